"""Host-side arithmetic of bench.py, on the CPU: the paired standard error
behind the FP32-vs-FP64 error bars, and the expected face events per step
behind the label-lookup roofline."""
import math
import os

import numpy as np

from conftest import make_workload

NT = os.cpu_count() or 1


def _bench():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _walkers(rng, W, S):
    return {"A": rng.uniform(0, 0.5, W), "phase": rng.normal(size=(W, S, 3))}


def test_paired_sigma_is_the_standard_error_of_the_paired_differences():
    """Against the definition computed directly, for a walker count that
    spans several chunks; 0 for identical forms."""
    import torch
    bench = _bench()
    rng = np.random.default_rng(1)
    W, S = 5000, 2
    wl = make_workload(np.zeros((2, 2, 2)), n_steps=4, G=np.ones((S, 4)), dirs=rng.normal(size=(40, 3)),
                       b=np.linspace(0, 3, 60))
    b_s = np.array([0.7, 1.3])
    w64 = _walkers(rng, W, S)
    w32 = {"A": w64["A"] + rng.normal(scale=1e-3, size=W), "phase": w64["phase"] + rng.normal(scale=1e-2, size=(W, S, 3))}
    sig = bench.paired_sigma(torch, wl, b_s, w64, w32, dev="cpu")
    assert sig.shape == (S, 40, 60)
    q = np.sqrt(wl.b[None, :] / b_s[:, None])
    for s in range(S):
        terms = []
        for wk in (w32, w64):
            al = np.exp(-wk["A"])
            phi = (wk["phase"][:, s, :] @ wl.dirs.T)[:, :, None] * q[s][None, None, :]
            terms.append((al / al.mean())[:, None, None] * np.exp(-1j * phi))
        d = terms[0] - terms[1]
        expect = np.sqrt((np.abs(d - d.mean(0)) ** 2).mean(0) / W)
        np.testing.assert_allclose(sig[s], expect, rtol=1e-9, atol=1e-15)
    assert np.all(bench.paired_sigma(torch, wl, b_s, w64, w64, dev="cpu") == 0.0)


def test_events_per_step_matches_the_oracle_counts(oracle_lib):
    """1.5 ds / l_p per label, averaged over where the walkers are: with a
    dead label and unequal D the prediction equals the oracle's mean face
    events per step."""
    bench = _bench()
    rng = np.random.default_rng(2)
    lab = rng.integers(0, 3, size=(6, 6, 6))
    D = np.array([2.0, 0.6, 1.0])
    wl = make_workload(lab, voxel_um=0.2, D=D, dt=1e-3, n_steps=50, n_walkers=20000, dead=[0, 0, 1], seed=3)
    r = oracle_lib.run(wl, n_threads=NT)
    per = r["counts"][:, 0] / wl.n_steps
    assert abs(per.mean() - bench.events_per_step(wl)) < 4.5 * per.std() / math.sqrt(wl.n_walkers)
    frac = np.bincount(lab.ravel(), minlength=3) / lab.size      # the volume fraction over every label
    naive = float((frac * 1.5 * np.sqrt(6 * D * wl.dt) / wl.voxel_um).sum())
    assert abs(per.mean() - naive) > 4.5 * per.std() / math.sqrt(wl.n_walkers)
