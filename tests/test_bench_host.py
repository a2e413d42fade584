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


def test_every_library_name_bench_uses_exists():
    """bench.py reaches the library only through the package: every `rms.X`
    it names is exported (caught on the CPU, before any GPU run)."""
    import re
    import paper_2012_06478_gb300 as rms
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = set(re.findall(r"\brms\.([A-Za-z_][A-Za-z0-9_]*)", open(os.path.join(root, "bench.py")).read()))
    missing = sorted(n for n in names if not hasattr(rms, n))
    assert not missing, missing


def test_operation_counts_of_the_axon_workload():
    """The method's per-walker-step operation counts for the 200x200x400
    axon workload, by hand from the itemised lists: 0.735 face events per
    walker-step, a gradient on half of the steps, one shape, no relaxation."""
    import rms_inputs as ri
    bench = _bench()
    wl = ri.workload("axons-200x200x400")
    ev, g_frac, S, relax = bench._step_profile(wl)
    assert abs(ev - 1.5 * math.sqrt(6 * 2.0 * 2e-4) / 0.1) < 1e-12   # one D everywhere
    assert abs(g_frac - 0.5) < 1e-12 and S == 1 and not relax
    assert abs(bench.method_ops(wl) - (40 + 28 + 3 + 12 + 13 * ev + 6 + 0.5 * (12 + 15) + 3)) < 1e-9
    assert abs(bench.fp64_ops(wl) - (20 + 3 + 4.5 + 5 * ev + 7 + 0.5 * (12 + 6))) < 1e-9


def test_rooflines_divide_algorithmic_work_by_measured_peaks():
    import rms_inputs as ri
    bench = _bench()
    wl = ri.workload("axons-200x200x400")
    live = {"sm_count": 152, "gather_per_s": 4e11, "fp64_add_per_s": 6e11, "fp64_mul_per_s": 5e11}
    pk = {"hbm_gbs": 6800.0}
    ws, ms = 2e9, 30.0
    rate = ws / (ms * 1e-3)
    r = bench.rooflines(wl, "fp32", ws, ms, pk, live, 2000.0, "k", profiled=False)
    ev = bench.events_per_step(wl)
    rl = r["rooflines"]
    assert abs(rl["label_lookup_l2"]["frac"] - ev * rate / 4e11) < 1e-12
    assert abs(rl["label_lookup_hbm"]["frac"] - 2 * ev * rate / 6.8e12) < 1e-12
    assert abs(rl["issue_floor"]["frac"] - bench.method_ops(wl) * rate / (152 * 128 * 2e9)) < 1e-12
    assert r["roofline"]["name"] == max(rl, key=lambda k: rl[k]["frac"])
    assert r["roofline"]["traffic"] is None                        # no matching profile
    r64 = bench.rooflines(wl, "fp64", ws, ms, pk, live, 2000.0, "k", profiled=False)
    assert abs(r64["rooflines"]["fp64_pipe"]["frac"] - bench.fp64_ops(wl) * rate / 5e11) < 1e-12
    assert "issue_floor" not in r64["rooflines"]


def test_fp32_vs_fp64_verdicts_at_every_recording_time():
    """The bars are applied at every recording time and axis: one bad K at one
    time flips dK_within_bar and names that time as the worst."""
    import torch
    bench = _bench()
    rng = np.random.default_rng(3)
    W, n_rec = 400, 5
    wl = make_workload(np.zeros((2, 2, 2)), dt=1e-3, n_steps=50, rec_steps=np.arange(10, 51, 10),
                       dirs=np.eye(3), b=np.array([0.0, 1.0]))
    M = np.zeros((n_rec, 22))
    t = wl.rec_steps * wl.dt
    M[:, 0] = W
    for j, col in enumerate((1, 4, 6)):            # xx, yy, zz: D = 2 along every axis
        M[:, col] = W * 2 * 2.0 * t
    for col in (7, 17, 21):                        # xxxx, yyyy, zzzz: K = 0.5
        M[:, col] = 3.5 * (M[:, 1] / W) ** 2 * W
    S = np.ones((1, 3, 2), complex)
    wk = {"i": np.zeros((W, 3), np.int32), "A": np.zeros(W), "phase": rng.normal(size=(W, 1, 3))}
    ok = bench.fp32_vs_fp64(torch, wl, np.array([1.0]), (S, M, float(W)), (S, M.copy(), float(W)), wk, wk,
                            dev="cpu")
    assert ok["dD_within_bar"] and ok["dK_within_bar"] and ok["dS_within_flat_bar"] and ok["decorrelated_walkers"] == 0
    M2 = M.copy()
    M2[3, 17] *= 1.01                              # K_yy at the 4th time off by 0.035 > 0.01 * 0.5
    bad = bench.fp32_vs_fp64(torch, wl, np.array([1.0]), (S, M2, float(W)), (S, M, float(W)), wk, wk, dev="cpu")
    assert not bad["dK_within_bar"] and bad["dD_within_bar"]
    assert bad["dK_worst"]["axis"] == "y" and abs(bad["dK_worst"]["t_ms"] - t[3]) < 1e-12
    assert abs(bad["dK_worst"]["K64"] - 0.5) < 1e-9
    assert bad["per_time"]["dK_over_bar"][3] > 1 and max(bad["per_time"]["dK_over_bar"][:3]) == 0


def test_morton_passes_and_launch_count():
    """The radix passes bench.py counts for RMS_MORTON: 3 key bits per bit of
    the largest coordinate, coordinates shifted to at most 8 bits, 8 key bits
    per pass (a 32^3 volume: 15 key bits, 2 passes; 200x200x400 and 512^3:
    24 key bits, 3 passes; one voxel: no pass)."""
    bench = _bench()
    assert bench.morton_passes((32, 32, 32)) == 2
    assert bench.morton_passes((200, 200, 400)) == 3
    assert bench.morton_passes((512, 512, 512)) == 3
    assert bench.morton_passes((1024, 1024, 1024)) == 3
    assert bench.morton_passes((4, 4, 4)) == 1
    assert bench.morton_passes((1, 1, 1)) == 0
