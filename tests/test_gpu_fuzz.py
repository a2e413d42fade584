"""Randomised parity: seeded random configurations that mix every option at
once -- grid shapes, label counts, walls and periodic axes, dead labels,
per-label D, T1, T2 and relaxation modes, per-pair kappa (some zero), the
three interactions, absorbing membranes, spin concentrations with fixed or
optimal lambda or Baxter's rule, 1-8 waveform shapes, walker ids past 2^32,
odd slice lengths, recording steps -- and, on some cases, a run cut and
resumed and the invariant checks.  The plain FP64 form must equal the CPU
oracle bit for bit on every walker (state, checksum, counts), with moments
and signal to 1e-12."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload
from test_gpu_parity import assert_moments_close, assert_signal_close, assert_walkers_equal

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
ERR_LEAPS = 16


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


@pytest.fixture(scope="module")
def oracle():
    import oracle
    oracle.build()
    return oracle


def random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    shape = tuple(int(x) for x in rng.integers(1, 9, size=3))   # (nz, ny, nx)
    L = int(rng.integers(1, 7))
    lab = rng.integers(0, L, size=shape)
    lab.flat[0] = 0
    dead = (rng.uniform(size=L) < 0.25).astype(np.uint8)
    dead[0] = 0                                                 # at least one live voxel
    D = rng.uniform(0.3, 3.0, size=L)
    l_p = float(rng.choice([0.1, 0.2, 0.5]))
    dt = float(rng.uniform(0.1, 0.95)) * l_p ** 2 / (6 * D.max())
    K = rng.uniform(0, 4.0, size=(L, L)) * (rng.uniform(size=(L, L)) < 0.7)
    T2 = np.where(rng.uniform(size=L) < 0.7, rng.uniform(5, 100, size=L), np.inf)
    T1 = np.where(rng.uniform(size=L) < 0.5, rng.uniform(100, 900, size=L), np.inf)
    n_steps = int(rng.choice([0, 1, 7, 64, 200]))
    S = int(rng.integers(1, 9)) if n_steps else 1
    G = rng.normal(size=(max(S, 1), n_steps)) * (rng.uniform(size=(max(S, 1), n_steps)) < 0.4)
    mode = rng.integers(0, 3, size=n_steps).astype(np.uint8) if (n_steps and rng.uniform() < 0.5) else None
    rec = np.unique(rng.integers(1, n_steps + 1, size=int(rng.integers(0, 6)))) if n_steps else np.zeros(0, np.int64)
    W = int(rng.choice([1, 33, 128, 129, 600]))
    periodic = tuple(int(x) for x in rng.integers(0, 2, size=3))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=K, T2=T2, T1=T1, dt=dt, n_steps=n_steps,
                       G=G if S else np.zeros((1, n_steps)), dirs=rng.normal(size=(3, 3)),
                       b=np.array([0.0, 0.7]), rec_steps=rec, n_walkers=W, seed=int(rng.integers(1, 2 ** 40)),
                       periodic=periodic, dead=dead, mode=mode, interaction=int(rng.integers(0, 3)))
    if rng.uniform() < 0.4:
        R = rng.uniform(0, 0.3, size=(L, L))
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R)
    if rng.uniform() < 0.4:
        wl = wl.with_(conc=rng.uniform(0.3, 1.5, size=L), lam=float(rng.choice([-1.0, 0.0, 0.5, 1.0])),
                      perm_model=int(rng.uniform() < 0.3))
    extras = dict(walker_begin=int(rng.choice([0, 12345, 2 ** 33 + 7])), spl=int(rng.choice([0, 1, 13, 64])),
                  cut=int(rng.integers(1, n_steps)) if (n_steps > 1 and rng.uniform() < 0.3) else 0,
                  checked=bool(rng.uniform() < 0.3))
    return wl, extras


@pytest.mark.parametrize("seed", range(40))
def test_random_configuration(rms, oracle, seed):
    wl, ex = random_case(seed)
    kw = dict(hash_=True, walkers=True, counts=True, walker_begin=ex["walker_begin"],
              steps_per_launch=ex["spl"], checked=ex["checked"])
    if ex["cut"]:
        part = rms.simulate(wl, rms.RMS_FP64, step_end=ex["cut"], **kw)
        state = {k: part[k] for k in ("i", "o", "i0", "o0", "c", "A", "phase", "hash")}
        state.update(step=ex["cut"], moments=part["moments"])
        g = rms.simulate(wl, rms.RMS_FP64, resume=state, **kw)
        cnt_first = part["counts"]
    else:
        g = rms.simulate(wl, rms.RMS_FP64, **kw)
        cnt_first = 0
    o = oracle.run(wl, ex["walker_begin"], ex["walker_begin"] + wl.n_walkers, n_threads=NT, hash_=True)
    assert o["err"] & ~ERR_LEAPS == 0, o["err"]
    assert_walkers_equal(g, o)
    # counts restart at a resume: the two parts add up to the oracle's
    np.testing.assert_array_equal(g["counts"] + cnt_first, o["counts"])
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    S_o, asum_o = oracle.readout(o, wl)
    if asum_o > 0:
        assert_signal_close(g["S"], S_o)
    assert abs(g["alpha_sum"] - asum_o) <= 1e-12 * max(asum_o, 1e-300)
