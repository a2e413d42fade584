"""Parity of the CUDA path with the CPU FP64 oracle for absorbing membranes
(Sec. 2.1.3, magnetization transfer): per-pair surface relaxivity rho, a
saturation trial at every membrane event, saturated walkers with weight 0
(A = +inf).  Plain FP64 form bit for bit (saturations included); FP32 form
paired with it."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload
from test_gpu_parity import _rand_case, assert_moments_close, assert_signal_close, assert_walkers_equal

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
EC, RS, ERL = 0, 1, 2
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


def _with_rho(wl, seed, hi):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, hi, (wl.n_labels, wl.n_labels))
    np.fill_diagonal(R, 0.0)
    return wl.with_(rho=R)


@pytest.mark.parametrize("interaction", [EC, RS, ERL])
@pytest.mark.parametrize("case", [
    dict(seed=31),
    dict(seed=32, S=1, periodic=(0, 0, 0)),
    dict(seed=33, S=2, dead=[0, 0, 1, 0], W=1000),
    dict(seed=34, shape=(1, 1, 2), L=2, W=500, S=8),
])
def test_random_substrates_bit_exact(rms, oracle, case, interaction):
    wl = _with_rho(_rand_case(**case), case["seed"], 0.05).with_(interaction=interaction)
    g = rms.simulate(wl, rms.RMS_FP64, hash_=True, steps_per_launch=37, walkers=True)
    o = oracle.run(wl, n_threads=NT, hash_=True)
    assert o["err"] & ~ERR_LEAPS == 0
    assert g["leap_limit"] == bool(o["err"] & ERR_LEAPS)
    assert_walkers_equal(g, o)
    if case["seed"] == 31:  # a case with membranes everywhere: some walkers saturate, not all
        assert 0 < np.isinf(g["A"]).mean() < 1
    S_o, asum_o = oracle.readout(o, wl)
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)
    assert abs(g["alpha_sum"] - asum_o) <= 1e-12 * max(asum_o, 1e-300)


def test_axons_full_with_absorption(rms, oracle):
    """The benchmark workload (200 axons, 1e6 walkers x 1e5 steps) with every
    membrane absorbing (rho = 0.02 um/ms), in the bench launch shape: sampled
    walkers bit for bit in the plain form; the FP32 form within its bars plus
    at most the bar again in paired standard errors, with noise-limited
    comparisons counted (most walkers saturate, so the paired noise of the
    drifted walkers is large against the few that remain)."""
    import rms_inputs as ri
    from test_gpu_fullsize import _check_fp32
    wl = ri.workload("axons-200x200x400")
    R = np.full((wl.n_labels, wl.n_labels), 0.02)
    np.fill_diagonal(R, 0.0)
    wl = wl.with_(rho=R)
    W = wl.n_walkers
    g64 = rms.simulate(wl, rms.RMS_FP64, walkers=True)
    assert 0.05 < 1 - np.isinf(g64["A"]).mean() < 0.95
    for b, e in ((0, 16), (W // 2, W // 2 + 16), (W - 16, W)):
        o = oracle.run(wl, b, e, n_threads=NT, hash_=False)
        assert o["err"] == 0
        for k in ("i", "o", "c", "A", "phase"):
            np.testing.assert_array_equal(g64[k][b:e], o[k].astype(g64[k].dtype), err_msg=k)
    g32 = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    dec, _ = _check_fp32(wl, g64, g32, paired=False)
    assert dec <= 0.05 * W


@pytest.mark.parametrize("interaction", [EC, RS])
def test_fp32_form_paired_with_plain_form(rms, oracle, interaction):
    """FP32 and FP64 forms draw the same MT words, so the saturated walkers
    are almost the same ones; the FP32 export shows them as +inf; signals
    and the unsaturated sum agree."""
    rng = np.random.default_rng(42)
    lab = rng.integers(0, 4, size=(12, 10, 11))
    D = np.array([2.0, 0.6, 1.3, 2.5])
    dt = 0.9 * (0.2 ** 2) / (6 * D.max())
    n = 2000
    G = np.zeros((1, n))
    G[0, :600], G[0, 1000:1600] = 1.0, -1.0
    wl = make_workload(lab, voxel_um=0.2, D=D, kappa=rng.uniform(0.01, 0.05, (4, 4)), T2=[40.0, 60.0, 80.0, 30.0],
                       dt=dt, n_steps=n, G=G, dirs=rng.normal(size=(6, 3)) / math.sqrt(3),
                       b=np.array([0.0, 0.5, 2.0]), rec_steps=np.array([1000, 2000]), n_walkers=20000, seed=12,
                       interaction=interaction, rho=0.02)
    g64 = rms.simulate(wl, rms.RMS_FP64, walkers=True)
    g32 = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    s64, s32 = np.isinf(g64["A"]), np.isinf(g32["A"])
    assert 0.05 < s64.mean() < 0.95
    assert (s64 == s32).mean() > 0.98
    assert np.abs(g32["S"] - g64["S"]).max() <= 1e-3
    assert abs(g32["alpha_sum"] - g64["alpha_sum"]) <= 0.01 * g64["alpha_sum"]


def test_serving_refuses_absorbing_membranes(rms):
    from paper_2012_06478_gb300 import _lib
    wl = _with_rho(_rand_case(35, W=10, n_steps=5), 35, 0.3)
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, kappa=wl.kappa, rho=wl.rho)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    srv = rms.Server()
    try:
        with pytest.raises(rms.RmsError) as e:
            srv.submit(seq, 10, 1, rms.RMS_FP64)
        assert e.value.status == _lib.RMS_E_INVALID_ARG
    finally:
        srv.close()
        seq.close()
        sub.close()


def test_saturation_probability_above_one_warns(rms):
    """P_MT > 1 is clamped to 1 with the RMS_W_PROB_RANGE warning."""
    from paper_2012_06478_gb300 import _lib
    wl = _rand_case(36, W=10, n_steps=5)
    R = np.full((wl.n_labels, wl.n_labels), 1e4)
    np.fill_diagonal(R, 0.0)
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, kappa=wl.kappa * 0, rho=R)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    assert seq.status == _lib.RMS_W_PROB_RANGE
    seq.close()
    sub.close()
