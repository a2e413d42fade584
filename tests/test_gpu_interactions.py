"""Parity of the CUDA path with the CPU FP64 oracle for the alternative
particle-membrane interactions: rejection sampling (App. B) and the
equal-step-length random leap (App. A).

Plain FP64 form: every walker's final state, relaxation exponent, phases and
trajectory checksum are bit-identical to the oracle's, and an ERL step that
uses up its draws is reported by both sides.  FP32 form: paired with the FP64
form (same random numbers), |dS| <= 1e-3."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload
from test_gpu_parity import _rand_case, assert_moments_close, assert_signal_close, assert_walkers_equal

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
RS, ERL = 1, 2
ERR_LEAPS = 16  # oracle error bit: an ERL step used up its draws


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


def run_both(rms, oracle, wl, spl=0, w_begin=0, n=None, hash_=True):
    W = wl.n_walkers if n is None else n
    g = rms.simulate(wl, rms.RMS_FP64, n_walkers=W, hash_=hash_, walker_begin=w_begin, steps_per_launch=spl,
                     walkers=True)
    o = oracle.run(wl, w_begin, w_begin + W, n_threads=NT, hash_=hash_)
    assert o["err"] & ~ERR_LEAPS == 0
    assert g["leap_limit"] == bool(o["err"] & ERR_LEAPS)
    S_o, asum_o = oracle.readout(o, wl)
    return g, o, S_o, asum_o


@pytest.mark.parametrize("interaction", [RS, ERL])
@pytest.mark.parametrize("case", [
    dict(seed=21),
    dict(seed=22, S=1, periodic=(0, 0, 0)),
    dict(seed=23, S=2, dead=[0, 0, 1, 0], W=1000),
    dict(seed=24, shape=(1, 1, 2), L=2, W=500, S=8),
    dict(seed=25, W=1, n_steps=50),
])
def test_random_substrates_bit_exact(rms, oracle, case, interaction):
    """Random labels, per-label D, T1, T2 and relaxation modes, per-pair
    kappa (refusals by failed Bernoulli trials), dead labels and walls:
    every walker bit for bit, launches sliced every 37 steps."""
    wl = _rand_case(**case).with_(interaction=interaction)
    g, o, S_o, asum_o = run_both(rms, oracle, wl, spl=37)
    assert_walkers_equal(g, o)
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)
    assert abs(g["alpha_sum"] - asum_o) <= 1e-12 * asum_o


@pytest.mark.parametrize("interaction", [RS, ERL])
def test_impermeable_slabs_bit_exact(rms, oracle, interaction):
    """Impermeable slabs (the geometry of App. A and B): many refused steps,
    ERL redraws, T2 weighting of the steps a walker stays."""
    lab = np.broadcast_to(np.array([0] * 6 + [1] * 6), (3, 3, 12))
    n = 400
    G = np.zeros((1, n))
    G[0, :100], G[0, 300:] = 1.0, -1.0
    wl = make_workload(lab, voxel_um=0.1, D=2.0, kappa=0.0, T2=[50.0, 70.0], dt=5e-4, n_steps=n, G=G,
                       b=np.array([0.0, 1.0]), rec_steps=np.array([100, 400]), n_walkers=5000, seed=3,
                       interaction=interaction)
    g, o, S_o, _ = run_both(rms, oracle, wl)
    assert_walkers_equal(g, o)
    assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)


def test_erl_leap_limit_is_reported(rms, oracle):
    """Every voxel its own impermeable cell and ds = 0.95 voxel: near a
    voxel's centre no direction is admissible (|n_a| ds < 1/2 for all three
    axes needs ds < sqrt(3)/2), so those ERL steps use up their 64 draws and
    the walker stays; both sides flag it and still agree bit for bit."""
    lab = np.arange(27).reshape(3, 3, 3)
    D, l_p = 2.0, 0.1
    dt = (0.95 * l_p) ** 2 / (6 * D)
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=20, n_walkers=3000, seed=5,
                       interaction=ERL)
    g, o, _, _ = run_both(rms, oracle, wl)
    assert g["leap_limit"]
    assert_walkers_equal(g, o)
    np.testing.assert_array_equal(g["i"], g["i0"])


def test_axons_sampled_walkers(rms, oracle):
    """The benchmark geometry (200 undulating axons, kappa 0.01 um/ms: almost
    every membrane event refused) at 1e6 walkers, 1000 steps, default
    launches: sampled walkers bit for bit for both interactions."""
    import rms_inputs as ri
    base = ri.workload("axons-200x200x400")
    n = 1000
    base = base.with_(n_steps=n, G=base.G[:, :n], rec_steps=np.array([n]))
    W = base.n_walkers
    for interaction in (RS, ERL):
        wl = base.with_(interaction=interaction)
        g = rms.simulate(wl, rms.RMS_FP64, walkers=True)
        for b, e in ((0, 16), (W // 2, W // 2 + 16), (W - 16, W)):
            o = oracle.run(wl, b, e, n_threads=NT, hash_=False)
            assert o["err"] == 0
            for k in ("i", "o", "c", "A", "phase"):
                np.testing.assert_array_equal(g[k][b:e], o[k].astype(g[k].dtype), err_msg=f"{k} {interaction}")


@pytest.mark.parametrize("interaction", [RS, ERL])
def test_fp32_form_paired_with_plain_form(rms, oracle, interaction):
    """FP32 and FP64 forms draw the same random numbers; a refusal differs
    only where a face lies within the FP32 rounding drift, so almost every
    walker ends in the same voxel and the signals agree within 1e-3."""
    rng = np.random.default_rng(41)
    lab = rng.integers(0, 4, size=(12, 10, 11))
    D = np.array([2.0, 0.6, 1.3, 2.5])
    dt = 0.9 * (0.2 ** 2) / (6 * D.max())
    n = 2000
    G = np.zeros((2, n))
    G[0, :600], G[0, 1000:1600] = 1.0, -1.0
    G[1, 100:200], G[1, 1800:1900] = 1.0, -1.0
    wl = make_workload(lab, voxel_um=0.2, D=D, kappa=rng.uniform(0.01, 0.05, (4, 4)), T2=[40.0, 60.0, 80.0, 30.0],
                       dt=dt, n_steps=n, G=G, dirs=rng.normal(size=(6, 3)) / math.sqrt(3),
                       b=np.array([0.0, 0.5, 2.0]), rec_steps=np.array([1000, 2000]), n_walkers=20000, seed=9,
                       interaction=interaction)
    g64 = rms.simulate(wl, rms.RMS_FP64, walkers=True)
    g32 = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    same = np.all(g64["i"] == g32["i"], axis=1).mean()
    assert same > 0.98, same
    assert np.abs(g32["S"] - g64["S"]).max() <= 1e-3
    o = oracle.run(wl, 0, 64, n_threads=NT)
    np.testing.assert_array_equal(g64["i"][:64], o["i"])


def test_unknown_interaction_is_rejected(rms):
    from paper_2012_06478_gb300 import _lib
    wl = _rand_case(26, W=10, n_steps=5)
    with pytest.raises(rms.RmsError) as e:
        rms.simulate(wl, rms.RMS_FP64, interaction=3)
    assert e.value.status == _lib.RMS_E_INVALID_ARG
