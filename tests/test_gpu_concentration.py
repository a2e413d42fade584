"""Parity of the CUDA path with the CPU FP64 oracle for spin concentrations
(App. C.2: initial density ~ c, the generalised Eq. 3 with (c2/c1)^lambda)
and Baxter's permeation rule (App. C.3): plain FP64 form bit for bit."""
import os

import numpy as np
import pytest

from test_gpu_parity import _rand_case, assert_moments_close, assert_signal_close, assert_walkers_equal

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


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


def _conc_case(seed, lam, perm_model, interaction=0, **kw):
    wl = _rand_case(seed, **kw)
    rng = np.random.default_rng(seed + 100)
    conc = rng.uniform(0.3, 1.5, wl.n_labels)
    return wl.with_(conc=conc, lam=lam, perm_model=perm_model, interaction=interaction)


@pytest.mark.parametrize("lam,perm_model,interaction", [
    (0.3, 0, 0), (-1.0, 0, 0), (1.0, 0, 1), (-1.0, 1, 0), (-1.0, 1, 2),
])
@pytest.mark.parametrize("case", [
    dict(seed=51),
    dict(seed=52, S=2, dead=[0, 0, 1, 0], W=1000, periodic=(0, 1, 1)),
])
def test_random_substrates_bit_exact(rms, oracle, case, lam, perm_model, interaction):
    """Random labels, per-label D, T1/T2 modes, per-pair kappa, dead labels
    and walls, with spin concentrations: every walker bit for bit (the
    concentration-weighted start included)."""
    wl = _conc_case(lam=lam, perm_model=perm_model, interaction=interaction, **case)
    g = rms.simulate(wl, rms.RMS_FP64, hash_=True, steps_per_launch=37, walkers=True)
    o = oracle.run(wl, n_threads=NT, hash_=True)
    assert o["err"] & ~16 == 0
    assert_walkers_equal(g, o)
    S_o, asum_o = oracle.readout(o, wl)
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)


def test_axons_sampled_walkers(rms, oracle):
    """The 200-axon geometry (1e6 walkers, 1000 steps, default launches) with
    the bath at 0.6 of the axons' spin concentration, for the generalised
    Eq. 3 (optimal lambda) and Baxter's rule: sampled walkers bit for bit."""
    import rms_inputs as ri
    base = ri.workload("axons-200x200x400")
    n = 1000
    base = base.with_(n_steps=n, G=base.G[:, :n], rec_steps=np.array([n]))
    conc = np.ones(base.n_labels)
    conc[0] = 0.6
    W = base.n_walkers
    for perm_model in (0, 1):
        wl = base.with_(conc=conc, lam=-1.0, perm_model=perm_model)
        g = rms.simulate(wl, rms.RMS_FP64, walkers=True)
        for b, e in ((0, 16), (W // 2, W // 2 + 16), (W - 16, W)):
            o = oracle.run(wl, b, e, n_threads=NT, hash_=False)
            assert o["err"] == 0
            for k in ("i", "o", "i0", "o0", "c", "A", "phase"):
                np.testing.assert_array_equal(g[k][b:e], o[k].astype(g[k].dtype), err_msg=f"{k} {perm_model}")


def test_fp32_start_matches_fp64(rms):
    """Both precision forms draw the same concentration-weighted start."""
    wl = _conc_case(53, -1.0, 0, W=5000)
    g64 = rms.simulate(wl, rms.RMS_FP64, n_walkers=5000, walkers=True)
    g32 = rms.simulate(wl, rms.RMS_FP32, n_walkers=5000, walkers=True)
    np.testing.assert_array_equal(g64["i0"], g32["i0"])
    np.testing.assert_allclose(g64["o0"], g32["o0"], atol=1e-7)


def test_extreme_contrast_and_bad_arguments_are_rejected(rms):
    """A start-acceptance rate (volume mean of c / c_max) below 1/200, a
    non-positive concentration, lambda > 1 or an unknown model: refused."""
    from paper_2012_06478_gb300 import _lib
    lab = np.zeros((10, 10, 10), np.uint16)
    lab[0, 0, 0] = 1
    D = np.array([1.0, 1.0])
    for kw in (dict(conc=np.array([1e-3, 1.0])), dict(conc=np.array([1.0, 0.0])),
               dict(conc=np.array([1.0, 1.0]), lam=2.0), dict(perm_model=5)):
        with pytest.raises(rms.RmsError) as e:
            rms.rms_create_substrate(lab, 0.2, D, kappa_scalar=0.1, **kw)
        assert e.value.status == _lib.RMS_E_INVALID_ARG, kw
    sub = rms.rms_create_substrate(lab, 0.2, D, kappa_scalar=0.1, conc=np.array([1e-2, 1.0]))
    sub.close()
