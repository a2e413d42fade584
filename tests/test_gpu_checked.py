"""RMS_CHECKED: the verification kernel checks the walker invariants after
every step (voxel coordinates in range, flat index consistent, the walker's
label equal to its voxel's, offsets in [0,1]).  On substrates exercising
every path (walls, dead labels, permeable and absorbing membranes, spin
concentrations, every interaction) no check fires, and checking changes no
result."""
import numpy as np
import pytest

from test_gpu_parity import _rand_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


@pytest.mark.parametrize("interaction", [0, 1, 2])
@pytest.mark.parametrize("extras", ["plain", "mt-conc"])
def test_checked_runs_pass_and_change_nothing(rms, interaction, extras):
    wl = _rand_case(61, periodic=(0, 1, 1), dead=[0, 0, 1, 0], W=2000, n_steps=400).with_(interaction=interaction)
    if extras == "mt-conc":
        R = np.full((wl.n_labels, wl.n_labels), 0.05)
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R, conc=np.array([1.0, 0.6, 1.0, 1.3]), lam=-1.0)
    for prec in (rms.RMS_FP64, rms.RMS_FP32):
        a = rms.simulate(wl, prec, hash_=True, walkers=True)
        b = rms.simulate(wl, prec, checked=True, walkers=True)   # raises RmsError on a broken invariant
        if prec == rms.RMS_FP64:
            for k in ("i", "o", "c", "A", "phase", "hash"):
                np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a["S"], b["S"])
