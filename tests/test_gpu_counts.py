"""RMS_COUNTS: per walker, face events, crossings into another label and
reflections (RS/ERL: steps a refused walker stayed).  The plain FP64 form
counts exactly what the CPU oracle counts, walker by walker; at scale the
mean number of face events per step is the closed form 1.5 ds / l_p."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload
from test_gpu_parity import _rand_case

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


@pytest.mark.parametrize("interaction,mt", [(0, False), (0, True), (1, False), (2, True)])
def test_counts_equal_the_oracle(rms, oracle, interaction, mt):
    wl = _rand_case(81, periodic=(0, 1, 1), W=1500, n_steps=300).with_(interaction=interaction)
    if mt:
        R = np.full((wl.n_labels, wl.n_labels), 0.05)
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R)
    g = rms.simulate(wl, rms.RMS_FP64, counts=True, walkers=True, steps_per_launch=53)
    o = oracle.run(wl, n_threads=NT)
    np.testing.assert_array_equal(g["counts"], o["counts"])
    np.testing.assert_array_equal(g["i"], o["i"])
    assert g["counts"][:, 1].sum() > 0 and g["counts"][:, 2].sum() > 0


def test_face_events_per_step_at_scale(rms):
    """One label, periodic: a uniform walker meets 1.5 ds / l_p faces per step
    on average (each axis: E|d_a| = s/2 faces, three axes)."""
    lab = np.zeros((16, 16, 16), np.uint16)
    l_p, D, dt, n, W = 0.1, 2.0, 2e-4, 200, 1_000_000
    wl = make_workload(lab, voxel_um=l_p, D=D, dt=dt, n_steps=n, n_walkers=W, seed=3)
    expect = 1.5 * math.sqrt(6 * D * dt) / l_p
    for prec in (rms.RMS_FP64, rms.RMS_FP32):
        g = rms.simulate(wl, prec, counts=True)
        ev = g["counts"][:, 0] / n
        assert abs(ev.mean() - expect) < 4.5 * ev.std() / math.sqrt(W), (prec, ev.mean(), expect)
        assert g["counts"][:, 1:].sum() == 0
