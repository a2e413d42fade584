"""End to end on the GPU: wide-pulse signals of a synthetic axon (a straight
voxelised cylinder, walkers inside only) through the host-side analysis.
Transverse to the axon, D_perp gives back the radius through Eq. r-mr
(Neuman's wide-pulse limit); the spherical mean of the b-shells follows
Eq. S-sph with D_a = D0."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


def _cylinder_workload(dirs, b, W):
    from conftest import make_workload
    import rms_inputs as ri
    l_p, r_vox, D0 = 0.05, 20, 2.0           # radius 1 um
    lab = ri.cylinder_labels(48, r_vox, nz=4)
    dt = 1.5e-4                              # ds = 0.042 um < l_p
    delta, Delta = 10.0, 12.0
    n = int(round((Delta + delta) / dt))
    G = ri.pgse(delta, Delta, dt, n)[None, :]
    wl = make_workload(lab, voxel_um=l_p, D=[D0, D0], dead=[1, 0], dt=dt, n_steps=n, G=G, dirs=dirs, b=b,
                       rec_steps=np.array([n]), n_walkers=W, seed=21)
    r_eff = math.sqrt((lab[0] == 1).sum() / math.pi) * l_p   # radius of the equal-area disk
    return wl, r_eff, delta, Delta, D0


def test_wide_pulse_radius_of_a_cylinder(rms):
    from paper_2012_06478_gb300 import analysis
    b = np.array([0.0, 25.0, 50.0, 100.0, 150.0, 200.0])
    dirs = np.eye(3)
    wl, r_eff, delta, Delta, D0 = _cylinder_workload(dirs, b, 200_000)
    g = rms.simulate(wl, rms.RMS_FP32)
    S = g["S"][0].real                                   # (3 dirs, n_b)
    Dp = []
    for d in (0, 1):
        c = np.polyfit(b[1:], np.log(S[d, 1:]), 2)     # ln S = -b D_perp + O(b^2)
        Dp.append(-c[1])
    D_perp = float(np.mean(Dp))
    r = analysis.r_mr(delta, Delta, D0, D_perp)
    assert abs(r - r_eff) < 0.05 * r_eff, (r, r_eff, D_perp)
    assert S[2, 1] < 1e-6                                # free along the axon: e^{-25*2}


def test_spherical_mean_of_a_cylinder(rms):
    from paper_2012_06478_gb300 import analysis
    import rms_inputs as ri
    b = np.linspace(16, 100, 8)
    dirs = ri.fibonacci_dirs(1000)
    wl, r_eff, delta, Delta, D0 = _cylinder_workload(dirs, np.r_[0.0, b], 100_000)
    g = rms.simulate(wl, rms.RMS_FP32)
    Sbar = analysis.spherical_mean(g["S"][0])[1:]
    beta, D_perp, D_a = analysis.fit_spherical_mean(b, Sbar)
    assert abs(D_a - D0) < 0.03 * D0, (D_a, D_perp)
    assert 0.0 < D_perp < 0.01
