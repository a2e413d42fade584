"""The FP32 form's read-out (Eq. 7): each term alpha e^{-i phi} is evaluated
in single precision (phase rounded to float, phi = q g.Phi_s and sincosf in
FP32, alpha rounded to float) and summed in FP64.  Against the FP64 read-out
of the same walkers (computed here on the host from the exported state) S
agrees within fp32_readout_bound(P), P = q sum_i |g_i| |Phi_i| over all
walkers and combinations: the roundings of Phi, g, q, the dot product and the
product move phi by at most about 6 P 2^-24, sincosf, alpha and the term's
product add about 4 2^-24.  FP32_READOUT_TOL is the bound at P = 20 rad
(7.4e-6, rounded up).  b = 0 gives S = 1 exactly; the sum of alpha is FP64."""
import math

import numpy as np
import pytest

from conftest import make_workload

pytestmark = pytest.mark.gpu

def fp32_readout_bound(P):
    return (6.0 * P + 4.0) * 2.0 ** -24


FP32_READOUT_TOL = 1e-5  # >= fp32_readout_bound(20)


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


def host_readout(wl, b_s, st):
    """S = sum alpha e^{-i q g.Phi_s} / sum alpha in FP64 (numpy), and sum alpha."""
    al = np.exp(-st["A"])
    S = np.zeros((b_s.size, wl.dirs.shape[0], wl.b.size), np.complex128)
    for s in range(b_s.size):
        gp = st["phase"][:, s, :] @ wl.dirs.T  # (W, n_dirs)
        for ib, b in enumerate(wl.b):
            q = math.sqrt(b / b_s[s]) if b > 0 else 0.0
            S[s, :, ib] = (al[:, None] * np.exp(-1j * q * gp)).sum(axis=0) / al.sum()
    return S, al.sum()


@pytest.mark.parametrize("seed,W", [(3, 20000), (4, 4097), (5, 1)])
def test_fp32_readout_against_fp64_terms(rms, seed, W):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 3, size=(10, 9, 12))
    n = 400
    G = np.zeros((2, n))
    G[0, :100], G[0, 250:350] = 1.0, -1.0                       # PGSE
    G[1] = np.cos(2 * np.pi * np.arange(n) / 200.0)             # an oscillating shape
    wl = make_workload(lab, voxel_um=0.2, D=[2.0, 1.0, 1.5], kappa=rng.uniform(0, 2, size=(3, 3)),
                       T2=[50.0, 70.0, 90.0], dt=2e-3, n_steps=n, G=G,
                       dirs=rng.normal(size=(9, 3)) / np.sqrt(3), b=np.array([0.0, 0.5, 2.0, 5.0]),
                       rec_steps=np.array([n]), n_walkers=W, seed=seed)
    res = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    S_h, asum_h = host_readout(wl, res["b_s"], res)
    P = max(math.sqrt(wl.b.max() / res["b_s"][s]) * (np.abs(res["phase"][:, s, :]) @ np.abs(wl.dirs).T).max()
            for s in range(res["b_s"].size))
    assert P <= 60.0, P  # the phases stay in the range the bound is meant for
    tol = fp32_readout_bound(P)
    assert np.abs(res["S"] - S_h).max() <= tol, (np.abs(res["S"] - S_h).max(), tol, P)
    assert abs(res["alpha_sum"] - asum_h) <= 1e-12 * asum_h
    assert np.all(res["S"][:, :, 0] == 1.0)  # b = 0
