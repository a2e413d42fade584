"""Pins of the oracle's magnetization-transfer (absorbing membrane) model,
Sec. 2.1.3: a walker meeting a membrane of surface relaxivity rho is
saturated with probability P_MT = rho ds C_3 / D0 and then has weight 0
(Eq. wt-mt); the mean-field rate is R = rho S/V.  Statistical checks use 4.5
standard errors."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload

NT = os.cpu_count() or 1
Z = 4.5
EC, RS, ERL = 0, 1, 2


def ds_of(D, dt):
    return math.sqrt(6.0 * D * dt)


def p_hat(rho, D, dt):
    """The probability the walker actually uses: floor(P_MT 2^32) / 2^32."""
    P = rho * ds_of(D, dt) / D * (2.0 / 3.0)
    return math.floor(P * 2.0 ** 32) / 2.0 ** 32


def slabs(a_vox):
    return np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))


def saturated(r):
    return np.isinf(r["A"])


@pytest.mark.parametrize("interaction", [EC, RS, ERL])
def test_paths_do_not_depend_on_absorption(oracle_lib, interaction):
    """MT draws have a stream of their own: with and without absorbing
    membranes every walker follows the same path; only the weights differ,
    and a saturated walker stays saturated (A = inf, alpha = 0)."""
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 3, size=(6, 5, 7))
    D = np.array([2.0, 0.8, 1.4])
    dt = 0.8 * 0.04 / (6 * D.max())
    base = dict(voxel_um=0.2, D=D, kappa=rng.uniform(0, 2.0, (3, 3)), T2=[50.0, 70.0, 90.0], dt=dt, n_steps=200,
                G=rng.normal(size=(1, 200)), rec_steps=np.array([50, 200]), n_walkers=3000, seed=4,
                interaction=interaction)
    a = oracle_lib.run(make_workload(lab, **base), n_threads=NT)
    b = oracle_lib.run(make_workload(lab, rho=rng.uniform(0, 0.05, (3, 3)), **base), n_threads=NT)
    for k in ("i", "o", "c", "phase"):
        np.testing.assert_array_equal(a[k], b[k])
    sat = saturated(b)
    assert 0.05 < sat.mean() < 0.95
    np.testing.assert_array_equal(a["A"][~sat], b["A"][~sat])
    assert b["moments"][-1, 0] <= a["moments"][-1, 0]


@pytest.mark.parametrize("interaction", [EC, RS])
def test_one_step_saturation_is_rho_s_over_v(oracle_lib, interaction):
    """Uniform start between absorbing planes a apart (a > 2 ds): a step from
    a distance h < ds meets the plane with probability (1 - h/ds)/2, so a
    fraction ds/(2a) of walkers meets one in the first step and ds/(2a) P_MT
    are saturated.  With ds^2 = 6 D dt and C_3 = 2/3 this is rho (S/V) dt
    whatever D: the mean-field rate R = rho S/V of Sec. 2.1.3, exact at
    t -> 0.  Alternate slabs have D = 2 and 0.5 (P_MT uses the walker's own
    D and ds).  RS cancels the step but the encounter still counts."""
    a_vox, l_p, dt, rho = 6, 0.1, 5e-4, 15.0
    D = np.array([2.0, 0.5])
    a = a_vox * l_p
    W = 1_000_000
    wl = make_workload(slabs(a_vox), voxel_um=l_p, D=D, dt=dt, n_steps=1, n_walkers=W, seed=7, rho=rho,
                       interaction=interaction)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    for c in (0, 1):
        P = p_hat(rho, D[c], dt)
        assert 0.3 < P < 0.9
        m = r["c"] == c
        f = saturated(r)[m].mean()
        expect = ds_of(D[c], dt) / (2 * a) * P
        assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / m.sum()), (c, f, expect)
        assert abs(expect - rho * (2 / a) * dt) < 1e-6 * expect + 2.0 ** -32


def test_membrane_into_a_dead_label_absorbs(oracle_lib):
    """Sec. 2.1.3 with the other side dead (e.g. myelin): walkers live only
    between the planes, the dead label is never entered, and the membrane
    still saturates: the first step's saturated fraction is again
    ds/(2a) P_MT."""
    a_vox, l_p, dt, rho, D = 6, 0.1, 5e-4, 15.0, 2.0
    a = a_vox * l_p
    W = 400_000
    wl = make_workload(slabs(a_vox), voxel_um=l_p, D=D, dt=dt, n_steps=1, n_walkers=W, seed=8, rho=rho,
                       dead=[0, 1])
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    assert np.all(r["c"] == 0)
    P = p_hat(rho, D, dt)
    f = saturated(r).mean()
    expect = ds_of(D, dt) / (2 * a) * P
    assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / W), (f, expect)


def test_one_step_saturation_under_erl(oracle_lib):
    """ERL redraws after every refused draw, and each refused draw meets the
    plane once: from u = h/ds < 1 the number of refused draws N is geometric
    with q = (1 - u)/2, so the walker stays unsaturated with probability
    E[(1 - P)^N] = (1 - q)/(1 - q + qP); integrated over the uniform start."""
    a_vox, l_p, D, dt, rho = 6, 0.1, 2.0, 5e-4, 30.0
    ds, a = ds_of(D, dt), a_vox * l_p
    P = p_hat(rho, D, dt)
    W = 1_000_000
    wl = make_workload(slabs(a_vox), voxel_um=l_p, D=D, dt=dt, n_steps=1, n_walkers=W, seed=8, rho=rho,
                       interaction=ERL)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    assert r["err"] == 0
    f = saturated(r).mean()
    u = (np.arange(200000) + 0.5) / 200000
    q = (1 - u) / 2
    expect = 2 * (ds / a) * np.mean(q * P / (1 - q + q * P))
    assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / W), (f, expect)
    assert f > 1.05 * ds / (2 * a) * P


def _brownstein_tarr(a, D, rho, t, n_modes=40):
    """Unsaturated fraction between absorbing planes a apart, uniform start:
    modes cos(xi x/l), l = a/2, with xi tan xi = rho l / D (Robin boundary
    D d_n rho + rho_s rho = 0), weights 2 sin^2 xi / (xi (xi + sin xi cos xi)),
    decay D xi^2 / l^2 (Brownstein & Tarr 1979)."""
    from scipy.optimize import brentq
    l = a / 2
    c = rho * l / D
    out = np.zeros_like(np.asarray(t, dtype=np.float64))
    for n in range(n_modes):
        lo, hi = n * math.pi + 1e-12, n * math.pi + math.pi / 2 - 1e-12
        xi = brentq(lambda x: x * math.tan(x) - c, lo, hi)
        w = 2 * math.sin(xi) ** 2 / (xi * (xi + math.sin(xi) * math.cos(xi)))
        out += w * np.exp(-D * xi * xi * np.asarray(t) / (l * l))
    return out


@pytest.mark.parametrize("interaction", [EC, RS])
def test_unsaturated_fraction_follows_brownstein_tarr(oracle_lib, interaction):
    """Between absorbing planes the unsaturated fraction (sum of alpha over
    walkers, no T2) follows the exact eigenmode solution with the surface
    relaxivity rho, through the crossover from the fast-diffusion limit
    exp(-rho S/V t)."""
    a_vox, l_p, D, dt, rho = 10, 0.1, 2.0, 5e-4, 1.0
    a = a_vox * l_p
    n, W = 4000, 40000
    rec = np.array([500, 1000, 2000, 4000])
    wl = make_workload(slabs(a_vox), voxel_um=l_p, D=D, dt=dt, n_steps=n, n_walkers=W, seed=9, rho=rho,
                       rec_steps=rec, interaction=interaction)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    f = r["moments"][:, 0] / W
    expect = _brownstein_tarr(a, D, rho, rec * dt)
    se = np.sqrt(expect * (1 - expect) / W)
    assert np.all(np.abs(f - expect) < Z * se + 0.01 * (1 - expect)), (f, expect)
    fast = np.exp(-rho * (2 / a) * rec * dt)
    assert np.all(f > fast)  # diffusion-limited: slower than the mean-field rate


def test_erl_saturation_persists_across_redraws(oracle_lib):
    """With the same seed, EC and RS make the same first-event MT trial in
    step 1, so in a slab (one membrane event per step at most) their
    saturated walkers coincide; ERL's saturated set contains them (its first
    draw is the same, later draws add trials)."""
    a_vox, l_p, D, dt, rho = 6, 0.1, 2.0, 5e-4, 30.0
    sat = {}
    for im in (EC, RS, ERL):
        wl = make_workload(slabs(a_vox), voxel_um=l_p, D=D, dt=dt, n_steps=1, n_walkers=100000, seed=10,
                           rho=rho, interaction=im)
        sat[im] = saturated(oracle_lib.run(wl, n_threads=NT, hash_=False))
    np.testing.assert_array_equal(sat[EC], sat[RS])
    assert np.all(sat[ERL][sat[EC]])
    assert sat[ERL].sum() > sat[EC].sum()


def test_each_membrane_event_is_an_independent_trial(oracle_lib):
    """Every voxel its own impermeable cell and ds = 0.9 voxel, so a step
    meets up to three membranes: among walkers whose first step has N face
    events, a fraction 1 - (1 - P_MT)^N is saturated."""
    lab = np.arange(64).reshape(4, 4, 4)
    l_p, D = 0.1, 2.0
    dt = (0.9 * l_p) ** 2 / (6 * D)
    rho = 0.5 * D / (ds_of(D, dt) * 2.0 / 3.0)  # P_MT ~ 1/2
    P = p_hat(rho, D, dt)
    W = 400_000
    wl = make_workload(lab, voxel_um=l_p, D=D, dt=dt, n_steps=1, n_walkers=W, seed=11, rho=rho)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    sat, events = saturated(r), r["counts"][:, 0]
    for N in (1, 2, 3):
        m = events == N
        assert m.sum() > 2000, N
        expect = 1 - (1 - P) ** N
        f = sat[m].mean()
        assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / m.sum()), (N, f, expect)
    assert not sat[events == 0].any()
