"""Pins of the oracle's alternative particle-membrane interactions against the
paper's closed forms: rejection sampling (App. B) and the equal-step-length
random leap (App. A).  Statistical checks use 4.5 standard errors."""
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


@pytest.mark.parametrize("interaction", [RS, ERL])
def test_walkers_never_leave_a_closed_voxel(oracle_lib, interaction):
    """Every face impermeable (each voxel its own label): a refused step is
    cancelled, so walkers never change voxel; RS walkers either stay exactly
    or make a whole step inside the voxel, ERL walkers always move exactly ds
    (a new direction is drawn until the step stays inside).  A refused step
    still lasts dt: the relaxation weight grows by dt/T2 either way."""
    lab = np.arange(64).reshape(4, 4, 4)
    dt, l_p, D, T2 = 1e-3, 0.2, 2.0, 0.05
    s = ds_of(D, dt) / l_p
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, T2=T2, dt=dt, n_steps=1, n_walkers=20000,
                       interaction=interaction)
    r = oracle_lib.run(wl, n_threads=NT)
    np.testing.assert_array_equal(r["i"], r["i0"])
    np.testing.assert_allclose(r["A"], dt / T2, rtol=1e-14)
    step = np.linalg.norm(r["o"] - r["o0"], axis=1)
    stayed = step == 0.0
    if interaction == RS:
        assert 0.2 < stayed.mean() < 0.9
        np.testing.assert_allclose(step[~stayed], s, rtol=1e-12)
    else:
        assert r["err"] == 0
        np.testing.assert_allclose(step, s, rtol=1e-12)


def test_rejection_stays_are_counted_at_the_refusal_rate(oracle_lib):
    """Rejection sampling in closed voxels: the start is uniform and stays
    uniform (App. B), and a step from a uniform point of the unit voxel along
    s n stays inside with probability prod_a (1 - s |n_a|), so the stays per
    step (the third count) average 1 - E_n prod_a (1 - s |n_a|) over
    directions (quadrature over the sphere).  No face event survives a
    refusal, and nothing crosses."""
    lab = np.arange(64).reshape(4, 4, 4)
    dt, l_p, D, n = 1e-3, 0.2, 2.0, 40
    s = ds_of(D, dt) / l_p
    W = 20000
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=n, n_walkers=W, seed=13, interaction=RS)
    r = oracle_lib.run(wl, n_threads=NT)
    cnt = r["counts"]
    assert np.all(cnt[:, 0] == 0) and np.all(cnt[:, 1] == 0)
    # E over the sphere: z uniform on [-1, 1], azimuth uniform (midpoint rule)
    m = 2000
    z = -1 + (np.arange(m) + 0.5) * (2.0 / m)
    ph = (np.arange(m) + 0.5) * (2 * math.pi / m)
    rr = np.sqrt(1 - z * z)[:, None]
    nx, ny, nz = np.abs(rr * np.cos(ph)), np.abs(rr * np.sin(ph)), np.abs(z)[:, None]
    stay_in = ((1 - s * nx) * (1 - s * ny) * (1 - s * nz)).mean()
    per = cnt[:, 2] / n
    expect = 1 - stay_in
    assert abs(per.mean() - expect) < Z * per.std() / math.sqrt(W), (per.mean(), expect)


def test_erl_leap_limit_near_the_centre_of_a_closed_voxel(oracle_lib):
    """App. A's redraw loop is capped at 64 draws (R21).  With ds = 0.95 voxel
    in closed voxels, a start within r < 0.95 - sqrt(3)/2 of the voxel's
    centre reaches at most sqrt(3)/2 + r: every direction leaves the voxel,
    so the walker stays for the step (one stay in the counts) and the run
    reports the leap-limit error bit (16).  Walkers elsewhere still move ds."""
    lab = np.arange(64).reshape(4, 4, 4)
    l_p, D = 0.1, 2.0
    dt = (0.95 * l_p) ** 2 / (6 * D)
    W = 40000
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=1, n_walkers=W, seed=14,
                       interaction=ERL)
    r = oracle_lib.run(wl, n_threads=NT)
    assert r["err"] & 16
    rc = np.linalg.norm(r["o0"] - 0.5, axis=1)
    trapped = rc < 0.95 - math.sqrt(3) / 2 - 1e-9
    assert trapped.sum() > 50
    np.testing.assert_array_equal(r["o"][trapped], r["o0"][trapped])
    np.testing.assert_array_equal(r["counts"][trapped, 2], 1)
    moved = np.linalg.norm(r["o"] - r["o0"], axis=1)
    free = rc > 0.2
    np.testing.assert_allclose(moved[free & (moved > 0)], 0.95, rtol=1e-12)
    assert (moved[free] > 0).mean() > 0.9


def _slab_positions(r, a_vox):
    """Distance (voxels) of each walker to the nearest wall of its slab."""
    x = np.mod(r["i"][:, 0], 2 * a_vox) + r["o"][:, 0]
    x = np.where(x >= a_vox, x - a_vox, x)
    return np.minimum(x, a_vox - x)


@pytest.mark.parametrize("interaction", [RS, ERL])
def test_density_next_to_a_wall(oracle_lib, interaction):
    """App. A, Eq. A.1 (d = 3): under ERL the density a distance h <= ds from
    an impermeable membrane is p(h) = (1 + h/ds)/2 of the bulk; rejection
    sampling keeps it uniform (App. B)."""
    a_vox, l_p, D, dt = 6, 0.1, 2.0, 5e-4
    ds = ds_of(D, dt) / l_p                          # 0.775 voxel
    W = 200000
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=400, n_walkers=W, seed=12,
                       interaction=interaction)
    r = oracle_lib.run(wl, n_threads=NT)
    h = _slab_positions(r, a_vox) / ds               # in units of ds
    edges = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    bulk = (h >= 1.0).sum() / (a_vox / 2 / ds - 1.0)  # walkers per unit of h in the bulk
    for lo, hi in zip(edges[:-1], edges[1:]):
        n = ((h >= lo) & (h < hi)).sum()
        ratio = n / (bulk * (hi - lo))
        expect = 1.0 if interaction == RS else 0.5 * (1 + 0.5 * (lo + hi))
        assert abs(ratio - expect) < Z * math.sqrt(n) / (bulk * (hi - lo)) + 0.01, (lo, hi, ratio, expect)


def _erl_msd(a, ds, m=200000):
    """Long-time <(x - x0)^2> = Var(x0) + Var(x): x0 uniform on the slab, x from
    the ERL stationary density p(h) (Eq. A.1) -- the pore shrinkage of Eq. A.8
    at first order in ds."""
    x = (np.arange(m) + 0.5) / m * a
    h = np.minimum(x, a - x)
    p = np.where(h < ds, 0.5 * (1 + h / ds), 1.0)
    p /= p.sum()
    mean = (p * x).sum()
    var = (p * (x - mean) ** 2).sum()
    return a * a / 12 + var


def test_erl_pore_shrinkage(oracle_lib):
    """App. A: between impermeable planes ERL measures a pore narrowed by
    about ds/8 on each side (Eq. A.8); the long-time MSD follows the ERL
    stationary density (second order in ds: + ds^2/8), well below the
    elastic-collision a^2/6."""
    a_vox, l_p, D, dt = 4, 0.1, 2.0, 5e-4
    a = a_vox * l_p
    ds = ds_of(D, dt)                                 # ds / a = 0.19
    W, n = 80000, 800                                 # t = 5 a^2 / D
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=n, n_walkers=W, seed=13,
                       interaction=ERL)
    r = oracle_lib.run(wl, n_threads=NT)
    assert r["err"] == 0
    dx = oracle_lib.displacement(r, l_p)[:, 0]
    x2 = dx ** 2
    expect = _erl_msd(a, ds)
    first_order = (a * a - a * ds / 2) / 6
    assert abs(expect - first_order - ds * ds / 8) < ds ** 3 / a
    assert abs(x2.mean() - expect) < Z * x2.std() / math.sqrt(W), (x2.mean(), expect)
    assert x2.mean() < 0.93 * a * a / 6


def _dpar(a, ds, dt, interaction, m=200000):
    """D parallel to the planes of a slab of width a > 2 ds.  Per step, from a
    distance h = u ds to a wall, the allowed directions are cos(theta) >= -u
    (theta from the wall normal); averaging ds^2 sin^2(theta) cos^2(phi) over
    them gives ds^2 (2 + 3u - u^3) / 12 for RS (refused steps count as zero)
    and ds^2 (2 + u - u^2) / 6 for ERL (the leap is uniform over the allowed
    set); both equal ds^2 / 3 past u = 1.  Parallel increments have zero mean
    given the past, so D_par is their mean over the stationary density
    (uniform for RS, p(h) of Eq. A.1 for ERL) over 2 dt (App. A and B)."""
    x = (np.arange(m) + 0.5) / m * a
    u = np.minimum(np.minimum(x, a - x) / ds, 1.0)
    if interaction == RS:
        z2, rho = ds * ds * (2 + 3 * u - u ** 3) / 12, np.ones_like(u)
    else:
        z2, rho = ds * ds * (2 + u - u * u) / 6, 0.5 * (1 + u)
    return (rho * z2).sum() / rho.sum() / (2 * dt)


@pytest.mark.parametrize("interaction", [RS, ERL])
def test_diffusivity_along_the_walls(oracle_lib, interaction):
    """App. A (Eq. erl-axial) and App. B (Eq. rs-axial): near a membrane RS
    slows diffusion parallel to it, D_par = D0 (1 - 3/16 (S/V) ds), and ERL
    speeds it up, D_par = D0 (1 + 1/16 (S/V) ds), both at first order in ds."""
    a_vox = 6 if interaction == RS else 3
    l_p, D, dt = 0.1, 2.0, 5e-4
    a = a_vox * l_p
    ds = ds_of(D, dt)
    W, n = (160000, 400) if interaction == RS else (320000, 1000)
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=n, n_walkers=W, seed=14,
                       interaction=interaction)
    r = oracle_lib.run(wl, n_threads=NT)
    assert r["err"] == 0
    dy = oracle_lib.displacement(r, l_p)[:, 1:]
    y2 = (dy ** 2).sum(axis=1) / 2                    # y and z alike
    Dpar = y2.mean() / (2 * n * dt)
    se = y2.std() / math.sqrt(W) / (2 * n * dt)
    expect = _dpar(a, ds, dt, interaction)
    sign = -3.0 if interaction == RS else 1.0
    first_order = D * (1 + sign / 16.0 * (2 / a) * ds)
    assert abs(expect - first_order) < 2 * D * (ds / a) ** 2
    assert abs(Dpar - expect) < Z * se, (Dpar, expect, se)
    if interaction == RS:
        assert Dpar < 0.96 * D
    else:
        assert Dpar > 1.01 * D


def test_rs_exchange_rate(oracle_lib):
    """App. B and Fig. C1: with the permeation probability of Eq. 3 (at equal
    D: P/(1-P) = kappa ds C_3 / D0), rejection sampling gives the genuine
    permeability -- the exchange fraction follows the exact eigenmode
    solution, as for elastic collisions."""
    from test_oracle_pins import _exchange_fraction
    l_p, D, dt, kappa = 0.2, 2.0, 1e-3, 0.02
    a = 3 * l_p
    n, W = 6000, 20000
    lab = np.broadcast_to(np.array([0, 0, 0, 1, 1, 1]), (2, 2, 6))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=kappa, dt=dt, n_steps=n, n_walkers=W, seed=15,
                       interaction=RS)
    r = oracle_lib.run(wl, n_threads=NT)
    c0 = lab[np.mod(r["i0"][:, 2], 2), np.mod(r["i0"][:, 1], 2), np.mod(r["i0"][:, 0], 6)]
    stay = (r["c"] == c0).mean()
    expect = _exchange_fraction(a, D, kappa, n * dt)
    assert abs(stay - expect) < Z * math.sqrt(0.25 / W) + 0.005, (stay, expect)
