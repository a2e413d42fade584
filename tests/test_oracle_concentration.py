"""Pins of the oracle's permeation with spin concentrations (App. C.2: the
generalised Eq. 3 with (c2/c1)^lambda factors and the finite-step
correction) and of Baxter's concentration rule (App. C.3, with its effective
permeability kappa' = kappa0' / (1 - beta), kappa0' = sqrt(D2 / (6 dt)) / C_3).
Statistical checks use 4.5 standard errors."""
import math
import os

import numpy as np
import pytest

from conftest import make_workload

NT = os.cpu_count() or 1
Z = 4.5


def _stay_fraction(a1, a2, D1, D2, kappa, f12, f21, t, n=200):
    """Periodic pair of slabs (widths a1, a2; D1, D2) with membranes of flux
    j = kappa (rho1 f12 - rho2 f21) from 1 to 2 and continuous D d_x rho:
    the fraction of walkers that start uniformly in slab 1 and are in it at
    time t.  Finite volumes (n cells per slab; at a membrane the half-cell
    diffusion resistances h f / (2 D) add to 1/kappa), propagated exactly by
    the matrix exponential; kappa = inf is no barrier."""
    from scipy.linalg import expm
    h = np.r_[np.full(n, a1 / n), np.full(n, a2 / n)]
    D = np.r_[np.full(n, D1), np.full(n, D2)]
    N = 2 * n
    M = np.zeros((N, N))
    ik = 0.0 if math.isinf(kappa) else 1.0 / kappa
    for i in range(N):
        j = (i + 1) % N
        if (i < n) == (j < n):
            cl = cr = D[i] / h[i]
        else:
            fl, fr = (f12, f21) if i < n else (f21, f12)
            den = ik + h[i] * fl / (2 * D[i]) + h[j] * fr / (2 * D[j])
            cl, cr = fl / den, fr / den
        M[i, i] -= cl / h[i]
        M[i, j] += cr / h[i]
        M[j, i] += cl / h[j]
        M[j, j] -= cr / h[j]
    rho0 = np.r_[np.ones(n), np.zeros(n)]
    r = expm(M * t) @ rho0
    return float((r[:n] * h[:n]).sum() / (rho0 * h).sum())


def _lambda12(lam, c1, c2, D1, D2):
    return 1.0 / (1.0 + c2 * math.sqrt(D2) / (c1 * math.sqrt(D1))) if lam < 0 else lam


def slabs(a1, a2):
    return np.broadcast_to(np.array([0] * a1 + [1] * a2), (2, 2, a1 + a2))


def start_label(r, lab):
    n = lab.shape[2]
    return lab[0, 0, np.mod(r["i0"][:, 0], n)]


def test_solver_reduces_to_the_eigenmode_solution():
    """f = 1 and equal D: the finite-volume solution equals the exact
    eigenmode series of the symmetric exchange problem."""
    from test_oracle_pins import _exchange_fraction
    assert abs(_stay_fraction(0.6, 0.6, 2.0, 2.0, 0.02, 1, 1, 6.0) - _exchange_fraction(0.6, 2.0, 0.02, 6.0)) < 1e-6


def test_equal_concentrations_change_nothing(oracle_lib):
    """c the same for every label: (c2/c1)^lambda = 1 and every start is
    accepted, so every walker follows the same path bit for bit."""
    rng = np.random.default_rng(5)
    lab = rng.integers(0, 3, size=(5, 6, 7))
    D = np.array([2.0, 0.7, 1.3])
    dt = 0.8 * 0.04 / (6 * D.max())
    base = dict(voxel_um=0.2, D=D, kappa=rng.uniform(0, 1.0, (3, 3)), T2=[40.0, 60.0, 80.0], dt=dt, n_steps=150,
                G=rng.normal(size=(1, 150)), n_walkers=2000, seed=3)
    a = oracle_lib.run(make_workload(lab, **base), n_threads=NT)
    b = oracle_lib.run(make_workload(lab, conc=[2.5, 2.5, 2.5], lam=-1.0, **base), n_threads=NT)
    for k in ("i", "o", "i0", "o0", "c", "A", "phase", "hash"):
        np.testing.assert_array_equal(a[k], b[k])


def test_initial_density_follows_concentration(oracle_lib):
    """App. C.2: at equilibrium the spin density is proportional to c, so
    walkers start in label l with probability c_l V_l / sum c V."""
    lab = slabs(3, 5)
    conc = np.array([1.0, 0.3])
    W = 400000
    wl = make_workload(lab, voxel_um=0.2, D=[2.0, 1.0], kappa=0.1, dt=1e-3, n_steps=0, n_walkers=W, seed=8,
                       conc=conc)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    assert r["err"] == 0
    f = (r["c"] == 0).mean()
    expect = conc[0] * 3 / (conc[0] * 3 + conc[1] * 5)
    assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / W), (f, expect)


def test_start_offsets_stay_uniform_with_concentrations(oracle_lib):
    """The concentration-weighted start changes only how often each label is
    chosen: inside the chosen voxel the offset stays uniform on every axis,
    in the low-concentration label too (the acceptance uses a word of its
    own, not one of the offset's)."""
    lab = slabs(3, 5)
    conc = np.array([1.0, 0.3])
    W = 200000
    wl = make_workload(lab, voxel_um=0.2, D=[2.0, 1.0], kappa=0.1, dt=1e-3, n_steps=0, n_walkers=W, seed=9,
                       conc=conc)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    assert r["err"] == 0
    for c in (0, 1):
        m = r["c"] == c
        for a in range(3):
            h, _ = np.histogram(r["o0"][m, a], bins=10, range=(0, 1))
            e = m.sum() / 10
            assert np.all(np.abs(h - e) < Z * math.sqrt(e)), (c, a, h, e)


@pytest.mark.parametrize("model", ["kappa-lambda0", "kappa-optimal", "baxter"])
def test_threshold_ratio_keeps_equilibrium(oracle_lib, model):
    """P12 / P21 = c2 sqrt(D2) / (c1 sqrt(D1)) for every pair, which keeps
    the density ratio c1/c2 (App. C.2); Baxter's rule has P = 1 from the
    low-flux side."""
    L = 4
    rng = np.random.default_rng(9)
    D = rng.uniform(0.5, 2.5, L)
    conc = rng.uniform(0.2, 1.5, L)
    dt = 0.5 * 0.04 / (6 * D.max())
    lam = {"kappa-lambda0": 0.0, "kappa-optimal": -1.0, "baxter": -1.0}[model]
    wl = make_workload(np.arange(L).reshape(1, 1, L), voxel_um=0.2, D=D, kappa=0.05, dt=dt, conc=conc, lam=lam,
                       perm_model=1 if model == "baxter" else 0)
    T, _ = oracle_lib.thresholds(wl)
    for a in range(L):
        for b in range(L):
            if a == b:
                continue
            ratio = conc[b] * math.sqrt(D[b]) / (conc[a] * math.sqrt(D[a]))
            if model == "baxter":
                expect = min(ratio, 1.0) * 2.0 ** 32
                assert abs(float(T[a, b]) - min(expect, 2.0 ** 32 - 1)) <= 1.0
            else:
                assert abs(T[a, b] / T[b, a] - ratio) < 1e-6 * ratio + 2.0 / T[b, a]
                # App. C.2 read backwards: the input permeability is the genuine one,
                # kappa = kappa0 / (1 - alpha_lambda), alpha_lambda = (P12 + P21) / 2,
                # with kappa0 = P12 D1 / (ds1 C_3 f12)
                P12, P21 = T[a, b] / 2.0 ** 32, T[b, a] / 2.0 ** 32
                l12 = _lambda12(lam, conc[a], conc[b], D[a], D[b]) if (lam < 0 or a < b) else 1 - lam
                f12 = (conc[b] / conc[a]) ** l12
                kappa0 = P12 * D[a] / (math.sqrt(6 * D[a] * dt) * (2.0 / 3.0) * f12)
                assert abs(kappa0 / (1 - (P12 + P21) / 2) - 0.05) < 1e-6


@pytest.mark.parametrize("model", ["kappa", "baxter"])
def test_equilibrium_is_stationary(oracle_lib, model):
    """Start at the equilibrium (density ~ c, unequal D): the occupancy of
    each compartment stays c_l V_l / sum c V and the density stays flat
    inside each compartment."""
    lab = slabs(3, 4)
    conc = np.array([1.0, 0.4])
    W, n = 200000, 1500
    wl = make_workload(lab, voxel_um=0.2, D=[2.0, 0.7], kappa=0.5, dt=1e-3, n_steps=n, n_walkers=W, seed=10,
                       conc=conc, lam=0.5, perm_model=1 if model == "baxter" else 0)
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    assert r["err"] == 0
    moved = (r["c"] != start_label(r, lab)).mean()
    assert moved > 0.1
    f = (r["c"] == 0).mean()
    expect = conc[0] * 3 / (conc[0] * 3 + conc[1] * 4)
    assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / W), (f, expect)
    col = np.mod(r["i"][:, 0], 7)
    counts = np.bincount(col, minlength=7).astype(float)
    for cols, cl in ((range(0, 3), 0), (range(3, 7), 1)):
        per = counts[list(cols)]
        mean = W * expect / 3 if cl == 0 else W * (1 - expect) / 4
        assert np.all(np.abs(per - mean) < Z * np.sqrt(mean)), (cl, per, mean)


@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0, -1.0])
def test_exchange_with_concentrations(oracle_lib, lam):
    """The generalised Eq. 3 gives the genuine permeability kappa of the
    flux j = kappa (rho1 (c2/c1)^lambda - rho2 (c2/c1)^(lambda-1)): the
    fraction of walkers still in their starting slab follows the
    two-compartment solution with that jump condition (for fixed lambda and
    the alpha-minimising one), far from the same kappa without the factors."""
    D1, D2, c1, c2 = 2.0, 1.0, 1.0, 0.5
    l_p, dt, kappa = 0.2, 1e-3, 0.1
    a = 3 * l_p
    lab = slabs(3, 3)
    l12 = _lambda12(lam, c1, c2, D1, D2)
    f12, f21 = (c2 / c1) ** l12, (c1 / c2) ** (1 - l12)
    for t in (1.0, 3.0):
        n, W = int(round(t / dt)), 40000
        wl = make_workload(lab, voxel_um=l_p, D=[D1, D2], kappa=kappa, dt=dt, n_steps=n, n_walkers=W, seed=6,
                           conc=[c1, c2], lam=lam)
        r = oracle_lib.run(wl, n_threads=NT, hash_=False)
        m = start_label(r, lab) == 0
        f = (r["c"][m] == 0).mean()
        se = math.sqrt(f * (1 - f) / m.sum())
        expect = _stay_fraction(a, a, D1, D2, kappa, f12, f21, t)
        assert abs(f - expect) < Z * se + 0.003, (t, f, expect)
        assert abs(f - _stay_fraction(a, a, D1, D2, kappa, 1.0, 1.0, t)) > 10 * se


def test_baxter_effective_permeability(oracle_lib):
    """App. C.3: Baxter's rule behaves as a membrane of permeability
    kappa' = kappa0' / (1 - beta), kappa0' = sqrt(D2 / (6 dt)) / C_3 (side 2
    the low-flux one), beta = (P12 + P21) / 2 -- finite, and growing as
    1/sqrt(dt) -- in the jump condition j = kappa' (rho1 c2/c1 - rho2): at two
    time steps the exchange follows that kappa' (within a first-order
    allowance of 0.004) and not the barrier-free limit kappa' -> inf."""
    D1, D2, c1, c2 = 2.0, 1.0, 1.0, 0.5
    l_p = 0.2
    a = 5 * l_p
    lab = slabs(5, 5)
    P12 = c2 * math.sqrt(D2) / (c1 * math.sqrt(D1))
    beta = (P12 + 1.0) / 2
    for dt in (1e-3, 3e-3):
        kp = math.sqrt(D2 / (6 * dt)) / (2.0 / 3.0) / (1 - beta)
        t = 0.06
        n, W = int(round(t / dt)), 400000
        wl = make_workload(lab, voxel_um=l_p, D=[D1, D2], kappa=1.0, dt=dt, n_steps=n, n_walkers=W, seed=5,
                           conc=[c1, c2], perm_model=1)
        r = oracle_lib.run(wl, n_threads=NT, hash_=False)
        m = start_label(r, lab) == 0
        f = (r["c"][m] == 0).mean()
        se = math.sqrt(f * (1 - f) / m.sum())
        expect = _stay_fraction(a, a, D1, D2, kp, c2 / c1, 1.0, n * dt)
        free = _stay_fraction(a, a, D1, D2, math.inf, c2 / c1, 1.0, n * dt)
        assert abs(f - expect) < Z * se + 0.004, (dt, f, expect)
        assert f - free > Z * se + 0.004, (dt, f, free)
