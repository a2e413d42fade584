"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against a result obtained without it: closed forms
of the discrete walk, textbook limits of restricted diffusion, invariants the
paper states, and brute-force enumeration of single steps.  Statistical checks
use 4.5 standard errors estimated from the same run.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from conftest import make_workload

NT = os.cpu_count() or 1
Z = 4.5


def ds_of(D, dt):
    return math.sqrt(6.0 * D * dt)


# ------------------------------------------------------------ free walk (P2)

@pytest.mark.parametrize("n", [1, 2, 8])
def test_free_walk_moments(oracle_lib, n):
    """No membranes: per-axis <dx^2> = n ds^2/3 and
    <dx^4> = n ds^4/5 + 3 n (n-1) (ds^2/3)^2 (sums of n isotropic steps of
    length ds: one step projects to ds u with u uniform on [-1,1]);
    at n = 1 every displacement has length exactly ds (Eq. 1)."""
    W = 40000
    wl = make_workload(np.zeros((8, 8, 8)), voxel_um=0.2, D=2.0, dt=1e-3, n_steps=n, n_walkers=W,
                       seed=11 + n)
    r = oracle_lib.run(wl, n_threads=NT)
    assert r["err"] == 0
    dx = oracle_lib.displacement(r, wl.voxel_um)
    ds = ds_of(2.0, 1e-3)
    if n == 1:
        np.testing.assert_allclose(np.linalg.norm(dx, axis=1), ds, rtol=1e-13)
    m2x = ds * ds / 3
    m4x = n * ds ** 4 / 5 + 3 * n * (n - 1) * m2x ** 2
    for a in range(3):
        x2, x4 = dx[:, a] ** 2, dx[:, a] ** 4
        assert abs(x2.mean() - n * m2x) < Z * x2.std() / math.sqrt(W)
        assert abs(x4.mean() - m4x) < Z * x4.std() / math.sqrt(W)
    # every one of the 22 moment sums against the isotropic-step expectation:
    # a product with an odd power of some axis averages 0; x_a^2 x_b^2 (a != b)
    # averages n ds^4/15 + n (n-1) (ds^2/3)^2 (one step: <u_a^2 u_b^2> = 1/15)
    M = r["moments"][-1]
    np.testing.assert_allclose(M[0], W, rtol=1e-14)
    m22 = n * ds ** 4 / 15 + n * (n - 1) * m2x ** 2
    for q, name in enumerate(oracle_lib.MOMENT_NAMES[1:], start=1):
        powers = [name.count(ax) for ax in "xyz"]
        prod = np.prod([dx[:, a] ** powers[a] for a in range(3)], axis=0)
        if any(p % 2 for p in powers):
            expect = 0.0
        elif len(name) == 2:
            expect = n * m2x
        elif 4 in powers:
            expect = m4x
        else:
            expect = m22
        assert abs(M[q] / W - expect) < Z * prod.std() / math.sqrt(W), (name, M[q] / W, expect)
        # and the sum the oracle accumulated is that of its exported final positions
        assert abs(M[q] - prod.sum()) <= 1e-12 * np.abs(prod).sum(), name


def test_face_events_per_step(oracle_lib):
    """In a lattice the number of faces crossed by one step is the sum over
    axes of the number of integer planes crossed, expectation
    3 E|n_x| s = 1.5 ds / l_p."""
    W, n = 20000, 10
    wl = make_workload(np.zeros((8, 8, 8)), voxel_um=0.2, D=2.0, dt=1e-3, n_steps=n, n_walkers=W)
    r = oracle_lib.run(wl, n_threads=NT)
    ev = r["counts"][:, 0] / n
    assert abs(ev.mean() - 1.5 * ds_of(2.0, 1e-3) / 0.2) < Z * ev.std() / math.sqrt(W)
    assert r["counts"][:, 1].sum() == 0 and r["counts"][:, 2].sum() == 0


def test_free_walk_signal_exact(oracle_lib):
    """Free walk: phi = q sum_j g.dx_j H_j with H_j = dt sum_{k>=j} G_k and
    independent isotropic steps dx_j of length ds, so
    E e^{-i phi} = prod_j sinc(q H_j ds) exactly (sinc x = sin x / x)."""
    W, n, dt = 40000, 60, 1e-3
    G = np.zeros(n)
    G[:20] = 1.0
    G[40:60] = -1.0
    wl = make_workload(np.zeros((8, 8, 8)), voxel_um=0.2, D=2.0, dt=dt, n_steps=n, G=G,
                       dirs=np.array([[1, 0, 0], [0, 0.6, 0.8]]), b=np.array([0.0, 0.5, 1.0, 2.0]),
                       n_walkers=W, seed=5)
    r = oracle_lib.run(wl, n_threads=NT)
    S, asum = oracle_lib.readout(r, wl)
    assert asum == W
    bs = oracle_lib.bvalue(G, dt)
    H = dt * np.cumsum(G[::-1])[::-1]
    ds = ds_of(2.0, dt)
    for ib, b in enumerate(wl.b):
        q = math.sqrt(b / bs)
        x = q * H * ds
        expect = np.prod(np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x)))
        for g in range(2):
            phi = q * (r["phase"][:, 0, :] @ wl.dirs[g])
            se = max(np.cos(phi).std(), 1e-3) / math.sqrt(W)
            assert abs(S[0, g, ib].real - expect) < Z * se, (b, g, S[0, g, ib], expect)
            assert abs(S[0, g, ib].imag) < Z * max(np.sin(phi).std(), 1e-3) / math.sqrt(W)
    # b = 0 gives S = 1 exactly (Eq. 7: S = 1 without diffusion weighting)
    assert np.all(S[0, :, 0] == 1.0)


def test_bvalue_discrete_sum_exact():
    """b_s = dt sum_{j=1..N} F_{j-1}^2 with F_j = dt sum_{k<=j} G_k, compared
    with exact rational arithmetic on the same binary inputs, and with the
    continuous-time delta^2 (Delta - delta/3) (Sec. 2.3) to O(dt)."""
    import oracle
    import rms_inputs as ri
    dt = 2.0 ** -10
    n = 4 * 1024
    G = ri.pgse(1.0, 3.0, dt, n)
    bs = oracle.bvalue(G, dt)
    F = Fraction(0)
    acc = Fraction(0)
    fdt = Fraction(dt)
    for j in range(n):
        acc += F * F
        F += fdt * Fraction(float(G[j]))
    exact = fdt * acc
    assert abs(Fraction(bs) - exact) <= exact * Fraction(1, 10 ** 15)
    assert abs(bs - 1.0 * (3.0 - 1.0 / 3.0)) < 4 * dt


# ------------------------------------------------------- single steps (P7, P8)

def _lattice_wl(labels, kappa, D=2.0, dt=1e-3, voxel=0.2):
    return make_workload(labels, voxel_um=voxel, D=D, kappa=kappa, dt=dt, n_steps=1)


def test_corner_reflector(oracle_lib):
    """Fig. 2: three impermeable faces at a corner send n -> -n; the
    unfolded end point o + s n is mirrored on every axis."""
    lab = np.arange(8).reshape(2, 2, 2)
    wl = _lattice_wl(lab, 0.0, D=2.0, dt=1e-3)
    s = ds_of(2.0, 1e-3) / 0.2
    n0 = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    o0 = np.array([0.8, 0.85, 0.9])
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [0, 0, 0], o0, 0, n0.copy())
    assert err == 0
    np.testing.assert_array_equal(i, [0, 0, 0])
    np.testing.assert_allclose(o, 2.0 - (o0 + s * n0), rtol=0, atol=1e-14)
    np.testing.assert_array_equal(n, -n0)
    assert list(counts) == [3, 0, 3] and c == 0


def test_cross_into_other_diffusivity_keeps_time_fraction(oracle_lib):
    """Crossing at fraction t of the step into a label with step length s2
    continues for the remaining fraction 1 - t at s2 (the remaining time
    is kept); T2 weights accrue per segment (Eq. 5)."""
    lab = np.array([[[0, 1]]])
    D = np.array([2.0, 0.5])
    wl = make_workload(lab, voxel_um=0.2, D=D, kappa=1e6, T2=np.array([40.0, 80.0]), dt=1e-3,
                       n_steps=1)
    s1, s2 = ds_of(2.0, 1e-3) / 0.2, ds_of(0.5, 1e-3) / 0.2
    o_x = 1.0 - 0.3 * s1
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [0, 0, 0], [o_x, 0.5, 0.5], 0, [1.0, 0, 0],
                                                      perm=[0, 0, 0])
    assert err == 0 and c == 1 and list(i) == [1, 0, 0]
    np.testing.assert_allclose(o[0], 0.7 * s2, atol=1e-14)
    np.testing.assert_allclose(A, 0.3 * 1e-3 / 40.0 + 0.7 * 1e-3 / 80.0, rtol=1e-12)
    # the same event with a PERM word above the threshold reflects
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [0, 0, 0], [o_x, 0.5, 0.5], 0, [1.0, 0, 0],
                                                      perm=[0xFFFFFFFF] * 3)
    assert c == 0 and list(i) == [0, 0, 0] and n[0] == -1.0
    np.testing.assert_allclose(o[0], 1.0 - 0.7 * s1, atol=1e-14)


def test_non_periodic_edge_is_a_wall(oracle_lib):
    lab = np.zeros((1, 1, 2))
    wl = make_workload(lab, voxel_um=0.2, D=2.0, dt=1e-3, n_steps=1, periodic=(0, 1, 1))
    s = ds_of(2.0, 1e-3) / 0.2
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [1, 0, 0], [0.95, 0.5, 0.5], 0, [1.0, 0, 0])
    assert list(i) == [1, 0, 0] and n[0] == -1.0
    np.testing.assert_allclose(o[0], 1.0 - (s - 0.05), atol=1e-14)


def _brute_force_step(labels, T, s, i, o, c, n, perm):
    """Equal step length in every label.  Reflections on an axis-aligned face
    change only that axis's component, so each axis's face time is
    t_a = dist_a / |d_a| from the start, independent of the other axes; sort
    the events by time (ties: lower axis), take the crossing decisions in
    that order, then unfold each axis: crossed -> p - 1 (or p + 1),
    reflected -> 2 - p (or -p), untouched -> p, with p = o + s n."""
    nz, ny, nx = labels.shape
    N = (nx, ny, nz)
    d = s * np.asarray(n, float)
    hits = []
    for a in range(3):
        if d[a] > 0 and 1 - o[a] < d[a]:
            hits.append(((1 - o[a]) / d[a], a))
        elif d[a] < 0 and o[a] < -d[a]:
            hits.append((o[a] / -d[a], a))
    hits.sort()
    i = list(i)
    crossed, reflected = set(), set()
    for e, (_, a) in enumerate(hits):
        j = list(i)
        j[a] += 1 if d[a] > 0 else -1
        c2 = int(labels[j[2] % N[2], j[1] % N[1], j[0] % N[0]])
        if c2 == c or perm[e] < T[c, c2]:
            i, c = j, c2
            crossed.add(a)
        else:
            reflected.add(a)
    p = np.asarray(o) + d
    o2 = p.copy()
    n2 = np.array(n, float)
    for a in range(3):
        if a in crossed:
            o2[a] = p[a] - 1 if d[a] > 0 else p[a] + 1
        elif a in reflected:
            o2[a] = 2 - p[a] if d[a] > 0 else -p[a]
            n2[a] = -n2[a]
    return i, o2, c, n2, len(hits), len(crossed), len(reflected), [t for t, _ in hits]


def test_single_steps_match_brute_force(oracle_lib):
    """2x2x2 periodic lattice of random labels and permeabilities; random
    starts, directions and PERM words; every branch of the face walk."""
    rng = np.random.default_rng(7)
    checked = branches = 0
    for trial in range(400):
        lab = rng.integers(0, 3, size=(2, 2, 2))
        K = rng.uniform(0, 30.0, size=(3, 3))
        wl = _lattice_wl(lab, K, D=2.0, dt=1.5e-3, voxel=0.2)
        T, svec = oracle_lib.thresholds(wl)
        s = svec[0]
        i0 = list(rng.integers(-3, 3, size=3))
        c0 = int(lab[i0[2] % 2, i0[1] % 2, i0[0] % 2])
        v = rng.normal(size=3)
        n0 = v / np.linalg.norm(v)
        o0 = rng.uniform(0, 1, size=3)
        perm = [int(x) for x in rng.integers(0, 2 ** 32, size=3, dtype=np.uint64)]
        ref = _brute_force_step(lab, T, s, i0, o0, c0, n0, perm)
        times = ref[7]
        if any(abs(x - 1) < 1e-9 for x in times) or any(abs(a - b) < 1e-9 for a in times for b in times
                                                        if a is not b):
            continue
        i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, i0, o0, c0, n0.copy(), perm=perm)
        assert err == 0
        assert list(i) == list(ref[0]) and c == ref[2], trial
        np.testing.assert_allclose(o, ref[1], atol=1e-12)
        np.testing.assert_array_equal(n, ref[3])
        assert counts[0] == ref[4] and counts[2] == ref[6]
        checked += 1
        branches += ref[4]
    assert checked > 300 and branches > 300


# -------------------------------------------------- restricted diffusion (P3, P4)

def test_slab_long_time_limit(oracle_lib):
    """Impermeable slabs of width a: per-axis MSD normal to the walls -> a^2/6
    (twice the variance of a uniform density on [0, a]), free along the
    walls; narrow-pulse S(q) -> sinc^2(q a / 2) (Eq. A.2 with a uniform
    long-time propagator)."""
    a_vox, l_p, D, dt = 8, 0.2, 2.0, 1e-3
    a = a_vox * l_p
    n = 6400                                    # t = 5 a^2 / D
    W = 20000
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    G = np.zeros(n)
    G[0], G[-1] = 1.0, -1.0                     # narrow pulses: phase ~ q dt (x_1 - x_N)
    qa2 = np.array([math.pi / 2, math.pi, 1.5 * math.pi])
    import oracle
    bs = oracle.bvalue(G, dt)
    qeff = qa2 * 2 / a
    b = (qeff / dt) ** 2 * bs
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=n, G=G,
                       dirs=np.array([[1.0, 0, 0]]), b=b, n_walkers=W, seed=3)
    r = oracle_lib.run(wl, n_threads=NT)
    dx = oracle_lib.displacement(r, l_p)
    x2 = dx[:, 0] ** 2
    assert abs(x2.mean() - a * a / 6) < Z * x2.std() / math.sqrt(W)
    for ax in (1, 2):
        y2 = dx[:, ax] ** 2
        assert abs(y2.mean() - n * ds_of(D, dt) ** 2 / 3) < Z * y2.std() / math.sqrt(W)
    S, _ = oracle_lib.readout(r, wl)
    for k, x in enumerate(qa2):
        expect = (math.sin(x) / x) ** 2
        assert abs(S[0, 0, k].real - expect) < Z / math.sqrt(W) + 2e-3, (x, S[0, 0, k], expect)


def test_short_time_surface_to_volume_law(oracle_lib):
    """Mitra, Sen, Schwartz & Halperin (1992): D(t)/D0 = 1 - 4/(9 sqrt(pi))
    (S/V) sqrt(D0 t) at short times; slabs of width a have S/V = 2/a exactly
    on the voxel grid."""
    a_vox, l_p, D, dt = 30, 0.1, 2.0, 2e-4
    a = a_vox * l_p
    n = 1000
    t = n * dt
    W = 40000
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=0.0, dt=dt, n_steps=n, n_walkers=W, seed=9)
    r = oracle_lib.run(wl, n_threads=NT)
    dx = oracle_lib.displacement(r, l_p)
    r2 = (dx ** 2).sum(axis=1)
    Dt = r2.mean() / (6 * t)
    se = r2.std() / math.sqrt(W) / (6 * t)
    expect = D * (1 - 4 / (9 * math.sqrt(math.pi)) * (2 / a) * math.sqrt(D * t))
    assert abs(Dt - expect) < Z * se + 0.004 * D, (Dt, expect, se)
    assert D - Dt > 0.08 * D      # the restriction is seen at all


# ------------------------------------------------------ permeation (P5, P6)

def test_uniform_density_kept_across_unequal_diffusivity(oracle_lib):
    """Sec. 2.1.2 and App. C: elastic collisions with the corrected P keep a
    uniform density; P_{1->2} ds_1 = P_{2->1} ds_2 balances the flux across
    a membrane between D1 != D2 (the remaining-time rule after a crossing is
    part of what this checks)."""
    l_p, dt = 0.1, 5e-4
    D = np.array([2.0, 0.5])
    n, W = 4000, 20000
    lab = np.broadcast_to(np.array([0] * 10 + [1] * 10), (2, 2, 20))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=3.0, dt=dt, n_steps=n, n_walkers=W, seed=21)
    r = oracle_lib.run(wl, n_threads=NT)
    assert r["err"] == 0 and r["counts"][:, 1].sum() > 5 * W
    f1 = (r["c"] == 0).mean()
    assert abs(f1 - 0.5) < Z * math.sqrt(0.25 / W)
    x = (np.mod(r["i"][:, 0], 20) + r["o"][:, 0])
    hist, _ = np.histogram(x, bins=20, range=(0, 20))
    expect = W / 20
    assert np.all(np.abs(hist - expect) < Z * math.sqrt(expect)), hist
    T, _ = oracle_lib.thresholds(wl)
    ratio = T[0, 1] / T[1, 0]
    np.testing.assert_allclose(ratio, math.sqrt(D[1] / D[0]), rtol=1e-6)


def _exchange_fraction(a, D, kappa, t, nmodes=200):
    """Symmetric periodic slabs (width a, membranes kappa): fraction of walkers
    that start in slab 1 and are in it at t.  Antisymmetric modes cos(k x)
    with (k a / 2) tan(k a / 2) = kappa a / D, decay D k^2."""
    from scipy.optimize import brentq
    frac = 0.5
    g = kappa * a / D
    for m in range(nmodes):
        lo, hi = m * math.pi + 1e-12, m * math.pi + math.pi / 2 - 1e-12
        x = brentq(lambda x: x * math.tan(x) - g, lo, hi)
        k = 2 * x / a
        integ = 2 * math.sin(k * a / 2) / k
        norm = a / 2 + math.sin(k * a) / (2 * k)
        # h = +1/2 on slab 1, -1/2 on slab 2; its projection on the mode
        c = 0.5 * integ / norm
        frac += c * integ / a * math.exp(-D * k * k * t)
    return frac


def test_two_compartment_exchange(oracle_lib):
    """Exchange between slabs through permeable membranes: the fraction of
    walkers still in their starting slab follows the exact eigenmode
    solution, which in the barrier-limited case kappa a / D << 1 is
    Kaerger's f1 + (1 - f1) exp(-(k12 + k21) t), k = 2 kappa / a."""
    l_p, D, dt, kappa = 0.2, 2.0, 1e-3, 0.02
    a = 3 * l_p
    n, W = 6000, 20000
    lab = np.broadcast_to(np.array([0, 0, 0, 1, 1, 1]), (2, 2, 6))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=kappa, dt=dt, n_steps=n, n_walkers=W, seed=4)
    r = oracle_lib.run(wl, n_threads=NT)
    c0 = lab[np.mod(r["i0"][:, 2], 2), np.mod(r["i0"][:, 1], 2), np.mod(r["i0"][:, 0], 6)]
    stay = (r["c"] == c0).mean()
    t = n * dt
    expect = _exchange_fraction(a, D, kappa, t)
    karger = 0.5 + 0.5 * math.exp(-(4 * kappa / a) * t)
    assert abs(expect - karger) < 0.01
    assert abs(stay - expect) < Z * math.sqrt(0.25 / W), (stay, expect)


# ----------------------------------------------------------- relaxation (P10)

def test_relaxation_weights(oracle_lib):
    """Eq. 5: alpha = exp(-sum_i t_i / T^(i)).  Impermeable compartments:
    each walker stays in its label, so A = t / T2(label) up to rounding;
    steps flagged T1 use T1 instead."""
    n, dt, W = 500, 1e-3, 2000
    lab = np.broadcast_to(np.array([0] * 4 + [1] * 4), (2, 2, 8))
    mode = np.zeros(n, np.uint8)
    mode[100:200] = 1
    mode[300:320] = 2
    T2 = np.array([30.0, 70.0])
    T1 = np.array([500.0, 900.0])
    wl = make_workload(lab, voxel_um=0.2, D=2.0, kappa=0.0, T2=T2, T1=T1, dt=dt, n_steps=n,
                       n_walkers=W, mode=mode)
    r = oracle_lib.run(wl, n_threads=NT)
    c = r["c"]
    expect = (380 * dt) / T2[c] + (100 * dt) / T1[c]
    np.testing.assert_allclose(r["A"], expect, rtol=1e-12)
    M = r["moments"][-1]
    np.testing.assert_allclose(M[0], np.exp(-expect).sum(), rtol=1e-12)


def test_dead_label_never_entered(oracle_lib):
    """Sec. 2.2 item 1: no walker starts in or steps into dead space."""
    lab = np.zeros((8, 8, 8), np.uint16)
    lab[:, 2:5, 2:6] = 1
    wl = make_workload(lab, voxel_um=0.2, D=2.0, kappa=50.0, dt=1e-3, n_steps=300, n_walkers=3000,
                       dead=[0, 1])
    r = oracle_lib.run(wl, n_threads=NT)
    assert np.all(r["c"] == 0)
    c0 = lab[np.mod(r["i0"][:, 2], 8), np.mod(r["i0"][:, 1], 8), np.mod(r["i0"][:, 0], 8)]
    assert np.all(c0 == 0)
    assert r["counts"][:, 2].sum() > 0


def test_uniform_initial_density(oracle_lib):
    """Sec. 2.2 item 1: initial positions uniform over non-dead voxels."""
    lab = np.zeros((4, 4, 4), np.uint16)
    lab[0] = 1
    W = 64000
    wl = make_workload(lab, voxel_um=0.2, D=2.0, dt=1e-3, n_steps=0, n_walkers=W, dead=[0, 1])
    r = oracle_lib.run(wl, n_threads=NT)
    v = np.mod(r["i0"][:, 0], 4) + 4 * (np.mod(r["i0"][:, 1], 4) + 4 * np.mod(r["i0"][:, 2], 4))
    cnt = np.bincount(v, minlength=64)
    assert np.all(cnt[:16] == 0)
    e = W / 48
    assert np.all(np.abs(cnt[16:] - e) < Z * math.sqrt(e))
    for a in range(3):
        h, _ = np.histogram(r["o0"][:, a], bins=10, range=(0, 1))
        assert np.all(np.abs(h - W / 10) < Z * math.sqrt(W / 10))


def test_initial_position_uniform_jointly(oracle_lib):
    """Sec. 2.2 item 1, jointly: the start point (voxel and offset together)
    is uniform over the live volume, so each octant of each live voxel holds
    1/(8 n_live) of the walkers.  Per-axis histograms cannot see a word
    shared between two offsets, or between the voxel draw and an offset;
    either empties whole octants here."""
    lab = np.zeros((4, 4, 4), np.uint16)
    lab[0] = 1
    W = 192_000
    wl = make_workload(lab, voxel_um=0.2, D=2.0, dt=1e-3, n_steps=0, n_walkers=W, dead=[0, 1], seed=5)
    r = oracle_lib.run(wl, n_threads=NT)
    v = np.mod(r["i0"][:, 0], 4) + 4 * (np.mod(r["i0"][:, 1], 4) + 4 * np.mod(r["i0"][:, 2], 4))
    octant = (r["o0"] >= 0.5).astype(np.int64) @ np.array([1, 2, 4])
    cnt = np.bincount(v * 8 + octant, minlength=64 * 8)[16 * 8:]
    e = W / cnt.size
    assert np.all(np.abs(cnt - e) < Z * math.sqrt(e)), (cnt.min(), cnt.max(), e)
    chi2 = float(((cnt - e) ** 2 / e).sum())
    dof = cnt.size - 1
    assert abs(chi2 - dof) < Z * math.sqrt(2 * dof), chi2


def test_start_voxels_on_a_non_cubic_grid(oracle_lib):
    """Sec. 2.2 item 1 on a 3 x 5 x 4 grid (x, y, z) with an irregular dead
    label: every walker starts in a live voxel with that voxel's label, and
    the live voxels are equally likely (the raster order is x fastest, so a
    decode that mixes up the axis sizes breaks both)."""
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 3, size=(4, 5, 3))  # (nz, ny, nx)
    dead = np.array([0, 0, 1], np.uint8)
    W = 60_000
    wl = make_workload(lab, voxel_um=0.2, D=2.0, dt=1e-3, n_steps=0, n_walkers=W, dead=dead, seed=6)
    r = oracle_lib.run(wl, n_threads=NT)
    x, y, z = r["i0"][:, 0], r["i0"][:, 1], r["i0"][:, 2]
    assert x.min() >= 0 and x.max() < 3 and y.min() >= 0 and y.max() < 5 and z.min() >= 0 and z.max() < 4
    np.testing.assert_array_equal(lab[z, y, x], r["c"])
    live = dead[lab] == 0
    cnt = np.bincount((z * 5 + y) * 3 + x, minlength=60).reshape(4, 5, 3)
    assert np.all(cnt[~live] == 0)
    e = W / live.sum()
    assert np.all(np.abs(cnt[live] - e) < Z * math.sqrt(e)), (cnt[live].min(), cnt[live].max(), e)


def test_readout_weights_are_the_relaxation_weights(oracle_lib):
    """Eq. 5 and Eq. 7: S = sum alpha e^{-i phi} / sum alpha.  One label with
    T2 = TE / 2: every walker has alpha = e^{-2}, so sum alpha = W e^{-2}, and
    alpha cancels from S, which stays the exact free-walk signal
    prod_j sinc(q H_j ds)."""
    W, n, dt = 40000, 60, 1e-3
    G = np.zeros(n)
    G[:20] = 1.0
    G[40:60] = -1.0
    T2 = n * dt / 2.0
    wl = make_workload(np.zeros((8, 8, 8)), voxel_um=0.2, D=2.0, T2=T2, dt=dt, n_steps=n, G=G,
                       dirs=np.array([[1.0, 0, 0]]), b=np.array([0.0, 1.0]), n_walkers=W, seed=15)
    r = oracle_lib.run(wl, n_threads=NT)
    S, asum = oracle_lib.readout(r, wl)
    assert abs(asum - W * math.exp(-2.0)) < 1e-12 * asum
    assert abs(S[0, 0, 0] - 1.0) < 1e-12
    bs = oracle_lib.bvalue(G, dt)
    H = dt * np.cumsum(G[::-1])[::-1]
    x = math.sqrt(1.0 / bs) * H * ds_of(2.0, dt)
    expect = np.prod(np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x)))
    phi = math.sqrt(1.0 / bs) * r["phase"][:, 0, 0]
    assert abs(S[0, 0, 1].real - expect) < Z * np.cos(phi).std() / math.sqrt(W), (S[0, 0, 1], expect)


def test_tied_face_times_go_to_the_lower_axis(oracle_lib):
    """Two faces met at the same time (a diagonal step from a symmetric
    point): the x face is the step's event 0 and takes the first Bernoulli
    word, the y face event 1 and the second.  With the first word crossing
    and the second reflecting, the walker ends one voxel along x, mirrored
    in y (unfolded end point: x - 1, 2 - y)."""
    lab = np.zeros((2, 2, 2), np.int64)
    lab[:, 0, 1], lab[:, 1, 0], lab[:, 1, 1] = 1, 2, 3
    wl = _lattice_wl(lab, 5.0, D=2.0, dt=1e-3, voxel=0.2)
    T, svec = oracle_lib.thresholds(wl)
    s = svec[0]
    assert 0 < T[0, 1] < 2 ** 32 - 1 and T[1, 3] > 0
    n0 = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    o0 = np.array([0.8, 0.8, 0.5])
    assert (1 - 0.8) / (s * n0[0]) < 1.0
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [0, 0, 0], o0, 0, n0.copy(), perm=[0, 2 ** 32 - 1, 0])
    assert err == 0
    np.testing.assert_array_equal(i, [1, 0, 0])
    assert c == 1
    p = o0 + s * n0
    np.testing.assert_allclose(o, [p[0] - 1.0, 2.0 - p[1], 0.5], atol=1e-12)
    np.testing.assert_array_equal(n, [n0[0], -n0[1], 0.0])
    assert list(counts) == [2, 1, 1]


def test_trajectory_independent_of_thread_split(oracle_lib):
    wl = make_workload(np.arange(8).reshape(2, 2, 2) % 3, voxel_um=0.2, D=2.0, kappa=5.0, dt=1e-3,
                       n_steps=200, n_walkers=500, seed=99)
    r1 = oracle_lib.run(wl, n_threads=1)
    r2 = oracle_lib.run(wl, n_threads=7)
    r3 = oracle_lib.run(wl, w_begin=100, w_end=300, n_threads=3)
    for k in ("i", "o", "c", "A", "phase", "hash"):
        np.testing.assert_array_equal(r1[k], r2[k])
        np.testing.assert_array_equal(r1[k][100:300], r3[k])


def test_each_face_decision_is_an_independent_trial(oracle_lib):
    """Every voxel its own label, one kappa for every pair and ds = 0.9
    voxel, so a step meets up to three membranes (Sec. 2.2 items 3-4): with
    equal D the number N of face events is set by the start and the
    direction alone, and each event crosses with the same P, on its own
    Bernoulli word.  Among walkers with N events the crossings are then
    Binomial(N, P), with P = T/2^32 of the threshold table and T from Eq. 3
    at P ~ 1/2 (a shared or reused word would put no mass on 0 < k < N)."""
    lab = np.arange(64).reshape(4, 4, 4)
    l_p, D = 0.1, 2.0
    dt = (0.9 * l_p) ** 2 / (6 * D)
    kappa = D / (ds_of(D, dt) * 2.0 / 3.0)        # kappa ds C3 / D = 1: P = 1/2 by Eq. 3
    W = 400_000
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=kappa, dt=dt, n_steps=1, n_walkers=W, seed=12)
    T, _ = oracle_lib.thresholds(wl)
    P = float(T[0, 1]) / 2.0 ** 32
    assert abs(P - 0.5) < 1e-9 and np.all(T[~np.eye(64, dtype=bool)] == T[0, 1])
    r = oracle_lib.run(wl, n_threads=NT, hash_=False)
    ev, cross, refl = r["counts"][:, 0], r["counts"][:, 1], r["counts"][:, 2]
    np.testing.assert_array_equal(ev, cross + refl)   # every face is a membrane
    for N in (1, 2, 3):
        m = ev == N
        n = int(m.sum())
        assert n > 2000, N
        for k in range(N + 1):
            expect = math.comb(N, k) * P ** k * (1 - P) ** (N - k)
            f = float((cross[m] == k).mean())
            assert abs(f - expect) < Z * math.sqrt(expect * (1 - expect) / n), (N, k, f, expect)


def test_finite_step_permeability_correction(oracle_lib):
    """App. C, Eq. C.7: with the uncorrected P of Eq. 2 the walk realises
    kappa / (1 - alpha), alpha = (P12 + P21) / 2; Eq. 3 removes this to first
    order.  Coarse steps (ds = 0.15 a, alpha ~ 0.17) make the difference
    large: the exchange fraction must follow the exact solution for the
    input kappa (the uncorrected P lands ~0.024 below it), allowing 0.003 for
    second-order step effects."""
    D, kappa, ds, l_p, a_vox = 1.0, 2.0, 0.15, 0.2, 5
    dt = ds * ds / (6 * D)
    a = a_vox * l_p
    n, W = 67, 200000
    lab = np.broadcast_to(np.array([0] * a_vox + [1] * a_vox), (2, 2, 2 * a_vox))
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=kappa, dt=dt, n_steps=n, n_walkers=W, seed=4)
    r = oracle_lib.run(wl, n_threads=NT)
    c0 = lab[np.mod(r["i0"][:, 2], 2), np.mod(r["i0"][:, 1], 2), np.mod(r["i0"][:, 0], 2 * a_vox)]
    stay = (r["c"] == c0).mean()
    expect = _exchange_fraction(a, D, kappa, n * dt)
    T, _ = oracle_lib.thresholds(wl)
    alpha = T[0, 1] / 2.0 ** 32
    assert alpha > 0.15
    uncorrected = _exchange_fraction(a, D, kappa / (1 - alpha), n * dt)
    assert expect - uncorrected > 0.015
    assert abs(stay - expect) < Z * math.sqrt(0.25 / W) + 0.003, (stay, expect, uncorrected)


def test_direction_sampler_closed_form(oracle_lib):
    """The direction of words (x0, x1) is (r cos phi, r sin phi, z) with
    z = 1 - 2 (x0 + 1/2) 2^-32, r = sqrt(1 - z^2), phi = 2 pi (x1 + 1/2) 2^-32
    (Archimedes: z uniform on [-1, 1] gives a uniform point of the sphere);
    checked against libm on words covering every octant and its edges."""
    rng = np.random.default_rng(17)
    words = list(rng.integers(0, 2 ** 32, size=(3000, 2), dtype=np.uint64))
    for o in range(8):
        for m in (0, 1, 0x1FFFFFFE, 0x1FFFFFFF, 0x0FFFFFFF):
            words.append(np.array([int(rng.integers(0, 2 ** 32)), (o << 29) | m], dtype=np.uint64))
    words += [np.array([0, 0], np.uint64), np.array([2 ** 32 - 1, 2 ** 32 - 1], np.uint64)]
    for x0, x1 in words:
        n = oracle_lib.direction_from_words(int(x0), int(x1))
        z = 1.0 - 2.0 * (int(x0) + 0.5) * 2.0 ** -32
        phi = 2 * math.pi * (int(x1) + 0.5) * 2.0 ** -32
        r = math.sqrt((1 - z) * (1 + z))  # 1 - z and 1 + z are exact
        np.testing.assert_allclose(n, [r * math.cos(phi), r * math.sin(phi), z], rtol=0, atol=1e-15)
        assert abs(np.dot(n, n) - 1.0) < 1e-15


def test_speed_change_brings_a_face_inside_the_step(oracle_lib):
    """Hand-derived step: from o = (0.95, 0.75, 0.5) with n = (0.6, 0.8, 0) in
    a slow label (D = 0.5), the x face is crossed at t1 = 0.05 / (0.6 s0) into
    a fast label (D = 3); at the old speed the y face (0.25 away) would lie
    beyond the step (0.25 / (0.8 s0) > 1), at the new speed it is met at
    t2 = t1 + (0.25 - 0.8 s0 t1) / (0.8 s1) < 1 and reflects (impermeable)."""
    lab = np.array([[[0, 1], [2, 2]]])            # (z, y, x): (0,0)=0, (1,0)=1, y=1 row = 2
    D = np.array([0.5, 3.0, 1.0])
    K = np.zeros((3, 3))
    K[0, 1] = 1e6                                 # 0 -> 1 always crosses, 1 -> 2 never
    dt, l_p = 1e-3, 0.2
    wl = make_workload(lab, voxel_um=l_p, D=D, kappa=K, dt=dt, n_steps=1, periodic=(1, 1, 0))
    s0, s1 = ds_of(0.5, dt) / l_p, ds_of(3.0, dt) / l_p
    t1 = 0.05 / (0.6 * s0)
    assert 0.25 / (0.8 * s0) > 1.0
    t2 = t1 + (0.25 - 0.8 * s0 * t1) / (0.8 * s1)
    assert t2 < 1.0
    i, o, c, A, n, counts, err = oracle_lib.walk_once(wl, [0, 0, 0], [0.95, 0.75, 0.5], 0, [0.6, 0.8, 0.0],
                                                      perm=[0, 0, 0])
    assert err == 0 and list(i) == [1, 0, 0] and c == 1
    np.testing.assert_allclose(o, [(1 - t1) * 0.6 * s1, 1 - (1 - t2) * 0.8 * s1, 0.5], atol=1e-14)
    np.testing.assert_array_equal(n, [0.6, -0.8, 0.0])
    assert list(counts) == [2, 1, 1]
