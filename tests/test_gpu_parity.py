"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Plain FP64 form: every walker's final voxel, offset, label, relaxation
exponent, phase vectors and trajectory checksum are bit-identical to the
oracle's; the signal agrees to 1e-12 * max(|S|, 1e-3) and the moment sums to
1e-12 of their magnitude (summation order differs).  FP32 form: |dS| <= 1e-3,
|dD|/D <= 1%, |dK| <= 0.01 max(|K|, 0.1).
"""
import math
import os

import numpy as np
import pytest

from conftest import make_workload

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


def assert_walkers_equal(g, o, sl=slice(None)):
    for k in ("i", "o", "c", "A", "phase", "hash"):
        a, b = g[k], o[k][sl] if sl != slice(None) else o[k]
        if k in ("i", "c"):
            b = b.astype(a.dtype)
        bad = np.nonzero(~(a == b).reshape(a.shape[0], -1).all(axis=1))[0]
        assert bad.size == 0, f"{k}: {bad.size} walkers differ, first {bad[:5]}: gpu {a[bad[0]]} oracle {b[bad[0]]}"
    np.testing.assert_array_equal(g["i0"], o["i0"][sl] if sl != slice(None) else o["i0"])
    np.testing.assert_array_equal(g["o0"], o["o0"][sl] if sl != slice(None) else o["o0"])


def moment_scale(M):
    """Per-entry magnitude bound of the moment sums: sum alpha |products| is at
    most (M_ii + M_jj)/2 for second order and sum alpha r^4 for fourth order."""
    M = np.atleast_2d(M)
    sc = np.zeros_like(M)
    sc[:, 0] = np.abs(M[:, 0])
    d2 = {0: M[:, 1], 1: M[:, 4], 2: M[:, 6]}
    p = 1
    for a in range(3):
        for b in range(a, 3):
            sc[:, p] = 0.5 * (d2[a] + d2[b])
            p += 1
    r4 = M[:, 7] + M[:, 17] + M[:, 21] + 2 * (M[:, 10] + M[:, 12] + M[:, 19])
    sc[:, 7:] = r4[:, None]
    return sc


def assert_moments_close(Mg, Mo, rtol=1e-12):
    sc = moment_scale(Mo)
    assert np.all(np.abs(Mg - Mo) <= rtol * sc + 1e-300), np.max(np.abs(Mg - Mo) / (sc + 1e-300))


def assert_signal_close(Sg, So, tol=1e-12):
    err = np.abs(Sg - So) / np.maximum(np.abs(So), 1e-3)
    assert err.max() <= tol, err.max()


def run_both(rms, oracle, wl, precision=None, hash_=True, spl=0, w_begin=0, n=None):
    precision = rms.RMS_FP64 if precision is None else precision
    W = wl.n_walkers if n is None else n
    g = rms.simulate(wl, precision, n_walkers=W, hash_=hash_, walker_begin=w_begin, steps_per_launch=spl,
                     walkers=True)
    o = oracle.run(wl, w_begin, w_begin + W, n_threads=NT, hash_=hash_)
    assert o["err"] == 0
    S_o, asum_o = oracle.readout(o, wl)
    return g, o, S_o, asum_o


def test_cylinder_plain_fp64_bit_exact(rms, oracle):
    """The plain FP64 check case in full: 32^3 cylinder, 1e4 walkers, 5000 steps."""
    import rms_inputs as ri
    wl = ri.workload("cylinder-32^3")
    g, o, S_o, asum_o = run_both(rms, oracle, wl)
    assert_walkers_equal(g, o)
    assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)
    assert abs(g["alpha_sum"] - asum_o) <= 1e-12 * asum_o


def _rand_case(seed, shape=(7, 5, 6), L=4, n_steps=300, W=777, S=3, periodic=(1, 1, 0), dead=None, mode=True):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, L, size=shape)
    D = rng.uniform(0.5, 2.5, size=L)
    dt = 0.9 * (0.2 ** 2) / (6 * D.max())
    K = rng.uniform(0, 3.0, size=(L, L))
    T2 = rng.uniform(30, 90, size=L)
    T1 = rng.uniform(500, 900, size=L)
    G = rng.normal(size=(S, n_steps)) * (rng.uniform(size=(S, n_steps)) < 0.3)
    md = rng.integers(0, 3, size=n_steps).astype(np.uint8) if mode else None
    rec = np.unique(rng.integers(1, n_steps + 1, size=7)) if n_steps else np.zeros(0, np.int64)
    return make_workload(lab, voxel_um=0.2, D=D, kappa=K, T2=T2, T1=T1, dt=dt, n_steps=n_steps, G=G,
                         dirs=rng.normal(size=(5, 3)) / math.sqrt(3), b=np.array([0.0, 0.3, 1.7]),
                         rec_steps=rec, n_walkers=W, seed=seed, periodic=periodic, dead=dead, mode=md)


@pytest.mark.parametrize("case", [
    dict(seed=1),
    dict(seed=2, S=1, periodic=(0, 0, 0)),
    dict(seed=3, S=5, shape=(3, 9, 4), W=129),
    dict(seed=4, S=2, dead=[0, 0, 1, 0], W=1000),
    dict(seed=5, W=1, n_steps=50),
    dict(seed=6, W=300, n_steps=0),
    dict(seed=7, shape=(1, 1, 2), L=2, W=500, S=8),
    dict(seed=8, mode=False, L=1, W=4096, shape=(4, 4, 4)),
])
def test_random_substrates_bit_exact(rms, oracle, case):
    wl = _rand_case(**case)
    g, o, S_o, asum_o = run_both(rms, oracle, wl, spl=37)
    assert_walkers_equal(g, o)
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)


def test_slicing_and_sharding_do_not_change_trajectories(rms, oracle):
    wl = _rand_case(11, W=2000, n_steps=400)
    a = rms.simulate(wl, rms.RMS_FP64, hash_=True, steps_per_launch=400, walkers=True)
    b = rms.simulate(wl, rms.RMS_FP64, hash_=True, steps_per_launch=13, walkers=True)
    s1 = rms.simulate(wl, rms.RMS_FP64, n_walkers=700, hash_=True, walkers=True)
    s2 = rms.simulate(wl, rms.RMS_FP64, n_walkers=1300, walker_begin=700, hash_=True, walkers=True)
    for k in ("i", "o", "c", "A", "phase", "hash"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], np.concatenate([s1[k], s2[k]]))
    assert_moments_close(s1["moments"] + s2["moments"], a["moments"])
    np.testing.assert_array_equal(a["S"], b["S"])


def test_fp32_form_against_oracle(rms, oracle):
    """FP32 form on the cylinder case: signal and D(t), K(t) against the FP64 oracle."""
    import rms_inputs as ri
    wl = ri.workload("cylinder-32^3")
    g = rms.simulate(wl, rms.RMS_FP32)
    o = oracle.run(wl, n_threads=NT, hash_=False)
    S_o, _ = oracle.readout(o, wl)
    assert np.abs(g["S"] - S_o).max() <= 1e-3
    check_dk(g["moments"], o["moments"], wl)


def test_fp32_form_paired_with_plain_form_at_unequal_diffusivity(rms, oracle):
    """FP32 and FP64 forms draw the same random numbers, so at the workloads'
    permeabilities (P ~ 1e-3 per membrane event) their walkers stay paired:
    almost every walker ends in the same voxel, and the signals agree far
    inside 1e-3 -- including after crossings into labels of other D.  (Each
    FP32 position carries a rounding drift that grows like sqrt(steps); a
    membrane decision differs only when a face lies within that drift, so at
    large P the two forms decorrelate while staying statistically equal.)"""
    rng = np.random.default_rng(31)
    lab = rng.integers(0, 4, size=(12, 10, 11))
    D = np.array([2.0, 0.6, 1.3, 2.5])
    dt = 0.9 * (0.2 ** 2) / (6 * D.max())
    n = 3000
    G = np.zeros((2, n))
    G[0, :800], G[0, 1500:2300] = 1.0, -1.0
    G[1, 100:200], G[1, 2800:2900] = 1.0, -1.0
    wl = make_workload(lab, voxel_um=0.2, D=D, kappa=rng.uniform(0.01, 0.05, (4, 4)), T2=[40.0, 60.0, 80.0, 30.0],
                       dt=dt, n_steps=n, G=G, dirs=rng.normal(size=(6, 3)) / math.sqrt(3),
                       b=np.array([0.0, 0.5, 2.0]), rec_steps=np.array([1000, 2000, 3000]), n_walkers=20000, seed=8)
    g64 = rms.simulate(wl, rms.RMS_FP64, walkers=True)
    g32 = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    same = np.all(g64["i"] == g32["i"], axis=1).mean()
    assert same > 0.99, same
    assert np.abs(g32["S"] - g64["S"]).max() <= 1e-3
    o = oracle.run(wl, 0, 64, n_threads=NT)
    np.testing.assert_array_equal(g64["i"][:64], o["i"])


def dk(M, t):
    """D and K along x, y, z from the 22 moment sums (Sec. 2.3, narrow pulse)."""
    a = M[:, 0]
    m2 = np.stack([M[:, 1], M[:, 4], M[:, 6]], 1) / a[:, None]
    m4 = np.stack([M[:, 7], M[:, 17], M[:, 21]], 1) / a[:, None]
    return m2 / (2 * t[:, None]), m4 / m2 ** 2 - 3


def check_dk(Mg, Mo, wl):
    t = wl.rec_steps * wl.dt
    Dg, Kg = dk(Mg, t)
    Do, Ko = dk(Mo, t)
    assert np.all(np.abs(Dg - Do) <= 0.01 * Do), np.max(np.abs(Dg - Do) / Do)
    assert np.all(np.abs(Kg - Ko) <= 0.01 * np.maximum(np.abs(Ko), 0.1)), np.max(np.abs(Kg - Ko))


def test_errors_and_cancel(rms, oracle):
    from paper_2012_06478_gb300 import _lib
    wl = _rand_case(12, W=1000, n_steps=200)
    # step longer than a voxel
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D * 10, kappa=wl.kappa)
    with pytest.raises(rms.RmsError) as e:
        rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    assert e.value.status == _lib.RMS_E_STEP_TOO_LARGE
    sub.close()
    # P > 1 is clamped with a warning
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, kappa=wl.kappa * 1e6)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    assert seq.status == _lib.RMS_W_PROB_RANGE
    # a label outside the tables
    with pytest.raises(rms.RmsError):
        rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D[:2])
    # busy handles
    run = rms.rms_run(seq, 1000, 1)
    with pytest.raises(rms.RmsError) as e:
        seq.close()
    assert e.value.status == _lib.RMS_E_BUSY
    # cancel: the run reports it, the context stays usable
    rms.rms_cancel(run)
    with pytest.raises(rms.RmsError) as e:
        rms.rms_read_signal(run)
    assert e.value.status == _lib.RMS_E_CANCELLED
    run.close()
    seq.close()
    sub.close()
    g = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True)
    o = oracle.run(wl, n_threads=NT)
    assert_walkers_equal(g, o)


def test_labels_from_device_tensor(rms, oracle):
    import torch
    wl = _rand_case(13, W=500, n_steps=100)
    lab = torch.from_numpy(wl.labels.astype(np.int16)).cuda()
    sub = rms.rms_create_substrate(lab, wl.voxel_um, wl.D, T2=wl.T2, T1=wl.T1, kappa=wl.kappa,
                                   periodic=wl.periodic)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps, mode=wl.mode)
    run = rms.rms_run(seq, 500, wl.seed, flags=rms.RMS_TRAJ_HASH)
    g = rms.rms_read_walkers(run)
    o = oracle.run(wl, n_threads=NT)
    assert_walkers_equal(g, o)
    run.close()
    seq.close()
    sub.close()
