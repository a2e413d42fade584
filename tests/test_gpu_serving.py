"""Continuous-batching serving loop: requests of different substrates,
sizes, sequences and precisions run together in the batched kernels, are
admitted as memory frees up, and each result equals the one rms_run gives
for the same request alone (FP64: bit for bit; FP32: to 1e-6)."""
import math

import numpy as np
import pytest

from conftest import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available()
    import paper_2012_06478_gb300 as rms
    return rms


def _cases():
    import rms_inputs as ri
    rng = np.random.default_rng(5)
    out = []
    cyl = ri.workload("cylinder-32^3").with_(n_steps=600, G=ri.pgse(0.2, 0.4, 1e-3, 600)[None, :],
                                             rec_steps=np.arange(100, 601, 100))
    out.append((cyl, 3000, 1))
    lab = rng.integers(0, 4, size=(9, 10, 11))
    G = rng.normal(size=(3, 400)) * (rng.uniform(size=(3, 400)) < 0.3)
    rnd = make_workload(lab, voxel_um=0.2, D=[2.0, 1.0, 1.5, 0.7], kappa=rng.uniform(0, 2, (4, 4)),
                        T2=[40.0, 60.0, 80.0, 100.0], dt=6e-4, n_steps=400, G=G, dirs=ri.fibonacci_dirs(7),
                        b=np.array([0.0, 1.0, 3.0]), rec_steps=np.array([50, 400]), n_walkers=5000, seed=9)
    out.append((rnd, 5000, 9))
    ax = ri.axon_labels(40, 40, 32, 0.1, 6, seed=3)
    L = int(ax.max()) + 1
    axw = make_workload(ax, voxel_um=0.1, D=2.0, kappa=0.05, dt=2e-4, n_steps=700,
                        G=ri.pgse(0.04, 0.08, 2e-4, 700)[None, :], dirs=ri.fibonacci_dirs(12),
                        b=np.array([0.0, 2.0]), rec_steps=np.array([700]), n_walkers=20000, seed=4)
    assert axw.n_labels == L
    out.append((axw, 20000, 4))
    return out


def _open(rms, wl):
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, T2=wl.T2, T1=wl.T1, kappa=wl.kappa,
                                   periodic=wl.periodic)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps, mode=wl.mode)
    return sub, seq


@pytest.mark.parametrize("policy", [0, 1])
def test_requests_alone_and_in_the_mix(rms, policy):
    cases = _cases()
    handles = [_open(rms, wl) for wl, _, _ in cases]
    jobs = []
    for (wl, W, seed), (sub, seq) in zip(cases, handles):
        for prec in (rms.RMS_FP64, rms.RMS_FP32):
            run = rms.rms_run(seq, W, seed, prec)
            jobs.append((seq, W, seed, prec, rms.rms_read_signal(run)))
            run.close()
    # a budget that holds only part of the requests at once: the rest queue
    srv = rms.Server(memory_budget_bytes=12 << 20, max_active=4, steps_per_tick=64, policy=policy)
    tickets = [srv.submit(seq, W, seed, prec) for seq, W, seed, prec, _ in jobs]
    tickets += [srv.submit(seq, W, seed, prec) for seq, W, seed, prec, _ in jobs]  # the same again
    results = [srv.wait(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    srv.close()
    for k, (S, M, a) in enumerate(results):
        seq, W, seed, prec, (S0, M0, a0) = jobs[k % len(jobs)]
        if prec == rms.RMS_FP64:
            np.testing.assert_array_equal(S, S0)
            np.testing.assert_array_equal(M, M0)
            assert a == a0
        else:
            np.testing.assert_allclose(S, S0, rtol=0, atol=1e-6)
            np.testing.assert_allclose(M, M0, rtol=1e-6)
    assert st["completed"] == len(tickets)
    assert st["peak_in_flight"] >= 2            # requests overlapped on the device
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["graph_updates"] + st["graph_instantiations"] == st["ticks"]
    for sub, seq in handles:
        seq.close()
        sub.close()


def test_size_aware_policy_lets_small_requests_fill_the_tick(rms):
    """RMS_SERVE_FILL: next to a request whose blocks span several waves of
    the GPU, a small request advances several waves' worth of steps per tick
    (fewer ticks than steps / steps_per_tick), with the same result as alone;
    under RMS_SERVE_STEPS it takes one tick per steps_per_tick steps."""
    import rms_inputs as ri
    n = 4096
    big = ri.workload("cylinder-32^3").with_(n_steps=n, G=ri.pgse(0.5, 1.0, 1e-3, n)[None, :],
                                             rec_steps=np.array([n]))
    sub, seq = _open(rms, big)
    W_big, W_small = 1_200_000, 2000   # > 6 waves of 128-walker blocks on 152 SMs x 8 slots; one block row
    ref = rms.rms_run(seq, W_small, 77, rms.RMS_FP32)
    S0, M0, a0 = rms.rms_read_signal(ref)
    ref.close()
    ticks = {}
    for policy in (rms.RMS_SERVE_STEPS, rms.RMS_SERVE_FILL):
        srv = rms.Server(max_active=4, steps_per_tick=128, policy=policy)
        tb = srv.submit(seq, W_big, 5, rms.RMS_FP32)
        ts = srv.submit(seq, W_small, 77, rms.RMS_FP32)
        while not srv.poll(ts):
            pass
        ticks[policy] = srv.request_info(ts)["ticks"]
        S, M, a = srv.wait(ts)
        np.testing.assert_allclose(S, S0, rtol=0, atol=1e-6)
        np.testing.assert_allclose(M, M0, rtol=1e-6)
        srv.wait(tb)
        srv.close()
    assert ticks[rms.RMS_SERVE_STEPS] == n // 128
    assert ticks[rms.RMS_SERVE_FILL] <= n // 128 // 2, ticks
    seq.close()
    sub.close()


def test_cancel_and_busy(rms):
    wl, W, seed = _cases()[0]
    sub, seq = _open(rms, wl)
    srv = rms.Server(max_active=1, steps_per_tick=16)
    t1 = srv.submit(seq, W, seed)
    t2 = srv.submit(seq, W, seed)
    t3 = srv.submit(seq, W, seed)
    srv.cancel(t3)
    with pytest.raises(rms.RmsError) as e:
        seq.close()                              # still referenced by queued requests
    assert e.value.status == -8
    S1, _, _ = srv.wait(t1)
    S2, _, _ = srv.wait(t2)
    np.testing.assert_array_equal(S1, S2)
    with pytest.raises(rms.RmsError) as e:
        srv.wait(t3)
    assert e.value.status == -7
    srv.close()
    seq.close()
    sub.close()


def test_destroy_with_work_in_flight(rms):
    wl, W, seed = _cases()[2]
    sub, seq = _open(rms, wl)
    srv = rms.Server(max_active=2, steps_per_tick=8)
    for _ in range(5):
        srv.submit(seq, W, seed, rms.RMS_FP32)
    srv.close()                                  # cancels what is queued or running
    seq.close()
    sub.close()
    # the device is still usable
    r = rms.simulate(wl.with_(n_steps=10, G=wl.G[:, :10], rec_steps=np.array([10])), rms.RMS_FP64,
                     n_walkers=100)
    assert math.isfinite(r["alpha_sum"])
