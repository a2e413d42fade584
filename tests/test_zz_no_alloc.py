"""The allocation-free signal read-out (rms_readout_noalloc) against the
read-out rms_run performs, through the C ABI.

rms_readout_noalloc exists for callers that may not allocate device memory
where they need the signal (a serving loop sharing the GPU with other
streams, where cudaMalloc/cudaFree could synchronise the device; an
application whose device memory all sits in its own fixed pool).  The caller
owns every input and output buffer -- here torch tensors -- and the library
uses only its fixed internal scratch.  Two calls in a row, on different
runs, must each match the regular path: to 1e-12 for a plain FP64 run, whose
read-out has the same FP64 terms, and, for an FP32-form run (whose read-out
evaluates each term in single precision), within the bound of that read-out
that tests/test_gpu_readout.py uses.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from conftest import make_workload
from test_gpu_readout import FP32_READOUT_TOL

pytestmark = pytest.mark.gpu


def _workload(seed, W):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 3, size=(6, 7, 8))
    n = 240
    G = np.zeros((2, n))
    G[0, :60], G[0, 120:180] = 1.0, -1.0
    G[1, 10:30], G[1, 200:220] = 1.0, -1.0
    return make_workload(lab, voxel_um=0.2, D=[2.0, 1.0, 1.5], kappa=rng.uniform(0, 2, size=(3, 3)),
                         T2=[50.0, 70.0, 90.0], dt=2e-3, n_steps=n, G=G,
                         dirs=rng.normal(size=(7, 3)) / np.sqrt(3), b=np.array([0.0, 0.5, 2.0, 5.0]),
                         rec_steps=np.array([n]), n_walkers=W, seed=seed)


def _noalloc(torch, lib, st, bs, wl):
    dev = torch.device("cuda")
    phase = torch.from_numpy(np.ascontiguousarray(st["phase"])).to(dev)
    A = torch.from_numpy(st["A"]).to(dev)
    b_s = torch.from_numpy(bs).to(dev)
    dirs = torch.from_numpy(np.ascontiguousarray(wl.dirs)).to(dev)
    b = torch.from_numpy(wl.b).to(dev)
    S, nd, nb = phase.shape[1], wl.dirs.shape[0], wl.b.size
    re = torch.zeros(S * nd * nb, dtype=torch.float64, device=dev)
    im = torch.zeros_like(re)
    asum = torch.zeros(1, dtype=torch.float64, device=dev)
    rc = lib.rms_readout_noalloc(phase.data_ptr(), A.data_ptr(), phase.shape[0], S, b_s.data_ptr(), nd,
                                 dirs.data_ptr(), nb, b.data_ptr(), re.data_ptr(), im.data_ptr(), asum.data_ptr(),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, (re.cpu().numpy() + 1j * im.cpu().numpy()).reshape(S, nd, nb), float(asum.item())


def test_noalloc_readout_matches_regular_readout_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_2012_06478_gb300 as rms
    from paper_2012_06478_gb300 import _lib
    cases = [(_workload(21, 9000), rms.RMS_FP64), (_workload(22, 5003), rms.RMS_FP32)]
    for wl, prec in cases:  # two calls in a row
        sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, T2=wl.T2, kappa=wl.kappa)
        seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
        run = rms.rms_run(seq, wl.n_walkers, wl.seed, prec)
        S_ref, _, asum_ref = rms.rms_read_signal(run)
        st = rms.rms_read_walkers(run)
        bs = rms.rms_sequence_bvalues(seq)
        rc, S, asum = _noalloc(torch, _lib.lib, st, bs, wl)
        assert rc == _lib.RMS_OK, _lib.last_error()
        if prec == rms.RMS_FP64:
            err = np.abs(S - S_ref) / np.maximum(np.abs(S_ref), 1e-3)
            assert err.max() <= 1e-12, err.max()
        else:
            assert np.abs(S - S_ref).max() <= FP32_READOUT_TOL, np.abs(S - S_ref).max()
        assert abs(asum - asum_ref) <= 1e-12 * asum_ref
        run.close()
        seq.close()
        sub.close()


def test_noalloc_at_its_chunk_cap_allocates_nothing():
    """Many combinations (1 shape x 500 directions x 100 b-values) over 3e5
    walkers: the scratch holds only 10 walker chunks where rms_run's read-out
    uses 74, so each chunk covers 30000 walkers.  The result still equals the
    regular read-out, on two calls in a row, and the second call leaves the
    device's free memory unchanged (the first may load the library's device
    code on this device, which takes the scratch array's memory)."""
    import torch
    import paper_2012_06478_gb300 as rms
    from paper_2012_06478_gb300 import _lib
    rng = np.random.default_rng(23)
    lab = rng.integers(0, 2, size=(8, 8, 8))
    n = 40
    G = np.zeros((1, n))
    G[0, :10], G[0, 20:30] = 1.0, -1.0
    wl = make_workload(lab, voxel_um=0.2, D=[2.0, 1.2], kappa=0.3, T2=[60.0, 45.0], dt=2e-3, n_steps=n, G=G,
                       dirs=rng.normal(size=(500, 3)) / np.sqrt(3), b=np.linspace(0.0, 40.0, 100),
                       rec_steps=np.array([n]), n_walkers=300_000, seed=23)
    n_combo = 500 * 100
    assert (8 * 1024 * 1024 // 8) // (2 * (n_combo + 1)) < -(-wl.n_walkers // 4096)   # the cap binds
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, T2=wl.T2, kappa=wl.kappa)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    run = rms.rms_run(seq, wl.n_walkers, wl.seed, rms.RMS_FP64)
    S_ref, _, asum_ref = rms.rms_read_signal(run)
    st = rms.rms_read_walkers(run)
    bs = rms.rms_sequence_bvalues(seq)
    for call in range(2):
        rc, S, asum = _noalloc(torch, _lib.lib, st, bs, wl)
        assert rc == _lib.RMS_OK, _lib.last_error()
        err = np.abs(S - S_ref) / np.maximum(np.abs(S_ref), 1e-3)
        assert err.max() <= 1e-12, (call, err.max())
        assert abs(asum - asum_ref) <= 1e-12 * asum_ref
    run.close()
    seq.close()
    sub.close()
    # the second call took no device memory: measured around a third call with
    # its inputs and outputs already in place
    phase = torch.from_numpy(np.ascontiguousarray(st["phase"])).cuda()
    A = torch.from_numpy(st["A"]).cuda()
    b_s, dirs, b = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (bs, wl.dirs, wl.b))
    re = torch.zeros(n_combo, dtype=torch.float64, device="cuda")
    im = torch.zeros_like(re)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    rc = _lib.lib.rms_readout_noalloc(phase.data_ptr(), A.data_ptr(), wl.n_walkers, 1, b_s.data_ptr(), 500,
                                      dirs.data_ptr(), 100, b.data_ptr(), re.data_ptr(), im.data_ptr(), None,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == _lib.RMS_OK
    assert torch.cuda.mem_get_info()[0] == before


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2012_06478_gb300 import _lib
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    # 8 shapes x 1000 directions x 100 b-values needs 2*(8e5+1) doubles > 8 MiB / 8
    rc = _lib.lib.rms_readout_noalloc(p, p, 1, 8, p, 1000, p, 100, p, p, p, p, None)
    assert rc == _lib.RMS_E_INVALID_ARG
    assert "scratch" in _lib.last_error()
