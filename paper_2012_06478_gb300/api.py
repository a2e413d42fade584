"""Python face of the C ABI, with the same names (argument marshalling only).

    sub = rms_create_substrate(labels, voxel_um, D, T2=..., kappa=..., stream=...)
    seq = rms_set_sequence(sub, dt_ms, G, dirs, b, rec_steps)
    run = rms_run(seq, n_walkers, seed, precision=RMS_FP64)
    S, moments, alpha_sum = rms_read_signal(run)

Inputs may be numpy arrays (host) or, for the label volume, a CUDA tensor
(device); torch supplies device memory and the stream, nothing else.  The
handles free their device memory when closed or garbage collected.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence as Seq

import numpy as np

from . import _lib as L
from ._lib import (RMS_CHECKED, RMS_COUNTS, RMS_EC, RMS_MORTON, RMS_ERL, RMS_FP32, RMS_FP64, RMS_PEAK_FP64_ADD, RMS_PEAK_FP64_FMA,
                   RMS_PEAK_FP64_MUL, RMS_PEAK_GATHER, RMS_PEAK_GATHER_DEP, RMS_RS, RMS_SERVE_FILL, RMS_SERVE_STEPS,
                   RMS_TRAJ_HASH, RmsError, check)

__all__ = ["rms_create_substrate", "rms_set_sequence", "rms_run", "rms_read_signal", "rms_read_walkers",
           "rms_read_counts", "rms_read_slots", "rms_cancel", "rms_run_query", "rms_destroy_run", "rms_destroy_sequence",
           "rms_destroy_substrate", "rms_sequence_bvalues", "rms_run_step_time_ms", "simulate", "current_stream",
           "RMS_FP32", "RMS_FP64", "RMS_TRAJ_HASH", "RMS_CHECKED", "RMS_COUNTS", "RMS_MORTON", "RMS_EC", "RMS_RS", "RMS_ERL",
           "RmsError", "MOMENT_NAMES", "Server", "rms_measure_peak", "rms_device_sm_count", "rms_read_partials",
           "rms_normalise_partials", "rms_philox4x32_10", "RMS_PEAK_FP64_ADD", "RMS_PEAK_FP64_MUL", "RMS_PEAK_FP64_FMA",
           "RMS_PEAK_GATHER", "RMS_PEAK_GATHER_DEP", "RMS_SERVE_STEPS", "RMS_SERVE_FILL"]

MOMENT_NAMES = ["1", "xx", "xy", "xz", "yy", "yz", "zz", "xxxx", "xxxy", "xxxz", "xxyy", "xxyz", "xxzz", "xyyy",
                "xyyz", "xyzz", "xzzz", "yyyy", "yyyz", "yyzz", "yzzz", "zzzz"]


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 if torch has no CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Substrate:
    def __init__(self, handle, shape_xyz, n_labels, keep=None):
        self.handle = handle
        self.shape_xyz = shape_xyz
        self.n_labels = n_labels
        self._keep = keep

    def close(self):
        if self.handle:
            check(L.lib.rms_destroy_substrate(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sequence:
    def __init__(self, handle, sub, n_steps, n_shapes, n_dirs, n_b, n_rec, status):
        self.handle = handle
        self.sub = sub
        self.n_steps, self.n_shapes, self.n_dirs, self.n_b, self.n_rec = n_steps, n_shapes, n_dirs, n_b, n_rec
        self.status = status

    def close(self):
        if self.handle:
            check(L.lib.rms_destroy_sequence(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Run:
    def __init__(self, handle, seq, n_walkers, precision, flags, interaction=RMS_EC):
        self.handle = handle
        self.seq = seq
        self.n_walkers = n_walkers
        self.precision = precision
        self.flags = flags
        self.interaction = interaction
        self.status = L.RMS_OK  # RMS_W_LEAP_LIMIT once a read reports it

    def close(self):
        if self.handle:
            check(L.lib.rms_destroy_run(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rms_create_substrate(labels, voxel_um: float, D, T2=None, T1=None, kappa=None, kappa_scalar: float = 0.0,
                         dead=None, periodic=(1, 1, 1), n_labels: Optional[int] = None,
                         stream: Optional[int] = None, rho=None, conc=None, lam: float = -1.0,
                         perm_model: int = 0) -> Substrate:
    """labels: (nz, ny, nx) uint16 numpy array or CUDA tensor (x fastest).
    rho: optional (L, L) surface relaxivity (um/ms) of absorbing membranes.
    conc, lam, perm_model: spin concentration per label, the exponent lambda
    (< 0: the optimal one) and the permeation model (0 nominal kappa,
    1 Baxter)."""
    on_device = hasattr(labels, "is_cuda") and labels.is_cuda
    if on_device:
        import torch
        assert labels.dtype in (torch.uint16, torch.int16) and labels.is_contiguous()
        nz, ny, nx = labels.shape
        lab_ptr = labels.data_ptr()
        keep_lab = labels
    else:
        lab = np.ascontiguousarray(labels, dtype=np.uint16)
        nz, ny, nx = lab.shape
        lab_ptr = lab.ctypes.data
        keep_lab = lab
    Dv = _host(D, np.float64)
    Lc = int(n_labels if n_labels is not None else Dv.size)
    T2v, T1v = _host(T2, np.float64), _host(T1, np.float64)
    Kv = _host(kappa, np.float64)
    Rv = _host(rho, np.float64)
    Cv = _host(conc, np.float64)
    deadv = _host(dead, np.uint8)
    d = L.SubstrateDesc()
    d.labels = lab_ptr
    d.labels_on_device = 1 if on_device else 0
    d.nx, d.ny, d.nz = nx, ny, nz
    d.voxel_um = float(voxel_um)
    d.periodic = (C.c_int32 * 3)(*[int(p) for p in periodic])
    d.n_labels = Lc
    d.D, d.T2, d.T1, d.kappa = _ptr(Dv), _ptr(T2v), _ptr(T1v), _ptr(Kv)
    d.kappa_scalar = float(kappa_scalar)
    d.rho = _ptr(Rv)
    d.conc = _ptr(Cv)
    d.lam = float(lam)
    d.perm_model = int(perm_model)
    d.dead = _ptr(deadv)
    d.stream = current_stream() if stream is None else stream
    h = C.c_void_p()
    check(L.lib.rms_create_substrate(C.byref(d), C.byref(h)))
    return Substrate(h, (nx, ny, nz), Lc, keep=None if not on_device else keep_lab)


def rms_set_sequence(sub: Substrate, dt_ms: float, G, dirs, b, rec_steps: Seq[int] = (), mode=None) -> Sequence:
    Gv = np.ascontiguousarray(np.atleast_2d(np.asarray(G, np.float64)))
    S, N = Gv.shape
    dv = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
    bv = np.ascontiguousarray(np.asarray(b, np.float64).ravel())
    rv = np.ascontiguousarray(np.asarray(rec_steps, np.int64).ravel())
    mv = _host(mode, np.uint8)
    d = L.SequenceDesc()
    d.dt_ms = float(dt_ms)
    d.n_steps = N
    d.n_shapes = S
    d.G = Gv.ctypes.data if N else None
    d.mode = _ptr(mv)
    d.n_dirs = dv.shape[0]
    d.dirs = dv.ctypes.data
    d.n_b = bv.size
    d.b = bv.ctypes.data
    d.n_rec = rv.size
    d.rec_steps = rv.ctypes.data if rv.size else None
    h = C.c_void_p()
    st = check(L.lib.rms_set_sequence(sub.handle, C.byref(d), C.byref(h)), allow=(L.RMS_OK, L.RMS_W_PROB_RANGE))
    return Sequence(h, sub, N, S, dv.shape[0], bv.size, rv.size, st)


def rms_sequence_bvalues(seq: Sequence) -> np.ndarray:
    out = np.zeros(seq.n_shapes)
    check(L.lib.rms_sequence_bvalues(seq.handle, out.ctypes.data))
    return out


def rms_run(seq: Sequence, n_walkers: int, seed: int, precision: int = RMS_FP64, flags: int = 0,
            walker_begin: int = 0, steps_per_launch: int = 0, stream: Optional[int] = None,
            interaction: int = RMS_EC, resume: Optional[dict] = None, step_end: int = 0) -> Run:
    """rms_run, or rms_run_range when `resume` (a state: `step` plus the arrays
    rms_read_walkers returns and optionally `moments`) or `step_end` is given."""
    d = L.RunDesc()
    d.n_walkers = int(n_walkers)
    d.walker_begin = int(walker_begin)
    d.seed = int(seed)
    d.precision = int(precision)
    d.flags = int(flags)
    d.steps_per_launch = int(steps_per_launch)
    d.interaction = int(interaction)
    d.stream = current_stream() if stream is None else stream
    h = C.c_void_p()
    if resume is None and not step_end:
        check(L.lib.rms_run(seq.handle, C.byref(d), C.byref(h)))
    else:
        keep = []
        st = None
        if resume is not None:
            st = L.RunState()
            st.step = int(resume["step"])
            for name, dt in (("i", np.int32), ("o", np.float64), ("i0", np.int32), ("o0", np.float64),
                             ("c", np.int32), ("A", np.float64), ("phase", np.float64), ("hash", np.uint64),
                             ("moments", np.float64)):
                a = resume.get(name)
                if a is not None:
                    a = np.ascontiguousarray(a, dtype=dt)
                    keep.append(a)
                    setattr(st, name, a.ctypes.data)
        check(L.lib.rms_run_range(seq.handle, C.byref(d), C.byref(st) if st is not None else None, int(step_end),
                                  C.byref(h)))
    return Run(h, seq, int(n_walkers), precision, flags, int(interaction))


def rms_run_query(run: Run) -> bool:
    """True when finished."""
    return check(L.lib.rms_run_query(run.handle), allow=(L.RMS_OK, L.RMS_E_NOT_READY)) == L.RMS_OK


def rms_cancel(run: Run) -> None:
    check(L.lib.rms_cancel(run.handle))


def rms_read_signal(run: Run):
    """(S complex (n_shapes, n_dirs, n_b), moments (n_rec, 22), alpha_sum)."""
    q = run.seq
    n = q.n_shapes * q.n_dirs * q.n_b
    re, im = np.zeros(n), np.zeros(n)
    mom = np.zeros((q.n_rec, 22))
    asum = np.zeros(1)
    run.status = check(L.lib.rms_read_signal(run.handle, re.ctypes.data, im.ctypes.data,
                                             mom.ctypes.data if q.n_rec else None, asum.ctypes.data),
                       allow=(L.RMS_OK, L.RMS_W_LEAP_LIMIT))
    return (re + 1j * im).reshape(q.n_shapes, q.n_dirs, q.n_b), mom, float(asum[0])


def rms_read_partials(run: Run):
    """Unnormalised reductions for combining walker shards: (sum of alpha
    e^{-i phi} complex (n_shapes, n_dirs, n_b), moments (n_rec, 22), sum alpha)."""
    q = run.seq
    n = q.n_shapes * q.n_dirs * q.n_b
    re, im = np.zeros(n), np.zeros(n)
    mom = np.zeros((q.n_rec, 22))
    asum = np.zeros(1)
    run.status = check(L.lib.rms_read_partials(run.handle, re.ctypes.data, im.ctypes.data, asum.ctypes.data,
                                               mom.ctypes.data if q.n_rec else None),
                       allow=(L.RMS_OK, L.RMS_W_LEAP_LIMIT))
    return (re + 1j * im).reshape(q.n_shapes, q.n_dirs, q.n_b), mom, float(asum[0])


def rms_normalise_partials(num, alpha_sum: float) -> np.ndarray:
    """S = num / sum alpha (Eq. 7), computed by the library."""
    num = np.asarray(num, np.complex128)
    re = np.ascontiguousarray(num.real.ravel())
    im = np.ascontiguousarray(num.imag.ravel())
    sr, si = np.zeros(re.size), np.zeros(re.size)
    check(L.lib.rms_normalise_partials(re.size, re.ctypes.data, im.ctypes.data, float(alpha_sum), sr.ctypes.data,
                                       si.ctypes.data))
    return (sr + 1j * si).reshape(num.shape)


def rms_philox4x32_10(ctr, key, stream: Optional[int] = None):
    """The library's Philox4x32-10 on CUDA tensors ctr (n, 4) and key (n, 2)
    of dtype int32/uint32; returns an (n, 4) tensor of words (same dtype)."""
    import torch
    assert ctr.is_cuda and key.is_cuda and ctr.is_contiguous() and key.is_contiguous()
    n = ctr.shape[0]
    assert ctr.shape == (n, 4) and key.shape == (n, 2) and ctr.element_size() == 4 and key.element_size() == 4
    out = torch.empty_like(ctr)
    check(L.lib.rms_philox4x32_10(ctr.data_ptr(), key.data_ptr(), n, out.data_ptr(),
                                  current_stream() if stream is None else stream))
    return out


def rms_read_walkers(run: Run) -> dict:
    W, S = run.n_walkers, run.seq.n_shapes
    out = dict(i=np.zeros((W, 3), np.int32), o=np.zeros((W, 3)), i0=np.zeros((W, 3), np.int32),
               o0=np.zeros((W, 3)), c=np.zeros(W, np.int32), A=np.zeros(W), phase=np.zeros((W, S, 3)),
               hash=np.zeros(W, np.uint64))
    run.status = check(L.lib.rms_read_walkers(run.handle, *[out[k].ctypes.data for k in
                                                            ("i", "o", "i0", "o0", "c", "A", "phase", "hash")]),
                       allow=(L.RMS_OK, L.RMS_W_LEAP_LIMIT))
    return out


def rms_read_counts(run: Run) -> np.ndarray:
    """(W, 3) int64: face events, crossings into another label, reflections
    (or RS/ERL stays) per walker; the run needs RMS_COUNTS."""
    out = np.zeros((run.n_walkers, 3), np.int64)
    run.status = check(L.lib.rms_read_counts(run.handle, out.ctypes.data), allow=(L.RMS_OK, L.RMS_W_LEAP_LIMIT))
    return out


def rms_read_slots(run: Run) -> np.ndarray:
    """W int32: the walker (relative to walker_begin) in each slot of the
    run's device state (identity unless RMS_MORTON)."""
    out = np.zeros(run.n_walkers, np.int32)
    run.status = check(L.lib.rms_read_slots(run.handle, out.ctypes.data), allow=(L.RMS_OK, L.RMS_W_LEAP_LIMIT))
    return out


def rms_run_step_time_ms(run: Run) -> float:
    ms = C.c_float()
    check(L.lib.rms_run_step_time_ms(run.handle, C.byref(ms)))
    return float(ms.value)


def rms_destroy_run(run: Run) -> None:
    run.close()


def rms_destroy_sequence(seq: Sequence) -> None:
    seq.close()


def rms_destroy_substrate(sub: Substrate) -> None:
    sub.close()


def simulate(wl, precision: int = RMS_FP64, n_walkers: Optional[int] = None, seed: Optional[int] = None,
             hash_: bool = False, walker_begin: int = 0, steps_per_launch: int = 0, walkers: bool = False,
             stream: Optional[int] = None, interaction: Optional[int] = None, checked: bool = False,
             resume: Optional[dict] = None, step_end: int = 0, counts: bool = False, morton: bool = False) -> dict:
    """Run one workload (an rms_inputs.Workload) end to end through the C ABI.
    The interaction defaults to the workload's (elastic collision if unset);
    `leap_limit` in the result is True when an ERL step used up its draws.
    `resume` / `step_end` run part of the sequence (rms_run_range): a result
    with walkers=True and its `moments` is a state to resume from, given the
    number of steps it took as `step`.  `morton` re-buckets the walkers in
    Morton order of their voxel before every step launch (RMS_MORTON)."""
    sub = rms_create_substrate(wl.labels, wl.voxel_um, wl.D, T2=wl.T2, T1=wl.T1, kappa=wl.kappa, dead=wl.dead,
                               periodic=wl.periodic, stream=stream, rho=getattr(wl, "rho", None),
                               conc=getattr(wl, "conc", None), lam=getattr(wl, "lam", -1.0),
                               perm_model=getattr(wl, "perm_model", 0))
    G = np.asarray(wl.G, np.float64)
    G = G.reshape(-1, wl.n_steps) if wl.n_steps else np.zeros((G.shape[0] if G.ndim == 2 else 1, 0))
    seq = rms_set_sequence(sub, wl.dt, G, wl.dirs, wl.b, wl.rec_steps, mode=wl.mode)
    run = rms_run(seq, wl.n_walkers if n_walkers is None else n_walkers, wl.seed if seed is None else seed,
                  precision,
                  (RMS_TRAJ_HASH if hash_ else 0) | (RMS_CHECKED if checked else 0) | (RMS_COUNTS if counts else 0)
                  | (RMS_MORTON if morton else 0),
                  walker_begin,
                  steps_per_launch, stream,
                  int(getattr(wl, "interaction", RMS_EC)) if interaction is None else int(interaction),
                  resume=resume, step_end=step_end)
    S, mom, asum = rms_read_signal(run)
    num, _, _ = rms_read_partials(run)
    res = dict(S=S, num=num, moments=mom, alpha_sum=asum, status=seq.status, step_ms=rms_run_step_time_ms(run),
               b_s=rms_sequence_bvalues(seq), leap_limit=run.status == L.RMS_W_LEAP_LIMIT)
    if walkers:
        res.update(rms_read_walkers(run))
    if counts:
        res["counts"] = rms_read_counts(run)
    if morton:
        res["slots"] = rms_read_slots(run)
    run.close()
    seq.close()
    sub.close()
    return res


def rms_measure_peak(kind: int, volume_elems: int = 0, target_ms: float = 20.0, reps: int = 3,
                     stream: Optional[int] = None):
    """(rate per second, ms of the best launch) of one machine peak
    (include/rms_peaks.h: RMS_PEAK_FP64_ADD/MUL/FMA, RMS_PEAK_GATHER[_DEP])."""
    rate, ms = C.c_double(), C.c_double()
    check(L.lib.rms_measure_peak(int(kind), int(volume_elems), float(target_ms), int(reps),
                                 current_stream() if stream is None else stream, C.byref(rate), C.byref(ms)))
    return float(rate.value), float(ms.value)


def rms_device_sm_count() -> int:
    n = C.c_int32()
    check(L.lib.rms_device_sm_count(C.byref(n)))
    return int(n.value)


class Server:
    """The continuous-batching serving loop (rms_server_* in include/rms.h)."""

    STATS = ("p50_ms", "p99_ms", "mean_ms", "walker_steps_per_s", "completed", "in_flight", "queued",
             "peak_in_flight", "ticks", "graph_updates", "graph_instantiations")

    def __init__(self, memory_budget_bytes: int = 0, max_active: int = 0, steps_per_tick: int = 0,
                 policy: int = L.RMS_SERVE_STEPS):
        cfg = L.ServerConfig(int(memory_budget_bytes), int(max_active), int(steps_per_tick), int(policy))
        h = C.c_void_p()
        check(L.lib.rms_server_create(C.byref(cfg), C.byref(h)))
        self.handle = h
        self._shapes = {}

    def submit(self, seq: Sequence, n_walkers: int, seed: int, precision: int = RMS_FP64) -> int:
        t = C.c_int64()
        check(L.lib.rms_server_submit(self.handle, seq.handle, int(n_walkers), int(seed), int(precision),
                                      C.byref(t)))
        self._shapes[t.value] = seq
        return t.value

    def poll(self, ticket: int) -> bool:
        return check(L.lib.rms_server_poll(self.handle, ticket), allow=(L.RMS_OK, L.RMS_E_NOT_READY)) == L.RMS_OK

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(S complex (n_shapes, n_dirs, n_b), moments (n_rec, 22), alpha_sum)."""
        q = self._shapes[ticket]
        n = q.n_shapes * q.n_dirs * q.n_b
        re, im = np.zeros(n), np.zeros(n)
        mom = np.zeros((q.n_rec, 22))
        asum = np.zeros(1)
        check(L.lib.rms_server_wait(self.handle, ticket, int(timeout_ms), re.ctypes.data, im.ctypes.data,
                                    mom.ctypes.data if q.n_rec else None, asum.ctypes.data))
        del self._shapes[ticket]
        return (re + 1j * im).reshape(q.n_shapes, q.n_dirs, q.n_b), mom, float(asum[0])

    def request_info(self, ticket: int) -> dict:
        """Timing of a finished request (before wait() releases it)."""
        out = np.zeros(4)
        check(L.lib.rms_server_request_info(self.handle, ticket, out.ctypes.data))
        return dict(queue_ms=out[0], latency_ms=out[1], walker_steps=out[2], ticks=int(out[3]))

    def cancel(self, ticket: int) -> None:
        check(L.lib.rms_server_cancel(self.handle, ticket))

    def stats(self) -> dict:
        out = np.zeros(11)
        check(L.lib.rms_server_stats(self.handle, out.ctypes.data))
        return dict(zip(self.STATS, out.tolist()))

    def close(self):
        if self.handle:
            check(L.lib.rms_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
