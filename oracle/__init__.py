"""CPU FP64 oracle for the RMS random-walker step -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it
and shares no code with it.  The arithmetic lives in ``rms_oracle.c`` (plain
C, FP64, no FMA contraction); this file only builds it with gcc and marshals
numpy arrays through ctypes.

Parity status per function (see the header of ``rms_oracle.c`` for the
passages each follows):
  philox4x32_10      pinned: Random123 known-answer vectors and cuRAND's host
                     Philox4x32-10 generator
  run / walk_once    pinned: free-walk closed forms, corner reflector,
                     hand-derived single steps, impermeable long-time limits,
                     short-time S/V law, uniform equilibrium at unequal D,
                     two-compartment exchange, finite-step permeability
  readout / bvalue   pinned: b = delta^2 (Delta - delta/3), S = 1 at b = 0,
                     exact free-walk signal prod_j sinc(q |F_j| ds)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rms_oracle.c")
# RMS_ORACLE_SANITIZE=1: a separate build under AddressSanitizer and
# UndefinedBehaviorSanitizer (the process must preload the ASan runtime)
_SANITIZE = os.environ.get("RMS_ORACLE_SANITIZE") == "1"
_LIB = os.path.join(_HERE, "librms_oracle_san.so" if _SANITIZE else "librms_oracle.so")
_lib = None

MOMENT_NAMES = (["1"] + [a + b for i, a in enumerate("xyz") for b in "xyz"[i:]] +
                ["".join(t) for t in
                 [(a, b, c, d) for ia, a in enumerate("xyz") for ib, b in enumerate("xyz") if ib >= ia
                  for ic, c in enumerate("xyz") if ic >= ib for d in "xyz"[ic:]]])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        san = (["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]
               if _SANITIZE else [])
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", *san,
                               "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("voxel_um", C.c_double), ("periodic", C.c_int32 * 3),
        ("labels", C.c_void_p), ("n_labels", C.c_int32),
        ("D", C.c_void_p), ("T2", C.c_void_p), ("T1", C.c_void_p), ("kappa", C.c_void_p),
        ("dead", C.c_void_p),
        ("dt", C.c_double), ("n_steps", C.c_int64), ("n_shapes", C.c_int32),
        ("G", C.c_void_p), ("mode", C.c_void_p), ("n_rec", C.c_int32), ("rec_steps", C.c_void_p),
        ("seed", C.c_uint64), ("w_begin", C.c_int64), ("w_end", C.c_int64),
        ("n_threads", C.c_int32), ("hash", C.c_int32), ("interaction", C.c_int32),
        ("rho", C.c_void_p), ("conc", C.c_void_p), ("lam", C.c_double), ("perm_model", C.c_int32),
    ]


class _Output(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("i", "o", "i0", "o0", "c", "A", "phase", "hash", "counts", "moments")]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.rmso_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.rmso_philox_many.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.rmso_run.argtypes = [C.POINTER(_Config), C.POINTER(_Output)]
        _lib.rmso_run.restype = C.c_int
        _lib.rmso_readout.argtypes = [C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int64, C.c_double, C.c_int32, C.c_void_p, C.c_int32,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.rmso_bvalue.argtypes = [C.c_void_p, C.c_int64, C.c_double]
        _lib.rmso_bvalue.restype = C.c_double
        _lib.rmso_perm_prob.argtypes = [C.c_double] * 5
        _lib.rmso_perm_prob.restype = C.c_double
        _lib.rmso_step_length.argtypes = [C.c_double, C.c_double]
        _lib.rmso_step_length.restype = C.c_double
        _lib.rmso_threshold.argtypes = [C.c_double]
        _lib.rmso_threshold.restype = C.c_uint32
        _lib.rmso_mix64.argtypes = [C.c_uint64]
        _lib.rmso_mix64.restype = C.c_uint64
        _lib.rmso_walk_once.argtypes = [C.POINTER(_Config), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        _lib.rmso_walk_once.restype = C.c_int
        _lib.rmso_thresholds.argtypes = [C.POINTER(_Config), C.c_void_p, C.c_void_p]
        _lib.rmso_thresholds.restype = C.c_int
        _lib.rmso_direction.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_void_p]
        _lib.rmso_direction.restype = C.c_int
        _lib.rmso_direction_from_words.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr (n, 4) uint32 under keys key (n, 2)."""
    ctr = np.ascontiguousarray(np.atleast_2d(ctr), dtype=np.uint32)
    key = np.ascontiguousarray(np.atleast_2d(key), dtype=np.uint32)
    if key.shape[0] == 1 and ctr.shape[0] > 1:
        key = np.ascontiguousarray(np.repeat(key, ctr.shape[0], axis=0))
    out = np.empty_like(ctr)
    lib().rmso_philox_many(ctr.shape[0], ctr.ctypes.data, key.ctypes.data, out.ctypes.data)
    return out


def step_length(D: float, dt: float) -> float:
    return lib().rmso_step_length(D, dt)


def perm_prob(kappa, D1, ds1, D2, ds2) -> float:
    return lib().rmso_perm_prob(kappa, D1, ds1, D2, ds2)


def threshold(P: float) -> int:
    return int(lib().rmso_threshold(P))


def mix64(z: int) -> int:
    return int(lib().rmso_mix64(z))


def direction(seed: int, w: int, k: int) -> np.ndarray:
    n = np.zeros(3)
    if lib().rmso_direction(seed, w, k, n.ctypes.data):
        raise RuntimeError("direction sampler ran out of draws")
    return n


def direction_from_words(x0: int, x1: int) -> np.ndarray:
    n = np.zeros(3)
    lib().rmso_direction_from_words(x0, x1, n.ctypes.data)
    return n


class _Keep:
    """Keeps the contiguous arrays a _Config points at alive."""

    def __init__(self):
        self.refs = []

    def __call__(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def _config(wl, keep: _Keep, w_begin=0, w_end=None, n_threads=None, hash_=True,
            n_steps=None) -> _Config:
    nx, ny, nz = wl.shape_xyz
    cfg = _Config()
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.voxel_um = wl.voxel_um
    cfg.periodic = (C.c_int32 * 3)(*[int(p) for p in wl.periodic])
    cfg.labels = keep(wl.labels, np.uint16).ctypes.data
    cfg.n_labels = wl.n_labels
    cfg.D = keep(wl.D, np.float64).ctypes.data
    cfg.T2 = keep(wl.T2, np.float64).ctypes.data
    cfg.T1 = keep(wl.T1, np.float64).ctypes.data
    cfg.kappa = keep(wl.kappa, np.float64).ctypes.data
    cfg.dead = keep(wl.dead, np.uint8).ctypes.data
    cfg.dt = wl.dt
    ns = wl.n_steps if n_steps is None else n_steps
    cfg.n_steps = ns
    G = np.asarray(wl.G, np.float64)
    G = keep(G.reshape(-1, wl.n_steps)[:, :ns] if wl.n_steps > 0 else G.reshape(1, 0), np.float64)
    cfg.n_shapes = G.shape[0]
    cfg.G = G.ctypes.data
    cfg.mode = None if wl.mode is None else keep(wl.mode[:ns], np.uint8).ctypes.data
    rec = keep(np.asarray(wl.rec_steps)[np.asarray(wl.rec_steps) <= ns], np.int64)
    cfg.n_rec = rec.size
    cfg.rec_steps = rec.ctypes.data if rec.size else None
    cfg.seed = wl.seed
    cfg.w_begin = w_begin
    cfg.w_end = wl.n_walkers if w_end is None else w_end
    cfg.n_threads = n_threads or os.cpu_count() or 1
    cfg.hash = 1 if hash_ else 0
    cfg.interaction = int(getattr(wl, "interaction", 0))
    rho = getattr(wl, "rho", None)
    cfg.rho = None if rho is None else keep(rho, np.float64).ctypes.data
    conc = getattr(wl, "conc", None)
    cfg.conc = None if conc is None else keep(conc, np.float64).ctypes.data
    cfg.lam = float(getattr(wl, "lam", -1.0))
    cfg.perm_model = int(getattr(wl, "perm_model", 0))
    return cfg


def run(wl, w_begin: int = 0, w_end: Optional[int] = None, n_threads: Optional[int] = None,
        hash_: bool = True, n_steps: Optional[int] = None) -> dict:
    """Run walkers [w_begin, w_end) of workload wl (first n_steps steps).

    Returns per-walker arrays i, o, i0, o0 (W, 3), c, A (W,), phase (W, S, 3),
    hash (W,), counts (W, 3) = (face events, crossings, reflections), and
    moments (n_rec, 22) summed over these walkers."""
    keep = _Keep()
    cfg = _config(wl, keep, w_begin, w_end, n_threads, hash_, n_steps)
    W = cfg.w_end - cfg.w_begin
    S = cfg.n_shapes
    res = dict(i=np.zeros((W, 3), np.int32), o=np.zeros((W, 3)), i0=np.zeros((W, 3), np.int32),
               o0=np.zeros((W, 3)), c=np.zeros(W, np.int32), A=np.zeros(W),
               phase=np.zeros((W, S, 3)), hash=np.zeros(W, np.uint64), counts=np.zeros((W, 3), np.int64),
               moments=np.zeros((cfg.n_rec, 22)))
    out = _Output(*[_p(res[k]) for k in ("i", "o", "i0", "o0", "c", "A", "phase", "hash", "counts",
                                          "moments")])
    err = lib().rmso_run(C.byref(cfg), C.byref(out))
    res["err"] = int(err)
    res["rec_steps"] = np.asarray(wl.rec_steps)[np.asarray(wl.rec_steps) <= cfg.n_steps]
    return res


def bvalue(G: np.ndarray, dt: float) -> float:
    G = np.ascontiguousarray(G, np.float64)
    return lib().rmso_bvalue(G.ctypes.data, G.size, dt)


def readout(res: dict, wl, n_steps: Optional[int] = None):
    """Signal S (n_shapes, n_dirs, n_b) complex and sum of alpha."""
    ns = wl.n_steps if n_steps is None else n_steps
    G = np.asarray(wl.G, np.float64)
    G = np.ascontiguousarray(G.reshape(-1, wl.n_steps)[:, :ns] if wl.n_steps > 0 else G.reshape(1, 0))
    phase = np.ascontiguousarray(res["phase"], np.float64)
    A = np.ascontiguousarray(res["A"], np.float64)
    dirs = np.ascontiguousarray(wl.dirs, np.float64)
    b = np.ascontiguousarray(wl.b, np.float64)
    S, nd, nb = G.shape[0], dirs.shape[0], b.size
    re = np.zeros((S, nd, nb))
    im = np.zeros((S, nd, nb))
    asum = np.zeros(1)
    lib().rmso_readout(A.size, S, phase.ctypes.data, A.ctypes.data, G.ctypes.data, ns, wl.dt, nd,
                       dirs.ctypes.data, nb, b.ctypes.data, re.ctypes.data, im.ctypes.data,
                       asum.ctypes.data)
    return re + 1j * im, float(asum[0])


def thresholds(wl):
    keep = _Keep()
    cfg = _config(wl, keep, 0, 0)
    L = wl.n_labels
    T = np.zeros((L, L), np.uint32)
    s = np.zeros(L)
    err = lib().rmso_thresholds(C.byref(cfg), T.ctypes.data, s.ctypes.data)
    if err:
        raise RuntimeError(f"oracle error {err}")
    return T, s


def walk_once(wl, i, o, c, n, perm=(0, 0, 0), A=0.0, mode=0):
    """One face walk of a single walker with a given direction n and given
    PERM words (no random draws).  Returns (i, o, c, A, n, counts, err)."""
    keep = _Keep()
    cfg = _config(wl, keep, 0, 0)
    ii = np.array(i, np.int64)
    oo = np.array(o, np.float64)
    cc = np.array([c], np.int32)
    AA = np.array([A], np.float64)
    nn = np.array(n, np.float64)
    pp = np.zeros(4, np.uint32)
    pp[:len(perm)] = perm
    counts = np.zeros(3, np.int64)
    err = lib().rmso_walk_once(C.byref(cfg), ii.ctypes.data, oo.ctypes.data, cc.ctypes.data,
                               AA.ctypes.data, nn.ctypes.data, pp.ctypes.data, mode, counts.ctypes.data)
    return ii, oo, int(cc[0]), float(AA[0]), nn, counts, int(err)


def displacement(res: dict, voxel_um: float) -> np.ndarray:
    """Final displacement (um) per walker, the same expression the oracle uses."""
    return voxel_um * ((res["i"] - res["i0"]).astype(np.float64) + (res["o"] - res["o0"]))
