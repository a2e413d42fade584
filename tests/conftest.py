import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long statistical test")


def make_workload(labels, voxel_um=0.2, D=2.0, kappa=0.0, T2=math.inf, T1=math.inf, dt=1e-3,
                  n_steps=100, G=None, dirs=None, b=None, rec_steps=None, n_walkers=1000, seed=1,
                  periodic=(1, 1, 1), dead=None, mode=None, name="test", interaction=0, rho=None, conc=None,
                  lam=-1.0, perm_model=0):
    """A Workload from per-label scalars or arrays (tests only)."""
    import rms_inputs as ri
    labels = np.ascontiguousarray(labels, dtype=np.uint16)
    L = int(labels.max()) + 1

    def per_label(v):
        v = np.asarray(v, dtype=np.float64)
        return np.full(L, float(v)) if v.ndim == 0 else v.astype(np.float64)

    Dv, T2v, T1v = per_label(D), per_label(T2), per_label(T1)
    K = np.asarray(kappa, dtype=np.float64)
    if K.ndim == 0:
        K = np.full((L, L), float(K))
    K = K.copy()
    np.fill_diagonal(K, 0.0)
    if G is None:
        G = np.zeros((1, n_steps))
    G = np.asarray(G, dtype=np.float64)
    G = G.reshape(-1, n_steps) if n_steps > 0 else G.reshape(1, 0)
    if dirs is None:
        dirs = np.eye(3)
    if b is None:
        b = np.array([0.0])
    if rec_steps is None:
        rec_steps = np.array([n_steps], dtype=np.int64)
    dead = np.zeros(L, np.uint8) if dead is None else np.asarray(dead, np.uint8)
    return ri.Workload(name, labels, float(voxel_um), tuple(int(p) for p in periodic), Dv, T2v, T1v, K,
                       dead, float(dt), int(n_steps), G, mode, np.asarray(dirs, np.float64),
                       np.asarray(b, np.float64), np.asarray(rec_steps, np.int64), int(n_walkers), int(seed),
                       int(interaction), _pair_table(rho, L),
                       None if conc is None else np.asarray(conc, np.float64), float(lam), int(perm_model))


def _pair_table(v, L):
    """None, or an (L, L) table from a scalar or an array (diagonal zeroed)."""
    if v is None:
        return None
    R = np.asarray(v, dtype=np.float64)
    R = np.full((L, L), float(R)) if R.ndim == 0 else R.copy()
    np.fill_diagonal(R, 0.0)
    return R


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
