"""b_s of each waveform shape (Sec. 2.3: b = dt sum_j F_{j-1}^2, F_j the
running integral of the unit-amplitude gradient), computed on the GPU with
the waveform staged through shared memory in chunks of 2048 steps, is the
oracle's sequential compensated sum bit for bit (the same operations in the
same order), and matches the closed form delta^2 (Delta - delta/3) of a
step-aligned PGSE.  Lengths cover one step, a partial chunk, exact chunks, a
ragged last chunk, several shapes and N = 0."""
import numpy as np
import pytest

import rms_inputs as ri
from conftest import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


def _bvalues(rms, G, dt):
    S, N = G.shape
    wl = make_workload(np.zeros((2, 2, 2)), voxel_um=0.2, D=1.0, dt=dt, n_steps=N, G=G, n_walkers=1,
                       rec_steps=np.zeros(0, np.int64))
    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps)
    out = rms.rms_sequence_bvalues(seq)
    seq.close()
    sub.close()
    return out


@pytest.mark.parametrize("N", [1, 7, 2047, 2048, 2049, 4096, 65537, 100000])
def test_bvalue_against_the_oracle(rms, N):
    import oracle
    oracle.build()
    rng = np.random.default_rng(N)
    G = np.stack([rng.normal(size=N), np.cos(np.arange(N) * 0.01), (rng.uniform(size=N) < 0.2) * 1.0])
    dt = 2e-4
    got = _bvalues(rms, G, dt)
    for s in range(G.shape[0]):
        want = oracle.bvalue(np.ascontiguousarray(G[s]), dt)
        assert got[s] == want, (s, got[s], want)


def test_bvalue_pgse_closed_form(rms):
    dt, n = 2e-4, 100000                                   # delta = 5, Delta = 15 ms, TE = 20 ms
    G = ri.pgse(5.0, 15.0, dt, n)[None, :]
    got = _bvalues(rms, G, dt)
    assert abs(got[0] - 25.0 * (15.0 - 5.0 / 3.0)) <= 1e-9 * 25.0 * 15.0, got[0]


def test_bvalue_of_no_steps_is_zero(rms):
    assert np.array_equal(_bvalues(rms, np.zeros((1, 0)), 1e-3), np.zeros(1))
