"""The seeded input generators: deterministic, and shaped as documented."""
import numpy as np

import rms_inputs as ri


def test_cylinder_cross_section():
    lab = ri.cylinder_labels(32, 10.0)
    assert lab.shape == (32, 32, 32) and lab.dtype == np.uint16
    # every z-slice identical; area close to pi r^2 = 314.16 voxels
    assert all((lab[z] == lab[0]).all() for z in range(32))
    assert abs(int(lab[0].sum()) - np.pi * 100) < 5


def test_pgse_and_ogse_waveforms():
    dt, n = 1e-3, 5000
    G = ri.pgse(1.0, 3.0, dt, n)
    assert G.sum() == 0.0 and G[:1000].min() == 1.0 and G[3000:4000].max() == -1.0
    assert np.count_nonzero(G) == 2000
    O = ri.ogse(100.0, 1e-3, 20000)
    assert abs(O.sum()) < 1e-9 and np.abs(O).max() <= 1.0 + 1e-12


def test_directions_unit():
    d = ri.fibonacci_dirs(30)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=1e-14)
    assert abs(d.mean(axis=0)).max() < 0.05


def test_axon_generator_deterministic():
    a = ri.axon_labels(60, 60, 40, 0.1, 8, seed=2)
    b = ri.axon_labels(60, 60, 40, 0.1, 8, seed=2)
    c = ri.axon_labels(60, 60, 40, 0.1, 8, seed=3)
    assert (a == b).all() and not (a == c).all()
    assert a.max() <= 8 and 0.05 < (a > 0).mean() < 0.6
    # beads: the cross-section of an axon varies along z
    area = (a == 1).sum(axis=(1, 2))
    assert area.max() > area.min()


def test_serving_requests_seeded():
    r1 = ri.serving_requests(20, 4)
    assert r1 == ri.serving_requests(20, 4)
    assert all(1e4 <= r["n_walkers"] <= 1e6 and 6 <= r["n_dirs"] <= 64 for r in r1)
