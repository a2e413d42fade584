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


def test_axon_generator_follows_the_recipe():
    """The 200-axon recipe on a shorter stack (20 x 20 x 8 um, 0.1 um voxels):
    every axon is present, the narrowest cross-section of each axon (away
    from its beads) gives back the base radius distribution Gamma(6.25, 0.08)
    clipped at 0.15 um (mean 0.5, sd 0.2), about half the volume is
    intra-axonal, and the volume continues across the periodic z boundary."""
    import math
    nz = 80
    lab = ri.axon_labels(200, 200, nz, 0.1, 200, seed=2)
    present = np.unique(lab)
    assert present[0] == 0 and list(present[1:]) == list(range(1, 201))
    area = np.stack([np.bincount(lab[z].ravel(), minlength=201) for z in range(nz)])  # (z, label)
    r_min = np.sqrt(area[:, 1:].min(axis=0) / math.pi) * 0.1
    assert abs(r_min.mean() - 0.5) < 4.5 * 0.2 / math.sqrt(200), r_min.mean()
    assert 0.15 < r_min.std() < 0.25, r_min.std()
    assert r_min.min() >= 0.15 - 0.1
    assert 0.4 < (lab > 0).mean() < 0.7
    step = [(lab[z] != lab[z + 1]).mean() for z in range(nz - 1)]
    assert (lab[nz - 1] != lab[0]).mean() <= 3 * max(step)


def test_voronoi_generator_is_the_periodic_nearest_seed_map():
    """Every voxel centre takes its nearest seed under the periodic (minimum
    image) distance: checked by brute force over all seeds on a 16^3 grid."""
    n, cells, seed = 16, 20, 7
    lab = ri.voronoi_labels(n, cells, seed)
    seeds = np.random.default_rng(seed).uniform(0, n, size=(cells, 3))   # the generator's seed draw
    g = np.arange(n) + 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([x, y, z], axis=-1)[..., None, :]                        # (n, n, n, 1, 3)
    d = np.abs(p - seeds)
    d = np.minimum(d, n - d)
    expect = np.argmin((d * d).sum(axis=-1), axis=-1)
    np.testing.assert_array_equal(lab, expect)
    assert len(np.unique(lab)) == cells


def test_ogse_waveform_b_value():
    """Cosine OGSE, n periods per lobe at frequency f: q(t) = sin(2 pi f t)/(2 pi f)
    over each lobe, so b = 2 int_0^T q^2 dt = n / (4 pi^2 f^3) (ms/um^2 for f in
    1/ms); the step-averaged waveform's discrete b_s tends to it as dt -> 0."""
    import math
    import oracle
    oracle.build()
    for f_hz, n_per in ((100.0, 1), (40.0, 2)):
        f = f_hz * 1e-3
        dt = 4e-4
        n = int(math.ceil(2 * n_per / f / dt)) + 10
        G = ri.ogse(f_hz, dt, n, n_periods=n_per)
        exact = n_per / (4 * math.pi ** 2 * f ** 3)
        assert abs(oracle.bvalue(G, dt) - exact) < 1e-3 * exact, (f_hz, oracle.bvalue(G, dt), exact)
        assert abs(G.sum()) < 1e-9 and np.all(G[int(2 * n_per / f / dt) + 2:] == 0.0)
