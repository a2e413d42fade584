"""Seeded synthetic inputs for the RMS random-walker step.

This module is the only code shared by the CUDA path and the CPU oracle.  It
builds inputs only -- label volumes, per-label parameter tables, gradient
waveforms, directions, b-values, recording steps -- and holds none of the
method's arithmetic (no step length, permeation probability, phase, weight or
b-value computation; those live separately on each side).

The paper's own substrate (an EM segmentation of 227 mouse corpus-callosum
axons, Sec. 3.1) is not available; the generators below stand in for it with
the same kind of structure: a voxelised label volume (Sec. 2.1.1, one uint16
label per isotropic voxel) of beaded, undulating axons in an extra-axonal bath
(Sec. 3.2: caliber variation, undulation by the 1-harmonic model of App. D),
plus a simple cylinder, slabs, boxes and a periodic Voronoi tessellation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "cylinder_labels", "slab_labels", "box_labels", "axon_labels",
    "voronoi_labels", "pgse", "ogse", "fibonacci_dirs", "axis_dirs",
    "uniform_tables", "workload", "WORKLOADS", "serving_requests", "serving_geometry", "serving_tables",
    "SERVING_GEOMETRIES",
]


@dataclasses.dataclass
class Workload:
    """Everything one simulation needs.  Arrays are numpy, host side.

    labels     uint16 (nz, ny, nx), C order, so x is fastest in memory
    voxel_um   voxel edge l_p (um)
    periodic   3 ints (x, y, z)
    D, T2, T1  float64 per label (um^2/ms, ms, ms; inf = no relaxation)
    kappa      float64 (L, L) membrane permeability between labels (um/ms)
    dead       uint8 per label (1 = no walker starts in or enters it)
    dt         time step (ms); n_steps steps
    G          float64 (n_shapes, n_steps) unit-amplitude effective gradient,
               the average of g(t)/|g| over each step
    mode       uint8 per step or None (0 T2 weighting, 1 T1, 2 none)
    dirs       float64 (n_dirs, 3) unit gradient directions
    b          float64 b-values (ms/um^2)
    rec_steps  int64 increasing recording steps in [1, n_steps]
    n_walkers, seed
    interaction 0 elastic collision, 1 rejection sampling, 2 equal-step-length
               random leap (the particle-membrane interaction of a run)
    rho        float64 (L, L) surface relaxivity (um/ms) of the membrane met from
               label r towards label c (magnetization transfer), or None
    conc       float64 per label spin concentration, or None (all equal)
    lam        exponent lambda of (c2/c1) in the generalised permeation
               probability, in [0, 1]; < 0 picks the minimiser of alpha_lambda
    perm_model 0 nominal permeability kappa, 1 Baxter's concentration rule
               (kappa > 0 then only marks a permeable pair)
    """
    name: str
    labels: np.ndarray
    voxel_um: float
    periodic: tuple
    D: np.ndarray
    T2: np.ndarray
    T1: np.ndarray
    kappa: np.ndarray
    dead: np.ndarray
    dt: float
    n_steps: int
    G: np.ndarray
    mode: Optional[np.ndarray]
    dirs: np.ndarray
    b: np.ndarray
    rec_steps: np.ndarray
    n_walkers: int
    seed: int
    interaction: int = 0
    rho: Optional[np.ndarray] = None
    conc: Optional[np.ndarray] = None
    lam: float = -1.0
    perm_model: int = 0

    @property
    def n_labels(self) -> int:
        return int(self.D.shape[0])

    @property
    def shape_xyz(self):
        nz, ny, nx = self.labels.shape
        return nx, ny, nz

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------- substrates

def cylinder_labels(n: int = 32, radius_vox: float = 10.0, nz: Optional[int] = None) -> np.ndarray:
    """A z-aligned cylinder (label 1) in a label-0 bath on an n x n x nz grid.
    Voxel (x, y, .) is inside iff (x + 1/2 - n/2)^2 + (y + 1/2 - n/2)^2 <= r^2."""
    nz = n if nz is None else nz
    c = np.arange(n) + 0.5 - n / 2.0
    inside = (c[None, :] ** 2 + c[:, None] ** 2) <= radius_vox ** 2   # [y, x]
    return np.broadcast_to(inside.astype(np.uint16), (nz, n, n)).copy()


def slab_labels(widths: Sequence[int], ny: int = 4, nz: int = 4) -> np.ndarray:
    """Slabs stacked along x with the given widths (voxels); slab m has label m."""
    lab = np.concatenate([np.full(w, m, dtype=np.uint16) for m, w in enumerate(widths)])
    return np.broadcast_to(lab[None, None, :], (nz, ny, lab.size)).copy()


def box_labels(n_box: int, cells: int, wall_label: bool = False) -> np.ndarray:
    """A cubic lattice of cells^3 cubic pores, each n_box voxels on a side,
    pore m labelled m (every face between pores is a membrane)."""
    n = n_box * cells
    idx = np.arange(n) // n_box
    lab = idx[None, None, :] + cells * (idx[None, :, None] + cells * idx[:, None, None])
    return lab.astype(np.uint16)


def axon_labels(nx: int, ny: int, nz: int, voxel_um: float, n_axons: int, seed: int,
                r_shape: float = 6.25, r_scale: float = 0.08, r_min: float = 0.15,
                bead_spacing: float = 4.0, bead_amp=(0.2, 0.6), bead_sigma: float = 0.5,
                max_attempts: int = 20000) -> np.ndarray:
    """Beaded, undulating z-aligned axons (labels 1..n_axons) in a label-0 bath.

    * axis positions: random sequential addition on the periodic xy torus,
      largest radius first, no two base disks overlapping;
    * base radii: Gamma(k = r_shape, theta = r_scale) um (mean 0.5, sd 0.2 for
      the defaults), clipped below at r_min;
    * undulation: one harmonic (App. D), wavelength L_z/m with m in {1, 2},
      amplitude w0 = 0.02 lambda U(0.5, 1.5), random plane and phase;
    * beads: r(z) = r0 (1 + sum_b a_b exp(-(z - z_b)^2 / 2 sigma^2)), bead
      centres Poisson with mean spacing bead_spacing, a_b ~ U(bead_amp),
      periodic in z;
    * a voxel takes the axon with the smallest d / r(z) <= 1 (ties to the
      lower label), else the bath.
    """
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = nx * voxel_um, ny * voxel_um, nz * voxel_um
    r0 = np.maximum(rng.gamma(r_shape, r_scale, size=n_axons), r_min)
    r0 = np.sort(r0)[::-1]
    cx = np.zeros(n_axons)
    cy = np.zeros(n_axons)
    for a in range(n_axons):
        for _ in range(max_attempts):
            x, y = rng.uniform(0, Lx), rng.uniform(0, Ly)
            if a == 0:
                break
            dx = np.abs(cx[:a] - x)
            dx = np.minimum(dx, Lx - dx)
            dy = np.abs(cy[:a] - y)
            dy = np.minimum(dy, Ly - dy)
            if np.all(dx * dx + dy * dy >= (r0[:a] + r0[a]) ** 2):
                break
        else:
            raise RuntimeError("random sequential addition did not converge")
        cx[a], cy[a] = x, y
    z = (np.arange(nz) + 0.5) * voxel_um
    best = np.full((nz, ny, nx), np.inf)
    lab = np.zeros((nz, ny, nx), dtype=np.uint16)
    xs = (np.arange(nx) + 0.5) * voxel_um
    ys = (np.arange(ny) + 0.5) * voxel_um
    for a in range(n_axons):
        m = rng.integers(1, 3)
        lam = Lz / m
        w0 = 0.02 * lam * rng.uniform(0.5, 1.5)
        plane = rng.uniform(0, 2 * np.pi)
        ph = rng.uniform(0, 2 * np.pi)
        wz = w0 * np.cos(2 * np.pi * z / lam + ph)
        ccx = cx[a] + wz * np.cos(plane)
        ccy = cy[a] + wz * np.sin(plane)
        n_beads = rng.poisson(Lz / bead_spacing)
        zb = rng.uniform(0, Lz, size=n_beads)
        ab = rng.uniform(bead_amp[0], bead_amp[1], size=n_beads)
        dz = np.abs(z[:, None] - zb[None, :])
        dz = np.minimum(dz, Lz - dz)
        rz = r0[a] * (1.0 + (ab[None, :] * np.exp(-dz ** 2 / (2 * bead_sigma ** 2))).sum(axis=1))
        reach = rz.max() + w0 + voxel_um
        ix0 = int(math.floor((cx[a] - reach) / voxel_um))
        ix1 = int(math.ceil((cx[a] + reach) / voxel_um))
        iy0 = int(math.floor((cy[a] - reach) / voxel_um))
        iy1 = int(math.ceil((cy[a] + reach) / voxel_um))
        ixs = np.arange(ix0, ix1 + 1)
        iys = np.arange(iy0, iy1 + 1)
        px = (ixs + 0.5) * voxel_um
        py = (iys + 0.5) * voxel_um
        ddx = px[None, None, :] - ccx[:, None, None]
        ddy = py[None, :, None] - ccy[:, None, None]
        ddx -= Lx * np.round(ddx / Lx)
        ddy -= Ly * np.round(ddy / Ly)
        ratio = np.sqrt(ddx * ddx + ddy * ddy) / rz[:, None, None]
        gx = np.mod(ixs, nx)
        gy = np.mod(iys, ny)
        sub = best[:, gy[:, None], gx[None, :]]
        take = (ratio <= 1.0) & (ratio < sub)
        sub = np.where(take, ratio, sub)
        best[:, gy[:, None], gx[None, :]] = sub
        cur = lab[:, gy[:, None], gx[None, :]]
        lab[:, gy[:, None], gx[None, :]] = np.where(take, np.uint16(a + 1), cur)
    return lab


def voronoi_labels(n: int, n_cells: int, seed: int) -> np.ndarray:
    """Periodic Voronoi tessellation of an n^3 grid: voxel centre -> index of
    the nearest of n_cells uniform seeds (periodic distance), labels 0..n_cells-1."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(0, n, size=(n_cells, 3))
    tree = cKDTree(seeds, boxsize=n)
    lab = np.empty((n, n, n), dtype=np.uint16)
    g = np.arange(n) + 0.5
    yy, xx = np.meshgrid(g, g, indexing="ij")
    for zi in range(n):
        pts = np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, g[zi])], axis=1)
        _, idx = tree.query(pts, workers=-1)
        lab[zi] = idx.reshape(n, n).astype(np.uint16)
    return lab


# ---------------------------------------------------------------- tables

def uniform_tables(n_labels: int, D: float, kappa: float = 0.0, T2: float = math.inf,
                   T1: float = math.inf):
    """Per-label tables with one value for every label and one kappa for
    every membrane (every face between two different labels)."""
    Dv = np.full(n_labels, float(D))
    K = np.full((n_labels, n_labels), float(kappa))
    np.fill_diagonal(K, 0.0)
    return Dv, np.full(n_labels, float(T2)), np.full(n_labels, float(T1)), K, np.zeros(n_labels, np.uint8)


# ---------------------------------------------------------------- sequences

def _snap(x: float) -> float:
    r = round(x)
    return float(r) if abs(x - r) < 1e-9 else x


def _box_average(t0: float, t1: float, dt: float, n_steps: int) -> np.ndarray:
    """Fraction of each step [(k-1)dt, k dt] covered by [t0, t1]."""
    a, b = _snap(t0 / dt), _snap(t1 / dt)
    k = np.arange(n_steps, dtype=np.float64)
    return np.clip(np.minimum(b, k + 1) - np.maximum(a, k), 0.0, 1.0)


def pgse(delta: float, Delta: float, dt: float, n_steps: int, t0: float = 0.0) -> np.ndarray:
    """Pulsed-gradient spin echo, effective (unit amplitude) gradient averaged
    over each step: +1 on [t0, t0+delta], -1 on [t0+Delta, t0+Delta+delta]."""
    return (_box_average(t0, t0 + delta, dt, n_steps)
            - _box_average(t0 + Delta, t0 + Delta + delta, dt, n_steps))


def ogse(freq_hz: float, dt: float, n_steps: int, n_periods: int = 1, t0: float = 0.0) -> np.ndarray:
    """Cosine oscillating-gradient spin echo, two lobes of n_periods periods:
    g = cos(2 pi f (t - t0)) in lobe 1 and the negated copy in lobe 2 right
    after it, zero elsewhere; averaged over each step."""
    f = freq_hz * 1e-3  # 1/ms
    T = n_periods / f
    t = np.arange(n_steps + 1) * dt

    def lobe(start, sign):
        tt = np.clip(t, start, start + T)
        prim = np.sin(2 * np.pi * f * (tt - start)) / (2 * np.pi * f)
        return sign * np.diff(prim) / dt

    return lobe(t0, 1.0) + lobe(t0 + T, -1.0)


def axis_dirs() -> np.ndarray:
    return np.eye(3)


def fibonacci_dirs(n: int) -> np.ndarray:
    """n nearly uniform unit vectors (Fibonacci sphere)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = np.pi * (3.0 - np.sqrt(5.0)) * k
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _rec(n_steps: int, every: int) -> np.ndarray:
    return np.arange(every, n_steps + 1, every, dtype=np.int64)


# ---------------------------------------------------------------- workloads

def _cylinder32() -> Workload:
    """Plain FP64 check case: 32^3 grid, 0.2 um voxels, periodic; one z-aligned
    cylinder of radius 2 um (label 1) in a label-0 bath, impermeable; D = 2
    for both; 1e4 walkers; dt = 1e-3 ms, 5000 steps; PGSE delta = 1,
    Delta = 3 ms; b in {0, 1} along x, y, z; recording every 50 steps."""
    lab = cylinder_labels(32, 10.0)
    D, T2, T1, K, dead = uniform_tables(2, 2.0, 0.0)
    dt, n = 1e-3, 5000
    return Workload("cylinder-32^3", lab, 0.2, (1, 1, 1), D, T2, T1, K, dead, dt, n,
                    pgse(1.0, 3.0, dt, n)[None, :], None, axis_dirs(), np.array([0.0, 1.0]),
                    _rec(n, 50), 10_000, 1)


def _axons(nx, ny, nz, n_axons, seed, D_in, D_ex, kappa, T2_in, T2_ex, dt, n_steps,
           shapes, n_walkers, dirs, b, rec_every, name, kappa_per_axon=None) -> Workload:
    lab = axon_labels(nx, ny, nz, 0.1, n_axons, seed)
    L = n_axons + 1
    D = np.full(L, float(D_in))
    D[0] = D_ex
    T2 = np.full(L, float(T2_in))
    T2[0] = T2_ex
    T1 = np.full(L, math.inf)
    if kappa_per_axon is None:
        K = np.full((L, L), float(kappa))
    else:
        # two membranes in series between touching axons; the bath has none
        k = np.concatenate([[math.inf], kappa_per_axon])
        with np.errstate(divide="ignore"):
            K = 1.0 / (1.0 / k[:, None] + 1.0 / k[None, :])
    np.fill_diagonal(K, 0.0)
    return Workload(name, lab, 0.1, (1, 1, 1), D, T2, T1, K, np.zeros(L, np.uint8), dt, n_steps,
                    shapes, None, dirs, b, _rec(n_steps, rec_every), n_walkers, seed)


def _axons200() -> Workload:
    """FP64-vs-FP32 workload: 200 x 200 x 400 grid, 0.1 um voxels; 200 beaded,
    undulating axons; D = 2 everywhere; kappa = 0.01 um/ms; 1e6 walkers,
    1e5 steps of dt = 2e-4 ms; PGSE delta = 5, Delta = 15 ms; 30 directions
    x b = 0..10 ms/um^2; recording every 1000 steps."""
    dt, n = 2e-4, 100_000
    return _axons(200, 200, 400, 200, 2, 2.0, 2.0, 0.01, math.inf, math.inf, dt, n,
                  pgse(5.0, 15.0, dt, n)[None, :], 1_000_000, fibonacci_dirs(30),
                  np.arange(11, dtype=np.float64), 1000, "axons-200x200x400")


def _axons400() -> Workload:
    """FP32 workload with T2 and unequal D: 400^3 grid, 0.1 um voxels, 800 axons
    (the 200-axon density); D_in = 2, D_ex = 1.5; T2 60 / 40 ms; kappa
    log-uniform 0.005-0.05 per axon; 4e6 walkers; dt = 4e-4 ms over 100 ms
    (2.5e5 steps, the length of one 20 Hz lobe pair); PGSE delta = 3,
    Delta = 7 ms and cosine OGSE at 20, 40, 60, 80, 100 Hz."""
    dt, n = 4e-4, 250_000
    rng = np.random.default_rng(3)
    kap = np.exp(rng.uniform(np.log(0.005), np.log(0.05), size=800))
    shapes = np.stack([pgse(3.0, 7.0, dt, n)] + [ogse(f, dt, n) for f in (20, 40, 60, 80, 100)])
    return _axons(400, 400, 400, 800, 3, 2.0, 1.5, None, 60.0, 40.0, dt, n, shapes, 4_000_000,
                  fibonacci_dirs(30), np.array([0.0, 0.5, 1.0, 2.0, 3.0]), 2500,
                  "axons-400^3-t2-ogse", kappa_per_axon=kap)


def _voronoi512() -> Workload:
    """Large FP32 workload: 512^3 grid, 0.1 um voxels, 1000 periodic Voronoi
    cells; D ~ U(0.5, 2.5), per-pair kappa ~ U(0, 0.05) (symmetric),
    T1 ~ U(600, 1000), T2 ~ U(40, 100) ms; 1e7 walkers, 2e4 steps of
    dt = 1e-4 ms; PGSE delta = 0.5, Delta = 1.5 ms; 64 directions x 8
    b-values; recording every 200 steps."""
    L = 1000
    lab = voronoi_labels(512, L, 5)
    rng = np.random.default_rng(5)
    D = rng.uniform(0.5, 2.5, size=L)
    T1 = rng.uniform(600, 1000, size=L)
    T2 = rng.uniform(40, 100, size=L)
    K = rng.uniform(0.0, 0.05, size=(L, L))
    K = np.triu(K, 1)
    K = K + K.T
    dt, n = 1e-4, 20_000
    return Workload("voronoi-512^3", lab, 0.1, (1, 1, 1), D, T2, T1, K, np.zeros(L, np.uint8), dt, n,
                    pgse(0.5, 1.5, dt, n)[None, :], None, fibonacci_dirs(64),
                    np.array([0.25, 0.5, 1, 2, 3, 4, 6, 8], dtype=np.float64), _rec(n, 200),
                    10_000_000, 5)


WORKLOADS = {
    "cylinder-32^3": _cylinder32,
    "axons-200x200x400": _axons200,
    "axons-400^3-t2-ogse": _axons400,
    "voronoi-512^3": _voronoi512,
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]()


# ---------------------------------------------------------------- serving load

SERVING_GEOMETRIES = 2  # label volumes per (kind, size) in the serving pool


def serving_geometry(kind: str, n: int, geometry_seed: int) -> np.ndarray:
    """Label volume of a serving request: the cylinder, axon or Voronoi
    generator at n^3 with 0.1 um voxels (axons at the 200-axon workload's
    areal density, Voronoi cells at the 512^3 workload's cell density)."""
    rng = np.random.default_rng(1000 * n + geometry_seed)
    if kind == "cylinder":
        return cylinder_labels(n, n * rng.uniform(0.2, 0.4))
    if kind == "axons":
        return axon_labels(n, n, n, 0.1, max(2, int(round(200 * (n / 200.0) ** 2))), seed=40 + n + 7 * geometry_seed)
    return voronoi_labels(n, max(8, int(1000 * (n / 512.0) ** 3)), seed=50 + n + 7 * geometry_seed)


def serving_tables(kind: str, n_labels: int, params_seed: int):
    """Per-label tissue tables of a serving request, drawn per request by the
    recipe of its generator's workload: the cylinder with D ~ U(0.5, 2.5) per
    label, kappa log-uniform 0.005-0.05 um/ms, T2 ~ U(40, 100) ms; axons with
    D_in = 2, D_ex = 1.5, per-axon kappa log-uniform 0.005-0.05 (two
    membranes in series between axons), T2 60 / 40 ms; Voronoi cells with
    D ~ U(0.5, 2.5), per-pair kappa ~ U(0, 0.05), T1 ~ U(600, 1000),
    T2 ~ U(40, 100) ms.  Returns D, T2, T1, kappa (L, L)."""
    rng = np.random.default_rng(params_seed)
    L = n_labels
    T1 = np.full(L, math.inf)
    if kind == "cylinder":
        D = rng.uniform(0.5, 2.5, size=L)
        T2 = rng.uniform(40, 100, size=L)
        K = np.full((L, L), math.exp(rng.uniform(math.log(0.005), math.log(0.05))))
    elif kind == "axons":
        D = np.full(L, 2.0)
        D[0] = 1.5
        T2 = np.full(L, 60.0)
        T2[0] = 40.0
        k = np.concatenate([[math.inf], np.exp(rng.uniform(math.log(0.005), math.log(0.05), size=L - 1))])
        with np.errstate(divide="ignore"):
            K = 1.0 / (1.0 / k[:, None] + 1.0 / k[None, :])
    else:
        D = rng.uniform(0.5, 2.5, size=L)
        T1 = rng.uniform(600, 1000, size=L)
        T2 = rng.uniform(40, 100, size=L)
        K = np.triu(rng.uniform(0.0, 0.05, size=(L, L)), 1)
        K = K + K.T
    np.fill_diagonal(K, 0.0)
    return D, T2, T1, K


def serving_requests(n: int, seed: int, sizes=(32, 64, 128, 256), walkers=(1e4, 1e6),
                     steps=(1e3, 5e4), dirs=(6, 64)):
    """A seeded stream of simulation requests: each a substrate kind from
    {cylinder, axons, voronoi} at n^3, log-uniform walkers and steps, a
    uniform number of directions.  Returns a list of dicts (no arrays)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        out.append(dict(
            kind=["cylinder", "axons", "voronoi"][int(rng.integers(0, 3))],
            n=int(sizes[int(rng.integers(0, len(sizes)))]),
            n_walkers=int(round(math.exp(rng.uniform(math.log(walkers[0]), math.log(walkers[1]))))),
            n_steps=int(round(math.exp(rng.uniform(math.log(steps[0]), math.log(steps[1]))))),
            n_dirs=int(rng.integers(dirs[0], dirs[1] + 1)),
            seed=int(rng.integers(0, 2 ** 63 - 1)),
            geometry=int(rng.integers(0, SERVING_GEOMETRIES)),
        ))
    return out
