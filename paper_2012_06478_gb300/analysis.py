"""Host-side analysis of simulated signals (Sec. 2.3 and Sec. 3.2 of
Lee, Fieremans & Novikov, arXiv 2012.06478): the wide-pulse cumulant (DKI)
fit, the spherical (orientational) mean of each b-shell and its
intra-axonal power law (Eq. S-sph), and the MR-measured radius (Eq. r-mr).

These run on the signals the engine returns (numpy, float64); none of them
touches walkers.
"""
from __future__ import annotations

import itertools
import math
from typing import Tuple

import numpy as np

__all__ = ["dki_design", "dki_fit", "spherical_mean", "fit_spherical_mean", "r_mr", "mean_kurtosis_along"]

# index pairs (i <= j) and quadruples (i <= j <= k <= l) of the symmetric
# tensors, with their multiplicities in the full sums
_PAIRS = [(i, j) for i in range(3) for j in range(i, 3)]
_QUADS = [q for q in itertools.combinations_with_replacement(range(3), 4)]


def _multiplicity(idx) -> int:
    return len(set(itertools.permutations(idx)))


def dki_design(b: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Rows (one per direction and b): the coefficients of the 6 unique D_ij
    and the 15 unique A_ijkl = Dbar^2 W_ijkl in
      ln S = -b sum_ij n_ij D_ij + (b^2 / 6) sum_ijkl n_ijkl A_ijkl,
    n_ij = g_i g_j, n_ijkl = g_i g_j g_k g_l (the cumulant expansion of
    Sec. 2.3, wide pulses; Jensen et al. 2005)."""
    b = np.asarray(b, np.float64)
    g = np.asarray(dirs, np.float64)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    rows = []
    for gd in g:
        nd = np.array([_multiplicity(p) * gd[p[0]] * gd[p[1]] for p in _PAIRS])
        nk = np.array([_multiplicity(q) * gd[q[0]] * gd[q[1]] * gd[q[2]] * gd[q[3]] for q in _QUADS])
        for bb in b:
            rows.append(np.concatenate([-bb * nd, (bb * bb / 6.0) * nk]))
    return np.array(rows)


def _full2(v) -> np.ndarray:
    D = np.zeros((3, 3))
    for (i, j), x in zip(_PAIRS, v):
        D[i, j] = D[j, i] = x
    return D


def _full4(v) -> np.ndarray:
    W = np.zeros((3, 3, 3, 3))
    for q, x in zip(_QUADS, v):
        for p in set(itertools.permutations(q)):
            W[p] = x
    return W


def dki_fit(b: np.ndarray, dirs: np.ndarray, S: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Least-squares fit of the cumulant expansion to signals S (n_dirs, n_b)
    at b-values b (S normalised to 1 at b = 0; b = 0 columns are skipped).
    Returns the diffusion tensor D (3, 3) and the kurtosis tensor W
    (3, 3, 3, 3), W = A / Dbar^2 with Dbar = tr(D) / 3.  Needs at least 6
    directions and two nonzero b-values, and 15 directions for W."""
    b = np.asarray(b, np.float64)
    S = np.asarray(S)
    keep = b > 0
    y = np.log(np.abs(S[:, keep])).reshape(-1)
    X = dki_design(b[keep], dirs)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    D = _full2(coef[:6])
    Dbar = np.trace(D) / 3.0
    W = _full4(coef[6:]) / (Dbar * Dbar)
    return D, W


def mean_kurtosis_along(D: np.ndarray, W: np.ndarray, g: np.ndarray) -> Tuple[float, float]:
    """Apparent D and K along unit direction g: D_g = g.D.g,
    K_g = (Dbar / D_g)^2 W_ijkl g_i g_j g_k g_l."""
    g = np.asarray(g, np.float64) / np.linalg.norm(g)
    Dg = float(g @ D @ g)
    Dbar = np.trace(D) / 3.0
    Wg = float(np.einsum("ijkl,i,j,k,l->", W, g, g, g, g))
    return Dg, (Dbar / Dg) ** 2 * Wg


def spherical_mean(S: np.ndarray) -> np.ndarray:
    """Orientational average of each b-shell: S has shape (..., n_dirs, n_b)
    with the directions spread uniformly over the sphere (Sec. 3.2)."""
    return np.asarray(S).real.mean(axis=-2)


def fit_spherical_mean(b: np.ndarray, Sbar: np.ndarray) -> Tuple[float, float, float]:
    """Fit of Eq. S-sph, Sbar(b) = beta exp(-b D_perp) b^(-1/2), in its
    linear form ln(Sbar sqrt(b)) = ln(beta) - b D_perp over the given
    shells (b > 0, in the regime where the power law holds).  Returns
    (beta, D_perp, D_a) with beta = sqrt(pi / (4 D_a))."""
    b = np.asarray(b, np.float64)
    Sbar = np.asarray(Sbar, np.float64)
    keep = b > 0
    slope, icpt = np.polyfit(b[keep], np.log(Sbar[keep] * np.sqrt(b[keep])), 1)
    beta = math.exp(icpt)
    return beta, -slope, math.pi / (4.0 * beta * beta)


def r_mr(delta: float, t: float, D0: float, D_perp: float) -> float:
    """Eq. r-mr: the MR-measured radius [48/7 delta (t - delta/3) D0 D_perp]^(1/4)
    (um, with delta, t in ms, D in um^2/ms)."""
    return (48.0 / 7.0 * delta * (t - delta / 3.0) * D0 * D_perp) ** 0.25
