"""Pins of the host-side analysis (Sec. 2.3 wide-pulse cumulant fit, Sec. 3.2
spherical mean and Eq. r-mr) against closed forms and the paper's printed
worked value."""
import math
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def an():
    import __graft_entry__
    __graft_entry__._builder().build()
    from paper_2012_06478_gb300 import analysis
    return analysis


def fib_dirs(n):
    import rms_inputs as ri
    return ri.fibonacci_dirs(n)


def test_r_mr_reproduces_the_printed_value(an):
    """Sec. 3.2: D_perp = 1.6e-4 um^2/ms at (t, delta) = (20, 7.1) ms is an
    MR radius of 0.72 um (tests/golden/r_mr_sec3.txt)."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "r_mr_sec3.txt"))
            if l.strip() and not l.startswith("#")]
    for t, delta, D0, Dp, r, dec in rows:
        assert round(an.r_mr(float(delta), float(t), float(D0), float(Dp)), int(dec)) == float(r)


def test_r_mr_inverts_the_wide_pulse_cylinder_limit(an):
    """Neuman's wide-pulse limit for a cylinder of radius r,
    D_perp = 7 r^4 / (48 D0 delta (t - delta/3)), gives r_MR = r."""
    for r, delta, t, D0 in ((0.5, 7.1, 20.0, 2.0), (1.3, 35.1, 50.9, 1.7)):
        Dp = 7 * r ** 4 / (48 * D0 * delta * (t - delta / 3))
        assert abs(an.r_mr(delta, t, D0, Dp) - r) < 1e-12


def test_dki_fit_recovers_a_gaussian_tensor(an):
    """S = exp(-b g.D.g): the fit returns D exactly and W = 0."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    D = Q @ np.diag([2.0, 0.6, 0.3]) @ Q.T
    g = fib_dirs(30)
    b = np.array([0.0, 0.5, 1.0, 1.5, 2.0])
    S = np.exp(-b[None, :] * np.einsum("di,ij,dj->d", g, D, g)[:, None])
    Df, Wf = an.dki_fit(b, g, S)
    np.testing.assert_allclose(Df, D, atol=1e-10)
    assert np.abs(Wf).max() < 1e-8


def test_dki_fit_recovers_the_kurtosis_of_a_tensor_mixture(an):
    """Two Gaussian compartments (fractions f, 1 - f; tensors D1, D2): along
    g the cumulants are D_g = <g.D.g> and K_g = 3 Var(g.D.g) / D_g^2
    (Jensen et al. 2005).  Noiseless signals at small b: the fit's
    directional D and K match within the O(b^3) truncation."""
    f = 0.4
    D1 = np.diag([1.8, 0.4, 0.4])
    D2 = np.diag([0.9, 0.9, 0.9])
    g = fib_dirs(64)
    b = np.linspace(0.02, 0.3, 8)
    d1, d2 = (np.einsum("di,ij,dj->d", g, M, g) for M in (D1, D2))
    S = f * np.exp(-b[None, :] * d1[:, None]) + (1 - f) * np.exp(-b[None, :] * d2[:, None])
    Df, Wf = an.dki_fit(np.r_[0.0, b], g, np.c_[np.ones(len(g)), S])
    for gd in (np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([1.0, 1.0, 1.0]) / math.sqrt(3)):
        a1, a2 = gd @ D1 @ gd, gd @ D2 @ gd
        Dg = f * a1 + (1 - f) * a2
        Kg = 3 * f * (1 - f) * (a1 - a2) ** 2 / Dg ** 2
        Dfit, Kfit = an.mean_kurtosis_along(Df, Wf, gd)
        assert abs(Dfit - Dg) < 0.005 * Dg
        assert abs(Kfit - Kg) < 0.05 * max(Kg, 0.1), (gd, Kfit, Kg)


def test_spherical_mean_of_a_stick(an):
    """A stick (axial D_a, radial D_perp) along a random axis: the
    orientational mean over dense uniform directions equals the closed form
    exp(-b D_perp) sqrt(pi / (4 b (D_a - D_perp))) erf(sqrt(b (D_a - D_perp))),
    and the fit of Eq. S-sph over the paper's high-b shells (16-100
    ms/um^2) returns D_perp and D_a - D_perp (its beta = sqrt(pi/(4 D_a))
    sees the axial excess)."""
    rng = np.random.default_rng(2)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    Da, Dp = 2.0, 2e-3
    g = fib_dirs(4000)
    b = np.linspace(16, 100, 18)
    c2 = (g @ n) ** 2
    S = np.exp(-b[None, :] * (Dp + (Da - Dp) * c2[:, None]))
    Sbar = an.spherical_mean(S)
    from scipy.special import erf
    exact = np.exp(-b * Dp) * np.sqrt(np.pi / (4 * b * (Da - Dp))) * erf(np.sqrt(b * (Da - Dp)))
    np.testing.assert_allclose(Sbar, exact, rtol=2e-3)
    beta, Dp_fit, Da_fit = an.fit_spherical_mean(b, exact)
    assert abs(Dp_fit - Dp) < 1e-9
    assert abs(Da_fit - (Da - Dp)) < 1e-9
