"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one oracle routine against a closed form, a library routine,
an exact quadrature identity or an exact property of the transform (Parseval,
the Laplacian eigenvalues, solid-body rotation, the adjoint identity), chosen
so that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""

import math

import numpy as np
import pytest
from scipy import special

from paper_1908_06097_gb300 import inputs

OCT, FULL = 0, 1


# ------------------------------------------------------------------ closed forms
# Ferrers functions without the Condon-Shortley phase for n <= 4, written in the
# latitude phi (mu = sin phi, sin(colatitude) = cos phi) so that they can be
# differentiated exactly by the complex-step method.
def _ferrers(n, m, phi):
    mu, s = np.sin(phi), np.cos(phi)
    table = {
        (0, 0): 1.0 + 0 * mu,
        (1, 0): mu, (1, 1): s,
        (2, 0): (3 * mu**2 - 1) / 2, (2, 1): 3 * mu * s, (2, 2): 3 * s**2,
        (3, 0): (5 * mu**3 - 3 * mu) / 2, (3, 1): 1.5 * (5 * mu**2 - 1) * s,
        (3, 2): 15 * mu * s**2, (3, 3): 15 * s**3,
        (4, 0): (35 * mu**4 - 30 * mu**2 + 3) / 8, (4, 1): 2.5 * (7 * mu**3 - 3 * mu) * s,
        (4, 2): 7.5 * (7 * mu**2 - 1) * s**2, (4, 3): 105 * mu * s**3, (4, 4): 105 * s**4,
    }
    return table[(n, m)]


def pbar_closed(n, m, phi):
    """Orthonormal P_n^m(sin phi): sqrt((2n+1)/2 (n-m)!/(n+m)!) times the Ferrers function."""
    c = math.sqrt((2 * n + 1) / 2 * math.factorial(n - m) / math.factorial(n + m))
    return c * _ferrers(n, m, phi)


def dpbar_dphi(n, m, phi):
    """d/dphi of pbar_closed by the complex step (exact to rounding)."""
    h = 1e-30
    return np.imag(pbar_closed(n, m, phi + 1j * h)) / h


def y_real(n, m, phi, lam, re=1.0, im=0.0):
    """Grid field of the single coefficient a_n^m = re + i im under the real convention."""
    p = pbar_closed(n, m, phi)
    if m == 0:
        return re * p + 0 * lam
    return 2 * p * (re * np.cos(m * lam) - im * np.sin(m * lam))


def grid_coords(orc, kind, N, T):
    nlon, _, npts = orc.grid(kind, N, T)
    x, _ = orc.gauss(2 * N)
    phi = np.concatenate([np.full(nl, np.arcsin(xk)) for nl, xk in zip(nlon, x)])
    lam = np.concatenate([2 * np.pi * np.arange(nl) / nl for nl in nlon])
    return phi, lam


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------- Gauss nodes
def test_gauss_closed_forms(orc):
    x, w = orc.gauss(2)
    assert np.allclose(x, [1 / math.sqrt(3), -1 / math.sqrt(3)], rtol=0, atol=2.3e-16)
    assert np.allclose(w, [1, 1], rtol=0, atol=1e-15)
    x, w = orc.gauss(3)
    assert np.allclose(x, [math.sqrt(0.6), 0, -math.sqrt(0.6)], rtol=0, atol=2.3e-16)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], rtol=0, atol=1e-15)


@pytest.mark.parametrize("nlat", [1, 4, 7, 32, 160, 200])
def test_gauss_vs_numpy_leggauss(orc, nlat):
    x, w = orc.gauss(nlat)
    xr, wr = np.polynomial.legendre.leggauss(nlat)
    # numpy's weights carry ~3e-13 relative error at nlat = 200; the long-double
    # build pins ours more tightly
    assert np.abs(x - xr[::-1]).max() < 4e-16
    assert np.abs(w - wr[::-1]).max() < 5e-13 * wr.max()
    xl, wl = orc.gauss(nlat, long_double=True)
    assert np.abs(w - wl).max() < 1e-14 * wl.max()
    assert abs(w.sum() - 2) < 1e-14
    assert np.all(np.diff(x) < 0) and np.all(x == -x[::-1])


def test_gauss_integrates_monomials_exactly(orc):
    nlat = 40
    x, w = orc.gauss(nlat)
    for k in range(2 * nlat):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x**k) - exact) < 2e-15


def test_gauss_large_sum(orc):
    x, w = orc.gauss(2560)
    assert abs(w.sum() - 2) < 1e-13
    xl, wl = orc.gauss(2560, long_double=True)
    assert np.abs(x - xl).max() < 4e-16


# ------------------------------------------------------------- Legendre functions
@pytest.mark.parametrize("x", [0.93, 0.31, -0.55, 1e-3])
def test_plm_closed_forms(orc, x):
    phi = math.asin(x)
    for m in range(5):
        p = orc.plm(m, 4, x)
        for n in range(m, 5):
            assert abs(p[n - m] - pbar_closed(n, m, phi)) < 2e-15


@pytest.mark.parametrize("m", [0, 1, 3, 10, 25])
def test_plm_vs_scipy_lpmv(orc, m):
    """scipy's Ferrers function carries the (-1)^m phase; the normalisation is by factorials."""
    for x in [0.8, -0.2, 0.05]:
        p = orc.plm(m, 40, x)
        for n in range(m, 41):
            norm = math.exp(0.5 * (math.log((2 * n + 1) / 2) + math.lgamma(n - m + 1) - math.lgamma(n + m + 1)))
            ref = (-1) ** m * special.lpmv(m, n, x) * norm
            assert abs(p[n - m] - ref) < 1e-12 * max(1.0, abs(ref))


def test_plm_quadrature_orthonormal(orc):
    T, nlat = 79, 160
    x, w = orc.gauss(nlat)
    for m in [0, 1, 2, 17, 40, 78, 79]:
        P = np.array([orc.plm(m, T, xk) for xk in x])  # [lat][n]
        G = (P * w[:, None]).T @ P
        assert np.abs(G - np.eye(T - m + 1)).max() < 1e-13


def test_plm_sectoral_extended_range(orc):
    """P_m^m = sqrt((2m+1)/2 (2m)!)/(2^m m!) sin^m(theta): checked in log form where it
    is tiny but representable, and 0 where it lies below the FP64 range."""
    for m, s in [(1279, 0.62), (900, 0.7), (600, 0.5), (1279, 0.95)]:
        x = math.sqrt(1 - s * s)
        logv = (0.5 * math.log((2 * m + 1) / 2) + 0.5 * math.lgamma(2 * m + 1) - m * math.log(2)
                - math.lgamma(m + 1) + m * math.log(s))
        got = orc.plm(m, m, x)[0]
        assert got > 0 and abs(math.log(got) - logv) < 1e-11
    assert orc.plm(1279, 1279, math.sqrt(1 - 1e-4))[0] == 0.0
    # columns that start below the FP64 range and grow with n agree with the
    # long-double build wherever they are representable
    for m, s in [(600, 0.2), (300, 0.02), (1000, 0.55)]:
        x = math.sqrt(1 - s * s)
        p, pl = orc.plm(m, 1280, x), orc.plm(m, 1280, x, long_double=True)
        big = np.abs(pl) > 1e-290
        assert np.all(np.abs(p[big] / pl[big] - 1) < 1e-11)
        assert np.all(np.abs(p[~big]) < 1e-280)


def test_hlm_vs_complex_step(orc):
    """H_n^m = (1 - mu^2) dP/dmu = cos(phi) dP/dphi, against the closed forms."""
    for x in [0.7, -0.25, 0.02]:
        phi = math.asin(x)
        for m in range(4):
            h = orc.hlm(m, 3, x)
            for n in range(m, 4):
                assert abs(h[n - m] - math.cos(phi) * dpbar_dphi(n, m, phi)) < 5e-15


def test_hlm_vs_finite_difference_high_degree(orc):
    m, T = 7, 120
    x0, dx = 0.4, 1e-5
    h = orc.hlm(m, T, x0)
    fd = (orc.plm(m, T + 1, x0 + dx)[:-1] - orc.plm(m, T + 1, x0 - dx)[:-1]) / (2 * dx)
    assert np.abs(h - (1 - x0 * x0) * fd).max() < 1e-6 * np.abs(h).max()


# -------------------------------------------------------------------- transforms
@pytest.mark.parametrize("kind", [OCT, FULL])
def test_inverse_single_modes_closed_form(orc, kind):
    T, N = 8, 9
    phi, lam = grid_coords(orc, kind, N, T)
    nc = inputs.ncoef(T)
    for n in range(5):
        for m in range(n + 1):
            for re, im in [(1.0, 0.0), (0.0, 1.0), (0.3, -0.7)]:
                spec = np.zeros((1, nc, 2))
                spec[0, inputs.coef_index(T, n, m)] = [re, im]
                g = orc.inverse(T, kind, N, spec)[0]
                ref = y_real(n, m, phi, lam, re, 0.0 if m == 0 else im)
                assert np.abs(g - ref).max() < 1e-14


@pytest.mark.parametrize("kind", [OCT, FULL])
def test_derivatives_single_modes(orc, kind):
    T, N = 6, 7
    phi, lam = grid_coords(orc, kind, N, T)
    nc = inputs.ncoef(T)
    for n in range(5):
        for m in range(n + 1):
            spec = np.zeros((1, nc, 2))
            spec[0, inputs.coef_index(T, n, m)] = [0.6, -0.8 if m else 0.0]
            g, dl, dp = orc.inverse(T, kind, N, spec, deriv=True)
            ref_dl = 0 * phi if m == 0 else 2 * m * pbar_closed(n, m, phi) * (
                -0.6 * np.sin(m * lam) + 0.8 * np.cos(m * lam))
            ref_dp = dpbar_dphi(n, m, phi) * (1.0 if m == 0 else 2 * (0.6 * np.cos(m * lam) + 0.8 * np.sin(m * lam)))
            if m == 0:
                ref_dp = 0.6 * dpbar_dphi(n, m, phi)
            assert np.abs(dl[0] - ref_dl).max() < 1e-13
            assert np.abs(dp[0] - ref_dp).max() < 1e-13


def test_roundtrip_full_gaussian_exact(orc):
    T, N = 31, 32
    a = inputs.spectral_fields(T, 3, inputs.SEED_BASE)
    g = orc.inverse(T, FULL, N, a)
    b = orc.direct(T, FULL, N, g)
    assert relmax(b, a) < 1e-13
    e, _ = orc.roundtrip_defect(T, FULL, N)
    assert e == 0.0


def test_roundtrip_octahedral_within_defect(orc):
    """On O80 the only round-trip error is the quadrature mass of the polar rings a
    wavenumber skips; the defect matrix bounds it."""
    T, N = 79, 80
    a = inputs.spectral_fields(T, 2, inputs.SEED_BASE)
    g = orc.inverse(T, OCT, N, a)
    b = orc.direct(T, OCT, N, g)
    e, em = orc.roundtrip_defect(T, OCT, N)
    ns, ms = inputs.coef_nm(T)
    for f in range(2):
        for m in range(T + 1):
            sel = ms == m
            bound = em[m] * np.abs(a[f, sel]).sum() * 2 + 1e-14
            assert np.abs(b[f, sel] - a[f, sel]).max() <= bound


def _pbar_scipy(n, m, x):
    """Orthonormal P_n^m(x) without the Condon-Shortley phase, from scipy's lpmv
    (which carries the phase) and the factorial normalisation."""
    c = math.sqrt((2 * n + 1) / 2 * math.exp(math.lgamma(n - m + 1) - math.lgamma(n + m + 1)))
    return c * (-1) ** m * special.lpmv(m, n, x)


def _skipped_mass_numpy(T, N):
    """E_m = max_{n,n'} |sum over the rings that do not carry m of w_k P_n^m P_n'^m|,
    computed here from numpy's Gauss-Legendre rule, scipy's Legendre functions and
    the octahedral ring rule (ring i from a pole has 4i+16 points and carries
    m <= min(T, (4i+16)/2 - 1)); nothing of the oracle is used."""
    x, w = np.polynomial.legendre.leggauss(2 * N)
    x, w = x[::-1], w[::-1]  # north first
    nlon = inputs.octahedral_nlon(N)
    mmax = np.minimum(T, nlon // 2 - 1)
    em = np.zeros(T + 1)
    for m in range(T + 1):
        skip = np.nonzero(mmax < m)[0]
        if len(skip) == 0:
            continue
        P = np.array([[_pbar_scipy(n, m, x[k]) for k in skip] for n in range(m, T + 1)])
        M = (P * w[skip][None, :]) @ P.T
        em[m] = np.abs(M).max()
    return em


# Coarse octahedral grids O(N) with 2N >= T + 1: Gauss-Legendre on 2N nodes is
# still exact for the degree-2T products, but the rings that carry fewer than
# T+1 wavenumbers reach mid-latitudes, so the skipped quadrature mass is 6e-3
# (T=31 on O16) and 0.22 (T=47 on O24) instead of the ~1e-12 of O(T+1), and a
# wrong exclusion rule or weight shows.
COARSE = [(31, 16), (47, 24)]


@pytest.mark.parametrize("T,N", COARSE + [(79, 80)])
def test_roundtrip_defect_vs_numpy_skipped_mass(orc, T, N):
    """The oracle's defect table equals the quadrature mass of the skipped rings
    computed independently (numpy nodes and weights, scipy Legendre functions)."""
    e, em = orc.roundtrip_defect(T, OCT, N)
    ref = _skipped_mass_numpy(T, N)
    assert np.all(ref[: 10] == 0)  # ring 1 (20 points) carries m <= 9
    if N < T + 1:
        assert ref.max() > 1e-3
        np.testing.assert_allclose(em, ref, rtol=1e-10, atol=1e-15)
    else:  # O(T+1): the mass is near rounding; agreement to the rounding level
        np.testing.assert_allclose(em, ref, rtol=1e-6, atol=1e-16)
    assert e == pytest.approx(ref.max(), rel=1e-6)


@pytest.mark.parametrize("T,N", COARSE)
def test_roundtrip_defect_equals_brute_force_identity_defect(orc, T, N):
    """Brute force: direct(inverse(e_j)) for every real and imaginary unit
    vector e_j.  Its deviation from the identity, per wavenumber m, is minus
    the skipped-ring quadrature matrix, so its largest entry per m equals the
    defect table entry E_m."""
    nc = inputs.ncoef(T)
    ns, ms = inputs.coef_nm(T)
    cols = []
    for part in (0, 1):
        basis = np.zeros((nc, nc, 2))
        basis[np.arange(nc), np.arange(nc), part] = 1.0
        cols.append(orc.direct(T, OCT, N, orc.inverse(T, OCT, N, basis)))
    _, em = orc.roundtrip_defect(T, OCT, N)
    assert em.max() > 1e-3
    for m in range(T + 1):
        sel = np.nonzero(ms == m)[0]
        dev = []
        for part in (0, 1):
            if m == 0 and part == 1:
                continue  # Im a_n^0 is not carried
            D = cols[part][np.ix_(sel, sel)][:, :, part]  # response in the same part
            dev.append(np.abs(D.T - np.eye(len(sel))).max())
            # no leakage into the other part or another wavenumber
            other = np.delete(np.arange(nc), sel)
            assert np.abs(cols[part][np.ix_(sel, other)]).max() < 1e-13
            assert np.abs(cols[part][np.ix_(sel, sel)][:, :, 1 - part]).max() < 1e-13
        assert max(dev) == pytest.approx(em[m], rel=1e-10, abs=1e-14), m


def test_parseval_full_grid(orc):
    T, N = 24, 25
    a = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 7)
    g = orc.inverse(T, FULL, N, a)
    nlon, _, _ = orc.grid(FULL, N, T)
    x, w = orc.gauss(2 * N)
    wpt = np.concatenate([np.full(nl, wk / nl) for nl, wk in zip(nlon, w)])
    ns, ms = inputs.coef_nm(T)
    for f in range(2):
        lhs = np.dot(wpt, g[f] ** 2)
        rhs = (a[f, ms == 0, 0] ** 2).sum() + 2 * (a[f, ms > 0] ** 2).sum()
        assert abs(lhs - rhs) < 1e-13 * rhs


def test_direct_vs_numpy_rfft_on_one_ring(orc):
    """The ring analysis equals numpy's FFT: a field that depends on longitude only
    through one ring's samples is checked via its coefficients on the full grid."""
    T, N = 15, 16
    a = inputs.spectral_fields(T, 1, inputs.SEED_BASE + 3)
    g = orc.inverse(T, FULL, N, a)[0]
    nlon, mmax, _ = orc.grid(FULL, N, T)
    ring = g[: nlon[0]]
    F = np.fft.rfft(ring) / nlon[0]
    x, w = orc.gauss(2 * N)
    # F_m on ring 0 must equal sum_n a_n^m P_n^m(x_0)
    for m in range(mmax[0] + 1):
        P = orc.plm(m, T, x[0])
        sel = slice(inputs.coef_index(T, m, m), inputs.coef_index(T, T, m) + 1)
        ref = np.dot(a[0, sel, 0], P) + 1j * (np.dot(a[0, sel, 1], P) if m else 0)
        assert abs(F[m] - ref) < 1e-14 * max(1, abs(ref))


@pytest.mark.parametrize("kind,T,N", [(FULL, 15, 16), (OCT, 15, 16)])
def test_oracle_fp64_vs_long_double(orc, kind, T, N):
    a = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 1)
    g = orc.inverse(T, kind, N, a, deriv=True)
    gl = orc.inverse(T, kind, N, a, deriv=True, long_double=True)
    for u, v in zip(g, gl):
        assert relmax(u, v) < 1e-14
    b = orc.direct(T, kind, N, g[0])
    bl = orc.direct(T, kind, N, g[0], long_double=True)
    assert relmax(b, bl) < 1e-14


# --------------------------------------------------------------------------- uv
def test_solid_body_rotation(orc):
    """psi = -Omega sin(phi) gives u = Omega cos(phi), v = 0 exactly."""
    T, N, Om = 10, 11, 0.37
    nc = inputs.ncoef(T)
    vor = np.zeros((1, nc, 2))
    div = np.zeros((1, nc, 2))
    # sin(phi) = sqrt(2/3) P_1^0 ; zeta = -n(n+1) psi = 2 Omega sqrt(2/3)
    vor[0, inputs.coef_index(T, 1, 0), 0] = 2 * Om * math.sqrt(2 / 3)
    for kind in (OCT, FULL):
        phi, lam = grid_coords(orc, kind, N, T)
        u, v = orc.inverse_uv(T, kind, N, vor, div)
        assert np.abs(u[0] - Om * np.cos(phi)).max() < 1e-15
        assert np.abs(v[0]).max() < 1e-15
        z, d = orc.direct_uv(T, kind, N, u, v)
        assert np.abs(z - vor).max() < 4e-15 and np.abs(d).max() < 4e-15


@pytest.mark.parametrize("n,m", [(1, 1), (2, 0), (3, 2), (4, 1), (4, 4)])
def test_direct_uv_laplacian_eigenvalue(orc, n, m):
    """Winds built analytically from psi = Y_n^m (or chi = Y_n^m) give zeta (or D) =
    -n(n+1) at (n, m) and zero elsewhere."""
    T, N = 6, 7
    nc = inputs.ncoef(T)
    for kind in (OCT, FULL):
        phi, lam = grid_coords(orc, kind, N, T)
        c = 1.0 if m == 0 else 2.0
        p, dp = pbar_closed(n, m, phi), dpbar_dphi(n, m, phi)
        # psi: u = -d psi/d phi, v = (1/cos phi) d psi/d lambda
        u = -c * dp * np.cos(m * lam)
        v = -c * m * p * np.sin(m * lam) / np.cos(phi)
        z, d = orc.direct_uv(T, kind, N, u[None], v[None])
        ref = np.zeros((1, nc, 2))
        ref[0, inputs.coef_index(T, n, m), 0] = -n * (n + 1)
        assert np.abs(z - ref).max() < 1e-12 and np.abs(d).max() < 1e-12
        # chi: u = (1/cos phi) d chi/d lambda, v = d chi/d phi  -> D
        z, d = orc.direct_uv(T, kind, N, v[None], (-u)[None])
        assert np.abs(d - ref).max() < 1e-12 and np.abs(z).max() < 1e-12


def test_inverse_uv_then_direct_uv_identity(orc):
    T, N = 20, 21
    vor = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 11)
    div = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 12)
    vor[:, 0] = 0  # the n = 0 mode has no wind
    div[:, 0] = 0
    u, v = orc.inverse_uv(T, FULL, N, vor, div, radius=2.5)
    z, d = orc.direct_uv(T, FULL, N, u, v, radius=2.5)
    assert relmax(z, vor) < 1e-13 and relmax(d, div) < 1e-13


def test_inverse_uv_vs_derivatives(orc):
    """u cos(phi) = -cos(phi) dpsi/dphi + dchi/dlambda with psi, chi from the scalar inverse."""
    T, N = 12, 13
    vor = inputs.spectral_fields(T, 1, inputs.SEED_BASE + 5)
    div = inputs.spectral_fields(T, 1, inputs.SEED_BASE + 6)
    ns, _ = inputs.coef_nm(T)
    fac = np.where(ns > 0, -1.0 / np.maximum(ns * (ns + 1), 1), 0.0)[None, :, None]
    psi, chi = vor * fac, div * fac
    _, psil, psip = orc.inverse(T, OCT, N, psi, deriv=True)
    _, chil, chip = orc.inverse(T, OCT, N, chi, deriv=True)
    phi, _ = grid_coords(orc, OCT, N, T)
    u, v = orc.inverse_uv(T, OCT, N, vor, div)
    assert relmax(u, -psip + chil / np.cos(phi)) < 1e-13
    assert relmax(v, psil / np.cos(phi) + chip) < 1e-13


# --------------------------------------------------------------------- adjoints
def _spec_dot(a, b):
    # real inner product on (Re, Im) pairs without Im a_n^0 (m = 0 rows come first)
    return float(np.sum(a * b))


@pytest.mark.parametrize("kind", [OCT, FULL])
def test_adjoint_dot_products(orc, kind):
    T, N = 23, 24
    _, _, npts = orc.grid(kind, N, T)
    x = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 20)
    y = inputs.grid_values(npts, 2, inputs.SEED_BASE + 21)
    Ax = orc.inverse(T, kind, N, x)
    ATy = orc.inverse_adjoint(T, kind, N, y)
    lhs, rhs = float(np.sum(Ax * y)), _spec_dot(x, ATy)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    s = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 22)
    By = orc.direct(T, kind, N, y)
    BTs = orc.direct_adjoint(T, kind, N, s)
    lhs, rhs = _spec_dot(By, s), float(np.sum(y * BTs))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_brute_force_tiny(orc):
    """Columns of the inverse map by unit vectors give its matrix; its transpose must
    equal the adjoint applied to unit grid vectors."""
    T, N = 3, 4
    nc = inputs.ncoef(T)
    _, _, npts = orc.grid(OCT, N, T)
    ns, ms = inputs.coef_nm(T)
    cols = []
    for c in range(nc):
        for r in range(2):
            if r == 1 and ms[c] == 0:
                continue
            e = np.zeros((1, nc, 2))
            e[0, c, r] = 1
            cols.append(orc.inverse(T, OCT, N, e)[0])
    A = np.array(cols).T  # [npts][nspec]
    ATy = orc.inverse_adjoint(T, OCT, N, np.eye(npts))  # [npts][nc][2]
    mask = np.ones((nc, 2), bool)
    mask[ms == 0, 1] = False
    AT = ATy[:, mask]  # [npts][nspec]
    assert np.abs(AT - A).max() < 1e-13


def test_inverse_rings_matches_full_inverse(orc):
    """The ring-subset inverse returns exactly the full inverse's values on the
    selected rings (same code path, other rings skipped)."""
    T, N = 31, 32
    a = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 990)
    g, dl, dp = orc.inverse(T, 0, N, a, deriv=True)
    nlon, _, _ = orc.grid(0, N, T)
    off = np.concatenate([[0], np.cumsum(nlon)])
    rings = [0, 5, 31, 32, 63]
    gs, dls, dps = orc.inverse_rings(T, 0, N, a, rings, deriv=True)
    for k in rings:
        assert np.array_equal(gs[k], g[:, off[k]:off[k + 1]])
        assert np.array_equal(dls[k], dl[:, off[k]:off[k + 1]])
        assert np.array_equal(dps[k], dp[:, off[k]:off[k + 1]])


# ----------------------------------------------------- restricted variants
def test_restricted_variants_equal_the_full_routines(orc):
    """The wavenumber- and ring-restricted routines (used to check sampled
    outputs of the largest configurations) compute exactly what the full,
    pinned routines compute on the selected entries, and nothing elsewhere."""
    T, N = 31, 32
    a = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 11)
    b = inputs.spectral_fields(T, 2, inputs.SEED_BASE + 12)
    ns, ms = inputs.coef_nm(T)
    sel_m = [0, 1, 9, 10, 17, 31]
    pick = np.isin(ms, sel_m)
    g = orc.inverse(T, OCT, N, a)
    full = orc.direct(T, OCT, N, g)
    part = orc.direct_m(T, OCT, N, g, sel_m)
    assert np.array_equal(part[:, pick], full[:, pick])
    assert not part[:, ~pick].any()
    u, v = orc.inverse_uv(T, OCT, N, a, b)
    rings = [0, 5, 31, 32, 63]
    ur, vr = orc.inverse_uv_rings(T, OCT, N, a, b, rings)
    nlon, _, _ = orc.grid(OCT, N, T)
    off = np.concatenate([[0], np.cumsum(nlon)])
    for k in rings:
        assert np.array_equal(ur[k], u[:, off[k]:off[k + 1]])
        assert np.array_equal(vr[k], v[:, off[k]:off[k + 1]])
    zf, df = orc.direct_uv(T, OCT, N, u, v)
    zp, dp = orc.direct_uv_m(T, OCT, N, u, v, sel_m)
    assert np.array_equal(zp[:, pick], zf[:, pick]) and np.array_equal(dp[:, pick], df[:, pick])
    assert not zp[:, ~pick].any() and not dp[:, ~pick].any()
