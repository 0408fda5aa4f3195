"""Seeded synthetic inputs for the spectral-transform dwarf.

This module is the only code shared by the CUDA path's tests/benchmarks and
the CPU oracle.  It holds the input recipe and the storage layout of the
arrays, and none of the transform's arithmetic.

Recipe (the spectral fields of the dwarf's test cases, Sec. 3.1.4 TCo639 and
the TCo1279/TCo1999 resolutions of Sec. 3.2.2, which the paper names without
giving their data):

* spectral coefficient a_n^m = (g1 + i g2) / sqrt(2) * (n + 1)^-1.5 with
  g1, g2 standard normals drawn from ``numpy.random.Generator(PCG64(seed))``
  in [field][coef][re, im] order; Im a_n^0 = 0 because the fields are real;
* grid values (adjoint / cotangent inputs) are standard normals from the same
  generator family.

Layouts (the library's I/O convention):

* spectral: float64 [nfld][ncoef][2], m-major: m = 0..T, then n = m..T,
  ncoef = (T+1)(T+2)/2;
* grid: float64 [nfld][npts], rings north -> south, each from lambda = 0
  eastward.
"""

import numpy as np

SEED_BASE = 1908060970


def ncoef(T):
    """Number of triangular-truncation coefficients, (T+1)(T+2)/2."""
    return (T + 1) * (T + 2) // 2


def coef_nm(T):
    """(n, m) of every coefficient in the m-major storage order."""
    ms = np.concatenate([np.full(T + 1 - m, m, dtype=np.int64) for m in range(T + 1)])
    ns = np.concatenate([np.arange(m, T + 1, dtype=np.int64) for m in range(T + 1)])
    return ns, ms


def coef_index(T, n, m):
    """Storage index of (n, m): m(2T+3-m)/2 + (n - m)."""
    return m * (2 * T + 3 - m) // 2 + (n - m)


def spectral_fields(T, nfld, seed, slope=-1.5):
    """Seeded complex-Gaussian coefficients scaled by (n+1)^slope."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((nfld, ncoef(T), 2))
    ns, ms = coef_nm(T)
    a = g / np.sqrt(2.0) * ((ns + 1.0) ** slope)[None, :, None]
    a[:, ms == 0, 1] = 0.0
    return np.ascontiguousarray(a)


def grid_values(npts, nfld, seed):
    """Seeded standard-normal grid fields [nfld][npts]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.standard_normal((nfld, npts)))


def octahedral_nlon(N):
    """Ring lengths of the octahedral grid O(N), north -> south.

    The northern ring i (1..N from the pole) has 4i + 16 points; the southern
    hemisphere mirrors it.  This is the grid definition, not transform
    arithmetic, and both sides may use it to size their arrays.
    """
    north = 4 * np.arange(1, N + 1, dtype=np.int64) + 16
    return np.concatenate([north, north[::-1]])


def full_gaussian_nlon(N):
    """Ring lengths of the full (regular) Gaussian grid: 4N points on every ring."""
    return np.full(2 * N, 4 * N, dtype=np.int64)
