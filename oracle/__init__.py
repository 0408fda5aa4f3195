"""CPU oracle of the spherical-harmonic transform (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never loads it, and it imports nothing from the product.

``st_oracle.c`` holds the plain FP64 definitions (see its header); this file
compiles it with gcc (OpenMP) into ``_st_oracle.so`` and a long-double build
``_st_oracle_ld.so``, and marshals numpy arrays through ctypes.

Arrays: spectral float64 [nfld][ncoef][2] (m-major, n = m..T); grid float64
[nfld][npts], rings north -> south.  ``kind`` 0 = octahedral (ring i from the
pole has 4i+16 points), 1 = full Gaussian (4N points per ring).
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "st_oracle.c")
_LIBS = {False: os.path.join(_HERE, "_st_oracle.so"), True: os.path.join(_HERE, "_st_oracle_ld.so")}
_cache = {}

OCTAHEDRAL = 0
FULL_GAUSSIAN = 1


def build(force=False):
    """Compile both oracle builds (FP64 and long double) with gcc + OpenMP."""
    for ld, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", out + ".tmp", _SRC, "-lm"]
        if ld:
            cmd.insert(1, "-DORACLE_LONG_DOUBLE")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


def _lib(long_double=False):
    if long_double not in _cache:
        build()
        lib = ctypes.CDLL(_LIBS[long_double])
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_grid.argtypes = [i, i, i, ip, ip]
        lib.or_grid.restype = ctypes.c_long
        lib.or_gauss.argtypes = [i, d, d]
        lib.or_plm.argtypes = [i, i, ctypes.c_double, d]
        lib.or_hlm.argtypes = [i, i, ctypes.c_double, d]
        lib.or_inverse.argtypes = [i, i, i, i, d, d, d, d]
        lib.or_inverse_rings.argtypes = [i, i, i, i, d, d, d, d, ctypes.c_void_p]
        lib.or_direct.argtypes = [i, i, i, i, d, d]
        lib.or_direct_m.argtypes = [i, i, i, i, d, d, ctypes.c_void_p]
        lib.or_inverse_uv_rings.argtypes = [i, i, i, i, ctypes.c_double, d, d, d, d, ctypes.c_void_p]
        lib.or_direct_uv_m.argtypes = [i, i, i, i, ctypes.c_double, d, d, d, d, ctypes.c_void_p]
        lib.or_inverse_uv.argtypes = [i, i, i, i, ctypes.c_double, d, d, d, d]
        lib.or_direct_uv.argtypes = [i, i, i, i, ctypes.c_double, d, d, d, d]
        lib.or_inverse_adjoint.argtypes = [i, i, i, i, d, d]
        lib.or_direct_adjoint.argtypes = [i, i, i, i, d, d]
        lib.or_roundtrip_defect.argtypes = [i, i, i, d]
        lib.or_roundtrip_defect.restype = ctypes.c_double
        lib.or_num_threads.restype = ctypes.c_int
        _cache[long_double] = lib
    return _cache[long_double]


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def ncoef(T):
    return (T + 1) * (T + 2) // 2


def grid(kind, N, T):
    """(nlon, mmax, npts) of the 2N rings."""
    nlon = (ctypes.c_int * (2 * N))()
    mmax = (ctypes.c_int * (2 * N))()
    npts = _lib().or_grid(kind, N, T, nlon, mmax)
    return np.array(nlon, dtype=np.int64), np.array(mmax, dtype=np.int64), int(npts)


def gauss(nlat, long_double=False):
    """Gauss-Legendre nodes (descending, north first) and weights."""
    x = np.zeros(nlat)
    w = np.zeros(nlat)
    _check(_lib(long_double).or_gauss(nlat, _p(x), _p(w)), "gauss")
    return x, w


def plm(m, nmax, x, long_double=False):
    """P_n^m(x) for n = m..nmax (orthonormal, no Condon-Shortley phase)."""
    out = np.zeros(nmax - m + 1)
    _check(_lib(long_double).or_plm(m, nmax, float(x), _p(out)), "plm")
    return out


def hlm(m, nmax, x, long_double=False):
    """H_n^m(x) = (1-x^2) dP_n^m/dx for n = m..nmax."""
    out = np.zeros(nmax - m + 1)
    _check(_lib(long_double).or_hlm(m, nmax, float(x), _p(out)), "hlm")
    return out


def inverse(T, kind, N, spec, deriv=False, long_double=False):
    """spec [nfld][ncoef][2] -> grid [nfld][npts] (and d/dlambda, d/dphi if deriv)."""
    spec = np.ascontiguousarray(spec, dtype=np.float64)
    nfld = spec.shape[0]
    npts = grid(kind, N, T)[2]
    out = np.zeros((nfld, npts))
    dl = np.zeros((nfld, npts)) if deriv else None
    dp = np.zeros((nfld, npts)) if deriv else None
    _check(_lib(long_double).or_inverse(T, kind, N, nfld, _p(spec), _p(out), _p(dl), _p(dp)), "inverse")
    return (out, dl, dp) if deriv else out


def inverse_rings(T, kind, N, spec, rings, deriv=False, long_double=False):
    """``inverse`` evaluated on the listed rings only: returns {ring: values}
    (and the d/dlambda, d/dphi dicts if deriv), each [nfld][nlon]."""
    spec = np.ascontiguousarray(spec, dtype=np.float64)
    nfld = spec.shape[0]
    nlon, _, npts = grid(kind, N, T)
    off = np.concatenate([[0], np.cumsum(nlon)])
    sel = np.zeros(2 * N, dtype=np.uint8)
    sel[list(rings)] = 1
    out = np.zeros((nfld, npts))
    dl = np.zeros((nfld, npts)) if deriv else None
    dp = np.zeros((nfld, npts)) if deriv else None
    _check(_lib(long_double).or_inverse_rings(T, kind, N, nfld, _p(spec), _p(out), _p(dl), _p(dp),
                                              sel.ctypes.data_as(ctypes.c_void_p)), "inverse_rings")
    pick = lambda a: {k: a[:, off[k]:off[k + 1]].copy() for k in rings}
    return (pick(out), pick(dl), pick(dp)) if deriv else pick(out)


def direct(T, kind, N, g, long_double=False):
    """grid [nfld][npts] -> spec [nfld][ncoef][2]."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    nfld = g.shape[0]
    out = np.zeros((nfld, ncoef(T), 2))
    _check(_lib(long_double).or_direct(T, kind, N, nfld, _p(g), _p(out)), "direct")
    return out


def _mask(n, idx):
    sel = np.zeros(n, dtype=np.uint8)
    sel[list(idx)] = 1
    return sel


def direct_m(T, kind, N, g, ms, long_double=False):
    """``direct`` for the wavenumbers in ms only: returns spec [nfld][ncoef][2]
    with the coefficients of every other m set to 0."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros((g.shape[0], ncoef(T), 2))
    sel = _mask(T + 1, ms)
    _check(_lib(long_double).or_direct_m(T, kind, N, g.shape[0], _p(g), _p(out),
                                         sel.ctypes.data_as(ctypes.c_void_p)), "direct_m")
    return out


def inverse_uv_rings(T, kind, N, vor, div, rings, radius=1.0, long_double=False):
    """``inverse_uv`` on the listed rings only: ({ring: u}, {ring: v}), each [nfld][nlon]."""
    vor = np.ascontiguousarray(vor, dtype=np.float64)
    div = np.ascontiguousarray(div, dtype=np.float64)
    nfld = vor.shape[0]
    nlon, _, npts = grid(kind, N, T)
    off = np.concatenate([[0], np.cumsum(nlon)])
    u = np.zeros((nfld, npts))
    v = np.zeros((nfld, npts))
    sel = _mask(2 * N, rings)
    _check(_lib(long_double).or_inverse_uv_rings(T, kind, N, nfld, radius, _p(vor), _p(div), _p(u), _p(v),
                                                 sel.ctypes.data_as(ctypes.c_void_p)), "inverse_uv_rings")
    pick = lambda a: {k: a[:, off[k]:off[k + 1]].copy() for k in rings}
    return pick(u), pick(v)


def direct_uv_m(T, kind, N, u, v, ms, radius=1.0, long_double=False):
    """``direct_uv`` for the wavenumbers in ms only (other coefficients 0)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    nfld = u.shape[0]
    vor = np.zeros((nfld, ncoef(T), 2))
    div = np.zeros((nfld, ncoef(T), 2))
    sel = _mask(T + 1, ms)
    _check(_lib(long_double).or_direct_uv_m(T, kind, N, nfld, radius, _p(u), _p(v), _p(vor), _p(div),
                                            sel.ctypes.data_as(ctypes.c_void_p)), "direct_uv_m")
    return vor, div


def inverse_uv(T, kind, N, vor, div, radius=1.0, long_double=False):
    """(vorticity, divergence) spectra -> (u, v) grid fields."""
    vor = np.ascontiguousarray(vor, dtype=np.float64)
    div = np.ascontiguousarray(div, dtype=np.float64)
    nfld = vor.shape[0]
    npts = grid(kind, N, T)[2]
    u = np.zeros((nfld, npts))
    v = np.zeros((nfld, npts))
    _check(_lib(long_double).or_inverse_uv(T, kind, N, nfld, radius, _p(vor), _p(div), _p(u), _p(v)),
           "inverse_uv")
    return u, v


def direct_uv(T, kind, N, u, v, radius=1.0, long_double=False):
    """(u, v) grid fields -> (vorticity, divergence) spectra."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    nfld = u.shape[0]
    vor = np.zeros((nfld, ncoef(T), 2))
    div = np.zeros((nfld, ncoef(T), 2))
    _check(_lib(long_double).or_direct_uv(T, kind, N, nfld, radius, _p(u), _p(v), _p(vor), _p(div)),
           "direct_uv")
    return vor, div


def inverse_adjoint(T, kind, N, grid_cot, long_double=False):
    """Transpose of ``inverse``: grid cotangent -> spectral cotangent."""
    g = np.ascontiguousarray(grid_cot, dtype=np.float64)
    out = np.zeros((g.shape[0], ncoef(T), 2))
    _check(_lib(long_double).or_inverse_adjoint(T, kind, N, g.shape[0], _p(g), _p(out)), "inverse_adjoint")
    return out


def direct_adjoint(T, kind, N, spec_cot, long_double=False):
    """Transpose of ``direct``: spectral cotangent -> grid cotangent."""
    s = np.ascontiguousarray(spec_cot, dtype=np.float64)
    npts = grid(kind, N, T)[2]
    out = np.zeros((s.shape[0], npts))
    _check(_lib(long_double).or_direct_adjoint(T, kind, N, s.shape[0], _p(s), _p(out)), "direct_adjoint")
    return out


def roundtrip_defect(T, kind, N):
    """(max_m E_m, E_m array): quadrature defect of the rings each m skips."""
    em = np.zeros(T + 1)
    e = _lib().or_roundtrip_defect(T, kind, N, _p(em))
    return e, em


def num_threads():
    return int(_lib().or_num_threads())
