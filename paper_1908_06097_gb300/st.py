"""Python binding of the C-ABI spectral-transform library (libst_gb300.so).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  Tensors are float64 CUDA tensors in the layouts of
include/st.h (spectral [nfld, ncoef, 2], grid [nfld, npts]); calls enqueue on
torch's current CUDA stream.  There is no CPU fallback: importing this module
without the built library raises.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libst_gb300.so")

ST_OK, ST_ERR_ARG, ST_ERR_CUDA, ST_ERR_NOMEM, ST_ERR_UNSUPPORTED, ST_ERR_TIMEOUT, ST_ERR_CHECK = range(7)
OCTAHEDRAL, FULL_GAUSSIAN = 0, 1
FP64, FP32, BF16X3, BF16X6 = 0, 1, 2, 3
FLAG_AUTOTUNE = 1
FLAG_STAGE_TIMING = 2
FLAG_CHECKS = 4
FLAG_OTF = 8
FLAG_DF64 = 16
STAGES = ["pre", "leg_inv", "c2r", "r2c", "leg_dir", "post"]

_PREC_NAMES = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3, "bf16x6": BF16X6}


class StError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"st error {code}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("N", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("radius", ctypes.c_double), ("flags", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


_lib = None

# exported names of include/st.h
EXPORTS = ["st_plan_create", "st_plan_destroy", "st_plan_info", "st_plan_latitudes", "st_inv_transform",
           "st_dir_transform", "st_inv_transform_deriv", "st_inv_transform_uv", "st_dir_transform_uv",
           "st_inv_adjoint", "st_dir_adjoint", "st_group_create", "st_group_inv", "st_group_dir",
           "st_group_destroy", "st_group_last_launches", "st_sync_status", "st_last_error",
           "st_plan_last_launches", "st_plan_stage_times", "st_plan_tuning", "st_inv_transform_noalloc",
           "st_plan_set_wait_limit", "st_debug_fail_alloc", "st_debug_corrupt_worklist", "st_debug_poison_workspaces",
           "st_plan_set_partition", "st_exchange_counts", "st_exchange_pack", "st_exchange_unpack",
           "st_inv_legendre", "st_inv_fourier", "st_dir_fourier", "st_dir_legendre", "st_debug_convert"]


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libst_gb300.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i = ctypes.c_int
    lib.st_plan_create.argtypes = [ctypes.POINTER(vp), i, _Grid, i, ctypes.POINTER(_Opts)]
    lib.st_plan_destroy.argtypes = [vp]
    lib.st_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                 ctypes.POINTER(i), ctypes.POINTER(ctypes.POINTER(i)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_long))]
    lib.st_plan_latitudes.argtypes = [vp, vp, vp]
    for name, n in [("st_inv_transform", 3), ("st_dir_transform", 3), ("st_inv_adjoint", 3),
                    ("st_dir_adjoint", 3), ("st_inv_transform_deriv", 5), ("st_inv_transform_uv", 5),
                    ("st_dir_transform_uv", 5)]:
        getattr(lib, name).argtypes = [vp] * (n + 1)
    lib.st_group_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i]
    lib.st_group_inv.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.st_group_dir.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.st_group_destroy.argtypes = [vp]
    lib.st_group_last_launches.argtypes = [vp]
    lib.st_inv_transform_noalloc.argtypes = [vp] * 4
    lib.st_sync_status.argtypes = [vp]
    lib.st_last_error.restype = ctypes.c_char_p
    lib.st_plan_last_launches.argtypes = [vp]
    lib.st_plan_tuning.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.st_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long), i]
    lib.st_plan_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.st_debug_fail_alloc.argtypes = [i]
    lib.st_debug_corrupt_worklist.argtypes = [vp, i]
    lib.st_debug_poison_workspaces.argtypes = [vp, vp]
    lib.st_plan_set_partition.argtypes = [vp, i, i, vp, vp]
    lib.st_exchange_counts.argtypes = [vp, i, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                       ctypes.POINTER(i)]
    lib.st_exchange_pack.argtypes = [vp, i, vp, vp]
    lib.st_exchange_unpack.argtypes = [vp, i, vp, vp]
    for name in ("st_inv_legendre", "st_inv_fourier", "st_dir_fourier", "st_dir_legendre"):
        getattr(lib, name).argtypes = [vp, vp, vp]
    lib.st_debug_convert.argtypes = [vp, vp, vp, ctypes.c_long, vp]
    if path == _LIB_PATH:
        _lib = lib
    return lib


def last_error():
    return load().st_last_error().decode()


def _check(rc):
    if rc != ST_OK:
        raise StError(rc, last_error())


def _ptr(t):
    if t is None:
        return None
    import torch

    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A transform plan: truncation T, grid (kind, N), nfld fields per call."""

    def __init__(self, T, nfld, N=None, kind=OCTAHEDRAL, prec="fp64", radius=1.0, flags=0, tune_cache=None):
        lib = load()
        self.T, self.nfld = T, nfld
        self.N = N if N is not None else T + 1
        self.kind = kind
        self.prec = _PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
        h = ctypes.c_void_p()
        opts = _Opts(self.prec, radius, flags, tune_cache.encode() if tune_cache else None)
        _check(lib.st_plan_create(ctypes.byref(h), T, _Grid(kind, self.N), nfld, ctypes.byref(opts)))
        self._h = h
        npts, ncoef, nlat = ctypes.c_long(), ctypes.c_long(), ctypes.c_int()
        nlon_p = ctypes.POINTER(ctypes.c_int)()
        roff_p = ctypes.POINTER(ctypes.c_long)()
        _check(lib.st_plan_info(h, ctypes.byref(npts), ctypes.byref(ncoef), ctypes.byref(nlat),
                                ctypes.byref(nlon_p), ctypes.byref(roff_p)))
        self.npts, self.ncoef, self.nlat = npts.value, ncoef.value, nlat.value
        self.nlon = np.array(nlon_p[: self.nlat], dtype=np.int64)
        self.ring_off = np.array(roff_p[: self.nlat + 1], dtype=np.int64)

    @property
    def handle(self):
        return self._h

    def latitudes(self):
        mu = np.zeros(self.nlat)
        w = np.zeros(self.nlat)
        _check(load().st_plan_latitudes(self._h, mu.ctypes.data_as(ctypes.c_void_p),
                                        w.ctypes.data_as(ctypes.c_void_p)))
        return mu, w

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().st_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- transforms (outputs are written in place) -------------------------
    def inv(self, spec, grid, stream=None):
        _check(load().st_inv_transform(self._h, _ptr(spec), _ptr(grid), _stream(stream)))

    def dir(self, grid, spec, stream=None):
        _check(load().st_dir_transform(self._h, _ptr(grid), _ptr(spec), _stream(stream)))

    def inv_deriv(self, spec, grid=None, dlam=None, dphi=None, stream=None):
        _check(load().st_inv_transform_deriv(self._h, _ptr(spec), _ptr(grid), _ptr(dlam), _ptr(dphi),
                                             _stream(stream)))

    def inv_uv(self, vor, div, u, v, stream=None):
        _check(load().st_inv_transform_uv(self._h, _ptr(vor), _ptr(div), _ptr(u), _ptr(v), _stream(stream)))

    def dir_uv(self, u, v, vor, div, stream=None):
        _check(load().st_dir_transform_uv(self._h, _ptr(u), _ptr(v), _ptr(vor), _ptr(div), _stream(stream)))

    def inv_adjoint(self, grid_cot, spec_cot, stream=None):
        _check(load().st_inv_adjoint(self._h, _ptr(grid_cot), _ptr(spec_cot), _stream(stream)))

    def dir_adjoint(self, spec_cot, grid_cot, stream=None):
        _check(load().st_dir_adjoint(self._h, _ptr(spec_cot), _ptr(grid_cot), _stream(stream)))

    def sync_status(self):
        return load().st_sync_status(self._h)

    def last_launches(self):
        return load().st_plan_last_launches(self._h)

    def set_wait_limit(self, clocks):
        """Bound (SM clocks) of the tensor-core kernels' waits; 0 = default."""
        _check(load().st_plan_set_wait_limit(self._h, int(clocks)))

    def tuning(self):
        """(inverse, direct) Legendre tile widths: defaults or the autotuner's choice."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().st_plan_tuning(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def stage_times(self):
        """(ms, launches) per stage since the last call (plan made with FLAG_STAGE_TIMING)."""
        ms = (ctypes.c_double * 6)()
        n = (ctypes.c_long * 6)()
        _check(load().st_plan_stage_times(self._h, ms, n, 6))
        return list(ms), list(n)

    # -- allocation helpers ---------------------------------------------------
    def spec_empty(self, nfld=None, device="cuda"):
        import torch

        return torch.empty((nfld or self.nfld, self.ncoef, 2), dtype=torch.float64, device=device)

    def grid_empty(self, nfld=None, device="cuda"):
        import torch

        return torch.empty((nfld or self.nfld, self.npts), dtype=torch.float64, device=device)


class Group:
    """Several plans whose stages each run as one grouped kernel launch."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(load().st_group_create(ctypes.byref(h), arr, len(self.plans)))
        self._h = h

    def _arrs(self, xs):
        return (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])

    def inv(self, specs, grids, stream=None):
        _check(load().st_group_inv(self._h, self._arrs(specs), self._arrs(grids), _stream(stream)))

    def dir(self, grids, specs, stream=None):
        _check(load().st_group_dir(self._h, self._arrs(grids), self._arrs(specs), _stream(stream)))

    def last_launches(self):
        return load().st_group_last_launches(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().st_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
