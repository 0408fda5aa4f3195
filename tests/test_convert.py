"""The library's integer-only float/double conversions against the hardware.

The ring FFTs and the spectral kernels convert between FP64 I/O and FP32
arithmetic with integer operations (dbl2flt_rn, to_dbl) instead of the narrow
FP64 pipe.  Through the C-ABI self-test hook, every value here must convert
bit for bit as the GPU's own round-to-nearest-even conversion does (torch's
.float() / .double() on the device): ties, the subnormal range, the overflow
boundary, infinities and NaN (compared as NaN), signed zeros.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _edge_values():
    f32 = np.finfo(np.float32)
    vals = []
    for x in [1.0, 1.5, 3.1, 2.0**-126, 2.0**-127, 2.0**-140, 2.0**-149, 3 * 2.0**-149, 2.0**-150, 1.5 * 2.0**-150,
              2.0**-151, float(f32.max), 2.0**127, 65504.0, 1e-40]:
        xf = np.float32(x)
        with np.errstate(over="ignore"):  # the step above FLT_MAX is inf, replaced below
            up = np.nextafter(xf, np.float32(np.inf))
        if not np.isfinite(up):
            up = np.float64(f32.max) + 2.0**103  # one float ulp above FLT_MAX, in double
        mid = (float(xf) + float(up)) / 2
        for v in [float(xf), mid, np.nextafter(mid, 0.0), np.nextafter(mid, np.inf), float(up)]:
            vals += [v, -v]
    vals += [0.0, -0.0, np.inf, -np.inf, np.nan, 1e300, -1e300, 1e-300, 5e-324, 3 * 2.0**-1074]
    rng = np.random.default_rng(7)
    vals += list(rng.standard_normal(50000) * 10.0 ** rng.uniform(-50, 40, 50000))
    vals += list(rng.uniform(-1, 1, 50000) * 2.0 ** rng.uniform(-155, -120, 50000))
    return np.array(vals, dtype=np.float64)


def test_conversions_match_hardware():
    from paper_1908_06097_gb300 import st

    lib = st.load()
    x = torch.from_numpy(_edge_values()).cuda()
    n = x.numel()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    back = torch.empty(n, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.st_debug_convert(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(back.data_ptr()), n, s) == 0
    ref = x.float()
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(out), nan)
    o, r = out[~nan].view(torch.int32), ref[~nan].view(torch.int32)
    bad = (o != r).nonzero()
    assert bad.numel() == 0, (x[~nan][bad[:5, 0]].tolist(), o[bad[:5, 0]].tolist(), r[bad[:5, 0]].tolist())
    ref_back = out.double()
    assert torch.equal(torch.isnan(back), torch.isnan(ref_back))
    keep = ~torch.isnan(ref_back)
    assert torch.equal(back[keep].view(torch.int64), ref_back[keep].view(torch.int64))
    assert lib.st_debug_convert(None, None, None, 1, None) == st.ST_ERR_ARG
