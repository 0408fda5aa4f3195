"""The allocation-free inverse transform (st_inv_transform_noalloc).

Callers that cannot allocate device memory while they transform (code under
an allocator hook, a frozen memory pool) get an inverse transform whose
scratch lives in a static device array.  Called through the C ABI:
  - it matches st_inv_transform and the FP64 oracle on two calls in a row;
  - two plans of different shapes alternate on the shared array, after a
    call that filled the array with NaN (a transform of NaN inputs): a call
    that read any scratch element it had not written would return NaN;
  - after the first call (set-up) a call allocates no device memory;
  - plans whose scratch does not fit the array are rejected.
This file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1908_06097_gb300 import st

    lib = st.load()
    lib.st_inv_transform_noalloc.argtypes = [ctypes.c_void_p] * 4
    return lib


def _noalloc(lib, p, a, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.st_inv_transform_noalloc(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        stream)


def _rel(x, ref):
    return max(float(np.abs(x[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in range(len(ref)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_matches_inverse_twice(prec, tol):
    from paper_1908_06097_gb300 import st

    lib = _lib()
    T, nfld = 79, 10
    p = st.Plan(T, nfld, prec=prec)
    for call in range(2):
        a = torch.from_numpy(inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 900 + call)).cuda()
        ref = p.grid_empty()
        out = torch.full_like(ref, float("nan"))
        p.inv(a, ref)
        assert _noalloc(lib, p, a, out) == 0, st.last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        for f in range(nfld):
            assert np.abs(o[f] - r[f]).max() <= tol * np.abs(r[f]).max()
    assert p.sync_status() == 0
    p.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_two_shapes_over_poisoned_scratch(orc, prec, tol):
    from paper_1908_06097_gb300 import st

    lib = _lib()
    shapes = [(79, 10), (47, 7)]
    plans = [st.Plan(T, nf, prec=prec) for T, nf in shapes]
    ins = [inputs.spectral_fields(T, nf, inputs.SEED_BASE + 910 + T) for T, nf in shapes]
    refs = [orc.inverse(T, 0, T + 1, a) for (T, nf), a in zip(shapes, ins)]
    dev = [torch.from_numpy(a).cuda() for a in ins]
    outs = [p.grid_empty() for p in plans]
    # set-up call, then NaN through the larger plan: its operand and Fourier
    # rows in the array become NaN
    assert _noalloc(lib, plans[0], dev[0], outs[0]) == 0, st.last_error()
    nan_in = torch.full_like(dev[0], float("nan"))
    assert _noalloc(lib, plans[0], nan_in, outs[0]) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(4):
        i = (call + 1) % 2  # the smaller plan first, over the NaN left by the larger one
        outs[i].fill_(float("nan"))
        assert _noalloc(lib, plans[i], dev[i], outs[i]) == 0, st.last_error()
        torch.cuda.synchronize()
        got = outs[i].cpu().numpy()
        assert np.isfinite(got).all(), (call, shapes[i])
        assert _rel(got, refs[i]) < tol, (call, shapes[i])
    # nothing was allocated by these calls
    assert torch.cuda.mem_get_info()[0] == free0
    for p in plans:
        assert p.sync_status() == 0
        p.close()


def test_noalloc_rejects_oversized_and_split_plans():
    from paper_1908_06097_gb300 import st

    lib = _lib()
    p = st.Plan(319, 20, prec="fp64")
    a, g = p.spec_empty(), p.grid_empty()
    rc = lib.st_inv_transform_noalloc(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert rc == st.ST_ERR_ARG
    assert "static" in st.last_error()
    p.close()
    q = st.Plan(31, 2, prec="bf16x6")
    a, g = q.spec_empty(), q.grid_empty()
    rc = lib.st_inv_transform_noalloc(q.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert rc == st.ST_ERR_UNSUPPORTED
    q.close()
