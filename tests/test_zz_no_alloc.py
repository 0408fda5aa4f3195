"""The allocation-free inverse transform (st_inv_transform_noalloc).

Callers that cannot allocate device memory while they transform get an
inverse transform whose scratch lives in a static device array.  Called
through the C ABI, it must reproduce st_inv_transform on two calls in a row:
the second call reuses the array the first one left behind.  It also rejects
plans whose scratch does not fit the array.  This file is named so that pytest
collects it last.
"""

import ctypes

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_matches_inverse_twice(prec, tol):
    from paper_1908_06097_gb300 import st

    lib = st.load()
    lib.st_inv_transform_noalloc.argtypes = [ctypes.c_void_p] * 4
    T, nfld = 79, 10
    p = st.Plan(T, nfld, prec=prec)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        a = torch.from_numpy(inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 900 + call)).cuda()
        ref = p.grid_empty()
        out = torch.full_like(ref, float("nan"))
        p.inv(a, ref)
        rc = lib.st_inv_transform_noalloc(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          stream)
        assert rc == 0, st.last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        for f in range(nfld):
            assert np.abs(o[f] - r[f]).max() <= tol * np.abs(r[f]).max()
    assert p.sync_status() == 0
    p.close()


def test_noalloc_rejects_oversized_plan():
    from paper_1908_06097_gb300 import st

    lib = st.load()
    lib.st_inv_transform_noalloc.argtypes = [ctypes.c_void_p] * 4
    p = st.Plan(319, 20, prec="fp64")
    a, g = p.spec_empty(), p.grid_empty()
    rc = lib.st_inv_transform_noalloc(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert rc == st.ST_ERR_ARG
    assert "static" in st.last_error()
    p.close()
