"""GPU parity up the truncation ladder: TCo319 and TCo639, 4 fields.

The full inverse (grid of every ring) and the direct transform of the GPU's
own grid are compared element by element with the FP64 oracle, per field
max|x - x_ref| / max|x_ref|: 1e-12 for FP64, 1e-5 for FP32 and BF16X6.  The
oracle results are computed once per truncation and shared by the
precisions.  (TCo79-255 are covered by test_gpu_parity.py, TCo719 by
test_long_rings.py, TCo1279 by test_fullsize.py.)
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NF = 4
TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x6": 1e-5}
_REF = {}


def _ref(orc, T):
    if T not in _REF:
        a = inputs.spectral_fields(T, NF, inputs.SEED_BASE + 600 + T)
        _REF[T] = (a, orc.inverse(T, 0, T + 1, a))
    return _REF[T]


def _rel(x, ref):
    return max(float(np.abs(x[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in range(len(ref)))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x6"])
@pytest.mark.parametrize("T", [319, 639])
def test_inverse_and_direct_vs_oracle(orc, T, prec):
    from paper_1908_06097_gb300 import st

    a, g_ref = _ref(orc, T)
    p = st.Plan(T, NF, prec=prec)
    g = p.grid_empty()
    p.inv(torch.from_numpy(a).cuda(), g)
    s = p.spec_empty()
    p.dir(g, s)
    torch.cuda.synchronize()
    assert p.sync_status() == 0
    gh = g.cpu().numpy()
    e_inv = _rel(gh, g_ref)
    s_ref = orc.direct(T, 0, T + 1, gh)
    e_dir = _rel(s.cpu().numpy(), s_ref)
    p.close()
    assert e_inv <= TOL[prec] and e_dir <= TOL[prec], (e_inv, e_dir)
