"""GPU parity of the full-length ring transforms (8192 points, one per CTA).

From TCo680 on, the equatorial ring pairs need the largest chirp-z length,
8192 points, which fills a CTA of the FP32 kernels (also used by the split
paths).  Such a CTA holds a single transform, so no two fields share their
Fourier-row accesses there, unlike the shorter transforms of the other
tests.  TCo719 with 3 fields (an odd count, so the d/dphi half of the
operand starts at an odd column) runs them in both directions.
Element-by-element against the FP64 oracle, per field max-relative: 1e-5
for the grid, d/dphi and the direct spectra.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

T, NFLD = 719, 3
TOL = 1e-5
TOL_DPHI = {"fp32": 1e-5, "bf16x6": 1e-5}


def relmax_fields(x, ref):
    return max(np.abs(x[f] - ref[f]).max() / max(np.abs(ref[f]).max(), 1e-300) for f in range(ref.shape[0]))


@pytest.fixture(scope="module")
def case(orc):
    a = inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 719)
    g_ref, _, dp_ref = orc.inverse(T, 0, T + 1, a, deriv=True)
    s_ref = orc.direct(T, 0, T + 1, g_ref)
    return a, g_ref, dp_ref, s_ref


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_full_length_rings_vs_oracle(case, prec):
    from paper_1908_06097_gb300 import st

    st.load()
    a, g_ref, dp_ref, s_ref = case
    p = st.Plan(T, NFLD, prec=prec)
    # the equatorial ring pairs use the 8192-point transform
    assert max(p.nlon) + 2 * (T + 1) - 2 > 4096
    g, dp = p.grid_empty(), p.grid_empty()
    p.inv_deriv(torch.from_numpy(a).cuda(), g, None, dp)
    s = p.spec_empty()
    p.dir(torch.from_numpy(g_ref).cuda(), s)
    torch.cuda.synchronize()
    assert relmax_fields(g.cpu().numpy(), g_ref) < TOL
    assert relmax_fields(dp.cpu().numpy(), dp_ref) < TOL_DPHI[prec]
    assert relmax_fields(s.cpu().numpy(), s_ref) < TOL
    assert p.sync_status() == 0
    p.close()
