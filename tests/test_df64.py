"""FP64 plans with double-float Legendre contractions (ST_FLAG_DF64).

The Legendre kernels stage the FP64 table and operands as pairs of FP32
values and accumulate in pairs (about 2^-47 per operation against FP64's
2^-53); everything else is the FP64 path.  Its error bound is the FP64 one
times 2^6, but what it reaches is the FP64 path's own error (the FP64
recurrences and FFTs dominate; at TCo1279 5.7e-13 against 5.4e-13), so it is
held to the FP64 gate of 1e-12, max-relative per field against the FP64
oracle.  The direct winds (vorticity, divergence), whose two terms cancel by
about 1e3 near the poles at m = 1, would make the path's own 2^-47 rounding
visible there; the kernels run the tiles of m <= 1 in FP64 for that reason,
and the winds are held to 1e-12 like every other output.  Checked here,
through the C ABI:
  - every transform against the oracle at truncations with one and several
    64-row tiles, ragged column tiles (odd field counts) and polar rings
    (TCo255);
  - agreement with the FP64 path (the same tables and FFTs), within the gate;
  - the adjoints against the oracle's;
  - the unsupported combinations are refused.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_DF = 1e-12


def _rel(x, ref):
    return max(float(np.abs(x[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in range(len(ref)))


@pytest.mark.parametrize("T,nfld", [(79, 3), (159, 5), (255, 2)])
def test_df64_matches_oracle(orc, T, nfld):
    from paper_1908_06097_gb300 import st

    N = T + 1
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 90 + T)
    b = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 91 + T)
    p = st.Plan(T, nfld, prec="fp64", flags=st.FLAG_DF64)
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    g, dl, dp = p.grid_empty(), p.grid_empty(), p.grid_empty()
    p.inv_deriv(ad, g, dl, dp)
    s = p.spec_empty()
    p.dir(g, s)
    u, v = p.grid_empty(), p.grid_empty()
    p.inv_uv(ad, bd, u, v)
    z, d = p.spec_empty(), p.spec_empty()
    p.dir_uv(u, v, z, d)
    torch.cuda.synchronize()
    assert p.sync_status() == 0
    g_ref, dl_ref, dp_ref = orc.inverse(T, 0, N, a, deriv=True)
    errs = {"grid": _rel(g.cpu().numpy(), g_ref), "dlam": _rel(dl.cpu().numpy(), dl_ref),
            "dphi": _rel(dp.cpu().numpy(), dp_ref)}
    s_ref = orc.direct(T, 0, N, g.cpu().numpy())
    errs["direct"] = _rel(s.cpu().numpy(), s_ref)
    u_ref, v_ref = orc.inverse_uv(T, 0, N, a, b)
    errs["u"] = _rel(u.cpu().numpy(), u_ref)
    errs["v"] = _rel(v.cpu().numpy(), v_ref)
    z_ref, d_ref = orc.direct_uv(T, 0, N, u.cpu().numpy(), v.cpu().numpy())
    errs["vor"] = _rel(z.cpu().numpy(), z_ref)
    errs["div"] = _rel(d.cpu().numpy(), d_ref)
    msg = ", ".join(f"{k} {v:.3g}" for k, v in errs.items())
    assert max(errs.values()) <= TOL_DF, msg
    p.close()


def test_df64_agrees_with_fp64_and_adjoints(orc):
    from paper_1908_06097_gb300 import st

    T, nfld = 200, 4
    N = T + 1
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 92)
    y = inputs.grid_values(inputs.octahedral_nlon(N).sum(), nfld, inputs.SEED_BASE + 93)
    ad, yd = torch.from_numpy(a).cuda(), torch.from_numpy(y).cuda()
    out = {}
    for name, flags in (("df", st.FLAG_DF64), ("fp64", 0)):
        p = st.Plan(T, nfld, prec="fp64", flags=flags)
        g = p.grid_empty()
        p.inv(ad, g)
        s = p.spec_empty()
        p.dir(g, s)
        ia = p.spec_empty()
        p.inv_adjoint(yd, ia)
        da = p.grid_empty()
        p.dir_adjoint(ad, da)
        torch.cuda.synchronize()
        assert p.sync_status() == 0
        out[name] = [x.cpu().numpy() for x in (g, s, ia, da)]
        p.close()
    for x, ref in zip(out["df"], out["fp64"]):
        assert _rel(x, ref) <= TOL_DF
    ia_ref = orc.inverse_adjoint(T, 0, N, y)
    da_ref = orc.direct_adjoint(T, 0, N, a)
    assert _rel(out["df"][2], ia_ref) <= TOL_DF
    assert _rel(out["df"][3], da_ref) <= TOL_DF


def test_df64_refusals():
    from paper_1908_06097_gb300 import st

    for prec, flags in (("fp32", st.FLAG_DF64), ("bf16x6", st.FLAG_DF64), ("fp64", st.FLAG_DF64 | st.FLAG_OTF)):
        with pytest.raises(st.StError) as e:
            st.Plan(79, 2, prec=prec, flags=flags)
        assert e.value.code == st.ST_ERR_UNSUPPORTED
    p = st.Plan(79, 2, prec="fp64", flags=st.FLAG_DF64)
    with pytest.raises(st.StError) as e:
        st.Group([p])
    assert e.value.code == st.ST_ERR_UNSUPPORTED
    p.close()
