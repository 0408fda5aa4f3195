"""FP64 plans with on-the-fly Legendre functions (ST_FLAG_OTF).

The Legendre kernels regenerate P_n^m by its recurrence instead of reading a
stored table; the direct kernel restarts the recurrence from checkpoints every
128 degrees.  Checked here, through the C ABI:
  - every transform of the plan against the FP64 oracle at 1e-12, at
    truncations below and above one checkpoint block (T+1 = 80, 160, 256),
    with field counts that leave ragged column tiles;
  - agreement with the stored-table FP64 path to rounding;
  - the plan holds no table (device memory);
  - the unsupported combinations are refused;
  - TCo1279: sampled rings of the inverse (and d/dphi) against the
    long-double oracle, and sampled wavenumbers of the direct transform of
    the GPU's grid against the oracle's direct transform of the same grid.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    return max(float(np.abs(x[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in range(len(ref)))


@pytest.mark.parametrize("T,nfld", [(79, 3), (159, 5), (255, 2)])
def test_otf_matches_oracle(orc, T, nfld):
    from paper_1908_06097_gb300 import st

    N = T + 1
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 60 + T)
    b = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 61 + T)
    p = st.Plan(T, nfld, prec="fp64", flags=st.FLAG_OTF)
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
    assert _rel(g.cpu().numpy(), g_ref) < 1e-12
    assert _rel(dl.cpu().numpy(), dl_ref) < 1e-12
    assert _rel(dp.cpu().numpy(), dp_ref) < 1e-12
    s_ref = orc.direct(T, 0, N, g.cpu().numpy())
    assert _rel(s.cpu().numpy(), s_ref) < 1e-12
    u_ref, v_ref = orc.inverse_uv(T, 0, N, a, b)
    assert _rel(u.cpu().numpy(), u_ref) < 1e-12
    assert _rel(v.cpu().numpy(), v_ref) < 1e-12
    z_ref, d_ref = orc.direct_uv(T, 0, N, u.cpu().numpy(), v.cpu().numpy())
    assert _rel(z.cpu().numpy(), z_ref) < 1e-12
    assert _rel(d.cpu().numpy(), d_ref) < 1e-12
    p.close()


def test_otf_agrees_with_stored_table_and_adjoints(orc):
    from paper_1908_06097_gb300 import st

    T, nfld = 200, 4
    a = torch.from_numpy(inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 62)).cuda()
    y = torch.from_numpy(inputs.grid_values(inputs.octahedral_nlon(T + 1).sum(), nfld, inputs.SEED_BASE + 63)).cuda()
    po = st.Plan(T, nfld, prec="fp64", flags=st.FLAG_OTF)
    ps = st.Plan(T, nfld, prec="fp64")
    out = {}
    for name, p in (("otf", po), ("stored", ps)):
        g = p.grid_empty()
        p.inv(a, g)
        s = p.spec_empty()
        p.dir(g, s)
        ia = p.spec_empty()
        p.inv_adjoint(y, ia)
        da = p.grid_empty()
        p.dir_adjoint(a, da)
        torch.cuda.synchronize()
        out[name] = [x.cpu().numpy() for x in (g, s, ia, da)]
    for x, r in zip(out["otf"], out["stored"]):
        assert _rel(x, r) < 1e-13
    ia_ref = orc.inverse_adjoint(T, 0, T + 1, y.cpu().numpy())
    assert _rel(out["otf"][2], ia_ref) < 1e-12
    po.close()
    ps.close()


def test_otf_plan_holds_no_table():
    from paper_1908_06097_gb300 import st

    T, nfld = 639, 1
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    po = st.Plan(T, nfld, prec="fp64", flags=st.FLAG_OTF)
    f1 = torch.cuda.mem_get_info()[0]
    ps = st.Plan(T, nfld, prec="fp64")
    f2 = torch.cuda.mem_get_info()[0]
    # the stored FP64 table at T=639 is 0.88 GB; the checkpoints are ~1/64 of it
    assert (f1 - f2) - (f0 - f1) > 0.7e9
    po.close()
    ps.close()


def test_otf_unsupported_combinations():
    from paper_1908_06097_gb300 import st

    with pytest.raises(st.StError) as e:
        st.Plan(31, 1, prec="bf16x6", flags=st.FLAG_OTF)
    assert e.value.code == st.ST_ERR_UNSUPPORTED
    p = st.Plan(31, 1, prec="fp64", flags=st.FLAG_OTF)
    with pytest.raises(st.StError) as e:
        st.Group([p])
    assert e.value.code == st.ST_ERR_UNSUPPORTED
    p.close()


def test_otf_full_size_sampled(orc):
    """TCo1279 (8 fields): inverse with d/dphi on sampled rings against the
    long-double oracle (d/dphi with the same polar allowance as the stored
    FP64 path: four times the FP64 oracle's own deviation), and the direct
    transform on sampled wavenumbers against the oracle's direct of the
    GPU's grid."""
    from paper_1908_06097_gb300 import st

    T, nfld = 1279, 8
    rings = [0, 1, 40, 320, 900, 1279, 1280, 1700, 2400, 2558, 2559]
    ms = [0, 1, 2, 37, 127, 128, 129, 320, 639, 1000, 1151, 1152, 1278, 1279]
    fields = [0, nfld - 1]
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 64)
    p = st.Plan(T, nfld, prec="fp64", flags=st.FLAG_OTF)
    g, dp = p.grid_empty(), p.grid_empty()
    p.inv_deriv(torch.from_numpy(a).cuda(), g, None, dp)
    s = p.spec_empty()
    p.dir(g, s)
    torch.cuda.synchronize()
    assert p.sync_status() == 0
    off = p.ring_off
    gh, dh, sh = g[fields].cpu().numpy(), dp[fields].cpu().numpy(), s.cpu().numpy()
    p.close()
    gl, _, dl = orc.inverse_rings(T, 0, T + 1, a[fields], rings, deriv=True, long_double=True)
    g8, _, d8 = orc.inverse_rings(T, 0, T + 1, a[fields], rings, deriv=True)
    for i in range(len(fields)):
        for x, ref, o64, name in ((gh, gl, g8, "grid"), (dh, dl, d8, "dphi")):
            scale = max(np.abs(ref[k][i]).max() for k in rings)
            err = max(np.abs(x[i, off[k]:off[k + 1]] - ref[k][i]).max() for k in rings) / scale
            e64 = max(np.abs(o64[k][i] - ref[k][i]).max() for k in rings) / scale
            assert err <= max(1e-12, 4 * e64), (name, i, err, e64)
    ref = orc.direct_m(T, 0, T + 1, gh, ms, long_double=True)
    ns, mm = inputs.coef_nm(T)
    pick = np.isin(mm, ms)
    for i, f in enumerate(fields):
        err = np.abs(sh[f][pick] - ref[i][pick]).max() / np.abs(ref[i][pick]).max()
        assert err <= 1e-12, (f, err)
