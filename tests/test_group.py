"""Grouped launches (st_group_*) and CUDA-graph capture.

A group runs the transforms of several plans (different truncations and
field counts) as one kernel launch per stage (FP64 groups add one launch per
member with polar rings, whose rows are recomputed in double-double).  Every member's result must be
bit-identical to the same plan's own transform: the kernels are the same and
each output element is produced by exactly one CTA, only the CTA order
differs.  A group call captured in a CUDA graph must replay to the same bits
with new input values in the captured buffers.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MEMBERS = [(79, 3), (159, 1), (47, 5), (79, 2), (31, 4)]  # (T, fields)


@pytest.fixture(scope="module")
def st():
    from paper_1908_06097_gb300 import st as _st

    _st.load()
    return _st


def _spectra(members, seed):
    return [torch.from_numpy(inputs.spectral_fields(T, nf, seed + 17 * i)).cuda() for i, (T, nf) in enumerate(members)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x6"])
def test_group_matches_plans_bitwise(st, prec):
    plans = [st.Plan(T, nf, prec=prec) for T, nf in MEMBERS]
    g = st.Group(plans)
    specs = _spectra(MEMBERS, inputs.SEED_BASE + 4)
    grids = [p.grid_empty() for p in plans]
    g.inv(specs, grids)
    # FP64: one more launch per member with polar rings (cos(phi) < 0.012),
    # whose Fourier rows are recomputed in double-double as by the plans
    npol = sum(1 for p in plans if np.sqrt(1 - p.latitudes()[0][0] ** 2) < 0.012) if prec == "fp64" else 0
    assert g.last_launches() == 3 + npol
    outs = [p.spec_empty() for p in plans]
    g.dir(grids, outs)
    # split precisions: the ring FFT writes the FP32 operand, one more kernel
    # splits it into the bf16 planes
    assert g.last_launches() == (4 if prec in ("bf16x3", "bf16x6") else 3)
    for p, a, gr, o in zip(plans, specs, grids, outs):
        gr_ref, o_ref = p.grid_empty(), p.spec_empty()
        p.inv(a, gr_ref)
        p.dir(gr_ref, o_ref)
        torch.cuda.synchronize()
        assert torch.equal(gr, gr_ref)
        assert torch.equal(o, o_ref)
        assert p.sync_status() == 0
    g.close()
    for p in plans:
        p.close()


def test_group_rejects_mixed_precision_and_null(st):
    p1, p2 = st.Plan(15, 1, prec="fp64"), st.Plan(15, 1, prec="fp32")
    with pytest.raises(st.StError):
        st.Group([p1, p2])
    g = st.Group([p1])
    lib = st.load()
    import ctypes

    nulls = (ctypes.c_void_p * 1)(None)
    s = p1.spec_empty()
    good = (ctypes.c_void_p * 1)(s.data_ptr())
    assert lib.st_group_inv(g._h, good, nulls, None) == st.ST_ERR_ARG
    assert lib.st_group_dir(g._h, nulls, good, None) == st.ST_ERR_ARG
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_group_cuda_graph_replay(st, prec):
    members = [(79, 4), (159, 2), (31, 3)]
    plans = [st.Plan(T, nf, prec=prec) for T, nf in members]
    g = st.Group(plans)
    specs = _spectra(members, inputs.SEED_BASE + 40)
    grids = [p.grid_empty() for p in plans]
    outs = [p.spec_empty() for p in plans]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):  # warm-up on the capture stream (first-call set-up)
        g.inv(specs, grids, stream)
        g.dir(grids, outs, stream)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        g.inv(specs, grids, stream)
        g.dir(grids, outs, stream)
    new = _spectra(members, inputs.SEED_BASE + 41)
    for a, b in zip(specs, new):
        a.copy_(b)
    graph.replay()
    torch.cuda.synchronize()
    for p, a, gr, o in zip(plans, new, grids, outs):
        gr_ref, o_ref = p.grid_empty(), p.spec_empty()
        p.inv(a, gr_ref)
        p.dir(gr_ref, o_ref)
        torch.cuda.synchronize()
        assert torch.equal(gr, gr_ref)
        assert torch.equal(o, o_ref)
    del graph
    g.close()
    for p in plans:
        p.close()


def test_plan_calls_capture_in_graph(st, orc):
    """A plan's inverse-with-derivatives call captured in a graph replays to the
    oracle's values for new inputs."""
    T, nf = 63, 2
    p = st.Plan(T, nf, prec="fp64")
    a = torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 50)).cuda()
    g, dp = p.grid_empty(), p.grid_empty()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        p.inv_deriv(a, g, None, dp, stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        p.inv_deriv(a, g, None, dp, stream)
    b = inputs.spectral_fields(T, nf, inputs.SEED_BASE + 51)
    a.copy_(torch.from_numpy(b))
    graph.replay()
    torch.cuda.synchronize()
    g_ref, _, dp_ref = orc.inverse(T, 0, T + 1, b, deriv=True)
    for f in range(nf):
        assert np.abs(g.cpu().numpy()[f] - g_ref[f]).max() <= 1e-12 * np.abs(g_ref[f]).max()
        assert np.abs(dp.cpu().numpy()[f] - dp_ref[f]).max() <= 1e-12 * np.abs(dp_ref[f]).max()
    del graph
    p.close()


GM = [(639, 3), (159, 2), (79, 4), (319, 1)]  # a TCo639 member among smaller ones
GM_RINGS = [0, 1, 97, 400, 639, 640, 1100, 1279]
GM_MS = [0, 1, 2, 45, 320, 638, 639]
GM_TOL = {"fp64": 1e-12, "bf16x6": 1e-5}


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_group_member_t639_vs_oracle(st, orc, prec):
    """The TCo639 member of a group against the oracle: its inverse on sampled
    rings (long-double oracle), and its direct transform of the group's own
    grid on sampled wavenumbers (FP64 oracle of the same grid), each relative
    to the field's largest sampled value."""
    plans = [st.Plan(T, nf, prec=prec) for T, nf in GM]
    g = st.Group(plans)
    specs = _spectra(GM, inputs.SEED_BASE + 60)
    grids = [p.grid_empty() for p in plans]
    outs = [p.spec_empty() for p in plans]
    g.inv(specs, grids)
    g.dir(grids, outs)
    torch.cuda.synchronize()
    T, nf = GM[0]
    a = specs[0].cpu().numpy()
    gh = grids[0].cpu().numpy()
    off = plans[0].ring_off
    ref = orc.inverse_rings(T, 0, T + 1, a, GM_RINGS, long_double=True)
    for f in range(nf):
        scale = max(np.abs(ref[k][f]).max() for k in GM_RINGS)
        err = max(np.abs(gh[f, off[k]:off[k + 1]] - ref[k][f]).max() for k in GM_RINGS) / scale
        assert err <= GM_TOL[prec], ("inverse", f, err)
    sref = orc.direct_m(T, 0, T + 1, gh, GM_MS)
    ns, ms = inputs.coef_nm(T)
    sel = np.isin(ms, GM_MS)
    got = outs[0].cpu().numpy()
    for f in range(nf):
        err = np.abs(got[f][sel] - sref[f][sel]).max() / np.abs(sref[f][sel]).max()
        assert err <= GM_TOL[prec], ("direct", f, err)
    for p in plans:
        assert p.sync_status() == 0
    g.close()
    for p in plans:
        p.close()
