"""NaN canaries in the workspaces.

Before every transform the plan's workspaces that each call rewrites (the
Fourier buffer / direct operand, the inverse operand / direct result, the
split planes) are filled with all-ones bytes, a NaN in every precision
(st_debug_poison_workspaces).  Every output must be bit-identical to the same
call on clean workspaces: no kernel may read an entry that its call has not
written, padding rows and columns of ragged tiles included.  Field counts
leave ragged column tiles; TCo127 has polar rings, whose rows are recomputed.
"""

import ctypes

import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ops(p, a, b, y):
    """(name, call) for every transform of the plan; each call returns its outputs."""
    def inv_deriv():
        g, dl, dp = p.grid_empty(), p.grid_empty(), p.grid_empty()
        p.inv_deriv(a, g, dl, dp)
        return g, dl, dp

    def direct():
        s = p.spec_empty()
        p.dir(y, s)
        return (s,)

    def inv_uv():
        u, v = p.grid_empty(), p.grid_empty()
        p.inv_uv(a, b, u, v)
        return u, v

    def dir_uv():
        z, d = p.spec_empty(), p.spec_empty()
        p.dir_uv(y, y.flip(0), z, d)
        return z, d

    def adjoints():
        ia, da = p.spec_empty(), p.grid_empty()
        p.inv_adjoint(y, ia)
        p.dir_adjoint(a, da)
        return ia, da

    return [("inv_deriv", inv_deriv), ("dir", direct), ("inv_uv", inv_uv), ("dir_uv", dir_uv),
            ("adjoints", adjoints)]


@pytest.mark.parametrize("prec,df", [("fp64", False), ("fp64", True), ("fp32", False), ("bf16x3", False),
                                     ("bf16x6", False)])
@pytest.mark.parametrize("T,nf", [(79, 3), (127, 5)])
def test_poisoned_workspaces_leave_results_unchanged(prec, df, T, nf):
    from paper_1908_06097_gb300 import st

    lib = st.load()
    p = st.Plan(T, nf, prec=prec, flags=st.FLAG_DF64 if df else 0)
    a = torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 500 + T)).cuda()
    b = torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 501 + T)).cuda()
    y = torch.from_numpy(inputs.grid_values(int(inputs.octahedral_nlon(T + 1).sum()), nf,
                                            inputs.SEED_BASE + 502 + T)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for name, op in _ops(p, a, b, y):
        clean = [x.clone() for x in op()]
        assert lib.st_debug_poison_workspaces(p.handle, stream) == 0
        poisoned = op()
        torch.cuda.synchronize()
        for i, (c, q) in enumerate(zip(clean, poisoned)):
            assert torch.equal(c, q), (name, i)
    assert p.sync_status() == 0
    p.close()
