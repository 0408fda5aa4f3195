"""The Legendre tile-width autotuner (ST_FLAG_AUTOTUNE, tune_cache).

A plan created with the flag times the candidate tile widths on its own
workspaces and keeps the fastest; its transforms must stay within the
oracle tolerance.  The choice is appended to the cache file, and a later plan
with the same key takes it from there without timing (shown by planting a
choice in the file).  A group with an autotuned member tunes its merged
launches and must still match the members' own transforms bitwise.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x6": 1e-5}
CANDS = {"fp64": (64, 32), "fp32": (128, 64), "bf16x6": (128, 64)}


@pytest.fixture(scope="module")
def st():
    from paper_1908_06097_gb300 import st as _st

    _st.load()
    return _st


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x6"])
def test_autotuned_plan_matches_oracle_and_caches(st, orc, prec, tmp_path):
    T, nf = 79, 70  # more than one 64-column tile
    cache = str(tmp_path / "tune.txt")
    p = st.Plan(T, nf, prec=prec, flags=st.FLAG_AUTOTUNE, tune_cache=cache)
    bi, bd = p.tuning()
    assert bi in CANDS[prec] and bd in CANDS[prec]
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith(f"legendre T={T} ") and f"inv={bi} dir={bd}" in lines[0]
    a = inputs.spectral_fields(T, nf, inputs.SEED_BASE + 61)
    g = p.grid_empty()
    p.inv(torch.from_numpy(a).cuda(), g)
    s = p.spec_empty()
    p.dir(g, s)
    torch.cuda.synchronize()
    g_ref = orc.inverse(T, 0, T + 1, a)
    gh = g.cpu().numpy()
    for f in range(0, nf, 23):
        assert np.abs(gh[f] - g_ref[f]).max() <= TOL[prec] * np.abs(g_ref[f]).max()
    p.close()
    # a planted choice is read back without timing
    other_i, other_d = [c for c in CANDS[prec] if c != bi][0], [c for c in CANDS[prec] if c != bd][0]
    with open(cache, "a") as f:
        f.write(lines[0].split(" inv=")[0] + f" inv={other_i} dir={other_d}\n")
    q = st.Plan(T, nf, prec=prec, flags=st.FLAG_AUTOTUNE, tune_cache=cache)
    assert q.tuning() == (other_i, other_d)
    assert len(open(cache).read().splitlines()) == 2
    q.close()


def test_autotuned_group_matches_members(st):
    members = [(79, 40), (47, 3), (159, 2)]
    plans = [st.Plan(T, nf, prec="bf16x6", flags=st.FLAG_AUTOTUNE if i == 0 else 0)
             for i, (T, nf) in enumerate(members)]
    g = st.Group(plans)
    specs = [torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 70 + i)).cuda()
             for i, (T, nf) in enumerate(members)]
    grids = [p.grid_empty() for p in plans]
    g.inv(specs, grids)
    torch.cuda.synchronize()
    for p, a, gr in zip(plans, specs, grids):
        ref = p.grid_empty()
        p.inv(a, ref)
        torch.cuda.synchronize()
        # tile widths may differ between the group and the plan: same tolerance
        # as the split path's parity gate, relative to each field's maximum
        d = (gr - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)
        assert float(d.max()) <= 1e-6
    g.close()
    for p in plans:
        p.close()
