"""The two forms of the tensor-core Legendre kernels give the same bits.

The persistent kernel (the default: one CTA per SM over the tile list,
warp-specialised, accumulators reused across tiles) and the one-tile kernel
(one CTA per tile, selected with ST_TC_ONE_TILE=1 when the library loads)
issue the same MMAs in the same order into freshly zeroed accumulators and
combine them the same way, so every output must be bit-identical.  The
one-tile run happens in a child process, since the choice is read once per
process.  Sizes span several row and column tiles, a ragged column tile and
both split precisions.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1908_06097_gb300 import inputs, st
T, nf, prec, out = int(sys.argv[2]), int(sys.argv[3]), sys.argv[4], sys.argv[5]
st.load()
p = st.Plan(T, nf, prec=prec)
a = torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 300 + T)).cuda()
b = torch.from_numpy(inputs.spectral_fields(T, nf, inputs.SEED_BASE + 301 + T)).cuda()
g, dp = p.grid_empty(), p.grid_empty()
p.inv_deriv(a, g, None, dp)
s = p.spec_empty()
p.dir(g, s)
u, v = p.grid_empty(), p.grid_empty()
p.inv_uv(a, b, u, v)
z, d = p.spec_empty(), p.spec_empty()
p.dir_uv(u, v, z, d)
torch.cuda.synchronize()
assert p.sync_status() == 0
np.savez(out, *[x.cpu().numpy() for x in (g, dp, s, u, v, z, d)])
"""


def _run(T, nf, prec, out, one_tile):
    env = dict(os.environ)
    env.pop("ST_TC_ONE_TILE", None)
    if one_tile:
        env["ST_TC_ONE_TILE"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(T), str(nf), prec, out], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("T,nf", [(255, 37), (639, 5)])
def test_persistent_and_one_tile_kernels_agree_bitwise(tmp_path, prec, T, nf):
    pers = _run(T, nf, prec, str(tmp_path / "p.npz"), False)
    one = _run(T, nf, prec, str(tmp_path / "o.npz"), True)
    for k in pers.files:
        assert np.array_equal(pers[k], one[k]), k
