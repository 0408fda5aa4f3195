"""The halves of the decomposed transform and the exchange kernels, on one GPU.

R partitioned plans stand for R ranks of the paper's decomposition (each owns
some wavenumbers and some ring pairs).  The test runs them one after another
in one process: every rank's first half, then the all-to-all emulated by
device copies between the ranks' pack and unpack buffers (no kernel of one
rank waits on another), then every rank's second half.  The assembled grid
and spectra must equal the unpartitioned plan's transforms bit for bit (the
same kernels compute every row), and a rank must not write outside its own
rings and wavenumbers.
"""

import ctypes

import numpy as np
import pytest

from paper_1908_06097_gb300 import dist, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _exchange_all(engines, d):
    """The all-to-all of direction d among the emulated ranks (device copies)."""
    R = len(engines)
    sends = [e.pack(d) for e in engines]
    counts = [e.counts(d) for e in engines]
    row_bytes = counts[0][2]
    recvs = []
    for r in range(R):
        parts = []
        for s in range(R):
            send_rows = counts[s][0]
            start = sum(send_rows[:r]) * row_bytes
            parts.append(sends[s][start:start + send_rows[r] * row_bytes])
        assert sum(p.numel() for p in parts) == sum(counts[r][1]) * row_bytes
        recvs.append(torch.cat(parts) if parts else torch.empty(0, dtype=torch.uint8, device="cuda"))
    for e, rv in zip(engines, recvs):
        e.unpack(d, rv if rv.numel() else torch.empty(1, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
@pytest.mark.parametrize("T,nfld,R", [(79, 3, 3), (159, 2, 2)])
def test_decomposed_equals_whole(prec, T, nfld, R):
    from paper_1908_06097_gb300 import st

    N = T + 1
    mo, ro = dist.partition(T, N, R)
    a = torch.from_numpy(inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 80 + T)).cuda()
    whole = st.Plan(T, nfld, prec=prec)
    g_ref, s_ref = whole.grid_empty(), whole.spec_empty()
    whole.inv(a, g_ref)
    whole.dir(g_ref, s_ref)
    plans = [st.Plan(T, nfld, prec=prec) for _ in range(R)]
    engines = [dist.LibEngine(p, R, r, mo, ro) for r, p in enumerate(plans)]
    grids = [torch.full_like(g_ref, float("nan")) for _ in range(R)]
    specs = [torch.full_like(s_ref, float("nan")) for _ in range(R)]
    for e in engines:
        e.inv_legendre(a)
    _exchange_all(engines, 0)
    for e, g in zip(engines, grids):
        e.inv_fourier(g)
    for e in engines:
        e.dir_fourier(g_ref)
    _exchange_all(engines, 1)
    for e, s in zip(engines, specs):
        e.dir_legendre(s)
    torch.cuda.synchronize()
    off = whole.ring_off
    ns, ms = inputs.coef_nm(T)
    g_all = torch.full_like(g_ref, float("nan"))
    s_all = torch.full_like(s_ref, float("nan"))
    for r in range(R):
        for k in range(2 * N):
            kp = k if k < N else 2 * N - 1 - k
            ring = grids[r][:, off[k]:off[k + 1]]
            if ro[kp] == r:
                g_all[:, off[k]:off[k + 1]] = ring
            else:
                assert torch.isnan(ring).all()
        own = torch.from_numpy(mo[ms] == r).cuda()
        s_all[:, own] = specs[r][:, own]
        assert torch.isnan(specs[r][:, ~own]).all()
    assert torch.equal(g_all, g_ref)
    assert torch.equal(s_all, s_ref)
    for p in plans + [whole]:
        assert p.sync_status() == 0
        p.close()


def test_partition_argument_errors():
    from paper_1908_06097_gb300 import st

    lib = st.load()
    p = st.Plan(31, 1, prec="fp64")
    bad = np.full(32, 5, dtype=np.int32)
    ro = np.zeros(32, dtype=np.int32)
    assert lib.st_plan_set_partition(p.handle, 2, 0, bad.ctypes.data_as(ctypes.c_void_p),
                                     ro.ctypes.data_as(ctypes.c_void_p)) == st.ST_ERR_ARG
    cnt = (ctypes.c_long * 2)()
    assert lib.st_exchange_counts(p.handle, 0, cnt, cnt, None) == st.ST_ERR_ARG  # no partition yet
    p.close()
