"""Failure detection of the library, exercised without a GPU fault.

  - Bounded waits: the tensor-core Legendre kernels bound every mbarrier wait
    by the plan's wait limit.  A limit of a few dozen clocks makes the waits
    run out; the call must report ST_ERR_TIMEOUT through st_sync_status, the
    context must stay usable, and with the default limit restored the same
    plan must again match the oracle.
  - Work-list checks: a work-list entry overwritten with an out-of-range value
    (a test hook) is caught by the kernel's own check, skipped and reported
    as ST_ERR_CHECK; with the entry restored the results are bit-identical.
  - Input checks (ST_FLAG_CHECKS): a non-finite spectral coefficient or grid
    value is reported as ST_ERR_CHECK; finite inputs are not.
  - Allocation failures: the n-th device allocation of plan creation is made
    to fail (a test hook); creation returns ST_ERR_NOMEM, frees what it had
    allocated, and a plan created afterwards is correct.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

T, NFLD = 79, 6


def _oracle_inverse(orc, a):
    return orc.inverse(T, 0, T + 1, a)


def _relerr(x, ref):
    return max(float(np.abs(x[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in range(len(ref)))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_wait_limit_runs_out_then_recovers(orc, prec):
    from paper_1908_06097_gb300 import st

    a = inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 40)
    ref = _oracle_inverse(orc, a)
    p = st.Plan(T, NFLD, prec=prec)
    ad = torch.from_numpy(a).cuda()
    g = p.grid_empty()
    s = p.spec_empty()
    p.set_wait_limit(32)
    p.inv(ad, g)
    assert p.sync_status() == st.ST_ERR_TIMEOUT
    p.dir(g, s)  # the direct kernel's waits run out as well
    assert p.sync_status() == st.ST_ERR_TIMEOUT
    p.set_wait_limit(0)  # default
    p.inv(ad, g)
    assert p.sync_status() == st.ST_OK
    assert _relerr(g.cpu().numpy(), ref) < 1e-5
    p.dir(g, s)
    assert p.sync_status() == st.ST_OK
    with pytest.raises(st.StError):
        p.set_wait_limit(-1)
    p.close()


@pytest.mark.parametrize("what", [1, 2], ids=["legendre_tile", "fft_item"])
@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_corrupt_work_list_entry_is_caught(prec, what):
    from paper_1908_06097_gb300 import st

    lib = st.load()
    a = torch.from_numpy(inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 41)).cuda()
    p = st.Plan(T, NFLD, prec=prec)
    g0, g1 = p.grid_empty(), p.grid_empty()
    p.inv(a, g0)
    assert p.sync_status() == st.ST_OK
    assert lib.st_debug_corrupt_worklist(p.handle, what) == st.ST_OK
    p.inv(a, g1)
    assert p.sync_status() == st.ST_ERR_CHECK
    assert lib.st_debug_corrupt_worklist(p.handle, 0) == st.ST_OK
    p.inv(a, g1)
    assert p.sync_status() == st.ST_OK
    assert torch.equal(g0, g1)
    assert lib.st_debug_corrupt_worklist(p.handle, 3) == st.ST_ERR_ARG
    p.close()


def test_checks_flag_reports_non_finite_input():
    from paper_1908_06097_gb300 import st

    a = inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 42)
    p = st.Plan(T, NFLD, prec="fp64", flags=st.FLAG_CHECKS)
    q = st.Plan(T, NFLD, prec="fp64")
    g = p.grid_empty()
    p.inv(torch.from_numpy(a).cuda(), g)
    assert p.sync_status() == st.ST_OK
    bad = a.copy()
    bad[3, 17, 0] = np.nan
    p.inv(torch.from_numpy(bad).cuda(), g)
    assert p.sync_status() == st.ST_ERR_CHECK
    q.inv(torch.from_numpy(bad).cuda(), g)  # without the flag nothing is checked
    assert q.sync_status() == st.ST_OK
    # the direct transform checks its grid input
    p.inv(torch.from_numpy(a).cuda(), g)
    s = p.spec_empty()
    p.dir(g, s)
    assert p.sync_status() == st.ST_OK
    g[2, 1000] = float("inf")
    p.dir(g, s)
    assert p.sync_status() == st.ST_ERR_CHECK
    p.close()
    q.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_allocation_failure_is_clean(orc, prec):
    from paper_1908_06097_gb300 import st

    lib = st.load()
    a = inputs.spectral_fields(31, 3, inputs.SEED_BASE + 43)
    ref = orc.inverse(31, 0, 32, a)
    warm = st.Plan(31, 3, prec=prec)  # modules loaded, tables of another T cached
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for n in range(1, 200):
            assert lib.st_debug_fail_alloc(n) == st.ST_OK
            try:
                p = st.Plan(47, 3, prec=prec)
            except st.StError as e:
                assert e.code == st.ST_ERR_NOMEM, e
                failures += 1
                torch.cuda.synchronize()
                # nothing of the failed creation stays allocated
                assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20), n
                continue
            p.close()  # n is past the last allocation: creation succeeded
            break
        else:
            pytest.fail("plan creation never succeeded")
    finally:
        lib.st_debug_fail_alloc(0)
    assert failures > 10
    p = st.Plan(31, 3, prec=prec)
    g = p.grid_empty()
    p.inv(torch.from_numpy(a).cuda(), g)
    assert p.sync_status() == st.ST_OK
    assert _relerr(g.cpu().numpy(), ref) < (1e-12 if prec == "fp64" else 1e-5)
    p.close()
    warm.close()
