"""Backward passes through the adjoint kernels (torch.autograd.Function).

The workload is TCo399 on O400 with 137 levels x 2 fields (274 fields, FP64).
The scalar loss is the area-weighted sum of squares of the grid values after
the inverse transform, L = sum_p w_p g_p^2, with w_p the Gauss weight of
p's ring divided by the ring length.  Checks:
  - dot-product test <A x, y> = <x, A^T y> to 1e-12 (FP64) for the inverse
    and the direct transform (A^T is the backward pass);
  - the gradient of L against central finite differences on 20 random
    spectral directions.  L is quadratic, so a central difference is exact
    for any step up to rounding; the step moves x by 10 % of its norm, which
    keeps the rounding of the two loss values far below the 1e-8 gate;
  - the backward pass against the FP64 CPU oracle's adjoint on a few fields.
"""

import numpy as np
import pytest

from paper_1908_06097_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

T, N, NFLD = 399, 400, 274


@pytest.fixture(scope="module")
def plan():
    from paper_1908_06097_gb300 import st

    st.load()
    p = st.Plan(T, NFLD, prec="fp64")
    yield p
    p.close()


def _dot(a, b):
    return float((a.double() * b.double()).sum())


def _area_weights(p):
    _, w = p.latitudes()
    wp = np.repeat(w / p.nlon, p.nlon)
    return torch.from_numpy(wp).cuda()


def test_dot_product_inverse_and_direct(plan):
    from paper_1908_06097_gb300 import autograd as ag

    g = torch.Generator(device="cpu").manual_seed(1908)
    x = torch.from_numpy(inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 3)).cuda()
    y = torch.randn(NFLD, plan.npts, generator=g, dtype=torch.float64).cuda()
    # inverse: <A x, y> = <x, A^T y>
    xr = x.clone().requires_grad_(True)
    gx = ag.inverse(xr, plan)
    (gx * y).sum().backward()
    lhs = _dot(gx.detach(), y)
    rhs = _dot(x, xr.grad)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
    # direct: <B y, s> = <y, B^T s>
    s = torch.from_numpy(inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 4)).cuda()
    yr = y.clone().requires_grad_(True)
    by = ag.direct(yr, plan)
    (by * s).sum().backward()
    lhs = _dot(by.detach(), s)
    rhs = _dot(y, yr.grad)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_gradient_finite_differences(plan):
    from paper_1908_06097_gb300 import autograd as ag

    wp = _area_weights(plan)
    x0 = torch.from_numpy(inputs.spectral_fields(T, NFLD, inputs.SEED_BASE + 3)).cuda()

    def loss(x):
        g = ag.inverse(x, plan)
        return (wp * g * g).sum()

    x = x0.clone().requires_grad_(True)
    loss(x).backward()
    grad = x.grad.clone()
    ns, ms = inputs.coef_nm(T)
    rng = np.random.default_rng(1908060973)
    for _ in range(20):
        d = rng.standard_normal(x0.shape)
        d[:, ms == 0, 1] = 0.0  # Im a_n^0 does not enter the transform
        d = torch.from_numpy(d).cuda()
        h = 0.1 * float(x0.norm()) / float(d.norm())
        with torch.no_grad():
            fd = (float(loss(x0 + h * d)) - float(loss(x0 - h * d))) / (2 * h)
        an = _dot(grad, d)
        assert abs(fd - an) <= 1e-8 * max(abs(an), 1e-300), (fd, an)


def test_backward_matches_oracle_adjoint(plan, orc):
    from paper_1908_06097_gb300 import autograd as ag

    fields = [0, 137, 273]
    y = inputs.grid_values(plan.npts, NFLD, inputs.SEED_BASE + 5)
    x = torch.zeros(NFLD, plan.ncoef, 2, dtype=torch.float64, device="cuda", requires_grad=True)
    g = ag.inverse(x, plan)
    g.backward(torch.from_numpy(y).cuda())
    ref = orc.inverse_adjoint(T, 0, N, y[fields])
    got = x.grad.cpu().numpy()[fields]
    for i in range(len(fields)):
        assert np.abs(got[i] - ref[i]).max() <= 1e-12 * np.abs(ref[i]).max()
