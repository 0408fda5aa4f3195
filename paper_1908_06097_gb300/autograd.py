"""Differentiable spherical-harmonic transforms (torch.autograd.Function).

The forward passes call the library's inverse / direct transforms; the
backward passes call its hand-written adjoint kernels (st_inv_adjoint,
st_dir_adjoint: the transposed Legendre contraction with the adjoint ring
FFT).  The adjoints are taken under the real Euclidean inner products on the
grid values and on the (Re, Im) spectral pairs; Im a_n^0 does not enter the
transform, so its gradient is 0.  All tensors are contiguous float64 CUDA
tensors in the layouts of include/st.h; the plan fixes T, the grid and the
field count.
"""

import torch


class InverseSHT(torch.autograd.Function):
    """grid = A spec (st_inv_transform); backward: spec_grad = A^T grid_grad."""

    @staticmethod
    def forward(ctx, spec, plan):
        grid = plan.grid_empty()
        plan.inv(spec.contiguous(), grid)
        ctx.plan = plan
        return grid

    @staticmethod
    def backward(ctx, grid_grad):
        spec_grad = ctx.plan.spec_empty()
        ctx.plan.inv_adjoint(grid_grad.contiguous(), spec_grad)
        return spec_grad, None


class DirectSHT(torch.autograd.Function):
    """spec = B grid (st_dir_transform); backward: grid_grad = B^T spec_grad."""

    @staticmethod
    def forward(ctx, grid, plan):
        spec = plan.spec_empty()
        plan.dir(grid.contiguous(), spec)
        ctx.plan = plan
        return spec

    @staticmethod
    def backward(ctx, spec_grad):
        grid_grad = ctx.plan.grid_empty()
        ctx.plan.dir_adjoint(spec_grad.contiguous(), grid_grad)
        return grid_grad, None


def inverse(spec, plan):
    """Differentiable inverse transform: spec [nfld, ncoef, 2] -> grid [nfld, npts]."""
    return InverseSHT.apply(spec, plan)


def direct(grid, plan):
    """Differentiable direct transform: grid [nfld, npts] -> spec [nfld, ncoef, 2]."""
    return DirectSHT.apply(grid, plan)
