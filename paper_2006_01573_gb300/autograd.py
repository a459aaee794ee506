"""PyTorch autograd wrappers of the differentiable projector (argument
marshalling only: every projection and gradient runs in libctis).

* :func:`project` -- ``H f`` as a function of the datacube ``f`` and the PSF tap
  values ``v`` (``Plan.export_taps`` order). Backward: ``dL/df = H^T gy``
  (Eq. 14) and ``dL/dv_t = sum_{p,r} f_s(p, r) gy(x_t + p, y_t + r)``.
* :func:`unrolled_nll` -- the Poisson negative log-likelihood after k EM
  updates (Eq. 2) as a function of ``v`` (and of the initial guess), with the
  gradient through the updates, including ``h = H^T 1``, computed natively with
  checkpointed iterates.

Both load the given values into the plan (``Plan.set_values``) before they
project, so one plan serves a whole optimisation of the PSF values. Several
live graphs may share one plan: a backward pass whose forward projected with
other values than the plan now holds loads its own values again first.
"""
from __future__ import annotations

import torch


def _load_values(plan, vals):
    plan.set_values(vals)


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, vals, plan):
        _load_values(plan, vals)
        ctx.plan = plan
        ctx.version = plan.values_version
        ctx.save_for_backward(f, vals.detach().clone())
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, gy):
        f, vals = ctx.saved_tensors
        plan = ctx.plan
        if plan.values_version != ctx.version:
            # another forward loaded other values since: the adjoint below
            # must apply the H this forward used
            _load_values(plan, vals)
            ctx.version = plan.values_version
        gy = gy.contiguous().float()
        df = plan.adjoint(gy) if ctx.needs_input_grad[0] else None
        dv = plan.psf_grad(f.contiguous(), gy) if ctx.needs_input_grad[1] else None
        return df, dv, None


def project(plan, f, vals):
    """``H f`` with H built from ``vals`` (differentiable in ``f`` and ``vals``)."""
    return _Project.apply(f, vals, plan)


class _UnrolledNll(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, f0, plan, g, k):
        _load_values(plan, vals)
        nll, dval, df0 = plan.unrolled_nll_grad(g, k, f0=f0, want_df0=f0 is not None)
        ctx.save_for_backward(dval, df0 if df0 is not None else torch.empty(0))
        ctx.has_f0 = f0 is not None
        return nll

    @staticmethod
    def backward(ctx, gout):
        dval, df0 = ctx.saved_tensors
        dv = (gout * dval).to(dval.dtype) if ctx.needs_input_grad[0] else None
        d0 = (gout * df0).to(df0.dtype) if ctx.has_f0 and ctx.needs_input_grad[1] else None
        return dv, d0, None, None, None


def unrolled_nll(plan, vals, g, k: int, f0=None):
    """Poisson NLL ``sum q - g log q`` of ``q = H f^(k)`` after k EM updates
    from ``f0`` (ones when None), differentiable in ``vals`` and ``f0``."""
    return _UnrolledNll.apply(vals, f0, plan, g, k)
