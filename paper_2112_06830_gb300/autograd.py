"""torch.autograd wrapper of the photometry path.

``photometry(ctx, params, set_id, precision)`` returns AB magnitudes [G, Q] and
is differentiable with respect to ``params`` [12, G] (rows 0..10; the redshift
row 11 gets a zero gradient); the rows after z (nebular axis, old-star dust,
tabulated SFR) take the gradient rows after row 10.  Forward and backward both run in libdsps: the
backward calls dsps_photometry_vjp, which recomputes the forward sums it needs
instead of storing spectra.
"""
from __future__ import annotations

import torch

from . import dsps


class DSPSPhotometry(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, context, set_id, precision):
        mags = context.photometry(params, set_id, precision=precision)
        fctx.save_for_backward(params)
        fctx.context = context
        fctx.set_id = set_id
        fctx.precision = precision
        return mags

    @staticmethod
    def backward(fctx, grad_mags):
        (params,) = fctx.saved_tensors
        _, pbar = fctx.context.photometry_vjp(params, fctx.set_id, grad_mags.contiguous(),
                                              precision=fctx.precision, want_mags=False)
        grad = torch.zeros_like(params)
        # gradient rows 0..10 are parameter rows 0..10; the rows after them
        # (nebular axis, old-star dust, SFR table) are the parameter rows after
        # z (row 11)
        grad[: dsps.DSPS_NGRAD] = pbar[: dsps.DSPS_NGRAD]
        extra = pbar.shape[0] - dsps.DSPS_NGRAD
        if extra:
            grad[12:12 + extra] = pbar[dsps.DSPS_NGRAD:]
        return grad, None, None, None


def photometry(context: "dsps.Context", params: torch.Tensor, set_id: int,
               precision: int = dsps.DSPS_PREC_BF16X3) -> torch.Tensor:
    """Differentiable AB magnitudes of the galaxies in ``params`` [12, G]."""
    return DSPSPhotometry.apply(params, context, set_id, precision)
