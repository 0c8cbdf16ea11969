"""Calibration of the kernel width sigma against a target mean synapse length.

The expected mean synapse length m(sigma) (msp_length_loss: an axonal element
of t reaches dendrite s with probability w_s K(t,s)/u(t), Eq. 1 with the
kernel of Eq. 8) grows with sigma.  Newton's method on m(sigma) - target, with
dm/dsigma from the library's adjoint sums, finds the sigma whose mean
synapse length is the target; every step redoes the pair lists of the
attraction at the new width (the octree stays).

    from paper_2301_10570_gb300 import calibrate, msp
    ctx = msp.MSP(params)                 # cutoff 5, no translations
    ctx.build_tree(pos, type_, ones, ones, ones)
    sigma, history = calibrate.calibrate_sigma(ctx, type_, vac_axon, w_e, w_i, 1000.0)
"""
from __future__ import annotations


def calibrate_sigma(ctx, type_, vac_axon, w_e, w_i, target, sigma0=None, iters=12, rtol=1e-4):
    """Returns (sigma, history of (sigma, m, dm/dsigma)).  Steps are limited
    to a factor of 2; the loop stops when |m - target| <= rtol * target."""
    sigma = float(sigma0 if sigma0 is not None else ctx.params["sigma"])
    history = []
    for _ in range(iters):
        ctx.set_sigma(sigma)
        ctx.attraction()
        r = ctx.length_loss(type_, vac_axon, w_e, w_i, target, grad=False)
        history.append((sigma, r["mean"], r["dmean_dsigma"]))
        err = r["mean"] - target
        if abs(err) <= rtol * abs(target):
            break
        d = r["dmean_dsigma"]
        step = sigma - err / d if d > 0 else sigma * (0.5 if err > 0 else 2.0)
        sigma = min(max(step, 0.5 * sigma), 2.0 * sigma)
    return sigma, history
