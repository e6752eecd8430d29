"""Differentiable ray transmission through the nested geometry.

T_r = exp(-sum_m sigma_m l_m(r; theta)) for deterministic rays r without
collisions, as a torch.autograd.Function whose forward and backward are the
library's CUDA kernels (transmission_fwd / transmission_bwd):
  dT/dsigma_m = -l_m T
  dT/dtheta_j = -T sum_m sigma_m dl_m/dtheta_j,  theta = (r_fuel, r_clad, r_guide, pitch)
with dl_m/dtheta from the moved crossing points, dt/dtheta = -(df/dtheta) /
(grad f . Omega) at every crossing (segments recomputed in the backward pass,
not stored).  The geometry depends on theta, so a parametric geometry object
rebuilds the flattened description when the radii or the pitch change.
"""
from __future__ import annotations

import torch

from . import inputs
from . import native


class ParametricCore:
    """The three-level rect core of the transmission workload as a function
    of theta = (r_fuel, r_clad, r_guide, pitch): rebuilt on change."""

    def __init__(self, exact: bool = False, tracker: int = native.TRACKER_AUTO, **geom_kw):
        self.exact = exact
        self.tracker = tracker
        self.geom_kw = geom_kw
        self._key = None
        self.geom = None

    def geometry(self, theta: torch.Tensor) -> native.Geometry:
        vals = tuple(float(v) for v in theta.detach().cpu().tolist())
        if vals != self._key:
            desc = inputs.config2(r_fuel=vals[0], r_clad=vals[1], r_guide=vals[2], pitch=vals[3], **self.geom_kw)
            self.geom = native.Geometry(inputs.to_json(desc), exact=self.exact)
            self._key = vals
        return self.geom


class Transmission(torch.autograd.Function):
    """T = transmission(rays, sigma, theta, core): rays (n, 6) float64 on the
    GPU; sigma (n_materials,) and theta (4,) float64 tensors with gradients."""

    @staticmethod
    def forward(ctx, rays, sigma, theta, core: ParametricCore):
        g = core.geometry(theta)
        T, _ = g.transmission_fwd(rays, sigma.detach().contiguous(), tracker=core.tracker, lens=False)
        ctx.save_for_backward(rays, sigma, theta)
        ctx.core = core
        return T

    @staticmethod
    def backward(ctx, gT):
        rays, sigma, theta = ctx.saved_tensors
        g = ctx.core.geometry(theta)
        grad = g.transmission_bwd(rays, sigma.detach().contiguous(), float(theta[3]), gT.contiguous(),
                                  tracker=ctx.core.tracker)
        nm = sigma.shape[0]
        return None, grad[:nm].to(sigma.dtype), grad[nm:].to(theta.dtype), None


def transmission(rays, sigma, theta, core: ParametricCore):
    return Transmission.apply(rays, sigma, theta, core)
