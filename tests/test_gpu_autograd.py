"""Hand-written transmission backward behind torch.autograd.Function:
against central finite differences of the CUDA forward (h = 1e-6) and the
oracle's analytic gradient."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N
from paper_2406_13849_gb300.autograd import ParametricCore, transmission

pytestmark = pytest.mark.gpu

R_OUT = 0.5 * 3 * 5 * 1.26 * 1.2
KW = dict(n_core=3, n_assm=5, height=20.0, r_outer=R_OUT)


def _setup(n=4000):
    rays = torch.from_numpy(I.boundary_rays(n, r_outer=R_OUT, height=20.0, seed=31).packed()).cuda()
    sigma = torch.tensor([0.9, 0.4, 0.2, 0.6], dtype=torch.float64, device="cuda", requires_grad=True)
    theta = torch.tensor([0.41, 0.475, 0.56, 1.26], dtype=torch.float64, device="cuda", requires_grad=True)
    return rays, sigma, theta


def test_autograd_matches_oracle_analytic():
    rays, sigma, theta = _setup()
    core = ParametricCore(**KW)
    w = torch.from_numpy(np.random.default_rng(4).normal(size=rays.shape[0])).cuda()
    T = transmission(rays, sigma, theta, core)
    loss = (w * T).sum()
    loss.backward()
    desc = I.config2(r_fuel=0.41, r_clad=0.475, r_guide=0.56, pitch=1.26, sigma=sigma.detach().cpu().numpy(), **KW)
    ref = O.Geometry(I.to_json(desc), O.MODE_RECT).transmission(rays.cpu().numpy(), sigma.detach().cpu().numpy(),
                                                                pitch=1.26)
    assert np.allclose(T.detach().cpu().numpy(), ref["T"], rtol=1e-12, atol=0)
    expect = (w.cpu().numpy()[:, None] * ref["dT"]).sum(0)
    got = np.concatenate([sigma.grad.cpu().numpy(), theta.grad.cpu().numpy()])
    assert np.allclose(got, expect, rtol=1e-9, atol=1e-13 * np.abs(expect).max())


def test_autograd_against_central_differences():
    # per ray: central differences of the CUDA forward (h = 1e-6) against the
    # analytic derivative (the oracle's per-ray terms, which the CUDA backward
    # reproduces in test_autograd_matches_oracle_analytic)
    rays, sigma, theta = _setup(3000)
    h = 1e-6
    base = torch.cat([sigma.detach(), theta.detach()])
    desc = I.config2(r_fuel=0.41, r_clad=0.475, r_guide=0.56, pitch=1.26, sigma=sigma.detach().cpu().numpy(), **KW)
    ref = O.Geometry(I.to_json(desc), O.MODE_RECT).transmission(rays.cpu().numpy(), sigma.detach().cpu().numpy(),
                                                                pitch=1.26)

    def f(v):
        with torch.no_grad():
            return transmission(rays, v[:4].clone(), v[4:].clone(), ParametricCore(**KW)).cpu().numpy()

    T0 = f(base)
    for j in range(8):
        e = torch.zeros(8, dtype=torch.float64, device="cuda")
        e[j] = h
        fd = (f(base + e) - f(base - e)) / (2 * h)
        an = ref["dT"][:, j]
        err = np.abs(fd - an) / np.maximum(np.abs(an), 1e-3 * np.abs(T0) + 1e-300)
        touched = np.abs(an) > 0
        if touched.any():
            assert np.median(err[touched]) < 1e-6, j
            assert np.quantile(err[touched], 0.95) < 1e-3, j
