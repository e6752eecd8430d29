"""transmission_bwd_noalloc: the backward pass for callers that cannot
allocate device memory (its scratch is a fixed array in the library's device
image).  Checked through the C-ABI against transmission_bwd, which takes a
caller-allocated work buffer, on two calls in a row.  This file sorts last so
that a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu


def _case():
    r_out = 0.5 * 3 * 5 * 1.26 * 1.2
    desc = I.small_core(height=20.0, r_outer=r_out)
    g = N.Geometry(I.to_json(desc))
    rays = torch.from_numpy(I.boundary_rays(50_000, r_outer=r_out, height=20.0, seed=21).packed()).cuda()
    sigma = torch.tensor(desc["sigma"], dtype=torch.float64, device="cuda")
    return g, rays, sigma


def test_noalloc_backward_matches_allocating_backward_twice():
    g, rays, sigma = _case()
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        gT = torch.randn(rays.shape[0], dtype=torch.float64, device="cuda", generator=gen)
        ref = g.transmission_bwd(rays, sigma, 1.26, gT)
        out = torch.full_like(ref, float("nan"))
        st = g.lib.transmission_bwd_noalloc(g.h, N.TRACKER_AUTO, rays.shape[0], N._ptr(rays), N._ptr(sigma),
                                            ctypes.c_double(1.26), N._ptr(gT), N._ptr(out), N._stream())
        torch.cuda.synchronize()
        assert st == 0, g.lib.trk_last_error().decode()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.allclose(a, b, rtol=1e-10, atol=1e-14 * np.abs(b).max()), (call, a, b)


def test_noalloc_rejects_too_many_rays():
    g, rays, sigma = _case()
    n_big = 40_000_000
    st = g.lib.transmission_bwd_noalloc(g.h, N.TRACKER_AUTO, n_big, N._ptr(rays), N._ptr(sigma),
                                        ctypes.c_double(1.26), N._ptr(rays), N._ptr(sigma), N._stream())
    assert st == -4
    assert "at most" in g.lib.trk_last_error().decode()
