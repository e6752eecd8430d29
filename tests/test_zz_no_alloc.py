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
    # Both paths run the same kernels and the same fixed-order reduction, so
    # the gradients must agree bit for bit.  The second call uses fewer rays:
    # partial sums the first call left in the shared array past the second
    # call's blocks must not reach its result.
    g, rays, sigma = _case()
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call, n in enumerate((rays.shape[0], rays.shape[0] - 12_345)):
        r = rays[:n].contiguous()
        gT = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
        ref = g.transmission_bwd(r, sigma, 1.26, gT)
        out = torch.full_like(ref, float("nan"))
        st = g.lib.transmission_bwd_noalloc(g.h, N.TRACKER_AUTO, n, N._ptr(r), N._ptr(sigma),
                                            ctypes.c_double(1.26), N._ptr(gT), N._ptr(out), N._stream())
        torch.cuda.synchronize()
        assert st == 0, g.lib.trk_last_error().decode()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b), (call, a, b)


def test_noalloc_python_wrapper():
    # the binding's wrapper makes the geometry's device current itself
    g, rays, sigma = _case()
    gT = torch.ones(rays.shape[0], dtype=torch.float64, device="cuda")
    ref = g.transmission_bwd(rays, sigma, 1.26, gT)
    out = torch.full_like(ref, float("nan"))
    N.transmission_bwd_noalloc(g, rays, sigma, 1.26, gT, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_too_many_rays():
    # The size check comes before any pointer is looked at, so null buffers
    # suffice: nothing can launch even if the check were to regress (the
    # backward pass would then refuse the null pointers).
    g, rays, sigma = _case()
    n_big = 1_000_000_000
    st = g.lib.transmission_bwd_noalloc(g.h, N.TRACKER_AUTO, n_big, None, None, ctypes.c_double(1.26), None, None,
                                        N._stream())
    assert st == -4
    assert "at most" in g.lib.trk_last_error().decode()
