"""The moment filter G (Eqs. moment1/moment2) and its transpose G^T (Sec. 4, the
gradient carried back through the filter) through the C ABI, against the
oracle's separable filter in fp64: G element by element, G^T against the
oracle's autograd of <G x, y> (the transpose is what that gradient is).

Cases span several 32 x 32 tiles with a ragged tail, both boundary rules, the
Gaussian and the box filter, the largest radius of the tiled kernel and one
above it (two 1-D passes), maps smaller than the filter, a single texel, and a
full 2048 x 2048 light map."""
import numpy as np
import pytest
import torch

from oracle import dsm_oracle as O

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-5, 1e-4

CASES = [  # res, sigma, radius, kind, boundary
    (64, 2.0, 0, 0, 0),
    (77, 2.0, 6, 0, 1),
    (100, 1.5, 0, 1, 0),
    (45, 3.0, 15, 1, 1),
    (45, 3.0, 15, 0, 0),
    (300, 8.0, 20, 0, 0),
    (130, 4.0, 16, 0, 1),
    (5, 3.0, 8, 0, 0),
    (7, 2.0, 10, 1, 1),
    (1, 2.0, 0, 0, 0),
    (2048, 2.0, 0, 0, 0),
]


def _ctx():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    return dsm.Context()


def _check(got, exp, what):
    got = got.astype(np.float64)
    bad = np.abs(got - exp) > ATOL + RTOL * np.abs(exp)
    assert not bad.any(), f"{what}: {bad.sum()} texels off, max diff {np.abs(got - exp).max():.3g}"


@pytest.mark.parametrize("res,sigma,radius,kind,boundary", CASES)
def test_filter_and_transpose_match_oracle(res, sigma, radius, kind, boundary):
    g = torch.Generator().manual_seed(1000 + res + radius)
    x = torch.rand((res, res, 2), generator=g, dtype=torch.float64)
    y = torch.rand((res, res, 2), generator=g, dtype=torch.float64) - 0.5
    w = O.filter_weights(sigma, radius, kind)
    ctx = _ctx()
    xd = x.float().cuda().contiguous()
    yd = y.float().cuda().contiguous()
    md = torch.full_like(xd, float("nan"))
    gd = torch.full_like(yd, float("nan"))
    ctx.filter_moments(xd, md, sigma, radius, kind, boundary)
    ctx.filter_moments_adjoint(yd, gd, sigma, radius, kind, boundary)
    ctx.sync()
    # the oracle sees the float32-rounded inputs the GPU sees
    xr32 = xd.cpu().double().requires_grad_(True)
    m32 = O.separable_filter(xr32, w, boundary)
    (m32 * yd.cpu().double()).sum().backward()
    _check(md.cpu().numpy(), m32.detach().numpy(), "G x")
    _check(gd.cpu().numpy(), xr32.grad.numpy(), "G^T y")
    ctx.close()


def test_filter_rejects_bad_arguments():
    from paper_2308_10896_b300 import dsm
    ctx = _ctx()
    a = torch.zeros((8, 8, 2), device="cuda")
    b = torch.zeros_like(a)
    for args in ((2.0, 33, 0, 0), (2.0, 0, 2, 0), (2.0, 0, 0, 2), (0.0, 0, 0, 0)):
        with pytest.raises(dsm.DsmError):
            ctx.filter_moments(a, b, *args)
        with pytest.raises(dsm.DsmError):
            ctx.filter_moments_adjoint(a, b, *args)
    ctx.close()
