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


# every radius the filter takes (1 to 32: the tiled kernel up to 15, two 1-D
# passes above), each map side a multiple of 16 (the TMA-staged path, radius up
# to 8) or ragged, the kinds and boundaries in turn
SWEEP = [(48 if r % 2 else 37, 0.4 * r + 0.3, r, (r // 2) % 2, (r // 4) % 2) for r in range(1, 33)]


@pytest.mark.parametrize("res,sigma,radius,kind,boundary", SWEEP, ids=[f"r{c[2]}" for c in SWEEP])
def test_filter_radius_sweep_matches_oracle(res, sigma, radius, kind, boundary):
    test_filter_and_transpose_match_oracle(res, sigma, radius, kind, boundary)


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


TMA_CASES = [  # res, sigma, radius, kind, boundary: sides that are multiples of 16 take the TMA path
    (64, 2.0, 0, 0, 0),
    (48, 1.5, 3, 0, 1),
    (96, 2.0, 5, 1, 0),
    (160, 3.0, 8, 0, 0),
    (32, 1.0, 7, 0, 0),
    (2048, 2.0, 0, 0, 0),
    (2048, 1.0, 1, 1, 1),
]


@pytest.mark.parametrize("res,sigma,radius,kind,boundary", TMA_CASES)
def test_filter_shapes_are_bit_identical(res, sigma, radius, kind, boundary):
    """The TMA-staged kernel (shape 0), the fused kernel with plain loads
    (shape 2) and the two 1-D passes (shape 1): the forward results are
    bit-identical, the transposes of the tiled kernels too (the two-pass
    transpose applies y then x, so it agrees to rounding)."""
    g = torch.Generator().manual_seed(7000 + res + radius)
    x = torch.rand((res, res, 2), generator=g).cuda().contiguous()
    y = (torch.rand((res, res, 2), generator=g) - 0.5).cuda().contiguous()
    ctx = _ctx()
    out = {}
    for shape in (0, 2, 1):
        ctx.set_tuning(filter_shape=shape)
        m = torch.full_like(x, float("nan"))
        gin = torch.full_like(y, float("nan"))
        ctx.filter_moments(x, m, sigma, radius, kind, boundary)
        ctx.filter_moments_adjoint(y, gin, sigma, radius, kind, boundary)
        ctx.sync()
        out[shape] = (m.cpu(), gin.cpu())
    assert torch.equal(out[0][0], out[2][0]) and torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[2][1])
    assert torch.allclose(out[0][1], out[1][1], rtol=1e-5, atol=1e-6)


def test_bounded_wait_records_timeout_and_context_survives():
    """The bounded-wait failure path without a GPU fault: a wait that nothing
    completes gives up, dsm_sync reports DSM_ERR_TIMEOUT, and the context then
    renders the same frame as before."""
    import scenes
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    r = dsm.Renderer(scenes.tiny_scene(3, res=64, img=32))
    img0 = r.forward().clone()
    r.ctx.sync()
    r.ctx.bounded_wait_probe(arrive=True)
    r.ctx.sync()
    r.ctx.bounded_wait_probe(arrive=False)
    with pytest.raises(dsm.DsmError) as err:
        r.ctx.sync()
    assert err.value.status == dsm.DSM_ERR_TIMEOUT
    img1 = r.forward().clone()
    r.ctx.sync()
    assert torch.equal(img0, img1)
