"""The paper's Jacobian experiment (Sec. 5, shadow map resolution and filter
kernel; supplementary Sec. B) as a functional test of the GPU path: a square
occluder, slightly rotated, over a receiver under an orthogonal directional
light; x is the occluder's horizontal translation, L = sum(W * image) with
fixed weights W, and dL/dx is the sum of the occluder vertices' x gradients.

- dL/dx from the backward pass equals the central difference of the rendered
  images at a step far below a texel (no event of the method is crossed).
- Over a step of one texel the difference quotient averages over the method's
  events.  With triangles much larger than a texel it stays close to dL/dx;
  with the paper's ~130k-face tessellation (triangles a third of a texel) the
  antialiasing misses primitive boundaries, the shadow map's Jacobian is
  sparse, and dL/dx falls well below it (the paper's observation).
- The filter is applied to the shadow map's Jacobian too, so the image's
  Jacobian dI/dx spreads over more pixels as the kernel grows."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

TEXEL = 3.0 / 256     # texel of the 256^2 map in world units
H = 2e-3              # step of the support test (0.17 texels)


def _render_shifted(dsm, r, base, occ, t):
    v = base.clone()
    v[occ, 0] += t
    return r.forward(verts=v.contiguous()).clone()


def _grad_and_differences(dsm, n, steps):
    sc = scenes.tessellated_occluder(n=n)
    r = dsm.Renderer(sc)
    occ = torch.as_tensor(sc["occluder"], device="cuda")
    base = r.verts.clone()
    W = torch.randn((128, 128, 4), generator=torch.Generator().manual_seed(3)).cuda()
    r.forward(verts=base)
    dv, _, _ = r.backward(W.contiguous())
    grad = float(dv[occ, 0].double().sum())
    fds = []
    for h in steps:
        lp = float((_render_shifted(dsm, r, base, occ, h).double() * W.double()).sum())
        lm = float((_render_shifted(dsm, r, base, occ, -h).double() * W.double()).sum())
        fds.append((lp - lm) / (2 * h))
    return grad, fds


def test_coarse_occluder_gradient_matches_central_differences():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    grad, (fd_small, fd_texel) = _grad_and_differences(dsm, 4, (1e-4, TEXEL))   # 32 triangles
    assert abs(grad) > 1.0
    assert abs(fd_small - grad) <= 0.05 * abs(grad), f"small-step difference {fd_small} vs gradient {grad}"
    assert 0.7 < grad / fd_texel < 1.5, f"one-texel difference {fd_texel} vs gradient {grad}"


def test_tessellated_occluder_gives_a_sparse_jacobian():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    grad, (fd_texel,) = _grad_and_differences(dsm, 256, (TEXEL,))   # 131,072 triangles
    assert np.sign(grad) == np.sign(fd_texel)
    assert grad / fd_texel < 0.5, f"gradient {grad} vs one-texel difference {fd_texel}"


def test_jacobian_support_grows_with_the_filter():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    support = []
    for sigma in (0.75, 1.5, 3.0):          # kernel sizes 5, 7, 13
        sc = scenes.tessellated_occluder(n=256, sigma=sigma)
        r = dsm.Renderer(sc)
        occ = torch.as_tensor(sc["occluder"], device="cuda")
        base = r.verts.clone()
        J = (_render_shifted(dsm, r, base, occ, H) - _render_shifted(dsm, r, base, occ, -H))[..., :3].sum(-1) / (2 * H)
        J = J.abs().cpu().numpy()
        support.append(int((J > 1e-2 * J.max()).sum()))
    assert support[0] < support[1] < support[2], support
