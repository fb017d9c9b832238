"""The allocation-free filter entry point (dsm_filter_moments_noalloc) gives the
same moment maps as dsm_filter_moments, call after call, through the C ABI.

It exists for callers that must not allocate device memory while they run (a
fixed-budget real-time loop, code inside a stream capture, a host application
that owns the memory pool); its intermediate map is a static device array of the
library.  This file is collected last so that a run stopping at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-5, 1e-4


def _lib():
    from paper_2308_10896_b300 import dsm
    return dsm, dsm.load_library()


def _reference(dsm, inp, sigma, radius, kind, boundary):
    ctx = dsm.Context()
    out = torch.empty_like(inp)
    ctx.filter_moments(inp, out, sigma, radius, kind, boundary)
    torch.cuda.synchronize()
    ctx.close()
    return out


@pytest.mark.parametrize("res,sigma,radius,kind,boundary", [(300, 2.0, 0, 0, 0), (1024, 1.5, 0, 0, 1), (77, 1.0, 2, 1, 0)])
def test_noalloc_filter_matches_existing_entry_point(res, sigma, radius, kind, boundary):
    dsm, lib = _lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cpu").manual_seed(res)
    for call in range(2):                               # two calls in a row share the static array
        inp = torch.rand((res, res, 2), generator=g).cuda().contiguous()
        ref = _reference(dsm, inp, sigma, radius, kind, boundary)
        out = torch.full_like(inp, float("nan"))
        st = lib.dsm_filter_moments_noalloc(ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()), res,
                                            ctypes.c_float(sigma), radius, kind, boundary, ctypes.c_void_p(stream))
        assert st == dsm.DSM_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        o, r = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(o - r) <= ATOL + RTOL * np.abs(r)), f"call {call}: max diff {np.abs(o - r).max()}"


def test_noalloc_filter_rejects_maps_above_its_static_size():
    dsm, lib = _lib()
    torch.cuda.set_device(0)
    inp = torch.zeros((1025, 1025, 2), device="cuda")
    out = torch.zeros_like(inp)
    st = lib.dsm_filter_moments_noalloc(ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1025,
                                        ctypes.c_float(2.0), 0, 0, 0, None)
    assert st == dsm.DSM_ERR_CAPACITY
