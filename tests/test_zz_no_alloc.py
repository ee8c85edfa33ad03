"""The allocation-free correction entry point (ctrex_correct_static).

It exists for callers that cannot let the library call cudaMalloc (their own
allocator already holds the device memory, or they run in a loop or callback
where allocating is not allowed); its reduction scratch is a static device
array shared by every call.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run everything else.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2609_30166_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def _rel(a, b):
    a, b = a.double().cpu(), b.double().cpu()
    return float((a - b).norm() / b.norm())


def _call(ct, p, q, rowsum, eps_R, dev):
    r = torch.full_like(p, float("nan"))
    sums = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    rc = ct.load_library().ctrex_correct_static(
        ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(rowsum.data_ptr()),
        ctypes.c_void_p(r.data_ptr()), ct.F32 if p.dtype == torch.float32 else ct.BF16, p.numel(),
        ctypes.c_float(eps_R), ctypes.c_void_p(sums.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert rc == ct.OK
    torch.cuda.synchronize()
    return r, sums


def test_correct_static_matches_fused_correction_twice(ct):
    """FP32: same r and residual norms as ctrex_fwd_correct (1e-5), twice."""
    cfg = inputs.CIRCULAR_64
    ctx = ct.context_for(cfg)
    dev = torch.device("cuda", torch.cuda.current_device())
    phantom = inputs.phantom(cfg).to(torch.float32).to(dev)
    x = (phantom * 0.8).contiguous()
    p = ctx.fwd_project(phantom)
    # existing entry point: fused projection + correction
    r_ref, sums_ref = ctx.fwd_correct(x, p)
    # inputs of the allocation-free one: q = A x, rowsum = A 1
    rowsum = torch.empty(p.shape, dtype=torch.float32, device=dev)
    q = ctx.fwd_project(x, rowsum=rowsum)
    eps_R = 1e-6 * cfg.vox
    for _ in range(2):  # the static scratch keeps the previous call's contents
        r, sums = _call(ct, p, q, rowsum, eps_R, dev)
        assert _rel(r, r_ref) <= 1e-5
        assert np.allclose(sums.cpu().numpy(), sums_ref.cpu().numpy(), rtol=1e-5, atol=0.0)
    # the Python wrapper takes the same path
    r2, _ = ct.correct_static(p, q, rowsum, eps_R=eps_R)
    torch.cuda.synchronize()
    assert _rel(r2, r_ref) <= 1e-5
    # and both equal the FP64 oracle's correction on the same inputs
    import oracle

    r_o, e2_o, p2_o = oracle.correct(p.double().cpu().numpy(), q.double().cpu().numpy(),
                                     rowsum.double().cpu().numpy(), eps_R)
    assert _rel(r2, torch.from_numpy(r_o)) <= 1e-5
    assert np.allclose(sums.cpu().numpy(), [e2_o, p2_o], rtol=1e-5, atol=0.0)
    ctx.close()


def test_correct_static_bf16_storage_twice(ct):
    """BF16 storage: equal to the FP32 call on the same rounded inputs up to
    one output rounding (4e-3), on two calls in a row."""
    cfg = inputs.CIRCULAR_64
    ctx = ct.context_for(cfg)
    dev = torch.device("cuda", torch.cuda.current_device())
    phantom = inputs.phantom(cfg).to(torch.float32).to(dev)
    p16 = ctx.fwd_project(phantom).to(torch.bfloat16).contiguous()
    rowsum = torch.empty(p16.shape, dtype=torch.float32, device=dev)
    q16 = ctx.fwd_project((phantom * 0.8).contiguous(), rowsum=rowsum, out_dtype=torch.bfloat16)
    eps_R = 1e-6 * cfg.vox
    r32, s32 = _call(ct, p16.float().contiguous(), q16.float().contiguous(), rowsum, eps_R, dev)
    for _ in range(2):
        r16, s16 = _call(ct, p16, q16, rowsum, eps_R, dev)
        assert _rel(r16, r32) <= 4e-3
        assert np.allclose(s16.cpu().numpy(), s32.cpu().numpy(), rtol=1e-5, atol=0.0)
    ctx.close()


def test_correct_static_rejects_oversize_before_launch(ct):
    lib = ct.load_library()
    buf = torch.zeros(4, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    rc = lib.ctrex_correct_static(ptr, ptr, ptr, ptr, ct.F32, ct.CORRECT_STATIC_MAX_N + 1, ctypes.c_float(0.0),
                                  None, None)
    assert rc == -2  # CTREX_E_SHAPE, nothing enqueued
    assert lib.ctrex_correct_static(ptr, ptr, ptr, ptr, 7, 4, ctypes.c_float(0.0), None, None) == -3
    assert lib.ctrex_correct_static(ptr, ptr, ptr, ptr, ct.F32, -1, ctypes.c_float(0.0), None, None) == -2
