"""The bounded waits of the persistent tensor-core convolutions, exercised.

Every mbarrier wait in the conv kernels gives up after a bounded number of
polls; a role that gives up raises a shared abort flag, the others leave
their loops, and after the CTA's final barrier the producer waits for the
last copy of every pipeline stage and the MMA warp for every MMA it issued
(bounded waits) before TMEM and shared memory are released.  Here a build
of the conv translation unit whose epilogue waits give up after one poll
runs the forward and the weight gradient: the kernels must come back (no
hang), set the status word, and leave the device usable -- a normal
convolution right after, in the same process, still matches the FP64
oracle (TMEM was released, nothing landed in shared memory after exit).
Every other wait keeps its normal bound."""

import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def variant(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    out = str(tmp_path_factory.mktemp("conv_abort") / "libconv_epi_wait1.so")
    src = os.path.join(_build.CSRC, "conv_tc.cu")
    cmd = [_build.nvcc()] + _build.ARCH + _build.FLAGS + ["-DCTREX_CONV_EPI_WAIT_LIMIT=1", "-shared", src, "-o", out]
    subprocess.run(cmd, check=True)
    lib = ctypes.CDLL(out)
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.ctrex_conv3d_fwd.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, i, i, vp, vp]
    lib.ctrex_conv3d_fwd.restype = i
    lib.ctrex_conv3d_wgrad.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp, vp]
    lib.ctrex_conv3d_wgrad.restype = i
    return ctrex, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_expired_epilogue_wait_recovers(variant):
    ct, lib = variant
    from oracle import conv

    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(21)
    # 2 x 64^3 x 16 channels: the forward runs the kx-folded kernel (1024
    # output tiles of 16 x 32 in items of 4 planes, several tiles per CTA, so
    # the MMA warp also reaches its accumulator-release waits).  The weight
    # gradient takes 32 output channels: layers with 16 use the
    # register-blocked kernel, which has no mbarrier waits.
    nb, d, h, w, cin, cout, cg = 2, 64, 64, 64, 16, 16, 32
    x = torch.as_tensor(rng.normal(size=(nb, d, h, w, cin)), dtype=torch.float32).to(torch.bfloat16).to(dev)
    wt = torch.as_tensor(rng.normal(size=(cout, 27, cin)) / 20.0, dtype=torch.float32).to(torch.bfloat16).to(dev)
    dy = torch.as_tensor(rng.normal(size=(nb, d, h, w, cg)), dtype=torch.float32).to(torch.bfloat16).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    # forward with the one-poll epilogue
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    y = torch.empty((nb, d, h, w, cout), dtype=torch.float32, device=dev)
    rc = lib.ctrex_conv3d_fwd(_p(x), _p(wt), None, _p(y), 0, nb, d, h, w, cin, cout, 0, _p(st), stream)
    torch.cuda.synchronize()
    assert rc == 0
    fwd_status = int(st.item())
    # weight gradient with the one-poll epilogue
    st.zero_()
    dw = torch.zeros((cg, 27, cin), dtype=torch.float32, device=dev)
    rc = lib.ctrex_conv3d_wgrad(_p(x), _p(dy), _p(dw), nb, d, h, w, cin, cg, _p(st), stream)
    torch.cuda.synchronize()
    assert rc == 0
    wg_status = int(st.item())
    print(f"status word after the expired waits: forward {fwd_status}, weight gradient {wg_status}")
    assert fwd_status == 1 and wg_status == 1
    # the normal library, right after, in the same process
    xs, ws_, dys = x[:1, :24, :20, :18], wt, dy[:1, :24, :20, :18]
    xs, dys = xs.contiguous(), dys.contiguous()
    y_ref = conv.conv3d(xs.double().cpu().numpy(), ws_.double().cpu().numpy())
    w32 = rng.normal(size=(cg, 27, cin))  # dW does not depend on the weights
    _, dw_ref = conv.conv3d_grads(xs.double().cpu().numpy(), w32, dys.double().cpu().numpy())
    y2 = ct.conv3d(xs, ws_, out_dtype=torch.float32)
    dw2 = ct.conv3d_wgrad(xs, dys)
    ct.conv_status_check(dev)
    e_y = float(np.linalg.norm(y2.double().cpu().numpy() - y_ref) / np.linalg.norm(y_ref))
    e_w = float(np.linalg.norm(dw2.double().cpu().numpy() - dw_ref) / np.linalg.norm(dw_ref))
    print(f"normal convolution afterwards: forward rel.L2 {e_y:.2e}, weight gradient {e_w:.2e}")
    assert e_y <= 1e-4 and e_w <= 1e-4
