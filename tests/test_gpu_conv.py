"""tcgen05 implicit-GEMM 3x3x3 convolution vs the FP64 conv oracle, fed the
same BF16-rounded inputs.  Products of BF16 values are exact and the tensor
cores accumulate in FP32, so FP32 outputs agree to 1e-4 relative L2 (the
bound set for the conv kernels); BF16 outputs add one rounding (4e-3)."""

import numpy as np
import pytest
import torch

from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def _bf(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16)


# channel counts: 1 (scalar gathers), 8 and 24 (16-byte im2col copies), the
# rest multiples of 16 (brick-staged input, TMA; filters resident or
# streamed, several N tiles); spatial sizes ragged against the 16 x 16 and
# 16 x 8 output tiles, several tiles per plane
@pytest.mark.parametrize("shape,cin,cout", [((1, 6, 7, 9), 1, 16), ((1, 6, 7, 9), 16, 48), ((2, 5, 8, 6), 48, 32),
                                            ((1, 8, 8, 8), 32, 192), ((1, 4, 4, 4), 96, 128),
                                            ((2, 3, 17, 19), 8, 16), ((1, 5, 9, 11), 24, 40),
                                            ((1, 4, 35, 21), 32, 24), ((2, 3, 18, 40), 16, 16),
                                            ((1, 3, 20, 19), 32, 160), ((1, 2, 17, 18), 192, 64)])
def test_conv_fwd_matches_oracle(ct, shape, cin, cout):
    from oracle import conv

    rng = np.random.default_rng(cin * 1000 + cout)
    x = _bf(rng.normal(size=shape + (cin,)))
    wt = _bf(rng.normal(size=(cout, 27, cin)) / np.sqrt(27 * cin))
    bias = rng.normal(size=cout).astype(np.float32)
    ref = conv.conv3d(x.double().numpy(), wt.double().numpy(), bias.astype(np.float64), relu=True)
    y = ct.conv3d(x.cuda(), wt.cuda(), torch.as_tensor(bias).cuda(), relu=True, out_dtype=torch.float32)
    ct.conv_status_check()
    assert rel_l2(y.double().cpu().numpy(), ref) <= 1e-4
    y16 = ct.conv3d(x.cuda(), wt.cuda(), torch.as_tensor(bias).cuda(), relu=True, out_dtype=torch.bfloat16)
    assert rel_l2(y16.double().cpu().numpy(), ref) <= 4e-3


# weight gradient: input channels 16, 48 (16-channel chunks), 32 (32-channel
# chunks), 8 and 24 (the split-K kernel); 136 output channels span two 128-row
# tiles, the second mostly empty; ragged spatial sizes against the 16 x 16
# position tiles
@pytest.mark.parametrize("shape,cin,cout", [((1, 6, 7, 9), 16, 16), ((2, 5, 6, 7), 48, 32), ((1, 8, 8, 8), 32, 64),
                                            ((1, 3, 17, 18), 32, 136), ((2, 4, 5, 6), 8, 16),
                                            ((1, 3, 19, 33), 24, 24)])
def test_conv_grads_match_oracle(ct, shape, cin, cout):
    from oracle import conv

    rng = np.random.default_rng(cin + 7 * cout)
    x = _bf(rng.normal(size=shape + (cin,)))
    wt = _bf(rng.normal(size=(cout, 27, cin)) / np.sqrt(27 * cin))
    dy = _bf(rng.normal(size=shape + (cout,)))
    dx_ref, dw_ref = conv.conv3d_grads(x.double().numpy(), wt.double().numpy(), dy.double().numpy())
    dx = ct.conv3d(dy.cuda(), ct.flip_weights(wt.cuda()), out_dtype=torch.float32)
    dw = ct.conv3d_wgrad(x.cuda(), dy.cuda())
    ct.conv_status_check()
    assert rel_l2(dx.double().cpu().numpy(), dx_ref) <= 1e-4
    assert rel_l2(dw.double().cpu().numpy(), dw_ref) <= 1e-4
