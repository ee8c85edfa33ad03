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
                                            ((1, 3, 20, 19), 32, 160), ((1, 2, 17, 18), 192, 64),
                                            ((1, 5, 19, 33), 16, 16), ((2, 4, 9, 7), 16, 16), ((1, 4, 21, 26), 32, 32),
                                            ((1, 3, 17, 45), 48, 16), ((1, 3, 16, 64), 16, 32)])
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
# position tiles; 16 output channels (the register-blocked kernel) with
# ragged 16 x 32 tiles, and with three input-channel chunks whose tiles a
# CTA's range crosses
@pytest.mark.parametrize("shape,cin,cout", [((1, 6, 7, 9), 16, 16), ((2, 5, 6, 7), 48, 32), ((1, 8, 8, 8), 32, 64),
                                            ((1, 3, 17, 18), 32, 136), ((2, 4, 5, 6), 8, 16),
                                            ((1, 3, 19, 33), 24, 24), ((2, 7, 35, 40), 16, 16),
                                            ((2, 16, 40, 70), 48, 16)])
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


def test_conv_fullsize_sampled(ct):
    """The U-Net's widest layer at the size the bench times (2 x 128^3, 16 ->
    16 channels, the persistent TMA kernels): forward outputs at sampled
    voxels against direct FP64 sums over the 27 taps, and sampled weight
    derivatives against FP64 dot products over all 4.2 M voxels.  The weight
    gradient uses positive inputs: its FP32 accumulation over millions of
    voxels then stays far inside the 1e-4 bound (with zero-mean inputs the
    cancellation would scale the relative error by ~sqrt(n))."""
    rng = np.random.default_rng(128)
    shape = (2, 128, 128, 128)
    cin = cout = 16
    x = _bf(rng.normal(size=shape + (cin,)))
    wt = _bf(rng.normal(size=(cout, 27, cin)) / np.sqrt(27 * cin))
    y = ct.conv3d(x.cuda(), wt.cuda(), out_dtype=torch.float32)
    ct.conv_status_check()
    xp = np.pad(x.double().numpy(), ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    w64 = wt.double().numpy().reshape(cout, 3, 3, 3, cin)
    n = 64
    idx = np.stack([rng.integers(0, s, n) for s in shape], axis=1)
    ref = np.stack([np.einsum("oabci,abci->o", w64, xp[b, z:z + 3, yy:yy + 3, xx:xx + 3, :]) for b, z, yy, xx in idx])
    got = y[tuple(torch.as_tensor(idx[:, a]) for a in range(4))].double().cpu().numpy()
    e_y = rel_l2(got, ref)
    # weight gradient, positive inputs
    xq = _bf(rng.uniform(0.0, 1.0, size=shape + (cin,)))
    dq = _bf(rng.uniform(0.0, 1.0, size=shape + (cout,)))
    dw = ct.conv3d_wgrad(xq.cuda(), dq.cuda())
    ct.conv_status_check()
    xqp = np.pad(xq.double().numpy(), ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dq64 = dq.double().numpy()
    m = 24
    co_s, tap_s, ci_s = rng.integers(0, cout, m), rng.integers(0, 27, m), rng.integers(0, cin, m)
    ref_w = []
    for co, tap, ci in zip(co_s, tap_s, ci_s):
        kz, ky, kx = tap // 9, (tap // 3) % 3, tap % 3
        xs = xqp[:, kz:kz + 128, ky:ky + 128, kx:kx + 128, ci]
        ref_w.append(float(np.tensordot(dq64[..., co], xs, axes=4)))
    got_w = dw.double().cpu().numpy()[co_s, tap_s, ci_s]
    e_w = rel_l2(got_w, np.array(ref_w))
    print(f"conv 2 x 128^3 16->16: sampled outputs rel.L2 {e_y:.3e}, sampled weight derivatives {e_w:.3e}")
    assert e_y <= 1e-4 and e_w <= 1e-4
