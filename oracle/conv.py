"""FP64 CPU oracle of the 3x3x3 'same' convolution used by the warm-start
network (test infrastructure only).  Plain PyTorch CPU float64 ops; the
library routine conv3d is one step, itself pinned by brute-force loops in
tests/test_oracle_pins.py.

Layouts match the CUDA path: x [N, D, H, W, Cin] (channels last),
wt [Cout, 27, Cin] with tap = kz*9 + ky*3 + kx (offsets -1, 0, +1).
"""

import numpy as np
import torch


def _w5(wt):
    wt = torch.as_tensor(np.asarray(wt, dtype=np.float64))
    cout, _, cin = wt.shape
    return wt.reshape(cout, 3, 3, 3, cin).permute(0, 4, 1, 2, 3).contiguous()  # [Cout, Cin, kz, ky, kx]


def conv3d(x, wt, bias=None, relu=False):
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64)).permute(0, 4, 1, 2, 3)
    b = None if bias is None else torch.as_tensor(np.asarray(bias, dtype=np.float64))
    y = torch.nn.functional.conv3d(xt, _w5(wt), b, padding=1)
    if relu:
        y = torch.relu(y)
    return y.permute(0, 2, 3, 4, 1).contiguous().numpy()


def conv3d_grads(x, wt, dy):
    """(dx, dw) of L = <dy, conv3d(x, wt)>: dx like x, dw [Cout, 27, Cin]."""
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64)).permute(0, 4, 1, 2, 3).contiguous().requires_grad_(True)
    w5 = _w5(wt).requires_grad_(True)
    y = torch.nn.functional.conv3d(xt, w5, None, padding=1)
    dyt = torch.as_tensor(np.asarray(dy, dtype=np.float64)).permute(0, 4, 1, 2, 3)
    (y * dyt).sum().backward()
    dx = xt.grad.permute(0, 2, 3, 4, 1).contiguous().numpy()
    cout, cin = w5.shape[0], w5.shape[1]
    dw = w5.grad.permute(0, 2, 3, 4, 1).reshape(cout, 27, cin).contiguous().numpy()
    return dx, dw
