"""Host-side checks of constants compiled into the CUDA kernels (no GPU)."""

import math

import numpy as np

from paper_2609_30166_gb300 import inputs


def test_cylinder_sampler_arctangent_coefficients():
    # the polynomial arctangent of the cylindrical sampler (its coefficients
    # are read from the kernel header): within 2e-7 rad of the true angle over
    # all octants when evaluated in FP32 Horner form
    import os
    import re

    hdr = open(os.path.join(os.path.dirname(inputs.__file__), "csrc", "cylinder.cuh")).read()
    body = hdr[hdr.index("cyl_angle"):hdr.index("return copysignf")]
    coef = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    assert len(coef) == 8  # highest power first
    ang = np.linspace(-math.pi, math.pi, 200001)
    x, y = np.cos(ang).astype(np.float32), np.sin(ang).astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    z = (np.minimum(ax, ay) / np.maximum(ax, ay)).astype(np.float32)
    t = (z * z).astype(np.float32)
    p = np.float32(coef[0])
    for ci in coef[1:]:
        p = (p * t + np.float32(ci)).astype(np.float32)
    a = (p * z).astype(np.float64)
    a = np.where(ay > ax, math.pi / 2 - a, a)
    a = np.where(x < 0, math.pi - a, a)
    a = np.copysign(a, y)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(np.angle(np.exp(1j * (a - ref))))
    assert err.max() < 2e-7
