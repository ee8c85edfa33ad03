"""Coefficients of the arctangent used by the cylindrical sampler
(csrc/cylinder.cuh): atan(z) ~ z * (c0 + c1 z^2 + ... + c7 z^14) on [0, 1],
fitted by least squares at Chebyshev nodes of z in [0, 1] on the relative
error, then refined by a few Lawson (iteratively reweighted) passes toward
the minimax fit.  Run it to print the coefficients and the maximum error of
the FP64 polynomial and of its FP32 Horner evaluation."""

import numpy as np


def fit(degree=8, nodes=4000, passes=60):
    k = np.arange(nodes)
    z = 0.5 * (1.0 - np.cos(np.pi * (k + 0.5) / nodes))  # Chebyshev nodes on [0, 1]
    z = z[z > 1e-6]
    t = z * z
    V = np.vander(t, degree, increasing=True) * z[:, None]  # columns z t^i
    f = np.arctan(z)
    w = np.ones_like(z)
    for _ in range(passes):
        sw = np.sqrt(w)[:, None]
        c, *_ = np.linalg.lstsq(V * sw / f[:, None], sw[:, 0], rcond=None)  # relative error weights
        e = np.abs(V @ c / f - 1.0)
        w = w * (e / e.max() + 1e-3)
        w /= w.sum()
    return c


def horner32(c, z):
    z = z.astype(np.float32)
    t = z * z
    acc = np.float32(c[-1])
    for ci in c[-2::-1]:
        acc = np.float32(acc) * t + np.float32(ci)
    return acc * z


if __name__ == "__main__":
    c = fit()
    zz = np.linspace(0.0, 1.0, 2_000_001)
    p64 = (np.vander(zz * zz, len(c), increasing=True) * zz[:, None]) @ c
    p32 = horner32(c.astype(np.float32), zz).astype(np.float64)
    print("coefficients:", ", ".join(f"{v:.9e}f" for v in c.astype(np.float32)))
    print(f"max |error| FP64 polynomial {np.abs(p64 - np.arctan(zz)).max():.3e} rad")
    print(f"max |error| FP32 evaluation {np.abs(p32 - np.arctan(zz)).max():.3e} rad")
