"""Shared test helpers: oracle problems built from the seeded input configs."""

import numpy as np

from paper_2609_30166_gb300 import inputs


def oracle_problem(cfg, P=None, theta=None, coef=None, s_view=None):
    import oracle

    if P is None:
        P = inputs.projection_matrices(cfg)
    vox = (cfg.vox,) * 3
    return oracle.Problem(P, cfg.vol_shape, vox, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox,
                          theta=theta, coef=coef, s_view=s_view,
                          margin=cfg.margin if (theta is not None or coef is not None) else 0.0)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def ray_points(cfg, view, sub=0):
    """Source and pixel-centre positions of every pixel of one view, from the
    trajectory definition itself (no projection matrix involved)."""
    srcs, ctrs, us, vs = inputs.detector_frames(cfg)
    s, c, u, v = srcs[view, sub], ctrs[view, sub], us[view, sub], vs[view, sub]
    d0 = c - 0.5 * (cfg.nu - 1) * u - 0.5 * (cfg.nv - 1) * v
    iu = np.arange(cfg.nu)
    iv = np.arange(cfg.nv)
    pix = d0[None, None, :] + iv[:, None, None] * v[None, None, :] + iu[None, :, None] * u[None, None, :]
    return s, pix  # pix [nv, nu, 3]
