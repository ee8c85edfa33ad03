"""Extended field of view (Sec. 3.6, Sec. 4.3.2): SIRT for an offset
centre-of-rotation scan whose backprojector edge is moved per view and per
iteration to a random column between the physical detector edge and the
projected centre of rotation.  The forward projector always sees the whole
detector; the backprojector windows are set through ``ctrex_set_bp_window``.
"""

from __future__ import annotations

from . import inputs


def sirt_random_edge(ctx, cfg, x, p, n_iter, u_cor, seed=0, alpha=1.0):
    """n_iter SIRT iterations, windows re-drawn before each; returns the
    residual history (residual of the iterate before each update)."""
    hist = []
    for it in range(n_iter):
        ctx.set_bp_window(inputs.efov_windows(cfg, u_cor, seed + it))
        _, h, _ = ctx.sirt_iterate(x, p, 1, alpha=alpha)
        hist.append(float(h[0]))
    ctx.set_bp_window(None)
    return hist
