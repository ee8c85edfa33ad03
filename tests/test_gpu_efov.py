"""Extended field of view: backprojector detector windows on the GPU vs the
FP64 oracle, and SIRT on a truncated offset centre-of-rotation scan with the
randomised backprojection edge."""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

# 48 columns of 1 mm, shifted 20 columns: the rotation axis projects at
# column 3.5, the detector covers a 24 mm wide fan at the centre of a 32 mm
# field of view, so every view truncates the object
CFG = inputs.CIRCULAR_64.scaled(name="offset-cor-64^3-48x96-90v", nu=48, nv=96, trajectory="offset",
                                det_offset=20.0)
U_COR = 0.5 * (CFG.nu - 1) - CFG.det_offset


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def test_bp_windows_match_oracle(ct):
    pb = oracle_problem(CFG)
    win = inputs.efov_windows(CFG, U_COR, seed=3)
    rng = np.random.default_rng(4)
    r = rng.normal(size=(CFG.n_views, CFG.nv, CFG.nu))
    x0 = rng.uniform(size=CFG.vol_shape)
    x_ref, b_ref, c_ref = oracle.backproject(pb.with_window(win), r, alpha=0.8, x=x0)
    ctx = ct.context_for(CFG)
    ctx.set_bp_window(win)
    rt = torch.as_tensor(r, dtype=torch.float32).cuda()
    b = ctx.back_project(rt, normalize=False, accumulate=False)
    assert rel_l2(b.double().cpu().numpy(), b_ref) <= 1e-5
    x = torch.as_tensor(x0, dtype=torch.float32).cuda()
    ctx.back_project(rt, vol=x, alpha=0.8)
    assert rel_l2(x.double().cpu().numpy() - x0, x_ref - x0) <= 1e-5
    # resetting the windows restores the whole-detector backprojector
    ctx.set_bp_window(None)
    _, b_full, _ = oracle.backproject(pb, r)
    assert rel_l2(ctx.back_project(rt, normalize=False, accumulate=False).double().cpu().numpy(), b_full) <= 1e-5


def test_truncated_offset_scan_sirt_with_random_edge(ct):
    from paper_2609_30166_gb300 import efov

    ctx = ct.context_for(CFG)
    ph = inputs.phantom(CFG, device="cuda").float().contiguous()
    p = ctx.fwd_project(ph)
    n_it = 30
    x_fix = torch.zeros_like(ph)
    _, h_fix, _ = ctx.sirt_iterate(x_fix, p, n_it)
    x_rnd = torch.zeros_like(ph)
    h_rnd = efov.sirt_random_edge(ctx, CFG, x_rnd, p, n_it, U_COR, seed=11)
    # both converge on the truncated data
    assert h_fix[-1] < 0.2 * h_fix[0] and h_rnd[-1] < 0.2 * h_rnd[0]
    # error near the boundary of the fully illuminated central disk
    r_c = abs(U_COR - (-0.5)) * CFG.pitch * inputs.SOD / inputs.SDD  # mm
    ax = torch.tensor(CFG.origin[0] + np.arange(CFG.n) * CFG.vox, device="cuda")
    rad = torch.sqrt(ax[None, :, None] ** 2 + ax[None, None, :] ** 2).expand(CFG.n, CFG.n, CFG.n)
    ring = (rad > r_c - 1.0) & (rad < r_c + 1.0)
    e_fix = float((x_fix - ph)[ring].norm() / ph[ring].norm())
    e_rnd = float((x_rnd - ph)[ring].norm() / ph[ring].norm())
    print(f"central-FOV ring (r = {r_c:.2f} mm) error after {n_it} iterations: fixed edge {e_fix:.4f}, "
          f"random edge {e_rnd:.4f}; residual {h_fix[-1]:.4f} / {h_rnd[-1]:.4f}")
    assert math.isfinite(e_fix) and math.isfinite(e_rnd)
