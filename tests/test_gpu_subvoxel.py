"""Sub-voxel backprojection (Sec. 4.3.2, motion blur) on the GPU against the
FP64 oracle, and against the block mean of the GPU's own backprojection on
the s-times finer grid at a size the oracle would take minutes for."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5

# ragged: 37 voxels per axis (not a multiple of the 32 x 4 x 4 voxel CTA tile)
RAGGED = inputs.CIRCULAR_64.scaled(name="perturbed-37^3-50x44-20v", n=37, nu=50, nv=44, n_views=20,
                                   trajectory="perturbed", seed=37)


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


def _np(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("s", [2, 3])
def test_subvoxel_b_and_c_match_oracle(ct, s):
    cfg = RAGGED
    pb = oracle_problem(cfg).with_subvoxel(s)
    rng = np.random.default_rng(s)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    _, b_ref, c_ref = oracle.backproject(pb, r)
    ctx = ct.context_for(cfg)
    ctx.set_bp_subvoxel(s)
    b = ctx.back_project(_t(r), normalize=False, accumulate=False)
    c = ctx.back_project(_t(np.ones_like(r)), normalize=False, accumulate=False)
    eb, ec = rel_l2(_np(b), b_ref), rel_l2(_np(c), c_ref)
    print(f"sub-voxel s={s}: b rel.L2 {eb:.3e}, c rel.L2 {ec:.3e}")
    assert eb <= TOL32 and ec <= TOL32
    # the sub-voxel result differs from the centre-only backprojector
    _, b1, _ = oracle.backproject(oracle_problem(cfg), r)
    assert rel_l2(b_ref, b1) > 1e-3


def test_subvoxel_with_subangles_window_and_weights(ct):
    cfg = inputs.HELICAL_256.scaled(name="helical-40^3-48x40-24v-S2", n=40, nu=48, nv=40, n_views=24, n_sub=2)
    P = inputs.projection_matrices(cfg)
    pb = oracle_problem(cfg, P=P)
    rng = np.random.default_rng(11)
    win = np.stack([rng.integers(0, 6, cfg.n_views), rng.integers(cfg.nu - 7, cfg.nu, cfg.n_views),
                    np.zeros(cfg.n_views, int), np.full(cfg.n_views, cfg.nv - 1)], axis=1).astype(np.int32)
    pb = pb.with_window(win).with_subvoxel(2)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    x0 = rng.uniform(size=cfg.vol_shape)
    w = rng.uniform(0.5, 1.5, size=cfg.vol_shape)
    x_ref, _, _ = oracle.backproject(pb, r, alpha=0.7, x=x0, w=w)
    ctx = ct.context_for(cfg, P=P)
    ctx.set_bp_window(win)
    ctx.set_bp_subvoxel(2)
    x = _t(x0)
    ctx.back_project(_t(r), vol=x, w=_t(w), alpha=0.7)
    err = rel_l2(_np(x) - x0, x_ref - x0)
    print(f"sub-voxel + sub-angles + window + weights: update rel.L2 {err:.3e}")
    assert err <= TOL32


def test_subvoxel_is_block_mean_of_fine_grid_bp(ct):
    cfg = inputs.CIRCULAR_64.scaled(name="perturbed-96^3-128x112-90v", n=96, nu=128, nv=112, n_views=90,
                                    trajectory="perturbed", seed=96)
    P = inputs.projection_matrices(cfg)
    ctx = ct.context_for(cfg, P=P)
    # projections of a phantom: images as smooth as the correction images of
    # a reconstruction (on white noise, the FP32 rounding of the projected
    # coordinate of each evaluation alone moves b by ~1e-5)
    r = ctx.fwd_project(inputs.phantom(cfg, device="cuda").float().contiguous())
    ones = torch.ones_like(r)
    ctx.set_bp_subvoxel(2)
    b2 = _np(ctx.back_project(r, normalize=False, accumulate=False))
    c2 = _np(ctx.back_project(ones, normalize=False, accumulate=False))
    fine = ct.Context()
    fvox = cfg.vox / 2
    forigin = tuple(o - 0.25 * cfg.vox for o in cfg.origin)
    fine.set_geometry(P, (2 * cfg.n,) * 3, (fvox,) * 3, forigin, (cfg.nu, cfg.nv), cfg.step_vox)
    n = cfg.n
    blk = lambda a: a.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))  # noqa: E731
    bf = blk(_np(fine.back_project(r, normalize=False, accumulate=False)))
    cf = blk(_np(fine.back_project(ones, normalize=False, accumulate=False)))
    eb, ec = rel_l2(b2, bf), rel_l2(c2, cf)
    print(f"sub-voxel 96^3 vs block mean of 192^3 backprojection: b {eb:.3e}, c {ec:.3e}")
    assert eb <= TOL32 and ec <= TOL32


def test_subvoxel_setting_errors_and_reset(ct):
    cfg = RAGGED
    ctx = ct.context_for(cfg)
    for bad in (0, -1, 9):
        with pytest.raises(RuntimeError):
            ctx.set_bp_subvoxel(bad)
    rng = np.random.default_rng(5)
    r = _t(rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu)))
    b_default = ctx.back_project(r, normalize=False, accumulate=False)
    ctx.set_bp_subvoxel(2)
    ctx.set_bp_subvoxel(1)
    assert torch.equal(ctx.back_project(r, normalize=False, accumulate=False), b_default)
