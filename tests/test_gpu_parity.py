"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 storage 1e-5 relative L2 (the contract for every
projector, correction and backprojection result); BF16 storage is compared
against the oracle run on the same BF16-rounded inputs at 4e-3 relative L2
(one output rounding is 2^-9 relative; sums stay FP32).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 4e-3


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def _gpu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dtype).cuda().contiguous()


def _np(t):
    return t.detach().double().cpu().numpy()


def _bf16_round(a):
    return torch.as_tensor(a).to(torch.bfloat16).double().numpy()


def _ctx(ct, cfg, P=None, vol_shape=None, vox=None, origin=None):
    if P is None:
        P = inputs.projection_matrices(cfg)
    c = ct.Context()
    c.set_geometry(P, vol_shape or cfg.vol_shape, vox or (cfg.vox,) * 3, origin or cfg.origin,
                   (cfg.nu, cfg.nv), cfg.step_vox)
    return c, P


@pytest.fixture(scope="module")
def c1(ct):
    cfg = inputs.CIRCULAR_64
    vol = inputs.phantom(cfg).numpy()
    pb = oracle_problem(cfg)
    proj, rs = oracle.forward(pb, vol)
    return cfg, vol, pb, proj, rs


# ---------------------------------------------------------------------------
# Forward projector
# ---------------------------------------------------------------------------

def test_forward_fp32_circular64(ct, c1):
    cfg, vol, pb, proj, rs = c1
    c, _ = _ctx(ct, cfg)
    rowsum = torch.empty((cfg.n_views, cfg.nv, cfg.nu), device="cuda")
    out = c.fwd_project(_gpu(vol), rowsum=rowsum)
    assert rel_l2(_np(out), proj) <= TOL32
    assert rel_l2(_np(rowsum), rs) <= TOL32
    # exact sample count agrees with the FP64 count up to rounding of ceil()
    n_gpu = c.count_samples()
    n_ref = oracle.count_samples(pb)
    assert abs(n_gpu - n_ref) <= 1e-6 * n_ref + 100


def test_forward_ragged_anisotropic_perturbed(ct):
    cfg = inputs.CIRCULAR_64.scaled(nu=77, nv=53, n_views=7, trajectory="perturbed", seed=21)
    shape = (23, 29, 37)  # nz, ny, nx
    vox = (0.8, 0.7, 1.1)
    origin = tuple(-0.5 * (n - 1) * v for n, v in zip(shape[::-1], vox))
    P = inputs.projection_matrices(cfg)
    rng = np.random.default_rng(1)
    vol = rng.uniform(size=shape)
    pb = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv), 0.5)
    proj, rs = oracle.forward(pb, vol)
    c, _ = _ctx(ct, cfg, P=P, vol_shape=shape, vox=vox, origin=origin)
    rowsum = torch.empty((cfg.n_views, cfg.nv, cfg.nu), device="cuda")
    out = c.fwd_project(_gpu(vol), rowsum=rowsum)
    assert rel_l2(_np(out), proj) <= TOL32
    assert rel_l2(_np(rowsum), rs) <= TOL32
    # backprojection on the same ragged grid
    r = rng.normal(size=proj.shape)
    _, b, cc = oracle.backproject(pb, r)
    got_b = c.back_project(_gpu(r), normalize=False, accumulate=False)
    assert rel_l2(_np(got_b), b) <= TOL32


def test_forward_subangles_helical(ct):
    cfg = inputs.HELICAL_256.scaled(n=48, nu=64, nv=48, n_views=24, z_span=12.0)
    vol = inputs.phantom(cfg, seed=3).numpy()
    pb = oracle_problem(cfg)
    proj, rs = oracle.forward(pb, vol)
    c, _ = _ctx(ct, cfg)
    rowsum = torch.empty((cfg.n_views, cfg.nv, cfg.nu), device="cuda")
    out = c.fwd_project(_gpu(vol), rowsum=rowsum)
    assert rel_l2(_np(out), proj) <= TOL32
    assert rel_l2(_np(rowsum), rs) <= TOL32
    # matched sub-angle backprojection
    r = np.random.default_rng(2).normal(size=proj.shape)
    _, b, cc = oracle.backproject(pb, r)
    got = c.back_project(_gpu(r), normalize=False, accumulate=False)
    assert rel_l2(_np(got), b) <= TOL32


def test_forward_view_subset_and_empty(ct, c1):
    cfg, vol, pb, proj, rs = c1
    c, _ = _ctx(ct, cfg)
    views = [17, 3, 89, 3, 40]
    out = c.fwd_project(_gpu(vol), view_idx=views)
    assert rel_l2(_np(out), proj[views]) <= TOL32
    empty = c.fwd_project(_gpu(vol), view_idx=np.zeros(0, np.int32))
    assert empty.shape == (0, cfg.nv, cfg.nu)
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# Fused correction and residual norms
# ---------------------------------------------------------------------------

def test_fwd_correct_circular64(ct, c1):
    cfg, vol, pb, proj, rs = c1
    rng = np.random.default_rng(3)
    x = vol * rng.uniform(0.5, 1.5, size=vol.shape)
    q, rsx = oracle.forward(pb, x)
    r_ref, s0, s1 = oracle.correct(proj, q, rsx, pb.eps_R)
    c, _ = _ctx(ct, cfg)
    r, sums = c.fwd_correct(_gpu(x), _gpu(proj))
    assert rel_l2(_np(r), r_ref) <= TOL32
    s = sums.cpu().numpy()
    assert s[0] == pytest.approx(s0, rel=1e-4)
    assert s[1] == pytest.approx(s1, rel=1e-5)
    # fixed-order reduction: bitwise reproducible
    r2, sums2 = c.fwd_correct(_gpu(x), _gpu(proj))
    assert torch.equal(sums, sums2) and torch.equal(r, r2)


# ---------------------------------------------------------------------------
# Backprojection and update
# ---------------------------------------------------------------------------

def test_backproject_circular64(ct, c1):
    cfg, vol, pb, proj, rs = c1
    rng = np.random.default_rng(4)
    r = rng.normal(size=proj.shape)
    w = rng.uniform(0.2, 1.0, size=vol.shape)
    x0 = rng.uniform(size=vol.shape)
    x_ref, b_ref, c_ref = oracle.backproject(pb, r, w=w, alpha=0.7, x=x0)
    c, _ = _ctx(ct, cfg)
    b = c.back_project(_gpu(r), normalize=False, accumulate=False)
    assert rel_l2(_np(b), b_ref) <= TOL32
    ones = c.back_project(_gpu(np.ones_like(r)), normalize=False, accumulate=False)
    assert rel_l2(_np(ones), c_ref) <= TOL32
    x = _gpu(x0)
    c.back_project(_gpu(r), vol=x, w=_gpu(w), alpha=0.7, normalize=True, accumulate=True)
    assert rel_l2(_np(x) - x0, x_ref - x0) <= TOL32


# ---------------------------------------------------------------------------
# SIRT (Eq. (1), all views)
# ---------------------------------------------------------------------------

def test_sirt_circular64(ct, c1):
    cfg, vol, pb, proj, rs = c1
    x_ref, hist_ref, done_ref, _ = oracle.sirt(pb, proj, cfg.sirt_iters)
    c, _ = _ctx(ct, cfg)
    x = torch.zeros(cfg.vol_shape, device="cuda")
    x, hist, done = c.sirt_iterate(x, _gpu(proj), cfg.sirt_iters)
    assert done == done_ref == cfg.sirt_iters
    assert rel_l2(_np(x), x_ref) <= TOL32
    assert np.allclose(hist, hist_ref, rtol=1e-4)
    assert hist[-1] < 0.5 * hist[0]


def test_sirt_restart_is_bitwise(ct, c1):
    cfg, vol, pb, proj, rs = c1
    c, _ = _ctx(ct, cfg)
    p = _gpu(proj)
    a = torch.zeros(cfg.vol_shape, device="cuda")
    c.sirt_iterate(a, p, 6)
    b = torch.zeros(cfg.vol_shape, device="cuda")
    c.sirt_iterate(b, p, 3)
    saved = b.cpu().clone()
    b2 = saved.cuda()
    c.sirt_iterate(b2, p, 3)
    assert torch.equal(a, b2)


def test_sirt_tolerance_stop_and_host_path(ct, c1):
    cfg, vol, pb, proj, rs = c1
    c, _ = _ctx(ct, cfg)
    x = torch.zeros(cfg.vol_shape, device="cuda")
    _, hist, done = c.sirt_iterate(x, _gpu(proj), 50, tol=0.2)
    assert 0 < done < 50 and hist[done] <= 0.2 and hist[done - 1] > 0.2
    xh = torch.zeros(cfg.vol_shape, dtype=torch.float32).pin_memory()
    ph = torch.as_tensor(proj, dtype=torch.float32).pin_memory()
    xh, hist_h, done_h = c.sirt_host(xh, ph, 4)
    xd = torch.zeros(cfg.vol_shape, device="cuda")
    xd, hist_d, done_d = c.sirt_iterate(xd, _gpu(proj), 4)
    # the host path's first iteration projects while the projections upload
    # and corrects afterwards: the same correction images (so the same
    # iterates, bitwise), only that residual norm summed in another order
    assert done_h == done_d == 4
    assert torch.equal(xh, xd.cpu()) and np.array_equal(hist_h[1:], hist_d[1:])
    assert np.allclose(hist_h[:1], hist_d[:1], rtol=1e-6, atol=0)
    # stopping on the tolerance at the first residual: no update applied
    xh0 = torch.zeros(cfg.vol_shape, dtype=torch.float32).pin_memory()
    xh0, hist0, done0 = c.sirt_host(xh0, ph, 4, tol=10.0)
    assert done0 == 0 and not xh0.any() and np.isclose(hist0[0], hist_d[0], rtol=1e-6)


# ---------------------------------------------------------------------------
# BF16 storage (FP32 accumulation)
# ---------------------------------------------------------------------------

def test_bf16_storage_forward_and_backproject(ct, c1):
    cfg, vol, pb, proj, rs = c1
    vol16 = _bf16_round(vol)
    ref16, _ = oracle.forward(pb, vol16)
    c, _ = _ctx(ct, cfg)
    out = c.fwd_project(_gpu(vol, torch.bfloat16), out_dtype=torch.bfloat16)
    assert out.dtype == torch.bfloat16
    assert rel_l2(_np(out), ref16) <= TOL16
    out32 = c.fwd_project(_gpu(vol, torch.bfloat16), out_dtype=torch.float32)
    assert rel_l2(_np(out32), ref16) <= TOL32
    r = _bf16_round(np.random.default_rng(5).normal(size=proj.shape))
    _, b_ref, _ = oracle.backproject(pb, r)
    b = c.back_project(_gpu(r, torch.bfloat16), normalize=False, accumulate=False)
    assert rel_l2(_np(b), b_ref) <= TOL32
    b16 = c.back_project(_gpu(r, torch.bfloat16), normalize=False, accumulate=False, vol_dtype=torch.bfloat16)
    assert rel_l2(_np(b16), b_ref) <= TOL16


def test_bf16_sirt_error_is_bounded(ct, c1):
    cfg, vol, pb, proj, rs = c1
    x_ref, hist_ref, _, _ = oracle.sirt(pb, proj, cfg.sirt_iters)
    c, _ = _ctx(ct, cfg)
    x = torch.zeros(cfg.vol_shape, device="cuda", dtype=torch.bfloat16)
    x, hist, done = c.sirt_iterate(x, _gpu(proj, torch.bfloat16), cfg.sirt_iters)
    err = rel_l2(_np(x), x_ref)
    print(f"BF16-storage SIRT ({cfg.sirt_iters} it.) rel.L2 vs FP64 oracle: {err:.3e}")
    assert err <= 5e-2, err
    assert abs(hist[-1] - hist_ref[-1]) <= 0.1 * hist_ref[-1] + 3e-3


# ---------------------------------------------------------------------------
# Matched adjoint and motion
# ---------------------------------------------------------------------------

def test_adjoint_matches_oracle_and_dot_product(ct):
    cfg = inputs.CIRCULAR_64.scaled(n=40, nu=48, nv=44, n_views=12, trajectory="perturbed", seed=8)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(6)
    y = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    ref = oracle.adjoint(pb, y)
    c, _ = _ctx(ct, cfg)
    got = c.adjoint_project(_gpu(y))
    assert rel_l2(_np(got), ref) <= TOL32
    x = rng.normal(size=cfg.vol_shape)
    Ax = _np(c.fwd_project(_gpu(x)))
    lhs, rhs = (Ax * y).sum(), (x * _np(got)).sum()
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Ax) * np.linalg.norm(y)


@pytest.fixture(scope="module")
def motion(ct):
    cfg = inputs.MOTION_FD_32.scaled(nu=40, nv=36, n_views=10)
    th, co, sv = inputs.motion_params(cfg)
    vol = inputs.phantom(cfg).numpy()
    pb = oracle_problem(cfg, theta=th, coef=co, s_view=sv)
    c, _ = _ctx(ct, cfg)
    c.set_motion(_gpu(th), _gpu(co), _gpu(sv), cfg.margin)
    return cfg, th, co, sv, vol, pb, c


def test_motion_forward_and_adjoint(ct, motion):
    cfg, th, co, sv, vol, pb, c = motion
    ref, rs = oracle.forward(pb, vol)
    rowsum = torch.empty((cfg.n_views, cfg.nv, cfg.nu), device="cuda")
    out = c.fwd_project(_gpu(vol), rowsum=rowsum)
    assert rel_l2(_np(out), ref) <= TOL32
    assert rel_l2(_np(rowsum), rs) <= TOL32
    y = np.random.default_rng(7).normal(size=ref.shape)
    assert rel_l2(_np(c.adjoint_project(_gpu(y))), oracle.adjoint(pb, y)) <= TOL32


def test_motion_gradient(ct, motion):
    cfg, th, co, sv, vol, pb, c = motion
    g = np.random.default_rng(8).normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    gt_ref, gc_ref = oracle.motion_grad(pb, vol, g)
    gt, gc = c.motion_grad(_gpu(vol), _gpu(g))
    et, ec = rel_l2(_np(gt), gt_ref), rel_l2(_np(gc), gc_ref)
    print(f"motion gradient rel.L2: theta {et:.3e}, coef {ec:.3e}")
    assert et <= TOL32 and ec <= TOL32


# ---------------------------------------------------------------------------
# Error paths
# ---------------------------------------------------------------------------

def test_error_paths(ct, c1):
    cfg, vol, pb, proj, rs = c1
    c, P = _ctx(ct, cfg)
    bad = P.copy()
    bad[5, 0, :, 0] = 0.0
    with pytest.raises(ct.CtrexError, match="GEOMETRY"):
        c.set_geometry(bad, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv))
    c, _ = _ctx(ct, cfg)
    out = c.fwd_project(_gpu(vol), view_idx=[0, 400, 1])  # 400 is out of range
    with pytest.raises(ct.CtrexError, match="DEVICE_CHECK"):
        c.device_status()
    c.device_status()  # flag cleared
    assert float(out[1].abs().max()) == 0.0
    with pytest.raises(ct.CtrexError, match="STATE"):
        c.motion_grad(_gpu(vol), torch.zeros((cfg.n_views, cfg.nv, cfg.nu), device="cuda"))
    with pytest.raises(TypeError):
        c.fwd_project(_gpu(vol, torch.float64))
