"""Multi-resolution ROI (Sec. 3.7, simultaneous projection of a coarse
context grid and a fine ROI grid) on the GPU against the FP64 oracle,
element by element through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex


def _t(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dtype).cuda().contiguous()


def _np(t):
    return t.detach().double().cpu().numpy()


def _blobs(shape, vox, origin, seed=5):
    """A smooth analytic object (12 Gaussian blobs) sampled at the voxel
    centres of a grid, so both resolutions see the same object."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-9, 9, size=(12, 3))
    s = rng.uniform(1.0, 3.5, size=12)
    a = rng.uniform(0.2, 1.0, size=12)
    nz, ny, nx = shape
    X = origin[0] + np.arange(nx) * vox[0]
    Y = origin[1] + np.arange(ny) * vox[1]
    Z = origin[2] + np.arange(nz) * vox[2]
    vol = np.zeros(shape)
    for ci, si, ai in zip(c, s, a):
        vol += ai * (np.exp(-((Z - ci[2]) ** 2) / si ** 2)[:, None, None]
                     * np.exp(-((Y - ci[1]) ** 2) / si ** 2)[None, :, None]
                     * np.exp(-((X - ci[0]) ** 2) / si ** 2)[None, None, :])
    return vol


def _setup():
    """Context grid 37 x 33 x 29 at 0.8 mm (ragged); an ROI of 30 x 27 x 23 at
    0.35 mm whose box is not aligned to the context voxels."""
    cfg = inputs.CIRCULAR_64.scaled(name="perturbed-64^2-24v", nu=64, nv=64, n_views=24, trajectory="perturbed",
                                    seed=81)
    P = inputs.projection_matrices(cfg)
    shape, vox = (29, 33, 37), (0.8, 0.8, 0.8)
    origin = tuple(-0.5 * (n - 1) * 0.8 for n in (37, 33, 29))
    rshape, rvox = (23, 27, 30), (0.35, 0.35, 0.35)
    rorigin = (-3.9, -5.2, -2.7)
    xc = _blobs(shape, vox, origin)
    xf = _blobs(rshape, rvox, rorigin)
    pb = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv)).with_roi(rshape, rvox, rorigin)
    return cfg, P, shape, vox, origin, rshape, rvox, rorigin, xc, xf, pb


def _ctx(ct, cfg, P, shape, vox, origin, rshape, rvox, rorigin):
    c = ct.Context()
    c.set_geometry(P, shape, vox, origin, (cfg.nu, cfg.nv), cfg.step_vox)
    c.set_roi(rshape, rvox, rorigin)
    return c


def test_roi_forward_rowsum_and_count(ct):
    cfg, P, shape, vox, origin, rshape, rvox, rorigin, xc, xf, pb = _setup()
    x = np.concatenate([xc.ravel(), xf.ravel()])
    proj, rs = oracle.forward(pb, x)
    c = _ctx(ct, cfg, P, shape, vox, origin, rshape, rvox, rorigin)
    rowsum = torch.empty(proj.shape, device="cuda")
    out = c.fwd_project(_t(x), rowsum=rowsum)
    e, er = rel_l2(_np(out), proj), rel_l2(_np(rowsum), rs)
    print(f"ROI forward rel.L2 {e:.3e}, row sums {er:.3e}")
    assert e <= TOL32 and er <= TOL32
    # the ROI part alone, through the same call
    xr = np.concatenate([np.zeros(xc.size), xf.ravel()])
    pr, _ = oracle.forward(pb, xr)
    assert np.abs(pr).max() > 0.2 * np.abs(proj).max()
    assert rel_l2(_np(c.fwd_project(_t(xr))), pr) <= TOL32
    n_gpu, n_ref = c.count_samples(), oracle.count_samples(pb)
    print(f"ROI samples: GPU {n_gpu}, oracle {n_ref}")
    assert abs(n_gpu - n_ref) <= 1e-4 * n_ref


def test_roi_correction_backprojection_and_sirt(ct):
    cfg, P, shape, vox, origin, rshape, rvox, rorigin, xc, xf, pb = _setup()
    x = np.concatenate([xc.ravel(), xf.ravel()])
    proj, _ = oracle.forward(pb, x)
    c = _ctx(ct, cfg, P, shape, vox, origin, rshape, rvox, rorigin)
    x0 = 0.7 * x
    q, rsx = oracle.forward(pb, x0)
    r_ref, e2, p2 = oracle.correct(proj, q, rsx, pb.eps_R)
    r, sums = c.fwd_correct(_t(x0), _t(proj))
    scale = np.where(rsx > pb.eps_R, proj / np.where(rsx > 0, rsx, 1.0), 0.0)
    err = float(np.linalg.norm(_np(r) - r_ref) / np.linalg.norm(scale))
    print(f"ROI correction |dr| / |R p| = {err:.3e}")
    assert err <= TOL32 and np.allclose(_np(sums), [e2, p2], rtol=1e-4)
    # backprojection onto both grids, weighted update
    rng = np.random.default_rng(82)
    w = rng.uniform(0.5, 1.5, size=x.size)
    x_ref, b_ref, c_ref = oracle.backproject(pb, r_ref, alpha=0.9, x=x0, w=w)
    b = c.back_project(_t(r_ref), normalize=False, accumulate=False)
    cc = c.back_project(torch.ones_like(_t(r_ref)), normalize=False, accumulate=False)
    eb, ec = rel_l2(_np(b), b_ref), rel_l2(_np(cc), c_ref)
    xg = _t(x0)
    c.back_project(_t(r_ref), vol=xg, w=_t(w), alpha=0.9)
    eu = rel_l2(_np(xg) - x0, x_ref - x0)
    print(f"ROI backprojection: b {eb:.3e}, c {ec:.3e}, update {eu:.3e}")
    assert eb <= TOL32 and ec <= TOL32 and eu <= TOL32
    nc = xc.size
    assert np.abs(_np(b)[nc:]).max() > 0.0  # the ROI grid receives its own update
    # SIRT on both grids
    xs_ref, hist_ref, done_ref, _ = oracle.sirt(pb, proj, 5)
    xs = torch.zeros(x.size, device="cuda")
    xs, hist, done = c.sirt_iterate(xs, _t(proj), 5)
    es = rel_l2(_np(xs), xs_ref)
    print(f"ROI SIRT 5 iterations: rel.L2 {es:.3e}, residual {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert done == done_ref == 5 and es <= TOL32
    assert np.allclose(hist, hist_ref, rtol=1e-4)


def test_roi_state_errors(ct):
    cfg, P, shape, vox, origin, rshape, rvox, rorigin, xc, xf, pb = _setup()
    c = ct.Context()
    c.set_geometry(P, shape, vox, origin, (cfg.nu, cfg.nv), cfg.step_vox)
    with pytest.raises(ct.CtrexError):  # leaves the context box
        c.set_roi(rshape, rvox, (-20.0, -5.2, -2.7))
    c.set_roi(rshape, rvox, rorigin)
    with pytest.raises(ct.CtrexError):
        c.set_projector("joseph")
    with pytest.raises(ct.CtrexError):
        c.adjoint_project(torch.zeros((cfg.n_views, cfg.nv, cfg.nu), device="cuda"))
    th = torch.as_tensor(inputs.identity_theta(cfg.n_views), dtype=torch.float32).cuda()
    with pytest.raises(ct.CtrexError):
        c.set_motion(th)
    # removing the ROI restores the single-grid projector
    c.set_roi(None)
    ref, _ = oracle.forward(oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv)), xc)
    assert rel_l2(_np(c.fwd_project(_t(xc))), ref) <= TOL32


def test_roi_fullsize_sampled():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    rc = inputs.ROI_FOCUS
    b = rc.base
    P = inputs.projection_matrices(b)
    c = ctrex.context_for(b, P=P)
    c.set_roi(rc.roi_shape, (rc.roi_vox,) * 3, rc.roi_origin)
    xc, xf = inputs.roi_phantom(rc, device="cuda")
    x = torch.cat([xc.flatten(), xf.flatten()]).to(torch.float32).contiguous()
    p = c.fwd_project(x)
    pb = oracle.Problem(P, b.vol_shape, (b.vox,) * 3, b.origin, (b.nu, b.nv)).with_roi(
        rc.roi_shape, (rc.roi_vox,) * 3, rc.roi_origin)
    x64 = x.double().cpu().numpy()
    rng = np.random.default_rng(256)
    n = 160
    views = rng.integers(0, b.n_views, n).astype(np.int32)
    # pixels around the ROI's shadow (the central quarter of the detector)
    iu = rng.integers(3 * b.nu // 8, 5 * b.nu // 8, n)
    iv = rng.integers(3 * b.nv // 8, 5 * b.nv // 8, n)
    ref, _ = oracle.forward_rays(pb, x64, views, iu.astype(float), iv.astype(float))
    got = p[torch.as_tensor(views, dtype=torch.long), torch.as_tensor(iv), torch.as_tensor(iu)]
    e = rel_l2(got.double().cpu().numpy(), ref)
    print(f"ROI full size, {n} sampled rays: rel.L2 {e:.3e}")
    assert e <= TOL32
    # correction and backprojection at sampled voxels of both grids
    r, _ = c.fwd_correct((0.9 * x).contiguous(), p)
    bb = c.back_project(r, normalize=False, accumulate=False)
    nc = xc.numel()
    vox = np.concatenate([rng.integers(0, nc, 16), rng.integers(nc, x.numel(), 16)])
    r64 = r.double().cpu().numpy()
    b_ref, _ = oracle.backproject_voxels(pb, r64, vox)
    eb = rel_l2(bb[torch.as_tensor(vox)].double().cpu().numpy(), b_ref)
    print(f"ROI full size backprojection, 32 sampled voxels of both grids: rel.L2 {eb:.3e}")
    assert eb <= TOL32
