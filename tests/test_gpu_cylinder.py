"""Aligned cylindrical domain (Sec. 3.5): the CUDA projector, correction,
backprojector and SIRT on (r, phi, z) grids against the FP64 oracle, element
by element, through the C ABI; the full-size vial workload on sampled rays
and voxels."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 4e-3

# ragged: 21 rings (not a multiple of 32), 50 sectors, 27 slices (odd)
SMALL = inputs.CYL_SMALL.scaled(name="cylinder-21x50x27-64^2-60v", n_r=21, n_phi=50, n_z=27)


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


def _problem(cc, P=None):
    if P is None:
        P = inputs.projection_matrices(cc.base)
    b = cc.base
    return oracle.cylinder_problem(P, cc.n_r, cc.n_phi, cc.n_z, cc.dr, cc.dz, (b.nu, b.nv),
                                   pose=inputs.cylinder_pose(cc), step_vox=cc.step_vox)


@pytest.fixture(scope="module")
def small():
    cc = SMALL
    P = inputs.projection_matrices(cc.base)
    pb = _problem(cc, P)
    vol = inputs.cyl_phantom(cc).numpy()
    proj, rs = oracle.forward(pb, vol)
    return cc, P, pb, vol, proj, rs


def test_cylinder_forward_and_rowsum(ct, small):
    cc, P, pb, vol, proj, rs = small
    ctx = ct.context_for_cylinder(cc, P=P)
    rowsum = torch.empty(proj.shape, device="cuda")
    out = ctx.fwd_project(_t(vol), rowsum=rowsum)
    e, er = rel_l2(_np(out), proj), rel_l2(_np(rowsum), rs)
    print(f"cylinder forward rel.L2 {e:.3e}, row sums {er:.3e}")
    assert e <= TOL32 and er <= TOL32
    assert (rs > 0).mean() > 0.3  # the cylinder covers a good part of the detector
    n_gpu, n_ref = ctx.count_samples(), oracle.count_samples(pb)
    assert abs(n_gpu - n_ref) <= 1e-6 * n_ref + 100


def test_cylinder_correction(ct, small):
    cc, P, pb, vol, proj, rs = small
    ctx = ct.context_for_cylinder(cc, P=P)
    x = 0.8 * vol
    q, rsx = oracle.forward(pb, x)
    r_ref, e2, p2 = oracle.correct(proj, q, rsx, pb.eps_R)
    r, sums = ctx.fwd_correct(_t(x), _t(proj))
    # p - A x cancels: compare against the scale of R p
    scale = np.where(rsx > pb.eps_R, proj / np.where(rsx > 0, rsx, 1.0), 0.0)
    err = float(np.linalg.norm(_np(r) - r_ref) / np.linalg.norm(scale))
    print(f"cylinder correction |dr| / |R p| = {err:.3e}")
    assert err <= TOL32
    assert np.allclose(_np(sums), [e2, p2], rtol=1e-4)


def test_cylinder_backprojection_variants(ct, small):
    cc, P, pb, vol, proj, rs = small
    ctx = ct.context_for_cylinder(cc, P=P)
    rng = np.random.default_rng(31)
    r = proj / np.maximum(rs, 1e-3)  # smooth images, like a correction
    _, b_ref, c_ref = oracle.backproject(pb, r)
    b = ctx.back_project(_t(r), normalize=False, accumulate=False)
    c = ctx.back_project(_t(np.ones_like(r)), normalize=False, accumulate=False)
    eb, ec = rel_l2(_np(b), b_ref), rel_l2(_np(c), c_ref)
    print(f"cylinder BP: b {eb:.3e}, c {ec:.3e}")
    assert eb <= TOL32 and ec <= TOL32
    # normalised, weighted, windowed update, then with sub-voxel points
    x0 = rng.uniform(size=cc.vol_shape)
    w = rng.uniform(0.5, 1.5, size=cc.vol_shape)
    b_ = cc.base
    win = np.stack([rng.integers(0, 8, b_.n_views), rng.integers(b_.nu - 9, b_.nu, b_.n_views),
                    np.zeros(b_.n_views, int), np.full(b_.n_views, b_.nv - 1)], axis=1).astype(np.int32)
    ctx.set_bp_window(win)
    for s in (1, 2):
        ctx.set_bp_subvoxel(s)
        x_ref, _, _ = oracle.backproject(pb.with_window(win).with_subvoxel(s), r, alpha=0.6, x=x0, w=w)
        x = _t(x0)
        ctx.back_project(_t(r), vol=x, w=_t(w), alpha=0.6)
        err = rel_l2(_np(x) - x0, x_ref - x0)
        print(f"cylinder BP update (window, weights, sub-voxel {s}): {err:.3e}")
        assert err <= TOL32


def test_cylinder_sirt(ct, small):
    cc, P, pb, vol, proj, rs = small
    x_ref, hist_ref, done_ref, _ = oracle.sirt(pb, proj, 6)
    ctx = ct.context_for_cylinder(cc, P=P)
    x = torch.zeros(cc.vol_shape, device="cuda")
    x, hist, done = ctx.sirt_iterate(x, _t(proj), 6)
    err = rel_l2(_np(x), x_ref)
    print(f"cylinder SIRT 6 iterations: rel.L2 {err:.3e}, residual {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert done == done_ref == 6
    assert err <= TOL32
    assert np.allclose(hist, hist_ref, rtol=1e-4)
    assert hist[-1] < 0.5 * hist[0]


def test_cylinder_bf16_volume(ct, small):
    cc, P, pb, vol, proj, rs = small
    ctx = ct.context_for_cylinder(cc, P=P)
    v16 = torch.as_tensor(vol).to(torch.bfloat16)
    ref, _ = oracle.forward(pb, v16.double().numpy())
    out = ctx.fwd_project(v16.cuda().contiguous(), out_dtype=torch.float32)
    e = rel_l2(_np(out), ref)
    print(f"cylinder forward, BF16 volume: rel.L2 {e:.3e}")
    assert e <= TOL32  # same rounded input on both sides, FP32 accumulation


def test_cylinder_error_paths(ct, small):
    cc, P, pb, vol, proj, rs = small
    ctx = ct.context_for_cylinder(cc, P=P)
    g = torch.zeros((cc.base.n_views,) + ctx.det_shape, device="cuda")
    with pytest.raises(ct.CtrexError):
        ctx.adjoint_project(g)
    th = torch.as_tensor(inputs.identity_theta(cc.base.n_views), dtype=torch.float32).cuda()
    with pytest.raises(ct.CtrexError):
        ctx.set_motion(th)
    b = cc.base
    bad = inputs.cylinder_pose(cc).copy()
    bad[0, 0] *= 1.01  # not a rotation
    for kw in (dict(pose=bad), dict(n_phi=2), dict(dr=0.0)):
        args = dict(n_r=cc.n_r, n_phi=cc.n_phi, n_z=cc.n_z, dr=cc.dr, dz=cc.dz, pose=inputs.cylinder_pose(cc))
        args.update(kw)
        c2 = ct.Context()
        with pytest.raises(ct.CtrexError):
            c2.set_geometry_cylinder(P, args["n_r"], args["n_phi"], args["n_z"], args["dr"], args["dz"],
                                     (b.nu, b.nv), pose=args["pose"])
    # switching back to a Cartesian grid restores the box projector
    cart = b
    ctx.set_geometry(P, cart.vol_shape, (cart.vox,) * 3, cart.origin, (cart.nu, cart.nv), cart.step_vox)
    ph = inputs.phantom(cart).numpy()
    from tests.helpers import oracle_problem

    ref, _ = oracle.forward(oracle_problem(cart, P=P), ph)
    assert rel_l2(_np(ctx.fwd_project(_t(ph))), ref) <= TOL32


def test_cylinder_vial_fullsize_sampled():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    cc = inputs.CYL_VIAL
    P = inputs.projection_matrices(cc.base)
    ctx = ctrex.context_for_cylinder(cc, P=P)
    vol = inputs.cyl_phantom(cc, device="cuda").to(torch.float32).contiguous()
    p = ctx.fwd_project(vol)
    pb = _problem(cc, P)
    vol64 = vol.double().cpu().numpy()
    rng = np.random.default_rng(256)
    n = 160
    views = rng.integers(0, cc.base.n_views, n).astype(np.int32)
    # pixels inside the vial's shadow (columns 25-75 %, rows 20-65 % of the detector)
    iu = rng.integers(cc.base.nu // 4, 3 * cc.base.nu // 4, n)
    iv = rng.integers(cc.base.nv // 5, 13 * cc.base.nv // 20, n)
    ref, _ = oracle.forward_rays(pb, vol64, views, iu.astype(float), iv.astype(float))
    del vol64
    got = p[torch.as_tensor(views, dtype=torch.long), torch.as_tensor(iv), torch.as_tensor(iu)]
    assert (ref > 0).sum() > 120
    e = rel_l2(got.double().cpu().numpy(), ref)
    print(f"vial forward, {n} sampled rays: rel.L2 {e:.3e}")
    assert e <= TOL32
    # one SIRT step's correction and backprojection at sampled voxels
    x = (0.9 * vol).contiguous()
    r, sums = ctx.fwd_correct(x, p)
    b = ctx.back_project(r, normalize=False, accumulate=False)
    vox = rng.integers(0, b.numel(), 32)
    r64 = r.double().cpu().numpy()
    b_ref, _ = oracle.backproject_voxels(pb, r64, vox)
    del r64
    eb = rel_l2(b.flatten()[torch.as_tensor(vox)].double().cpu().numpy(), b_ref)
    print(f"vial backprojection, sampled voxels: rel.L2 {eb:.3e}")
    assert eb <= TOL32
