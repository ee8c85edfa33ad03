"""Classical Joseph projector on the GPU against the FP64 oracle, element by
element through the C ABI: ragged anisotropic grids, rays of every principal
axis, sub-angles, the fused correction, SIRT, BF16 storage, and the
full-size workload on sampled rays."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

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


def _top_view(nu, nv, D=300.0, f=None):
    """A view from below the volume, on the z axis: its rays run mostly
    along z (the volume fills about 80 % of the detector)."""
    f = f or 6.0 * nu
    uc, vc = 0.5 * (nu - 1), 0.5 * (nv - 1)
    return np.array([[f, 0.0, uc, uc * D], [0.0, f, vc, vc * D], [0.0, 0.0, 1.0, D]])


def _ragged():
    """Anisotropic 37 x 29 x 23 grid, a perturbed circular scan plus two views
    along the z axis, so rays of all three principal axes occur."""
    cfg = inputs.CIRCULAR_64.scaled(name="perturbed-48x40-18v", nu=48, nv=40, n_views=16,
                                    trajectory="perturbed", seed=61)
    P = inputs.projection_matrices(cfg)[:, 0]
    P = np.concatenate([P, _top_view(cfg.nu, cfg.nv)[None], _top_view(cfg.nu, cfg.nv, D=260.0)[None]])
    shape, vox = (23, 29, 37), (0.9, 1.1, 1.3)
    origin = tuple(-0.5 * (n - 1) * v for n, v in zip((37, 29, 23), vox))
    vol = inputs.phantom(inputs.CIRCULAR_64.scaled(n=40)).numpy()[:23, :29, :37].copy()
    return cfg, P, shape, vox, origin, vol


def _ctx(ct, P, shape, vox, origin, det, step=0.5):
    c = ct.Context()
    c.set_geometry(P, shape, vox, origin, det, step)
    c.set_projector("joseph")
    return c


def test_joseph_forward_rowsum_count_ragged(ct):
    cfg, P, shape, vox, origin, vol = _ragged()
    pb = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv)).with_joseph()
    proj, rs = oracle.forward(pb, vol)
    c = _ctx(ct, P, shape, vox, origin, (cfg.nu, cfg.nv))
    rowsum = torch.empty(proj.shape, device="cuda")
    out = c.fwd_project(_t(vol), rowsum=rowsum)
    e, er = rel_l2(_np(out), proj), rel_l2(_np(rowsum), rs)
    print(f"Joseph forward (ragged, anisotropic, 3 principal axes) rel.L2 {e:.3e}, row sums {er:.3e}")
    assert e <= TOL32 and er <= TOL32
    for v in (16, 17):  # the views along z see the volume
        assert np.abs(proj[v]).max() > 0.1 * np.abs(proj).max()
    n_gpu, n_ref = c.count_samples(), oracle.count_samples(pb)
    print(f"Joseph slice crossings: GPU {n_gpu}, oracle {n_ref}")
    assert abs(n_gpu - n_ref) <= 1e-4 * n_ref
    # the trilinear projector gives different numbers on the same rays
    c.set_projector("trilinear")
    assert rel_l2(_np(c.fwd_project(_t(vol))), proj) > 1e-4


def test_joseph_subangles_correction_and_sirt(ct):
    cfg = inputs.CIRCULAR_64.scaled(name="circular-48^3-64^2-40v-S2", n=48, nu=64, nv=64, n_views=40, n_sub=2)
    P = inputs.projection_matrices(cfg)
    pb = oracle_problem(cfg, P=P).with_joseph()
    vol = inputs.phantom(cfg).numpy()
    proj, rs = oracle.forward(pb, vol)
    c = _ctx(ct, P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv))
    e = rel_l2(_np(c.fwd_project(_t(vol))), proj)
    print(f"Joseph forward with 2 sub-angles: rel.L2 {e:.3e}")
    assert e <= TOL32
    # fused correction
    x = 0.8 * vol
    q, rsx = oracle.forward(pb, x)
    r_ref, e2, p2 = oracle.correct(proj, q, rsx, pb.eps_R)
    r, sums = c.fwd_correct(_t(x), _t(proj))
    scale = np.where(rsx > pb.eps_R, proj / np.where(rsx > 0, rsx, 1.0), 0.0)
    err = float(np.linalg.norm(_np(r) - r_ref) / np.linalg.norm(scale))
    print(f"Joseph correction |dr| / |R p| = {err:.3e}")
    assert err <= TOL32
    assert np.allclose(_np(sums), [e2, p2], rtol=1e-4)
    # SIRT with the Joseph forward and the voxel-driven backprojector
    x_ref, hist_ref, done_ref, _ = oracle.sirt(pb, proj, 6)
    xg = torch.zeros(cfg.vol_shape, device="cuda")
    xg, hist, done = c.sirt_iterate(xg, _t(proj), 6)
    es = rel_l2(_np(xg), x_ref)
    print(f"Joseph SIRT 6 iterations: rel.L2 {es:.3e}, residual {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert done == done_ref == 6 and es <= TOL32
    assert np.allclose(hist, hist_ref, rtol=1e-4)


def test_joseph_bf16_volume(ct):
    cfg, P, shape, vox, origin, vol = _ragged()
    v16 = torch.as_tensor(vol).to(torch.bfloat16)
    pb = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv)).with_joseph()
    ref, _ = oracle.forward(pb, v16.double().numpy())
    c = _ctx(ct, P, shape, vox, origin, (cfg.nu, cfg.nv))
    out = c.fwd_project(v16.cuda().contiguous(), out_dtype=torch.float32)
    e = rel_l2(_np(out), ref)
    print(f"Joseph forward, BF16 volume: rel.L2 {e:.3e}")
    assert e <= TOL32


def test_joseph_state_errors(ct):
    cfg = inputs.CIRCULAR_64
    c = _ctx(ct, inputs.projection_matrices(cfg), cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv))
    g = torch.zeros((cfg.n_views, cfg.nv, cfg.nu), device="cuda")
    with pytest.raises(ct.CtrexError):
        c.adjoint_project(g)
    th = torch.as_tensor(inputs.identity_theta(cfg.n_views), dtype=torch.float32).cuda()
    with pytest.raises(ct.CtrexError):
        c.set_motion(th)
    with pytest.raises(KeyError):
        c.set_projector("siddon")
    with pytest.raises(ct.CtrexError):
        c._check(c.lib.ctrex_set_projector(c._h, 7))
    # the cylindrical domain resets to, and keeps, the trilinear projector
    cc = inputs.CYL_SMALL
    c.set_geometry_cylinder(inputs.projection_matrices(cc.base), cc.n_r, cc.n_phi, cc.n_z, cc.dr, cc.dz,
                            (cc.base.nu, cc.base.nv), pose=inputs.cylinder_pose(cc))
    with pytest.raises(ct.CtrexError):
        c.set_projector("joseph")
    # motion first, then Joseph: refused
    c2 = ct.context_for(cfg)
    c2.set_motion(th)
    with pytest.raises(ct.CtrexError):
        c2.set_projector("joseph")


def test_joseph_fullsize_sampled():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    cfg = inputs.PERTURBED_512
    P = inputs.projection_matrices(cfg)
    ctx = ctrex.context_for(cfg, P=P)
    ctx.set_projector("joseph")
    vol = inputs.phantom(cfg, device="cuda").to(torch.float32).contiguous()
    p = ctx.fwd_project(vol)
    pb = oracle_problem(cfg, P=P).with_joseph()
    vol64 = vol.double().cpu().numpy()
    rng = np.random.default_rng(512)
    n = 200
    views = rng.integers(0, cfg.n_views, n).astype(np.int32)
    iu = rng.integers(0, cfg.nu, n)
    iv = rng.integers(0, cfg.nv, n)
    ref, _ = oracle.forward_rays(pb, vol64, views, iu.astype(float), iv.astype(float))
    del vol64
    got = p[torch.as_tensor(views, dtype=torch.long), torch.as_tensor(iv), torch.as_tensor(iu)]
    assert (ref > 0).sum() > 100
    e = rel_l2(got.double().cpu().numpy(), ref)
    print(f"Joseph full size, {n} sampled rays: rel.L2 {e:.3e}")
    assert e <= TOL32
