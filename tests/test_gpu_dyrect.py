"""Event-based 4D model (Sec. 3.3: initial values, final values and a
transition time per voxel) on the GPU against the FP64 oracle, element by
element through the C ABI: projection and row sums, the fused correction,
the split backprojection with weights and relaxation, the adjoint with
respect to both value fields, SIRT, BF16 storage, and sampled rays and
voxels of the 512^3 bench workload."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import rel_l2

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


def _t(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dtype).cuda().contiguous()


def _np(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture(scope="module")
def scene():
    # 40^3 (not a multiple of the 32 x 4 x 4 backprojection tiles: ragged
    # edges), perturbed views, 10 changing regions
    cfg = inputs.CIRCULAR_64.scaled(name="dyrect-40^3-56x48-30v", n=40, nu=56, nv=48, n_views=30,
                                    trajectory="perturbed", seed=17)
    P = inputs.projection_matrices(cfg)
    mu0, mu1, tau = (f.numpy() for f in inputs.dyrect_fields(cfg, n_events=10))
    tv = inputs.view_times(cfg)
    # the GPU holds tau in FP32: the oracle takes the same values
    tau = tau.astype(np.float32).astype(np.float64)
    tv = tv.astype(np.float32).astype(np.float64)
    pb = oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)
    return cfg, P, np.stack([mu0, mu1]), tau, tv, pb.with_dyrect(tau, tv)


def _ctx(ct, cfg, P, tau, tv):
    c = ct.context_for(cfg, P=P)
    c.set_dyrect(_t(tau), _t(tv))
    return c


def test_dyrect_forward_rowsum_and_correction(ct, scene):
    cfg, P, x, tau, tv, pb = scene
    c = _ctx(ct, cfg, P, tau, tv)
    proj, rs = oracle.forward(pb, x)
    rowsum = torch.empty(proj.shape, device="cuda")
    out = c.fwd_project(_t(x), rowsum=rowsum)
    e, er = rel_l2(_np(out), proj), rel_l2(_np(rowsum), rs)
    # the frames differ: the model is exercised, not the static projector
    stat, _ = oracle.forward(oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv),
                                            cfg.step_vox), x[0])
    print(f"event-model forward rel.L2 {e:.3e}, row sums {er:.3e} (differs from the mu0 projection by "
          f"{rel_l2(proj, stat):.2e})")
    assert rel_l2(proj, stat) > 1e-2
    assert e <= TOL32 and er <= TOL32
    x0 = 0.8 * x
    q, rsx = oracle.forward(pb, x0)
    r_ref, e2, p2 = oracle.correct(proj, q, rsx, pb.eps_R)
    r, sums = c.fwd_correct(_t(x0), _t(proj))
    scale = np.where(rsx > pb.eps_R, proj / np.where(rsx > 0, rsx, 1.0), 0.0)
    err = float(np.linalg.norm(_np(r) - r_ref) / np.linalg.norm(scale))
    print(f"event-model correction |dr| / |R p| = {err:.3e}")
    assert err <= TOL32 and np.allclose(_np(sums), [e2, p2], rtol=1e-4)
    c.close()


def test_dyrect_backprojection_weights_and_adjoint(ct, scene):
    cfg, P, x, tau, tv, pb = scene
    c = _ctx(ct, cfg, P, tau, tv)
    rng = np.random.default_rng(11)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    w = rng.uniform(0.3, 1.0, size=x.shape)
    x0 = rng.uniform(size=x.shape)
    x1, b, cc = oracle.backproject(pb, r, w=w, alpha=0.8, x=x0)
    got = c.back_project(_t(r), vol=_t(x0), w=_t(w), alpha=0.8, normalize=True, accumulate=True)
    e = rel_l2(_np(got) - x0, x1 - x0)
    assert (b[0] != 0).sum() > 0 and (b[1] != 0).sum() > 0
    # unnormalised, overwriting: b itself
    gb = c.back_project(_t(r), vol=torch.zeros(x.shape, device="cuda"), alpha=1.0, normalize=False,
                        accumulate=False)
    eb = rel_l2(_np(gb), b)
    y = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    adj = c.adjoint_project(_t(y))
    ea = rel_l2(_np(adj), oracle.adjoint(pb, y))
    print(f"event-model BP update rel.L2 {e:.3e}, b {eb:.3e}, adjoint {ea:.3e}")
    assert e <= TOL32 and eb <= TOL32 and ea <= TOL32
    c.close()


def test_dyrect_sirt_and_bf16(ct, scene):
    cfg, P, x, tau, tv, pb = scene
    c = _ctx(ct, cfg, P, tau, tv)
    proj, _ = oracle.forward(pb, x)
    x_ref, hist_ref, done_ref, _ = oracle.sirt(pb, proj, 6)
    xg = torch.zeros(x.shape, device="cuda")
    xg, hist, done = c.sirt_iterate(xg, _t(proj), 6)
    e = rel_l2(_np(xg), x_ref)
    print(f"event-model SIRT 6 iterations rel.L2 {e:.3e}; residual {hist[-1]:.4e} (oracle {hist_ref[-1]:.4e})")
    assert done == done_ref == 6 and e <= TOL32
    assert np.allclose(hist, hist_ref, rtol=1e-4)
    # BF16 storage of both value fields, FP32 accumulation: against the
    # oracle on the same BF16-rounded inputs
    x16 = _t(x, torch.bfloat16)
    want, _ = oracle.forward(pb, _np(x16))
    got = c.fwd_project(x16, out_dtype=torch.float32)
    e16 = rel_l2(_np(got), want)
    print(f"event-model BF16 volume forward rel.L2 {e16:.3e}")
    assert e16 <= TOL32
    c.close()


def test_dyrect_brick_shortcut_paths(ct, scene):
    """The per-brick shortcut of the projector: with one transition time for
    the whole volume every interior footprint takes one field (mu0 for the
    views before it, mu1 after), which must give the static projections of
    those fields; with NaN transition times in a few voxels (their taps take
    mu1, t < NaN being false) their bricks take the per-tap path, and the
    result must still match the oracle."""
    cfg, P, x, tau, tv, pb = scene
    t_mid = float(np.float32(0.5 * (tv[14] + tv[15])))
    c = _ctx(ct, cfg, P, np.full_like(tau, t_mid), tv)
    got = _np(c.fwd_project(_t(x)))
    st = ct.context_for(cfg, P=P)
    p0, p1 = _np(st.fwd_project(_t(x[0]))), _np(st.fwd_project(_t(x[1])))
    e0, e1 = rel_l2(got[:15], p0[:15]), rel_l2(got[15:], p1[15:])
    print(f"uniform transition time: early views vs static mu0 {e0:.2e}, late views vs static mu1 {e1:.2e}")
    assert e0 <= 1e-6 and e1 <= 1e-6
    c.close()
    st.close()
    tau_nan = tau.copy()
    rng = np.random.default_rng(3)
    idx = rng.integers(0, tau.size, size=40)
    tau_nan.flat[idx] = np.nan
    c = _ctx(ct, cfg, P, tau_nan, tv)
    ref, _ = oracle.forward(oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv),
                                           cfg.step_vox).with_dyrect(tau_nan, tv), x)
    e = rel_l2(_np(c.fwd_project(_t(x))), ref)
    print(f"NaN transition times in 40 voxels: forward vs oracle {e:.2e}")
    assert e <= TOL32
    c.close()


def test_dyrect_refusals(ct, scene):
    cfg, P, x, tau, tv, pb = scene
    c = _ctx(ct, cfg, P, tau, tv)
    f = lambda a: torch.as_tensor(a, dtype=torch.float32).cuda().contiguous()  # noqa: E731
    th, co, sv = inputs.motion_params(cfg.scaled(motion=True, margin=0.5))
    for call in (lambda: c.set_motion(f(th), f(co), f(sv), 0.5), lambda: c.set_bp_subvoxel(2),
                 lambda: c.set_projector("joseph"), lambda: c.set_roi((8, 8, 8), (0.2,) * 3, (0.0,) * 3)):
        with pytest.raises(ct.CtrexError) as ei:
            call()
        assert ei.value.code == -9  # CTREX_E_STATE
    c.set_dyrect(None)
    assert c.vol_shape == cfg.vol_shape
    c.close()


def test_dyrect_fullsize_sampled(ct):
    """The bench's event workload: the perturbed 512^3 geometry with the
    event scene; sampled rays of every part of the detector and sampled
    voxels of the whole volume against the oracle."""
    cfg = inputs.PERTURBED_512
    P = inputs.projection_matrices(cfg)
    mu0, mu1, tau = inputs.dyrect_fields(cfg, device="cuda")
    tv = inputs.view_times(cfg)
    c = ct.context_for(cfg, P=P)
    tau32 = tau.to(torch.float32).contiguous()
    tv32 = torch.as_tensor(tv, dtype=torch.float32, device="cuda")
    c.set_dyrect(tau32, tv32)
    x = torch.stack([mu0, mu1]).to(torch.float32).contiguous()
    del mu0, mu1
    proj = c.fwd_project(x)
    x64 = _np(x)
    pb = oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)
    pb = pb.with_dyrect(_np(tau32), tv.astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(912)
    views = rng.integers(0, cfg.n_views, size=200).astype(np.int32)
    iu = rng.integers(0, cfg.nu, size=200)
    iv = rng.integers(0, cfg.nv, size=200)
    ref, _ = oracle.forward_rays(pb, x64, views, iu.astype(float), iv.astype(float))
    got = proj[torch.as_tensor(views, dtype=torch.long), torch.as_tensor(iv), torch.as_tensor(iu)]
    e = rel_l2(_np(got), ref)
    # backprojection of the workload's own correction images at sampled
    # voxels, both value fields (not white noise: at u ~ 768 an FP32 detector
    # coordinate resolves ~5e-5 pixel, which bilinear samples of noise turn
    # into a relative error of that size)
    r, _ = c.fwd_correct((0.8 * x).contiguous(), proj)
    b = c.back_project(r, vol=torch.zeros(x.shape, device="cuda"), normalize=False, accumulate=False)
    vox = rng.integers(0, cfg.n ** 3, size=24)
    bv_ref, _ = oracle.backproject_voxels(pb, _np(r), vox)
    bv = _np(b).reshape(2, -1)[:, vox]
    eb = rel_l2(bv, bv_ref)
    print(f"event model, 512^3 x 720 views: 200 sampled rays rel.L2 {e:.3e}; 24 sampled voxels (both fields) "
          f"{eb:.3e}")
    assert (ref > 0).sum() > 50
    assert e <= TOL32 and eb <= TOL32
    c.close()
