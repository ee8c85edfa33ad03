"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check is a closed form, an
analytic line integral, an identity of the operators (adjointness, partition of
unity, linearity), an invariance of the projection-matrix formulation
(Sec. 2.2), brute force on an 8^3 grid, or finite differences.  A plausible
slip in the oracle (dropped term, wrong sign, swapped axis, transposed matrix)
fails at least one of them.
"""

import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, ray_points, rel_l2


def small(cfg=None, **kw):
    base = inputs.CIRCULAR_64 if cfg is None else cfg
    return base.scaled(**kw)


# ---------------------------------------------------------------------------
# P1: closed form for axis-aligned rays through a row of voxel centres
# ---------------------------------------------------------------------------

def _row_closed_form(row, vox):
    # truncated-midpoint samples at index -1/4, 1/4, ..., N - 3/4 with weight vox/2
    return vox * (row.sum() - (row[0] + row[-1]) / 8.0)


@pytest.mark.parametrize("n", [9, 13])
def test_p1_axis_rays_closed_form(n):
    cfg = small(n=n, nu=n, nv=n, n_views=4)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(11)
    vol = rng.uniform(0.0, 1.0, size=cfg.vol_shape)
    proj, rs = oracle.forward(pb, vol)
    c = (n - 1) // 2
    # view 0: source on -x, central ray along +x through row (z=c, y=c)
    assert proj[0, c, c] == pytest.approx(_row_closed_form(vol[c, c, :], cfg.vox), rel=1e-13)
    # view 1: angle 90 deg, central ray along +y through column (z=c, x=c)
    assert proj[1, c, c] == pytest.approx(_row_closed_form(vol[c, :, c], cfg.vox), rel=1e-13)
    # all-ones volume: row sum = vox (N - 1/4)
    assert rs[0, c, c] == pytest.approx(cfg.vox * (n - 0.25), rel=1e-13)
    # off-centre detector rows through voxel-centre rows are not axis aligned;
    # the central column of view 0 with an all-ones volume obeys the same rule
    ones_proj, _ = oracle.forward(pb, np.ones(cfg.vol_shape))
    assert ones_proj[0, c, c] == pytest.approx(cfg.vox * (n - 0.25), rel=1e-13)


def test_p1_z_ray_closed_form():
    n = 11
    cfg = small(n=n, nu=n, nv=n, n_views=1)
    pitch = cfg.pitch
    P = inputs.cone_matrix([0.0, 0.0, -inputs.SOD], [0.0, 0.0, inputs.SDD - inputs.SOD],
                           [pitch, 0.0, 0.0], [0.0, pitch, 0.0], n, n)
    pb = oracle_problem(cfg, P=P[None, None])
    rng = np.random.default_rng(12)
    vol = rng.uniform(0.0, 1.0, size=cfg.vol_shape)
    proj, _ = oracle.forward(pb, vol)
    c = (n - 1) // 2
    assert proj[0, c, c] == pytest.approx(_row_closed_form(vol[:, c, c], cfg.vox), rel=1e-13)


# ---------------------------------------------------------------------------
# P2: analytic ellipsoid line integrals (chord length x density)
# ---------------------------------------------------------------------------

def _analytic_ellipsoids(cfg, ells, views):
    out = []
    for view in views:
        s, pix = ray_points(cfg, view)
        d = pix - s
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        tot = np.zeros(pix.shape[:2])
        for e in ells:
            Q = (e.rot / e.semi_axes[None, :]).T       # q = Q (x - c)
            a0 = (s - e.centre) @ Q.T                   # [3]
            a1 = d @ Q.T                                # [nv, nu, 3]
            A = (a1 * a1).sum(-1)
            B = 2.0 * (a1 * a0).sum(-1)
            C = (a0 * a0).sum() - 1.0
            disc = B * B - 4 * A * C
            chord = np.where(disc > 0, np.sqrt(np.maximum(disc, 0)) / A, 0.0)
            tot += e.density * chord
        out.append(tot)
    return np.stack(out)


def test_p2_ellipsoid_chords_converge():
    errs = []
    for n in (64, 128):
        cfg = small(n=n, n_views=6)
        ells, blobs = inputs.draw_objects(cfg)
        vol = inputs.voxelize(cfg, ells, blobs).numpy()
        pb = oracle_problem(cfg)
        proj, _ = oracle.forward(pb, vol)
        ref = _analytic_ellipsoids(cfg, ells, range(cfg.n_views))
        errs.append(rel_l2(proj, ref))
    assert errs[0] <= 2e-2, errs
    assert errs[0] / errs[1] >= 1.7, errs


# ---------------------------------------------------------------------------
# P3: analytic Gaussian line integral (erf), second-order convergence
# ---------------------------------------------------------------------------

def _gauss_line(s, d, blob, t0, t1):
    c = blob.centre
    tc = (c - s) @ d
    b2 = ((c - s) ** 2).sum() - tc * tc
    sg = blob.sigma
    k = blob.amplitude * math.exp(-0.5 * b2 / (sg * sg)) * sg * math.sqrt(math.pi / 2)
    return k * (erf((t1 - tc) / (sg * math.sqrt(2))) - erf((t0 - tc) / (sg * math.sqrt(2))))


def test_p3_gaussian_blob_second_order():
    """Ray through the centre of an isotropic Gaussian, nearly along x.

    Leading-order error of (voxel average over 4^3 sub-samples) + (trilinear
    interpolation) + (truncated-midpoint quadrature) relative to the exact erf
    integral: along the ray both the voxel smoothing and the quadrature of the
    piecewise-linear interpolant integrate to zero; across the ray the
    projected Gaussian G is box-smoothed in y and z (factor 1 - 2 h^2 / 24 s^2)
    and bilinearly interpolated at fractional offsets (fy, fz) (error
    -fy(1-fy) h^2 / 2s^2 - fz(1-fz) h^2 / 2s^2).  So
        rel.err = -(h/s)^2 [1/12 + (fy(1-fy) + fz(1-fz)) / 2] + O(h^4).
    """
    blob = inputs.Blob(np.array([0.7, -0.4, 0.3]), 3.0, 1.0)
    for n in (32, 64, 128):
        cfg = small(n=n, nu=48, nv=48, n_views=1, n_ellipsoids=0)
        vol = inputs.voxelize(cfg, [], [blob]).numpy()
        pb = oracle_problem(cfg)
        srcs, ctrs, ua, va = inputs.detector_frames(cfg)
        s = srcs[0, 0]
        # detector point on the line source -> blob centre (trajectory definition)
        d = blob.centre - s
        d /= np.linalg.norm(d)
        nrm = np.cross(ua[0, 0], va[0, 0])
        d0 = ctrs[0, 0] - 0.5 * (cfg.nu - 1) * ua[0, 0] - 0.5 * (cfg.nv - 1) * va[0, 0]
        hit = s + d * (((d0 - s) @ nrm) / (d @ nrm)) - d0
        u = hit @ ua[0, 0] / (ua[0, 0] @ ua[0, 0])
        v = hit @ va[0, 0] / (va[0, 0] @ va[0, 0])
        val, _ = oracle.forward_rays(pb, vol, [0], [u], [v])
        exact = _gauss_line(s, d, blob, -1e3, 1e3)
        err = val[0] / exact - 1.0
        g = (blob.centre - np.array(cfg.origin)) / cfg.vox
        fy, fz = g[1] - math.floor(g[1]), g[2] - math.floor(g[2])
        pred = -(cfg.vox / blob.sigma) ** 2 * (1.0 / 12.0 + 0.5 * (fy * (1 - fy) + fz * (1 - fz)))
        assert abs(err - pred) <= 0.1 * abs(pred), (n, err, pred)


def test_p3_gaussian_blob_detector():
    """Whole detector, sigma = 6 voxels: second-order error below 1e-2."""
    cfg = small(n=64, nu=48, nv=48, n_views=2, n_ellipsoids=0)
    blob = inputs.Blob(np.array([0.7, -0.4, 0.3]), 3.0, 1.0)
    vol = inputs.voxelize(cfg, [], [blob]).numpy()
    proj, _ = oracle.forward(oracle_problem(cfg), vol)
    ref = np.zeros_like(proj)
    for view in range(cfg.n_views):
        s, pix = ray_points(cfg, view)
        for iv in range(cfg.nv):
            for iu in range(cfg.nu):
                d = pix[iv, iu] - s
                d /= np.linalg.norm(d)
                ref[view, iv, iu] = _gauss_line(s, d, blob, -1e3, 1e3)
    assert rel_l2(proj, ref) <= 1e-2


# ---------------------------------------------------------------------------
# P4: adjoint dot-product test <Ax, y> = <x, A^T y>
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["plain", "subangles", "motion", "perturbed"])
def test_p4_adjoint_dot_product(variant):
    rng = np.random.default_rng(4)
    if variant == "plain":
        cfg = small(n=16, nu=20, nv=18, n_views=5)
        pb = oracle_problem(cfg)
    elif variant == "subangles":
        cfg = small(n=16, nu=20, nv=18, n_views=5, n_sub=3)
        pb = oracle_problem(cfg)
    elif variant == "perturbed":
        cfg = small(n=16, nu=20, nv=18, n_views=5, trajectory="perturbed", seed=7)
        pb = oracle_problem(cfg)
    else:
        cfg = small(inputs.MOTION_FD_32, n=16, nu=20, nv=18, n_views=5)
        th, co, sv = inputs.motion_params(cfg)
        pb = oracle_problem(cfg, theta=th, coef=co, s_view=sv)
    x = rng.normal(size=cfg.vol_shape)
    y = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    Ax, _ = oracle.forward(pb, x)
    ATy = oracle.adjoint(pb, y)
    lhs, rhs = float((Ax * y).sum()), float((x * ATy).sum())
    scale = np.linalg.norm(Ax) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale


# ---------------------------------------------------------------------------
# P5: brute force on an 8^3 grid
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def dense8():
    cfg = small(n=8, nu=10, nv=9, n_views=4, trajectory="perturbed", seed=5)
    pb = oracle_problem(cfg)
    nvox = 8 ** 3
    nray = cfg.n_views * cfg.nv * cfg.nu
    A = np.zeros((nray, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = oracle.forward(pb, e.reshape(cfg.vol_shape))[0].ravel()
    B = np.zeros((nvox, nray))
    for i in range(nray):
        e = np.zeros(nray)
        e[i] = 1.0
        B[:, i] = oracle.backproject(pb, e.reshape(cfg.n_views, cfg.nv, cfg.nu))[1].ravel()
    return cfg, pb, A, B


def test_p5_dense_adjoint_is_transpose(dense8):
    cfg, pb, A, _ = dense8
    nray = A.shape[0]
    AT = np.zeros((A.shape[1], nray))
    for i in range(0, nray, 1):
        e = np.zeros(nray)
        e[i] = 1.0
        AT[:, i] = oracle.adjoint(pb, e.reshape(cfg.n_views, cfg.nv, cfg.nu)).ravel()
    assert np.max(np.abs(AT - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert (A >= 0).all() and A.sum() > 0


def test_p5_linearity_and_rowsum(dense8):
    cfg, pb, A, _ = dense8
    rng = np.random.default_rng(5)
    x = rng.normal(size=cfg.vol_shape)
    Ax, rs = oracle.forward(pb, x)
    assert np.allclose(Ax.ravel(), A @ x.ravel(), rtol=0, atol=1e-12 * np.abs(Ax).max())
    assert np.allclose(rs.ravel(), A.sum(axis=1), rtol=0, atol=1e-13)


def test_p5_backprojector_column_sums(dense8):
    cfg, pb, _, B = dense8
    _, _, c = oracle.backproject(pb, np.ones((cfg.n_views, cfg.nv, cfg.nu)))
    assert np.allclose(c.ravel(), B.sum(axis=1), atol=1e-13)
    assert (B >= 0).all()


def _frame_projection(frame, X):
    """Detector coordinates (u, v) of points X [..., 3] and whether each lies
    in front of the source, by line/plane intersection with the detector
    plane of one frame (s, d0, u_axis, v_axis): no projection matrix."""
    s, d0, ua, va = frame
    nrm = np.cross(ua, va)
    den = (X - s) @ nrm
    t = ((d0 - s) @ nrm) / np.where(den == 0, np.inf, den)
    rel = s + t[..., None] * (X - s) - d0
    G = np.array([[ua @ ua, ua @ va], [ua @ va, va @ va]])
    uv = np.linalg.solve(G, np.stack([rel @ ua, rel @ va], axis=-1)[..., None])[..., 0]
    return uv[..., 0], uv[..., 1], t > 0


def _dense_bp_independent(frames, shape, vox, origin, nu, nv):
    """Dense backprojector B [voxels, rays] from its definition (Sec. 4.1
    backprojection operator, reading R4): the voxel centre projected through
    each (view, sub-angle) frame, bilinear weights on the four neighbouring
    pixels, pixels outside [0, nu-1] x [0, nv-1] and points behind the source
    contributing nothing, each sub-angle weighted 1/S.  Also returns how many
    (voxel, frame) footprints straddle the detector edge."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([origin[0] + X * vox[0], origin[1] + Y * vox[1], origin[2] + Z * vox[2]], -1).reshape(-1, 3)
    n_views, n_sub = len(frames), len(frames[0])
    B = np.zeros((len(pts), n_views * nv * nu))
    straddle = total = 0
    for k in range(n_views):
        for sub in range(n_sub):
            u, v, front = _frame_projection(frames[k][sub], pts)
            for j in range(len(pts)):
                if not front[j]:
                    continue
                iu0, iv0 = math.floor(u[j]), math.floor(v[j])
                fu, fv = u[j] - iu0, v[j] - iv0
                inside = 0
                for dv, wv in ((0, 1.0 - fv), (1, fv)):
                    for du, wu in ((0, 1.0 - fu), (1, fu)):
                        iu, iv = iu0 + du, iv0 + dv
                        if 0 <= iu <= nu - 1 and 0 <= iv <= nv - 1:
                            inside += 1
                            B[j, (k * nv + iv) * nu + iu] += wu * wv / n_sub
                total += 1
                straddle += 0 < inside < 4
    return B, straddle, total


def _dense_bp_oracle(pb, n_views):
    nray = n_views * pb.nv * pb.nu
    B = np.zeros((pb.nx * pb.ny * pb.nz, nray))
    for i in range(nray):
        e = np.zeros(nray)
        e[i] = 1.0
        B[:, i] = oracle.backproject(pb, e.reshape(n_views, pb.nv, pb.nu))[1].ravel()
    return B


def test_p5_backprojector_equals_independent_dense_definition():
    # A detector narrower than the projected volume, so that many footprints
    # cross its edges, with perturbed views and two sub-angles per view.
    cfg = small(n=8, nu=5, nv=4, n_views=3, trajectory="perturbed", seed=5, det_width=40.0)
    srcs, ctrs, us, vs = inputs.detector_frames(cfg)
    P1 = inputs.projection_matrices(cfg)
    # second sub-angle: the same frame rotated by 7 degrees about z
    Rz = inputs.rot_z(math.radians(7.0))
    frames, P = [], np.zeros((cfg.n_views, 2, 3, 4))
    for k in range(cfg.n_views):
        f = []
        for sub, R in enumerate((np.eye(3), Rz)):
            s, c, ua, va = R @ srcs[k, 0], R @ ctrs[k, 0], R @ us[k, 0], R @ vs[k, 0]
            d0 = c - 0.5 * (cfg.nu - 1) * ua - 0.5 * (cfg.nv - 1) * va
            f.append((s, d0, ua, va))
            P[k, sub] = inputs.cone_matrix(s, c, ua, va, cfg.nu, cfg.nv)
        frames.append(f)
    assert np.allclose(P[:, 0], P1[:, 0])
    pb = oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)
    B_ind, straddle, total = _dense_bp_independent(frames, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin,
                                                   cfg.nu, cfg.nv)
    assert straddle >= 0.2 * total
    B = _dense_bp_oracle(pb, cfg.n_views)
    assert np.max(np.abs(B - B_ind)) <= 1e-13
    _, _, c = oracle.backproject(pb, np.ones((cfg.n_views, cfg.nv, cfg.nu)))
    assert np.allclose(c.ravel(), B_ind.sum(axis=1), rtol=0, atol=1e-13)


def test_p5_backprojector_skips_points_behind_the_source():
    # Sources inside the volume: the voxels behind each source get nothing
    # from that view (depth <= 0), the rest follow the bilinear definition.
    shape, vox, nu, nv = (8, 8, 8), (4.0, 4.0, 4.0), 12, 11
    origin = (-14.0, -14.0, -14.0)
    frames, P = [], []
    for ang, src in ((0.0, (-3.0, 0.5, 0.2)), (2.1, (1.5, -2.5, -0.7))):
        R = inputs.rot_z(ang)
        s = R @ np.array([src[0], 0.0, 0.0]) + np.array([0.0, src[1], src[2]])
        c = s + R @ np.array([60.0, 0.0, 0.0])
        ua, va = R @ np.array([0.0, 6.0, 0.0]), np.array([0.0, 0.0, 6.0])
        d0 = c - 0.5 * (nu - 1) * ua - 0.5 * (nv - 1) * va
        frames.append([(s, d0, ua, va)])
        P.append(inputs.cone_matrix(s, c, ua, va, nu, nv)[None])
    P = np.stack(P)
    pb = oracle.Problem(P, shape, vox, origin, (nu, nv), 0.5)
    B_ind, _, _ = _dense_bp_independent(frames, shape, vox, origin, nu, nv)
    Z, Y, X = np.meshgrid(*(np.arange(8),) * 3, indexing="ij")
    pts = np.stack([origin[0] + X * 4.0, origin[1] + Y * 4.0, origin[2] + Z * 4.0], -1).reshape(-1, 3)
    behind = ~_frame_projection(frames[0][0], pts)[2]
    assert 0.2 * len(pts) < behind.sum() < 0.8 * len(pts)
    B = _dense_bp_oracle(pb, 2)
    assert np.max(np.abs(B - B_ind)) <= 1e-13
    assert not B[behind, : nu * nv].any()


def test_p5_sirt_step_is_dense_formula(dense8):
    cfg, pb, A, B = dense8
    rng = np.random.default_rng(6)
    x0 = rng.uniform(0, 1, size=cfg.vol_shape)
    p = A @ rng.uniform(0, 1, size=A.shape[1])
    w = rng.uniform(0.2, 1.0, size=cfg.vol_shape)
    alpha = 0.7
    rowsum = A.sum(axis=1)
    R = np.where(rowsum > pb.eps_R, 1.0 / np.where(rowsum > 0, rowsum, 1), 0.0)
    colsum = B.sum(axis=1)
    C = np.where(colsum > oracle.EPS_C, 1.0 / np.where(colsum > 0, colsum, 1), 0.0)
    expect = x0.ravel() + alpha * w.ravel() * C * (B @ (R * (p - A @ x0.ravel())))
    x1, hist, done, ret = oracle.sirt(pb, p.reshape(cfg.n_views, cfg.nv, cfg.nu), 1, alpha=alpha,
                                      w=w, x0=x0)
    assert done == 1 and ret == 0
    assert np.allclose(x1.ravel(), expect, rtol=0, atol=1e-12)
    rho = np.linalg.norm(p - A @ x0.ravel()) / np.linalg.norm(p)
    assert hist[0] == pytest.approx(rho, rel=1e-12)


# ---------------------------------------------------------------------------
# P6: invariances of the projection-matrix formulation (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_p6_scale_invariance_and_sign():
    cfg = small(n=16, nu=20, nv=20, n_views=4, trajectory="perturbed", seed=3)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(7)
    vol = rng.uniform(size=cfg.vol_shape)
    ref, rs = oracle.forward(pb, vol)
    for kappa in (-2.5, 3.0, -1e-3):
        got, rs2 = oracle.forward(pb.with_P(pb.P * kappa), vol)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * ref.max())
        assert np.allclose(rs2, rs, rtol=0, atol=1e-12 * rs.max())
    r = rng.normal(size=ref.shape)
    _, b1, c1 = oracle.backproject(pb, r)
    _, b2, c2 = oracle.backproject(pb.with_P(pb.P * -4.0), r)
    assert np.allclose(b1, b2, atol=1e-12) and np.allclose(c1, c2, atol=1e-12)


def test_p6_rotation_about_z():
    cfg = small(n=16, nu=24, nv=20, n_views=3, trajectory="perturbed", seed=9)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(8)
    vol = rng.uniform(size=cfg.vol_shape)
    # rotate content by +90 deg about z: new(x, y) = old(y, -x)
    vol_r = np.ascontiguousarray(vol[:, ::-1, :].transpose(0, 2, 1))
    Rz = inputs.rot_z(math.pi / 2)
    P2 = pb.P.copy()
    P2[..., :3] = pb.P[..., :3] @ Rz.T
    ref, _ = oracle.forward(pb, vol)
    got, _ = oracle.forward(pb.with_P(P2), vol_r)
    assert np.allclose(got, ref, rtol=0, atol=1e-11 * ref.max())
    # the backprojector commutes with the same rotation
    r = rng.normal(size=ref.shape)
    _, b1, _ = oracle.backproject(pb, r)
    _, b2, _ = oracle.backproject(pb.with_P(P2), r)
    b1_r = b1[:, ::-1, :].transpose(0, 2, 1)
    assert np.allclose(b2, b1_r, rtol=0, atol=1e-11 * np.abs(b1).max())


def test_p6_view_order_and_linearity():
    cfg = small(n=16, nu=20, nv=20, n_views=5, trajectory="perturbed", seed=10)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(9)
    x, y = rng.uniform(size=cfg.vol_shape), rng.uniform(size=cfg.vol_shape)
    ref, _ = oracle.forward(pb, x)
    perm = np.array([3, 0, 4, 1, 2])
    got, _ = oracle.forward(pb, x, views=perm)
    assert np.array_equal(got, ref[perm])
    ay, _ = oracle.forward(pb, y)
    axy, _ = oracle.forward(pb, 2.0 * x - 3.0 * y)
    assert np.allclose(axy, 2.0 * ref - 3.0 * ay, atol=1e-12 * np.abs(axy).max())


# ---------------------------------------------------------------------------
# P7: special cases of the motion model (Sec. 2.2.2, Sec. 3.1, Sec. 3.4)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def motion_case():
    cfg = small(inputs.MOTION_FD_32, n=16, nu=20, nv=20, n_views=4)
    rng = np.random.default_rng(10)
    vol = np.zeros(cfg.vol_shape)
    vol[4:12, 4:12, 4:12] = rng.uniform(size=(8, 8, 8))  # interior content
    return cfg, vol


def test_p7_identity_motion_is_static(motion_case):
    cfg, vol = motion_case
    ref, rs = oracle.forward(oracle_problem(cfg), vol)
    pb = oracle_problem(cfg, theta=inputs.identity_theta(cfg.n_views), coef=np.zeros((8, 8, 8, 3)),
                        s_view=np.ones(cfg.n_views))
    pb0 = pb.with_motion(pb.theta, pb.coef, pb.s_view, margin=0.0)
    got, rs2 = oracle.forward(pb0, vol)
    assert np.array_equal(got, ref) and np.array_equal(rs2, rs)


def test_p7_constant_coefficients_are_translation(motion_case):
    cfg, vol = motion_case
    shift = np.array([2.0, -1.0, 1.0]) * cfg.vox          # whole voxels (x, y, z)
    coef = np.broadcast_to(shift, (8, 8, 8, 3)).copy()
    th = inputs.identity_theta(cfg.n_views)
    pb_c = oracle_problem(cfg, theta=th, coef=coef, s_view=np.ones(cfg.n_views))
    th_t = th.copy()
    th_t[:, 3:6] = shift
    pb_t = oracle_problem(cfg, theta=th_t, coef=np.zeros((8, 8, 8, 3)), s_view=np.ones(cfg.n_views))
    a, _ = oracle.forward(pb_c, vol)
    b, _ = oracle.forward(pb_t, vol)
    assert np.allclose(a, b, rtol=0, atol=1e-12 * a.max())
    # sampling mu(x + shift) equals sampling the volume shifted by -shift
    shifted = np.zeros_like(vol)
    shifted[3:11, 5:13, 2:10] = vol[4:12, 4:12, 4:12]      # z-1, y+1, x-2 voxels
    pb_s = oracle_problem(cfg, theta=th, coef=np.zeros((8, 8, 8, 3)), s_view=np.ones(cfg.n_views))
    c, _ = oracle.forward(pb_s, shifted)
    assert np.allclose(a, c, rtol=0, atol=1e-12 * a.max())


def test_p7_rotation_and_affine_conventions(motion_case):
    cfg, vol = motion_case
    zero = np.zeros((8, 8, 8, 3))
    # omega = (0, 0, pi/2): sampling mu(R x) equals sampling a rotated copy
    th = inputs.identity_theta(cfg.n_views)
    th[:, 2] = math.pi / 2
    a, _ = oracle.forward(oracle_problem(cfg, theta=th, coef=zero, s_view=np.zeros(cfg.n_views)), vol)
    # R (x, y) = (-y, x): new[z, iy, ix] = old at (-y, x) = old[z, ix, N-1-iy]
    vol_r = np.ascontiguousarray(vol[:, :, ::-1].transpose(0, 2, 1))
    pb_s = oracle_problem(cfg, theta=inputs.identity_theta(cfg.n_views), coef=zero,
                          s_view=np.zeros(cfg.n_views))
    b, _ = oracle.forward(pb_s, vol_r)
    assert np.allclose(a, b, rtol=0, atol=1e-11 * a.max())
    # A = permutation swapping x and y: mu(A x) = transposed volume
    th2 = inputs.identity_theta(cfg.n_views)
    th2[:, 6:15] = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]], float).reshape(9)
    c, _ = oracle.forward(oracle_problem(cfg, theta=th2, coef=zero, s_view=np.zeros(cfg.n_views)), vol)
    d, _ = oracle.forward(pb_s, np.ascontiguousarray(vol.transpose(0, 2, 1)))
    assert np.allclose(c, d, rtol=0, atol=1e-12 * c.max())


def test_p7_bspline_control_grid_reproduces_linear_fields():
    """Sec. 3.1 deformation on an 8^3 control grid, reading R6: point i of
    axis a sits at box_min_a + (i - 1) * box_a / 5.  A cubic B-spline
    reproduces linear functions, so coefficients c_i = a + G x_i (x_i the
    control-point positions from that statement) give u(x') = a + G x' and
    du/dx' = G inside the box; beyond it the coordinate is clamped to the box
    face, where u takes its face value and the clamped axis' column of the
    Jacobian vanishes."""
    shape, vox = (6, 7, 9), (1.3, 0.8, 1.1)          # (nz, ny, nx); vox (x, y, z)
    origin = (-4.0, 2.5, -3.0)
    n_xyz = shape[::-1]
    lo = np.array([origin[a] - 0.5 * vox[a] for a in range(3)])
    box = np.array([n_xyz[a] * vox[a] for a in range(3)])
    rng = np.random.default_rng(31)
    a0 = rng.normal(size=3)
    G = rng.normal(size=(3, 3)) * 0.05
    idx = np.arange(8)
    ctrl = [lo[a] + (idx - 1) * box[a] / 5.0 for a in range(3)]
    K, J_, I = np.meshgrid(idx, idx, idx, indexing="ij")      # coef[k][j][i]
    xc = np.stack([ctrl[0][I], ctrl[1][J_], ctrl[2][K]], axis=-1)
    coef = a0 + xc @ G.T
    cfg = small(n=8, nu=8, nv=8, n_views=2)
    pb = oracle.Problem(inputs.projection_matrices(cfg), shape, vox, origin, (8, 8), 0.5, coef=coef,
                        theta=inputs.identity_theta(2), s_view=np.ones(2))
    inside = lo + rng.uniform(0.0, 1.0, size=(400, 3)) * box
    u, J = oracle.displacement(pb, inside)
    assert np.max(np.abs(u - (a0 + inside @ G.T))) <= 1e-12
    assert np.max(np.abs(J - G)) <= 1e-12
    # beyond the box on one axis at a time: the face value, that column zero
    for ax in range(3):
        out = lo + rng.uniform(0.1, 0.9, size=(50, 3)) * box
        out[:25, ax] = lo[ax] - rng.uniform(0.2, 3.0, size=25)
        out[25:, ax] = lo[ax] + box[ax] + rng.uniform(0.2, 3.0, size=25)
        clamped = out.copy()
        clamped[:25, ax] = lo[ax]
        clamped[25:, ax] = lo[ax] + box[ax]
        u, J = oracle.displacement(pb, out)
        assert np.max(np.abs(u - (a0 + clamped @ G.T))) <= 1e-12
        G0 = G.copy()
        G0[:, ax] = 0.0
        assert np.max(np.abs(J - G0)) <= 1e-12


def test_p7_repeated_subangles_equal_single():
    cfg = small(n=16, nu=20, nv=20, n_views=3)
    P1 = inputs.projection_matrices(cfg)
    P3 = np.repeat(P1, 3, axis=1)
    rng = np.random.default_rng(12)
    vol = rng.uniform(size=cfg.vol_shape)
    a, ra = oracle.forward(oracle_problem(cfg, P=P1), vol)
    b, rb = oracle.forward(oracle_problem(cfg.scaled(n_sub=3), P=P3), vol)
    assert np.allclose(a, b, rtol=1e-14) and np.allclose(ra, rb, rtol=1e-14)


# ---------------------------------------------------------------------------
# P8: backprojector special cases (Sec. 4.1, Sec. 4.3.2)
# ---------------------------------------------------------------------------

def _projected_points(cfg, view, X):
    """Detector coordinates of points X [..., 3] by line/plane intersection,
    from the trajectory definition (no projection matrix)."""
    srcs, ctrs, us, vs = inputs.detector_frames(cfg)
    s, c, u, v = srcs[view, 0], ctrs[view, 0], us[view, 0], vs[view, 0]
    d0 = c - 0.5 * (cfg.nu - 1) * u - 0.5 * (cfg.nv - 1) * v
    nrm = np.cross(u, v)
    t = ((d0 - s) @ nrm) / ((X - s) @ nrm)
    hit = s + t[..., None] * (X - s)
    rel = hit - d0
    G = np.array([[u @ u, u @ v], [u @ v, v @ v]])
    coords = np.linalg.solve(G, np.stack([rel @ u, rel @ v], axis=-1)[..., None])[..., 0]
    return coords[..., 0], coords[..., 1]


def test_p8_interior_colsum_and_affine_images():
    cfg = small(n=16, nu=40, nv=40, n_views=5, trajectory="perturbed", seed=13)
    pb = oracle_problem(cfg)
    n = cfg.n
    idx = np.arange(n)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    pts = np.stack([cfg.origin[0] + X * cfg.vox, cfg.origin[1] + Y * cfg.vox,
                    cfg.origin[2] + Z * cfg.vox], axis=-1)
    rng = np.random.default_rng(13)
    coef = rng.normal(size=(cfg.n_views, 3))
    iu = np.arange(cfg.nu)[None, :]
    iv = np.arange(cfg.nv)[:, None]
    r = np.stack([coef[k, 0] + coef[k, 1] * iu + coef[k, 2] * iv for k in range(cfg.n_views)])
    _, b, c = oracle.backproject(pb, r)
    expect = np.zeros(cfg.vol_shape)
    interior = np.ones(cfg.vol_shape, bool)
    for k in range(cfg.n_views):
        u, v = _projected_points(cfg, k, pts)
        expect += coef[k, 0] + coef[k, 1] * u + coef[k, 2] * v
        interior &= (u >= 0) & (u <= cfg.nu - 1) & (v >= 0) & (v <= cfg.nv - 1)
    assert interior.sum() > 1000
    # bilinear interpolation reproduces affine images exactly
    assert np.allclose(b[interior], expect[interior], rtol=0, atol=1e-9)
    # interior voxels: column sum = number of views exactly
    assert np.allclose(c[interior], cfg.n_views, rtol=0, atol=1e-12)


def test_p8_weights_special_cases():
    cfg = small(n=16, nu=24, nv=24, n_views=4)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(14)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    x0 = rng.uniform(size=cfg.vol_shape)
    xa, _, _ = oracle.backproject(pb, r, x=x0)
    xb, _, _ = oracle.backproject(pb, r, x=x0, w=np.ones(cfg.vol_shape))
    xc, _, _ = oracle.backproject(pb, r, x=x0, w=np.zeros(cfg.vol_shape))
    assert np.array_equal(xa, xb)
    assert np.array_equal(xc, x0)
    w = rng.uniform(size=cfg.vol_shape)
    xd, _, _ = oracle.backproject(pb, r, x=x0, w=w, alpha=0.5)
    assert np.allclose(xd - x0, 0.5 * w * (xa - x0), atol=1e-13)


# ---------------------------------------------------------------------------
# P9: finite differences of the motion-aware forward (FP64)
# ---------------------------------------------------------------------------

def test_p9_motion_gradient_finite_differences():
    cfg = inputs.MOTION_FD_32.scaled(nu=24, nv=24, n_views=6)
    th, co, sv = inputs.motion_params(cfg)
    vol = inputs.phantom(cfg).numpy()
    pb = oracle_problem(cfg, theta=th, coef=co, s_view=sv)
    rng = np.random.default_rng(15)
    g = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    gt, gc = oracle.motion_grad(pb, vol, g)
    h = 1e-6

    def loss(theta=th, coef=co, views=None):
        p = oracle_problem(cfg, theta=theta, coef=coef, s_view=sv)
        proj, _ = oracle.forward(p, vol, views=views)
        gg = g if views is None else g[views]
        return float((proj * gg).sum())

    fd_t, an_t = [], []
    for view in (1, 4):
        for q in range(15):
            tp, tm = th.copy(), th.copy()
            tp[view, q] += h
            tm[view, q] -= h
            fd_t.append((loss(theta=tp, views=[view]) - loss(theta=tm, views=[view])) / (2 * h))
            an_t.append(gt[view, q])
    assert rel_l2(an_t, fd_t) <= 1e-5
    fd_c, an_c = [], []
    for (k, j, i, comp) in [(3, 3, 3, 0), (4, 3, 5, 1), (2, 5, 4, 2), (5, 4, 2, 0)]:
        cp, cm = co.copy(), co.copy()
        cp[k, j, i, comp] += h
        cm[k, j, i, comp] -= h
        fd_c.append((loss(coef=cp) - loss(coef=cm)) / (2 * h))
        an_c.append(gc[k, j, i, comp])
    assert rel_l2(an_c, fd_c) <= 1e-5
    # volume gradient of <g, A x> is A^T g: finite differences along a random direction
    dx = rng.normal(size=cfg.vol_shape)
    ATg = oracle.adjoint(pb, g)
    fd = (float((oracle.forward(pb, vol + dx)[0] * g).sum()) -
          float((oracle.forward(pb, vol - dx)[0] * g).sum())) / 2.0
    assert fd == pytest.approx(float((ATg * dx).sum()), rel=1e-10)


# ---------------------------------------------------------------------------
# Geometry reading R1: rejection of degenerate matrices
# ---------------------------------------------------------------------------

def test_geometry_rejects_singular_and_zero_depth():
    cfg = small(n=8, nu=8, nv=8, n_views=1)
    P = inputs.projection_matrices(cfg)
    bad = P.copy()
    bad[0, 0, :, 0] = 0.0  # singular left block
    with pytest.raises(ValueError):
        oracle.setup_views(oracle_problem(cfg, P=bad))
    bad2 = P.copy()
    bad2[0, 0, 2, :] = 0.0
    bad2[0, 0, 2, 0] = 1.0  # depth = x, zero at the volume centre
    with pytest.raises(ValueError):
        oracle.setup_views(oracle_problem(cfg, P=bad2))
    Pn, src, _ = oracle.setup_views(oracle_problem(cfg, P=-P))
    assert np.allclose(src[0, 0], [-inputs.SOD, 0, 0])
    assert np.allclose(Pn, P)


# ---------------------------------------------------------------------------
# Convolution oracle of the warm-start network: brute-force loops
# ---------------------------------------------------------------------------

def test_conv_oracle_matches_brute_force():
    from oracle import conv

    rng = np.random.default_rng(21)
    nb, d, h, w, cin, cout = 2, 4, 3, 5, 2, 3
    x = rng.normal(size=(nb, d, h, w, cin))
    wt = rng.normal(size=(cout, 27, cin))
    bias = rng.normal(size=cout)
    y = conv.conv3d(x, wt, bias)
    ref = np.zeros((nb, d, h, w, cout))
    for n in range(nb):
        for z in range(d):
            for yy in range(h):
                for xx in range(w):
                    for co in range(cout):
                        s = bias[co]
                        for kz in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                                    if 0 <= zz < d and 0 <= y2 < h and 0 <= x2 < w:
                                        s += wt[co, kz * 9 + ky * 3 + kx] @ x[n, zz, y2, x2]
                        ref[n, z, yy, xx, co] = s
    assert np.allclose(y, ref, atol=1e-12)
    # gradients: dx equals the convolution of dy with flipped, transposed taps;
    # dw by brute force
    dy = rng.normal(size=(nb, d, h, w, cout))
    dx, dw = conv.conv3d_grads(x, wt, dy)
    wflip = np.ascontiguousarray(wt[:, ::-1, :].transpose(2, 1, 0))
    assert np.allclose(dx, conv.conv3d(dy, wflip), atol=1e-12)
    dw_ref = np.zeros_like(wt)
    for co in range(cout):
        for t in range(27):
            kz, ky, kx = t // 9, (t // 3) % 3, t % 3
            for n in range(nb):
                for z in range(d):
                    for yy in range(h):
                        for xx in range(w):
                            zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                            if 0 <= zz < d and 0 <= y2 < h and 0 <= x2 < w:
                                dw_ref[co, t] += dy[n, z, yy, xx, co] * x[n, zz, y2, x2]
    assert np.allclose(dw, dw_ref, atol=1e-10)


# ---------------------------------------------------------------------------
# Ordered-subset SIRT (Sec. 2.3.2)
# ---------------------------------------------------------------------------

def test_os_sirt_single_subset_is_sirt():
    cfg = small(n=16, nu=20, nv=20, n_views=6, trajectory="perturbed", seed=31)
    pb = oracle_problem(cfg)
    p, _ = oracle.forward(pb, inputs.phantom(cfg.scaled(n_ellipsoids=4)).numpy())
    xs, hs, ds, _ = oracle.sirt(pb, p, 4)
    xo, ho, do, _ = oracle.os_sirt(pb, p, [list(range(cfg.n_views))], 4)
    assert ds == do == 4
    assert np.array_equal(xs, xo) and np.array_equal(hs, ho)


def test_os_sirt_cycle_is_dense_composition(dense8):
    cfg, pb, A, B = dense8
    rng = np.random.default_rng(32)
    p = A @ rng.uniform(0, 1, size=A.shape[1])
    w = rng.uniform(0.3, 1.0, size=A.shape[1])
    alpha = 0.8
    npix = cfg.nu * cfg.nv
    subsets = [[2, 0], [3], [1]]
    x = rng.uniform(0, 1, size=A.shape[1])
    x_ref = x.copy()
    acc = p2 = 0.0
    for S in subsets:
        rows = np.concatenate([np.arange(v * npix, (v + 1) * npix) for v in S])
        As, Bs = A[rows], B[:, rows]
        rs = As.sum(axis=1)
        R = np.where(rs > pb.eps_R, 1.0 / np.where(rs > 0, rs, 1), 0.0)
        cs = Bs.sum(axis=1)
        C = np.where(cs > oracle.EPS_C, 1.0 / np.where(cs > 0, cs, 1), 0.0)
        e = p[rows] - As @ x_ref
        acc += e @ e
        p2 += p[rows] @ p[rows]
        x_ref = x_ref + alpha * w * C * (Bs @ (R * e))
    xo, ho, do, _ = oracle.os_sirt(pb, p.reshape(cfg.n_views, cfg.nv, cfg.nu), subsets, 1, alpha=alpha,
                                   w=w.reshape(cfg.vol_shape), x0=x.reshape(cfg.vol_shape))
    assert do == 1
    assert np.allclose(xo.ravel(), x_ref, rtol=0, atol=1e-12)
    assert ho[0] == pytest.approx(np.sqrt(acc / p2), rel=1e-12)


def test_subset_schedules_partition_views():
    for sets in (inputs.subsets_cyclic(90, 10), inputs.subsets_cyclic(7, 3, spread=False),
                 inputs.subsets_random(90, 7, seed=3)):
        flat = sorted(v for s in sets for v in s)
        assert flat == list(range(max(flat) + 1))
    assert inputs.subsets_cyclic(8, 4)[:2] == [[0, 4], [2, 6]]  # bit-reversed visiting order


# ---------------------------------------------------------------------------
# Extended field of view: per-view backprojection windows (Sec. 3.6, 4.3.2)
# ---------------------------------------------------------------------------

def test_bp_window_equals_cropped_detector():
    cfg = small(n=16, nu=30, nv=24, n_views=5, trajectory="perturbed", seed=41)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(41)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    full = np.tile(np.array([0, cfg.nu - 1, 0, cfg.nv - 1], np.int32), (cfg.n_views, 1))
    _, b0, c0 = oracle.backproject(pb, r)
    _, b1, c1 = oracle.backproject(pb.with_window(full), r)
    assert np.array_equal(b0, b1) and np.array_equal(c0, c1)
    # a window [u0, u1] x [v0, v1] is the backprojector of a detector cropped to
    # it: shift the pixel origin by (u0, v0) and crop the images
    win = np.array([[3, 25, 2, 20], [0, 29, 5, 23], [7, 20, 0, 23], [1, 28, 1, 22], [10, 29, 4, 15]], np.int32)
    _, bw, cw = oracle.backproject(pb.with_window(win), r)
    bc, cc = np.zeros(cfg.vol_shape), np.zeros(cfg.vol_shape)
    for v in range(cfg.n_views):
        u0, u1, v0, v1 = win[v]
        T = np.array([[1.0, 0.0, -u0], [0.0, 1.0, -v0], [0.0, 0.0, 1.0]])
        Pc = (T @ pb.P[v, 0])[None, None]
        pv = oracle.Problem(Pc, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (u1 - u0 + 1, v1 - v0 + 1))
        _, bv, cv = oracle.backproject(pv, r[v:v + 1, v0:v1 + 1, u0:u1 + 1])
        bc += bv
        cc += cv
    assert np.allclose(bw, bc, atol=1e-12) and np.allclose(cw, cc, atol=1e-12)


# ---------------------------------------------------------------------------
# Sub-voxel backprojection (Sec. 4.3.2)
# ---------------------------------------------------------------------------

def test_subvoxel_bp_is_block_mean_of_fine_grid():
    cfg = small(n=8, nu=26, nv=22, n_views=4, trajectory="perturbed", seed=51)
    pb = oracle_problem(cfg)
    rng = np.random.default_rng(51)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    _, b1, c1 = oracle.backproject(pb.with_subvoxel(1), r)
    _, b0, c0 = oracle.backproject(pb, r)
    assert np.array_equal(b0, b1) and np.array_equal(c0, c1)
    s = 2
    _, bs, cs = oracle.backproject(pb.with_subvoxel(s), r)
    fine_vox = cfg.vox / s
    fine_origin = tuple(o - 0.5 * cfg.vox + 0.5 * fine_vox for o in cfg.origin)
    n2 = cfg.n * s
    pf = oracle.Problem(pb.P, (n2, n2, n2), (fine_vox,) * 3, fine_origin, (cfg.nu, cfg.nv))
    _, bf, cf = oracle.backproject(pf, r)
    blk = lambda a: a.reshape(cfg.n, s, cfg.n, s, cfg.n, s).mean(axis=(1, 3, 5))  # noqa: E731
    assert np.allclose(bs, blk(bf), atol=1e-12) and np.allclose(cs, blk(cf), atol=1e-12)


# ---------------------------------------------------------------------------
# Aligned cylindrical domain (Sec. 3.5, reading R13)
# ---------------------------------------------------------------------------

def _axial_P(x0, y0, D=300.0, f=40.0, uc=10.0, vc=10.0):
    """A projection whose source sits at (x0, y0, -D): the ray through pixel
    (uc, vc) runs along +z through (x0, y0)."""
    return np.array([[f, 0.0, uc, -f * x0 + uc * D],
                     [0.0, f, vc, -f * y0 + vc * D],
                     [0.0, 0.0, 1.0, D]])


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _pose(R, t):
    return np.hstack([R, np.asarray(t, float)[:, None]])


def test_cylinder_axial_rays_closed_form():
    # rays parallel to the cylinder axis: r and phi are constant, so the ray
    # reduces to the 1D truncated-midpoint rule of P1 along z on the values
    # the (r, phi) position selects
    n_r, n_p, n_z, dr, dz = 6, 12, 10, 1.5, 1.0
    rng = np.random.default_rng(13)
    vol = rng.uniform(0.0, 1.0, size=(n_z, n_p, n_r))
    dphi = 2 * math.pi / n_p

    def axial(r0, phi0):
        x0, y0 = r0 * math.cos(phi0), r0 * math.sin(phi0)
        pb = oracle.cylinder_problem(_axial_P(x0, y0)[None], n_r, n_p, n_z, dr, dz, (21, 21))
        val, rs = oracle.forward_rays(pb, vol, np.zeros(1, np.int32), np.array([10.0]), np.array([10.0]))
        return val[0], rs[0]

    def closed(col):
        return dz * (col.sum() - (col[0] + col[-1]) / 8.0)

    for i, j in ((2, 3), (5, 0), (0, 11)):
        val, rs = axial((i + 0.5) * dr, (j + 0.5) * dphi)
        assert val == pytest.approx(closed(vol[:, j, i]), rel=1e-12)
        assert rs == pytest.approx(dz * (n_z - 0.25), rel=1e-12)
    # inside the first ring centre the ring-0 value is used (clamp)
    val, _ = axial(0.2 * dr, 7.5 * dphi)
    assert val == pytest.approx(closed(vol[:, 7, 0]), rel=1e-12)
    # phi = 0 lies halfway between the last and the first sector (periodic)
    val, _ = axial(3.5 * dr, 0.0)
    assert val == pytest.approx(closed(0.5 * (vol[:, n_p - 1, 3] + vol[:, 0, 3])), rel=1e-12)
    # outside the bounding cylinder: nothing
    val, rs = axial(n_r * dr + 0.01, 1.0)
    assert val == 0.0 and rs == 0.0


def test_cylinder_rotation_about_axis_is_a_sector_roll():
    cfg = small(n=8, nu=24, nv=20, n_views=5, trajectory="perturbed", seed=21)
    P = inputs.projection_matrices(cfg)
    n_r, n_p, n_z, dr, dz = 5, 16, 7, 2.6, 3.8
    vol = np.random.default_rng(21).uniform(size=(n_z, n_p, n_r))
    m = 3
    tilt = _rot_x(0.2)
    pb0 = oracle.cylinder_problem(P, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv), pose=_pose(tilt, [0.4, -0.3, 0.2]))
    # frame rotated by m sectors about its own axis: a world point's sector index grows by m
    Rm = inputs.rot_z(m * 2 * math.pi / n_p)
    pbm = oracle.cylinder_problem(P, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv),
                                  pose=_pose(Rm @ tilt, Rm @ np.array([0.4, -0.3, 0.2])))
    a, ra = oracle.forward(pbm, vol)
    b, rb = oracle.forward(pb0, np.roll(vol, -m, axis=1))
    assert np.abs(a).max() > 1.0
    # equal up to the rounding of the rotated sample positions
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max() and np.abs(ra - rb).max() <= 1e-10 * np.abs(ra).max()


def test_cylinder_rigid_change_of_world_frame():
    # moving the scanner and the cylinder together by a rigid motion G changes nothing
    cfg = small(n=8, nu=24, nv=20, n_views=4, trajectory="perturbed", seed=22)
    P = inputs.projection_matrices(cfg)[:, 0]
    n_r, n_p, n_z, dr, dz = 5, 12, 6, 2.6, 4.0
    vol = np.random.default_rng(22).uniform(size=(n_z, n_p, n_r))
    pose = _pose(_rot_x(-0.15), [0.5, 0.2, -0.4])
    G = _pose(inputs.rot_z(0.7) @ _rot_x(0.3), [3.0, -2.0, 1.5])
    Gi = np.hstack([G[:, :3].T, -(G[:, :3].T @ G[:, 3])[:, None]])

    def compose(A, B):  # (A o B)(x) = A (B x) for 3x4 affine maps
        return np.hstack([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]])

    P2 = np.stack([Pv @ np.vstack([Gi, [0, 0, 0, 1]]) for Pv in P])  # P2 (G x) = P x
    pb1 = oracle.cylinder_problem(P, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv), pose=pose)
    pb2 = oracle.cylinder_problem(P2, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv), pose=compose(pose, Gi))
    a, _ = oracle.forward(pb1, vol)
    b, _ = oracle.forward(pb2, vol)
    assert np.abs(a).max() > 1.0 and np.allclose(a, b, rtol=1e-10, atol=1e-10)


def _cyl_centres_world(n_r, n_p, n_z, dr, dz, pose):
    """World positions of the cylinder voxel centres [n_z, n_p, n_r, 3]."""
    r = (np.arange(n_r) + 0.5) * dr
    phi = (np.arange(n_p) + 0.5) * 2 * math.pi / n_p
    z = (np.arange(n_z) - 0.5 * (n_z - 1)) * dz
    Z, PH, Rr = np.meshgrid(z, phi, r, indexing="ij")
    q = np.stack([Rr * np.cos(PH), Rr * np.sin(PH), Z], axis=-1)
    Rc, tc = pose[:, :3], pose[:, 3]
    return (q - tc) @ Rc  # Rc^T (q - tc), row-vector form


def test_cylinder_gaussian_line_integrals_converge():
    # a Cartesian Gaussian sampled at the cylinder voxel centres: the line
    # integrals converge to the analytic ones at second order
    cfg = small(n=8, nu=20, nv=20, n_views=3, trajectory="perturbed", seed=23)
    P = inputs.projection_matrices(cfg)[:, 0]
    pose = _pose(_rot_x(0.12) @ inputs.rot_z(0.3), [0.6, -0.4, 0.3])
    c = np.array([6.0, 3.0, -2.0])  # world centre of the blob
    sig = 2.5
    R, H = 16.0, 24.0
    # 48 rays through the blob's projection, shifted by up to a pixel
    rng = np.random.default_rng(23)
    views = (np.arange(48) % 3).astype(np.int32)
    offs = rng.uniform(-1.0, 1.0, size=(48, 2))
    h = np.einsum("vij,j->vi", P[views], np.append(c, 1.0))
    us = h[:, 0] / h[:, 2] + offs[:, 0]
    vs = h[:, 1] / h[:, 2] + offs[:, 1]
    # analytic integral of exp(-|x - c|^2 / sig^2) along each ray (the blob sits
    # well inside the cylinder): sig sqrt(pi) exp(-d^2 / sig^2), d = distance to c
    ref = []
    for v, u, w in zip(views, us, vs):
        M, p4 = P[v][:, :3], P[v][:, 3]
        s = -np.linalg.solve(M, p4)
        d = np.linalg.solve(M, np.array([u, w, 1.0]))
        d /= np.linalg.norm(d)
        e = c - s
        dist2 = e @ e - (e @ d) ** 2
        ref.append(sig * math.sqrt(math.pi) * math.exp(-dist2 / sig ** 2))
    ref = np.array(ref)
    errs = []
    for k in (1, 2, 4):
        n_r, n_p, n_z = 12 * k, 48 * k, 18 * k
        dr, dz = R / n_r, H / n_z
        X = _cyl_centres_world(n_r, n_p, n_z, dr, dz, pose)
        vol = np.exp(-((X - c) ** 2).sum(-1) / sig ** 2)
        pb = oracle.cylinder_problem(P, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv), pose=pose)
        val, _ = oracle.forward_rays(pb, vol, views, us, vs)
        errs.append(rel_l2(val, ref))
    # second order: each halving of (dr, dphi, dz) divides the error by ~4; a
    # misplaced grid (half-cell shift, wrong pose) would leave an O(h) or O(1) error
    assert errs[2] < 5e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_cylinder_bp_is_cartesian_bp_at_voxel_centres():
    cfg = small(n=8, nu=24, nv=22, n_views=6, trajectory="perturbed", seed=24)
    P = inputs.projection_matrices(cfg)
    n_r, n_p, n_z, dr, dz = 5, 14, 6, 2.8, 4.5
    pose = _pose(_rot_x(0.1), [0.3, 0.5, -0.2])
    pb = oracle.cylinder_problem(P, n_r, n_p, n_z, dr, dz, (cfg.nu, cfg.nv), pose=pose)
    r = np.random.default_rng(24).normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    _, b, c = oracle.backproject(pb, r)
    X = _cyl_centres_world(n_r, n_p, n_z, dr, dz, pose)
    rng = np.random.default_rng(25)
    for flat in rng.integers(0, b.size, 12):
        k, j, i = np.unravel_index(flat, b.shape)
        one = oracle.Problem(P, (1, 1, 1), (1.0, 1.0, 1.0), tuple(X[k, j, i]), (cfg.nu, cfg.nv))
        _, b1, c1 = oracle.backproject(one, r)
        assert b[k, j, i] == pytest.approx(b1[0, 0, 0], rel=1e-12, abs=1e-12)
        assert c[k, j, i] == pytest.approx(c1[0, 0, 0], rel=1e-12, abs=1e-12)
    # sub-voxel points of the cylinder are the centres of the 2x finer cylinder grid
    _, b2, c2 = oracle.backproject(pb.with_subvoxel(2), r)
    fine = oracle.cylinder_problem(P, 2 * n_r, 2 * n_p, 2 * n_z, dr / 2, dz / 2, (cfg.nu, cfg.nv), pose=pose)
    _, bf, cf = oracle.backproject(fine, r)
    blk = lambda a: a.reshape(n_z, 2, n_p, 2, n_r, 2).mean(axis=(1, 3, 5))  # noqa: E731
    assert np.allclose(b2, blk(bf), atol=1e-12) and np.allclose(c2, blk(cf), atol=1e-12)


def test_cylinder_refuses_adjoint():
    cfg = small(n=8, nu=12, nv=12, n_views=2)
    pb = oracle.cylinder_problem(inputs.projection_matrices(cfg), 4, 8, 4, 2.0, 2.0, (12, 12))
    with pytest.raises(ValueError):
        oracle.adjoint(pb, np.zeros((2, 12, 12)))


# ---------------------------------------------------------------------------
# Classical Joseph projector (reading R14)
# ---------------------------------------------------------------------------

def _x_axial_P(y0, z0, D=300.0, f=40.0, uc=10.0, vc=10.0):
    """Source at (-D, y0, z0): the ray through pixel (uc, vc) runs along +x."""
    return np.array([[0.0, f, 0.0, -f * y0],
                     [0.0, 0.0, f, -f * z0],
                     [0.0, 0.0, 0.0, 0.0]]) + np.array([[uc, 0, 0, uc * D], [vc, 0, 0, vc * D], [1.0, 0, 0, D]])


def _joseph_grid(n=(9, 7, 6), vox=(1.2, 0.9, 1.5)):
    origin = tuple(-0.5 * (k - 1) * v for k, v in zip(n, vox))
    return (n[2], n[1], n[0]), vox, origin


def test_joseph_axial_rays_closed_form():
    shape, vox, origin = _joseph_grid()
    vol = np.random.default_rng(41).uniform(size=shape)
    nz, ny, nx = shape
    for j, k, fy in ((3, 2, 0.0), (1, 4, 0.3), (5, 0, 0.75)):
        y0 = origin[1] + (j + fy) * vox[1]
        z0 = origin[2] + k * vox[2]
        pb = oracle.Problem(_x_axial_P(y0, z0)[None], shape, vox, origin, (21, 21)).with_joseph()
        val, rs = oracle.forward_rays(pb, vol, np.zeros(1, np.int32), np.array([10.0]), np.array([10.0]))
        row = (1.0 - fy) * vol[k, j, :] + (fy * vol[k, j + 1, :] if fy > 0 else 0.0)
        # one sample per slice, at every voxel centre of the row: no end corrections
        assert val[0] == pytest.approx(vox[0] * row.sum(), rel=1e-12)
        assert rs[0] == pytest.approx(vox[0] * nx, rel=1e-12)
    # the trilinear projector on the same ray has the end corrections of P1
    pb = oracle.Problem(_x_axial_P(origin[1] + 3 * vox[1], origin[2] + 2 * vox[2])[None], shape, vox, origin,
                        (21, 21), step_vox=0.5)
    row = vol[2, 3, :]
    val, _ = oracle.forward_rays(pb, vol, np.zeros(1, np.int32), np.array([10.0]), np.array([10.0]))
    assert val[0] != pytest.approx(vox[0] * row.sum(), rel=1e-6)


def _chord(src, d, lo, hi):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        ta, tb = (lo[a] - src[a]) / d[a], (hi[a] - src[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return t0, t1


def _joseph_linear_check(P, shape, vox, rng, n_rays=400, det=(40, 40), urange=(15, 25)):
    """Joseph on a linear volume against chord length x f(chord midpoint),
    for rays that cross both faces of their principal axis inside the grid;
    returns how many rays were checked."""
    n = (shape[2], shape[1], shape[0])
    origin = tuple(-0.5 * (k - 1) * v for k, v in zip(n, vox))
    c0, c = 0.4, np.array([0.05, -0.03, 0.02])
    Z, Y, X = np.meshgrid(*[origin[a] + np.arange(n[a]) * vox[a] for a in (2, 1, 0)], indexing="ij")
    vol = c0 + c[0] * X + c[1] * Y + c[2] * Z
    pb = oracle.Problem(P, shape, vox, origin, det).with_joseph()
    lo = np.array([origin[a] - 0.5 * vox[a] for a in range(3)])
    hi = np.array([origin[a] + (n[a] - 0.5) * vox[a] for a in range(3)])
    checked = 0
    for _ in range(n_rays):
        v = int(rng.integers(0, len(P)))
        u, w = rng.uniform(*urange, size=2)
        M, p4 = P[v][:, :3], P[v][:, 3]
        s = -np.linalg.solve(M, p4)
        d = np.linalg.solve(M, np.array([u, w, 1.0]))
        d /= np.linalg.norm(d)
        if d @ (-s) < 0:
            d = -d
        m = int(np.argmax(np.abs(d) / np.array(vox)))  # fastest index coordinate
        t0 = (lo[m] - s[m]) / d[m]
        t1 = (hi[m] - s[m]) / d[m]
        t0, t1 = min(t0, t1), max(t0, t1)
        ok = True
        for t in (t0, t1):
            p = s + t * d
            for a in range(3):
                if a != m and not (origin[a] + 1e-9 <= p[a] <= origin[a] + (n[a] - 1) * vox[a] - 1e-9):
                    ok = False
        if not ok:
            continue
        mid = s + 0.5 * (t0 + t1) * d
        val, rs = oracle.forward_rays(pb, vol, np.array([v], np.int32), np.array([u]), np.array([w]))
        L = t1 - t0
        assert val[0] == pytest.approx(L * (c0 + c @ mid), rel=1e-11)
        assert rs[0] == pytest.approx(L, rel=1e-11)
        checked += 1
    return checked


def test_joseph_linear_volume_and_row_sums_exact():
    # a linear function sampled at the voxel centres is reproduced exactly by
    # bilinear interpolation inside the grid, and the slice sum is the
    # midpoint rule over the chord between the two principal faces, exact for
    # a linear integrand: value = chord length x f(chord midpoint)
    cfg = small(n=8, nu=40, nv=40, n_views=6, trajectory="perturbed", seed=42)
    P = inputs.projection_matrices(cfg)[:, 0]
    rng = np.random.default_rng(42)
    assert _joseph_linear_check(P, (14, 13, 15), (1.0, 1.1, 0.9), rng) > 20
    # strongly anisotropic voxels, rays 60 degrees from x in the x-y plane:
    # |d_y| > |d_x| but the x index changes faster (0.5/0.8 > 0.87/2), so x
    # is the principal axis
    Ps = []
    for a in (58.0, 60.0, 62.0):
        e = np.array([math.cos(math.radians(a)), math.sin(math.radians(a)), 0.0])
        src = -200.0 * e
        uax = np.array([-e[1], e[0], 0.0]) * 0.5
        Ps.append(inputs.cone_matrix(src, 200.0 * e, uax, np.array([0.0, 0.0, 0.5]), 40, 40))
    assert _joseph_linear_check(np.array(Ps), (8, 12, 10), (0.8, 2.0, 1.0), rng, urange=(17, 23)) > 20


def test_joseph_axis_swap_equivariance():
    # swapping the x and y axes of the volume together with the geometry
    # leaves the projections unchanged (no axis is favoured)
    cfg = small(n=8, nu=20, nv=18, n_views=8, trajectory="perturbed", seed=43)
    P = inputs.projection_matrices(cfg)
    shape, vox, origin = (6, 7, 9), (1.3, 0.8, 1.1), (-4.0, -2.5, -3.0)
    vol = np.random.default_rng(43).uniform(size=shape)
    pb = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv)).with_joseph()
    S = np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], float)  # (x, y) swap
    P2 = P @ S
    pb2 = oracle.Problem(P2, (shape[0], shape[2], shape[1]), (vox[1], vox[0], vox[2]),
                         (origin[1], origin[0], origin[2]), (cfg.nu, cfg.nv)).with_joseph()
    a, ra = oracle.forward(pb, vol)
    b, rb = oracle.forward(pb2, vol.transpose(0, 2, 1))
    assert np.abs(a).max() > 1.0
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max() and np.abs(ra - rb).max() <= 1e-10 * np.abs(ra).max()


def test_joseph_gaussian_line_integrals_converge():
    # a Gaussian sampled at the voxel centres: second-order convergence to the
    # analytic line integrals, over rays whose principal axes are x, y and z
    c, sig = np.array([1.5, -1.0, 0.8]), 2.2
    cfg = small(n=8, nu=20, nv=20, n_views=4, trajectory="perturbed", seed=44)
    P = list(inputs.projection_matrices(cfg)[:, 0])
    # a view from above (rays mostly along z)
    P.append(np.array([[40.0, 0.0, 10.0, 10.0 * 300.0], [0.0, 40.0, 10.0, 10.0 * 300.0], [0.0, 0.0, 1.0, 300.0]]))
    P = np.array(P)
    rng = np.random.default_rng(44)
    views = np.repeat(np.arange(5), 10).astype(np.int32)
    h = np.einsum("vij,j->vi", P[views], np.append(c, 1.0))
    us = h[:, 0] / h[:, 2] + rng.uniform(-1, 1, len(views))
    vs = h[:, 1] / h[:, 2] + rng.uniform(-1, 1, len(views))
    ref, axes = [], set()
    for v, u, w in zip(views, us, vs):
        M, p4 = P[v][:, :3], P[v][:, 3]
        s = -np.linalg.solve(M, p4)
        d = np.linalg.solve(M, np.array([u, w, 1.0]))
        d /= np.linalg.norm(d)
        axes.add(int(np.argmax(np.abs(d))))
        e = c - s
        ref.append(sig * math.sqrt(math.pi) * math.exp(-(e @ e - (e @ d) ** 2) / sig ** 2))
    ref = np.array(ref)
    assert axes == {0, 1, 2}
    errs = []
    for k in (2, 4, 8):
        n = 12 * k
        vx = 24.0 / n
        org = -0.5 * (n - 1) * vx
        g = org + np.arange(n) * vx
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        vol = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / sig ** 2)
        pb = oracle.Problem(P, (n, n, n), (vx,) * 3, (org,) * 3, (cfg.nu, cfg.nv)).with_joseph()
        val, _ = oracle.forward_rays(pb, vol, views, us, vs)
        errs.append(rel_l2(val, ref))
    # h / sigma = 0.45, 0.23, 0.11: a half-voxel misplacement would halve the
    # error per level at best
    assert errs[2] < 5e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_joseph_refusals():
    cfg = small(n=8, nu=12, nv=12, n_views=2)
    pb = oracle_problem(cfg).with_joseph()
    with pytest.raises(ValueError):
        oracle.adjoint(pb, np.zeros((2, 12, 12)))
    th = inputs.identity_theta(2)
    with pytest.raises(ValueError):
        oracle.forward(pb.with_motion(theta=th), np.zeros(cfg.vol_shape))


# ---------------------------------------------------------------------------
# Multi-resolution ROI (reading R15)
# ---------------------------------------------------------------------------

def _roi_setup(nc=(12, 10, 8), vc=1.0, lo=(4, 3, 2), nroi=(4, 4, 3), ratio=2):
    """Context grid nc (x, y, z) of pitch vc centred at 0; an ROI covering the
    context voxels [lo, lo + nroi) at pitch vc / ratio (faces aligned)."""
    shape = (nc[2], nc[1], nc[0])
    origin = tuple(-0.5 * (n - 1) * vc for n in nc)
    vf = vc / ratio
    rn = tuple(k * ratio for k in nroi)
    rorigin = tuple(origin[a] + (lo[a] - 0.5) * vc + 0.5 * vf for a in range(3))
    return shape, (vc,) * 3, origin, (rn[2], rn[1], rn[0]), (vf,) * 3, rorigin


def test_roi_parts_equal_single_grid_projections():
    cfg = small(n=8, nu=30, nv=26, n_views=6, trajectory="perturbed", seed=71)
    P = inputs.projection_matrices(cfg)
    shape, vox, origin, rshape, rvox, rorg = _roi_setup(nc=(26, 24, 20), lo=(9, 8, 7), nroi=(8, 8, 6))
    base = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv))
    pb = base.with_roi(rshape, rvox, rorg)
    fine = oracle.Problem(P, rshape, rvox, rorg, (cfg.nu, cfg.nv))
    rng = np.random.default_rng(71)
    xc = rng.uniform(size=shape)
    xf = rng.uniform(size=rshape)
    nc = xc.size
    # ROI values only: the ROI piece of every ray is the fine grid's own clip
    a, ra = oracle.forward(pb, np.concatenate([np.zeros(nc), xf.ravel()]))
    b, _ = oracle.forward(fine, xf)
    assert np.abs(b).max() > 1.0 and np.allclose(a, b, rtol=1e-12, atol=1e-12)
    # context values only, on rays that miss the ROI box: the context projection
    c, _ = oracle.forward(pb, np.concatenate([xc.ravel(), np.zeros(xf.size)]))
    d, _ = oracle.forward(base, xc)
    _, rs_f = oracle.forward(fine, np.ones(rshape))
    miss = rs_f == 0.0
    assert miss.sum() > 100 and (~miss).sum() > 100
    assert np.allclose(c[miss], d[miss], rtol=1e-12, atol=1e-12)
    # and the two resolutions add
    e, _ = oracle.forward(pb, np.concatenate([xc.ravel(), xf.ravel()]))
    assert np.allclose(e, a + c, rtol=1e-12, atol=1e-12)


def test_roi_axial_ray_closed_form():
    # a ray along x through the centre of context row (j, k): context pieces
    # before and after the ROI, each the P1 rule with the context voxel just
    # inside the ROI entering through the last tap, and the ROI piece the P1
    # rule on the mean of the four ROI rows around the ray
    shape, vox, origin, rshape, rvox, rorg = _roi_setup()
    nz, ny, nx = shape
    rng = np.random.default_rng(72)
    xc = rng.uniform(size=shape)
    xf = rng.uniform(size=rshape)
    j, k = 4, 3  # inside the ROI's y range [3, 7) and z range [2, 5)
    y0 = origin[1] + j * vox[1]
    z0 = origin[2] + k * vox[2]
    pb = oracle.Problem(_x_axial_P(y0, z0)[None], shape, vox, origin, (21, 21)).with_roi(rshape, rvox, rorg)
    val, rs = oracle.forward_rays(pb, np.concatenate([xc.ravel(), xf.ravel()]), np.zeros(1, np.int32),
                                  np.array([10.0]), np.array([10.0]))
    lo, hi = 4, 8  # ROI covers context columns [4, 8)
    f = xc[k, j, :]
    entry, exit_ = f[:lo], f[hi:]
    vc = vox[0]
    ctx_in = vc * (entry.sum() - entry[0] / 8 - entry[-1] / 8 + f[lo] / 8)
    ctx_out = vc * (exit_.sum() - exit_[0] / 8 - exit_[-1] / 8 + f[hi - 1] / 8)
    # the ray sits halfway between ROI rows 2 (j - 3) * 2 + {0, 1} and slices 2 (k - 2) + {0, 1}
    jy, kz = 2 * (j - 3), 2 * (k - 2)
    g = 0.25 * (xf[kz, jy, :] + xf[kz, jy + 1, :] + xf[kz + 1, jy, :] + xf[kz + 1, jy + 1, :])
    roi_piece = rvox[0] * (g.sum() - g[0] / 8 - g[-1] / 8)
    assert val[0] == pytest.approx(ctx_in + roi_piece + ctx_out, rel=1e-11)
    ones = oracle.forward_rays(pb, np.ones(pb.vol_shape), np.zeros(1, np.int32), np.array([10.0]),
                               np.array([10.0]))[0][0]
    n_in, n_out, n_roi = lo, nx - hi, rshape[2]
    assert ones == pytest.approx(vc * (n_in - 1 / 8) + vc * (n_out - 1 / 8) + rvox[0] * (n_roi - 1 / 4), rel=1e-11)


def test_roi_backprojection_is_per_grid():
    cfg = small(n=8, nu=30, nv=26, n_views=5, trajectory="perturbed", seed=73)
    P = inputs.projection_matrices(cfg)
    shape, vox, origin, rshape, rvox, rorg = _roi_setup(nc=(26, 24, 20), lo=(9, 8, 7), nroi=(8, 8, 6))
    base = oracle.Problem(P, shape, vox, origin, (cfg.nu, cfg.nv))
    pb = base.with_roi(rshape, rvox, rorg)
    fine = oracle.Problem(P, rshape, rvox, rorg, (cfg.nu, cfg.nv))
    r = np.random.default_rng(73).normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    _, b, c = oracle.backproject(pb, r)
    _, bc, cc = oracle.backproject(base, r)
    _, bf, cf = oracle.backproject(fine, r)
    nc = bc.size
    assert np.array_equal(b[:nc], bc.ravel()) and np.array_equal(c[:nc], cc.ravel())
    assert np.array_equal(b[nc:], bf.ravel()) and np.array_equal(c[nc:], cf.ravel())
    vox_idx = np.array([0, 17, nc - 1, nc, nc + 100, b.size - 1])
    bv, cv = oracle.backproject_voxels(pb, r, vox_idx)
    assert np.array_equal(bv, b[vox_idx]) and np.array_equal(cv, c[vox_idx])

