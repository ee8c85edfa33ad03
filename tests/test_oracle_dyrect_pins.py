"""Pins of the oracle's event-based 4D model (Sec. 3.3, reading: view v sees
the initial value mu0_j where t_v < tau_j and the final value mu1_j
elsewhere; the backprojector splits Eq. (1) term 3 by the same rule).

Each check ties the event model to the static operators, which are pinned
on their own: the projection of a view equals the static projection of
that view's frame volume (built here voxel by voxel); the two backprojected
parts add up to the static backprojection and each equals the static
backprojection over its own views; the extreme transition times reduce to
the static model; the adjoint is the transpose; one SIRT step equals the
dense formula.
"""

import numpy as np
import pytest

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem


def _scene(n=16, nu=24, nv=22, views=7, seed=3):
    cfg = inputs.CIRCULAR_64.scaled(n=n, nu=nu, nv=nv, n_views=views, trajectory="perturbed", seed=seed)
    mu0, mu1, tau = (f.numpy() for f in inputs.dyrect_fields(cfg, n_events=10))
    tv = inputs.view_times(cfg)
    return cfg, mu0, mu1, tau, tv


def test_dyrect_projection_is_the_frame_projection():
    cfg, mu0, mu1, tau, tv = _scene()
    pb = oracle_problem(cfg)
    pbd = pb.with_dyrect(tau, tv)
    got, rs = oracle.forward(pbd, np.stack([mu0, mu1]))
    _, rs_static = oracle.forward(pb, mu0)
    mixed = 0
    for v in range(cfg.n_views):
        frame = np.where(tv[v] < tau, mu0, mu1)
        mixed += int((frame != mu0).any() and (frame != mu1).any())
        want, _ = oracle.forward(pb, frame, views=[v])
        assert np.allclose(got[v], want[0], rtol=0, atol=1e-13 * np.abs(want).max())
    assert mixed >= 3  # views that see some regions changed and others not
    assert np.array_equal(rs, rs_static)  # the row sums are the static ones


def test_dyrect_extreme_transition_times_are_static():
    cfg, mu0, mu1, tau, tv = _scene(views=5)
    pb = oracle_problem(cfg)
    vol = np.stack([mu0, mu1])
    for t_all, which in ((3.0, 0), (-1.0, 1)):
        pbd = pb.with_dyrect(np.full_like(tau, t_all), tv)
        got, _ = oracle.forward(pbd, vol)
        want, _ = oracle.forward(pb, vol[which])
        assert np.array_equal(got, want)
        r = np.random.default_rng(4).normal(size=(cfg.n_views, cfg.nv, cfg.nu))
        _, b, c = oracle.backproject(pbd, r)
        _, bs, cs = oracle.backproject(pb, r)
        assert np.array_equal(b[which], bs) and np.array_equal(c[which], cs)
        assert not b[1 - which].any() and not c[1 - which].any()


def test_dyrect_backprojection_splits_the_views():
    cfg, mu0, mu1, tau, tv = _scene(views=8)
    pb = oracle_problem(cfg)
    # two transition times only, so that each part is a static backprojection
    # over a known view subset
    t_star = 0.5 * (tv[3] + tv[4])
    tau2 = np.where(tau < 2.0, t_star, 2.0)
    assert (tau2 == t_star).sum() > 50
    pbd = pb.with_dyrect(tau2, tv)
    rng = np.random.default_rng(5)
    r = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    _, b, c = oracle.backproject(pbd, r)
    _, bs, cs = oracle.backproject(pb, r)
    assert np.allclose(b[0] + b[1], bs, rtol=0, atol=1e-12 * np.abs(bs).max())
    assert np.allclose(c[0] + c[1], cs, rtol=0, atol=1e-12)
    before, after = np.arange(4), np.arange(4, cfg.n_views)
    _, b_bef, c_bef = oracle.backproject(pb, r[before], views=before)
    _, b_aft, c_aft = oracle.backproject(pb, r[after], views=after)
    m = tau2 == t_star
    assert np.allclose(b[0][m], b_bef[m], rtol=0, atol=1e-12) and np.allclose(c[0][m], c_bef[m], rtol=0, atol=1e-12)
    assert np.allclose(b[1][m], b_aft[m], rtol=0, atol=1e-12) and np.allclose(c[1][m], c_aft[m], rtol=0, atol=1e-12)
    assert np.allclose(b[0][~m], bs[~m], rtol=0, atol=1e-12) and not b[1][~m].any()
    # each part is normalised by its own column sum
    x0 = rng.uniform(size=(2,) + cfg.vol_shape)
    x1, _, _ = oracle.backproject(pbd, r, x=x0, alpha=0.7)
    C = np.where(c > oracle.EPS_C, 1.0 / np.where(c > 0, c, 1.0), 0.0)
    assert np.allclose(x1, x0 + 0.7 * C * b, rtol=0, atol=1e-13)


def test_dyrect_adjoint_is_the_transpose():
    cfg, mu0, mu1, tau, tv = _scene(views=6)
    pbd = oracle_problem(cfg).with_dyrect(tau, tv)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2,) + cfg.vol_shape)
    y = rng.normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    Ax, _ = oracle.forward(pbd, x)
    ATy = oracle.adjoint(pbd, y)
    lhs, rhs = float((Ax * y).sum()), float((x * ATy).sum())
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)


def test_dyrect_sirt_step_is_the_dense_formula():
    cfg = inputs.CIRCULAR_64.scaled(n=8, nu=10, nv=9, n_views=4, trajectory="perturbed", seed=5)
    rng = np.random.default_rng(7)
    tau = rng.choice([0.2, 0.6, 2.0], size=cfg.vol_shape)
    tv = inputs.view_times(cfg)
    pbd = oracle_problem(cfg).with_dyrect(tau, tv)
    nunk, nray = 2 * 8 ** 3, cfg.n_views * cfg.nv * cfg.nu
    A = np.zeros((nray, nunk))
    for j in range(nunk):
        e = np.zeros(nunk)
        e[j] = 1.0
        A[:, j] = oracle.forward(pbd, e.reshape((2,) + cfg.vol_shape))[0].ravel()
    B = np.zeros((nunk, nray))
    for i in range(nray):
        e = np.zeros(nray)
        e[i] = 1.0
        B[:, i] = oracle.backproject(pbd, e.reshape(cfg.n_views, cfg.nv, cfg.nu))[1].ravel()
    # the unknown j of either part is seen only by the views its part owns
    AT = np.stack([oracle.adjoint(pbd, e.reshape(cfg.n_views, cfg.nv, cfg.nu)).ravel()
                   for e in np.eye(nray)[:: 7]], axis=1)
    assert np.allclose(AT, A[:: 7].T, rtol=0, atol=1e-14)
    x0 = rng.uniform(size=nunk)
    p = A @ rng.uniform(size=nunk)
    rowsum, colsum = A.sum(1), B.sum(1)
    R = np.where(rowsum > pbd.eps_R, 1.0 / np.where(rowsum > 0, rowsum, 1), 0.0)
    C = np.where(colsum > oracle.EPS_C, 1.0 / np.where(colsum > 0, colsum, 1), 0.0)
    expect = x0 + C * (B @ (R * (p - A @ x0)))
    x1, hist, done, ret = oracle.sirt(pbd, p.reshape(cfg.n_views, cfg.nv, cfg.nu), 1,
                                      x0=x0.reshape((2,) + cfg.vol_shape))
    assert done == 1 and ret == 0
    assert np.allclose(x1.ravel(), expect, rtol=0, atol=1e-12)


def test_dyrect_refuses_other_models():
    cfg, mu0, mu1, tau, tv = _scene(views=3)
    pbd = oracle_problem(cfg).with_dyrect(tau, tv)
    with pytest.raises(ValueError):
        oracle.forward(pbd.with_subvoxel(2), np.stack([mu0, mu1]))
    with pytest.raises(ValueError):
        oracle.forward(pbd.with_joseph(), np.stack([mu0, mu1]))
