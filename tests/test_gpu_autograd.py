"""torch.autograd around the CUDA projector: gradients against the FP64
oracle (whose own gradients are pinned to FP64 finite differences), and a
self-calibration run that recovers a rigid shift by gradient descent."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, autograd

    _build.build_library()
    return autograd


def test_autograd_gradients_match_oracle(ag):
    cfg = inputs.MOTION_FD_32.scaled(nu=40, nv=36, n_views=8)
    th, co, sv = inputs.motion_params(cfg)
    vol = inputs.phantom(cfg).numpy()
    proj = ag.Projector(cfg, s_view=sv)
    v = torch.tensor(vol, dtype=torch.float32, device="cuda", requires_grad=True)
    t = torch.tensor(th, dtype=torch.float32, device="cuda", requires_grad=True)
    c = torch.tensor(co, dtype=torch.float32, device="cuda", requires_grad=True)
    g = np.random.default_rng(3).normal(size=(cfg.n_views, cfg.nv, cfg.nu))
    out = proj(v, t, c)
    (out * torch.tensor(g, dtype=torch.float32, device="cuda")).sum().backward()
    pb = oracle_problem(cfg, theta=th, coef=co, s_view=sv)
    ref, _ = oracle.forward(pb, vol)
    assert rel_l2(out.detach().double().cpu().numpy(), ref) <= 1e-5
    assert rel_l2(v.grad.double().cpu().numpy(), oracle.adjoint(pb, g)) <= 1e-5
    gt, gc = oracle.motion_grad(pb, vol, g)
    assert rel_l2(t.grad.double().cpu().numpy(), gt) <= 1e-5
    assert rel_l2(c.grad.double().cpu().numpy(), gc) <= 1e-5


def test_self_calibration_recovers_rigid_shift(ag):
    """Fit one object translation (shared by all views) to data simulated with
    a known shift; a per-view shift along the source-detector axis would be
    nearly unobservable from its own view, a shared one is fixed by all."""
    cfg = inputs.MOTION_FD_32.scaled(n=32, nu=40, nv=40, n_views=12)
    vol = torch.tensor(inputs.phantom(cfg).numpy(), dtype=torch.float32, device="cuda")
    zero_coef = torch.zeros((8, 8, 8, 3), device="cuda")
    proj = ag.Projector(cfg, s_view=np.zeros(cfg.n_views))
    base = torch.tensor(inputs.identity_theta(cfg.n_views), dtype=torch.float32, device="cuda")
    t_true = torch.tensor([0.6, -0.4, 0.3], device="cuda")  # mm

    def theta_of(t):
        th = base.clone()
        th[:, 3:6] = t
        return th

    with torch.no_grad():
        p = proj(vol, theta_of(t_true), zero_coef)
    t = torch.zeros(3, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([t], lr=0.05)
    err0 = float((t.detach() - t_true).norm())
    for _ in range(100):
        opt.zero_grad()
        loss = ((proj(vol, theta_of(t), zero_coef) - p) ** 2).mean()
        loss.backward()
        opt.step()
    err = float((t.detach() - t_true).norm())
    assert err < 0.05 * err0, (err0, err)
