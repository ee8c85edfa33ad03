"""Ordered-subset SIRT (Eq. (1) with index sets P_k, Sec. 2.3.2) on the GPU
vs the FP64 oracle, and what subsets buy per pass over the data."""

import numpy as np
import pytest
import torch

import oracle
from paper_2609_30166_gb300 import inputs
from tests.helpers import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    cfg = inputs.CIRCULAR_64
    vol = inputs.phantom(cfg).numpy()
    pb = oracle_problem(cfg)
    proj, _ = oracle.forward(pb, vol)
    ctx = ctrex.context_for(cfg)
    return cfg, pb, proj, ctx


def _gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


@pytest.mark.parametrize("scheme", ["cyclic10", "random7", "sart"])
def test_os_sirt_matches_oracle(setup, scheme):
    cfg, pb, proj, ctx = setup
    if scheme == "cyclic10":
        subsets, cycles = inputs.subsets_cyclic(cfg.n_views, 10), 3
    elif scheme == "random7":
        subsets, cycles = inputs.subsets_random(cfg.n_views, 7, seed=5), 2
    else:
        subsets, cycles = [[v] for v in range(cfg.n_views)], 1
    rng = np.random.default_rng(9)
    w = rng.uniform(0.5, 1.0, size=cfg.vol_shape)
    x_ref, h_ref, d_ref, _ = oracle.os_sirt(pb, proj, subsets, cycles, alpha=0.9, w=w)
    x = torch.zeros(cfg.vol_shape, device="cuda")
    x, hist, done = ctx.os_sirt_iterate(x, _gpu(proj), subsets, cycles, alpha=0.9, w=_gpu(w))
    assert done == d_ref == cycles
    assert rel_l2(x.double().cpu().numpy(), x_ref) <= 1e-5
    assert np.allclose(hist, h_ref, rtol=1e-4)


def test_single_subset_is_sirt_bitwise(setup):
    cfg, pb, proj, ctx = setup
    p = _gpu(proj)
    a = torch.zeros(cfg.vol_shape, device="cuda")
    ctx.sirt_iterate(a, p, 4)
    b = torch.zeros(cfg.vol_shape, device="cuda")
    ctx.os_sirt_iterate(b, p, [list(range(cfg.n_views))], 4)
    assert torch.equal(a, b)


def test_subsets_converge_faster_per_data_pass(setup):
    cfg, pb, proj, ctx = setup
    p = _gpu(proj)
    x = torch.zeros(cfg.vol_shape, device="cuda")
    _, h_sirt, _ = ctx.sirt_iterate(x, p, 6)
    y = torch.zeros(cfg.vol_shape, device="cuda")
    _, h_os, _ = ctx.os_sirt_iterate(y, p, inputs.subsets_cyclic(cfg.n_views, 10), 5)
    # residual of x after 5 full passes: SIRT history entry 5 is rho(x_5)
    print(f"after 5 passes: SIRT {h_sirt[5]:.4e}, OS-SIRT(10) running residual of pass 5 {h_os[4]:.4e}")
    assert h_os[4] < 0.5 * h_sirt[5]
    # tolerance stop after a cycle
    z = torch.zeros(cfg.vol_shape, device="cuda")
    _, h, done = ctx.os_sirt_iterate(z, p, inputs.subsets_cyclic(cfg.n_views, 10), 50, tol=0.05)
    assert 0 < done < 50 and h[done - 1] <= 0.05
