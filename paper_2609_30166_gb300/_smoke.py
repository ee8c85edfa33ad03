"""One small invocation of the hot path on cuda:0, checked against the FP64
oracle: fused forward projection + correction, weighted backprojection with
normalisation and update (one SIRT iteration of Eq. (1)); then one 3x3x3
convolution of the warm-start network and its weight gradient on the
tensor cores against the FP64 conv oracle."""

import numpy as np
import torch


def run():
    import oracle

    from . import ctrex, inputs

    if not torch.cuda.is_available():
        raise RuntimeError("smoke needs a CUDA device")
    cfg = inputs.CIRCULAR_64.scaled(n=32, nu=48, nv=40, n_views=12)
    P = inputs.projection_matrices(cfg)
    vol = inputs.phantom(cfg).numpy()
    pb = oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)
    p_ref, _ = oracle.forward(pb, vol)
    x_ref, hist_ref, _, _ = oracle.sirt(pb, p_ref, 2)

    ctx = ctrex.context_for(cfg, P=P, device=0)
    dev = torch.device("cuda", 0)
    p = ctx.fwd_project(torch.as_tensor(vol, dtype=torch.float32, device=dev))
    err_p = float(np.linalg.norm(p.double().cpu().numpy() - p_ref) / np.linalg.norm(p_ref))
    x = torch.zeros(cfg.vol_shape, dtype=torch.float32, device=dev)
    x, hist, done = ctx.sirt_iterate(x, torch.as_tensor(p_ref, dtype=torch.float32, device=dev), 2)
    err_x = float(np.linalg.norm(x.double().cpu().numpy() - x_ref) / np.linalg.norm(x_ref))
    ctx.close()
    if not (err_p <= 1e-5 and err_x <= 1e-5 and done == 2):
        raise AssertionError(f"smoke parity failed: projection {err_p:.3e}, SIRT volume {err_x:.3e}")

    from oracle import conv

    rng = np.random.default_rng(3)
    xc = torch.as_tensor(rng.normal(size=(1, 4, 18, 20, 16)), dtype=torch.float32).to(torch.bfloat16)
    wc = torch.as_tensor(rng.normal(size=(16, 27, 16)) / 20.0, dtype=torch.float32).to(torch.bfloat16)
    dyc = torch.as_tensor(rng.normal(size=(1, 4, 18, 20, 16)), dtype=torch.float32).to(torch.bfloat16)
    y_ref = conv.conv3d(xc.double().numpy(), wc.double().numpy())
    _, dw_ref = conv.conv3d_grads(xc.double().numpy(), wc.double().numpy(), dyc.double().numpy())
    y = ctrex.conv3d(xc.to(dev), wc.to(dev), out_dtype=torch.float32)
    dw = ctrex.conv3d_wgrad(xc.to(dev), dyc.to(dev))
    ctrex.conv_status_check(dev)
    err_y = float(np.linalg.norm(y.double().cpu().numpy() - y_ref) / np.linalg.norm(y_ref))
    err_w = float(np.linalg.norm(dw.double().cpu().numpy() - dw_ref) / np.linalg.norm(dw_ref))
    if not (err_y <= 1e-4 and err_w <= 1e-4):
        raise AssertionError(f"smoke conv parity failed: forward {err_y:.3e}, weight gradient {err_w:.3e}")
    print(f"smoke ok: projection rel.L2 {err_p:.2e}, 2-iteration SIRT rel.L2 {err_x:.2e}, "
          f"conv {err_y:.2e}, conv weight gradient {err_w:.2e}")
