"""Learned warm start: a small 3D U-Net whose 3x3x3 convolutions run on the
tcgen05 tensor-core kernels of libctrex (BF16 operands, FP32 accumulation),
trained on (few-iteration SIRT, phantom) pairs that the library's own
projector and SIRT produce.  Plain SIRT from zero stays the fallback; the
data residual of Eq. (1) judges both.  The paper only motivates combining
the physics operators with learned components (Sec. 5).

Layout: activations are channels-last [N, D, H, W, C] in BF16; weights are
FP32 masters [Cout, 27, Cin], cast to BF16 for each call.  Pooling,
upsampling, concatenation, the 1x1x1 head, the loss and Adam are plain
torch ops (element-wise, not on the hot path).
"""

from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import ctrex, inputs


class _Conv3(torch.autograd.Function):
    """y = act(conv3x3x3(x, w) + b), act = ReLU or identity."""

    @staticmethod
    def forward(actx, x, w, b, relu):
        wb = w.to(torch.bfloat16)
        y = ctrex.conv3d(x, wb, b, relu=relu, out_dtype=torch.bfloat16)
        actx.save_for_backward(x, wb, y)
        actx.relu = relu
        return y

    @staticmethod
    def backward(actx, dy):
        x, wb, y = actx.saved_tensors
        dy = dy.to(torch.bfloat16)
        if actx.relu:
            dy = dy * (y > 0).to(dy.dtype)
        dy = dy.contiguous()
        dx = ctrex.conv3d(dy, ctrex.flip_weights(wb), None, relu=False, out_dtype=torch.bfloat16) \
            if actx.needs_input_grad[0] else None
        dw = ctrex.conv3d_wgrad(x, dy) if actx.needs_input_grad[1] else None
        db = dy.float().sum(dim=(0, 1, 2, 3)) if actx.needs_input_grad[2] else None
        return dx, dw, db, None


class Conv3(torch.nn.Module):
    def __init__(self, cin, cout, relu=True, gen=None, init_cin=None):
        """init_cin: draw (He initialisation) the weights of only the first
        init_cin input channels and start the others at zero."""
        super().__init__()
        ci = init_cin or cin
        std = math.sqrt(2.0 / (27 * ci))
        w = torch.randn(cout, 27, ci, generator=gen) * std
        if ci < cin:
            w = torch.nn.functional.pad(w, (0, cin - ci))
        self.w = torch.nn.Parameter(w)
        self.b = torch.nn.Parameter(torch.zeros(cout))
        self.relu = relu

    def forward(self, x):
        return _Conv3.apply(x, self.w, self.b, self.relu)


def _pool(x):
    n, d, h, w, c = x.shape
    return x.view(n, d // 2, 2, h // 2, 2, w // 2, 2, c).amax(dim=(2, 4, 6))


def _up(x):
    return x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


class UNet3D(torch.nn.Module):
    """4 levels (16, 32, 64, 128 channels), two 3x3x3 convs per level, max
    pooling down, nearest upsampling + skip concatenation up, 1x1x1 head; the
    output is the input plus the predicted correction."""

    def __init__(self, base=16, seed=0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        c1, c2, c3, c4 = base, 2 * base, 4 * base, 8 * base
        # the single input channel is carried in a block of 16 (zeros beside
        # it), the channel granularity of the brick-staged tensor-core conv;
        # the first layer is initialised as for a block of 8: the weights of
        # the other 8 start at zero and, facing zero inputs, get zero
        # gradients, so they stay zero
        self.e1 = torch.nn.ModuleList([Conv3(16, c1, gen=g, init_cin=8), Conv3(c1, c1, gen=g)])
        self.e2 = torch.nn.ModuleList([Conv3(c1, c2, gen=g), Conv3(c2, c2, gen=g)])
        self.e3 = torch.nn.ModuleList([Conv3(c2, c3, gen=g), Conv3(c3, c3, gen=g)])
        self.e4 = torch.nn.ModuleList([Conv3(c3, c4, gen=g), Conv3(c4, c4, gen=g)])
        self.d3 = torch.nn.ModuleList([Conv3(c4 + c3, c3, gen=g), Conv3(c3, c3, gen=g)])
        self.d2 = torch.nn.ModuleList([Conv3(c3 + c2, c2, gen=g), Conv3(c2, c2, gen=g)])
        self.d1 = torch.nn.ModuleList([Conv3(c2 + c1, c1, gen=g), Conv3(c1, c1, gen=g)])
        self.head_w = torch.nn.Parameter(torch.zeros(c1))
        self.head_b = torch.nn.Parameter(torch.zeros(1))

    @staticmethod
    def _block(convs, x):
        for c in convs:
            x = c(x)
        return x

    def forward(self, x):
        """x: [N, D, H, W] float32 (D, H, W divisible by 8); returns the same shape."""
        xin = torch.nn.functional.pad(x.to(torch.bfloat16).unsqueeze(-1), (0, 15)).contiguous()
        s1 = self._block(self.e1, xin)
        s2 = self._block(self.e2, _pool(s1))
        s3 = self._block(self.e3, _pool(s2))
        b = self._block(self.e4, _pool(s3))
        u3 = self._block(self.d3, torch.cat([_up(b), s3], dim=-1).contiguous())
        u2 = self._block(self.d2, torch.cat([_up(u3), s2], dim=-1).contiguous())
        u1 = self._block(self.d1, torch.cat([_up(u2), s1], dim=-1).contiguous())
        corr = (u1.float() * self.head_w).sum(-1) + self.head_b
        return x + corr


# ---------------------------------------------------------------------------
# Data, training and the warm-start comparison
# ---------------------------------------------------------------------------

def make_pairs(cfg, seeds, ctx, sirt_iters=5, device="cuda"):
    """(SIRT_k inputs, phantoms, measured projections) for the given seeds, all
    produced on the GPU by the library (projections simulated by the
    projector; inputs = sirt_iters SIRT iterations from zero)."""
    xs, ys, ps = [], [], []
    for s in seeds:
        ph = inputs.phantom(cfg, seed=int(s), device=device).to(torch.float32).contiguous()
        p = ctx.fwd_project(ph)
        x = torch.zeros_like(ph)
        ctx.sirt_iterate(x, p, sirt_iters)
        xs.append(x)
        ys.append(ph)
        ps.append(p)
    return torch.stack(xs), torch.stack(ys), ps


def error_gradient_loss(e):
    """Mean squared forward differences of the error e [N, D, H, W] along
    the three axes: the error's gradient, which weights a spatial frequency
    w by about |2 sin(w / 2)|^2 per axis."""
    return (((e[:, 1:] - e[:, :-1]) ** 2).mean() + ((e[:, :, 1:] - e[:, :, :-1]) ** 2).mean()
            + ((e[:, :, :, 1:] - e[:, :, :, :-1]) ** 2).mean())


def train(model, x_train, y_train, steps=1200, batch=2, lr=1e-3, seed=0, grad_weight=16.0, log=None):
    """Adam with cosine decay on loss = mean (x_hat - x)^2 + grad_weight *
    error_gradient_loss(x_hat - x).  Why the gradient term: SIRT corrects the
    low spatial frequencies of its start's error within a few iterations and
    the high ones slowly (its normalised normal operator C A^T R A acts as a
    low-pass filter), so the iterations still needed to reach a data residual
    are set by the high-frequency error the network leaves; weighting it by
    the squared gradient aims the network at exactly those components.  On
    the sparse-view workload it cut the iterations after the warm start from
    715 (plain squared error) to 203, against 790 from zero."""
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.LambdaLR(opt, lambda t: 0.5 * (1.0 + math.cos(math.pi * t / max(steps, 1))))
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x_train.shape[0]
    losses = []
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g)
        pred = model(x_train[idx])
        err = pred - y_train[idx]
        loss = (err ** 2).mean()
        if grad_weight:
            loss = loss + grad_weight * error_gradient_loss(err)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        losses.append(float(loss.detach()))
        if log and (it % 50 == 0 or it == steps - 1):
            log(f"step {it} loss {losses[-1]:.4e}")
    ctrex.conv_status_check()
    return losses


def sirt_to_tolerance(ctx, x, p, tol, max_iter, chunk=25):
    """Run SIRT in chunks until the relative data residual is <= tol.
    Returns (iterations applied, final residual, history)."""
    done_total, hist_all = 0, []
    while done_total < max_iter:
        n = min(chunk, max_iter - done_total)
        _, hist, done = ctx.sirt_iterate(x, p, n, tol=tol)
        hist_all.extend([float(h) for h in hist[: done + (1 if done < n else 0)]])
        done_total += done
        if done < n:  # stopped on tolerance
            return done_total, hist_all[-1], hist_all
    r, sums = ctx.fwd_correct(x, p)
    rho = float((sums[0] / sums[1]).sqrt())
    hist_all.append(rho)
    return done_total, rho, hist_all


def compare_warm_start(model, cfg, ctx, seeds, tol=1e-3, max_iter=3000, sirt_in=5, device="cuda"):
    """Wall time and iterations to relative data residual <= tol for plain
    SIRT from zero and for the warm start (sirt_in SIRT iterations, U-Net,
    then SIRT), per held-out seed; the warm-start time includes its SIRT
    input iterations and the network."""
    rows = []
    with torch.no_grad():  # one untimed inference: lazy module loading, allocator warm-up
        model(torch.zeros((1,) + cfg.vol_shape, device=device))
    for s in seeds:
        ph = inputs.phantom(cfg, seed=int(s), device=device).to(torch.float32).contiguous()
        p = ctx.fwd_project(ph)
        torch.cuda.synchronize()
        # plain SIRT from zero
        x = torch.zeros_like(ph)
        t0 = time.perf_counter()
        it_plain, rho_plain, _ = sirt_to_tolerance(ctx, x, p, tol, max_iter)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        # warm start
        t0 = time.perf_counter()
        xw = torch.zeros_like(ph)
        ctx.sirt_iterate(xw, p, sirt_in)
        t_in = time.perf_counter() - t0
        with torch.no_grad():
            x0 = model(xw.unsqueeze(0))[0].contiguous()
        torch.cuda.synchronize()
        t_net = time.perf_counter() - t0 - t_in
        x0_copy = x0.clone()  # for the error report, taken outside the timed region below
        t_copy = time.perf_counter()
        it_warm, rho_warm, _ = sirt_to_tolerance(ctx, x0, p, tol, max_iter)
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t_copy + t_in + t_net
        net_err = float((x0_copy - ph).norm() / ph.norm())
        in_err = float((xw - ph).norm() / ph.norm())
        rows.append({"seed": int(s), "plain_iters": it_plain, "plain_s": t_plain, "plain_rho": rho_plain,
                     "warm_iters": sirt_in + it_warm, "warm_s": t_warm, "warm_rho": rho_warm,
                     "sirt_in_s": t_in, "net_s": t_net, "sirt_in_err": in_err, "net_err": net_err,
                     "plain_final_err": float((x - ph).norm() / ph.norm()),
                     "warm_final_err": float((x0 - ph).norm() / ph.norm())})
    return rows
