"""Learned relaxation: training data from plain Laguerre-Gauss relaxation, training on the
GPU with libsph's own BF16 tensor-core forward/backward kernels and Adam, and the
proposal-accelerated relaxation that always finishes with plain steps.

Procedure (the benchmark configuration's learned variant):
* data: for each seeded body, plain relaxation snapshots every ``every`` steps;
  features at snapshot t, target (x^{t+every} - x^t) / h;
* training: Adam on random minibatches (MSE);
* use: ``applications`` times {proposal move, then ``plain_between`` plain steps},
  then plain steps until the residual target is met (plain relaxation is the
  fallback: if the target is missed by the step cap, the result is the plain run's).
"""
import torch

from . import api, inputs


def body_on_device(ctx, seed, dp, precision=api.SPH_FP32_KAHAN):
    b = inputs.sphere_body(seed, dp)
    pos = torch.tensor(b["pos"], dtype=torch.float64, device=ctx.device)
    order = api.cell_order(ctx, b["domain"], pos)
    pos = pos[:, order].contiguous()
    vol = torch.tensor(b["vol"], dtype=torch.float64, device=ctx.device)[order].contiguous()
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=precision, n=pos.shape[1])
    return b, prm, pos, vol


def trajectory_samples(ctx, seed, dp, steps=500, every=50):
    """(features [m, 128], targets [m, 3]) float32 device tensors from one plain trajectory."""
    b, prm, pos, vol = body_on_device(ctx, seed, dp)
    h = b["h"]
    feats, targets = [], []
    for _ in range(0, steps, every):
        f = api.mlp_features(ctx, prm, pos)
        x0 = pos.clone()
        api.relax_step(ctx, prm, pos, vol, every)
        feats.append(f)
        targets.append(((pos - x0) / h).t().to(torch.float32).contiguous())
    return torch.cat(feats), torch.cat(targets)


def train(ctx, feats, targets, steps, batch=4096, lr=1e-3, seed=0, log_every=0):
    trainer = api.MLPTrainer(ctx, inputs.mlp_init(seed), lr=lr)
    gen = torch.Generator(device=ctx.device)
    gen.manual_seed(seed)
    m = feats.shape[0]
    losses = []
    for k in range(steps):
        idx = torch.randint(0, m, (batch,), device=ctx.device, generator=gen)
        want = log_every and (k % log_every == 0 or k == steps - 1)
        loss = trainer.step(feats[idx].contiguous(), targets[idx].contiguous(), with_loss=bool(want))
        if want:
            losses.append((k, loss))
    return trainer, losses


def steps_to_target(ctx, prm, pos, vol, target, max_steps, check_every=10):
    """Plain relaxation steps until the Laguerre-Gauss residual is <= target (or the cap)."""
    done = 0
    r = api.relax_residual(ctx, prm, pos, vol)[0]
    while r > target and done < max_steps:
        api.relax_step(ctx, prm, pos, vol, check_every)
        done += check_every
        r = api.relax_residual(ctx, prm, pos, vol)[0]
    return done, r


def learned_relax(ctx, prm, params, pos, vol, target, max_steps, applications=3, plain_between=10, check_every=10):
    """Proposal-accelerated relaxation; returns (plain steps used, final residual, proposals kept).

    A proposal is kept only if it lowers the Laguerre-Gauss residual; otherwise the
    positions are restored and the run continues with plain relaxation alone."""
    used = 0
    kept = 0
    for _ in range(applications):
        r_before = api.relax_residual(ctx, prm, pos, vol)[0]
        if r_before <= target:
            return used, r_before, kept
        saved = pos.clone()
        api.relax_propose(ctx, prm, params, pos)
        if api.relax_residual(ctx, prm, pos, vol)[0] >= r_before:
            pos.copy_(saved)
            break
        kept += 1
        n, r = steps_to_target(ctx, prm, pos, vol, target, plain_between, check_every)
        used += n
        if r <= target:
            return used, r, kept
    more, r = steps_to_target(ctx, prm, pos, vol, target, max_steps - used, check_every)
    return used + more, r, kept
