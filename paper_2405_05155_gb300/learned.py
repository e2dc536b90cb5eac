"""Learned relaxation: training data from plain Laguerre-Gauss relaxation, training on the
GPU with libsph's own BF16 tensor-core forward/backward kernels and Adam, and the
proposal-accelerated relaxation that always finishes with plain steps.

Every step runs in libsph (this module only marshals arguments):
* data: sph_relax_samples -- for each seeded body, plain relaxation snapshots every
  ``every`` steps; features at snapshot t, target (x^{t+every} - x^t) / h;
* training: sph_mlp_train -- Adam on minibatches drawn and gathered on the device (MSE);
* use: sph_relax_run -- up to ``applications`` proposal moves, each kept only if it lowers
  the residual and followed by ``plain_between`` plain steps, then plain steps until the
  residual target is met; if the target is missed by the step cap, plain relaxation from
  the start is the fallback and gives the result.
"""
import torch

from . import api, inputs


def body_on_device(ctx, seed, dp, precision=api.SPH_FP32_KAHAN):
    """A seeded 8-sphere body (inputs.sphere_body) in cell order on the device."""
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
    return api.relax_samples(ctx, prm, pos, vol, steps // every, every)


def training_set(ctx, seeds, dp, steps=500, every=50):
    """Samples of several bodies, concatenated on the device."""
    feats, targets = [], []
    for seed in seeds:
        f, t = trajectory_samples(ctx, seed, dp, steps, every)
        feats.append(f)
        targets.append(t)
    return torch.cat(feats), torch.cat(targets)


def train(ctx, feats, targets, steps, batch=4096, lr=1e-3, seed=0, log_every=0):
    """Adam from the seeded initialisation; returns (trainer, [(step, loss), ...])."""
    trainer = api.MLPTrainer(ctx, inputs.mlp_init(seed), lr=lr)
    if not log_every:
        trainer.train(feats, targets, steps, batch=batch, seed=seed, with_loss=False)
        return trainer, []
    # the minibatch loss of steps 0, log_every, 2 log_every, ... and the last (each step's
    # loss is taken before its update)
    marks = sorted(set([0] + list(range(log_every, steps, log_every)) + [steps - 1]))
    losses, prev = [], -1
    for k in marks:
        losses.append((k, trainer.train(feats, targets, k - prev, batch=batch, seed=seed, with_loss=True)))
        prev = k
    return trainer, losses


def steps_to_target(ctx, prm, pos, vol, target, max_steps, check_every=10):
    """Plain relaxation steps until the Laguerre-Gauss residual is <= target (or the cap)."""
    r = api.relax_run(ctx, prm, pos, vol, target, max_steps, proposal=None, check_every=check_every)
    return r["steps"], r["residual"][0]


def learned_relax(ctx, prm, params, pos, vol, target, max_steps, applications=3, plain_between=10, check_every=10):
    """Proposal-accelerated relaxation; returns (plain steps used, final residual, proposals kept)."""
    r = api.relax_run(ctx, prm, pos, vol, target, max_steps, proposal=params, applications=applications,
                      plain_between=plain_between, check_every=check_every)
    return r["steps"], r["residual"][0], r["kept"]
