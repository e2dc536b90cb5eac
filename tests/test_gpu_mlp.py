"""GPU parity of the learned proposal (a12): features exact in ranking, BF16 tensor-core
forward and backward within 1e-2 relative L2 of the float64 oracle, Adam training that
lowers the loss like the oracle's, and the gain of the trained proposal."""
import numpy as np
import pytest
import torch

from helpers import cuda, host, odom, rel_l2, sorted_by_cells
from oracle import mlp as OM
from oracle import neighbors as ON
from oracle import relax as OR
from paper_2405_05155_gb300 import api, inputs, learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def test_features_parity(ctx):
    b = inputs.sphere_body(4, 1.0 / 24.0)
    pos, _ = sorted_by_cells(b["pos"], b["domain"])
    dom = odom(b["domain"])
    rp, col = ON.neighbors_cells(pos, dom)
    phi, _ = OR.sdf_spheres(pos, b["spheres"])
    X_o = OM.features(pos, rp, col, dom, phi)
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"])
    X = host(api.mlp_features(ctx, prm, cuda(pos)))
    # same neighbours in the same order: offsets agree to float32 rounding
    assert np.max(np.abs(X - X_o)) < 1e-6 * max(1.0, np.max(np.abs(X_o)))
    assert np.array_equal(X[:, :96] == 0.0, X_o[:, :96] == 0.0)


def test_features_parity_long_rows(ctx):
    # twice the density (each particle with a shifted copy): rows of more than 128
    # neighbours, ranked like the short ones
    b = inputs.sphere_body(4, 1.0 / 20.0)
    p = np.concatenate([b["pos"], b["pos"] + 0.31 * b["dp"] * np.array([[1.0], [0.7], [0.4]])], axis=1)
    pos, _ = sorted_by_cells(p, b["domain"])
    dom = odom(b["domain"])
    rp, col = ON.neighbors_cells(pos, dom.with_kappa(2.0))
    lens = np.diff(rp)
    assert lens.max() > 128 and lens.min() <= 128
    phi, _ = OR.sdf_spheres(pos, b["spheres"])
    X_o = OM.features(pos, rp, col, dom, phi)
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"])
    X = host(api.mlp_features(ctx, prm, cuda(pos)))
    assert np.max(np.abs(X - X_o)) < 1e-6 * max(1.0, np.max(np.abs(X_o)))
    assert np.array_equal(X[:, :96] == 0.0, X_o[:, :96] == 0.0)


def _batch(seed, rows):
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 128))
    X[:, :97] = rng.normal(scale=0.8, size=(rows, 97))
    T = rng.normal(scale=0.05, size=(rows, 3))
    return X, T


@pytest.mark.parametrize("rows", [7, 256, 5000])
def test_forward_parity(ctx, rows):
    flat = inputs.mlp_init(1)
    flat[OM.N_PARAM - 3:] = [0.01, -0.02, 0.03]
    X, _ = _batch(2, rows)
    y_o, _ = OM.forward(flat, X)
    y = host(api.mlp_forward(ctx, cuda(flat, torch.float32), cuda(X, torch.float32)))
    assert rel_l2(y, y_o) < 1e-2


@pytest.mark.parametrize("rows", [1, 127, 128, 129, 5000, 40000])
def test_forward_tcgen05_parity(ctx, rows):
    # fused tcgen05 forward: within the bfloat16 tolerance of the float64 oracle and
    # close to the mma.sync forward (same operands, different rounding order); ragged
    # last tiles and more tiles than SMs
    flat = inputs.mlp_init(1)
    flat[OM.N_PARAM - 3:] = [0.01, -0.02, 0.03]
    X, _ = _batch(3, rows)
    y_o, _ = OM.forward(flat, X)
    P, Xd = cuda(flat, torch.float32), cuda(X, torch.float32)
    y = host(api.mlp_forward_tc(ctx, P, Xd))
    assert np.all(np.isfinite(y))
    assert rel_l2(y, y_o) < 1e-2, rel_l2(y, y_o)
    y_mma = host(api.mlp_forward(ctx, P, Xd))
    assert rel_l2(y, y_mma) < 5e-3


@pytest.mark.parametrize("rows", [4096, 1000])
def test_gradient_parity_per_block(ctx, rows):
    # the training path's GEMMs run on tcgen05 (forward, products with the weights, split-K
    # weight gradients); 1000 rows: a ragged last tile and slices
    flat = inputs.mlp_init(5)
    X, T = _batch(6, rows)
    loss_o, g_o = OM.loss_and_grad(flat, X, T)
    g, loss = api.mlp_grad(ctx, cuda(flat, torch.float32), cuda(X, torch.float32), cuda(T, torch.float32))
    g = host(g)
    assert abs(loss - loss_o) < 1e-2 * loss_o
    off = 0
    for name, shape in OM.SHAPES:
        k = int(np.prod(shape))
        assert rel_l2(g[off:off + k], g_o[off:off + k]) < 1e-2, name
        off += k


def test_adam_training_tracks_the_oracle(ctx):
    flat = inputs.mlp_init(7)
    X, _ = _batch(8, 2048)
    # a smooth target the network can fit
    T = np.stack([np.tanh(X[:, 0]), 0.5 * X[:, 1] * X[:, 2], np.sin(X[:, 96])], axis=1) * 0.1
    trainer = api.MLPTrainer(ctx, flat, lr=1e-3)
    Xd, Td = cuda(X, torch.float32), cuda(T, torch.float32)
    gpu_losses = [trainer.step(Xd, Td, with_loss=True) for _ in range(60)]
    w, m, v = flat.copy(), np.zeros_like(flat), np.zeros_like(flat)
    cpu_losses = []
    for k in range(60):
        loss, g = OM.loss_and_grad(w, X, T)
        cpu_losses.append(loss)
        w, m, v = OM.adam(w, g, m, v, k + 1, 1e-3)
    assert gpu_losses[-1] < 0.5 * gpu_losses[0]
    assert abs(gpu_losses[-1] - cpu_losses[-1]) < 0.1 * cpu_losses[-1]
    # the parameters moved the same way (Adam steps are ~lr in size; BF16 moves a few signs)
    assert rel_l2(host(trainer.params) - flat, w - flat) < 0.2


def test_trained_proposal_reduces_relaxation_steps(ctx):
    # train on plain trajectories of a few small seeded bodies, then relax held-out bodies to
    # the residual plain relaxation reaches after 200 steps, with and without the proposal
    feats, targets = [], []
    for seed in range(12):
        f, t = learned.trajectory_samples(ctx, seed, 1.0 / 24.0, steps=300, every=50)
        feats.append(f)
        targets.append(t)
    feats, targets = torch.cat(feats), torch.cat(targets)
    trainer, losses = learned.train(ctx, feats, targets, steps=2000, batch=4096, lr=1e-3, log_every=500)
    assert losses[-1][1] < 0.2 * losses[0][1]
    gains = []
    for seed in (1000, 1001, 1002):
        b, prm, pos, vol = learned.body_on_device(ctx, seed, 1.0 / 24.0)
        ref = pos.clone()
        api.relax_step(ctx, prm, ref, vol, 20)
        target = api.relax_residual(ctx, prm, ref, vol)[0]
        p_plain = pos.clone()
        n_plain, r_plain = learned.steps_to_target(ctx, prm, p_plain, vol, target, 200, check_every=1)
        p_learn = pos.clone()
        n_learn, r_learn, kept = learned.learned_relax(ctx, prm, trainer.params, p_learn, vol, target, 200,
                                                       check_every=1)
        assert r_plain <= target and r_learn <= target
        gains.append((n_plain, n_learn, kept))
    print("plain steps, learned-run plain steps, proposals kept:", gains)
    # the proposal saves plain steps on every held-out body
    assert all(nl < npl for npl, nl, _ in gains)


# ---------------------------------------------------------------- the learned loop's ABI
def _splitmix64(x):
    # SplitMix64 as published with the generator (Steele, Lea and Flood, OOPSLA 2014),
    # written independently of the library: numpy uint64 wraps modulo 2^64
    with np.errstate(over="ignore"):
        z = np.uint64(x) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _draw(seed, step, batch, rows):
    key = _splitmix64(np.uint64(seed) ^ _splitmix64(np.uint64(step)))
    out = np.empty(batch, dtype=np.int64)
    for b in range(batch):
        with np.errstate(over="ignore"):
            z = int(_splitmix64(key + np.uint64(b)))
        out[b] = (z * rows) >> 64
    return out


def test_relax_samples_equal_the_composed_calls(ctx):
    # sph_relax_samples = features at x^t, `every` plain steps, (x^{t+every} - x^t)/h
    b, prm, pos, vol = learned.body_on_device(ctx, 5, 1.0 / 24.0)
    ref = pos.clone()
    f, t = api.relax_samples(ctx, prm, pos, vol, 3, 7)
    n = pos.shape[1]
    for k in range(3):
        fk = api.mlp_features(ctx, prm, ref)
        x0 = ref.clone()
        api.relax_step(ctx, prm, ref, vol, 7)
        tk = ((host(ref) - host(x0)) / b["h"]).T.astype(np.float32)
        assert torch.equal(f[k * n:(k + 1) * n], fk)
        assert np.array_equal(host(t[k * n:(k + 1) * n]), tk)
    assert torch.equal(pos, ref)


def test_mlp_train_draws_its_minibatches_as_documented(ctx):
    # sph_mlp_train = for each step t: the SplitMix64 minibatch of (seed, t), gathered, and
    # one sph_mlp_train_step; compared bit for bit with the host-drawn batches
    rows, batch, seed = 3000, 256, 77
    X, T = _batch(9, rows)
    Xd, Td = cuda(X, torch.float32), cuda(T, torch.float32)
    flat = inputs.mlp_init(2)
    a = api.MLPTrainer(ctx, flat, lr=1e-3)
    loss_a = a.train(Xd, Td, 4, batch=batch, seed=seed)
    b = api.MLPTrainer(ctx, flat, lr=1e-3)
    for step in range(1, 5):
        idx = torch.tensor(_draw(seed, step, batch, rows), device=Xd.device)
        loss_b = b.step(Xd[idx].contiguous(), Td[idx].contiguous(), with_loss=(step == 4))
    assert torch.equal(a.params, b.params) and torch.equal(a.m, b.m) and torch.equal(a.v, b.v)
    assert loss_a == loss_b and a.step_count == b.step_count == 4


def test_relax_run_plain_and_fallback(ctx):
    b, prm, pos, vol = learned.body_on_device(ctx, 6, 1.0 / 24.0, precision=api.SPH_FP64)
    r0 = api.relax_residual(ctx, prm, pos, vol)[0]
    # plain run to a reachable target, checked every 5 steps: the plain steps composed by hand
    ref = pos.clone()
    target = 0.9 * r0
    done, r = 0, r0
    while r > target and done < 100:
        api.relax_step(ctx, prm, ref, vol, 5)
        done += 5
        r = api.relax_residual(ctx, prm, ref, vol)[0]
    p = pos.clone()
    out = api.relax_run(ctx, prm, p, vol, target, 100, proposal=None, check_every=5)
    assert out["reached"] and out["steps"] == done and not out["fell_back"]
    assert torch.equal(p, ref) and out["residual"][0] == r
    # a proposal that only makes things worse (a network with large outputs) is undone; an
    # unreachable target then makes plain relaxation from the start the result
    bad = torch.tensor(inputs.mlp_init(3), dtype=torch.float32, device=ctx.device)
    bad[-3 - 3 * 128:-3] *= 3.0          # untrained, output layer tripled: random moves of ~h
    p = pos.clone()
    out = api.relax_run(ctx, prm, p, vol, 0.0, 12, proposal=bad, applications=3, plain_between=4, check_every=4)
    assert out["rejected"] == 1 and out["kept"] == 0
    assert out["fell_back"] and not out["reached"] and out["steps"] == 12
    plain = pos.clone()
    api.relax_step(ctx, prm, plain, vol, 12)
    assert torch.equal(p, plain)
