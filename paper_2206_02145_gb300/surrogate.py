"""Learned block propagator, 2D: the seeded problem sampler, training pairs
generated by the LB solver, the training loop and the LB-versus-network
comparison.

Every computation runs in the library's kernels (LB steps, normalisation,
targets, the network's forward / backward / Adam); this module schedules
them and gathers minibatches from device buffers.

Problems are closed channels, so that the solute invariant sum(U + phi(t-1))
of Eq. 13 is conserved and the propagator's drift check is meaningful:
periodic in x, half-way bounce-back walls in y, the flow driven by a body
force g with its steady Poiseuille profile u(y) = g (y + 1/2)(ny - 1/2 - y) /
(2 nu) as the initial velocity (nu = (tau_f - 1/2) / 3, Eq. 10), and a
seed at the centre (the origin of the interface rays).  The sweep draws the
supersaturation, seed size, flow speed, fold, anisotropy strength and
orientation, as the paper's parametric studies vary them.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (Sim, UNet, current_stream, lbpf_surrogate_advance, lbpf_surrogate_sample,
               lbpf_surrogate_target, lbpf_surrogate_train, surrogate_cfg)

__all__ = ["channel_problem", "make_sim", "default_cfg", "generate_pairs", "train_schedule",
           "train", "inference_net", "prediction_error", "surrogate_cfg",
           "lbpf_surrogate_advance"]


def channel_problem(rng: np.random.Generator, nx: int, ny: int, tau_f: float = 0.6,
                    w0: float = 2.0, noise: float = 0.01):
    """One draw of the sweep: (params for Sim, fields for Sim.init_fields)."""
    u0 = float(rng.uniform(0.25, 0.45))
    radius = float(rng.uniform(6.0, 16.0))
    umax = float(rng.uniform(0.0, 0.01))
    fold = int(rng.choice([4, 5]))
    eps = float(rng.uniform(0.02, 0.05))
    theta0 = float(rng.uniform(0.0, 2.0 * math.pi / fold))
    nu = (tau_f - 0.5) / 3.0
    g = 8.0 * nu * umax / (ny * ny)
    params = dict(dim=2, nx=nx, ny=ny, flow=1, bc=(0, 2, 0), fold=fold, eps_aniso=eps,
                  theta0=theta0, tau_f=tau_f, w0=w0, body_force=(g, 0.0, 0.0))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(x - nx // 2, y - ny // 2)
    phi = np.tanh((radius - r) / (math.sqrt(2.0) * w0))
    phi += noise * rng.uniform(-1.0, 1.0, size=phi.shape)
    U = np.full_like(phi, u0)
    ux = np.broadcast_to((g / (2.0 * nu) * (y[:, :1] + 0.5) * (ny - 0.5 - y[:, :1])),
                         phi.shape).copy()
    info = dict(u0=u0, radius=radius, umax=umax, fold=fold, eps=eps, theta0=theta0)
    return params, dict(phi=phi, U=U, ux=ux, uy=np.zeros_like(phi)), info


def make_sim(params: dict, fields: dict, stream: int | None = None) -> Sim:
    sim = Sim(stream=stream if stream is not None else current_stream(), **params)
    sim.init_fields(fields["phi"], fields["U"], None, fields["ux"], fields["uy"])
    return sim


def default_cfg(steps_per_block: int = 50, **kw):
    """Propagator settings for the channel problems: inputs (phi, U, ux, uy)
    shifted and scaled to O(1), outputs scaled by about four standard
    deviations of the change near the crystal over a 50-step block (measured
    on the sampler's trajectories), growing with the square root of the block
    length as diffusive changes do."""
    g = math.sqrt(steps_per_block / 50.0)
    kw.setdefault("res_scale", (0.02 * g, 0.012 * g, 0.0015 * g, 0.001 * g))
    return surrogate_cfg(steps_per_block=steps_per_block, shift=(0.0, 0.3, 0.0, 0.0),
                         scale=(1.0, 0.2, 0.01, 0.01), **kw)


def generate_pairs(n_traj: int, t_end: int, every: int, nx: int, ny: int, cfg, seed: int,
                   crop: int | None = None, t_start: int = 0, device="cuda"):
    """Pairs (x(t), target) from n_traj sampled problems, at t = t_start,
    t_start + every, ... < t_end: x(t) the normalised fields, target the
    normalised change over cfg.steps_per_block LB steps.  crop: keep only a
    band of `crop` rows centred on the seed, where the fields change, at full
    width (the network's deepest level needs the width); a convolutional
    network trained on bands applies to the whole domain.
    Returns device tensors X, T of shape [N, h, nx, 4]."""
    nb = cfg.steps_per_block
    assert every >= nb and (t_end - t_start) % every == 0
    per = (t_end - t_start) // every
    N = n_traj * per
    h, w = (crop, nx) if crop else (ny, nx)
    y0, x0 = (ny // 2 - h // 2, 0) if crop else (0, 0)
    X = torch.empty(N, h, w, 4, device=device)
    T = torch.empty_like(X)
    x0f = torch.empty(ny, nx, 4, device=device)
    x1f = torch.empty_like(x0f)
    tf = torch.empty_like(x0f)
    rng = np.random.default_rng(seed)
    k = 0
    for _ in range(n_traj):
        params, fields, _ = channel_problem(rng, nx, ny)
        sim = make_sim(params, fields)
        if t_start:
            sim.step(t_start)
        for _ in range(per):
            lbpf_surrogate_sample(sim, cfg, x0f)
            sim.step(nb)
            lbpf_surrogate_sample(sim, cfg, x1f)
            lbpf_surrogate_target(cfg, x0f, x1f, ny * nx, tf, current_stream())
            X[k].copy_(x0f[y0:y0 + h, x0:x0 + w])
            T[k].copy_(tf[y0:y0 + h, x0:x0 + w])
            sim.step(every - nb)
            k += 1
        sim.close()
    torch.cuda.synchronize()
    return X, T


def train_schedule(n_pairs: int, batch: int, steps: int, lr: float = 5e-4, seed: int = 0,
                   augment: bool = True):
    """The draws of the training loop: minibatch pair indices [steps, batch],
    mirror choices [steps] (0 none, 1 in y, 2 in x: the channel problems'
    mirror symmetries, y -> -y with uy -> -uy and x -> -x with ux -> -ux) and
    the cosine-decayed learning rate [steps], floored at 2 % of lr."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    idx = np.empty((steps, batch), np.int32)
    flip = np.zeros(steps, np.int32)
    rates = np.empty(steps, np.float32)
    for s in range(steps):
        idx[s] = torch.randint(0, n_pairs, (batch,), generator=g).numpy()
        if augment:
            flip[s] = int(torch.randint(0, 3, (1,), generator=g))
        a = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(steps, 1)))
        rates[s] = max(a, lr * 0.02)
    return idx, flip, rates


def train(net: UNet, X, T, steps: int, lr: float = 5e-4, seed: int = 0, log_every: int = 50,
          augment: bool = True):
    """Adam on random minibatches of net's batch size, cosine-decayed learning
    rate; with augment, each minibatch is mirrored in x or y (or left as is)
    at random.  The loop runs in the library (lbpf_surrogate_train).  Returns
    [(step, loss)] at every log_every-th step and the last."""
    idx, flip, rates = train_schedule(int(X.shape[0]), net.cfg.batch, steps, lr, seed, augment)
    losses = lbpf_surrogate_train(net, X, T, idx, flip, rates, log_every)
    at = [s + 1 for s in range(steps) if (s + 1) % log_every == 0 or s == steps - 1]
    return [(a, float(v)) for a, v in zip(at, losses)]


def inference_net(trained: UNet, nx: int, ny: int, stream: int | None = None) -> UNet:
    """A batch-1 network of the same architecture carrying trained's weights."""
    c = trained.cfg
    net = UNet(in_ch=c.in_ch, out_ch=c.out_ch, base_ch=c.base_ch, levels=c.levels, batch=1,
               height=ny, width=nx, seed=c.seed,
               stream=stream if stream is not None else current_stream())
    net.set_weights(trained.weights())
    return net


def prediction_error(net: UNet, X, T) -> tuple[float, float]:
    """Mean squared error of the network on pairs (X, T) and of predicting no
    change ("no network"), both in the normalised target units."""
    y = torch.empty_like(X[0])
    err = base = 0.0
    for k in range(X.shape[0]):
        net.forward(X[k], y)
        err += float(((y - T[k]) ** 2).mean())
        base += float((T[k] ** 2).mean())
    return err / X.shape[0], base / X.shape[0]
