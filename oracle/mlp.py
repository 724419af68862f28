"""FP64 reference of the learned beam: a Fourier-feature MLP
(az, za, nu, antenna) -> beam components.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64,
written from the definitions below; it shares nothing with the CUDA library.

The paper's beams are gridded (UVBeam) or analytic (Sec. 2.4); a learned
surrogate of per-antenna gridded beams is not in the paper, so the
definitions here are the surrogate's own:

  coordinates   x = (az / 2 pi, za / (pi/2), (nu - nu_mid) / nu_half)
  features      f(x) = [sin(2 pi B x), cos(2 pi B x), e_a]      (2 F + E values)
                with B a fixed F x 3 matrix and e_a the antenna's embedding
  layers        h_0 = f,  h_l = relu(W_l h_{l-1} + b_l)  (l = 1..L hidden)
                y = W_out h_L + b_out                     (n_out values)
  loss          mean over samples and outputs of (y - t)^2
  optimiser     Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g,
                v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)

Weights are stored as W_l[out][in] (row = output unit).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class MLP:
    B: np.ndarray                 # [F][3] Fourier frequencies
    emb: np.ndarray               # [n_ant][E]
    W: List[np.ndarray]           # W[l]: [out][in]; last is the output layer
    b: List[np.ndarray]
    nu_mid: float = 150e6
    nu_half: float = 52e6
    m: dict = field(default_factory=dict)   # Adam state
    v: dict = field(default_factory=dict)
    k: int = 0

    def params(self):
        d = {"emb": self.emb}
        for i, (w, bb) in enumerate(zip(self.W, self.b)):
            d[f"W{i}"] = w
            d[f"b{i}"] = bb
        return d


def coords(az, za, nu, nu_mid, nu_half):
    return np.stack([np.asarray(az) / (2 * np.pi), np.asarray(za) / (np.pi / 2),
                     (np.asarray(nu) - nu_mid) / nu_half], axis=-1)


def features(net: MLP, ant, az, za, nu):
    x = coords(az, za, nu, net.nu_mid, net.nu_half)          # [n][3]
    ph = 2 * np.pi * x @ net.B.T                               # [n][F]
    return np.concatenate([np.sin(ph), np.cos(ph), net.emb[np.asarray(ant)]], axis=1)


def forward(net: MLP, ant, az, za, nu, keep=False):
    h = features(net, ant, az, za, nu)
    acts = [h]
    for w, bb in zip(net.W[:-1], net.b[:-1]):
        h = np.maximum(h @ w.T + bb, 0.0)
        acts.append(h)
    y = h @ net.W[-1].T + net.b[-1]
    return (y, acts) if keep else y


def loss_and_grads(net: MLP, ant, az, za, nu, target):
    """MSE loss and its gradient with respect to every parameter."""
    y, acts = forward(net, ant, az, za, nu, keep=True)
    n = y.shape[0]
    r = y - target
    loss = float(np.mean(r * r))
    dy = 2.0 * r / r.size
    g = {}
    L = len(net.W) - 1
    d = dy
    for l in range(L, -1, -1):
        g[f"W{l}"] = d.T @ acts[l]
        g[f"b{l}"] = d.sum(axis=0)
        dh = d @ net.W[l]
        if l > 0:
            d = dh * (acts[l] > 0)
        else:
            d0 = dh
    E = net.emb.shape[1]
    ge = np.zeros_like(net.emb)
    np.add.at(ge, np.asarray(ant), d0[:, -E:])
    g["emb"] = ge
    return loss, g


def adam_step(net: MLP, grads: dict, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    net.k += 1
    for name, p in net.params().items():
        g = grads[name]
        m = net.m.setdefault(name, np.zeros_like(p))
        v = net.v.setdefault(name, np.zeros_like(p))
        m *= b1
        m += (1 - b1) * g
        v *= b2
        v += (1 - b2) * g * g
        mh = m / (1 - b1 ** net.k)
        vh = v / (1 - b2 ** net.k)
        p -= lr * mh / (np.sqrt(vh) + eps)
