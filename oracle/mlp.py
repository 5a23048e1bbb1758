"""FP64 reference MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatement of the warm-start network: an MLP with GELU hidden
activations (exact erf form), mean-squared error on affinely normalized
targets, hand-derived backward pass and Adam. It checks the GPU's BF16
tensor-core training and inference kernels. (The paper uses no neural network;
this network only proposes Newton initial guesses; the solve decides the answer.)
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


class OracleMLP:
    """Layers W_l (n_out x n_in), b_l; hidden layers GELU, last layer linear.
    Inputs are normalized as (x - in_shift) * in_scale; the network predicts
    normalized outputs t = (y - out_shift) * out_scale."""

    def __init__(self, sizes, in_shift, in_scale, out_shift, out_scale, weights=None):
        self.sizes = list(sizes)
        self.in_shift = np.asarray(in_shift, np.float64)
        self.in_scale = np.asarray(in_scale, np.float64)
        self.out_shift = np.asarray(out_shift, np.float64)
        self.out_scale = np.asarray(out_scale, np.float64)
        self.W = [np.asarray(w, np.float64).copy() for w in weights[0]]
        self.b = [np.asarray(b, np.float64).copy() for b in weights[1]]
        self.mW = [np.zeros_like(w) for w in self.W]
        self.vW = [np.zeros_like(w) for w in self.W]
        self.mb = [np.zeros_like(b) for b in self.b]
        self.vb = [np.zeros_like(b) for b in self.b]
        self.t = 0

    def forward(self, x, keep=False):
        a = (np.asarray(x, np.float64) - self.in_shift) * self.in_scale
        acts, zs = [a], []
        L = len(self.W)
        for l in range(L):
            z = a @ self.W[l].T + self.b[l]
            zs.append(z)
            a = gelu(z) if l < L - 1 else z
            acts.append(a)
        return (a, acts, zs) if keep else a

    def predict(self, x):
        """Physical outputs y = t / out_scale + out_shift."""
        return self.forward(x) / self.out_scale + self.out_shift

    def loss_and_grads(self, x, y):
        """MSE over batch and outputs on normalized targets; gradients dL/dW, dL/db."""
        t = (np.asarray(y, np.float64) - self.out_shift) * self.out_scale
        out, acts, zs = self.forward(x, keep=True)
        B, m = t.shape
        diff = out - t
        loss = float(np.sum(diff * diff) / (B * m))
        dz = 2.0 * diff / (B * m)
        L = len(self.W)
        gW = [None] * L
        gb = [None] * L
        for l in range(L - 1, -1, -1):
            gW[l] = dz.T @ acts[l]
            gb[l] = dz.sum(0)
            if l > 0:
                dz = (dz @ self.W[l]) * gelu_grad(zs[l - 1])
        return loss, gW, gb

    def adam_step(self, gW, gb, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        c1 = 1.0 - b1 ** self.t
        c2 = 1.0 - b2 ** self.t
        for l in range(len(self.W)):
            for P, g, mm, vv in ((self.W, gW, self.mW, self.vW), (self.b, gb, self.mb, self.vb)):
                mm[l] = b1 * mm[l] + (1 - b1) * g[l]
                vv[l] = b2 * vv[l] + (1 - b2) * g[l] * g[l]
                P[l] = P[l] - lr * (mm[l] / c1) / (np.sqrt(vv[l] / c2) + eps)
