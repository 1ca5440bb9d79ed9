"""FP64 CPU reference of the grain-optics surrogate: its training labels and the MLP
forward / backward.  TEST INFRASTRUCTURE ONLY (used by tests/ and bench.py's CPU
baseline leg, never by the product package).

Labels (what the network learns), from the method's own tables (Sec. 2.2: the
Mueller matrix may be supplied analytically, as tables, or by a network):
  input  u = (n_i, n_s, s): incident and scattered directions in the grain frame
         (unit vectors) and s in [-1, 1], the position of ln x between the first and
         last tabulated size parameter;
  P(Theta; s) = the bin tables interpolated linearly in the scattering angle and
         linearly in ln x between neighbouring bins;
  M    = the 4x4 scattering matrix in the scattering-plane basis (Sec. 2.1: the
         Stokes vector is rotated into the scattering plane, multiplied, rotated out),
         [[P11, P12, 0, 0], [P12, P22, 0, 0], [0, 0, P33, P34], [0, 0, -P34, P44]] for
         these tables; a network for aligned grains learns the general 16 entries as
         functions of both grain-frame directions;
  N(s) = max over the tabulated angles of the interpolated P11;
  outputs: ln M11 (= ln P11, 1/sr), the other 15 entries of M divided by M11
         (row-major, (0,0) left out), alpha1..3 at the polar angle of n_i (the
         extinction table, linear in theta'), ln N.  The logarithm and the ratios give
         every direction the same relative accuracy although P11 of a
         forward-scattering bin spans about three decades; the plane rotations stay
         exact geometry outside the network.
MLP: 16 (7 inputs, zero padded) -> 128 -> 128 -> 128 -> 128 -> 24 (20 used), SiLU
after every hidden layer, weights W_l [n_out][n_in], biases b_l.
"""
from __future__ import annotations

import math

import numpy as np


N_IN, N_IN_PAD, HIDDEN, N_OUT, N_OUT_PAD = 7, 16, 128, 20, 24
LAYERS = [(N_IN_PAD, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, N_OUT_PAD)]


# ----------------------------------------------------------------------------------
# labels
# ----------------------------------------------------------------------------------
def interp_bins(tabs, s):
    """Tables [n_bins][n_theta][6] interpolated linearly in ln x at s in [-1, 1]."""
    nb = tabs.shape[0]
    if nb == 1:  # a single size bin: nothing to interpolate in ln x
        return tabs[0].astype(np.float64)
    b = (min(max(s, -1.0), 1.0) + 1.0) * 0.5 * (nb - 1)
    k = min(int(math.floor(b)), nb - 2)
    f = b - k
    return (1.0 - f) * tabs[k].astype(np.float64) + f * tabs[k + 1].astype(np.float64)


def theta_interp(tab, mu):
    n_theta = tab.shape[0]
    x = math.acos(min(max(mu, -1.0), 1.0)) / math.pi * (n_theta - 1)
    j = min(int(math.floor(x)), n_theta - 2)
    f = x - j
    return (1.0 - f) * tab[j] + f * tab[j + 1]


def kext_interp(kext, cos_t):
    n = kext.shape[0]
    x = math.acos(min(max(cos_t, -1.0), 1.0)) / math.pi * (n - 1)
    j = min(int(math.floor(x)), n - 2)
    f = x - j
    return (1.0 - f) * kext[j].astype(np.float64) + f * kext[j + 1].astype(np.float64)


def label(u, tabs, kext):
    """20 targets for one input u = (n_i[3], n_s[3], s)."""
    ni, ns, s = np.asarray(u[0:3], float), np.asarray(u[3:6], float), float(u[6])
    tab = interp_bins(tabs, s)
    N = float(tab[:, 0].max())
    P11, P12, P22, P33, P34, P44 = theta_interp(tab, float(np.dot(ni, ns)))
    M = np.array([[P11, P12, 0.0, 0.0], [P12, P22, 0.0, 0.0], [0.0, 0.0, P33, P34], [0.0, 0.0, -P34, P44]])
    out = np.zeros(N_OUT)
    flat = M.ravel()
    out[0] = math.log(flat[0])
    out[1:16] = flat[1:16] / flat[0]
    out[16:19] = kext_interp(kext, ni[2])
    out[19] = math.log(N)
    return out


def matrix(out):
    """The 4x4 scattering-plane matrix encoded by the first 16 outputs."""
    out = np.asarray(out, dtype=float)
    r = np.concatenate([[1.0], out[1:16]])
    return math.exp(out[0]) * r.reshape(4, 4)


# ----------------------------------------------------------------------------------
# MLP
# ----------------------------------------------------------------------------------
def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def pad_inputs(u):
    u = np.atleast_2d(np.asarray(u, float))
    x = np.zeros((u.shape[0], N_IN_PAD))
    x[:, :N_IN] = u
    return x


def forward(params, x):
    """params: list of (W [n_out][n_in], b [n_out]); x [B][16].  Returns outputs
    [B][24] and the cache of pre-activations and layer inputs."""
    h = x
    cache = []
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if i < len(params) - 1 else z
    return h, cache


def loss_and_grads(params, x, t, weights):
    """Loss = sum_b sum_o w_o (y_bo - t_bo)^2 / (B * 20) over the 20 used outputs and
    the gradients of every W, b (backpropagation written out layer by layer)."""
    y, cache = forward(params, x)
    B = x.shape[0]
    r = y[:, :N_OUT] - t
    loss = float(np.sum(weights * r * r) / (B * N_OUT))
    dy = np.zeros_like(y)
    dy[:, :N_OUT] = 2.0 * weights * r / (B * N_OUT)
    grads = [None] * len(params)
    g = dy
    for i in range(len(params) - 1, -1, -1):
        h_in, z = cache[i]
        W, b = params[i]
        dz = g if i == len(params) - 1 else g * silu_grad(z)
        grads[i] = (dz.T @ h_in, dz.sum(axis=0))
        g = dz @ W
    return loss, grads
