"""FP64 oracle of the learned diagonal preconditioner (TEST INFRASTRUCTURE ONLY).

Nothing on the product path imports this module; the tests and the smoke check do.

The paper solves its linear systems without saying how they are preconditioned; the
learned preconditioner is an addition on top of the method, defined as follows.  For one
per-shift system (P_c H P_c - z) x = b, plane wave G gets the diagonal scaling

    plain    M_G = 1 / max(1, T_G / e_prec),  e_prec = 1.35 <r|T|r> / <r|r>  (r: the rhs given)
    Jacobi   J_G = 1 / max(|H_GG - z|, delta),  H_GG = T_G + <V_loc> + sum_p D_p |beta_p(G)|^2
    learned  M_G exp(f_theta(phi_G)),  phi_G = (T_G / (E_cut / 2), omega / 2.205 Ha, e_ref, <V_loc>)

with f_theta a 4 -> 64 -> 64 -> 1 perceptron with erf-GELU activations.  An untrained
network has a zero last layer, so it reproduces M.  A training pair is solved with M and
with J at several floors delta; the target of each of its plane waves is
log(clip(J_G / M_G, e^-3, e^3)) at the fastest floor (0 if M was fastest).  The loss is the
mean squared error; Adam (Kingma & Ba) updates FP32 master weights; the network evaluates
with its weights rounded to bfloat16 (round to nearest even), accumulating in FP32 on the
GPU and in FP64 here.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_IN, N_H = 4, 64
SHAPES = [("w1", (N_H, N_IN)), ("b1", (N_H,)), ("w2", (N_H, N_H)), ("b2", (N_H,)), ("w3", (1, N_H)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)       # 4545
HA_OMEGA_SCALE = 2.205                                   # Ha (60 eV)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even); returned as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    """x Phi(x) = x (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, feats, cache=False):
    """f_theta for rows feats [n][4]; returns [n] (and the activations when cache)."""
    p = unpack(theta)
    x = np.asarray(feats, dtype=np.float64)
    a1 = x @ p["w1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["w2"].T + p["b2"]
    h2 = gelu(a2)
    y = (h2 @ p["w3"].T + p["b3"])[:, 0]
    if cache:
        return y, (x, a1, h1, a2, h2)
    return y


def loss_and_grad(theta, feats, targets):
    """Mean squared error and its gradient with respect to theta (backpropagation)."""
    p = unpack(theta)
    y, (x, a1, h1, a2, h2) = forward(theta, feats, cache=True)
    n = len(y)
    r = y - np.asarray(targets, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = (2.0 / n) * r                     # d loss / d y
    g = {}
    g["w3"] = dy[None, :] @ h2
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] * p["w3"][0][None, :]
    da2 = dh2 * gelu_grad(a2)
    g["w2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["w2"]
    da1 = dh1 * gelu_grad(a1)
    g["w1"] = da1.T @ x
    g["b1"] = da1.sum(0)
    return loss, pack(g)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step count t starting at 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(rng):
    """He-uniform hidden layers, zero last layer (the untrained net reproduces M_G)."""
    p = {}
    for name, shp in SHAPES:
        if name.startswith("b") or name == "w3":
            p[name] = np.zeros(shp)
        else:
            lim = math.sqrt(6.0 / shp[1])
            p[name] = rng.uniform(-lim, lim, size=shp)
    return pack(p).astype(np.float32)


def plain_scaling(kin, b):
    """M_G = 1 / max(1, T_G / e_prec), e_prec = 1.35 <b|T|b> / <b|b>."""
    w = np.abs(np.asarray(b)) ** 2
    e_prec = 1.35 * float(np.sum(w * kin) / np.sum(w))
    return 1.0 / np.maximum(1.0, kin / e_prec)


def features(kin, ecut_ry, omega, e_ref, v_mean):
    kin = np.asarray(kin, dtype=np.float64)
    f = np.empty((len(kin), N_IN))
    f[:, 0] = kin / (0.5 * ecut_ry)
    f[:, 1] = omega / HA_OMEGA_SCALE
    f[:, 2] = e_ref
    f[:, 3] = v_mean
    return f


def h_diag(kin, v_mean, beta, dkb):
    """Diagonal of H in the plane-wave basis: T_G + V(0) + sum_p D_p |beta_p(G)|^2."""
    return np.asarray(kin) + v_mean + np.sum(np.asarray(dkb)[:, None] * np.abs(beta) ** 2, axis=0)


def jacobi_scaling(hdiag, z, delta):
    return 1.0 / np.maximum(np.abs(np.asarray(hdiag) - z), delta)


def targets(m, j):
    """log(clip(J / M, e^-3, e^3)); pass j = None when the plain scaling was fastest."""
    if j is None:
        return np.zeros_like(m)
    return np.clip(np.log(j / m), -3.0, 3.0)
