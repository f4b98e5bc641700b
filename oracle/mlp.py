"""Learned diagonal preconditioner: the per-Gaussian MLP, in float64.

The paper uses the Jacobi preconditioner M^-1 = 1 / diag(J^T J) (Sec. 3.3,
Algorithm 1). This module is the oracle for the learned replacement: a small
per-Gaussian network whose softplus output gives a positive diagonal D, so that
z = D r keeps PCG on a symmetric positive definite system. The paper has no
such network; the reading below is this project's:

  features phi (64) per Gaussian, from one image subset's linear system:
      log(M_k + 1e-12), k = 0..58    the subset's diag(J^T J)
      log-scale (3), opacity sigmoid(logit) (1)
      log(1 + entries)               cache entries that touch the Gaussian
  standardised with a per-feature mean and standard deviation;
  network  h1 = GELU(W1 phi + b1), h2 = GELU(W2 h1 + b2), o = W3 h2 + b3
           (64 -> 64 -> 64 -> 59, exact GELU x Phi(x))
  output   c = softplus(o), D_k = c_k / clamp(M_k)   (clamp as for Jacobi)
  weights  the network computes with its weight matrices rounded to bfloat16
           (round to nearest even from float32), its biases and everything else
           in float64 here; the weights kept and updated are masters, and the
           weight gradient is that of the rounded weights (bf16=False: exact).
           The biases are not rounded, so the initial network is exactly Jacobi
  init     W3 = 0, b3 = log(e - 1): c = 1, i.e. D = the Jacobi preconditioner
  loss     L = 1/2 log(||r_K||^2 / ||b||^2): the relative residual after K
           iterations of Algorithm 1 run with D in place of M^-1 (x0 = D b,
           z = D r) on the subset system A = J^T J + lambda clamp(M); its
           gradient in D is the reverse mode of those K iterations
           (unrolled_loss_and_grad), then the network's own reverse mode
  training Adam (beta1 0.9, beta2 0.999, eps 1e-8)

A warm-start loss (fit D b to the converged solution) was tried first and
rejected: it drives many entries of D towards zero, and PCG with that D no
longer converges.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf

from .solver import clamp_diag

N_IN, N_HID, N_OUT = 64, 64, 59
B3_INIT = math.log(math.e - 1.0)        # softplus(B3_INIT) = 1


@dataclass
class MLP:
    W1: np.ndarray   # (64, 64)  out x in
    b1: np.ndarray   # (64,)
    W2: np.ndarray   # (64, 64)
    b2: np.ndarray   # (64,)
    W3: np.ndarray   # (59, 64)
    b3: np.ndarray   # (59,)

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]

    def flat(self) -> np.ndarray:
        return np.concatenate([p.ravel() for p in self.params()])

    @staticmethod
    def from_flat(v: np.ndarray) -> "MLP":
        shapes = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]
        out, o = [], 0
        for s in shapes:
            n = int(np.prod(s))
            out.append(np.asarray(v[o:o + n], np.float64).reshape(s).copy())
            o += n
        return MLP(*out)


N_WEIGHTS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_OUT * N_HID + N_OUT


def init_mlp(seed: int, scale: float = 0.5) -> MLP:
    """Hidden layers ~ N(0, scale^2 / fan_in); output layer zero with bias log(e - 1)."""
    rng = np.random.default_rng([seed, 11])
    W1 = rng.standard_normal((N_HID, N_IN)) * (scale / math.sqrt(N_IN))
    W2 = rng.standard_normal((N_HID, N_HID)) * (scale / math.sqrt(N_HID))
    return MLP(W1, np.zeros(N_HID), W2, np.zeros(N_HID), np.zeros((N_OUT, N_HID)), np.full(N_OUT, B3_INIT))


def features(M: np.ndarray, params: np.ndarray, entries: np.ndarray) -> np.ndarray:
    """phi (N, 64) from diag(J^T J) (N, 59), the parameters (N, 59) and entries per Gaussian (N,)."""
    P = np.asarray(params, np.float64)
    return np.concatenate([
        np.log(np.asarray(M, np.float64) + 1e-12),
        P[:, 3:6],
        (1.0 / (1.0 + np.exp(-P[:, 10])))[:, None],
        np.log1p(np.asarray(entries, np.float64))[:, None],
    ], axis=1)


def standardizer(phi: np.ndarray):
    """Per-feature mean and standard deviation (std floored at 1e-6)."""
    mu = phi.mean(axis=0)
    sd = np.maximum(phi.std(axis=0), 1e-6)
    return mu, sd


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """x rounded to the nearest bfloat16 (the upper 16 bits of its float32,
    round half to even), as float64. bfloat16 keeps float32's sign and 8-bit
    exponent and the top 7 of its 23 mantissa bits."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def effective(net: MLP, bf16: bool = True) -> MLP:
    """The weights the network computes with: the matrices rounded to bfloat16
    (biases exact), or all exact."""
    if not bf16:
        return net
    return MLP(bf16_round(net.W1), net.b1, bf16_round(net.W2), net.b2, bf16_round(net.W3), net.b3)


def forward(net: MLP, phi_hat: np.ndarray, bf16: bool = True):
    """Returns (a1, h1, a2, h2, o) for standardised features (N, 64)."""
    net = effective(net, bf16)
    a1 = phi_hat @ net.W1.T + net.b1
    h1 = gelu(a1)
    a2 = h1 @ net.W2.T + net.b2
    h2 = gelu(a2)
    o = h2 @ net.W3.T + net.b3
    return a1, h1, a2, h2, o


def precond_diag(net: MLP, phi_hat: np.ndarray, M: np.ndarray, bf16: bool = True) -> np.ndarray:
    """D (N, 59) = softplus(o) / clamp(M)."""
    o = forward(net, phi_hat, bf16)[-1]
    return softplus(o) / clamp_diag(M)


def backward(net: MLP, phi_hat: np.ndarray, M: np.ndarray, dD: np.ndarray, bf16: bool = True):
    """Weight gradients (list matching net.params()) for an upstream gradient dL/dD (N, 59),
    taken at the weights the network computes with (see effective)."""
    a1, h1, a2, h2, o = forward(net, phi_hat, bf16)
    net = effective(net, bf16)
    do = dD / clamp_diag(M) * sigmoid(o)           # D = softplus(o) / clamp(M)
    gW3 = do.T @ h2
    gb3 = do.sum(axis=0)
    da2 = (do @ net.W3) * gelu_grad(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ net.W2) * gelu_grad(a1)
    gW1 = da1.T @ phi_hat
    gb1 = da1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


@dataclass
class Tape:
    """Forward values of the unrolled iterations kept for the reverse pass."""
    r: list          # r_0 .. r_K
    p: list          # p_0 .. p_{K-1}
    g: list          # g_i = A p_i
    rho: list        # rho_i = r_i . z_i, i = 0 .. K
    pg: list         # p_i . g_i
    alpha: list
    beta: list


def unrolled_pcg(apply_A, b: np.ndarray, d: np.ndarray, K: int):
    """K iterations of Algorithm 1 with the diagonal d as preconditioner:
    x0 = d b, r0 = b - A x0, z = d r, p0 = z0, then alpha = rho / p.Ap,
    r -= alpha A p, beta = rho_new / rho, p = z + beta p. Returns (x_K, tape)."""
    x = d * b
    r = b - apply_A(x)
    z = d * r
    p = z.copy()
    tp = Tape([r], [], [], [float(np.vdot(r, z))], [], [], [])
    for _ in range(K):
        g = apply_A(p)
        pg = float(np.vdot(p, g))
        alpha = tp.rho[-1] / pg
        x = x + alpha * p
        r = r - alpha * g
        z = d * r
        rho = float(np.vdot(r, z))
        beta = rho / tp.rho[-1]
        tp.p.append(p)
        tp.g.append(g)
        tp.pg.append(pg)
        tp.alpha.append(alpha)
        tp.beta.append(beta)
        tp.r.append(r)
        tp.rho.append(rho)
        p = z + beta * p
    return x, tp


def unrolled_loss_and_grad(apply_A, b: np.ndarray, d: np.ndarray, K: int):
    """L = 1/2 log(||r_K||^2 / ||b||^2) of unrolled_pcg and dL/dd, by reverse mode
    through the iterations (A symmetric, so the adjoint of g = A p is pbar += A gbar)."""
    _, tp = unrolled_pcg(apply_A, b, d, K)
    rK = tp.r[K]
    rr = float(np.vdot(rK, rK))
    L = 0.5 * math.log(rr / float(np.vdot(b, b)))
    dbar = np.zeros_like(d)
    rbar = rK / rr                                  # dL/dr_K
    pbar = np.zeros_like(d)                         # adjoint of p_{i+1}
    rhobar = [0.0] * (K + 1)
    for i in range(K - 1, -1, -1):
        r1, z1 = tp.r[i + 1], d * tp.r[i + 1]
        # p_{i+1} = z_{i+1} + beta_i p_i
        zbar = pbar.copy()
        betabar = float(np.vdot(pbar, tp.p[i]))
        pbar_i = tp.beta[i] * pbar
        # beta_i = rho_{i+1} / rho_i
        rhobar[i + 1] += betabar / tp.rho[i]
        rhobar[i] -= betabar * tp.rho[i + 1] / tp.rho[i] ** 2
        # rho_{i+1} = r_{i+1} . z_{i+1};  z_{i+1} = d r_{i+1}
        rbar = rbar + rhobar[i + 1] * z1
        zbar = zbar + rhobar[i + 1] * r1
        rbar = rbar + d * zbar
        dbar += r1 * zbar
        # r_{i+1} = r_i - alpha_i g_i
        alphabar = -float(np.vdot(rbar, tp.g[i]))
        gbar = -tp.alpha[i] * rbar
        # alpha_i = rho_i / (p_i . g_i)
        rhobar[i] += alphabar / tp.pg[i]
        pgbar = -alphabar * tp.rho[i] / tp.pg[i] ** 2
        # pg_i = p_i . g_i;  g_i = A p_i
        pbar_i = pbar_i + pgbar * tp.g[i]
        gbar = gbar + pgbar * tp.p[i]
        pbar = pbar_i + apply_A(gbar)
        # rbar now holds dL/dr_i (r_{i+1} depends on r_i with unit weight)
    # p_0 = z_0, rho_0 = r_0 . z_0, z_0 = d r_0
    r0 = tp.r[0]
    zbar = pbar + rhobar[0] * r0
    rbar = rbar + rhobar[0] * (d * r0) + d * zbar
    dbar += r0 * zbar
    # r_0 = b - A x_0, x_0 = d b
    dbar += b * (-apply_A(rbar))
    return L, dbar


def loss_and_grad(net: MLP, phi_hat: np.ndarray, M: np.ndarray, apply_A, b: np.ndarray, K: int,
                  bf16: bool = True):
    """Unrolled-PCG loss of the network's D on one system and its weight gradients."""
    D = precond_diag(net, phi_hat, M, bf16)
    L, dD = unrolled_loss_and_grad(apply_A, b, D, K)
    return L, backward(net, phi_hat, M, dD, bf16)


@dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: list = None
    v: list = None

    def step(self, net: MLP, grads: list) -> None:
        if self.m is None:
            self.m = [np.zeros_like(g) for g in grads]
            self.v = [np.zeros_like(g) for g in grads]
        self.t += 1
        for p, g, m, v in zip(net.params(), grads, self.m, self.v):
            m *= self.beta1
            m += (1 - self.beta1) * g
            v *= self.beta2
            v += (1 - self.beta2) * g * g
            mh = m / (1 - self.beta1 ** self.t)
            vh = v / (1 - self.beta2 ** self.t)
            p -= self.lr * mh / (np.sqrt(vh) + self.eps)
