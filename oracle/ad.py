"""Forward-mode automatic differentiation with dual numbers, vectorised over splats.

A ``Dual`` carries a value array ``v`` of shape (S,) and its derivative array
``d`` of shape (S, n) with respect to n seeded inputs. Every operation applies
the exact rule of differential calculus, so the derivative of a composite
function is exact up to float64 rounding. The oracle uses it to obtain the
per-splat Jacobian dy/dx of the projection (the last factor of the chain rule in
Eq. backward-pass of Sec. 3.3) without hand-deriving it.
"""
from __future__ import annotations

import numpy as np


class Dual:
    __slots__ = ("v", "d")
    __array_ufunc__ = None   # make NumPy defer to Dual's reflected operators

    def __init__(self, v, d):
        self.v = v
        self.d = d

    @staticmethod
    def seed(values: np.ndarray, index: int, n: int) -> "Dual":
        d = np.zeros((values.shape[0], n))
        d[:, index] = 1.0
        return Dual(values.astype(np.float64), d)

    @staticmethod
    def const(values, like: "Dual") -> "Dual":
        v = np.broadcast_to(np.asarray(values, np.float64), like.v.shape).copy()
        return Dual(v, np.zeros_like(like.d))

    # arithmetic -------------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.d + o.d)
        return Dual(self.v + o, self.d)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.d - o.d)
        return Dual(self.v - o, self.d)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.d)

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v * o.v, self.d * o.v[:, None] + o.d * self.v[:, None])
        o = np.asarray(o, np.float64)
        return Dual(self.v * o, self.d * (o[:, None] if o.ndim == 1 else o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Dual):
            q = self.v / o.v
            return Dual(q, (self.d - o.d * q[:, None]) / o.v[:, None])
        o = np.asarray(o, np.float64)
        return Dual(self.v / o, self.d / (o[:, None] if o.ndim == 1 else o))

    def __rtruediv__(self, o):
        q = o / self.v
        return Dual(q, -self.d * (q / self.v)[:, None])


def exp(a: Dual) -> Dual:
    e = np.exp(a.v)
    return Dual(e, a.d * e[:, None])


def sqrt(a: Dual) -> Dual:
    s = np.sqrt(a.v)
    return Dual(s, a.d * (0.5 / s)[:, None])


def sigmoid(a: Dual) -> Dual:
    s = 1.0 / (1.0 + np.exp(-a.v))
    return Dual(s, a.d * (s * (1.0 - s))[:, None])


def relu(a: Dual) -> Dual:
    """max(0, a); the derivative is taken as 0 where a < 0 (the clamped branch)."""
    keep = a.v >= 0.0
    return Dual(np.where(keep, a.v, 0.0), np.where(keep[:, None], a.d, 0.0))


def take(a: Dual, idx) -> Dual:
    return Dual(a.v[idx], a.d[idx])
