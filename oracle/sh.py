"""Real spherical harmonics up to degree 3 (the view-dependent colour of Sec. 3.1).

The paper models colour with "Spherical Harmonics coefficients of order 3"
(Sec. 3.1) and counts 48 SH coefficients per Gaussian (Sec. A). It does not
print the basis. This oracle uses the real orthonormal basis with the
Condon-Shortley phase: for degree l and order m,

    Y_lm = (-1)^m * N_lm * P_lm(x, y, z),

with P_lm the standard harmonic polynomial of the direction (x, y, z) and N_lm
its normalisation constant, built here from closed forms. Coefficient index k
runs l-major: k = l^2 + l + m.

Pinned in tests against scipy's complex spherical harmonics and against
orthonormality on the sphere.
"""
from __future__ import annotations

import math

# (l, m) of every coefficient index k.
LM = [(l, m) for l in range(4) for m in range(-l, l + 1)]


def _norm(l: int, m: int) -> float:
    """N_lm for the polynomial forms used in ``basis`` (closed forms)."""
    pi = math.pi
    table = {
        (0, 0): 0.5 * math.sqrt(1.0 / pi),
        (1, -1): math.sqrt(3.0 / (4 * pi)), (1, 0): math.sqrt(3.0 / (4 * pi)), (1, 1): math.sqrt(3.0 / (4 * pi)),
        (2, -2): 0.5 * math.sqrt(15.0 / pi), (2, -1): 0.5 * math.sqrt(15.0 / pi),
        (2, 0): 0.25 * math.sqrt(5.0 / pi),
        (2, 1): 0.5 * math.sqrt(15.0 / pi), (2, 2): 0.25 * math.sqrt(15.0 / pi),
        (3, -3): 0.25 * math.sqrt(35.0 / (2 * pi)), (3, -2): 0.5 * math.sqrt(105.0 / pi),
        (3, -1): 0.25 * math.sqrt(21.0 / (2 * pi)), (3, 0): 0.25 * math.sqrt(7.0 / pi),
        (3, 1): 0.25 * math.sqrt(21.0 / (2 * pi)), (3, 2): 0.25 * math.sqrt(105.0 / pi),
        (3, 3): 0.25 * math.sqrt(35.0 / (2 * pi)),
    }
    return table[(l, m)]


def _poly(l: int, m: int, x, y, z):
    """Harmonic polynomial P_lm; valid for unit (x, y, z). Works on floats, arrays and Duals."""
    if l == 0:
        return x * 0.0 + 1.0
    if l == 1:
        return {-1: y, 0: z, 1: x}[m]
    if l == 2:
        if m == -2:
            return x * y
        if m == -1:
            return y * z
        if m == 0:
            return 2.0 * (z * z) - x * x - y * y
        if m == 1:
            return x * z
        return x * x - y * y
    # l == 3
    if m == -3:
        return y * (3.0 * (x * x) - y * y)
    if m == -2:
        return x * y * z
    if m == -1:
        return y * (4.0 * (z * z) - x * x - y * y)
    if m == 0:
        return z * (2.0 * (z * z) - 3.0 * (x * x) - 3.0 * (y * y))
    if m == 1:
        return x * (4.0 * (z * z) - x * x - y * y)
    if m == 2:
        return z * (x * x - y * y)
    return x * (x * x - 3.0 * (y * y))


def basis(x, y, z):
    """List of the 16 basis values Y_k at unit directions (x, y, z)."""
    out = []
    for (l, m) in LM:
        s = -1.0 if (m % 2) else 1.0
        out.append(_poly(l, m, x, y, z) * (s * _norm(l, m)))
    return out
