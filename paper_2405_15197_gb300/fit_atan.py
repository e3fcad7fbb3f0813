"""Coefficients of the library's FP32 arctangent (lm_atan2 in csrc/lm_geom.cuh).

atan(r) is approximated on r in [0, 1] by r P(r^2) with P a polynomial of
degree 7 in t = r^2 (8 coefficients).  The fit minimises the largest
absolute error over a dense grid by Lawson's algorithm (iteratively
reweighted least squares converging to the minimax weights), in FP64; the
coefficients are then rounded to FP32.  lm_atan2 evaluates P by Horner's
rule with fused multiply-adds and maps other octants with
atan(y/x) = pi/2 - atan(x/y) and the sign rules of atan2.

  python -m paper_2405_15197_gb300.fit_atan     # prints the coefficients and
                                                # the FP32 evaluation error
"""
from __future__ import annotations

import numpy as np

DEGREE = 7
GRID = 20001
ITERS = 200


def fit():
    """FP64 minimax coefficients c[0..7] of P (P(t) = sum c_i t^i)."""
    r = np.linspace(0.0, 1.0, GRID)
    t = r * r
    V = r[:, None] * t[:, None] ** np.arange(DEGREE + 1)[None, :]
    f = np.arctan(r)
    w = np.full(GRID, 1.0 / GRID)
    c = None
    for _ in range(ITERS):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], f * sw, rcond=None)
        e = np.abs(V @ c - f)
        w = w * e
        s = w.sum()
        if s == 0.0:
            break
        w /= s
    return c


def coefficients_f32():
    return fit().astype(np.float32)


def _fma32(a, b, c):
    """FP32 fused multiply-add, emulated: the FP64 product of two FP32 values
    is exact, the sum is rounded once more to FP32."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def eval_f32(r, c32):
    """r P(r^2) evaluated as lm_atan2 does (FP32 Horner with FMAs)."""
    r = r.astype(np.float32)
    t = (r * r).astype(np.float32)
    p = np.full_like(r, c32[DEGREE])
    for i in range(DEGREE - 1, -1, -1):
        p = _fma32(p, t, np.full_like(r, c32[i]))
    return (r * p).astype(np.float32)


def max_error_f32(c32, n=2_000_001):
    r = np.linspace(0.0, 1.0, n).astype(np.float32)
    return float(np.abs(eval_f32(r, c32).astype(np.float64) - np.arctan(r.astype(np.float64))).max())


if __name__ == "__main__":
    c64 = fit()
    c32 = c64.astype(np.float32)
    r = np.linspace(0.0, 1.0, 200001)
    V = r[:, None] * (r * r)[:, None] ** np.arange(DEGREE + 1)[None, :]
    print("minimax error (FP64 coefficients):", np.abs(V @ c64 - np.arctan(r)).max())
    print("FP32 evaluation error:", max_error_f32(c32))
    for i in range(DEGREE, -1, -1):
        print(f"c[{i}] = {float(c32[i])!r}f")
