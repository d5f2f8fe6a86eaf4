"""Generate tll_poly.cuh: polynomial coefficients for the kernel's atan and
atanh on reduced ranges.

Method: odd functions written as f(w) = w * P(w^2); P is fitted by the Remez
exchange algorithm for minimax RELATIVE error of f on the interval, starting
from Chebyshev nodes (E. Remez 1934; e.g. J.-M. Muller, "Elementary
Functions", ch. 3).  Coefficients are computed here in float64 and rounded to
float32.  Run:  python gen_poly.py > tll_poly.cuh
"""
import math

import numpy as np


def remez_odd(f, a, b, deg, iters=40):
    """Minimax relative error of f(w) ~ w P(w^2) on w in [a, b] (a >= 0),
    P of degree deg in s = w^2.  Returns the coefficients of P (low first)
    and the max relative error (float64 evaluation)."""
    n = deg + 2                       # alternation points
    s_lo, s_hi = a * a, b * b
    k = np.arange(n)
    s = 0.5 * (s_lo + s_hi) - 0.5 * (s_hi - s_lo) * np.cos(np.pi * k / (n - 1))
    grid = np.linspace(s_lo, s_hi, 200001)
    target = lambda ss: f(np.sqrt(ss)) / np.sqrt(ss)   # P(s) ~ f(w)/w
    for _ in range(iters):
        # solve P(s_i) + (-1)^i E g(s_i) = target(s_i), g = |target| (relative)
        t = target(s)
        A = np.zeros((n, n))
        for j in range(deg + 1):
            A[:, j] = s ** j
        A[:, deg + 1] = (-1.0) ** k * np.abs(t)
        sol = np.linalg.solve(A, t)
        c = sol[:deg + 1]
        err = (np.polyval(c[::-1], grid) - target(grid)) / np.abs(target(grid))
        # new extrema: one per sign run
        idx = []
        start = 0
        sg = np.sign(err)
        for i in range(1, len(grid) + 1):
            if i == len(grid) or sg[i] != sg[start]:
                seg = np.arange(start, i)
                idx.append(seg[np.argmax(np.abs(err[seg]))])
                start = i
        if len(idx) < n:
            break
        # keep the n largest alternating extrema
        while len(idx) > n:
            e = np.abs(err[idx])
            if e[0] < e[-1]:
                idx.pop(0)
            else:
                idx.pop()
        s = grid[idx]
    err = (np.polyval(c[::-1], grid) - target(grid)) / np.abs(target(grid))
    return c, float(np.abs(err).max())


def f32_eval_err(f, c, a, b):
    """Max relative error of the kernel's evaluation order with float32
    coefficients: P = 1 + s Q(s), f(w) ~ w + (w s) Q(s), Horner for Q with
    each step rounded to float32 (as FMA does), the last step one FMA."""
    c32 = np.asarray(c, dtype=np.float32)
    w = np.linspace(max(a, 1e-6), b, 400001).astype(np.float32)
    s = (w * w).astype(np.float32)
    q = np.full_like(s, c32[-1])
    for cc in c32[-2:0:-1]:
        q = (q.astype(np.float64) * s + cc).astype(np.float32)
    ws = (w * s).astype(np.float32)
    r = (ws.astype(np.float64) * q + w).astype(np.float32)
    ref = f(w.astype(np.float64))
    return float(np.max(np.abs(r - ref) / np.abs(ref)))


def main():
    out = ["// tll_poly.cuh -- generated by gen_poly.py (Remez, relative error).",
           "// f(w) = w + (w^3) Q(w^2) with P = 1 + s Q(s); Q's coefficients,",
           "// low order first (P's constant term is exactly 1).",
           "#pragma once", ""]
    specs = [("ATAN", np.arctan, 0.0, 1.0, 9),
             ("ATANH", np.arctanh, 0.0, 0.5, 6)]
    for name, f, a, b, deg in specs:
        c, e64 = remez_odd(f, max(a, 1e-4), b, deg)
        c = np.asarray(c, dtype=np.float64)
        c[0] = 1.0
        e32 = f32_eval_err(f, c, a, b)
        out.append(f"// {name.lower()} on [{a}, {b}], degree {deg} in w^2: "
                   f"max rel err {e64:.2e} (float64), {e32:.2e} (float32 Horner)")
        body = ", ".join(f"{float(np.float32(x)):.9e}f" for x in c[1:])
        out.append(f"#define TLL_{name}_NC {deg}")
        out.append(f"#define TLL_{name}_COEFS {{{body}}}")
        out.append("")
    print("\n".join(out))


if __name__ == "__main__":
    main()
