"""Generates sqrt_table.cuh: the library's default piecewise rational
approximant of sqrt(x) on [0, 1] used by the refraction mapping of 2-bounce
chains (Sec. 3.4: six pieces of (c0 + c1 x) / (d0 + d1 x), error below
1e-3; the paper's own coefficients are in its supplement, which is not
available).  Each piece is the minimax fit over Chebyshev nodes of the
piece, by bisection on the error level with a linear feasibility program
(the differential-correction formulation of rational minimax fitting).
Breakpoints: chosen so that six pieces meet the bound (ratio-3 pieces fail
it near 0).

Run: python gen_sqrt_table.py > sqrt_table.cuh
"""
import numpy as np

BREAKS = (0.0, 4e-4, 7e-3, 0.048, 0.2, 0.65, 1.0)


def fit_piece(a, b, n=800):
    """Minimax (c0, c1, d1) on Chebyshev nodes of [a, b] by bisection on the
    error level h: for a fixed h the conditions
    |c0 + c1 x - sqrt(x) (1 + d1 x)| <= h (1 + d1 x), 1 + d1 x >= 1e-9,
    are linear in the unknowns, and a linear program decides feasibility."""
    from scipy.optimize import linprog
    k = np.arange(n)
    x = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / n)
    x = np.concatenate([x, [a, b]])
    f = np.sqrt(x)

    def feasible(h):
        # unknowns z = (c0, c1, d1)
        # c0 + c1 x - f - f d1 x - h - h d1 x <= 0
        A1 = np.stack([np.ones_like(x), x, -(f + h) * x], 1)
        b1 = f + h
        # -(c0 + c1 x - f - f d1 x) - h - h d1 x <= 0
        A2 = np.stack([-np.ones_like(x), -x, (f - h) * x], 1)
        b2 = h - f
        A3 = np.stack([np.zeros_like(x), np.zeros_like(x), -x], 1)
        b3 = np.full_like(x, 1.0 - 1e-9)
        r = linprog(np.zeros(3), A_ub=np.vstack([A1, A2, A3]), b_ub=np.concatenate([b1, b2, b3]),
                    bounds=[(None, None)] * 3, method="highs")
        return r.x if r.status == 0 else None

    lo, hi = 0.0, 0.05
    best = feasible(hi)
    assert best is not None
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        z = feasible(mid)
        if z is not None:
            hi, best = mid, z
        else:
            lo = mid
    err = np.max(np.abs((best[0] + best[1] * x) / (1 + best[2] * x) - f))
    return best, err


def main():
    rows, errs = [], []
    for a, b in zip(BREAKS[:-1], BREAKS[1:]):
        p, e = fit_piece(a, b)
        rows.append(p)
        errs.append(e)
    xs = np.linspace(0, 1, 2_000_001)
    k = np.clip(np.searchsorted(BREAKS, xs, side="right") - 1, 0, 5)
    P = np.array(rows)
    approx = (P[k, 0] + P[k, 1] * xs) / (1 + P[k, 2] * xs)
    total = np.max(np.abs(approx - np.sqrt(xs)))
    assert total < 1e-3, total
    print("// Generated by gen_sqrt_table.py; do not edit.")
    print(f"// Default six-piece rational approximant of sqrt on [0, 1]; max |error| = {total:.3e}.")
    print("#pragma once")
    print('#include "tt.cuh"')
    print("namespace spoly {")
    print("inline SqrtTable default_sqrt_table() {")
    print("  SqrtTable t;")
    for i, x in enumerate(BREAKS):
        print(f"  t.breaks[{i}] = {x!r};")
    for i, p in enumerate(rows):
        print(f"  t.c[{i}][0] = {float(p[0])!r};")
        print(f"  t.c[{i}][1] = {float(p[1])!r};")
        print(f"  t.c[{i}][2] = {float(p[2])!r};")
    print("  return t;")
    print("}")
    print("}  // namespace spoly")


if __name__ == "__main__":
    main()
