"""Generates laplace_gen.cuh: straight-line memoised Laplace expansions.

For a symmetric N x N Bezout matrix whose entry (i, j) is a polynomial of
degree <= ED - i - j (zero when negative), the determinant is expanded by
cofactors along each leading row, memoising the minors of the trailing rows
over column subsets (Sec. 4.2 of the paper).  Minors that vanish
structurally (no permutation through nonzero entries) are never formed.
Every coefficient of every minor becomes one scalar, so the emitted code is
straight-line and register-allocatable.

Run: python gen_laplace.py  (rewrites laplace_gen.cuh beside this file).
"""
from __future__ import annotations

import os
from functools import lru_cache

CONFIGS = [("R2", 2, 5), ("R3", 3, 5), ("R4", 4, 5), ("T2", 2, 7), ("T3", 3, 7), ("T4", 4, 7), ("T5", 5, 7),
           ("T6", 6, 7)]


def generate(name: str, N: int, ED: int, absolute: bool = False) -> str:
    """absolute=True emits the same memoised expansion over |E| with every
    term added: a bound on the sum of absolute values of all products that
    make each coefficient of the determinant (its rounding-error scale)."""
    def edeg(i, j):
        return ED - i - j

    @lru_cache(maxsize=None)
    def nonzero(row: int, mask: int) -> bool:
        if row == N:
            return mask == 0
        return any((mask >> j) & 1 and edeg(row, j) >= 0 and nonzero(row + 1, mask & ~(1 << j)) for j in range(N))

    def mdeg(row: int, mask: int) -> int:
        return sum(ED - i for i in range(row, N)) - sum(j for j in range(N) if (mask >> j) & 1)

    offs = {}
    o = 0
    for i in range(N):
        for j in range(i, N):
            offs[(i, j)] = o
            if edeg(i, j) >= 0:
                o += edeg(i, j) + 1
    sym = o
    RD = N * (ED - N + 1)

    def E(i, j, c):
        a, b = min(i, j), max(i, j)
        return f"E[{offs[(a, b)] + c}]"

    fname = f"laplace_abs_{name}" if absolute else f"laplace_{name}"
    what = "sum of |products| of the expansion" if absolute else "determinant"
    lines = [f"// {name}: N = {N}, entry degree <= {ED} - i - j, result degree <= {RD}; {what}.",
             "template <typename T>",
             f"SPOLY_D void {fname}(const T (&E)[{sym}], T (&r)[{RD + 1}]) {{"]
    row = N - 1
    for j in range(N):
        mask = 1 << j
        if not nonzero(row, mask):
            continue
        for c in range(mdeg(row, mask) + 1):
            lines.append(f"  const T m{mask}_{c} = {E(row, j, c)};")
    for row in range(N - 2, -1, -1):
        for mask in range(1, 1 << N):
            if bin(mask).count("1") != N - row or not nonzero(row, mask):
                continue
            terms = {}
            pos = 0
            for j in range(N):
                if not (mask >> j) & 1:
                    continue
                sub = mask & ~(1 << j)
                de, ds = edeg(row, j), mdeg(row + 1, sub)
                if de >= 0 and ds >= 0 and nonzero(row + 1, sub):
                    neg = (pos & 1) and not absolute
                    for x in range(de + 1):
                        for y in range(ds + 1):
                            terms.setdefault(x + y, []).append((neg, E(row, j, x), f"m{sub}_{y}"))
                pos += 1
            dm = mdeg(row, mask)
            for c in range(dm + 1):
                tl = terms.get(c, [])
                var = f"m{mask}_{c}"
                if not tl:
                    lines.append(f"  const T {var} = T(0);")
                    continue
                neg, e, m = tl[0]
                lines.append(f"  T {var} = {'-' if neg else ''}{e} * {m};")
                for neg, e, m in tl[1:]:
                    lines.append(f"  {var} = fma({'-' if neg else ''}{e}, {m}, {var});")
    full = (1 << N) - 1
    for c in range(RD + 1):
        lines.append(f"  r[{c}] = m{full}_{c};" if c <= mdeg(0, full) else f"  r[{c}] = T(0);")
    lines.append("}")
    return "\n".join(lines)


def main():
    out = ["// Generated by gen_laplace.py: straight-line memoised Laplace expansions of",
           "// the symmetric Bezout matrix (Sec. 4.2), and the same expansions over |E|",
           "// with every term added (the rounding-error scale of each coefficient).",
           "// Do not edit by hand.",
           "#pragma once",
           '#include "common.cuh"',
           "",
           "namespace spoly {",
           ""]
    for name, N, ED in CONFIGS:
        out.append(generate(name, N, ED))
        out.append("")
        out.append(generate(name, N, ED, absolute=True))
        out.append("")
    out.append("}  // namespace spoly")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "laplace_gen.cuh")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    return path


if __name__ == "__main__":
    print(main())
