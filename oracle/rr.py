"""FP64 CPU oracle of the 2-bounce reflection (RR) solve (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product path never does.  It shares no code with the
CUDA library.  The bivariate-polynomial helpers, the rational coordinate
mapping and the Bezout determinant are the ones of the TT oracle
(``oracle/tt.py``).

It follows the paper's steps for a chain x0 -> T1 -> T2 -> x3 of two
reflections, in plain numpy FP64:

1. Rational coordinate mapping (Sec. 3.4, Eq. eq_rct) with the scaled
   reflected direction of Eq. eq_431_di,
   D = -2 (d0 . n1) n1 + d0 |n1|^2, d0 = x1 - x0: a polynomial of degree 3
   in (u1, v1), exact (no square root), so a chain is one system.
2. Bivariate system in (u1, v1) (Sec. 3.5, Eq. eq_rr1): the endpoint
   coplanarity form at x2 and the product form (Eq. eq_pf_result) at x2,
   with d1 = x2 - x1 replaced by D and the kappa denominators of x2, n2 and
   t2 cleared (total degrees 9 and 15; Table tab_sum's 10 and 16 are upper
   bounds).
3. The Bezout matrix in u1 with hidden v1 (Eq. eq_bezout) at 2^12 + 1
   uniform v1 in [0, 1], the sign of its determinant, bisection of every
   sign change for the paper's 10 iterations (Sec. 4.2), continued to 1e-12.
4. u1 from a(u1, v1*) = 0, u2 from the mapping, path-space Newton on the
   exact constraint h x n = 0 (Eq. eq_ch, reflection: h = d1_hat - d0_hat)
   at both vertices, the reflection sidedness test (both neighbours on one
   side of the surface) and the in-triangle tests.
"""
from __future__ import annotations

import numpy as np

from . import F_EDGE, F_ILL_COND, F_NEWTON_REFINED, PATH_DTYPE
from . import tt
from .tt import (DEDUPE, DELTA, EDGE, ILL_COND_K2, N_INTERVALS, NEWTON_ITERS, PAPER_ITERS, RESIDUAL, ROOT_TOL,
                 TRIM)

SWITCH = 0.25


def reflected_direction(x0, x1, n1):
    """Eq. eq_431_di: the reflected direction at x1 scaled by |n1|^2 |d0|,
    -2 (d0 . n1) n1 + d0 |n1|^2 with d0 = x1 - x0 (polynomials)."""
    d0 = tt.vsub(x1, tt.vconst(x0))
    return tt.vsub(tt.vscale(d0, tt.vdot(n1, n1)), tt.vscale(n1, 2.0 * tt.vdot(d0, n1)))


def tangent_edge(x3, P1, P2, N2):
    """Edge of T2 in the tangent t2 = n2 x e of the product form at x2.
    Reading of the switch "if the equation degenerates" (Sec. 3.3), as for
    one bounce: with m = (x3 - c1) x n2c (c1 the centroid of T1, n2c the
    centroid normal of T2) the normal of the plane of incidence at x2, e21
    unless |m^ . e21^| < 0.25 and |m^ . e22^| > |m^ . e21^|, then e22."""
    m = np.cross(np.asarray(x3) - np.asarray(P1).mean(0), np.asarray(N2).mean(0))
    mn = np.linalg.norm(m)
    e1, e2 = P2[1] - P2[0], P2[2] - P2[0]
    if not mn > 0.0:
        return e1
    c1 = abs(m @ e1) / (mn * np.linalg.norm(e1))
    c2 = abs(m @ e2) / (mn * np.linalg.norm(e2))
    return e2 if (c1 < SWITCH and c2 > c1) else e1


def build_rr(x0, x3, P1, N1, P2, N2):
    """a (degree 9) and b (degree 15) of the RR system, and the mapping."""
    x0 = np.asarray(x0, float)
    x3 = np.asarray(x3, float)
    P1, N1, P2, N2 = (np.asarray(z, float) for z in (P1, N1, P2, N2))
    x1, n1 = tt.tri_polys(P1, N1)
    D = reflected_direction(x0, x1, n1)
    ut, vt, kap, tpar = tt.mapping(D, x1, P2)
    e21, e22 = P2[1] - P2[0], P2[2] - P2[0]
    X2 = tt.vadd(tt.vadd(tt.vscale(tt.vconst(P2[0]), kap), tt.vscale(tt.vconst(e21), ut)),
                 tt.vscale(tt.vconst(e22), vt))
    if tt.constant_normal(N2):
        # one normal over T2: used as is (a kappa factor common to a and b
        # would make the resultant vanish identically)
        M2 = tt.vconst(N2[0])
    else:
        M2 = tt.vadd(tt.vadd(tt.vscale(tt.vconst(N2[0]), kap), tt.vscale(tt.vconst(N2[1] - N2[0]), ut)),
                     tt.vscale(tt.vconst(N2[2] - N2[0]), vt))
    K2 = tt.vsub(tt.vscale(tt.vconst(x3), kap), X2)             # kappa d2
    a = tt.vdot(tt.vcross(D, tt.vsub(tt.vconst(x3), x1)), M2)   # coplanarity, endpoint difference form
    T2 = tt.vcross(M2, tt.vconst(tangent_edge(x3, P1, P2, N2)))
    b = tt.bp_add(tt.bp_mul(tt.vdot(D, M2), tt.vdot(K2, T2)),
                  tt.bp_mul(tt.vdot(D, T2), tt.vdot(K2, M2)))   # product form, Eq. eq_rr1
    return {"a": a, "b": b, "ut": ut, "vt": vt, "kap": kap, "tt": tpar}


# ----------------------------------------------------------- path space
def vertex_residual(xp, x, xn, n):
    """h x n / (|h| |n|) with h = d1_hat - d0_hat (Eq. eq_ch, reflection),
    and the reflection sidedness test: d0 . n and d1 . n of opposite signs
    (both neighbours on the same side)."""
    d0, d1 = x - xp, xn - x
    h = d1 / np.linalg.norm(d1) - d0 / np.linalg.norm(d0)
    r = np.cross(h, n) / (np.linalg.norm(h) * np.linalg.norm(n))
    s0, s1 = d0 @ n, d1 @ n
    return r, (s0 < 0) != (s1 < 0) and s0 != 0 and s1 != 0


def residuals(w, x0, x3, P1, N1, P2, N2):
    x1, n1, x2, n2 = tt.path_points(w, x0, x3, P1, N1, P2, N2)
    r1, ok1 = vertex_residual(x0, x1, x2, n1)
    r2, ok2 = vertex_residual(x1, x2, x3, n2)
    return r1, r2, ok1 and ok2, (x1, x2)


def newton_refine(w, x0, x3, P1, N1, P2, N2, iters=NEWTON_ITERS):
    """Path-space Newton on h_i x n_i = 0 at both vertices: four unknowns,
    two tangential components per vertex in a basis fixed at the start;
    Jacobian by central differences (as in the TT oracle)."""
    w = np.array(w, float)
    _, n1, _, n2 = tt.path_points(w, x0, x3, P1, N1, P2, N2)
    B1, B2 = tt._tangent_basis(n1), tt._tangent_basis(n2)

    def F(z):
        r1, r2, _, _ = residuals(z, x0, x3, P1, N1, P2, N2)
        return np.array([r1 @ B1[0], r1 @ B1[1], r2 @ B2[0], r2 @ B2[1]])

    for _ in range(iters):
        f = F(w)
        if np.max(np.abs(f)) < 1e-15:
            break
        J = np.empty((4, 4))
        h = 1e-7
        for k in range(4):
            e = np.zeros(4)
            e[k] = h
            J[:, k] = (F(w + e) - F(w - e)) / (2 * h)
        try:
            w = w - np.linalg.solve(J, f)
        except np.linalg.LinAlgError:
            break
    return w


# ---------------------------------------------------------------- solve
def v_roots(sysd, n_intervals=N_INTERVALS):
    """Roots v1* of the resultant in [0, 1] (Sec. 4.2, k = 2): signs of the
    Bezout determinant at n_intervals + 1 uniform samples, every sign change
    bisected (all together) for the paper's 10 iterations and on to 1e-12.
    A sample with det == 0 exactly is a root.  Returns [(v1*, flag)]."""
    da, db = tt.deg_u(sysd["a"]), tt.deg_u(sysd["b"])
    n = max(da, db)
    if da < 0 or db < 0 or n < 1:
        return [], da, db
    vs = np.linspace(0.0, 1.0, n_intervals + 1)
    sg, la = tt.det_sign(sysd, vs, n, da, db)
    roots = [(vs[m], 0) for m in range(1, n_intervals + 1) if sg[m] == 0.0]
    br = [m for m in range(n_intervals) if sg[m] * sg[m + 1] < 0]
    lo = vs[br].copy()
    hi = vs[np.array(br, int) + 1].copy()
    slo = sg[br].copy()
    flag = np.zeros(len(br), int)
    it = 0
    while len(br) and np.max(hi - lo) > ROOT_TOL:
        mid = 0.5 * (lo + hi)
        sm, _ = tt.det_sign(sysd, mid, n, da, db)
        zero = sm == 0.0
        left = (sm == slo) | zero
        lo = np.where(left, mid, lo)
        hi = np.where(left & ~zero, hi, mid)
        it += 1
        if it == PAPER_ITERS:
            # ill-conditioning after the paper's iterations, normalised
            # locally (as in the TT oracle)
            _, l_lo = tt.det_sign(sysd, lo, n, da, db)
            _, l_hi = tt.det_sign(sysd, hi, n, da, db)
            bi = np.array(br, int)
            lloc = np.max(np.stack([la[np.clip(bi + o, 0, n_intervals)] for o in (-2, -1, 0, 1, 2, 3)]), 0)
            rel = np.logaddexp(l_lo - lloc, l_hi - lloc)
            flag = np.where(rel < np.log(ILL_COND_K2), F_ILL_COND, 0)
    roots += [(0.5 * (a + b), int(f)) for a, b, f in zip(lo, hi, flag)]
    return roots, da, db


def solve_candidate(x0, x3, P1, N1, P2, N2, n_intervals=N_INTERVALS, v_solver="bisect"):
    """All admissible RR paths of one candidate: a list of dicts (uv (u1, v1,
    u2, v2), x1, x2, residual, flags, uv_unrefined).  v_solver="qz" finds the
    roots v1* by linearisation and QZ (oracle.qz) instead of sampling and
    bisection; the rest is unchanged."""
    x0, x3 = np.asarray(x0, float), np.asarray(x3, float)
    P1, N1, P2, N2 = (np.asarray(z, float) for z in (P1, N1, P2, N2))
    sysd = build_rr(x0, x3, P1, N1, P2, N2)
    if v_solver == "qz":
        from . import qz
        da, db = tt.deg_u(sysd["a"]), tt.deg_u(sysd["b"])
        roots = [] if da < 0 or db < 0 or max(da, db) < 1 else \
            [(float(v), 0) for v in qz.v_roots(sysd["a"], sysd["b"], da, db)]
    else:
        roots, da, db = v_roots(sysd, n_intervals)
    out = []
    for v1, vflag in roots:
        ac = tt.u_coeffs(sysd["a"][:da + 1], v1)[0]
        bc = tt.u_coeffs(sysd["b"][:db + 1], v1)[0]
        poly = ac if np.max(np.abs(ac)) > 0 else bc
        nz = np.nonzero(np.abs(poly) > TRIM * np.max(np.abs(poly)))[0]
        if nz.size == 0 or nz[-1] == 0:
            continue
        for r in np.roots(poly[:nz[-1] + 1][::-1]):
            if abs(r.imag) > 1e-6 * max(1.0, abs(r.real)):
                continue
            u1 = float(r.real)
            if not (-DELTA <= u1 <= 1.0 - v1 + DELTA):
                continue
            # b(u1, v1*) must vanish with a
            # measured against the magnitude bound of evaluating b
            # at (u1, v1*), sum_ij |b_ij| |u1|^i |v1*|^j (the coefficients of
            # b(., v1*) alone all vanish when b does not depend on u)
            babs = tt.u_coeffs(np.abs(sysd["b"][:db + 1]), abs(v1))[0]
            bs = np.sum(babs * np.maximum(1.0, abs(u1)) ** np.arange(babs.size))
            if abs(np.polynomial.polynomial.polyval(u1, bc)) > 1e-6 * bs:
                continue
            kap = tt.bp_eval(sysd["kap"], u1, v1)
            if kap == 0.0:
                continue
            w0 = np.array([u1, v1, tt.bp_eval(sysd["ut"], u1, v1) / kap, tt.bp_eval(sysd["vt"], u1, v1) / kap])
            w = newton_refine(w0, x0, x3, P1, N1, P2, N2)
            r1, r2, side_ok, (x1, x2) = residuals(w, x0, x3, P1, N1, P2, N2)
            res = max(np.linalg.norm(r1), np.linalg.norm(r2))
            if not side_ok or not (res < RESIDUAL):
                continue
            m1 = min(w[0], w[1], 1 - w[0] - w[1])
            m2 = min(w[2], w[3], 1 - w[2] - w[3])
            if m1 < 0 or m2 < 0:
                continue
            flags = vflag | F_NEWTON_REFINED
            if min(m1, m2) < EDGE:
                flags |= F_EDGE
            dup = False
            for p in out:
                if np.max(np.abs(p["uv"] - w)) <= DEDUPE:
                    p["flags"] |= flags
                    dup = True
            if not dup:
                out.append({"uv": w, "x1": x1, "x2": x2, "residual": res, "flags": flags, "uv_unrefined": w0})
    return out


def solve(tri, x_first, x_last, chains, n_intervals=N_INTERVALS, v_solver="bisect"):
    """RR solve of explicit chains (query, tri0, tri1) over a mesh in the
    library's SoA layout.  Returns a PATH_DTYPE array."""
    T = np.asarray(tri, float)
    recs = []
    for ci, (q, t1, t2) in enumerate(np.asarray(chains)):
        P1 = np.stack([T[0:3, t1], T[3:6, t1], T[6:9, t1]])
        N1 = np.stack([T[9:12, t1], T[12:15, t1], T[15:18, t1]])
        P2 = np.stack([T[0:3, t2], T[3:6, t2], T[6:9, t2]])
        N2 = np.stack([T[9:12, t2], T[12:15, t2], T[15:18, t2]])
        for p in solve_candidate(x_first[q], x_last[q], P1, N1, P2, N2, n_intervals, v_solver=v_solver):
            r = np.zeros(1, PATH_DTYPE)
            r["chain"], r["query"], r["tri0"], r["tri1"] = ci, q, t1, t2
            r["uv"][0] = p["uv"]
            r["x"][0, :3], r["x"][0, 3:] = p["x1"], p["x2"]
            r["residual"], r["flags"] = p["residual"], p["flags"]
            recs.append(r)
    if not recs:
        return np.zeros(0, PATH_DTYPE)
    return np.concatenate(recs)
