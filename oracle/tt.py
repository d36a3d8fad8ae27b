"""FP64 CPU oracle of the 2-bounce refraction (TT) solve (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product path never does.  It shares no code with the
CUDA library.

It follows the paper's steps for a chain x0 -> T1 -> T2 -> x3 of two
refractions (IORs eta_0, eta_1, eta_2), in plain numpy FP64:

1. Rational coordinate mapping (Sec. 3.4, Eq. eq_rct): the scaled refracted
   direction at x1 (Eq. eq_refr_rational), with sqrt(beta) replaced by a
   piecewise rational approximant (Sec. 3.4; the paper's coefficients are
   in its supplement, which is missing, so the pieces are fitted here:
   ``fit_sqrt_pieces``), then the Moller-Trumbore intersection with T2 as
   u2 = (u~, v~) / kappa.
2. Bivariate system in (u1, v1) (Sec. 3.5; Table tab_sum): the endpoint
   coplanarity form and the square form at x2, with x2 - x1 replaced by the
   mapped direction D and the kappa denominators of x2 and n2 cleared
   (total degrees 16 and 46; the table's 18 and 48 are upper bounds).
3. The Bezout matrix in u1 with hidden v1 by the explicit sum of
   Eq. eq_bezout, evaluated at 2^12 + 1 uniform v1 in [0, 1]; its
   determinant's sign from an LU factorisation with partial pivoting
   (numpy slogdet); bisection on every sign change for the paper's 10
   iterations (Sec. 4.2), continued to 1e-12.
4. u1 from a(u1, v1*) = 0 (companion eigenvalues), u2 from the mapping,
   then path-space Newton on the exact constraint h x n = 0 (Eq. eq_ch) at
   both vertices (at most 5 iterations), sidedness and in-triangle tests.

Readings where the paper is silent are listed with each function.
"""
from __future__ import annotations

import numpy as np
from scipy.signal import convolve2d

from . import F_EDGE, F_ILL_COND, F_NEWTON_REFINED, F_SQRT_SPLIT, PATH_DTYPE

DELTA = 1e-6
TRIM = 1e-13
RESIDUAL = 1e-9
EDGE = 1e-7
DEDUPE = 1e-9
N_INTERVALS = 4096
PAPER_ITERS = 10
ROOT_TOL = 1e-12
NEWTON_ITERS = 8
ILL_COND_K2 = 1e-7
# Reading: six pieces on [0, 1] chosen so that a (1,1) rational fit reaches
# the paper's error bound (< 1e-3) on each; pieces of ratio 3 fail it near 0.
SQRT_BREAKS = (0.0, 4e-4, 7e-3, 0.048, 0.2, 0.65, 1.0)


# ------------------------------------------------------------ sqrt pieces
def fit_sqrt_pieces(breaks=SQRT_BREAKS, n_grid=4000):
    """Minimax fit of sqrt(x) by (c0 + c1 x) / (1 + d1 x) on each piece
    (Sec. 3.4 form with d0 = 1): Nelder-Mead on the maximum absolute error
    over a uniform grid of the piece.  Returns an array [6][3] of
    (c0, c1, d1)."""
    from scipy.optimize import minimize
    out = []
    for a, b in zip(breaks[:-1], breaks[1:]):
        x = np.linspace(a, b, n_grid)
        f = np.sqrt(x)

        def err(p):
            return np.max(np.abs((p[0] + p[1] * x) / (1.0 + p[2] * x) - f))

        m = 0.5 * (a + b)
        starts = [[np.sqrt(m) / 3.0, 1.0 / np.sqrt(m), 1.0 / (3.0 * m)], [np.sqrt(a + 1e-12), 1.0, 1.0], [0.1, 3.0, 3.0]]
        best = None
        for s0 in starts:
            r = minimize(err, s0, method="Nelder-Mead", options={"xatol": 1e-13, "fatol": 1e-15, "maxiter": 40000})
            if best is None or r.fun < best.fun:
                best = r
        out.append(best.x)
    return np.array(out)


def sqrt_approx(x, table, breaks=SQRT_BREAKS):
    """Evaluates the piecewise approximant at x in [0, 1]."""
    x = np.asarray(x, float)
    k = np.clip(np.searchsorted(breaks, x, side="right") - 1, 0, len(breaks) - 2)
    c0, c1, d1 = table[k, 0], table[k, 1], table[k, 2]
    return (c0 + c1 * x) / (1.0 + d1 * x)


def piece_of(x, breaks=SQRT_BREAKS):
    return int(np.clip(np.searchsorted(breaks, x, side="right") - 1, 0, len(breaks) - 2))


# ------------------------------------------------- bivariate polynomials
# p(u, v) = sum_ij C[i, j] u^i v^j as a dense 2D array.
def bp_lin(c0, cu, cv):
    c = np.zeros((2, 2))
    c[0, 0], c[1, 0], c[0, 1] = c0, cu, cv
    return c


def bp_add(a, b):
    n = max(a.shape[0], b.shape[0])
    r = np.zeros((n, n))
    r[:a.shape[0], :a.shape[1]] += a
    r[:b.shape[0], :b.shape[1]] += b
    return r


def bp_mul(a, b):
    return convolve2d(a, b)


def bp_scale(a, s):
    return a * s


def vlin(p0, eu, ev):
    """Affine vector polynomial p0 + u eu + v ev."""
    return [bp_lin(p0[k], eu[k], ev[k]) for k in range(3)]


def vconst(x):
    return [np.array([[float(x[k])]]) for k in range(3)]


def vadd(a, b):
    return [bp_add(a[k], b[k]) for k in range(3)]


def vsub(a, b):
    return [bp_add(a[k], -b[k]) for k in range(3)]


def vscale(a, s):
    """Vector times a scalar polynomial (2D array) or a number."""
    if np.isscalar(s):
        return [a[k] * s for k in range(3)]
    return [bp_mul(a[k], s) for k in range(3)]


def vdot(a, b):
    return bp_add(bp_add(bp_mul(a[0], b[0]), bp_mul(a[1], b[1])), bp_mul(a[2], b[2]))


def vcross(a, b):
    return [bp_add(bp_mul(a[1], b[2]), -bp_mul(a[2], b[1])),
            bp_add(bp_mul(a[2], b[0]), -bp_mul(a[0], b[2])),
            bp_add(bp_mul(a[0], b[1]), -bp_mul(a[1], b[0]))]


def bp_eval(c, u, v):
    return np.polynomial.polynomial.polyval2d(u, v, c)


def u_coeffs(c, v):
    """Coefficients in u of p(u, v) at the numbers v: [len(v), deg_u + 1]."""
    v = np.atleast_1d(np.asarray(v, float))
    return np.stack([np.polynomial.polynomial.polyval(v, c[i]) for i in range(c.shape[0])], -1)


def deg_u(c):
    """Highest u-power whose coefficient polynomial is not negligible
    (max-abs above 1e-13 of the polynomial's max-abs)."""
    m = np.max(np.abs(c)) if c.size else 0.0
    if m == 0.0:
        return -1
    rows = np.max(np.abs(c), axis=1)
    nz = np.nonzero(rows > TRIM * m)[0]
    return int(nz[-1]) if nz.size else -1


# ------------------------------------------------------------ the system
def tri_polys(P, N):
    """Position and normal of a triangle as affine polynomials (Sec. 3.1):
    x = p0 + u (p1 - p0) + v (p2 - p0), n likewise."""
    P = np.asarray(P, float)
    N = np.asarray(N, float)
    return vlin(P[0], P[1] - P[0], P[2] - P[0]), vlin(N[0], N[1] - N[0], N[2] - N[0])


def refracted_direction(x0, x1, n1, eta_ratio, piece, table, s):
    """Scaled refracted direction at x1 (Eq. eq_refr_rational) with sqrt(beta)
    replaced by the rational piece, denominators cleared:
    Q eta' (d0 n^2 - (d0.n) n) - sqrt(s) (c0 s + c1 beta) n, with
    Q = s + d1 beta and x = beta / s the approximant's argument."""
    d0 = vsub(x1, vconst(x0))
    n2 = vdot(n1, n1)
    dd = vdot(d0, d0)
    dn = vdot(d0, n1)
    nd = bp_mul(n2, dd)
    beta = bp_add(nd, -(eta_ratio ** 2) * bp_add(nd, -bp_mul(dn, dn)))
    c0, c1, d1 = table[piece]
    Q = bp_add(np.array([[s]]), d1 * beta)
    tang = vsub(vscale(d0, n2), vscale(n1, dn))
    num = bp_add(np.array([[c0 * s]]), c1 * beta)
    return vsub(vscale(vscale(tang, eta_ratio), Q), vscale(vscale(n1, num), np.sqrt(s))), beta


def mapping(D, x1, P2):
    """Moller-Trumbore intersection of the ray x1 + t D with the plane of T2
    as polynomials (Eq. eq_rct): u~, v~, kappa, and the ray parameter's
    numerator t~ (t = t~ / kappa)."""
    P2 = np.asarray(P2, float)
    e1, e2 = P2[1] - P2[0], P2[2] - P2[0]
    s = vsub(x1, vconst(P2[0]))
    de2 = vcross(D, vconst(e2))
    ut = vdot(de2, s)
    se1 = vcross(s, vconst(e1))
    vt = vdot(se1, D)
    kap = vdot(de2, vconst(e1))
    tt = vdot(se1, vconst(e2))
    return ut, vt, kap, tt


def proj_vector(x0, x3, P1, N1, P2, N2):
    """Projection vector b of the square form at x2 (the switch of Sec. 3.3, read as for one bounce, applied to
    the second vertex): the first of (1,0,0), (0,0,1), (0,1,0) whose
    |m_hat . b| >= 0.25, m = (x3 - c1) x n2 at the centroids."""
    c1 = np.asarray(P1).mean(0)
    n2 = np.asarray(N2).mean(0)
    m = np.cross(np.asarray(x3) - c1, n2)
    mn = np.linalg.norm(m)
    m = m / mn if mn > 0 else m
    for b in (np.array([1.0, 0, 0]), np.array([0, 0, 1.0]), np.array([0, 1.0, 0])):
        if abs(m @ b) >= 0.25:
            return b
    return np.array([1.0, 0, 0])


def constant_normal(N):
    """True when the three vertex normals are parallel (relative 1e-12)."""
    u = [np.asarray(n, float) / np.linalg.norm(n) for n in N]
    return max(np.max(np.abs(u[1] - u[0])), np.max(np.abs(u[2] - u[0]))) < 1e-12


def build_tt(x0, x3, etas, P1, N1, P2, N2, piece, table):
    """a (degree 16) and b (degree 46) of the TT system, and the mapping."""
    x0 = np.asarray(x0, float)
    x3 = np.asarray(x3, float)
    P1, N1, P2, N2 = (np.asarray(z, float) for z in (P1, N1, P2, N2))
    x1, n1 = tri_polys(P1, N1)
    # reading: the refraction formula takes the normal on the incident side
    c1 = P1.mean(0)
    if (c1 - x0) @ N1.mean(0) > 0:
        n1 = vscale(n1, -1.0)
    ncen = N1.mean(0)
    s = float((ncen @ ncen) * ((c1 - x0) @ (c1 - x0)))
    D, beta = refracted_direction(x0, x1, n1, etas[0] / etas[1], piece, table, s)
    ut, vt, kap, tt = mapping(D, x1, P2)
    e21, e22 = P2[1] - P2[0], P2[2] - P2[0]
    X2 = vadd(vadd(vscale(vconst(P2[0]), kap), vscale(vconst(e21), ut)), vscale(vconst(e22), vt))
    if constant_normal(N2):
        # Reading: with one normal over T2, kappa n2 = kappa N would make kappa
        # a common factor of a and b and the resultant vanish identically;
        # the constant normal is used as is.
        M2 = vconst(N2[0])
    else:
        M2 = vadd(vadd(vscale(vconst(N2[0]), kap), vscale(vconst(N2[1] - N2[0]), ut)),
                  vscale(vconst(N2[2] - N2[0]), vt))
    # x2 - x1 = (t~ / kappa) D: the segment to x2 is parallel to D.  Writing
    # d1 through kappa (kappa d1 = X2 - kappa x1 = t~ D) would make t~ a
    # common factor of a and b and the resultant vanish identically, so the
    # constraints at x2 are written with D in place of d1 (reading).
    K2 = vsub(vscale(vconst(x3), kap), X2)         # kappa d2
    a = vdot(vcross(D, vsub(vconst(x3), x1)), M2)  # coplanarity (endpoint difference form), degree 16
    bv = proj_vector(x0, x3, P1, N1, P2, N2)
    p1 = vdot(vcross(D, M2), vconst(bv))
    p2 = vdot(vcross(K2, M2), vconst(bv))
    b = bp_add(etas[1] ** 2 * bp_mul(vdot(K2, K2), bp_mul(p1, p1)),
               -(etas[2] ** 2) * bp_mul(vdot(D, D), bp_mul(p2, p2)))  # square form, degree 46
    return {"a": a, "b": b, "ut": ut, "vt": vt, "kap": kap, "tt": tt, "beta": beta, "s": s}


# ------------------------------------------------------------ resultant
def bezout(ac, bc, n):
    """Bezout matrices of Eq. eq_bezout for a batch of coefficient vectors
    ac [S, n+1], bc [S, n+1] (padded with zeros).  The explicit sum
    B_ij = sum_{k=0}^{min(i, n-1-j)} (a_{i-k} b_{j+1+k} - b_{i-k} a_{j+1+k})
    is accumulated term k at a time over all (i, j) it reaches: i = k + i'
    and j with i', j in [0, n-1-k]."""
    S = ac.shape[0]
    B = np.zeros((S, n, n))
    for k in range(n):
        m = n - k
        B[:, k:, :m] += ac[:, :m, None] * bc[:, None, k + 1:n + 1] - bc[:, :m, None] * ac[:, None, k + 1:n + 1]
    return B


def det_sign(sys, v, n, da, db):
    """(sign, log|det|) of the Bezout matrix at the numbers v."""
    v = np.atleast_1d(v)
    ac = np.zeros((v.size, n + 1))
    bc = np.zeros((v.size, n + 1))
    ac[:, :da + 1] = u_coeffs(sys["a"][:da + 1], v)
    bc[:, :db + 1] = u_coeffs(sys["b"][:db + 1], v)
    return np.linalg.slogdet(bezout(ac, bc, n))


# ----------------------------------------------------------- path space
def _unit(x):
    return x / np.linalg.norm(x)


def vertex_residual(xp, x, xn, n, eta_in, eta_out):
    """h x n / (|h| |n|) with h = eta_out d1_hat - eta_in d0_hat (refraction,
    Eq. eq_ch), and the sidedness test (both directions on one side)."""
    d0, d1 = x - xp, xn - x
    h = eta_out * _unit(d1) - eta_in * _unit(d0)
    r = np.cross(h, n) / (np.linalg.norm(h) * np.linalg.norm(n))
    s0, s1 = d0 @ n, d1 @ n
    return r, (s0 < 0) == (s1 < 0) and s0 != 0 and s1 != 0


def _tangent_basis(n):
    n = _unit(n)
    a = np.eye(3)[np.argmin(np.abs(n))]
    t1 = _unit(np.cross(n, a))
    return t1, np.cross(n, t1)


def path_points(w, x0, x3, P1, N1, P2, N2):
    u1, v1, u2, v2 = w
    x1 = P1[0] + u1 * (P1[1] - P1[0]) + v1 * (P1[2] - P1[0])
    n1 = N1[0] + u1 * (N1[1] - N1[0]) + v1 * (N1[2] - N1[0])
    x2 = P2[0] + u2 * (P2[1] - P2[0]) + v2 * (P2[2] - P2[0])
    n2 = N2[0] + u2 * (N2[1] - N2[0]) + v2 * (N2[2] - N2[0])
    return x1, n1, x2, n2


def residuals(w, x0, x3, etas, P1, N1, P2, N2):
    x1, n1, x2, n2 = path_points(w, x0, x3, P1, N1, P2, N2)
    r1, ok1 = vertex_residual(x0, x1, x2, n1, etas[0], etas[1])
    r2, ok2 = vertex_residual(x1, x2, x3, n2, etas[1], etas[2])
    return r1, r2, ok1 and ok2, (x1, x2)


def newton_refine(w, x0, x3, etas, P1, N1, P2, N2, iters=NEWTON_ITERS):
    """Path-space Newton on h_i x n_i = 0 at both vertices: four unknowns,
    two tangential components per vertex in a basis fixed at the start;
    Jacobian by central differences."""
    w = np.array(w, float)
    _, n1, _, n2 = path_points(w, x0, x3, P1, N1, P2, N2)
    B1, B2 = _tangent_basis(n1), _tangent_basis(n2)

    def F(z):
        r1, r2, _, _ = residuals(z, x0, x3, etas, P1, N1, P2, N2)
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
def solve_candidate(x0, x3, etas, P1, N1, P2, N2, table, n_intervals=N_INTERVALS, keep_unrefined=False,
                    v_solver="bisect"):
    """All admissible TT paths of one candidate.  Returns a list of dicts
    (uv (u1, v1, u2, v2), x1, x2, residual, flags, uv_unrefined).
    v_solver="qz" finds the roots v1* by linearisation and QZ (oracle.qz)
    instead of sampling and bisection; the rest is unchanged."""
    x0, x3 = np.asarray(x0, float), np.asarray(x3, float)
    P1, N1, P2, N2 = (np.asarray(z, float) for z in (P1, N1, P2, N2))
    etas = tuple(float(e) for e in etas)
    # pieces of the sqrt approximant spanned by x = beta / s over the triangle
    c1 = P1.mean(0)
    nc = N1.mean(0)
    if (c1 - x0) @ nc > 0:
        nc = -nc
    s = float((nc @ nc) * ((c1 - x0) @ (c1 - x0)))
    er = etas[0] / etas[1]

    def xval(p, n):
        d = p - x0
        nd = (n @ n) * (d @ d)
        return (nd - er ** 2 * (nd - (d @ n) ** 2)) / s

    xs = [xval(c1, N1.mean(0))] + [xval(P1[i], N1[i]) for i in range(3)]
    pieces = sorted({piece_of(min(max(x, 0.0), 1.0)) for x in xs})
    split = len(pieces) > 1
    out = []
    vs = np.linspace(0.0, 1.0, n_intervals + 1)
    for piece in pieces:
        sysd = build_tt(x0, x3, etas, P1, N1, P2, N2, piece, table)
        da, db = deg_u(sysd["a"]), deg_u(sysd["b"])
        n = max(da, db)
        if da < 0 or db < 0 or n < 1:
            continue
        if v_solver == "qz":
            from . import qz
            roots = [(float(v), 0) for v in qz.v_roots(sysd["a"], sysd["b"], da, db)]
        else:
            sg, la = det_sign(sysd, vs, n, da, db)
            # sign changes; a sample with det == 0 exactly is a root belonging to
            # the interval on its left
            roots = [(vs[m], 0) for m in range(1, n_intervals + 1) if sg[m] == 0.0]
            br = [m for m in range(n_intervals) if sg[m] * sg[m + 1] < 0]
            lo = vs[br].copy()
            hi = vs[np.array(br, int) + 1].copy()
            slo = sg[br].copy()
            flag = np.zeros(len(br), int)
            it = 0
            # all brackets bisected together: the paper's 10 iterations, then on
            # to ROOT_TOL
            while len(br) and np.max(hi - lo) > ROOT_TOL:
                mid = 0.5 * (lo + hi)
                sm, _ = det_sign(sysd, mid, n, da, db)
                zero = sm == 0.0  # an exact root: collapse the bracket onto it
                left = (sm == slo) | zero
                lo = np.where(left, mid, lo)
                hi = np.where(left & ~zero, hi, mid)
                it += 1
                if it == PAPER_ITERS:
                    # ill-conditioning (k = 2), normalised locally: |det| across the
                    # bracket against the largest |det| of the five samples
                    # around it (|det| spans hundreds of orders of magnitude over
                    # [0, 1]); a simple root gives about 2^-10 / 2.5
                    _, l_lo = det_sign(sysd, lo, n, da, db)
                    _, l_hi = det_sign(sysd, hi, n, da, db)
                    bi = np.array(br, int)
                    lloc = np.max(np.stack([la[np.clip(bi + o, 0, n_intervals)] for o in (-2, -1, 0, 1, 2, 3)]), 0)
                    rel = np.logaddexp(l_lo - lloc, l_hi - lloc)
                    flag = np.where(rel < np.log(ILL_COND_K2), F_ILL_COND, 0)
            roots += [(0.5 * (a + b), int(f)) for a, b, f in zip(lo, hi, flag)]
        for v1, vflag in roots:
            ac = u_coeffs(sysd["a"][:da + 1], v1)[0]
            bc = u_coeffs(sysd["b"][:db + 1], v1)[0]
            poly = ac if np.max(np.abs(ac)) > 0 else bc
            nz = np.nonzero(np.abs(poly) > TRIM * np.max(np.abs(poly)))[0]
            if nz.size == 0 or nz[-1] == 0:
                continue
            rts = np.roots(poly[:nz[-1] + 1][::-1])
            for r in rts:
                if abs(r.imag) > 1e-6 * max(1.0, abs(r.real)):
                    continue
                u1 = float(r.real)
                if not (-DELTA <= u1 <= 1.0 - v1 + DELTA):
                    continue
                # measured against the magnitude bound of evaluating b
                # at (u1, v1*), sum_ij |b_ij| |u1|^i |v1*|^j (the coefficients of
                # b(., v1*) alone all vanish when b does not depend on u)
                babs = u_coeffs(np.abs(sysd["b"][:db + 1]), abs(v1))[0]
                bs = np.sum(babs * np.maximum(1.0, abs(u1)) ** np.arange(babs.size))
                if abs(np.polynomial.polynomial.polyval(u1, bc)) > 1e-6 * bs:
                    continue
                kap = bp_eval(sysd["kap"], u1, v1)
                if kap == 0.0:
                    continue
                w0 = np.array([u1, v1, bp_eval(sysd["ut"], u1, v1) / kap, bp_eval(sysd["vt"], u1, v1) / kap])
                if split:
                    # keep roots whose approximant argument lies in this piece
                    x1p, n1p, _, _ = path_points(w0, x0, x3, P1, N1, P2, N2)
                    n1o = -n1p if (c1 - x0) @ N1.mean(0) > 0 else n1p
                    if piece_of(min(max(xval(x1p, n1o), 0.0), 1.0)) != piece:
                        continue
                w = newton_refine(w0, x0, x3, etas, P1, N1, P2, N2)
                r1, r2, side_ok, (x1, x2) = residuals(w, x0, x3, etas, P1, N1, P2, N2)
                res = max(np.linalg.norm(r1), np.linalg.norm(r2))
                if not side_ok or not (res < RESIDUAL):
                    continue
                m1 = min(w[0], w[1], 1 - w[0] - w[1])
                m2 = min(w[2], w[3], 1 - w[2] - w[3])
                if m1 < 0 or m2 < 0:
                    continue
                flags = vflag | F_NEWTON_REFINED | (F_SQRT_SPLIT if split else 0)
                if min(m1, m2) < EDGE:
                    flags |= F_EDGE
                dup = False
                for p in out:
                    if np.max(np.abs(p["uv"] - w)) <= DEDUPE:
                        p["flags"] |= flags
                        if np.max(np.abs(w0 - w)) < np.max(np.abs(p["uv_unrefined"] - w)):
                            p["uv_unrefined"] = w0  # the bracket closest to the path
                        dup = True
                if not dup:
                    out.append({"uv": w, "x1": x1, "x2": x2, "residual": res, "flags": flags, "uv_unrefined": w0})
    return out


def solve(tri, x_first, x_last, eta, chains, table, n_intervals=N_INTERVALS, v_solver="bisect"):
    """TT solve of explicit chains (query, tri0, tri1) over a mesh in the
    library's SoA layout.  Returns (PATH_DTYPE array, unrefined (u, v) per
    path [n, 4])."""
    T = np.asarray(tri, float)
    recs, unref = [], []
    for ci, (q, t1, t2) in enumerate(np.asarray(chains)):
        P1 = np.stack([T[0:3, t1], T[3:6, t1], T[6:9, t1]])
        N1 = np.stack([T[9:12, t1], T[12:15, t1], T[15:18, t1]])
        P2 = np.stack([T[0:3, t2], T[3:6, t2], T[6:9, t2]])
        N2 = np.stack([T[9:12, t2], T[12:15, t2], T[15:18, t2]])
        for p in solve_candidate(x_first[q], x_last[q], eta[q], P1, N1, P2, N2, table, n_intervals,
                                 v_solver=v_solver):
            r = np.zeros(1, PATH_DTYPE)
            r["chain"], r["query"], r["tri0"], r["tri1"] = ci, q, t1, t2
            r["uv"][0] = p["uv"]
            r["x"][0, :3], r["x"][0, 3:] = p["x1"], p["x2"]
            r["residual"], r["flags"] = p["residual"], p["flags"]
            recs.append(r)
            unref.append(p["uv_unrefined"])
    if not recs:
        return np.zeros(0, PATH_DTYPE), np.zeros((0, 4))
    return np.concatenate(recs), np.array(unref)
