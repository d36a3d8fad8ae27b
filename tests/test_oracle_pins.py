"""Pins of the FP64 oracle against facts outside the oracle itself.

* Eq. eq_bezout + Sec. 4.2 Laplace: det of the Bezout matrix equals the
  Sylvester resultant (sympy) up to sign and the leading-coefficient power.
* Sec. 4.2 root isolation: exact Sturm counts (sympy) and planted roots.
* Table tab_sum / tab_equ: polynomial degrees for curved and face-normal input.
* Closed forms: a flat triangle with a constant normal has exactly the
  mirror-image point (R) or the unique Fermat/Snell point (T).
* Brute force: dense (u, v) search + Gauss-Newton on Eq. eq_ch itself, with
  no polynomial anywhere, finds the same solution set on curved triangles.
* Invariants: residual and in-triangle of every path, reciprocity, rigid
  motion, and the Bezout root-count bound.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2405_13409_gb300 import scenes

sympy = pytest.importorskip("sympy")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DEG = json.load(open(os.path.join(GOLDEN, "degrees.json")))


# ----------------------------------------------------------------- helpers
def _solve_single(tri18, x0, x2, type_, eta0=1.0, eta1=1.0):
    tri = np.asarray(tri18, dtype=np.float64).reshape(18, 1)
    x0 = np.asarray(x0, dtype=np.float64).reshape(1, 3)
    x2 = np.asarray(x2, dtype=np.float64).reshape(1, 3)
    eta = np.array([[eta0, eta1, 1.0]])
    types = np.array([[type_, type_]], dtype=np.int32)
    k = np.array([1], dtype=np.int32)
    chains = np.array([[0, 0, -1]], dtype=np.int32)
    paths, cnt = oracle.solve(tri, x0, x2, eta, types, k, chains, n_threads=1)
    return paths, cnt


def _batch(tri, x0, x2, type_, eta0=1.0, eta1=1.0):
    n = tri.shape[1]
    eta = np.tile([eta0, eta1, 1.0], (n, 1))
    types = np.full((n, 2), type_, dtype=np.int32)
    k = np.ones(n, dtype=np.int32)
    chains = np.stack([np.arange(n), np.arange(n), -np.ones(n)], axis=-1).astype(np.int32)
    return oracle.solve(tri, x0, x2, eta, types, k, chains)


def _tri_arrays(tri18):
    t = np.asarray(tri18).reshape(18)
    P = t[:9].reshape(3, 3)
    N = t[9:].reshape(3, 3)
    return P, N


def _bary(P, x):
    e1, e2 = P[1] - P[0], P[2] - P[0]
    A = np.stack([e1, e2], axis=1)
    uv, *_ = np.linalg.lstsq(A, x - P[0], rcond=None)
    return uv


# ------------------------------------------------ Bezout resultant (Eq. eq_bezout)
def _random_bipoly(rng, deg, lo=-4, hi=4):
    g = np.zeros((deg + 1, deg + 1))
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            g[i, j] = rng.integers(lo, hi + 1)
    if g[deg, 0] == 0:
        g[deg, 0] = 1 + rng.integers(0, 3)  # keep deg_u exact
    return g


def _grid_to_sympy(g, u, v):
    return sum(int(g[i, j]) * u ** i * v ** j for i in range(g.shape[0]) for j in range(g.shape[1]) if g[i, j])


@pytest.mark.parametrize("da,db", [(2, 4), (2, 6), (3, 3), (1, 2), (4, 2)])
def test_bezout_det_equals_sylvester_resultant(da, db):
    """det Bezout_n(a, b) = +-lc^(n-m) Res_Sylvester(a, b) exactly (integer input)."""
    u, v = sympy.symbols("u v")
    rng = np.random.default_rng(100 + 10 * da + db)
    dmax = max(da, db)
    for _ in range(6):
        ga = np.zeros((dmax + 1, dmax + 1))
        gb = np.zeros((dmax + 1, dmax + 1))
        ga[: da + 1, : da + 1] = _random_bipoly(rng, da)
        gb[: db + 1, : db + 1] = _random_bipoly(rng, db)
        r = oracle.resultant(ga, gb)
        A = sympy.Poly(_grid_to_sympy(ga, u, v), u)
        B = sympy.Poly(_grid_to_sympy(gb, u, v), u)
        res = sympy.resultant(A.as_expr(), B.as_expr(), u)
        m, n = min(da, db), max(da, db)
        lc = (B if db >= da else A).LC()
        expect = sympy.Poly(sympy.expand(lc ** (n - m) * res), v)
        ec = [float(c) for c in reversed(expect.all_coeffs())]
        got = list(r)
        ln = max(len(ec), len(got))
        ec += [0.0] * (ln - len(ec))
        got += [0.0] * (ln - len(got))
        ec, got = np.array(ec), np.array(got)
        ok_pos = np.array_equal(ec, got)
        ok_neg = np.array_equal(ec, -got)
        assert ok_pos or ok_neg, (da, db, ec, got)


# ------------------------------------------------ root isolation (Sec. 4.2)
def test_isolation_matches_exact_sturm_counts():
    x = sympy.symbols("x")
    rng = np.random.default_rng(7)
    lo, hi = sympy.Rational(-1, 10 ** 6), 1 + sympy.Rational(1, 10 ** 6)
    for deg in range(1, 13):
        for _ in range(8):
            c = rng.integers(-20, 21, deg + 1).astype(float)
            if c[-1] == 0:
                c[-1] = 1
            P = sympy.Poly(sum(int(ci) * x ** i for i, ci in enumerate(c)), x)
            if sympy.degree(sympy.gcd(P, P.diff(x))) > 0:
                continue  # repeated roots: the count of distinct roots differs by design
            exact = P.count_roots(lo, hi)
            roots, flags = oracle.isolate(c, float(lo), float(hi))
            simple = roots[(flags & oracle.F_TANGENT) == 0]
            assert simple.size == exact, (deg, c, roots, exact)


def test_isolation_recovers_planted_roots():
    rng = np.random.default_rng(11)
    for trial in range(200):
        k_in = rng.integers(0, 6)
        k_out = rng.integers(0, 4)
        k_cplx = rng.integers(0, 3)
        inside = np.sort(rng.uniform(0.0, 1.0, k_in))
        if k_in > 1 and np.min(np.diff(inside)) < 1e-3:
            continue
        outside = np.concatenate([rng.uniform(-3, -0.1, k_out // 2 + k_out % 2), rng.uniform(1.1, 3, k_out // 2)])
        p = np.array([rng.uniform(0.5, 2.0)])
        for r_ in np.concatenate([inside, outside]):
            p = np.convolve(p, [-r_, 1.0])
        for _ in range(k_cplx):
            re, im = rng.uniform(-1, 2), rng.uniform(0.05, 1.0)
            p = np.convolve(p, [re * re + im * im, -2 * re, 1.0])
        roots, flags = oracle.isolate(p, -1e-6, 1 + 1e-6)
        assert roots.size == inside.size, (trial, inside, roots)
        assert np.allclose(roots, inside, atol=1e-9)


def test_isolation_reports_tangent_root():
    p = np.convolve(np.convolve([-0.3, 1.0], [-0.3, 1.0]), [2.0, 1.0])  # (x-.3)^2 (x+2)
    roots, flags = oracle.isolate(p, -1e-6, 1 + 1e-6)
    assert roots.size == 1 and abs(roots[0] - 0.3) < 1e-7
    assert flags[0] & oracle.F_TANGENT and flags[0] & oracle.F_ILL_COND


# ------------------------------------------------ degrees (Table tab_sum / tab_equ)
def test_degrees_curved_and_face_normal():
    tri, x0, x2 = scenes.random_triangle_cases(3, 40, curved=True)
    for i in range(40):
        for type_, name in ((0, "R"), (1, "T")):
            x2i = x2[i].copy()
            if type_ == 1:
                x2i[2] = -x2i[2]
            a, b, info = oracle.system_k1(tri[:, i], x0[i], x2i, type_, 1.0, 1.5)
            assert [info["total_deg_a"], info["total_deg_b"]] == DEG["bivariate"][name]
    # Constant shading normal tilted off the face normal: the F column of
    # Table tab_equ is reached exactly.  With the geometric face normal,
    # (x1 - x0).n is constant on the plane, so the product form drops further
    # (the table counts degree with the neighbouring vertices free as well).
    tri, x0, x2 = scenes.random_triangle_cases(4, 40, flat_normal=True)
    rng = np.random.default_rng(4)
    for i in range(40):
        tilted = tri[:, i].copy()
        nt = tilted[9:12] + rng.normal(0, 0.3, 3)
        tilted[9:18] = np.tile(nt / np.linalg.norm(nt), 3)
        x2i = x2[i].copy()
        x2i[2] = -x2i[2]
        for t18, exact in ((tilted, True), (tri[:, i], False)):
            a, b, info = oracle.system_k1(t18, x0[i], x2[i], 0)
            ca = DEG["face_normal"]["coplanarity_endpoint_form"]
            cb = DEG["face_normal"]["product_form"]
            assert info["total_deg_a"] == ca
            assert info["total_deg_b"] == cb if exact else info["total_deg_b"] <= cb
            a, b, info = oracle.system_k1(t18, x0[i], x2i, 1, 1.0, 1.5)
            assert info["total_deg_a"] == ca
            sq = DEG["face_normal"]["square_form"]
            assert info["total_deg_b"] == sq if exact else info["total_deg_b"] <= sq


def test_resultant_degree_bound():
    """deg r <= deg(a) deg(b) (Bezout's theorem on the Sec. 3.5 degree pairs)
    plus (n - m) deg(lc_u b) for the leading-coefficient factor of the n x n
    Bezout determinant.  For R the product form with t = n x e1 has no u^4
    term (its coefficient is e1 . ((n1 - n0) x e1) = 0), so n = 3 and one
    spurious factor b_3(v) of degree 1 appears (t = n x e2 removes v^4
    instead); T keeps u-degree 6."""
    tri, x0, x2 = scenes.random_triangle_cases(5, 30)
    for i in range(30):
        for type_, name in ((0, "R"), (1, "T")):
            x2i = x2[i].copy()
            if type_ == 1:
                x2i[2] = -x2i[2]
            a, b, info = oracle.system_k1(tri[:, i], x0[i], x2i, type_, 1.0, 1.5)
            r = oracle.resultant(a, b)
            lc_deg = info["total_deg_b"] - info["deg_u_b"]
            extra = (info["deg_u_b"] - info["deg_u_a"]) * lc_deg
            if name == "R":  # t = n x e1 removes u^4; t = n x e2 removes v^4 instead
                assert info["deg_u_b"] == (3 if info["edge"] == 1 else 4)
            else:
                assert info["deg_u_b"] == 6
            assert len(r) - 1 <= DEG["resultant_degree_bound"][name] + extra


# ------------------------------------------------ closed forms
def _flat_cases(seed, n):
    tri, x0, x2 = scenes.random_triangle_cases(seed, n, flat_normal=True)
    return tri, x0, x2


def test_flat_reflection_is_mirror_image_point():
    tri, x0, x2 = _flat_cases(21, 3000)
    paths, cnt = _batch(tri, x0, x2, 0)
    hits = 0
    for i in range(tri.shape[1]):
        P, N = _tri_arrays(tri[:, i])
        n = N[0] / np.linalg.norm(N[0])
        s0 = np.dot(x0[i] - P[0], n)
        s2 = np.dot(x2[i] - P[0], n)
        got = paths[paths["chain"] == i]
        if s0 * s2 <= 0:
            assert got.size == 0
            continue
        xm = x0[i] - 2 * s0 * n  # mirror image of x0
        s = np.dot(P[0] - xm, n) / np.dot(x2[i] - xm, n)
        x1 = xm + s * (x2[i] - xm)
        u, v = _bary(P, x1)
        w = min(u, v, 1 - u - v)
        if abs(w) < 1e-6:
            continue
        if w < 0:
            assert got.size == 0, (i, u, v, got)
        else:
            hits += 1
            assert got.size == 1, (i, u, v, got)
            assert abs(got["uv"][0, 0] - u) < 1e-11 and abs(got["uv"][0, 1] - v) < 1e-11
    assert hits > 20


def _fermat_point(x0, x2, p0, n, eta0, eta1):
    """Minimiser of eta0 |x1-x0| + eta1 |x2-x1| over the plane (p0, n), by
    bisection on the derivative along the segment of the feet (convex)."""
    h0 = np.dot(x0 - p0, n)
    h2 = np.dot(x2 - p0, n)
    f0 = x0 - h0 * n
    f2 = x2 - h2 * n
    L = np.linalg.norm(f2 - f0)
    if L == 0:
        return f0
    lo, hi = 0.0, 1.0
    for _ in range(200):
        s = 0.5 * (lo + hi)
        d = eta0 * s * L * L / np.hypot(h0, s * L) - eta1 * (1 - s) * L * L / np.hypot(h2, (1 - s) * L)
        if d > 0:
            hi = s
        else:
            lo = s
    s = 0.5 * (lo + hi)
    return f0 + s * (f2 - f0)


def test_flat_refraction_is_fermat_point():
    tri, x0, x2 = _flat_cases(22, 3000)
    x2 = x2.copy()
    x2[:, 2] = -x2[:, 2]  # below the surface
    eta0, eta1 = 1.0, 1.5
    paths, cnt = _batch(tri, x0, x2, 1, eta0, eta1)
    hits = 0
    for i in range(tri.shape[1]):
        P, N = _tri_arrays(tri[:, i])
        n = N[0] / np.linalg.norm(N[0])
        got = paths[paths["chain"] == i]
        if np.dot(x0[i] - P[0], n) * np.dot(x2[i] - P[0], n) >= 0:
            assert got.size == 0
            continue
        x1 = _fermat_point(x0[i], x2[i], P[0], n, eta0, eta1)
        u, v = _bary(P, x1)
        w = min(u, v, 1 - u - v)
        if abs(w) < 1e-6:
            continue
        if w < 0:
            assert got.size == 0, (i, u, v, got)
        else:
            hits += 1
            assert got.size == 1, (i, u, v, got)
            assert abs(got["uv"][0, 0] - u) < 1e-10 and abs(got["uv"][0, 1] - v) < 1e-10
    assert hits > 20


# ------------------------------------------------ brute force (Eq. eq_ch only)
def _hn(P, N, x0, x2, uv, type_, eta0, eta1):
    u, v = uv
    x1 = P[0] + u * (P[1] - P[0]) + v * (P[2] - P[0])
    n = N[0] + u * (N[1] - N[0]) + v * (N[2] - N[0])
    d0 = x1 - x0
    d1 = x2 - x1
    if type_ == 0:
        h = d1 / np.linalg.norm(d1) - d0 / np.linalg.norm(d0)
    else:
        h = eta1 * d1 / np.linalg.norm(d1) - eta0 * d0 / np.linalg.norm(d0)
    return h, n, d0, d1


def _brute_force(P, N, x0, x2, type_, eta0, eta1, grid=160):
    """All (u, v) with h x n = 0 by dense search + Gauss-Newton, no polynomials."""
    g = np.linspace(-0.02, 1.02, grid)
    U, V = np.meshgrid(g, g, indexing="ij")
    X1 = P[0] + U[..., None] * (P[1] - P[0]) + V[..., None] * (P[2] - P[0])
    Nn = N[0] + U[..., None] * (N[1] - N[0]) + V[..., None] * (N[2] - N[0])
    D0 = X1 - x0
    D1 = x2 - X1
    D0 /= np.linalg.norm(D0, axis=-1, keepdims=True)
    D1 /= np.linalg.norm(D1, axis=-1, keepdims=True)
    H = (D1 - D0) if type_ == 0 else (eta1 * D1 - eta0 * D0)
    Hn = H / np.maximum(np.linalg.norm(H, axis=-1, keepdims=True), 1e-300)
    Nu = Nn / np.linalg.norm(Nn, axis=-1, keepdims=True)
    F = np.linalg.norm(np.cross(Hn, Nu), axis=-1)
    sols = []
    for i in range(1, grid - 1):
        for j in range(1, grid - 1):
            f = F[i, j]
            if f > 0.05 or U[i, j] + V[i, j] > 1.04:
                continue
            if f > F[i - 1:i + 2, j - 1:j + 2].min():
                continue
            uv = np.array([U[i, j], V[i, j]])

            def res(z):
                h, n, _, _ = _hn(P, N, x0, x2, z, type_, eta0, eta1)
                return np.cross(h, n / np.linalg.norm(n))

            for _ in range(60):
                r0 = res(uv)
                J = np.empty((3, 2))
                for c in range(2):
                    dz = np.zeros(2)
                    dz[c] = 1e-7
                    J[:, c] = (res(uv + dz) - res(uv - dz)) / 2e-7
                step, *_ = np.linalg.lstsq(J, -r0, rcond=None)
                uv = uv + step
                if np.linalg.norm(step) < 1e-15:
                    break
            h, n, d0, d1 = _hn(P, N, x0, x2, uv, type_, eta0, eta1)
            if np.linalg.norm(np.cross(h, n)) / (np.linalg.norm(h) * np.linalg.norm(n)) > 1e-11:
                continue
            if np.linalg.norm(h) <= 1e-9:
                continue
            s0, s1 = np.dot(d0, n), np.dot(d1, n)
            if type_ == 0 and np.sign(s0) == np.sign(s1):
                continue
            if type_ == 1 and np.sign(s0) != np.sign(s1):
                continue
            if any(np.max(np.abs(uv - s)) < 1e-8 for s in sols):
                continue
            sols.append(uv)
    return sols


def _planted_cases(seed, n, type_, eta0=1.0, eta1=1.5):
    """Curved triangles whose x2 lies on the exactly reflected / refracted ray
    (vector reflection law, vector Snell law) from x0 through a random
    interior point, so each case has at least one solution."""
    rng = np.random.default_rng(seed)
    tri, x0, _ = scenes.random_triangle_cases(seed, n, curved=True)
    x2 = np.empty_like(x0)
    for i in range(n):
        P, N = _tri_arrays(tri[:, i])
        u, v = rng.dirichlet([1.0, 1.0, 1.0])[1:]
        x1 = P[0] + u * (P[1] - P[0]) + v * (P[2] - P[0])
        nn = N[0] + u * (N[1] - N[0]) + v * (N[2] - N[0])
        nn /= np.linalg.norm(nn)
        d = (x1 - x0[i]) / np.linalg.norm(x1 - x0[i])
        c = -np.dot(d, nn)
        if type_ == 0:
            out = d + 2 * c * nn
        else:
            if c < 0:
                nn, c = -nn, -c
            r = eta0 / eta1
            out = r * d + (r * c - np.sqrt(1 - r * r * (1 - c * c))) * nn
        x2[i] = x1 + rng.uniform(0.5, 2.0) * out
    return tri, x0, x2


@pytest.mark.parametrize("type_", [0, 1])
def test_brute_force_matches_oracle_on_curved_triangles(type_):
    eta0, eta1 = 1.0, 1.5
    tri, x0, x2 = _planted_cases(30 + type_, 60, type_, eta0, eta1)
    paths, _ = _batch(tri, x0, x2, type_, eta0, eta1)
    total = 0
    for i in range(tri.shape[1]):
        P, N = _tri_arrays(tri[:, i])
        bf = [s for s in _brute_force(P, N, x0[i], x2[i], type_, eta0, eta1)
              if min(s[0], s[1], 1 - s[0] - s[1]) >= 0]
        got = paths[paths["chain"] == i]
        edge = lambda s: abs(min(s[0], s[1], 1 - s[0] - s[1])) < 1e-6
        for s in bf:
            m = np.max(np.abs(got["uv"][:, :2] - s), axis=1) if got.size else np.array([1.0])
            assert m.min() < 1e-8 or edge(s), (i, s, got["uv"])
        for g in got:
            s = g["uv"][:2]
            m = [np.max(np.abs(s - b)) for b in bf]
            assert (m and min(m) < 1e-8) or edge(s) or g["flags"] & oracle.F_ILL_COND, (i, s, bf)
        total += len(bf)
    assert total >= 55


# ------------------------------------------------ invariants
def test_paths_satisfy_constraint_and_lie_inside():
    s = scenes.reflect_scene()
    paths, cnt = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains)
    assert cnt["admissible"] == paths.size > 500
    assert np.all(paths["residual"] < 1e-9)
    u, v = paths["uv"][:, 0], paths["uv"][:, 1]
    assert np.all(u >= 0) and np.all(v >= 0) and np.all(u + v <= 1)


@pytest.mark.parametrize("type_", [0, 1])
def test_reciprocity(type_):
    eta0, eta1 = 1.0, 1.5
    tri, x0, x2 = _planted_cases(40 + type_, 300, type_, eta0, eta1)
    fwd, _ = _batch(tri, x0, x2, type_, eta0, eta1)
    bwd, _ = _batch(tri, x2, x0, type_, eta1, eta0)
    assert fwd.size > 250
    for g in fwd:
        b = bwd[bwd["chain"] == g["chain"]]
        edge = g["flags"] & (oracle.F_EDGE | oracle.F_ILL_COND)
        ok = b.size and np.max(np.abs(b["uv"][:, :2] - g["uv"][:2]), axis=1).min() < 1e-9
        assert ok or edge


@pytest.mark.parametrize("type_", [0, 1])
def test_rigid_motion_invariance(type_):
    rng = np.random.default_rng(50 + type_)
    tri, x0, x2 = _planted_cases(50 + type_, 300, type_)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    t = rng.normal(size=3)
    tri2 = tri.copy()
    for r in range(6):
        blk = tri[3 * r:3 * r + 3]
        tri2[3 * r:3 * r + 3] = Q @ blk + (t[:, None] if r < 3 else 0.0)
    a, _ = _batch(tri, x0, x2, type_, 1.0, 1.5)
    b, _ = _batch(tri2, x0 @ Q.T + t, x2 @ Q.T + t, type_, 1.0, 1.5)
    assert a.size > 250
    for g in a:
        m = b[b["chain"] == g["chain"]]
        ok = m.size and np.max(np.abs(m["uv"][:, :2] - g["uv"][:2]), axis=1).min() < 1e-9
        assert ok or g["flags"] & (oracle.F_EDGE | oracle.F_ILL_COND)
