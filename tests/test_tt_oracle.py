"""Pins of the 2-bounce refraction (TT) oracle: the rational sqrt pieces,
the rational coordinate mapping, the Bezout determinant, the flat-slab
closed form (Fermat), planted curved paths and a polynomial-free brute
force on a tiny slab."""
import json
import os

import numpy as np
import pytest

from oracle import tt

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    g = json.load(open(os.path.join(HERE, "golden", "sqrt_pieces.json")))
    assert tuple(g["breaks"]) == tt.SQRT_BREAKS
    return np.array(g["coeffs"])


def test_sqrt_pieces_error_bound():
    """Sec. 3.4: the six-piece approximant stays within 1e-3 of sqrt on [0, 1]."""
    x = np.linspace(0.0, 1.0, 1_000_001)
    err = np.abs(tt.sqrt_approx(x, _table()) - np.sqrt(x))
    assert err.max() < 1e-3, err.max()
    assert tt.piece_of(0.0) == 0 and tt.piece_of(1.0) == 5 and tt.piece_of(0.3) == 4


def _refl_dir(d, n):
    return -2.0 * (d @ n) * n + d * (n @ n)


def test_mapping_matches_ray_plane_intersection():
    """Eq. eq_rct with an exactly rational direction (the scaled reflected
    direction of Sec. 3.4) reproduces the textbook ray-plane intersection."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        P1 = rng.normal(size=(3, 3))
        N1 = rng.normal(size=(3, 3))
        P2 = rng.normal(size=(3, 3)) + [0, 0, -2]
        x0 = rng.normal(size=3) + [0, 0, 3]
        x1, n1 = tt.tri_polys(P1, N1)
        d0 = tt.vsub(x1, tt.vconst(x0))
        D = tt.vsub(tt.vscale(d0, tt.vdot(n1, n1)), tt.vscale(n1, 2.0 * tt.vdot(d0, n1)))
        ut, vt, kap, tpar = tt.mapping(D, x1, P2)
        u, v = rng.random(2)
        xx = P1[0] + u * (P1[1] - P1[0]) + v * (P1[2] - P1[0])
        nn = N1[0] + u * (N1[1] - N1[0]) + v * (N1[2] - N1[0])
        d = _refl_dir(xx - x0, nn)
        # textbook: solve xx + t d = p0 + a e1 + b e2
        A = np.stack([P2[1] - P2[0], P2[2] - P2[0], -d], 1)
        a, b, t = np.linalg.solve(A, xx - P2[0])
        k = tt.bp_eval(kap, u, v)
        assert abs(tt.bp_eval(ut, u, v) / k - a) < 1e-9 * (1 + abs(a))
        assert abs(tt.bp_eval(vt, u, v) / k - b) < 1e-9 * (1 + abs(b))
        assert abs(tt.bp_eval(tpar, u, v) / k - t) < 1e-9 * (1 + abs(t))


def test_refracted_direction_within_sqrt_error():
    """Eq. eq_refr_rational with the rational sqrt: the direction differs
    from Snell's refracted direction by no more than the approximant's
    error allows (|x - sqrt|, x = beta / s, scaled by |n|^2 |d|)."""
    rng = np.random.default_rng(1)
    table = _table()
    for _ in range(40):
        P1 = rng.normal(size=(3, 3)) * 0.1
        N1 = np.array([0, 0, 1.0]) + rng.normal(size=(3, 3)) * 0.1
        x0 = np.array([0.2, 0.1, 2.0])
        eta = 1 / 1.5
        x1, n1 = tt.tri_polys(P1, N1)
        c1 = P1.mean(0)
        s = float((N1.mean(0) @ N1.mean(0)) * ((c1 - x0) @ (c1 - x0)))
        xc = float((s - eta ** 2 * (s - ((c1 - x0) @ N1.mean(0)) ** 2)) / s)
        piece = tt.piece_of(xc)
        D, _ = tt.refracted_direction(x0, x1, n1, eta, piece, table, s)
        u, v = rng.random(2) * 0.5
        xx = P1[0] + u * (P1[1] - P1[0]) + v * (P1[2] - P1[0])
        nn = N1[0] + u * (N1[1] - N1[0]) + v * (N1[2] - N1[0])
        dh = (xx - x0) / np.linalg.norm(xx - x0)
        nh = nn / np.linalg.norm(nn)
        c = dh @ nh
        t = eta * (dh - c * nh) - np.sqrt(1 - eta ** 2 * (1 - c * c)) * nh
        Dv = np.array([tt.bp_eval(D[k], u, v) for k in range(3)])
        assert np.linalg.norm(Dv / np.linalg.norm(Dv) - t) < 5e-3


def test_bezout_determinant_is_resultant():
    """|det Bezout(a, b)| = |lc(b)|^(n - m) |Res(a, b)| (n = deg b >= m =
    deg a) on integer polynomials, against sympy's exact resultant."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(2)
    x = sympy.symbols("x")
    for m, n in [(3, 5), (4, 7), (2, 6), (5, 5)]:
        a = rng.integers(-5, 6, m + 1).astype(float)
        b = rng.integers(-5, 6, n + 1).astype(float)
        a[-1] = a[-1] or 3.0
        b[-1] = b[-1] or 2.0
        ac = np.zeros((1, n + 1))
        bc = np.zeros((1, n + 1))
        ac[0, :m + 1] = a
        bc[0, :n + 1] = b
        det = np.linalg.det(tt.bezout(ac, bc, n))[0]
        res = sympy.resultant(sum(int(c) * x ** i for i, c in enumerate(a)),
                              sum(int(c) * x ** i for i, c in enumerate(b)), x)
        want = abs(float(res)) * abs(b[-1]) ** (n - m)
        assert abs(abs(det) - want) <= 1e-9 * want, (m, n, det, want)


def _fermat(x0, x3, etas, P1, P2):
    from scipy.optimize import minimize
    e11, e12 = P1[1] - P1[0], P1[2] - P1[0]
    e21, e22 = P2[1] - P2[0], P2[2] - P2[0]

    def opl(w):
        x1 = P1[0] + w[0] * e11 + w[1] * e12
        x2 = P2[0] + w[2] * e21 + w[3] * e22
        return etas[0] * np.linalg.norm(x1 - x0) + etas[1] * np.linalg.norm(x2 - x1) + etas[2] * np.linalg.norm(x3 - x2)

    r = minimize(opl, np.full(4, 0.3), method="BFGS", options={"gtol": 1e-13})
    return r.x


@pytest.mark.parametrize("tilt", [0.0, 0.15])
def test_flat_slab_matches_fermat(tilt):
    """Two flat interfaces with constant normals: the exact TT path is the
    stationary point of the optical length (Fermat); the method, after its
    path-space refinement, returns exactly that path."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(3)
    n_inside = 0
    for _ in range(6):
        x0 = np.array([0.2, 0.1, 2.0]) + rng.normal(size=3) * 0.2
        x3 = np.array([0.0, 0.0, -1.0]) + rng.normal(size=3) * 0.4
        P1 = np.array([[-1.0, -1.0, 0.0], [1.5, -1.0, 0.0], [-1.0, 1.5, 0.0]])
        n1 = np.array([tilt, 0.0, 1.0])
        P1[:, 2] = -(P1[:, 0] * n1[0]) / n1[2]  # plane through the origin with normal n1
        P2 = P1 + [0.0, 0.0, -0.3]
        P2[:, 2] = -0.3 + 0.5 * tilt * P2[:, 1]
        n2 = np.cross(P2[1] - P2[0], P2[2] - P2[0])
        N1 = np.tile(n1, (3, 1))
        N2 = np.tile(n2, (3, 1))
        etas = (1.0, 1.5, 1.0)
        paths = tt.solve_candidate(x0, x3, etas, P1, N1, P2, N2, _table())
        want = _fermat(x0, x3, etas, P1, P2)
        margin = min(want[0], want[1], 1 - want[0] - want[1], want[2], want[3], 1 - want[2] - want[3])
        if margin < -1e-6:
            assert len(paths) == 0  # the only stationary path leaves a triangle
            continue
        assert margin > 1e-6
        n_inside += 1
        assert len(paths) == 1
        np.testing.assert_allclose(paths[0]["uv"], want, atol=1e-7)
        assert paths[0]["residual"] < 1e-9
        assert paths[0]["flags"] & tt.F_NEWTON_REFINED
    assert n_inside >= 3


def _refract(d, n, eta_in, eta_out):
    d = d / np.linalg.norm(d)
    n = n / np.linalg.norm(n)
    if d @ n > 0:
        n = -n
    e = eta_in / eta_out
    c = -(d @ n)
    k = 1 - e * e * (1 - c * c)
    if k < 0:
        return None
    return e * d + (e * c - np.sqrt(k)) * n


def _ray_tri(o, d, P):
    e1, e2 = P[1] - P[0], P[2] - P[0]
    pv = np.cross(d, e2)
    det = e1 @ pv
    if abs(det) < 1e-14:
        return None
    tv = o - P[0]
    u = (tv @ pv) / det
    qv = np.cross(tv, e1)
    return u, (d @ qv) / det, (e2 @ qv) / det


def planted_slab_cases(seed, n, n_cells=16, x0=None, x_range=None):
    """Exact TT paths traced through the slab generator's surfaces: a point
    of a top triangle, Snell refraction into the slab, the bottom triangle
    it hits, Snell refraction out, and the receiver on z = -1.  x0 defaults
    to the scene's light; x_range limits the top triangles to those whose
    first vertex has x in [lo, hi]."""
    from paper_2405_13409_gb300 import scenes
    s = scenes.slab_scene(seed=0, n_cells=n_cells, n_recv=4)
    T = s.tri
    half = T.shape[1] // 2
    rng = np.random.default_rng(seed)
    x0 = s.x_first[0] if x0 is None else np.asarray(x0, float)
    tops = np.arange(half) if x_range is None else np.where((T[0, :half] >= x_range[0]) & (T[0, :half] <= x_range[1]))[0]
    out = []
    while len(out) < n:
        t1 = int(tops[rng.integers(0, tops.size)])
        u, v = rng.random(2)
        if u + v > 1:
            u, v = 1 - u, 1 - v
        P1 = T[0:9, t1].reshape(3, 3)
        N1 = T[9:18, t1].reshape(3, 3)
        x1 = P1[0] + u * (P1[1] - P1[0]) + v * (P1[2] - P1[0])
        n1 = N1[0] + u * (N1[1] - N1[0]) + v * (N1[2] - N1[0])
        d1 = _refract(x1 - x0, n1, 1.0, 1.5)
        if d1 is None:
            continue
        hit = None
        for t2 in range(half, T.shape[1]):
            r = _ray_tri(x1, d1, T[0:9, t2].reshape(3, 3))
            if r and r[0] >= 0 and r[1] >= 0 and r[0] + r[1] <= 1 and r[2] > 0:
                hit = (t2, r)
                break
        if not hit:
            continue
        t2, (u2, v2, _) = hit
        P2 = T[0:9, t2].reshape(3, 3)
        N2 = T[9:18, t2].reshape(3, 3)
        x2 = P2[0] + u2 * (P2[1] - P2[0]) + v2 * (P2[2] - P2[0])
        n2 = N2[0] + u2 * (N2[1] - N2[0]) + v2 * (N2[2] - N2[0])
        d2 = _refract(x2 - x1, n2, 1.5, 1.0)
        if d2 is None or d2[2] >= 0:
            continue
        x3 = x2 + d2 * ((-1.0 - x2[2]) / d2[2])
        out.append((x0, x3, t1, t2, np.array([u, v, u2, v2]), P1, N1, P2, N2))
    return out


def test_planted_curved_slab_paths_found():
    table = _table()
    errs = []
    for (x0, x3, t1, t2, w, P1, N1, P2, N2) in planted_slab_cases(4, 8):
        paths = tt.solve_candidate(x0, x3, (1.0, 1.5, 1.0), P1, N1, P2, N2, table)
        d = [np.max(np.abs(p["uv"] - w)) for p in paths]
        assert d and min(d) < 1e-9, (t1, t2, d)
        p = paths[int(np.argmin(d))]
        assert p["residual"] < 1e-9
        errs.append(np.max(np.abs(p["uv_unrefined"] - p["uv"])))
    # the unrefined error of the rational approximation is reported, not a pin
    print("unrefined max |delta uv|", max(errs))


def _brute_force(x0, x3, etas, P1, N1, P2, N2, grid=8):
    """Polynomial-free exact solutions: from a (u1, v1) seed grid, trace the
    exact refracted ray into T2's plane for the (u2, v2) seed, then
    Gauss-Newton on the four tangential components of h x n = 0 written
    here from Snell's law (tangential continuity of eta d_hat)."""
    def F(w):
        x1 = P1[0] + w[0] * (P1[1] - P1[0]) + w[1] * (P1[2] - P1[0])
        n1 = N1[0] + w[0] * (N1[1] - N1[0]) + w[1] * (N1[2] - N1[0])
        x2 = P2[0] + w[2] * (P2[1] - P2[0]) + w[3] * (P2[2] - P2[0])
        n2 = N2[0] + w[2] * (N2[1] - N2[0]) + w[3] * (N2[2] - N2[0])
        out = []
        for xa, xb, xc, n, ea, eb in ((x0, x1, x2, n1, etas[0], etas[1]), (x1, x2, x3, n2, etas[1], etas[2])):
            di = (xb - xa) / np.linalg.norm(xb - xa)
            do = (xc - xb) / np.linalg.norm(xc - xb)
            nh = n / np.linalg.norm(n)
            g = ea * (di - (di @ nh) * nh) - eb * (do - (do @ nh) * nh)  # tangential mismatch
            a = np.cross(nh, [1.0, 0, 0] if abs(nh[0]) < 0.9 else [0, 1.0, 0])
            a /= np.linalg.norm(a)
            out += [g @ a, g @ np.cross(nh, a)]
        return np.array(out)

    sols = []
    for i in range(grid):
        for j in range(grid - i):
            u, v = (i + 0.5) / grid, (j + 0.5) / grid
            x1 = P1[0] + u * (P1[1] - P1[0]) + v * (P1[2] - P1[0])
            n1 = N1[0] + u * (N1[1] - N1[0]) + v * (N1[2] - N1[0])
            d1 = _refract(x1 - x0, n1, etas[0], etas[1])
            if d1 is None:
                continue
            r = _ray_tri(x1, d1, P2)
            if r is None:
                continue
            w = np.array([u, v, r[0], r[1]])
            for _ in range(20):
                f = F(w)
                J = np.stack([(F(w + h) - F(w - h)) / 2e-7 for h in np.eye(4) * 1e-7], 1)
                try:
                    w = w - np.linalg.lstsq(J, f, rcond=None)[0]
                except np.linalg.LinAlgError:
                    break
                if not np.all(np.isfinite(w)) or np.max(np.abs(w)) > 10:
                    break
            if not np.all(np.isfinite(w)) or np.max(np.abs(F(w))) > 1e-11:
                continue
            if min(w[0], w[1], 1 - w[0] - w[1], w[2], w[3], 1 - w[2] - w[3]) < 0:
                continue
            x1 = P1[0] + w[0] * (P1[1] - P1[0]) + w[1] * (P1[2] - P1[0])
            x2 = P2[0] + w[2] * (P2[1] - P2[0]) + w[3] * (P2[2] - P2[0])
            if not (x2[2] < x1[2]):  # travels down through the slab
                continue
            if all(np.max(np.abs(w - s)) > 1e-8 for s in sols):
                sols.append(w)
    return sols


def test_brute_force_tiny_slab():
    """2x2-cell surfaces, all (T1, T2) pairs for a receiver that a traced
    path reaches: every path the method returns is an exact solution, and
    its recall of the exact set is reported (the rational sqrt and the
    finite bisection make the method approximate, Sec. 6).  1024 initial
    intervals here to bound the test's time."""
    from paper_2405_13409_gb300 import scenes
    s = scenes.slab_scene(seed=0, n_cells=2, n_recv=2)
    T = s.tri
    half = T.shape[1] // 2
    table = _table()
    found = exact = matched = 0
    for (x0, x3, *_rest) in planted_slab_cases(5, 1, n_cells=2):
        for t1 in range(half):
            for t2 in range(half, T.shape[1]):
                P1, N1 = T[0:9, t1].reshape(3, 3), T[9:18, t1].reshape(3, 3)
                P2, N2 = T[0:9, t2].reshape(3, 3), T[9:18, t2].reshape(3, 3)
                ex = _brute_force(x0, x3, s.eta[0], P1, N1, P2, N2, grid=6)
                got = tt.solve_candidate(x0, x3, s.eta[0], P1, N1, P2, N2, table, n_intervals=1024)
                for p in got:
                    assert any(np.max(np.abs(p["uv"] - e)) < 1e-7 for e in ex) or p["flags"] & tt.F_EDGE, (t1, t2, p)
                found += len(got)
                exact += len(ex)
                matched += sum(any(np.max(np.abs(p["uv"] - e)) < 1e-7 for p in got) for e in ex)
    print("tiny slab: exact", exact, "method", found, "recall", matched / max(exact, 1))
    assert exact >= 1
    assert matched / exact >= 0.9
