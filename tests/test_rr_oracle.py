"""Pins of the 2-bounce reflection (RR) oracle: the scaled reflected
direction (Eq. eq_431_di) against the mirror law, the system degrees
against Table tab_sum, paths planted by forward ray tracing, reciprocity
(the reversed chain has the reversed paths), and the flat-mirror case,
which reduces to a one-bounce reflection towards the mirror image of x3
solved by the independent one-bounce oracle."""
import numpy as np
import pytest

import oracle
from oracle import rr, tt


def _refl(d, n):
    n = n / np.linalg.norm(n)
    return d - 2.0 * (d @ n) * n


def _corridor(rng, tilt=0.1):
    """A floor triangle (normals about +z) and a ceiling triangle (normals
    about -z) with perturbed vertices and shading normals."""
    P1 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]]) + rng.normal(size=(3, 3)) * 0.05
    N1 = np.array([0, 0, 1.0]) + rng.normal(size=(3, 3)) * tilt
    P2 = np.array([[0, 0, 1.0], [0, 1, 1.0], [1, 0, 1.0]]) + rng.normal(size=(3, 3)) * 0.05
    N2 = np.array([0, 0, -1.0]) + rng.normal(size=(3, 3)) * tilt
    return P1, N1, P2, N2


def _trace(x0, P1, N1, P2, N2, u1, v1, reach=0.4):
    """Forward trace: reflect at (u1, v1) on T1, intersect T2's plane,
    reflect there; x3 lies on the outgoing ray.  Returns (x3, w, t)."""
    x1 = P1[0] + u1 * (P1[1] - P1[0]) + v1 * (P1[2] - P1[0])
    n1 = N1[0] + u1 * (N1[1] - N1[0]) + v1 * (N1[2] - N1[0])
    d1 = _refl(x1 - x0, n1)
    A = np.stack([P2[1] - P2[0], P2[2] - P2[0], -d1], 1)
    u2, v2, t = np.linalg.solve(A, x1 - P2[0])
    x2 = x1 + t * d1
    n2 = N2[0] + u2 * (N2[1] - N2[0]) + v2 * (N2[2] - N2[0])
    d2 = _refl(d1, n2)
    return x2 + reach * d2 / np.linalg.norm(d2), np.array([u1, v1, u2, v2]), t


def test_reflected_direction_is_the_mirror_law():
    """Eq. eq_431_di: D(u, v) = |n|^2 |d0| times the mirror-reflected unit
    direction, exactly (a positive multiple)."""
    rng = np.random.default_rng(0)
    for _ in range(30):
        P1, N1, _, _ = _corridor(rng, 0.3)
        x0 = rng.normal(size=3) + [0, 0, 2]
        x1p, n1p = tt.tri_polys(P1, N1)
        D = rr.reflected_direction(x0, x1p, n1p)
        u, v = rng.random(2) * 0.5
        x1 = P1[0] + u * (P1[1] - P1[0]) + v * (P1[2] - P1[0])
        n1 = N1[0] + u * (N1[1] - N1[0]) + v * (N1[2] - N1[0])
        d0 = x1 - x0
        want = (n1 @ n1) * np.linalg.norm(d0) * _refl(d0 / np.linalg.norm(d0), n1)
        got = np.array([tt.bp_eval(D[k], u, v) for k in range(3)])
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_system_degrees_within_table_bounds():
    """Table tab_sum: RR degrees 10 and 16 (total); the u-degree of the
    Bezout matrix is at most 16."""
    rng = np.random.default_rng(1)
    P1, N1, P2, N2 = _corridor(rng)
    s = rr.build_rr([0.2, 0.2, 0.6], [0.6, 0.5, 0.4], P1, N1, P2, N2)
    for key, bound in (("a", 10), ("b", 16)):
        c = s[key]
        i, j = np.nonzero(np.abs(c) > 1e-14 * np.abs(c).max())
        assert (i + j).max() <= bound
    assert max(tt.deg_u(s["a"]), tt.deg_u(s["b"])) <= 16


def _planted(seed):
    rng = np.random.default_rng(seed)
    while True:
        P1, N1, P2, N2 = _corridor(rng)
        x0 = np.array([0.2, 0.2, 0.6]) + rng.normal(size=3) * 0.05
        u1, v1 = 0.2 + 0.25 * rng.random(), 0.2 + 0.25 * rng.random()
        x3, w, t = _trace(x0, P1, N1, P2, N2, u1, v1)
        if t > 0 and min(w[2], w[3], 1 - w[2] - w[3]) > 0.02:
            return x0, x3, P1, N1, P2, N2, w


@pytest.mark.parametrize("seed", [2, 3, 4, 5, 6])
def test_planted_paths_found(seed):
    """A path planted by forward tracing over curved (shading-normal)
    triangles is recovered to 1e-9; every path returned satisfies the
    reflection law at both vertices and lies in both triangles."""
    x0, x3, P1, N1, P2, N2, w = _planted(seed)
    out = rr.solve_candidate(x0, x3, P1, N1, P2, N2)
    assert any(np.max(np.abs(p["uv"] - w)) < 1e-9 for p in out), (w, [p["uv"] for p in out])
    for p in out:
        r1, r2, side, _ = rr.residuals(p["uv"], x0, x3, P1, N1, P2, N2)
        assert side and max(np.linalg.norm(r1), np.linalg.norm(r2)) < 1e-9
        u1, v1, u2, v2 = p["uv"]
        assert min(u1, v1, 1 - u1 - v1) >= 0 and min(u2, v2, 1 - u2 - v2) >= 0


@pytest.mark.parametrize("seed", [7, 8])
def test_reciprocity(seed):
    """Light paths are reversible: the chain x3 -> T2 -> T1 -> x0 has the
    same paths with the vertex order swapped."""
    x0, x3, P1, N1, P2, N2, w = _planted(seed)
    fwd = rr.solve_candidate(x0, x3, P1, N1, P2, N2)
    bwd = rr.solve_candidate(x3, x0, P2, N2, P1, N1)
    a = sorted(tuple(np.round(p["uv"], 8)) for p in fwd)
    b = sorted(tuple(np.round(np.r_[p["uv"][2:], p["uv"][:2]], 8)) for p in bwd)
    assert len(a) >= 1 and a == b


def test_flat_mirror_reduces_to_one_bounce():
    """With a flat second triangle (one normal), x0 -> T1 -> T2 -> x3 is the
    one-bounce reflection x0 -> T1 -> x3' (x3' the mirror image of x3 in
    T2's plane) whose segment x1 -> x3' crosses the plane inside T2.  The
    one-bounce paths come from the C oracle."""
    oracle.build()
    rng = np.random.default_rng(9)
    hits = 0
    for trial in range(6):
        P1 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]]) + rng.normal(size=(3, 3)) * 0.05
        N1 = np.array([0, 0, 1.0]) + rng.normal(size=(3, 3)) * 0.15
        P2 = np.array([[-2, -2, 1.0], [4, -2, 1.0], [-2, 4, 1.0]])  # large flat ceiling
        N2 = np.tile([0, 0, -1.0], (3, 1))
        x0 = np.array([0.3, 0.2, 0.5]) + rng.normal(size=3) * 0.05
        x3 = np.array([0.4, 0.5, 0.5]) + rng.normal(size=3) * 0.05
        x3m = x3.copy()
        x3m[2] = 2.0 - x3[2]  # mirror image in z = 1
        tri = np.zeros((18, 1))
        for v in range(3):
            tri[3 * v:3 * v + 3, 0] = P1[v]
            tri[9 + 3 * v:12 + 3 * v, 0] = N1[v]
        one, _ = oracle.solve(tri, x0[None], x3m[None], np.ones((1, 3)), np.zeros((1, 2), np.int32),
                              np.ones(1, np.int32), np.array([[0, 0, -1]], np.int32))
        want = []
        for p in one:
            u1, v1 = p["uv"][0], p["uv"][1]
            x1 = P1[0] + u1 * (P1[1] - P1[0]) + v1 * (P1[2] - P1[0])
            t = (1.0 - x1[2]) / (x3m[2] - x1[2])
            x2 = x1 + t * (x3m - x1)
            A = np.stack([P2[1] - P2[0], P2[2] - P2[0]], 1)
            u2, v2 = np.linalg.lstsq(A, x2 - P2[0], rcond=None)[0]
            if 0 < t < 1 and min(u2, v2, 1 - u2 - v2) >= 0:
                want.append((u1, v1, u2, v2))
        got = [p["uv"] for p in rr.solve_candidate(x0, x3, P1, N1, P2, N2)]
        assert len(got) == len(want), (trial, got, want)
        for w in want:
            assert any(np.max(np.abs(g - w)) < 1e-8 for g in got), (trial, w, got)
        hits += len(want)
    assert hits >= 4


def _tri(T, t):
    P = np.stack([T[0:3, t], T[3:6, t], T[6:9, t]])
    N = np.stack([T[9:12, t], T[12:15, t], T[15:18, t]])
    return P, N


def planted_corridor_cases(seed, n, n_cells=16, jitter=True):
    """Paths planted by forward tracing in the corridor scene: a light near
    the scene's, a random point of a random floor triangle, the mirror
    reflection to the ceiling triangle the ray hits (Moller-Trumbore over
    all of them), the reflection there; x3 on the outgoing ray at z = 0.5.
    jitter=False keeps the scene's light.  Returns [(x0, x3, t_floor,
    t_ceiling, (u1, v1, u2, v2))]."""
    from paper_2405_13409_gb300 import scenes
    s = scenes.corridor_scene(seed=0, n_cells=n_cells, n_recv=2)
    T = s.tri
    half = s.n_tris // 2
    C0 = T[0:3, half:].T
    E1 = T[3:6, half:].T - C0
    E2 = T[6:9, half:].T - C0
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        x0 = np.array([-0.6, 0.1, 0.5]) + (rng.normal(size=3) * [0.2, 0.2, 0.05] if jitter else 0.0)
        t1 = int(rng.integers(0, half))
        P1, N1 = _tri(T, t1)
        u1, v1 = rng.uniform(0.05, 0.9, 2)
        if u1 + v1 > 0.95:
            continue
        x1 = P1[0] + u1 * (P1[1] - P1[0]) + v1 * (P1[2] - P1[0])
        n1 = N1[0] + u1 * (N1[1] - N1[0]) + v1 * (N1[2] - N1[0])
        d1 = _refl(x1 - x0, n1)
        if d1[2] <= 0:
            continue
        # ray x1 + t d1 against every ceiling triangle
        pv = np.cross(d1, E2)
        det = np.einsum("ij,ij->i", E1, pv)
        sv = x1 - C0
        uu = np.einsum("ij,ij->i", sv, pv) / det
        qv = np.cross(sv, E1)
        vv = qv @ d1 / det
        tt_ = np.einsum("ij,ij->i", E2, qv) / det
        ok = (tt_ > 0) & (uu > 0.02) & (vv > 0.02) & (uu + vv < 0.98)
        if not ok.any():
            continue
        j = int(np.argmin(np.where(ok, tt_, np.inf)))
        P2, N2 = _tri(T, half + j)
        u2, v2 = uu[j], vv[j]
        x2 = x1 + tt_[j] * d1
        n2 = N2[0] + u2 * (N2[1] - N2[0]) + v2 * (N2[2] - N2[0])
        d2 = _refl(d1, n2)
        if d2[2] >= 0:
            continue
        x3 = x2 + ((0.5 - x2[2]) / d2[2]) * d2
        out.append((x0, x3, t1, half + j, np.array([u1, v1, u2, v2])))
    return out


def test_planted_corridor_paths_found():
    """The corridor mesh (heightfield mirrors): planted paths are recovered
    by the oracle from the mesh's SoA rows."""
    from paper_2405_13409_gb300 import scenes
    cases = planted_corridor_cases(20, 4)
    T = scenes.corridor_scene(seed=0, n_cells=16, n_recv=2).tri
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    chains = np.array([[i, c[2], c[3]] for i, c in enumerate(cases)], np.int32)
    ref = rr.solve(T, x0s, x3s, chains)
    for i, c in enumerate(cases):
        got = ref[ref["query"] == i]
        assert any(np.max(np.abs(p["uv"] - c[4])) < 1e-9 for p in got), (i, c[4], got["uv"])


def test_two_flat_mirrors_double_image():
    """Two flat parallel mirrors with face normals, floor z = 0 and ceiling
    z = h: the path is the straight line from x0 to the image of x3 mirrored
    in the ceiling and then in the floor (closed form).  It crosses the
    floor at x1 and the floor's image of the ceiling (z = -h) above x2.
    Here b does not depend on u1, and the path is still found."""
    rng = np.random.default_rng(12)
    F = np.array([[-2.0, -2.0, 0.0], [4.0, -2.0, 0.0], [-2.0, 4.0, 0.0]])
    for _ in range(8):
        h = rng.uniform(0.6, 1.5)
        x0 = np.r_[rng.uniform(-0.3, 0.3, 2), rng.uniform(0.2, 0.8) * h]
        x3 = np.r_[rng.uniform(-0.3, 0.3, 2) + 0.5, rng.uniform(0.2, 0.8) * h]
        img = np.r_[x3[:2], -(2.0 * h - x3[2])]  # ceiling image, then floor image
        t1 = x0[2] / (x0[2] - img[2])
        t2 = (x0[2] + h) / (x0[2] - img[2])
        x1 = x0 + t1 * (img - x0)
        x2 = np.r_[(x0 + t2 * (img - x0))[:2], h]
        E = np.stack([F[1] - F[0], F[2] - F[0]], 1)
        u1, v1 = np.linalg.lstsq(E, x1 - F[0], rcond=None)[0]
        u2, v2 = np.linalg.lstsq(E, x2 - (F[0] + [0, 0, h]), rcond=None)[0]
        out = rr.solve_candidate(x0, x3, F, np.tile([0, 0, 1.0], (3, 1)), F + [0, 0, h],
                                 np.tile([0, 0, -1.0], (3, 1)))
        assert len(out) == 1, out
        assert np.max(np.abs(out[0]["uv"] - [u1, v1, u2, v2])) < 1e-9, (out[0]["uv"], [u1, v1, u2, v2])
