"""Pins of the eigenvalue (linearisation + QZ) reference of the 2-bounce
resultant (oracle/qz.py, Sec. 4.2 "Discussion"): the companion pencil's
eigenvalues are the zeros of the exact determinant of random integer matrix
polynomials (sympy), det R(v1) equals the exact Sylvester resultant up to
the leading-coefficient factor, and the QZ-driven 2-bounce solves return the
closed-form and planted paths."""
import numpy as np
import pytest

from oracle import qz, rr, tt

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("n,d,seed", [(2, 3, 0), (3, 2, 1), (3, 4, 2), (4, 3, 3)])
def test_pencil_eigenvalues_are_the_determinant_zeros(n, d, seed):
    rng = np.random.default_rng(seed)
    R = rng.integers(-5, 6, size=(d + 1, n, n)).astype(float)
    v = sympy.symbols("v")
    M = sympy.Matrix(n, n, lambda i, j: sum(int(R[k, i, j]) * v ** k for k in range(d + 1)))
    det = sympy.Poly(sympy.expand(M.det()), v)
    want = np.array(sorted((complex(z) for z in det.nroots(n=30, maxsteps=200)), key=lambda z: (z.real, z.imag)))
    got = np.array(sorted(qz.matrix_poly_eigenvalues(R), key=lambda z: (z.real, z.imag)))
    assert got.size == want.size == det.degree()
    # match every exact zero to its nearest eigenvalue
    for z in want:
        assert np.min(np.abs(got - z)) <= 1e-7 * max(1.0, abs(z)), (z, got)


def test_determinant_is_the_sylvester_resultant():
    """det R(v1) of the polynomial-entry Bezout matrix equals +-lc(b)^(n-m)
    Res_u(a, b) exactly (sympy) at rational sample points, for bivariate
    integer polynomials of u-degrees (2, 3) and (3, 3)."""
    rng = np.random.default_rng(7)
    u, v = sympy.symbols("u v")
    for da, db in ((2, 3), (3, 3), (1, 4)):
        a = rng.integers(-4, 5, size=(da + 1, 3)).astype(float)
        b = rng.integers(-4, 5, size=(db + 1, 3)).astype(float)
        R = qz.bezout_matrix_poly(a, b, da, db)
        n = max(da, db)
        A = sum(int(a[i, j]) * u ** i * v ** j for i in range(da + 1) for j in range(3))
        B = sum(int(b[i, j]) * u ** i * v ** j for i in range(db + 1) for j in range(3))
        for vs in (sympy.Rational(1, 3), sympy.Rational(-2, 7), sympy.Rational(5, 4)):
            Av, Bv = sympy.Poly(A.subs(v, vs), u), sympy.Poly(B.subs(v, vs), u)
            res = sympy.resultant(Av, Bv, u)
            Mv = sympy.Matrix(n, n, lambda i, j: sum(sympy.Rational(int(R[k, i, j])) * vs ** k
                                                     for k in range(R.shape[0])))
            det = Mv.det()
            # the Bezout determinant of u-degrees (m, n) is +-lc(b)^(n-m) Res
            lcb = Bv.LC() if Bv.degree() == n else 0
            m = min(da, db)
            factor = lcb ** (n - m) if da < db else 1
            assert det == res * factor or det == -res * factor, (da, db, vs, det, res)


def test_qz_tt_flat_slab_matches_fermat():
    from .test_tt_oracle import _fermat
    rng = np.random.default_rng(5)
    P1 = np.array([[-1.0, -1.0, 0.0], [1.5, -1.0, 0.0], [-1.0, 1.5, 0.0]])
    P2 = P1 + [0.0, 0.0, -0.3]
    N = np.tile([0.0, 0.0, 1.0], (3, 1))
    pieces = tt.fit_sqrt_pieces()
    n_in = 0
    for _ in range(5):
        x0 = np.array([0.2, 0.1, 2.0]) + rng.normal(size=3) * 0.2
        x3 = np.array([0.0, 0.0, -1.0]) + rng.normal(size=3) * 0.3
        want = _fermat(x0, x3, (1.0, 1.5, 1.0), P1, P2)
        got = tt.solve_candidate(x0, x3, (1.0, 1.5, 1.0), P1, N, P2, N, pieces, v_solver="qz")
        inside = min(want[0], want[1], 1 - want[0] - want[1], want[2], want[3], 1 - want[2] - want[3]) > 1e-6
        if inside:
            n_in += 1
            assert len(got) == 1
            np.testing.assert_allclose(got[0]["uv"], want, atol=1e-7)
        else:
            assert not got
    assert n_in >= 2


def test_qz_rr_planted_corridor_paths():
    from .test_rr_oracle import planted_corridor_cases
    from paper_2405_13409_gb300 import scenes
    c = scenes.corridor_scene(seed=0, n_cells=16, n_recv=2)
    T = c.tri
    for x0, x3, t1, t2, w in planted_corridor_cases(41, 6):
        P1 = np.stack([T[0:3, t1], T[3:6, t1], T[6:9, t1]])
        N1 = np.stack([T[9:12, t1], T[12:15, t1], T[15:18, t1]])
        P2 = np.stack([T[0:3, t2], T[3:6, t2], T[6:9, t2]])
        N2 = np.stack([T[9:12, t2], T[12:15, t2], T[15:18, t2]])
        got = rr.solve_candidate(x0, x3, P1, N1, P2, N2, v_solver="qz")
        assert any(np.max(np.abs(p["uv"] - w)) < 1e-9 for p in got), (w, [p["uv"] for p in got])
