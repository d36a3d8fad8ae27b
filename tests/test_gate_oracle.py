"""Pins of the gate oracle (features, BF16 network, loss, gradient, Adam)
against closed forms, finite differences and invariances."""
import numpy as np
import pytest

from oracle import gate as G


def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


# ------------------------------------------------------------------ BF16
def test_bf16_rounding_known_values():
    u = 2.0 ** -7  # BF16 spacing just above 1
    x = np.array([1.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2.0 ** -20, -(1 + 3 * u / 2), 3.0, 0.0, 2.0 ** -130])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 3.0, 0.0, 2.0 ** -130])
    np.testing.assert_array_equal(G.bf16(x), want)


def test_bf16_error_bound():
    x = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10000)
    r = G.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))  # unit roundoff of an 8-bit significand


# --------------------------------------------------------------- network
def test_forward_closed_form_identity_network():
    th = np.zeros(G.N_PARAMS)
    W1 = np.zeros((G.N_IN, G.N_HID))
    W1[np.arange(24), np.arange(24)] = 1.0
    th[G.OFF_W1:G.OFF_B1] = W1.ravel()
    th[G.OFF_W2:G.OFF_B2] = np.eye(G.N_HID).ravel()
    th[G.OFF_W3:G.OFF_B3] = np.eye(G.N_HID).ravel()
    th[G.OFF_W4:G.OFF_B4] = 1.0
    th[G.OFF_B4] = -0.5
    f = np.random.default_rng(2).integers(-8, 9, size=(50, 24)) / 4.0  # exact in BF16
    z, _ = G.forward(th, f)
    np.testing.assert_array_equal(z, np.maximum(f, 0).sum(1) - 0.5)


def test_loss_closed_form_at_zero_logit():
    z = np.zeros(4)
    y = np.array([0, 1, 1, 0])
    assert G.loss(z, y, 3.0) == pytest.approx(np.log(2) * (1 + 3 + 3 + 1) / 4, rel=1e-14)


@pytest.mark.parametrize("quantize", [False, True])
def test_gradient_matches_finite_differences(quantize):
    """Central differences of the FP64 network's loss.  With quantize=True
    the perturbation is applied to b3, w4 and b4 only, where no rounding
    sits between the parameter and the loss."""
    rng = np.random.default_rng(3)
    th = rng.normal(size=G.N_PARAMS) * 0.3
    f = rng.normal(size=(40, 24))
    y = (rng.random(40) < 0.3).astype(float)
    L, g = G.grad(th, f, y, 2.5, quantize=quantize)
    assert L == pytest.approx(G.loss(G.forward(th, f, quantize)[0], y, 2.5), rel=1e-14)
    idx = rng.choice(G.N_PARAMS, 200, replace=False)
    if quantize:
        idx = np.arange(G.OFF_B3, G.N_PARAMS)
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (G.loss(G.forward(tp, f, quantize)[0], y, 2.5) - G.loss(G.forward(tm, f, quantize)[0], y, 2.5)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 2e-9, (i, fd, g[i])  # truncation + cancellation of the difference


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    th = rng.normal(size=10)
    g = rng.normal(size=10)
    t1, m, v = G.adam_step(th, np.zeros(10), np.zeros(10), g, 1, 1e-3)
    np.testing.assert_allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


# -------------------------------------------------------------- features
def _flat_cases(rng, n, size=2e-3):
    """Small flat triangles with one constant normal near the origin, the
    endpoints about two units above."""
    P = np.empty((n, 3, 3))
    N = np.empty((n, 3, 3))
    for k in range(n):
        c = rng.uniform(-0.3, 0.3, 3) * [1, 1, 0.1]
        nrm = G._unit(np.array([rng.normal() * 0.2, rng.normal() * 0.2, 1.0]))
        a = G._unit(np.cross(nrm, [1.0, 0.3, 0.0]))
        b = np.cross(nrm, a)
        pts = rng.uniform(-1, 1, (3, 2)) * size
        P[k] = c + pts[:, :1] * a + pts[:, 1:] * b
        N[k] = nrm
    return P, N


def _mirror_bary(x0, x2, P, n):
    """Closed form of the flat reflection: the segment from the mirror image
    of x0 to x2 meets the plane at the path vertex; its barycentric
    coordinates in the triangle."""
    n = n / np.linalg.norm(n)
    xm = x0 - 2 * np.dot(x0 - P[0], n) * n
    d = x2 - xm
    t = np.dot(P[0] - xm, n) / np.dot(d, n)
    x1 = xm + t * d
    A = np.stack([P[1] - P[0], P[2] - P[0]], 1)
    uv = np.linalg.lstsq(A, x1 - P[0], rcond=None)[0]
    return np.array([1 - uv.sum(), uv[0], uv[1]])


def test_flat_reflection_barycentrics_match_closed_form():
    rng = np.random.default_rng(5)
    n = 300
    P, N = _flat_cases(rng, n)
    x0 = np.tile([0.0, -2.0, 1.5], (n, 1)) + rng.normal(size=(n, 3)) * 0.1
    x2 = np.tile([1.0, 1.0, 2.0], (n, 1)) + rng.normal(size=(n, 3)) * 0.1
    # Normals tilted so the mirror point lands near the triangle: choose each
    # normal as the half vector at the centroid, perturbed by a fraction of
    # the triangle's angular size.
    for k in range(n):
        c = P[k].mean(0)
        h = G._unit(G._unit(x0[k] - c) + G._unit(x2[k] - c))
        nrm = G._unit(h + rng.normal(size=3) * 3e-4)
        a = G._unit(np.cross(nrm, [1.0, 0.3, 0.0]))
        b = np.cross(nrm, a)
        pts = rng.uniform(-1, 1, (3, 2)) * 2e-3
        P[k] = c + pts[:, :1] * a + pts[:, 1:] * b
        N[k] = nrm
    f = G.features(x0, x2, np.ones(n), np.ones(n), np.zeros(n, int), P, N)
    exact = np.array([_mirror_bary(x0[k], x2[k], P[k], N[k, 0]) for k in range(n)])
    # The features' affine model of the mismatch is exact to first order in
    # the triangle's angular size; compare where the root is near the
    # triangle (the error grows with the extrapolation distance).
    ok = ((exact > -0.5) & (exact < 1.5)).all(1) & (np.abs(f[:, 6:9].sum(1)) > 1e-3)
    assert ok.sum() > 100
    np.testing.assert_allclose(f[ok, 9:12], exact[ok], atol=2e-3)
    np.testing.assert_allclose(f[ok, 9:12].sum(1), 1.0, atol=1e-9)
    np.testing.assert_allclose(f[ok, 12], f[ok, 9:12].min(1))


def _snell_bary(x0, x2, P, n, e0, e1):
    """Flat refraction closed form: minimise the optical length
    e0 |x1 - x0| + e1 |x2 - x1| over the plane (Fermat; constant normal)."""
    from scipy.optimize import minimize
    A = np.stack([P[1] - P[0], P[2] - P[0]], 1)

    def opl(uv):
        x1 = P[0] + A @ uv
        return e0 * np.linalg.norm(x1 - x0) + e1 * np.linalg.norm(x2 - x1)

    r = minimize(opl, np.array([1 / 3, 1 / 3]), method="Nelder-Mead",
                 options={"xatol": 1e-12, "fatol": 1e-16, "maxiter": 4000})
    return np.array([1 - r.x.sum(), r.x[0], r.x[1]])


def test_flat_refraction_barycentrics_match_fermat():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(6)
    n = 60
    x0 = np.tile([0.0, 0.0, 2.0], (n, 1)) + rng.normal(size=(n, 3)) * 0.2
    x2 = np.tile([0.0, 0.0, -1.0], (n, 1)) + rng.normal(size=(n, 3)) * 0.5
    P = np.empty((n, 3, 3))
    N = np.empty((n, 3, 3))
    e0, e1 = np.ones(n), np.full(n, 1.5)
    for k in range(n):
        c = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.0])
        h = G._unit(e0[k] * G._unit(x0[k] - c) + e1[k] * G._unit(x2[k] - c))
        nrm = G._unit(h + rng.normal(size=3) * 5e-4)
        a = G._unit(np.cross(nrm, [1.0, 0.3, 0.0]))
        b = np.cross(nrm, a)
        pts = rng.uniform(-1, 1, (3, 2)) * 2e-3
        P[k] = c + pts[:, :1] * a + pts[:, 1:] * b
        N[k] = nrm
    f = G.features(x0, x2, e0, e1, np.ones(n, int), P, N)
    exact = np.array([_snell_bary(x0[k], x2[k], P[k], N[k, 0], e0[k], e1[k]) for k in range(n)])
    ok = ((exact > -0.5) & (exact < 1.5)).all(1) & (np.abs(f[:, 6:9].sum(1)) > 1e-3)
    assert ok.sum() > 20
    np.testing.assert_allclose(f[ok, 9:12], exact[ok], atol=2e-3)
    assert np.all(f[:, 23] == 1.0)


def _random_curved(rng, n):
    P = rng.normal(size=(n, 3, 3)) * 0.01 + rng.normal(size=(n, 1, 3)) * [0.5, 0.5, 0.05]
    N = np.array([0, 0, 1.0]) + rng.normal(size=(n, 3, 3)) * 0.1
    x0 = rng.normal(size=(n, 3)) * 0.3 + [0, -2, 1.5]
    x2 = rng.normal(size=(n, 3)) * 0.3 + [1, 1, 2]
    return x0, x2, P, N


def test_features_rigid_motion_invariant():
    rng = np.random.default_rng(7)
    n = 200
    x0, x2, P, N = _random_curved(rng, n)
    f = G.features(x0, x2, np.ones(n), np.ones(n), np.zeros(n, int), P, N)
    R, t = _rot(rng), rng.normal(size=3)
    g = G.features(x0 @ R.T + t, x2 @ R.T + t, np.ones(n), np.ones(n), np.zeros(n, int), P @ R.T + t, N @ R.T)
    np.testing.assert_allclose(g, f, atol=1e-9)


def test_features_cyclic_vertex_permutation():
    """Relabelling (p0, p1, p2) -> (p1, p2, p0) permutes the barycentric
    features the same way and the cross products cyclically."""
    rng = np.random.default_rng(8)
    n = 200
    x0, x2, P, N = _random_curved(rng, n)
    f = G.features(x0, x2, np.ones(n), np.ones(n), np.zeros(n, int), P, N)
    perm = [1, 2, 0]
    g = G.features(x0, x2, np.ones(n), np.ones(n), np.zeros(n, int), P[:, perm], N[:, perm])
    np.testing.assert_allclose(g[:, 9:12], f[:, 9:12][:, perm], atol=1e-9)
    np.testing.assert_allclose(g[:, [6, 7, 8]], f[:, [7, 8, 6]], atol=1e-9)
    np.testing.assert_allclose(g[:, 12:15], f[:, 12:15], atol=1e-9)


def test_feature_ranges_and_centroid():
    rng = np.random.default_rng(9)
    n = 500
    x0, x2, P, N = _random_curved(rng, n)
    f = G.features(x0, x2, np.ones(n), np.ones(n), np.zeros(n, int), P, N)
    assert np.all(np.abs(f[:, 0:6]) <= 1 + 1e-12)
    assert np.all(np.max(np.abs(f[:, 0:6]).reshape(n, 3, 2) ** 2 @ [1, 1], -1) >= 0)
    np.testing.assert_allclose(np.hypot(f[:, 0:6:2], f[:, 1:6:2]).max(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(f[:, [15, 17, 19]].sum(1), 0, atol=1e-12)
    np.testing.assert_allclose(f[:, [16, 18, 20]].sum(1), 0, atol=1e-12)
    assert np.all((f[:, 14] >= 0) & (f[:, 14] <= 1 + 1e-12))
    assert np.all(np.abs(f[:, 9:13]) <= 4)
    assert np.all(f[:, 23] == 0)
