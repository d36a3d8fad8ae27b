"""Pins of the visibility and contribution oracle (oracle/render.py; the
path phase's last steps, Sec. 4.3): the flat-mirror contribution equals the
inverse square law of the light's mirror image (closed form), curved
reflections and a flat refraction match the irradiance counted with traced
bundles of light rays, and the brute-force visibility test
sees a planted blocker and ignores the path's own triangles."""
import numpy as np
import pytest

import oracle
from oracle import render


def _mirror_tri(n=(0.0, 0.0, 1.0)):
    tri = np.zeros((18, 1))
    P = np.array([[-2.0, -2.0, 0.0], [3.0, -2.0, 0.0], [-2.0, 3.0, 0.0]])
    tri[0:9, 0] = P.ravel()
    tri[9:18, 0] = np.tile(n, 3)
    return tri, P


def test_flat_mirror_is_the_inverse_square_law_of_the_image():
    tri, P = _mirror_tri()
    rng = np.random.default_rng(1)
    for _ in range(20):
        x0 = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(0.5, 2.0)])
        xl = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(0.5, 2.0)])
        img = xl * [1, 1, -1]
        t = x0[2] / (x0[2] - img[2])
        x1 = x0 + t * (img - x0)
        f = render.contribution(tri, x0, [x1], xl, [0], [0], [1.0, 1.0], intensity=2.5)
        L = np.linalg.norm(x1 - x0) + np.linalg.norm(xl - x1)
        assert abs(f - 2.5 / L ** 2) <= 1e-6 * 2.5 / L ** 2, (f, 2.5 / L ** 2)


def _bundle_density(tri, t, x0, xl, x1, r=1e-3):
    """Irradiance at x0 from a unit point light at xl reflected by triangle t
    (interpolated normals), counted with a bundle of light rays: rays from
    the light through a grid of points on the triangle's plane around x1,
    mirror-reflected, counted where they cross a disc of radius r around x0
    perpendicular to the camera ray; a coarse grid finds the disc's
    pre-image and a fine 400 x 400 grid over it counts."""
    T = np.asarray(tri, float)[:, t]
    P, N = T[0:9].reshape(3, 3), T[9:18].reshape(3, 3)
    e1, e2 = P[1] - P[0], P[2] - P[0]
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm)
    a = e1 / np.linalg.norm(e1)
    b = np.cross(nrm, a)
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    axis = (x0 - x1) / np.linalg.norm(x0 - x1)

    def shoot(U, V):
        pts = x1 + U[:, None] * a + V[:, None] * b
        uv = np.linalg.solve(G, np.stack([(pts - P[0]) @ e1, (pts - P[0]) @ e2], 0))
        nn = N[0] + uv[0][:, None] * (N[1] - N[0]) + uv[1][:, None] * (N[2] - N[0])
        nn /= np.linalg.norm(nn, axis=1)[:, None]
        d_in = pts - xl
        dist = np.linalg.norm(d_in, axis=1)
        w_in = d_in / dist[:, None]
        dom = np.abs(w_in @ nrm) / dist ** 2  # solid angle per unit plane area
        w_out = w_in - 2.0 * np.sum(w_in * nn, 1)[:, None] * nn
        tt = ((x0 - pts) @ axis) / (w_out @ axis)
        hit = pts + tt[:, None] * w_out
        rad = np.linalg.norm(hit - x0 - ((hit - x0) @ axis)[:, None] * axis, axis=1)
        return rad < r, dom

    g = np.linspace(-80 * r, 80 * r, 801)
    U, V = (m.ravel() for m in np.meshgrid(g, g, indexing="ij"))
    inside, _ = shoot(U, V)
    assert inside.sum() >= 1
    h0 = g[1] - g[0]
    u0, u1 = U[inside].min() - 2 * h0, U[inside].max() + 2 * h0
    v0, v1 = V[inside].min() - 2 * h0, V[inside].max() + 2 * h0
    gu, gv = np.linspace(u0, u1, 400), np.linspace(v0, v1, 400)
    U, V = (m.ravel() for m in np.meshgrid(gu, gv, indexing="ij"))
    inside, dom = shoot(U, V)
    area = (gu[1] - gu[0]) * (gv[1] - gv[0])
    return np.sum(dom[inside]) * area / (np.pi * r * r)


def test_curved_reflection_matches_a_ray_bundle_count():
    """On curved triangles (interpolated normals) the contribution equals
    the irradiance counted with a traced bundle of light rays, an estimate
    that does not use the Jacobian; paths from the C++ oracle's solve of
    planted reflection cases."""
    from tests.test_oracle_pins import _planted_cases
    tri, x0, x2 = _planted_cases(5, 40, 0)
    n = tri.shape[1]
    chains = np.stack([np.arange(n), np.arange(n), -np.ones(n)], -1).astype(np.int32)
    ref, _ = oracle.solve(tri, x0, x2, np.ones((n, 3)), np.zeros((n, 2), np.int32), np.ones(n, np.int32), chains)
    assert ref.size >= 8
    for p in ref[:8]:
        q, t = int(p["query"]), int(p["tri0"])
        f = render.contribution(tri, x0[q], [p["x"][:3]], x2[q], [t], [0], [1.0, 1.0])
        est = _bundle_density(tri, t, x0[q], x2[q], p["x"][:3])
        assert abs(est - f) <= 0.03 * f, (q, est, f)


def test_flat_refraction_matches_a_ray_bundle_count():
    """Refraction through a flat interface: the contribution equals the
    density of a traced bundle of light rays at the camera (rays from the
    light through a fine grid of interface points, refracted by Snell's law,
    counted in a small disc around the camera), an estimate independent of
    the Jacobian."""
    tri, P = _mirror_tri()
    x0 = np.array([0.1, 0.05, -0.8])  # camera below the interface (in glass)
    xl = np.array([-0.2, 0.1, 1.0])   # light above it
    etas = [1.5, 1.0]                 # camera side eta0 = 1.5, light side 1.0
    # the refraction path by 1D search on the plane of incidence
    from scipy.optimize import minimize
    opl = lambda w: 1.5 * np.linalg.norm([w[0], w[1], 0] - x0) + np.linalg.norm(xl - [w[0], w[1], 0])
    w = minimize(opl, [0.0, 0.0], method="BFGS", options={"gtol": 1e-12}).x
    x1 = np.array([w[0], w[1], 0.0])
    f = render.contribution(tri, x0, [x1], xl, [0], [1], etas)
    # bundle: light rays through interface points near x1, refracted into the
    # glass; count the flux through a disc of radius r around the camera,
    # per unit solid angle of emission and per disc area
    r = 2e-3
    h = 2e-4
    g = np.arange(-60, 61) * h
    X, Y = np.meshgrid(x1[0] + g, x1[1] + g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], -1)
    d_in = pts - xl
    dist = np.linalg.norm(d_in, axis=1)
    w_in = d_in / dist[:, None]
    # solid angle of each grid point seen from the light: dA cos / dist^2
    dom = h * h * np.abs(w_in[:, 2]) / dist ** 2
    n = np.array([0.0, 0.0, 1.0])
    c = -(w_in @ n)
    eta = 1.0 / 1.5
    k = 1.0 - eta ** 2 * (1.0 - c ** 2)
    w_out = eta * w_in + (eta * c - np.sqrt(k))[:, None] * n
    # where each refracted ray crosses the plane perpendicular to the camera ray at x0
    axis = (x0 - x1) / np.linalg.norm(x0 - x1)
    t = ((x0 - pts) @ axis) / (w_out @ axis)
    hit = pts + t[:, None] * w_out
    inside = np.linalg.norm(hit - x0 - ((hit - x0) @ axis)[:, None] * axis, axis=1) < r
    flux = np.sum(dom[inside])  # light intensity 1: flux = emitted solid angle
    est = flux / (np.pi * r * r)
    assert abs(est - f) <= 0.03 * f, (est, f)


def test_visibility_sees_a_blocker_and_ignores_own_triangles():
    tri, P = _mirror_tri()
    x0 = np.array([0.0, 0.0, 1.0])
    xl = np.array([0.4, 0.0, 1.0])
    x1 = np.array([0.2, 0.0, 0.0])
    assert render.path_visible(tri, x0, [x1], xl, [0])
    blocker = np.zeros((18, 1))
    B = np.array([[-0.1, -0.3, 0.5], [0.4, -0.3, 0.5], [-0.1, 0.4, 0.5]])  # across the segment x0 -> x1
    blocker[0:9, 0] = B.ravel()
    blocker[9:18, 0] = np.tile([0.0, 0.0, 1.0], 3)
    both = np.concatenate([tri, blocker], 1)
    assert not render.path_visible(both, x0, [x1], xl, [0])
    # the same blocker moved off the segments does not block
    both[[0, 3, 6], 1] += 2.0
    assert render.path_visible(both, x0, [x1], xl, [0])
