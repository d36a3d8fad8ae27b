"""FP64 CPU oracle of the path phase's last two steps (TEST INFRASTRUCTURE):
the visibility test and the contribution of an admissible path (Sec. 4.3:
"conduct the visibility test ... evaluates its contribution"; Sec. 5.1,
glints), plus a glint image.

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; the
product path never does.  It shares no code with the CUDA library.

Visibility.  A path x0 -> x1 (-> x2) -> x_last is rejected when a segment
between consecutive vertices meets a triangle of the mesh strictly inside
it: ray parameter t in (eps, 1 - eps) with eps = 1e-9, where the segment's
own end triangles are excluded (reading: the paper states the test, not its
tolerance).  Brute force over every triangle (Moller-Trumbore in FP64).

Contribution.  The paper cites the generalised geometric term of specular
chains; its formula is not printed, so this module states a reading derived
from first principles: the contribution of an admissible path is the
irradiance at the camera point x0 from the point light (intensity I) at
x_last, carried through the chain.  The light emits I per unit solid angle;
a ray leaving it in direction omega_l(eps) = normalise(omega_l* + eps_a e_a
+ eps_b e_b) (omega_l* toward the chain's last vertex, e_a, e_b an
orthonormal basis perpendicular to it) is traced back through the planes of
the chain's triangles (interpolated normals; mirror reflection or Snell
refraction at each vertex) and leaves the first vertex y in direction
omega_out; it passes the camera at the transverse offset
|x0 - y| P_perp (omega_out - psi(y)), psi(y) the unit direction from y to
x0.  The irradiance is the emitted intensity over the area that a unit
solid angle of emission covers at the camera:

    f = rho I / ( |y - x0|^2 |det J| ),   J = d P_perp (omega_out - psi) / d eps,

with J by central differences (step 1e-6) and P_perp the two components
perpendicular to psi at the path.  rho = 1 (lossless interfaces; radiance
is invariant along the chain when eta_0 = eta_last).  The light is traced
outward rather than the camera ray backward because interpolated normals
make the ray map non-reciprocal: the two Jacobians differ, and the light's
emission is what reaches the camera.  For one flat mirror f reduces to
I / (|x0 - x1| + |x1 - x_last|)^2, the inverse square law of the light's
mirror image (the closed-form pin of this module); on curved triangles the
pins count a traced bundle of light rays at the camera.
"""
from __future__ import annotations

import numpy as np

EPS_T = 1e-9
FD_STEP = 1e-6


def _tri(T, t):
    T = np.asarray(T, float)
    return T[0:9, t].reshape(3, 3), T[9:18, t].reshape(3, 3)


def segment_hits(tri, a, b, exclude=()):
    """True when the segment a -> b meets a triangle (other than `exclude`)
    at a ray parameter strictly inside (EPS_T, 1 - EPS_T)."""
    T = np.asarray(tri, float)
    p0, p1, p2 = T[0:3].T, T[3:6].T, T[6:9].T
    d = np.asarray(b, float) - np.asarray(a, float)
    e1, e2 = p1 - p0, p2 - p0
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = np.asarray(a, float) - p0
    u = np.einsum("ij,ij->i", s, pv) * inv
    q = np.cross(s, e1)
    v = (q @ d) * inv
    t = np.einsum("ij,ij->i", e2, q) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > EPS_T) & (t < 1.0 - EPS_T)
    for e in exclude:
        if e >= 0:
            hit[e] = False
    return bool(np.any(hit))


def path_visible(tri, x0, verts, x_last, tris):
    """Visibility of x0 -> verts[0] (-> verts[1]) -> x_last; tris are the
    chain's triangle indices (each segment excludes its end triangles)."""
    pts = [np.asarray(x0, float)] + [np.asarray(v, float) for v in verts] + [np.asarray(x_last, float)]
    ends = [-1] + list(tris) + [-1]
    for i in range(len(pts) - 1):
        if segment_hits(tri, pts[i], pts[i + 1], exclude=(ends[i], ends[i + 1])):
            return False
    return True


def _unit(x):
    return x / np.linalg.norm(x)


def _scatter(w, n, typ, eta_in, eta_out):
    """Outgoing unit direction at a vertex with unit normal n (mirror
    reflection, or Snell refraction from eta_in to eta_out); None on total
    internal reflection."""
    if typ == 0:
        return w - 2.0 * (w @ n) * n
    if w @ n > 0:
        n = -n  # normal against the incident direction
    c = -(w @ n)
    r = eta_in / eta_out
    k = 1.0 - r * r * (1.0 - c * c)
    if k < 0:
        return None
    return r * w + (r * c - np.sqrt(k)) * n


def trace(tri, x0, w, tris, types, etas):
    """Traces the ray x0 + t w through the planes of the chain's triangles
    (barycentric extension beyond their edges).  Returns (last point, last
    direction) or None."""
    y, d = np.asarray(x0, float), _unit(np.asarray(w, float))
    for i, t in enumerate(tris):
        P, N = _tri(tri, t)
        e1, e2 = P[1] - P[0], P[2] - P[0]
        nrm = np.cross(e1, e2)
        den = d @ nrm
        if abs(den) < 1e-300:
            return None
        s = ((P[0] - y) @ nrm) / den
        y = y + s * d
        # barycentrics of y in the triangle's plane
        g = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
        rhs = np.array([(y - P[0]) @ e1, (y - P[0]) @ e2])
        u, v = np.linalg.solve(g, rhs)
        n = _unit(N[0] + u * (N[1] - N[0]) + v * (N[2] - N[0]))
        d = _scatter(d, n, int(types[i]), etas[i], etas[i + 1])
        if d is None:
            return None
        d = _unit(d)
    return y, d


def _perp_basis(w):
    a = np.cross(w, [1.0, 0.0, 0.0] if abs(w[0]) < 0.9 else [0.0, 1.0, 0.0])
    a = _unit(a)
    return a, np.cross(w, a)


def contribution(tri, x0, verts, x_last, tris, types, etas, intensity=1.0):
    """f = I / (|y - x0|^2 |det J|) of one admissible path x0 -> verts ->
    x_last (module docstring): the light at x_last traced back through the
    chain to the camera x0.  etas are eta_0 .. eta_k from the camera side;
    NaN when the traced perturbations fail."""
    x0, x_last = np.asarray(x0, float), np.asarray(x_last, float)
    rtris, rtypes, retas = list(tris)[::-1], list(types)[::-1], list(etas)[::-1]
    wl = _unit(np.asarray(verts[-1], float) - x_last)
    ea, eb = _perp_basis(wl)
    y_star = np.asarray(verts[0], float)
    psi = _unit(x0 - y_star)
    pa, pb = _perp_basis(psi)

    def F(da, db):
        r = trace(tri, x_last, wl + da * ea + db * eb, rtris, rtypes, retas)
        if r is None:
            return None
        y, d = r
        diff = d - _unit(x0 - y)
        return np.array([diff @ pa, diff @ pb])

    cols = []
    for da, db in ((FD_STEP, 0.0), (0.0, FD_STEP)):
        fp, fm = F(da, db), F(-da, -db)
        if fp is None or fm is None:
            return float("nan")
        cols.append((fp - fm) / (2.0 * FD_STEP))
    det = abs(np.linalg.det(np.stack(cols, 1)))
    if not det > 0:
        return float("nan")
    return float(intensity / ((y_star - x0) @ (y_star - x0)) / det)


def path_terms(tri, x_first, x_last, eta, types, paths, intensity=1.0, check_visibility=True):
    """Visibility (bool) and contribution (FP64) of every path of a
    PATH_DTYPE array (1 bounce: tri1 < 0)."""
    vis = np.ones(paths.size, bool)
    f = np.zeros(paths.size)
    for i, p in enumerate(paths):
        q = int(p["query"])
        k2 = int(p["tri1"]) >= 0
        tris = [int(p["tri0"])] + ([int(p["tri1"])] if k2 else [])
        verts = [p["x"][:3]] + ([p["x"][3:]] if k2 else [])
        tys = [int(types[q][0])] + ([int(types[q][1])] if k2 else [])
        et = [float(e) for e in eta[q][:len(tris) + 1]]
        if check_visibility:
            vis[i] = path_visible(tri, x_first[q], verts, x_last[q], tris)
        f[i] = contribution(tri, x_first[q], verts, x_last[q], tris, tys, et, intensity)
    return vis, f


def glint_image(paths, f, vis, width, height):
    """Sum of the contributions of the visible paths per pixel (a path's
    query is its pixel)."""
    img = np.zeros(width * height)
    q = paths["query"].astype(np.int64)
    np.add.at(img, q[vis], f[vis])
    return img.reshape(height, width)
