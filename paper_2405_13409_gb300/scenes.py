"""Seeded synthetic scene generators (inputs only).

This module produces the triangle meshes, endpoint queries and candidate
lists that both the CUDA path and the FP64 oracle consume.  It holds none of
the solver's arithmetic: no specular polynomial, resultant or root finding
lives here, only heightfield geometry, analytic normals and endpoint grids.

The scenes stand in for the paper's glint and caustic scenes (Sec. 5: brush,
relief, Plane, Pool), which are not available; they reproduce their shape:
curved triangles with interpolated vertex normals (Sec. 3.1, Eq. eq_xi and
eq_ni), a point light, and a grid of receivers or a pinhole camera.

Conventions shared by every generator
-------------------------------------
* Heightfield over [-1,1]^2 with (N+1)^2 vertices; vertex (i, j) sits at
  x = -1 + 2 i / N, y = -1 + 2 j / N.  Cell (i, j) is split into triangles
  (p00, p10, p11) and (p00, p11, p01), stored at index 2 (j N + i) + {0, 1}.
* Vertex normals are analytic, (-dz/dx, -dz/dy, 1) normalised; the solver
  interpolates them barycentrically (unnormalised, Eq. eq_ni).
* Mesh layout is SoA float64 of shape [18, T]: rows p0xyz, p1xyz, p2xyz,
  n0xyz, n1xyz, n2xyz.
* Receiver grids are inclusive linspaces over [-1.5, 1.5]^2.
* RNG is numpy.random.default_rng(seed); sinusoid parameters are drawn in
  the order a, f, g, p, q (four of each).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TYPE_R = 0
TYPE_T = 1


@dataclass
class Scene:
    """One solver workload: a mesh, endpoint queries and (optionally) chains.

    tri      float64 [18, T]  SoA triangle positions and vertex normals
    x_first  float64 [Q, 3]   separator x0 of each query
    x_last   float64 [Q, 3]   separator x_{k+1} of each query
    eta      float64 [Q, 3]   eta_0 .. eta_k (unused tail entries = 1)
    types    int32   [Q, 2]   scattering type per bounce (TYPE_R / TYPE_T)
    k        int32   [Q]      bounce count
    chains   int32   [C, 3]   explicit (query, tri0, tri1) list or None
    """

    name: str
    tri: np.ndarray
    x_first: np.ndarray
    x_last: np.ndarray
    eta: np.ndarray
    types: np.ndarray
    k: np.ndarray
    chains: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[1])

    @property
    def n_queries(self) -> int:
        return int(self.x_first.shape[0])


def _grid_vertices(n_cells: int):
    lin = np.linspace(-1.0, 1.0, n_cells + 1)
    xv, yv = np.meshgrid(lin, lin, indexing="xy")  # [j, i]
    return xv, yv


def heightfield_mesh(n_cells: int, z_fn, grad_fn, z_offset: float = 0.0) -> np.ndarray:
    """Triangulated heightfield with analytic vertex normals, SoA [18, T]."""
    xv, yv = _grid_vertices(n_cells)
    zv = z_fn(xv, yv) + z_offset
    gx, gy = grad_fn(xv, yv)
    nv = np.stack([-gx, -gy, np.ones_like(gx)], axis=-1)
    nv /= np.linalg.norm(nv, axis=-1, keepdims=True)
    pv = np.stack([xv, yv, zv], axis=-1)  # [j, i, 3]

    j, i = np.meshgrid(np.arange(n_cells), np.arange(n_cells), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    p00, p10, p11, p01 = pv[j, i], pv[j, i + 1], pv[j + 1, i + 1], pv[j + 1, i]
    n00, n10, n11, n01 = nv[j, i], nv[j, i + 1], nv[j + 1, i + 1], nv[j + 1, i]
    t = 2 * n_cells * n_cells
    tri = np.empty((18, t), dtype=np.float64)
    # triangle A = (p00, p10, p11) at even index, B = (p00, p11, p01) at odd index
    for slot, (a, b) in enumerate(((p00, p00), (p10, p11), (p11, p01))):
        tri[3 * slot:3 * slot + 3, 0::2] = a.T
        tri[3 * slot:3 * slot + 3, 1::2] = b.T
    for slot, (a, b) in enumerate(((n00, n00), (n10, n11), (n11, n01))):
        tri[9 + 3 * slot:9 + 3 * slot + 3, 0::2] = a.T
        tri[9 + 3 * slot:9 + 3 * slot + 3, 1::2] = b.T
    return tri


def sinusoid_params(seed: int):
    """Draw (a, f, g, p, q), four of each, in that order."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 1.0, 4)
    f = rng.uniform(1.0, 6.0, 4)
    g = rng.uniform(1.0, 6.0, 4)
    p = rng.uniform(0.0, 2.0 * math.pi, 4)
    q = rng.uniform(0.0, 2.0 * math.pi, 4)
    return a, f, g, p, q


def sinusoid_surface(seed: int, amplitude: float):
    """z = amplitude * sum_k a_k sin(f_k x + p_k) cos(g_k y + q_k) and its gradient."""
    a, f, g, p, q = sinusoid_params(seed)

    def z_fn(x, y):
        z = np.zeros_like(x)
        for k in range(4):
            z += a[k] * np.sin(f[k] * x + p[k]) * np.cos(g[k] * y + q[k])
        return amplitude * z

    def grad_fn(x, y):
        gx = np.zeros_like(x)
        gy = np.zeros_like(x)
        for k in range(4):
            gx += a[k] * f[k] * np.cos(f[k] * x + p[k]) * np.cos(g[k] * y + q[k])
            gy -= a[k] * g[k] * np.sin(f[k] * x + p[k]) * np.sin(g[k] * y + q[k])
        return amplitude * gx, amplitude * gy

    return z_fn, grad_fn


def receiver_grid(n: int, z: float, half: float = 1.5) -> np.ndarray:
    lin = np.linspace(-half, half, n)
    xr, yr = np.meshgrid(lin, lin, indexing="xy")
    return np.stack([xr.ravel(), yr.ravel(), np.full(n * n, z)], axis=-1)


def _queries(x_first, x_last, eta_row, types_row, k):
    q = x_last.shape[0]
    xf = np.broadcast_to(np.asarray(x_first, dtype=np.float64), (q, 3)).copy()
    eta = np.broadcast_to(np.asarray(eta_row, dtype=np.float64), (q, 3)).copy()
    types = np.broadcast_to(np.asarray(types_row, dtype=np.int32), (q, 2)).copy()
    kk = np.full(q, k, dtype=np.int32)
    return xf, np.ascontiguousarray(x_last, dtype=np.float64), eta, types, kk


def all_pairs(n_queries: int, n_tris: int) -> np.ndarray:
    """Exhaustive (query, tri, -1) list, triangle index fastest."""
    q = np.repeat(np.arange(n_queries, dtype=np.int32), n_tris)
    t = np.tile(np.arange(n_tris, dtype=np.int32), n_queries)
    return np.stack([q, t, np.full_like(t, -1)], axis=-1)


def reflect_scene(seed: int = 0, n_cells: int = 16, n_recv: int = 32) -> Scene:
    """1-bounce reflection: light (0.3,-0.2,2), 16x16-cell heightfield of
    amplitude 0.05, 32x32 receivers on z = 1, eta = 1, exhaustive pairs."""
    z_fn, grad_fn = sinusoid_surface(seed, 0.05)
    tri = heightfield_mesh(n_cells, z_fn, grad_fn)
    recv = receiver_grid(n_recv, 1.0)
    xf, xl, eta, types, k = _queries((0.3, -0.2, 2.0), recv, (1.0, 1.0, 1.0), (TYPE_R, TYPE_R), 1)
    return Scene("reflect_16x16_r32", tri, xf, xl, eta, types, k,
                 chains=all_pairs(recv.shape[0], tri.shape[1]),
                 meta={"seed": seed, "n_cells": n_cells, "n_recv": n_recv})


def refract_scene(seed: int = 0, n_cells: int = 64, n_recv: int = 256) -> Scene:
    """1-bounce refraction caustics: light (0,0,2), 64x64-cell heightfield of
    amplitude 0.08, glass below (eta 1 -> 1.5), 256x256 receivers on z = -1.
    Chains are left to the bounding-cone cull (chains = None)."""
    z_fn, grad_fn = sinusoid_surface(seed, 0.08)
    tri = heightfield_mesh(n_cells, z_fn, grad_fn)
    recv = receiver_grid(n_recv, -1.0)
    xf, xl, eta, types, k = _queries((0.0, 0.0, 2.0), recv, (1.0, 1.5, 1.0), (TYPE_T, TYPE_T), 1)
    return Scene("refract_64x64_r256", tri, xf, xl, eta, types, k, chains=None,
                 meta={"seed": seed, "n_cells": n_cells, "n_recv": n_recv})


def slab_scene(seed: int = 0, n_cells: int = 16, n_recv: int = 64, thickness: float = 0.3) -> Scene:
    """2-bounce TT slab: top heightfield (seed) at z = 0, bottom heightfield
    (seed + 1) at z = -0.3, both amplitude 0.05, eta = (1, 1.5, 1), light
    (0.2, 0.1, 2), 64x64 receivers on z = -1.  Triangles [0, T/2) are the top
    surface, [T/2, T) the bottom one.  Chains are left to the cone cull."""
    z1, g1 = sinusoid_surface(seed, 0.05)
    z2, g2 = sinusoid_surface(seed + 1, 0.05)
    top = heightfield_mesh(n_cells, z1, g1)
    bot = heightfield_mesh(n_cells, z2, g2, z_offset=-thickness)
    tri = np.concatenate([top, bot], axis=1)
    recv = receiver_grid(n_recv, -1.0)
    xf, xl, eta, types, k = _queries((0.2, 0.1, 2.0), recv, (1.0, 1.5, 1.0), (TYPE_T, TYPE_T), 2)
    return Scene("slab_tt_16x16_r64", tri, xf, xl, eta, types, k, chains=None,
                 meta={"seed": seed, "n_cells": n_cells, "n_recv": n_recv,
                       "top": (0, top.shape[1]), "bottom": (top.shape[1], tri.shape[1])})


def corridor_scene(seed: int = 0, n_cells: int = 16, n_recv: int = 16, height: float = 1.0) -> Scene:
    """2-bounce RR corridor between two mirrors: a floor heightfield (seed)
    at z = 0 with its normals up and a ceiling heightfield (seed + 1) at
    z = height with its normals turned down, both amplitude 0.05 over
    [-1, 1]^2; light (-0.6, 0.1, 0.5) between them; n_recv x n_recv
    receivers on z = 0.5 over [-0.8, 0.8]^2.  Triangles [0, T/2) are the
    floor, [T/2, T) the ceiling.  Chains are left to the caller."""
    z1, g1 = sinusoid_surface(seed, 0.05)
    z2, g2 = sinusoid_surface(seed + 1, 0.05)
    floor = heightfield_mesh(n_cells, z1, g1)
    ceil = heightfield_mesh(n_cells, z2, g2, z_offset=height)
    ceil[9:18] *= -1.0  # the ceiling reflects downwards
    tri = np.concatenate([floor, ceil], axis=1)
    recv = receiver_grid(n_recv, 0.5, half=0.8)
    xf, xl, eta, types, k = _queries((-0.6, 0.1, 0.5), recv, (1.0, 1.0, 1.0), (TYPE_R, TYPE_R), 2)
    return Scene(f"corridor_rr_{n_cells}x{n_cells}_r{n_recv}", tri, xf, xl, eta, types, k, chains=None,
                 meta={"seed": seed, "n_cells": n_cells, "n_recv": n_recv,
                       "floor": (0, floor.shape[1]), "ceiling": (floor.shape[1], tri.shape[1])})


def batched_scene(seed: int = 0, n_queries: int = 4096, c_min: float = 1e2, c_max: float = 1e5) -> Scene:
    """Batched mixed workload: independent queries with bounce count uniform
    in {1, 2} and candidate counts log-uniform in [c_min, c_max], each with
    its own geometry from the refraction or the slab generator (seed + 1 + q).

    1 bounce: the refraction heightfield (amplitude 0.08, eta 1 -> 1.5, light
    (0, 0, 2)) with max(64, ceil(sqrt(C / 2))) cells a side, so that it holds
    at least C triangles; the query's chains are C distinct triangles.
    2 bounces: the 16x16-cell slab (top at z = 0, bottom at z = -0.3, eta
    (1, 1.5, 1), light (0.2, 0.1, 2)); the chains are C distinct (top, bottom)
    pairs.  Receivers are uniform on z = -1 over [-1.5, 1.5]^2.  All meshes
    are concatenated; chains are grouped by query."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(1, 3, n_queries).astype(np.int32)
    counts = np.exp(rng.uniform(np.log(c_min), np.log(c_max), n_queries)).astype(np.int64)
    recv = np.column_stack([rng.uniform(-1.5, 1.5, (n_queries, 2)), np.full(n_queries, -1.0)])
    meshes, chains = [], []
    xf = np.empty((n_queries, 3))
    eta = np.tile(np.array([1.0, 1.5, 1.0]), (n_queries, 1))
    types = np.full((n_queries, 2), TYPE_T, dtype=np.int32)
    offset = 0
    for q in range(n_queries):
        qs = seed + 1 + q
        qrng = np.random.default_rng([seed, q])
        c = int(counts[q])
        if ks[q] == 1:
            n = max(64, int(math.ceil(math.sqrt(c / 2.0))))
            z_fn, grad_fn = sinusoid_surface(qs, 0.08)
            tri = heightfield_mesh(n, z_fn, grad_fn)
            t = qrng.choice(tri.shape[1], c, replace=False).astype(np.int64) + offset
            ch = np.column_stack([np.full(c, q), t, np.full(c, -1)])
            xf[q] = (0.0, 0.0, 2.0)
        else:
            z1, g1 = sinusoid_surface(qs, 0.05)
            z2, g2 = sinusoid_surface(qs + 1, 0.05)
            top = heightfield_mesh(16, z1, g1)
            bot = heightfield_mesh(16, z2, g2, z_offset=-0.3)
            tri = np.concatenate([top, bot], axis=1)
            nt = top.shape[1]
            pick = qrng.choice(nt * nt, c, replace=False).astype(np.int64)
            ch = np.column_stack([np.full(c, q), offset + pick // nt, offset + nt + pick % nt])
            xf[q] = (0.2, 0.1, 2.0)
        meshes.append(tri)
        chains.append(ch)
        offset += tri.shape[1]
    tri = np.ascontiguousarray(np.concatenate(meshes, axis=1))
    ch = np.concatenate(chains).astype(np.int32)
    return Scene(f"batched_{n_queries}", tri, xf, np.ascontiguousarray(recv), eta, types, ks, chains=ch,
                 meta={"seed": seed, "n_queries": n_queries, "counts": counts, "c_range": (c_min, c_max)})


def glint_surface(seed: int, n_terms: int = 64, n_cells: int = 1024):
    """Sum of random-phase plane waves of wavelength 2..20 cells, slope 0.02 each."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(2.0, 20.0, n_terms) * (2.0 / n_cells)
    theta = rng.uniform(0.0, 2.0 * math.pi, n_terms)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_terms)
    amp = 0.02 * lam / (2.0 * math.pi)
    kx = 2.0 * math.pi * np.cos(theta) / lam
    ky = 2.0 * math.pi * np.sin(theta) / lam

    def z_fn(x, y):
        z = np.zeros_like(x)
        for k in range(n_terms):
            z += amp[k] * np.sin(kx[k] * x + ky[k] * y + phi[k])
        return z

    def grad_fn(x, y):
        gx = np.zeros_like(x)
        gy = np.zeros_like(x)
        for k in range(n_terms):
            c = amp[k] * np.cos(kx[k] * x + ky[k] * y + phi[k])
            gx += c * kx[k]
            gy += c * ky[k]
        return gx, gy

    return z_fn, grad_fn, float(np.sum(amp))


@dataclass
class Camera:
    origin: np.ndarray
    target: np.ndarray
    up: np.ndarray
    vfov_deg: float
    width: int
    height: int

    def basis(self):
        fwd = self.target - self.origin
        fwd = fwd / np.linalg.norm(fwd)
        right = np.cross(fwd, self.up)
        right /= np.linalg.norm(right)
        upv = np.cross(right, fwd)
        return fwd, right, upv

    def as_array(self) -> np.ndarray:
        """float64 [16]: origin, forward, right, up, tan(vfov/2), aspect, width, height."""
        fwd, right, upv = self.basis()
        return np.concatenate([self.origin, fwd, right, upv,
                               [math.tan(math.radians(self.vfov_deg) / 2),
                                self.width / self.height, self.width, self.height]]).astype(np.float64)


def glint_scene(seed: int = 0, n_cells: int = 1024, res: int = 512, n_terms: int = 64) -> Scene:
    """Glints: 1024x1024-cell heightfield (2M triangles), pinhole camera at
    (0,-2,1.5) looking at the origin (up +z, vertical FOV 40 deg, 512x512),
    point light (1,1,2), reflection.  Each pixel is one query whose x0 is
    the pinhole and x_{k+1} the light; candidates come from the footprint
    grid builder."""
    z_fn, grad_fn, hmax = glint_surface(seed, n_terms, n_cells)
    tri = heightfield_mesh(n_cells, z_fn, grad_fn)
    cam = Camera(np.array([0.0, -2.0, 1.5]), np.zeros(3), np.array([0.0, 0.0, 1.0]), 40.0, res, res)
    q = res * res
    light = np.array([1.0, 1.0, 2.0])
    xl = np.broadcast_to(light, (q, 3)).copy()
    xf, xl, eta, types, k = _queries(cam.origin, xl, (1.0, 1.0, 1.0), (TYPE_R, TYPE_R), 1)
    return Scene("glints_1024_px512", tri, xf, xl, eta, types, k, chains=None,
                 meta={"seed": seed, "camera": cam, "hmax": hmax, "n_cells": n_cells})


def random_triangle_cases(seed: int, n: int, curved: bool = True, flat_normal: bool = False):
    """Tiny random single-triangle cases for pins: one triangle near the
    origin, x0 above and x2 at random positions.  Returns (tri [18, n],
    x0 [n, 3], x2 [n, 3])."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(-0.5, 0.5, (n, 3, 3))
    p[:, :, 2] *= 0.2
    if flat_normal:
        e1 = p[:, 1] - p[:, 0]
        e2 = p[:, 2] - p[:, 0]
        fn = np.cross(e1, e2)
        fn *= np.sign(fn[:, 2:3])
        fn /= np.linalg.norm(fn, axis=-1, keepdims=True)
        nrm = np.repeat(fn[:, None, :], 3, axis=1)
    else:
        nrm = rng.normal(0.0, 0.25 if curved else 0.0, (n, 3, 3))
        nrm[:, :, 2] += 1.0
        nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    tri = np.concatenate([p.reshape(n, 9), nrm.reshape(n, 9)], axis=1).T.copy()
    x0 = rng.uniform(-1.0, 1.0, (n, 3))
    x0[:, 2] = rng.uniform(0.8, 2.0, n)
    x2 = rng.uniform(-1.0, 1.0, (n, 3))
    x2[:, 2] = rng.uniform(0.8, 2.0, n)
    return tri, x0, x2
