"""Path-set comparison between the CUDA library and the FP64 oracle.

Solutions are matched by candidate key (query, tri0); within a key they are
paired greedily by the smallest max-norm distance over (u, v), accepted when
<= tol (1e-5: the solution tolerance the method is held to).  A solution
left unpaired is allowed only if the side that reports it flags it
ILL_COND or EDGE; their number must stay <= 1e-4 of the candidates.
"""
from collections import defaultdict

import numpy as np

FLAG_ILL_COND = 1
FLAG_EDGE = 2
ALLOWED = FLAG_ILL_COND | FLAG_EDGE


def _group(keys, uv, flags):
    g = defaultdict(list)
    for k, x, f in zip(keys, uv, flags):
        g[k].append((x, f))
    return g


def compare(gpu, ref, tol=1e-5):
    """gpu: binding.PATH_DTYPE array; ref: oracle.PATH_DTYPE array."""
    gk = list(zip(gpu["query"].tolist(), gpu["tri"][:, 0].tolist()))
    rk = list(zip(ref["query"].tolist(), ref["tri0"].tolist()))
    G = _group(gk, gpu["uv"][:, :2], gpu["flags"].tolist())
    R = _group(rk, ref["uv"][:, :2], ref["flags"].tolist())
    errs = []
    st = dict(matched=0, gpu_only_flagged=0, gpu_only_unflagged=0, ref_only_flagged=0, ref_only_unflagged=0)
    bad = []
    for key in set(G) | set(R):
        a = list(G.get(key, []))
        b = list(R.get(key, []))
        pairs = []
        for i, (x, _) in enumerate(a):
            for j, (y, _) in enumerate(b):
                pairs.append((float(np.max(np.abs(x - y))), i, j))
        pairs.sort()
        ua, ub = set(range(len(a))), set(range(len(b)))
        for d, i, j in pairs:
            if d > tol:
                break
            if i in ua and j in ub:
                ua.discard(i)
                ub.discard(j)
                errs.append(d)
                st["matched"] += 1
        for i in ua:
            if a[i][1] & ALLOWED:
                st["gpu_only_flagged"] += 1
            else:
                st["gpu_only_unflagged"] += 1
                bad.append(("gpu", key, a[i][0].tolist(), a[i][1]))
        for j in ub:
            if b[j][1] & ALLOWED:
                st["ref_only_flagged"] += 1
            else:
                st["ref_only_unflagged"] += 1
                bad.append(("ref", key, b[j][0].tolist(), b[j][1]))
    e = np.array(errs) if errs else np.zeros(1)
    st["max_err"] = float(e.max())
    st["p99_err"] = float(np.quantile(e, 0.99))
    st["bad"] = bad[:20]
    return st


def assert_parity(gpu, ref, n_candidates, tol=1e-5, min_recall=1.0, max_flagged_frac=1e-4):
    """min_recall < 1 allows that fraction of the reference's unflagged paths
    to be missing (mixed precision on inputs outside its accuracy range); the
    GPU may never report an unflagged path the reference lacks."""
    st = compare(gpu, ref, tol)
    assert st["gpu_only_unflagged"] == 0, st
    assert st["ref_only_unflagged"] <= (1.0 - min_recall) * max(1, ref.size), st
    flagged = st["gpu_only_flagged"] + st["ref_only_flagged"]
    assert flagged <= max(1, max_flagged_frac * n_candidates), st
    return st


# Pixel-footprint helpers for the glint tests (numpy, independent of the library).
def project_pixels(cam, x):
    o, f, r, u = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    th, asp, w, h = cam[12], cam[13], int(cam[14]), int(cam[15])
    d = x - o
    fz = d @ f
    sx = (d @ r) / (fz * th * asp)
    sy = (d @ u) / (fz * th)
    fx = (sx + 1) * 0.5 * w
    fy = (1 - sy) * 0.5 * h
    ok = (fz > 0) & (fx >= 0) & (fx < w) & (fy >= 0) & (fy < h)
    pix = np.floor(fy).astype(np.int64) * w + np.floor(fx).astype(np.int64)
    return np.where(ok, pix, -1)


def footprint_boxes(s, cam, qs):
    """Footprint box (xl, xh, yl, yh) of each pixel in qs: the xy box of its
    four corner rays between the mesh's z bounds (FP32-rounded, as the
    library takes them), with a 1e-5 relative margin; None where a corner
    ray never descends."""
    T = s.tri
    zs = T[[2, 5, 8]]
    zlo, zhi = float(np.float32(zs.min())), float(np.float32(zs.max()))
    o, f, r, u = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    th, asp, w, h = cam[12], cam[13], int(cam[14]), int(cam[15])
    out = []
    for q in qs:
        ix, iy = int(q) % w, int(q) // w
        pts = []
        for k in range(4):
            sx = -1 + 2 * (ix + (k & 1)) / w
            sy = 1 - 2 * (iy + (k >> 1)) / h
            d = f + sx * th * asp * r + sy * th * u
            if d[2] >= 0:
                pts = None
                break
            for z in (zlo, zhi):
                t = (z - o[2]) / d[2]
                pts.append(o + t * d)
        if pts is None:
            out.append(None)
            continue
        pts = np.array(pts)
        m = 1e-5 * (1 + max(abs(pts[:, 0].min()), abs(pts[:, 1].max())))
        out.append((pts[:, 0].min() - m, pts[:, 0].max() + m, pts[:, 1].min() - m, pts[:, 1].max() + m))
    return out


def footprint_numpy(s, cam):
    """Brute force: triangles whose xy bbox meets each pixel's footprint box."""
    T = s.tri
    xs, ys = T[[0, 3, 6]], T[[1, 4, 7]]
    txl, txh, tyl, tyh = xs.min(0), xs.max(0), ys.min(0), ys.max(0)
    w, h = int(cam[14]), int(cam[15])
    out = set()
    for q, b in enumerate(footprint_boxes(s, cam, range(w * h))):
        if b is None:
            continue
        xl, xh, yl, yh = b
        hit = np.where(~((txh < xl) | (txl > xh) | (tyh < yl) | (tyl > yh)))[0]
        out.update((q, int(t)) for t in hit)
    return out
