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
