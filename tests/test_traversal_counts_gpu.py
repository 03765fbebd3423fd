"""The work counters behind the traversal roofline, checked against an
independent count.

bench.py turns the kernels' node-visit and triangle-test counters into
algorithmic bytes.  Here a plain numpy walk of the node layout that
rp_bvh_build_host returns (the builder rp_scene_create uses) traces the same
rays in the kernel's order -- both child boxes of a node tested, a hit leaf's
triangles tested at once, the nearer inner child visited next and the other
pushed -- and counts every node visit and triangle test.  The device may
contract some FP32 products into fused multiply-adds, which can tip a box or
triangle test that sits on its boundary, so the totals must agree within
0.5 % and each ray's counts exactly for at least 98 % of the rays.  The
dynamic object is moved far outside the scene, so its BVH is culled by the
bounding-sphere test for every ray and only the static BVH is counted."""
import numpy as np
import pytest

from paper_2406_16302_gb300 import scenes as S

pytestmark = pytest.mark.gpu

F = np.float32


def _ints(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _rcp(x):
    x = F(x)
    if abs(x) < F(1e-20):
        x = F(np.copysign(F(1e-20), x))
    return F(1.0) / x


def _box(lo, hi, idv, oid, tmin, tmax):
    t0 = [_fma(lo[k], idv[k], -oid[k]) for k in range(3)]
    t1 = [_fma(hi[k], idv[k], -oid[k]) for k in range(3)]
    a = max(max(min(t0[0], t1[0]), min(t0[1], t1[1])), max(min(t0[2], t1[2]), tmin))
    b = min(min(max(t0[0], t1[0]), max(t0[1], t1[1])), min(max(t0[2], t1[2]), tmax))
    return a <= F(b * F(1.00000024)), a


def _setup(d):
    ad = np.abs(d)
    kz = (0 if ad[0] > ad[2] else 2) if ad[0] > ad[1] else (1 if ad[1] > ad[2] else 2)
    kx = 0 if kz == 2 else kz + 1
    ky = 0 if kx == 2 else kx + 1
    if d[kz] < 0:
        kx, ky = ky, kx
    return kx, ky, kz, F(d[kx] / d[kz]), F(d[ky] / d[kz]), F(F(1.0) / d[kz])


def _tri(w, o, v0, v1, v2, tmin, tmax):
    kx, ky, kz, Sx, Sy, Sz = w
    A, B, C = (v0 - o).astype(F), (v1 - o).astype(F), (v2 - o).astype(F)
    Ax, Ay = F(A[kx] - F(Sx * A[kz])), F(A[ky] - F(Sy * A[kz]))
    Bx, By = F(B[kx] - F(Sx * B[kz])), F(B[ky] - F(Sy * B[kz]))
    Cx, Cy = F(C[kx] - F(Sx * C[kz])), F(C[ky] - F(Sy * C[kz]))
    U, V, W = F(F(Cx * By) - F(Cy * Bx)), F(F(Ax * Cy) - F(Ay * Cx)), F(F(Bx * Ay) - F(By * Ax))
    if U == 0 or V == 0 or W == 0:
        U = F(np.float64(Cx) * np.float64(By) - np.float64(Cy) * np.float64(Bx))
        V = F(np.float64(Ax) * np.float64(Cy) - np.float64(Ay) * np.float64(Cx))
        W = F(np.float64(Bx) * np.float64(Ay) - np.float64(By) * np.float64(Ax))
    if (U < 0 or V < 0 or W < 0) and (U > 0 or V > 0 or W > 0):
        return None
    det = F(F(U + V) + W)
    if det == 0:
        return None
    T = F(F(F(U * F(Sz * A[kz])) + F(V * F(Sz * B[kz]))) + F(W * F(Sz * C[kz])))
    tt = F(T * F(F(1.0) / det))
    return tt if tmin < tt < tmax else None


def count_walk(bvh, o, d):
    """(node visits, triangle tests) of one closest-hit ray, tmin 0."""
    nodes, tris = bvh["nodes"], bvh["tris"]
    di = _ints(nodes[:, 12:16])
    o, d = o.astype(F), d.astype(F)
    idv = np.array([_rcp(d[0]), _rcp(d[1]), _rcp(d[2])], F)
    oid = (o * idv).astype(F)
    w = _setup(d)
    tmin, tmax = F(0.0), F(np.inf)
    nv = nt = 0
    node, stack = 0, []
    while True:
        nv += 1
        n = nodes[node]
        h0, t0 = _box(n[[0, 2, 8]], n[[1, 3, 9]], idv, oid, tmin, tmax)
        h1, t1 = _box(n[[4, 6, 10]], n[[5, 7, 11]], idv, oid, tmin, tmax)
        c0, c1 = di[node, 0], di[node, 1]
        for hs, cs, cnt in ((h0, c0, di[node, 2]), (h1, c1, di[node, 3])):
            if not hs or cs >= 0:
                continue
            for i in range(~cs, ~cs + cnt):
                nt += 1
                t = tris[i]
                tt = _tri(w, o, t[0:3], t[4:7], t[8:11], tmin, tmax)
                if tt is not None:
                    tmax = tt
        g0, g1 = h0 and c0 >= 0, h1 and c1 >= 0
        if g0 and g1:
            near, far = (c1, c0) if t1 < t0 else (c0, c1)
            stack.append(far)
            node = near
        elif g0:
            node = c0
        elif g1:
            node = c1
        elif stack:
            node = stack.pop()
        else:
            return nv, nt


@pytest.mark.parametrize("case", ["box_blob", "terrain"])
def test_node_and_triangle_counts_match_an_independent_walk(case):
    """The box scene (about 1.3k static triangles) and the terrain (about
    1.16M): rays from random points of the static scene's bounding box in
    random directions."""
    import torch
    from paper_2406_16302_gb300 import build, rp
    build.build()
    if case == "box_blob":
        scene, edit = S.cfg2_box_blob(width=16, height=16, blob_level=4)
    else:
        scene, edit = S.cfg3_terrain(width=16, height=16)
    far = edit.M1.copy()
    far[:, 3] += np.array([100.0, 0.0, 0.0], dtype=far.dtype)
    edit.M1, edit.M2 = far, far.copy()
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    bvh = rp.rp_bvh_build_host(scene.static_vertices, np.asarray(scene.static_triangles, np.uint32))
    lo = scene.static_vertices.min(0)
    hi = scene.static_vertices.max(0)
    rng = np.random.default_rng(21)
    n = 1500
    o = (lo + (hi - lo) * rng.uniform(0.02, 0.98, size=(n, 3))).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    t = torch.zeros(n, device="cuda")
    prim = torch.zeros(n, dtype=torch.int32, device="cuda")
    b1 = torch.zeros(n, device="cuda")
    b2 = torch.zeros(n, device="cuda")
    per_ray = []
    rp.rp_enable_stats(sc, True)
    # one launch per ray for the per-ray counts, then all rays in one launch
    for i in range(0, n, 10):
        rp.rp_trace_closest(sc, ed, 1, torch.from_numpy(o[i:i + 1]).cuda(),
                            torch.from_numpy(d[i:i + 1]).cuda(), t[:1], prim[:1], b1[:1], b2[:1])
        st = rp.rp_get_stats(sc)
        per_ray.append((st["nodes_closest"], st["tris_closest"]))
    rp.rp_trace_closest(sc, ed, 1, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                        t, prim, b1, b2)
    st = rp.rp_get_stats(sc)
    rp.rp_enable_stats(sc, False)
    assert st["rays_closest"] == n
    walks = [count_walk(bvh, o[i], d[i]) for i in range(n)]
    nv = sum(w[0] for w in walks)
    nt = sum(w[1] for w in walks)
    print(case, "kernel", st["nodes_closest"], st["tris_closest"], "walk", nv, nt)
    assert nv >= 5 * n
    assert abs(st["nodes_closest"] - nv) <= 0.005 * nv
    assert abs(st["tris_closest"] - nt) <= 0.005 * nt
    same = [per_ray[k] == walks[10 * k] for k in range(len(per_ray))]
    assert np.mean(same) >= 0.98, [(per_ray[k], walks[10 * k]) for k in range(len(per_ray))
                                   if not same[k]][:10]
