"""The host BVH builder behind rp_scene_create, checked on the CPU through
rp_bvh_build_host: every triangle sits in exactly one leaf, every child box
encloses what is below it, the depth fits the device traversal stack, and a
plain numpy traversal of the 64-byte node layout finds the same closest hit
as a brute-force test over all triangles."""
import numpy as np
import pytest

from paper_2406_16302_gb300 import scenes as S

STACK_DEPTH, MAX_DEPTH, MAX_LEAF = 40, 38, 8


@pytest.fixture(scope="module")
def rp():
    from paper_2406_16302_gb300 import build, rp as rp_mod
    build.build()
    rp_mod.lib()
    return rp_mod


def _ints(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def _meshes():
    box, _ = S.cfg2_box_blob(width=8, height=8, blob_level=3)
    yield "box_blob_static", box.static_vertices, box.static_triangles
    yield "blob", box.dyn_vertices, box.dyn_triangles
    rng = np.random.default_rng(4)
    v = rng.random((3000, 3)).astype(np.float32)
    yield "triangle_soup", v, rng.integers(0, 3000, (1000, 3)).astype(np.uint32)
    # every centroid equal: the builder must split by count, not by position
    t = np.array([[0, 1, 2]] * 40, dtype=np.uint32)
    yield "coincident", np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), t


def _check_structure(bvh, verts, tris):
    nodes, leaf_tris = bvh["nodes"], bvh["tris"]
    n = len(tris)
    ids = _ints(leaf_tris[:, 3])
    assert sorted(ids.tolist()) == list(range(n))            # each triangle once
    # the leaf copies hold the mesh's own vertices
    for k in range(3):
        np.testing.assert_array_equal(leaf_tris[:, 4 * k:4 * k + 3],
                                      np.asarray(verts, np.float32)[tris[ids, k]])
    assert 1 <= bvh["depth"] <= MAX_DEPTH < STACK_DEPTH
    d = _ints(nodes[:, 12:16])
    covered = np.zeros(n, dtype=int)
    seen_inner = np.zeros(len(nodes), dtype=int)
    for i in range(len(nodes)):
        boxes = [(nodes[i, [0, 2, 8]], nodes[i, [1, 3, 9]]),
                 (nodes[i, [4, 6, 10]], nodes[i, [5, 7, 11]])]
        for s in range(2):
            child, count = d[i, s], d[i, 2 + s]
            lo, hi = boxes[s]
            if child >= 0:
                seen_inner[child] += 1
                assert child > i                              # depth-first order
                cn = nodes[child]
                for lo2, hi2 in ((cn[[0, 2, 8]], cn[[1, 3, 9]]), (cn[[4, 6, 10]], cn[[5, 7, 11]])):
                    if np.all(lo2 <= hi2):
                        assert np.all(lo <= lo2) and np.all(hi2 <= hi)
            elif count > 0:
                first = ~child
                assert count <= MAX_LEAF or bvh["depth"] == MAX_DEPTH
                covered[first:first + count] += 1
                v = leaf_tris[first:first + count].reshape(-1, 3, 4)[:, :, :3].reshape(-1, 3)
                assert np.all(lo <= v.min(0)) and np.all(v.max(0) <= hi)
    assert np.all(covered == 1)                                # leaves partition the list
    assert seen_inner[0] == 0 and np.all(seen_inner[1:] == 1)  # a tree rooted at node 0


def _ray_tri(o, d, v0, v1, v2):
    """Moller-Trumbore in double; t or inf for each triangle."""
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    ok = np.abs(det) > 1e-18
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = o - v0
    u = np.einsum("ij,ij->i", s, p) * inv
    q = np.cross(s, e1)
    v = (q @ d) * inv
    t = np.einsum("ij,ij->i", e2, q) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-6)
    return np.where(hit, t, np.inf)


def _traverse(bvh, o, d):
    """Closest hit by walking the node layout with a stack (slab tests)."""
    nodes, leaf = bvh["nodes"].astype(np.float64), bvh["tris"].astype(np.float64)
    di = _ints(bvh["nodes"][:, 12:16])
    inv = 1.0 / np.where(d == 0, 1e-30, d)
    best, best_id = np.inf, -1
    stack = [0]
    while stack:
        i = stack.pop()
        for s in range(2):
            lo = nodes[i, [0, 2, 8]] if s == 0 else nodes[i, [4, 6, 10]]
            hi = nodes[i, [1, 3, 9]] if s == 0 else nodes[i, [5, 7, 11]]
            t0, t1 = (lo - o) * inv, (hi - o) * inv
            tn, tf = np.minimum(t0, t1).max(), np.maximum(t0, t1).min()
            if tn > tf * (1 + 1e-6) + 1e-9 or tf < 0 or tn > best:
                continue
            child, count = di[i, s], di[i, 2 + s]
            if child >= 0:
                stack.append(child)
            elif count > 0:
                first = ~child
                tv = leaf[first:first + count].reshape(-1, 3, 4)[:, :, :3]
                t = _ray_tri(o, d, tv[:, 0], tv[:, 1], tv[:, 2])
                k = int(np.argmin(t))
                if t[k] < best:
                    best, best_id = t[k], int(_ints(bvh["tris"][first + k, 3:4])[0])
    return best, best_id


@pytest.mark.parametrize("name", ["box_blob_static", "blob", "triangle_soup", "coincident"])
def test_bvh_structure(rp, name):
    verts, tris = next((v, t) for n, v, t in _meshes() if n == name)
    tris = np.asarray(tris, dtype=np.uint32)
    bvh = rp.rp_bvh_build_host(verts, tris)
    _check_structure(bvh, verts, tris)


@pytest.mark.parametrize("name", ["box_blob_static", "blob", "triangle_soup"])
def test_traversal_of_the_layout_matches_brute_force(rp, name):
    verts, tris = next((v, t) for n, v, t in _meshes() if n == name)
    tris = np.asarray(tris, dtype=np.uint32)
    bvh = rp.rp_bvh_build_host(verts, tris)
    V = np.asarray(verts, np.float64)
    v0, v1, v2 = V[tris[:, 0]], V[tris[:, 1]], V[tris[:, 2]]
    lo, hi = V.min(0), V.max(0)
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(150):
        o = lo + (hi - lo) * rng.random(3) * 1.2 - 0.1 * (hi - lo)
        target = lo + (hi - lo) * rng.random(3)
        d = target - o
        d /= np.linalg.norm(d)
        t_all = _ray_tri(o, d, v0, v1, v2)
        k = int(np.argmin(t_all))
        tb, idb = _traverse(bvh, o, d)
        if np.isinf(t_all[k]):
            assert np.isinf(tb)
            continue
        hits += 1
        assert abs(tb - t_all[k]) <= 1e-9 * max(1.0, t_all[k])
        assert idb == k or abs(t_all[idb] - t_all[k]) <= 1e-9 * max(1.0, t_all[k])
    assert hits > 50


def test_bad_meshes_are_refused(rp):
    v = np.zeros((3, 3), np.float32)
    with pytest.raises(rp.RPError) as e:
        rp.rp_bvh_build_host(v, np.array([[0, 1, 3]], np.uint32))
    assert e.value.status == 1
    with pytest.raises(rp.RPError):
        rp.rp_bvh_build_host(v, np.zeros((0, 3), np.uint32))
