"""The structure of the balance-heuristic denominator (Sec. 4.3) counted
against brute force.

A path of frame g is produced by one technique per dynamic vertex x_i --
(1) when x_i is the vertex next to the emitter, (2) when it is the first
vertex after the sensor, (3) otherwise -- by one ghost technique per crossing
of an edge with the object at its other-frame pose ((5) on the sensor edge,
(4) on the emitter edge, (6) in between; Sec. 4.2), and by path tracing.  The
paper's example figure of the seven techniques shows a path with one dynamic
vertex and four ghost crossings, which five techniques (besides path tracing)
can sample.  Here the crossings are counted by a plain numpy segment/triangle
test over every triangle of the ghost, independent of the oracle's BVH, and
the oracle's list of denominator terms must have exactly that composition.
"""
import collections

import numpy as np
import pytest

import oracle
from paper_2406_16302_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _world(v, M):
    M = np.asarray(M, dtype=np.float64)
    return np.asarray(v, dtype=np.float64) @ M[:, :3].T + M[:, 3]


def _segment_crossings(a, b, tris, eps=1e-5):
    """Number of triangles of tris (T, 3, 3) that the open segment a-b
    crosses (Moller-Trumbore, all triangles, no acceleration)."""
    e = b - a
    dist = np.linalg.norm(e)
    d = e / dist
    v0, v1, v2 = tris[:, 0], tris[:, 1], tris[:, 2]
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    ok = np.abs(det) > 1e-14
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = a - v0
    u = np.einsum("ij,ij->i", s, p) * inv
    q = np.cross(s, e1)
    v = (q @ d) * inv
    t = np.einsum("ij,ij->i", e2, q) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > eps) & (t < dist - eps)
    return int(hit.sum())


def _setup(shift):
    scene, edit = scenes.cfg1_box_sphere()
    M2 = np.array(edit.M1, dtype=np.float32).copy()
    M2[:, 3] += np.asarray(shift, dtype=np.float32)
    import dataclasses
    edit = dataclasses.replace(edit, M2=M2)
    return scene, edit


def _random_bary(rng):
    u, v = rng.random(2)
    if u + v > 1:
        u, v = 1 - u, 1 - v
    return u, v


def _points(scene, edit, g, prims, bary):
    sv = np.asarray(scene.static_vertices, dtype=np.float64)
    dw = _world(scene.dyn_vertices, edit.M1 if g == 1 else edit.M2)
    out = []
    for pr, (b1, b2) in zip(prims, bary):
        if pr < scene.n_static:
            tv = sv[scene.static_triangles[pr]]
        else:
            tv = dw[scene.dyn_triangles[pr - scene.n_static]]
        out.append((1 - b1 - b2) * tv[0] + b1 * tv[1] + b2 * tv[2])
    return out


def _expected(scene, edit, g, prims, bary, ghost_tris):
    k = len(prims) + 1
    cam = np.array(scene.camera.pos, dtype=np.float64)
    pts = [cam] + _points(scene, edit, g, prims, bary)
    want = collections.Counter({7: 1})
    for i in range(1, k - 1):
        if prims[i - 1] >= scene.n_static:
            want[1 if i == k - 2 else 2 if i == 1 else 3] += 1
    crossings = 0
    for j in range(k - 1):
        n = _segment_crossings(pts[j], pts[j + 1], ghost_tris)
        crossings += n
        if n:
            want[5 if j == 0 else 4 if j == k - 2 else 6] += n
    return want, crossings


@pytest.mark.parametrize("g", [1, 2])
def test_denominator_terms_match_brute_force_counts(g):
    scene, edit = _setup((0.45, 0.25, 0.15))
    o = oracle.Oracle(scene, edit)
    ghost = _world(scene.dyn_vertices, edit.M2 if g == 1 else edit.M1)[scene.dyn_triangles]
    emit = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    rng = np.random.default_rng(11 + g)
    n_ghost_terms = 0
    for trial in range(400):
        k = int(rng.integers(3, 7))
        prims = []
        for i in range(k - 2):
            if rng.random() < 0.4:
                prims.append(scene.n_static + int(rng.integers(scene.n_dyn)))
            else:
                prims.append(int(rng.integers(scene.n_static)))
        prims.append(int(rng.choice(emit)))
        bary = [_random_bary(rng) for _ in prims]
        tech, dens = o.mis_terms(g, prims, bary)
        want, crossings = _expected(scene, edit, g, prims, bary, ghost)
        got = collections.Counter(tech.tolist())
        assert got == want, (trial, prims, got, want)
        n_ghost_terms += crossings
        assert np.all(dens >= 0)
    assert n_ghost_terms > 100        # the sample exercises the ghost terms


def test_masked_techniques_leave_the_denominator():
    scene, edit = _setup((0.45, 0.25, 0.15))
    o = oracle.Oracle(scene, edit)
    rng = np.random.default_rng(5)
    emit = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    for _ in range(50):
        prims = [scene.n_static + int(rng.integers(scene.n_dyn)), int(rng.integers(scene.n_static)),
                 scene.n_static + int(rng.integers(scene.n_dyn)), int(rng.choice(emit))]
        bary = [_random_bary(rng) for _ in prims]
        t_all, d_all = o.mis_terms(1, prims, bary, tech_mask=oracle.MASK_SEVEN)
        t_four, d_four = o.mis_terms(1, prims, bary, tech_mask=oracle.MASK_ALL)
        assert set(t_four.tolist()) <= {1, 2, 3, 7}
        assert sorted(t_four.tolist()) == sorted(t for t in t_all.tolist() if t in (1, 2, 3, 7))
        # each term is the same number whichever others are enabled
        keep = np.isin(t_all, [1, 2, 3, 7])
        np.testing.assert_array_equal(np.sort(d_all[keep]), np.sort(d_four))


def test_figure_example_one_dynamic_vertex_four_crossings_five_techniques():
    """A path with one vertex on the object and two edges that each pass
    through the ghost (in and out): five techniques besides path tracing."""
    scene, edit = _setup((0.45, 0.25, 0.15))
    o = oracle.Oracle(scene, edit)
    g = 1
    ghost = _world(scene.dyn_vertices, edit.M2)[scene.dyn_triangles]
    emit = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    rng = np.random.default_rng(2024)
    found = None
    for _ in range(20000):
        k = 5
        dyn_at = int(rng.integers(1, k - 1))
        prims = [scene.n_static + int(rng.integers(scene.n_dyn)) if i == dyn_at
                 else int(rng.integers(scene.n_static)) for i in range(1, k - 1)]
        prims.append(int(rng.choice(emit)))
        bary = [_random_bary(rng) for _ in prims]
        want, crossings = _expected(scene, edit, g, prims, bary, ghost)
        if crossings == 4:
            found = (prims, bary, want)
            break
    assert found is not None
    prims, bary, want = found
    tech, dens = o.mis_terms(g, prims, bary)
    non_pt = [t for t in tech.tolist() if t != 7]
    assert len(non_pt) == 5
    assert collections.Counter(tech.tolist()) == want
    assert sum(want[t] for t in (4, 5, 6)) == 4


def test_static_path_without_crossings_has_only_path_tracing():
    scene, edit = _setup((0.45, 0.25, 0.15))
    o = oracle.Oracle(scene, edit)
    ghost = _world(scene.dyn_vertices, edit.M2)[scene.dyn_triangles]
    emit = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    rng = np.random.default_rng(3)
    seen = 0
    for _ in range(200):
        prims = [int(rng.integers(scene.n_static)) for _ in range(3)] + [int(rng.choice(emit))]
        bary = [_random_bary(rng) for _ in prims]
        want, crossings = _expected(scene, edit, 1, prims, bary, ghost)
        if crossings:
            continue
        tech, _ = o.mis_terms(1, prims, bary)
        assert tech.tolist() == [7]
        seen += 1
    assert seen > 50
