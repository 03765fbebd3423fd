"""Pins of edits that move several objects at once (Sec. 6, scenes with 1,
2, 4 and 8 moving objects) in the oracle: the objects form one dynamic set
with per-object transforms; the estimator stays unbiased against correlated
path tracing, the per-object world geometry matches an independent numpy
brute force, and paths through two moved objects are rejected by the
mapping."""
import numpy as np
import pytest

import oracle
from paper_2406_16302_gb300 import scenes
import helpers as H

KW = {"width": 8, "height": 8, "max_depth": 5}


@pytest.mark.parametrize("k,mask", [(3, 15), (8, 15), (3, 127)])
def test_several_moving_objects_keep_the_estimator_unbiased(k, mask):
    K = 24
    ek = ("objects", k, 0.1)
    corr = H.run_many("corr", "box_objects", KW, range(1000, 1000 + K), 1024, edit_kind=ek)
    res = H.run_many("res", "box_objects", KW, range(9000, 9000 + K), 128, mask=mask, edit_kind=ek)
    z, zs = H.zscores(res, corr)
    assert abs(corr.mean(0)).sum() > 0.0
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
    assert np.abs(z).max() < 6.0


def _numpy_closest(tris, o, d):
    """Moller-Trumbore against every triangle (numpy, one-sided test not
    applied: the oracle's traversal hits both sides)."""
    v0, v1, v2 = tris[:, 0], tris[:, 1], tris[:, 2]
    e1, e2 = v1 - v0, v2 - v0
    best = np.full(len(o), np.inf)
    for i in range(len(o)):
        p = np.cross(d[i], e2)
        det = np.einsum("ij,ij->i", e1, p)
        ok = np.abs(det) > 1e-14
        inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
        s = o[i] - v0
        u = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        v = (q @ d[i]) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
        hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
        if hit.any():
            best[i] = t[hit].min()
    return best


@pytest.mark.parametrize("frame", [1, 2])
def test_each_object_is_placed_by_its_own_transform(frame):
    full = scenes.box_objects(**KW)
    edits = scenes.move_objects(full, 3, 0.3)
    view = scenes.objects_view(full, [e.object for e in edits])
    o = oracle.Oracle(view, edits)
    # world triangles: static, then each object under its own frame transform
    sv = np.asarray(view.static_vertices, np.float64)
    tris = [sv[np.asarray(view.static_triangles, np.int64)]]
    dv = np.asarray(view.dyn_vertices, np.float64)[np.asarray(view.dyn_triangles, np.int64)]
    for i, e in enumerate(edits):
        M = np.asarray(e.M1 if frame == 1 else e.M2, np.float64)
        sel = view.dyn_instance == i
        tris.append(dv[sel] @ M[:, :3].T + M[:, 3])
    tris = np.concatenate(tris)
    rng = np.random.RandomState(3)
    n = 300
    orig = np.tile([0.0, -0.5, 0.8], (n, 1)) + rng.uniform(-0.1, 0.1, size=(n, 3))
    # aim at the moved objects' centres in this frame (and around them)
    tgt = np.array([tris[len(tris) - len(dv) + np.nonzero(view.dyn_instance == i)[0]].reshape(-1, 3)
                    .mean(0) for i in range(len(edits))])
    aim = tgt[rng.randint(0, len(tgt), n)] + rng.uniform(-0.12, 0.12, size=(n, 3))
    d = aim - orig
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t, prim, _, _ = o.closest_hit(frame, orig, d)
    want = _numpy_closest(tris, orig, d)
    fin = np.isfinite(want)
    assert np.array_equal(np.isfinite(t), fin)
    assert np.allclose(t[fin], want[fin], rtol=1e-9, atol=1e-12)
    dyn = prim[fin] >= view.n_static
    assert dyn.mean() > 0.2                      # the moved objects are hit


def test_paths_through_two_moved_objects_are_rejected():
    full = scenes.box_objects(width=16, height=16, max_depth=5)
    edits = scenes.move_objects(full, 8, 0.1)
    view = scenes.objects_view(full, [e.object for e in edits])
    o = oracle.Oracle(view, edits)
    rec = np.concatenate([o.dump(3, f, 16, 2, 0, o.n_roots(16)) for f in (1, 2)])
    assert (rec["status"] == 3).sum() > 0          # more than one dynamic vertex
    assert (rec["status"] == 0).sum() > 0


def test_an_edit_of_one_listed_object_is_the_single_object_edit():
    full = scenes.box_objects(**KW)
    e = scenes.move_objects(full, 1, 0.1)
    a = oracle.Oracle(scenes.object_view(full, 1), e[0]).render_residual(16, 3)
    b = oracle.Oracle(scenes.objects_view(full, [1]), e).render_residual(16, 3)
    assert np.array_equal(a, b)
