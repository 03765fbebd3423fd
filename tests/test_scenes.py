"""Host-side checks of the seeded input generators (no method arithmetic)."""
import numpy as np

from paper_2406_16302_gb300 import scenes as S


def test_object_view_moves_the_range_into_the_dynamic_mesh():
    scene, frames = S.cfg4_batch(n_objects=3, min_tris=200, max_tris=800, resolutions=(16,),
                                 spp_range=(1, 2))
    assert len(frames) == 3 and [f[0].object for f in frames] == [1, 2, 3]
    for k in (1, 2, 3):
        first, count = (int(v) for v in scene.object_ranges[k - 1])
        v = S.object_view(scene, k)
        assert v.n_static == scene.n_static - count and v.n_dyn == count
        want = np.asarray(scene.static_vertices)[np.asarray(scene.static_triangles)[first:first + count]]
        got = np.asarray(v.dyn_vertices)[np.asarray(v.dyn_triangles)]
        assert np.array_equal(want, got)
        # the other static triangles keep their order (emitters included)
        keep = np.ones(scene.n_static, bool)
        keep[first:first + count] = False
        assert np.array_equal(np.asarray(scene.static_triangles)[keep], v.static_triangles)
    assert S.object_view(scene, 0) is scene


def test_object_edits_are_rigid_and_small():
    scene, frames = S.cfg4_batch(n_objects=6, min_tris=200, max_tris=800)
    for e, w, h, spp in frames:
        R = np.asarray(e.M2, np.float64)[:, :3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        ang = np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))
        assert ang <= 10.0 + 1e-4
        assert np.array_equal(e.M1, S.translate((0, 0, 0)))
        assert w in (256, 512, 1024) and 64 <= spp <= 256


def test_uv_sphere_fast_equals_loop_builder():
    for seg, ring in [(6, 4), (13, 9)]:
        v1, t1 = S.uv_sphere(seg, ring)
        v2, t2 = S.uv_sphere_fast(seg, ring)
        assert np.allclose(v1, v2) and np.array_equal(t1, t2)
