"""Pins of the ghost techniques (4)-(6) in the oracle (Sec. 4.2): with any of
them enabled the residual estimator stays unbiased (agreement with
correlated path tracing), each adds its own samples, and without motion
there is no ghost and they produce nothing."""
import numpy as np
import pytest

import oracle
from paper_2406_16302_gb300 import scenes
import helpers as H

KW = {"width": 8, "height": 8, "max_depth": 5}


@pytest.mark.parametrize("mask", [8 | 16, 8 | 32, 8 | 64, 127])
def test_ghost_techniques_keep_the_estimator_unbiased(mask):
    K = 24
    corr = H.run_many("corr", "cfg1_box_sphere", KW, range(1000, 1000 + K), 1024)
    res = H.run_many("res", "cfg1_box_sphere", KW, range(9000, 9000 + K), 128, mask=mask)
    z, zs = H.zscores(res, corr)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
    assert np.abs(z).max() < 6.0


@pytest.mark.parametrize("tech", [4, 5, 6])
def test_ghost_techniques_sample_paths_through_the_ghost(tech):
    scene, edit = scenes.cfg1_box_sphere(**KW)
    o = oracle.Oracle(scene, edit)
    rec = np.concatenate([o.dump(tech, f, 16, 3, 0, o.n_roots(16), tech_mask=127) for f in (1, 2)])
    assert len(rec) > 50
    assert np.all(np.isfinite(rec["va"])) and np.all(np.isfinite(rec["vb"]))
    assert np.all(rec["tech"] == tech)


def test_ghost_techniques_need_motion():
    scene, edit = scenes.cfg2_box_blob(width=8, height=8, max_depth=5, blob_level=2)
    o = oracle.Oracle(scene, edit)
    assert np.all(o.render_residual(8, 1, tech_mask=oracle.MASK_GHOSTS) == 0.0)
    for tech in (4, 5, 6):
        assert len(o.dump(tech, 2, 8, 1, 0, o.n_roots(8), tech_mask=127)) == 0


@pytest.mark.parametrize("mask", [15, 127])
def test_without_path_mapping_the_estimator_stays_unbiased(mask):
    """Path mapping off: each frame's dynamic paths come from that frame's
    sampling alone; the residual still agrees with correlated path tracing."""
    K = 24
    corr = H.run_many("corr", "cfg1_box_sphere", KW, range(1000, 1000 + K), 1024)
    res = H.run_many("res_nomap", "cfg1_box_sphere", KW, range(11000, 11000 + K), 128, mask=mask)
    z, zs = H.zscores(res, corr)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4


def test_object_transform_mapping_stays_unbiased():
    """Mapping mode 1 (the object transform for every path) against correlated
    path tracing (mode 2, the default, is covered by the other residual pins)."""
    import multiprocessing as mp
    K = 24
    corr = H.run_many("corr", "cfg1_box_sphere", KW, range(1000, 1000 + K), 1024)
    res = H.run_many("res_objmap", "cfg1_box_sphere", KW, range(12000, 12000 + K), 128, mask=15)
    z, zs = H.zscores(res, corr)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
