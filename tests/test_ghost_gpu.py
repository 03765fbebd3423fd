"""Ghost techniques (4)-(6) on the GPU against the oracle, per sample: every
technique with all seven enabled (the ghost crossings enter every path's
balance-heuristic denominator), on a translated and on a rotated object."""
import numpy as np
import pytest

import oracle as O
from paper_2406_16302_gb300 import scenes as S
from test_gpu_parity import Tally, _compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_16302_gb300 import build, rp as binding
    build.build()
    binding.lib()
    return binding


def _rotating():
    scene, edit = S.cfg1_box_sphere(width=24, height=24, max_depth=6)
    edit.M2 = S.rotate_y_translate(25.0, (-0.22, -0.64, -0.1))
    edit.M1 = S.translate((-0.3, -0.64, -0.2))
    return scene, edit


CASES = [
    ("translate", lambda: S.cfg1_box_sphere(width=32, height=32, max_depth=6), 4),
    ("rotate", _rotating, 4),
]


@pytest.mark.parametrize("name,make,spp", CASES)
def test_seven_techniques_match_oracle(rp, name, make, spp):
    scene, edit = make()
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    ora = O.Oracle(scene, edit)
    N = sc.n_roots(spp)
    tally = Tally()
    for tech in (4, 5, 6, 1, 2, 3, 7):
        for frame in (1, 2):
            gpu = rp.dump_samples(sc, ed, tech, frame, spp, 31, 0, N, tech_mask=127)
            ref = ora.dump(tech, frame, spp, 31, 0, N, tech_mask=127)
            if tech in (4, 5, 6):
                assert len(ref) > 20, (tech, frame, len(ref))
            frac, n, bad = _compare(gpu, ref)
            tally.add(frac, n, bad, (name, tech, frame))
    tally.check()


def test_ghost_render_equals_oracle_image_statistically(rp):
    """The splatted image with all seven techniques against the oracle's
    image of the same seeds (identical up to the few diverging paths)."""
    scene, edit = S.cfg1_box_sphere(width=16, height=16, max_depth=5)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    img = rp.render_residual(sc, ed, 8, 77, tech_mask=127).cpu().numpy()
    ref = O.Oracle(scene, edit).render_residual(8, 77, tech_mask=127)
    assert np.all(np.isfinite(img))
    err = np.abs(img - ref).sum() / np.abs(ref).sum()
    assert err < 5e-3, err


def test_ghost_techniques_need_motion(rp):
    scene, edit = S.cfg2_box_blob(width=16, height=16, max_depth=5, blob_level=3)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    img = rp.render_residual(sc, ed, 4, 1, tech_mask=rp.RP_TECH_GHOSTS).cpu().numpy()
    assert np.all(img == 0.0)


def test_without_path_mapping_matches_oracle(rp):
    scene, edit = S.cfg1_box_sphere(width=24, height=24, max_depth=5)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    rp.rp_scene_set_mapping(sc, False)
    ora = O.Oracle(scene, edit)
    ora.set_mapping(False)
    N = sc.n_roots(4)
    tally = Tally()
    for tech in (1, 3, 5, 7):
        for frame in (1, 2):
            gpu = rp.dump_samples(sc, ed, tech, frame, 4, 5, 0, N, tech_mask=127)
            ref = ora.dump(tech, frame, 4, 5, 0, N, tech_mask=127)
            assert np.all(gpu["vb"] == 0.0)
            frac, n, bad = _compare(gpu, ref)
            tally.add(frac, n, bad, ("no mapping", tech, frame))
    tally.check()


@pytest.mark.parametrize("mode", [1, 2])
def test_mapping_modes_match_oracle(rp, mode):
    """Object-transform mapping for every path (1) and the default camera
    mapping for dynamic first edges (2), per sample against the oracle."""
    scene, edit = S.cfg1_box_sphere(width=32, height=32, max_depth=6)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    rp.rp_scene_set_mapping(sc, mode)
    ora = O.Oracle(scene, edit)
    ora.set_mapping(mode)
    N = sc.n_roots(4)
    tally = Tally()
    for tech in (1, 2, 3, 7):
        for frame in (1, 2):
            gpu = rp.dump_samples(sc, ed, tech, frame, 4, 9, 0, N)
            ref = ora.dump(tech, frame, 4, 9, 0, N)
            frac, n, bad = _compare(gpu, ref)
            tally.add(frac, n, bad, (mode, tech, frame))
    tally.check()
