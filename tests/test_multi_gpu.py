"""Edits that move several objects at once on the GPU, through the C ABI,
against the oracle on the equivalent several-object scene: per-sample
parity for contiguous and scattered objects (the latter through the static
skip mask), all seven techniques, closest hits, argument errors, and a
batch of several-object edits."""
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


CASES = [
    ("objects 1-3", None, 3, 15, (1, 2, 3, 7)),
    ("objects 2, 5, 7", [2, 5, 7], 3, 15, (1, 2, 3, 7)),
    ("objects 1-8", None, 8, 15, (1, 2, 3, 7)),
    ("objects 3, 1 (seven techniques)", [3, 1], 2, 127, (1, 2, 3, 7, 4, 5, 6)),
]


@pytest.mark.parametrize("label,objs,k,mask,techs", CASES)
def test_several_object_edit_matches_oracle(rp, label, objs, k, mask, techs):
    full = S.box_objects(width=32, height=32, max_depth=5)
    edits = S.move_objects(full, k, 0.12, objects=objs)
    sc = rp.Scene(full)
    ed = rp.Edit(sc, edits)
    ora = O.Oracle(S.objects_view(full, [e.object for e in edits]), edits)
    spp = 4
    N = sc.n_roots(spp)
    tally = Tally()
    for tech in techs:
        for frame in (1, 2):
            gpu = rp.dump_samples(sc, ed, tech, frame, spp, 23, 0, N, tech_mask=mask)
            ref = ora.dump(tech, frame, spp, 23, 0, N, tech_mask=mask)
            frac, n, bad = _compare(gpu, ref)
            tally.add(frac, n, bad, (label, tech, frame))
    tally.check()


def test_several_object_render_matches_sum_of_records(rp):
    full = S.box_objects(width=24, height=24, max_depth=5)
    edits = S.move_objects(full, 4, 0.1, objects=[4, 2, 8, 6])
    sc = rp.Scene(full)
    ed = rp.Edit(sc, edits)
    img = rp.render_residual(sc, ed, 8, 5, tech_mask=127).cpu().numpy()
    acc = np.zeros(sc.shape)
    for tech in (1, 2, 3, 7, 4, 5, 6):
        for frame in (1, 2):
            rec = rp.dump_samples(sc, ed, tech, frame, 8, 5, 0, sc.n_roots(8), tech_mask=127)
            for r in rec:
                if r["pix_a"] >= 0:
                    acc.reshape(-1, 3)[r["pix_a"]] += r["va"]
                if r["pix_b"] >= 0:
                    acc.reshape(-1, 3)[r["pix_b"]] += r["vb"]
    assert np.abs(acc).sum() > 0
    assert np.allclose(img, acc, rtol=1e-4, atol=1e-7 * np.abs(acc).max())


@pytest.mark.parametrize("frame", [1, 2])
def test_several_object_closest_hits(rp, frame):
    import torch
    full = S.box_objects(width=16, height=16, max_depth=5)
    edits = S.move_objects(full, 3, 0.3, objects=[2, 5, 7])
    view = S.objects_view(full, [e.object for e in edits])
    sc = rp.Scene(full)
    ed = rp.Edit(sc, edits)
    ora = O.Oracle(view, edits)
    rng = np.random.RandomState(9)
    n = 20000
    o = rng.uniform(-0.95, 0.95, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    t = torch.zeros(n, device="cuda")
    prim = torch.zeros(n, dtype=torch.int32, device="cuda")
    b1 = torch.zeros(n, device="cuda")
    b2 = torch.zeros(n, device="cuda")
    rp.rp_trace_closest(sc, ed, frame, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                        t, prim, b1, b2)
    tg = t.cpu().numpy()
    to, po, _, _ = ora.closest_hit(frame, o.astype(np.float64), d.astype(np.float64))
    hit = np.isfinite(to)
    assert np.array_equal(np.isfinite(tg), hit)
    pg = prim.cpu().numpy()
    dyn_g = pg >= full.n_static
    dyn_o = po >= view.n_static
    assert dyn_o.sum() > 100
    assert np.mean(dyn_g == dyn_o) > 0.999
    # the dynamic ids follow the edit's object order on both sides
    both = dyn_g & dyn_o
    assert np.mean(pg[both] - full.n_static == po[both] - view.n_static) > 0.999
    assert np.allclose(tg[hit], to[hit], rtol=1e-5, atol=2e-6)


def test_several_object_edit_errors(rp):
    full = S.box_objects(width=8, height=8, max_depth=4)
    sc = rp.Scene(full)
    e = S.move_objects(full, 8, 0.1)
    with pytest.raises(rp.RPError):
        rp.Edit(sc, [e[0], e[0]])                       # one object twice
    with pytest.raises(rp.RPError):
        rp.Edit(sc, [])                                 # no object
    bad = S.move_objects(full, 1, 0.1)[0]
    bad.object = 99
    with pytest.raises(rp.RPError):
        rp.Edit(sc, [e[1], bad])                        # out of range
    nine = e + [S.Edit(e[0].M1, e[0].M2, e[0].mat1, e[0].mat2, object=0)]
    with pytest.raises(rp.RPError):
        rp.Edit(sc, nine)                               # more than 8 objects
    ed = rp.Edit(sc, e[:2])
    g = rp.Guide(np.array([0, 0, 0, 1, 1, 1], np.float32), batch=256)
    rp.rp_scene_set_guide(sc, g)
    with pytest.raises(rp.RPError):
        rp.render_residual(sc, ed, 1, 1, tech_mask=4)   # the proposal needs one object
    rp.rp_scene_set_guide(sc, None)
    assert np.all(np.isfinite(rp.render_residual(sc, ed, 1, 1).cpu().numpy()))


def test_batch_of_several_object_edits(rp):
    import torch
    full = S.box_objects(width=32, height=32, max_depth=5)
    sc = rp.Scene(full)
    groups = [[1, 2], [3, 6, 8], [5], [7, 4, 2, 1]]
    eds = [rp.Edit(sc, S.move_objects(full, len(g), 0.1, objects=g)) for g in groups]
    outs = [torch.zeros((32, 32, 3), dtype=torch.float64, device="cuda") for _ in groups]
    items = [(eds[i], 32, 32, 3, 40 + i, 127, outs[i]) for i in range(len(groups))]
    b = rp.Batch(sc, items, config=(1 << 12, 2, 8))
    rp.rp_batch_launch(b)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        ref = rp.render_residual(sc, eds[i], 3, 40 + i, tech_mask=127).cpu().numpy()
        got = o.cpu().numpy()
        assert np.abs(ref).sum() > 0
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(ref).max())), i
