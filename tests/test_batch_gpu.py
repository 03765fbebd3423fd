"""Movable objects and batched edits on the GPU: an edit of any movable
object against the oracle on the equivalent single-object scene, a batch
(one CUDA graph over concurrent branches) against the items rendered one by
one, new seeds, and the autotuner."""
import dataclasses

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


def _small_batch(n_objects=4, res=32, max_depth=6):
    scene, frames = S.cfg4_batch(n_objects=n_objects, min_tris=400, max_tris=4000,
                                 max_depth=max_depth, resolutions=(res,), spp_range=(2, 6))
    cam = dataclasses.replace(scene.camera, width=res, height=res)
    return dataclasses.replace(scene, camera=cam), frames


def _with_size(scene, w, h):
    return dataclasses.replace(scene, camera=dataclasses.replace(scene.camera, width=w, height=h))


@pytest.mark.parametrize("k", [1, 3])
def test_movable_object_edit_matches_oracle(rp, k):
    """Moving object k of the static geometry is the single-object problem
    with that object as the dynamic mesh (the oracle's input)."""
    scene, frames = _small_batch()
    edit = frames[k - 1][0]
    assert edit.object == k
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    ora = O.Oracle(S.object_view(scene, k), edit)
    spp = 4
    N = sc.n_roots(spp)
    tally = Tally()
    for tech in (1, 2, 3, 7):
        for frame in (1, 2):
            gpu = rp.dump_samples(sc, ed, tech, frame, spp, 17, 0, N)
            ref = ora.dump(tech, frame, spp, 17, 0, N)
            frac, n, bad = _compare(gpu, ref)
            tally.add(frac, n, bad, (k, tech, frame))
    tally.check()


def test_movable_object_closest_hits(rp):
    """Static rays never hit the moved object's base pose; they hit the
    object under M_g instead (oracle with the object as dynamic mesh)."""
    import torch
    scene, frames = _small_batch()
    edit = frames[1][0]
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    view = S.object_view(scene, 2)
    ora = O.Oracle(view, edit)
    rng = np.random.RandomState(5)
    n = 20000
    o = rng.uniform(-0.95, 0.95, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    for frame in (1, 2):
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
        # the dynamic ids agree (n_static differs by the object's triangles)
        pg = prim.cpu().numpy()
        dyn_g = pg >= scene.n_static
        dyn_o = po >= view.n_static
        assert np.mean(dyn_g == dyn_o) > 0.999
        assert np.allclose(tg[hit], to[hit], rtol=1e-5, atol=2e-6)


def _items(rp, scene, frames, sizes, seeds):
    import torch
    scs, items, eds = {}, [], []
    for (edit, _, _, spp), (w, h), seed in zip(frames, sizes, seeds):
        key = (w, h)
        if key not in scs:
            scs[key] = rp.Scene(_with_size(scene, w, h))
        out = torch.zeros((h, w, 3), dtype=torch.float64, device="cuda")
        items.append((edit, w, h, spp, seed, 15, out))
    return scs, items


BATCH_MODES = [(1 << 12, 2, 8, 0),      # graph of per-wave launches over two branches
               (1 << 12, 2, 8, 1),      # persistent kernel, rounds of two waves
               (1 << 11, 16, 0, 1)]     # persistent kernel, rounds of up to 16 waves


@pytest.mark.parametrize("config", BATCH_MODES)
def test_batch_equals_items_rendered_one_by_one(rp, config):
    import torch
    scene, frames = _small_batch(n_objects=4)
    sizes = [(32, 32), (48, 24), (40, 40), (24, 48)]
    seeds = [11, 12, 13, 14]
    base = rp.Scene(scene)
    scs, items = _items(rp, scene, frames, sizes, seeds)
    edits = [rp.Edit(base, f[0]) for f in frames]
    bitems = [(edits[i],) + it[1:] for i, it in enumerate(items)]
    batch = rp.Batch(base, bitems, config=config)
    cfg, nodes = rp.rp_batch_info(batch)
    assert cfg == config and nodes >= 2
    rp.rp_batch_launch(batch)
    torch.cuda.synchronize()
    rp.rp_batch_status(batch)
    for i, (edit, w, h, spp, seed, mask, out) in enumerate(bitems):
        sc = scs[(w, h)]
        ed = rp.Edit(sc, frames[i][0])
        ref = rp.render_residual(sc, ed, spp, seed).cpu().numpy()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(ref).max())), i
    # new seeds, cleared images, second launch
    for it in bitems:
        it[-1].zero_()
    rp.rp_batch_set_seeds(batch, [21, 22, 23, 24])
    rp.rp_batch_launch(batch)
    torch.cuda.synchronize()
    for i, (edit, w, h, spp, seed, mask, out) in enumerate(bitems):
        sc = scs[(w, h)]
        ed = rp.Edit(sc, frames[i][0])
        ref = rp.render_residual(sc, ed, spp, 21 + i).cpu().numpy()
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_autotune_picks_a_candidate_and_keeps_the_result(rp):
    import torch
    scene, frames = _small_batch(n_objects=3)
    base = rp.Scene(scene)
    edits = [rp.Edit(base, f[0]) for f in frames]
    outs = [torch.zeros((32, 32, 3), dtype=torch.float64, device="cuda") for _ in frames]
    items = [(edits[i], 32, 32, frames[i][3], 5 + i, 15, outs[i]) for i in range(len(frames))]
    cfg, ms = rp.rp_batch_autotune(base, items, spp_divisor=2)
    assert ms > 0.0
    if cfg[3]:            # persistent mode: waves per round, resident blocks per SM
        assert cfg[1] in (4, 8, 16, 32) and cfg[2] in (0, 2, 4) and cfg[0] * cfg[1] <= 1 << 23
    else:                 # graph mode: branches, queue-kernel blocks per SM
        assert cfg[1] in (1, 2, 4) and cfg[2] in (0, 16, 32, 64, 128) and cfg[0] >= 256
    for o in outs:
        assert float(o.abs().sum()) == 0.0          # the autotuner leaves the images alone
    b1 = rp.Batch(base, items, config=cfg)
    rp.rp_batch_launch(b1)
    torch.cuda.synchronize()
    got = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    b2 = rp.Batch(base, items)
    rp.rp_batch_launch(b2)
    torch.cuda.synchronize()
    for a, b in zip(got, outs):
        assert torch.allclose(a, b, rtol=1e-9, atol=1e-15)


def test_full_size_images_are_finite(rp):
    """Walks through near-coincident vertices make per-edge factors of 1e8
    and more; the 256 x 256 x 64 spp renders must stay finite."""
    scene, edit = S.cfg2_box_blob()
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    for mask in (1, 2, 4, 8):
        img = rp.render_residual(sc, ed, 64, 710000, tech_mask=mask).cpu().numpy()
        assert np.all(np.isfinite(img)), mask
    for frame in (1, 2):
        assert np.all(np.isfinite(rp.render_primal(sc, ed, frame, 256, 720000).cpu().numpy()))


@pytest.mark.parametrize("persistent", [0, 1])
def test_batched_items_match_the_oracle(rp, persistent):
    """Two items of one batch against the FP64 oracle, in either batch mode:
    each item's residual image (its own image size, spp and seed) equals the
    oracle's render of the equivalent single-object scene at the same size,
    pixel by pixel within 1e-4 of the image's scale on at least 99.9 % of
    pixels."""
    import torch
    scene, frames = _small_batch(n_objects=4)
    sizes = [(32, 32), (40, 24)]
    seeds = [31, 32]
    base = rp.Scene(scene)
    edits = [rp.Edit(base, frames[i][0]) for i in range(2)]
    outs = [torch.zeros((h, w, 3), dtype=torch.float64, device="cuda") for w, h in sizes]
    items = [(edits[i], sizes[i][0], sizes[i][1], frames[i][3], seeds[i], 15, outs[i])
             for i in range(2)]
    batch = rp.Batch(base, items, config=(1 << 12, 2, 8, persistent))
    rp.rp_batch_launch(batch)
    torch.cuda.synchronize()
    rp.rp_batch_status(batch)
    for i, (w, h) in enumerate(sizes):
        edit = frames[i][0]
        view = _with_size(S.object_view(scene, edit.object), w, h)
        ref = O.Oracle(view, dataclasses.replace(edit, object=0)).render_residual(frames[i][3], seeds[i])
        got = outs[i].cpu().numpy()
        scale = np.abs(ref).max()
        assert scale > 0, i
        err = np.abs(got - ref)
        assert np.mean(err <= 1e-4 * scale) >= 0.999, (i, np.sort(err.ravel())[-5:] / scale)
        assert abs(got.sum() - ref.sum()) <= 1e-3 * np.abs(ref).sum(), i
