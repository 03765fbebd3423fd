"""rp_render_residual_f32_noalloc, the entry point for callers that cannot let
the library allocate device memory (hosts with their own memory pools, hard
memory caps, or no allocation allowed after start-up).  It must give the same
image as rp_render_residual_f32, whose scratch image is cudaMalloc'd, on
consecutive calls (the fixed scratch array keeps the previous call's sums
and has to be cleared each time), agree with the oracle, leave device memory
untouched, and refuse what its kernels do not run.  Kept in a file of its own
that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _scene(width=32, height=32):
    from paper_2406_16302_gb300 import build, rp, scenes
    build.build()
    scene, edit = scenes.cfg1_box_sphere(width=width, height=height)
    sc = rp.Scene(scene)
    return scene, edit, sc, rp.Edit(sc, edit)


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_2406_16302_gb300 import rp
    _, _, sc, ed = _scene()
    for call in range(2):
        ref = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        rp.rp_render_residual_f32(sc, ed, 4, 17, ref)
        out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        rp.rp_render_residual_f32_noalloc(sc, ed, 4, 17, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.abs(r).max() > 0
        assert np.allclose(o, r, rtol=1e-5, atol=1e-6 * np.abs(r).max()), call


def test_noalloc_matches_the_oracle():
    """The moving-sphere box at 24x24, 4 spp: per pixel within 1e-4 of the
    image's scale on at least 99 % of pixels (the float32 output rounds each
    FP64 sum once)."""
    import torch
    import oracle
    from paper_2406_16302_gb300 import rp
    scene, edit, sc, ed = _scene(24, 24)
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    rp.rp_render_residual_f32_noalloc(sc, ed, 4, 5, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy().astype(np.float64)
    o = oracle.Oracle(scene, edit).render_residual(4, 5)
    scale = np.abs(o).max()
    assert scale > 0
    frac = float(np.mean(np.abs(g - o) <= 1e-4 * scale))
    assert frac >= 0.99, (frac, float(np.abs(g - o).max() / scale))


def test_noalloc_allocates_no_device_memory():
    """After one call (which looks up the scratch array's address and loads
    the kernels), further calls change neither the device's free memory nor
    torch's allocator."""
    import torch
    from paper_2406_16302_gb300 import rp
    _, _, sc, ed = _scene()
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    rp.rp_render_residual_f32_noalloc(sc, ed, 2, 1, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for k in range(4):
        rp.rp_render_residual_f32_noalloc(sc, ed, 2, 2 + k, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocation.all.allocated", "segment.all.allocated", "allocated_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


def test_noalloc_rejects_ghost_techniques():
    import torch
    from paper_2406_16302_gb300 import rp
    _, _, sc, ed = _scene(16, 16)
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RPError) as e:
        rp.rp_render_residual_f32_noalloc(sc, ed, 1, 1, out, tech_mask=127)
    assert e.value.status == 5            # RP_ERR_UNSUPPORTED


def test_noalloc_rejects_images_beyond_its_scratch():
    import torch
    from paper_2406_16302_gb300 import rp
    _, _, sc, ed = _scene(2048, 1024)
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RPError) as e:
        rp.rp_render_residual_f32_noalloc(sc, ed, 1, 1, out)
    assert e.value.status == 1
    assert "RP_NOALLOC_MAX_PIXELS" in str(e.value)
