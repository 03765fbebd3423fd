"""rp_render_residual_f32_noalloc, the entry point for callers that cannot let
the library allocate device memory (hosts with their own memory pools, hard
memory caps, or no allocation allowed after start-up).  It must give the same
image as rp_render_residual_f32, whose scratch image is cudaMalloc'd, on
consecutive calls (the fixed scratch array keeps the previous call's sums
and has to be cleared each time).  Kept in a file of its own that pytest
collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_2406_16302_gb300 import build, rp, scenes
    build.build()
    scene, edit = scenes.cfg1_box_sphere(width=32, height=32)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    for call in range(2):
        ref = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        rp.rp_render_residual_f32(sc, ed, 4, 17, ref)
        out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        rp.rp_render_residual_f32_noalloc(sc, ed, 4, 17, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.abs(r).max() > 0
        assert np.allclose(o, r, rtol=1e-5, atol=1e-6 * np.abs(r).max()), call


def test_noalloc_rejects_images_beyond_its_scratch():
    import torch
    from paper_2406_16302_gb300 import build, rp, scenes
    build.build()
    scene, edit = scenes.cfg1_box_sphere(width=2048, height=1024)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RPError) as e:
        rp.rp_render_residual_f32_noalloc(sc, ed, 1, 1, out)
    assert e.value.status == 1
    assert "RP_NOALLOC_MAX_PIXELS" in str(e.value)
