"""Online training of the learned proposal of technique (3) on a synthetic
scene: renders with the guide attached (which gathers the samples), one
training step after each render, printing the weighted loss.

    python -m paper_2406_16302_gb300.train_guide --scene box_blob_side_light --size 256 \\
        --spp 8 --iters 4
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", default="box_blob_side_light",
                    choices=["box_blob_side_light", "cfg2_box_blob"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--spp", type=int, default=8)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--batch", type=int, default=1 << 20)
    ap.add_argument("--lr", type=float, default=1e-2)
    args = ap.parse_args(argv)
    import torch
    from . import build, rp, scenes
    build.build()
    rp.lib()
    scene, edit = getattr(scenes, args.scene)(width=args.size, height=args.size, max_depth=8,
                                               blob_level=5)
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    guide = rp.Guide(scenes.guide_box(scene.dyn_vertices), batch=args.batch, seed=1)
    rp.rp_scene_set_guide(sc, guide)
    for it in range(args.iters):
        rp.render_residual(sc, ed, args.spp, 100 + it, tech_mask=4)
        print("loss", rp.rp_guide_train_step(guide, lr=args.lr), flush=True)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
