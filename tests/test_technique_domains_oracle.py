"""Each technique alone estimates the residual over its own domain (Sec. 4.1
and the per-technique rows of the paper's technique figure).

With only technique t enabled, the balance heuristic keeps only t's
densities, so the estimator's mean is the integral of f2 - f1 over the paths
with a dynamic vertex where t samples it: (1) next to the emitter, (2) next
to the sensor, (3) in between.  The independent reference is plain path
tracing of both frames with the same seeds, each path counted only when it
lies in that domain (a filter on the path, no densities of the techniques).
On a material edit the geometry, hence the domain, is the same in both
frames and no path is rejected, so the two estimate the same image.
"""
import numpy as np
import pytest

import helpers as H

KW = {"width": 8, "height": 8, "max_depth": 5, "blob_level": 2}


@pytest.mark.parametrize("tech,bit", [(1, 1), (2, 2), (3, 4)])
def test_single_technique_matches_its_domain(tech, bit):
    K = 24
    ref = H.run_many("corr", "cfg2_box_blob", KW, range(9000, 9000 + K), 1024, domain=bit)
    res = H.run_many("res", "cfg2_box_blob", KW, range(9500, 9500 + K), 128, mask=bit)
    assert np.abs(ref).sum() > 0 and np.abs(res).sum() > 0
    z, zs = H.zscores(res, ref)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
    assert np.abs(z).max() < 6.0


def test_domains_partition_the_dynamic_paths():
    """The three domains together hold every path through the object once:
    on paths with a single dynamic vertex the filtered images add up to the
    filter with all three bits (same seeds, so the sums are exact up to
    rounding)."""
    import oracle
    from paper_2406_16302_gb300 import scenes as S
    scene, edit = S.cfg2_box_blob(**KW)
    o = oracle.Oracle(scene, edit)
    parts = [o.render_primal(2, 64, 5, domain=b) for b in (1, 2, 4)]
    union = o.render_primal(2, 64, 5, domain=7)
    total = o.render_primal(2, 64, 5)
    # a path with two dynamic vertices in different domains counts in both
    # parts but once in the union, so the parts can only exceed the union
    assert np.all(sum(parts) >= union - 1e-12)
    assert np.all(union <= total + 1e-12)
    assert union.sum() > 0
    # the blob is small: most paths through it touch it once, so the overlap
    # is a small fraction
    assert sum(parts).sum() <= 1.2 * union.sum()
