"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a published value, a closed form, an
independent estimator of the same integral, brute force or an invariant that
a plausible mistake (dropped term, wrong sign or index, swapped operand)
would break.  CPU only.
"""
import os

import numpy as np
import pytest

import helpers as H
from paper_2406_16302_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- random numbers --------------------------------------------------------

def test_philox_known_answers(oracle_mod):
    """Philox4x32-10 against the authors' published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(w, 16) for w in r]
        out = oracle_mod.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


# --- intersection ----------------------------------------------------------

@pytest.mark.parametrize("builder,kw", [("cfg1_box_sphere", {}),
                                        ("cfg2_box_blob", {"blob_level": 3})])
def test_bvh_closest_hit_matches_brute_force(oracle_mod, builder, kw):
    scene, edit = getattr(S, builder)(width=16, height=16, **kw)
    fast = oracle_mod.Oracle(scene, edit)
    slow = oracle_mod.Oracle(scene, edit, brute_force=True)
    rng = np.random.RandomState(7)
    o = rng.uniform(-0.95, 0.95, size=(3000, 3))
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for frame in (1, 2):
        t1, p1, u1, v1 = fast.closest_hit(frame, o, d)
        t2, p2, u2, v2 = slow.closest_hit(frame, o, d)
        assert np.array_equal(p1, p2)
        hit = p1 >= 0
        assert hit.mean() > 0.7          # the box front is open
        assert np.allclose(t1[hit], t2[hit], rtol=1e-12, atol=0)
        assert np.allclose(u1[hit], u2[hit], atol=1e-12)


def test_closest_hit_on_analytic_planes(oracle_mod):
    """Rays from inside the box hit the wall planes at the analytic distance."""
    scene, edit = S.cfg1_box_sphere(width=8, height=8)
    o = oracle_mod.Oracle(scene, edit)
    orig = np.array([[0.8, 0.5, 0.7]] * 5)
    dirs = np.array([[0, -1, 0], [0, 0, -1], [-1, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    t, prim, _, _ = o.closest_hit(1, orig, dirs)
    assert np.allclose(t, [1.5, 1.7, 1.8, 0.2, 0.5], rtol=1e-12)


# --- BSDF sampling and densities -------------------------------------------

MATS = [S.material(S.LAMBERT, (0.7, 0.5, 0.3)),
        S.material(S.GGX, alpha=0.3, f0=(0.04, 0.04, 0.04)),
        S.material(S.GGX, alpha=0.08, f0=(0.9, 0.6, 0.3))]


def _hemisphere_grid(m=400):
    ct = (np.arange(m) + 0.5) / m
    ph = (np.arange(2 * m) + 0.5) / (2 * m) * 2 * np.pi
    C, P = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - C * C)
    w = np.stack([st * np.cos(P), st * np.sin(P), C], -1).reshape(-1, 3)
    dw = (1.0 / m) * (2 * np.pi / (2 * m))
    return w, dw


@pytest.mark.parametrize("mi", range(len(MATS)))
def test_bsdf_energy_and_reciprocity(oracle_mod, mi):
    m = MATS[mi]
    n = np.array([0.0, 0.0, 1.0])
    w, dw = _hemisphere_grid(200)
    for theta in (0.0, 0.6, 1.2):
        wi = np.array([np.sin(theta), 0.0, np.cos(theta)])
        alb = np.zeros(3)
        for wo in w[::7]:
            rho, _ = oracle_mod.bsdf(m, n, wi, wo)
            rho2, _ = oracle_mod.bsdf(m, n, wo, wi)
            assert np.allclose(rho, rho2, rtol=1e-12)
            alb += rho * wo[2] * dw * 7
        if mi == 0:
            assert np.allclose(alb, m[1:4], rtol=2e-3)    # Lambert albedo exact
        else:
            assert np.all(alb <= 1.0 + 1e-2)


@pytest.mark.parametrize("mi", range(len(MATS)))
def test_sampling_matches_pdf(oracle_mod, mi):
    """Histogram of sampled directions against the pdf integrated per bin;
    the sampler also round-trips through its inverse."""
    m = MATS[mi]
    n = np.array([0.0, 0.0, 1.0])
    wc = np.array([np.sin(0.5), 0.0, np.cos(0.5)])
    rng = np.random.RandomState(mi)
    nb = 8
    counts = np.zeros((nb, nb))
    ns = 40000
    fails = 0
    for u1, u2 in rng.uniform(size=(ns, 2)):
        wo, ub = oracle_mod.bsdf_sample(m, n, wc, u1, u2)
        if wo is None:
            fails += 1
            continue
        assert abs(np.linalg.norm(wo) - 1) < 1e-12
        assert np.allclose(ub, [u1, u2], atol=1e-9) or abs(abs(ub[1] - u2) - 1) < 1e-9
        i = min(int(wo[2] ** 2 * nb), nb - 1)       # bins uniform in cos^2
        j = min(int((np.arctan2(wo[1], wo[0]) / (2 * np.pi) % 1.0) * nb), nb - 1)
        counts[i, j] += 1
    # expected counts from quadrature of the pdf
    w, dw = _hemisphere_grid(300)
    pdf = np.array([oracle_mod.bsdf(m, n, wc, wo)[1] for wo in w])
    ii = np.minimum((w[:, 2] ** 2 * nb).astype(int), nb - 1)
    jj = np.minimum(((np.arctan2(w[:, 1], w[:, 0]) / (2 * np.pi) % 1.0) * nb).astype(int), nb - 1)
    expect = np.zeros((nb, nb))
    np.add.at(expect, (ii, jj), pdf * dw)
    assert abs(expect.sum() + fails / ns - 1.0) < 5e-3       # pdf mass + failures = 1
    e = expect * ns
    sel = e > 20
    chi2 = ((counts[sel] - e[sel]) ** 2 / e[sel]).sum()
    dof = sel.sum()
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


def test_tangent_frames_orthonormal(oracle_mod):
    rng = np.random.RandomState(3)
    normals = list(np.eye(3)) + list(-np.eye(3)) + list(rng.normal(size=(200, 3)))
    for n in normals:
        n = n / np.linalg.norm(n)
        t, b = oracle_mod.tangent_frame(n)
        M = np.stack([t, b, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(t, b), n, atol=1e-12)


# --- primal path integral --------------------------------------------------

@pytest.mark.parametrize("albedo,depth", [(0.5, 4), (0.8, 3), (0.3, 6)])
def test_white_furnace(oracle_mod, albedo, depth):
    """Closed emissive box: every pixel is L * sum_{j<D} a^j exactly in
    expectation (Eq. pathIntegral with emission on every surface)."""
    scene, edit = S.furnace_box(albedo=albedo, radiance=1.0, max_depth=depth)
    o = oracle_mod.Oracle(scene, edit)
    reps = np.array([o.render_primal(1, 16, 100 + i) for i in range(32)])
    expect = sum(albedo ** j for j in range(depth))
    mean = reps.mean(0)
    se = reps.std(0, ddof=1) / np.sqrt(len(reps))
    z = (mean - expect) / se
    assert np.abs(z).max() < 5.0
    zg = (reps.mean() - expect) / (reps.mean(axis=(1, 2, 3)).std(ddof=1) / np.sqrt(len(reps)))
    assert abs(zg) < 4.0


def test_polygon_irradiance_helper():
    """The closed form used below against direct quadrature."""
    scene, edit = S.wall_and_quad()
    light_ids = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    t0, t1 = scene.static_triangles[light_ids[0]], scene.static_triangles[light_ids[1]]
    poly = scene.static_vertices[[t0[0], t0[1], t0[2], t1[2]]].astype(float)
    for x in ([0.3, -0.2, 0.0], [-0.8, 0.9, 0.0], [0.0, -0.7, 0.5]):
        x = np.array(x)
        e1 = H.polygon_irradiance(x[None], np.array([0, 0, 1.0]), poly, 10.0)[0]
        e2 = H.polygon_irradiance_quadrature(x, np.array([0, 0, 1.0]), poly, 10.0)
        assert abs(e1 / e2 - 1) < 1e-4


@pytest.mark.parametrize("frame", [1, 2])
def test_direct_lighting_closed_form(oracle_mod, frame):
    """Max depth 2 on the wall-and-quad scene equals the closed-form
    polygon irradiance image."""
    scene, edit = S.wall_and_quad()
    ref = H.wall_and_quad_closed_form(scene, edit, frame)
    o = oracle_mod.Oracle(scene, edit)
    reps = np.array([o.render_primal(frame, 16, 10 + i) for i in range(32)])
    z = (reps.mean(0) - ref) / (reps.std(0, ddof=1) / np.sqrt(len(reps)) + 1e-12)
    assert np.abs(z).max() < 5.0
    assert abs(reps.mean() / ref.mean() - 1) < 5e-3


# --- residual estimator ----------------------------------------------------

def test_residual_closed_form_moving_quad(oracle_mod):
    """Residual of the moving quad (techniques 1 and 7, camera-direction and
    object-transform mappings, two-way MIS) against the difference of the two
    closed-form images."""
    scene, edit = S.wall_and_quad()
    # 128 x 128 film samples per pixel: the camera-direction mapping makes the
    # estimate at the quad's silhouette precise enough to expose the
    # discretisation error of a coarser reference
    ref = (H.wall_and_quad_closed_form(scene, edit, 2, sub=128)
           - H.wall_and_quad_closed_form(scene, edit, 1, sub=128))
    reps = H.run_many("res", "wall_and_quad", {}, range(500, 516), 64)
    se = reps.std(0, ddof=1) / np.sqrt(len(reps))
    mean = reps.mean(0)
    nz = se > 0
    z = (mean[nz] - ref[nz]) / se[nz]
    assert np.abs(z).max() < 5.5
    assert np.sqrt((z ** 2).mean()) < 1.5
    # pixels the motion cannot affect get exactly nothing
    assert np.all(mean[~nz] == 0.0)
    assert np.all(np.abs(ref[~nz]) < 1e-12)
    zs = (reps.reshape(len(reps), -1).sum(1).mean() - ref.sum()) / (
        reps.reshape(len(reps), -1).sum(1).std(ddof=1) / np.sqrt(len(reps)))
    assert abs(zs) < 4.0


@pytest.mark.parametrize("builder,kw", [("cfg1_box_sphere", {"width": 8, "height": 8,
                                                               "max_depth": 5}),
                                        ("cfg2_box_blob", {"width": 8, "height": 8,
                                                           "max_depth": 5, "blob_level": 2})])
def test_identity_edit_is_exactly_zero(oracle_mod, builder, kw):
    """No motion and no material change: every sample is exactly 0."""
    scene, edit = getattr(S, builder)(**kw)
    o = oracle_mod.Oracle(scene, S.identity_edit(edit))
    img = o.render_residual(4, 11)
    assert np.all(img == 0.0)
    for tech in (1, 2, 3, 7):
        for frame in (1, 2):
            rec = o.dump(tech, frame, 4, 11, 0, 256)
            assert np.all(rec["va"] + rec["vb"] == 0.0)
    rec = o.dump(7, 2, 4, 11, 0, 256)
    assert len(rec) == 0 or np.all(rec["status"] == 0)


RESIDUAL_CASES = [
    ("cfg1_box_sphere", {"width": 8, "height": 8, "max_depth": 4}, 15),
    ("cfg1_box_sphere", {"width": 8, "height": 8, "max_depth": 6}, 15),
    ("cfg1_box_sphere", {"width": 8, "height": 8, "max_depth": 6}, 8 | 4),   # T3 + T7
    ("cfg2_box_blob", {"width": 8, "height": 8, "max_depth": 5, "blob_level": 2}, 15),
]


@pytest.mark.parametrize("builder,kw,mask", RESIDUAL_CASES)
def test_residual_matches_correlated_path_tracing(builder, kw, mask):
    """The residual estimator (any technique subset that includes path
    tracing with rejection) and correlated path tracing (the same primary
    samples in both frames) are independent unbiased estimators of I2 - I1."""
    K = 24
    corr = H.run_many("corr", builder, kw, range(1000, 1000 + K), 1024)
    res = H.run_many("res", builder, kw, range(3000, 3000 + K), 128, mask=mask)
    z, zs = H.zscores(res, corr)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
    assert np.abs(z).max() < 6.0


def test_residual_matches_independent_renders():
    """The plain definition: I2 - I1 from two independent primal renders."""
    kw = {"width": 6, "height": 6, "max_depth": 4}
    K = 24
    p2 = H.run_many("p2", "cfg1_box_sphere", kw, range(100, 100 + K), 2048)
    p1 = H.run_many("p1", "cfg1_box_sphere", kw, range(200, 200 + K), 2048)
    res = H.run_many("res", "cfg1_box_sphere", kw, range(300, 300 + K), 128)
    # difference of independent renders as K paired repeats
    z, zs = H.zscores(res, p2 - p1)
    assert abs(zs) < 4.0
    assert np.sqrt((z ** 2).mean()) < 1.4


@pytest.mark.parametrize("tech", [1, 2, 3, 7])
@pytest.mark.parametrize("frame", [1, 2])
@pytest.mark.parametrize("d_min", [None, 100.0])
def test_mapping_is_a_bijection_with_correct_jacobian(oracle_mod, tech, frame, d_min):
    """Every accepted pair maps back onto its base path (two-way mapping,
    Sec. 5), the two Jacobians multiply to one, and the per-vertex replay
    Jacobian equals finite differences of the mapping.  d_min = 100 disables
    reconnection so that every walk vertex is replayed."""
    scene, edit = S.cfg1_box_sphere(width=16, height=16, max_depth=6)
    if d_min is not None:
        scene.d_min = d_min
    o = oracle_mod.Oracle(scene, edit)
    r = o.check_mapping(tech, frame, 16, 5, 0, 4096)
    assert r["pairs"] > 50
    assert r["bad_inverse"] == 0
    assert r["max_pos_err"] < 1e-9
    assert r["max_jac_err"] < 1e-7
    if d_min is not None and tech in (1, 2, 3):
        assert r["fd_checked"] > 20
    if r["fd_checked"]:
        assert r["max_fd_err"] < 1e-5, r


def test_rotation_edit_mapping(oracle_mod):
    """Same checks with a rotating, translating object and glossy surfaces."""
    scene, edit = S.cfg1_box_sphere(width=16, height=16, max_depth=6)
    mats = scene.materials.copy()
    mats[0] = S.material(S.GGX, alpha=0.4, f0=(0.6, 0.6, 0.6))      # glossy grey walls
    scene.materials = mats
    c = edit.M1[:, 3].astype(np.float64)
    edit.M2 = S.rotate_y_translate(25.0, c + np.array([0.05, 0.02, 0.0]))
    o = oracle_mod.Oracle(scene, edit)
    total = 0
    for tech in (1, 2, 3, 7):
        for frame in (1, 2):
            r = o.check_mapping(tech, frame, 16, 9, 0, 4096)
            total += r["pairs"]
            assert r["bad_inverse"] == 0
            assert r["max_pos_err"] < 1e-9
            assert r["max_jac_err"] < 1e-7
            if r["fd_checked"]:
                assert r["max_fd_err"] < 1e-5, r
    assert total > 200


@pytest.mark.parametrize("alpha", [0.05, 0.3, 0.8])
def test_bsdf_textbook_values(oracle_mod, alpha):
    """Closed forms of the two BSDFs (Lambert; Walter et al. 2007 GGX with
    Smith masking and Schlick Fresnel): at normal incidence and normal exit
    D = 1 / (pi alpha^2), G = 1, F = F0, so f = F0 / (4 pi alpha^2); Lambert
    is rho / pi everywhere above the surface."""
    n = np.array([0.0, 0.0, 1.0])
    f0 = np.array([0.04, 0.5, 0.9])
    rho, _ = oracle_mod.bsdf(S.material(S.GGX, alpha=alpha, f0=tuple(f0)), n, n, n)
    np.testing.assert_allclose(rho, f0 / (4 * np.pi * alpha ** 2), rtol=1e-6)
    lam = S.material(S.LAMBERT, (0.7, 0.5, 0.3))
    wi = np.array([np.sin(0.4), 0.0, np.cos(0.4)])
    wo = np.array([0.0, np.sin(1.1), np.cos(1.1)])
    rho, _ = oracle_mod.bsdf(lam, n, wi, wo)
    np.testing.assert_allclose(rho, np.array([0.7, 0.5, 0.3]) / np.pi, rtol=1e-6)
    # below the surface nothing is reflected
    rho, _ = oracle_mod.bsdf(lam, n, wi, -wo)
    assert np.all(rho == 0)
