"""Pins of the oracle's learned-proposal arithmetic (technique (3)'s
light-side direction): the von Mises-Fisher density and sampler against
closed forms, the input encoding against known angles, the integer network's
wiring and rounding against hand-built networks, the float network's
gradient against finite differences, and unbiasedness of the guided
estimator against correlated path tracing."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2406_16302_gb300 import scenes
import helpers as H

KAPPAS = [0.02, 1.0, 30.0, 490.0]


def _frame(mu):
    t, b = oracle.tangent_frame(mu)
    return t, b


@pytest.mark.parametrize("kappa", KAPPAS)
def test_vmf_density_integrates_to_one(kappa):
    mu = np.array([0.3, -0.5, 0.8]); mu /= np.linalg.norm(mu)
    t, _ = _frame(mu)

    def f(c):   # density at angle arccos(c) from mu, times the ring 2 pi
        w = c * mu + math.sqrt(max(0.0, 1.0 - c * c)) * t
        return 2.0 * math.pi * oracle.vmf_pdf(mu, kappa, w)
    # split near c = 1 where a sharp lobe lives
    edges = [-1.0, 0.0, 1.0 - 10.0 / kappa if kappa > 10 else 0.5, 1.0]
    total = sum(integrate.quad(f, a, b, limit=200, epsabs=1e-13)[0] for a, b in zip(edges, edges[1:]))
    assert abs(total - 1.0) < 1e-7


@pytest.mark.parametrize("kappa", KAPPAS)
def test_vmf_sampler_matches_closed_form_cdf(kappa):
    """The cosine c = mu.w of a vMF sample has the CDF
    (exp(kappa (c - 1)) - exp(-2 kappa)) / (1 - exp(-2 kappa)) on [-1, 1];
    the azimuth about mu is uniform."""
    mu = np.array([-0.2, 0.9, 0.1]); mu /= np.linalg.norm(mu)
    t, b = _frame(mu)
    n = 4000
    rng = np.random.default_rng(7)
    u1 = (np.arange(n) + rng.random(n)) / n
    u2 = rng.permutation(n) / n + rng.random(n) / n
    ws = np.array([oracle.vmf_sample(mu, kappa, a, c) for a, c in zip(u1, u2)])
    assert np.allclose(np.linalg.norm(ws, axis=1), 1.0, atol=1e-12)
    c = np.sort(ws @ mu)
    cdf = (np.exp(kappa * (c - 1.0)) - math.exp(-2 * kappa)) / -math.expm1(-2 * kappa)
    ks = np.max(np.abs(cdf - (np.arange(n) + 0.5) / n))
    assert ks < 2.0 / n + 1e-9                 # stratified: far tighter than iid
    phi = np.arctan2(ws @ b, ws @ t) % (2 * math.pi)
    hist = np.histogram(phi, bins=16, range=(0, 2 * math.pi))[0]
    assert np.all(np.abs(hist - n / 16) < 6 * math.sqrt(n / 16))


def test_encoding_closed_form_values():
    box = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], dtype=np.float32)
    p = np.array([1.0 / 6.0, 0.0, 0.5])
    n = np.array([0.0, 1.0, 0.0])
    m = oracle.guide_encode(box, p, n)
    # x = 1/6: sin(pi/6) = 1/2, cos(pi/6) = sqrt(3)/2; sin(pi/3), cos(pi/3) ...
    assert m[0] == 64 and m[1] == round(128 * math.sqrt(3) / 2)
    assert m[2] == round(128 * math.sqrt(3) / 2) and m[3] == 64
    # y = 0: sin 0 = 0 and cos 0 = 1 -> 128, clamped to 127, for every octave
    assert np.all(m[12:24:2] == 0) and np.all(m[13:24:2] == 127)
    # z = 1/2: sin(pi/2) = 1, cos(pi/2) = 0, then sin(pi) = 0, cos(pi) = -1
    assert m[24] == 127 and m[25] == 0 and m[26] == 0 and m[27] == -127
    # normal (0, 1, 0): n_y = 1 -> sin(2^f pi) = 0, cos(2^f pi) = -1 then +1 ...
    assert m[48] == 0 and m[49] == -127 and m[51] == 127
    # raw coordinates and the constant
    assert list(m[72:75]) == [21, 0, 64] and list(m[75:78]) == [0, 127, 0]
    assert m[78] == 127 and m[79] == 0


def test_encoding_octave_two():
    box = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], dtype=np.float32)
    m = oracle.guide_encode(box, np.array([1.0 / 6.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]))
    # x = 1/6, octave f = 2: angle 4 pi / 6 = 2 pi / 3: sin = sqrt(3)/2, cos = -1/2
    assert m[4] == round(128 * math.sqrt(3) / 2) and m[5] == -64


def _identity_net(perm, out_exp, gain=2):
    W = np.zeros(20480, dtype=np.int32)
    off = [0, 5120, 9216, 13312, 17408]
    for o in range(64):
        W[off[0] + o * 80 + perm[o]] = 1
        for l in (1, 2, 3):
            W[off[l] + o * 64 + o] = 1
    for o in range(48):
        W[off[4] + o * 64 + o] = gain
    return W, np.zeros(4, dtype=np.int32), out_exp


def test_integer_network_wiring():
    """Layer 0 row o selects input perm[o]; hidden layers are identities; the
    output layer doubles: out[o] = 2 max(0, m[perm[o]]) / 2^e.  A transposed
    weight matrix or a dropped ReLU fails."""
    rng = np.random.default_rng(3)
    perm = rng.permutation(80)[:64]
    W, sh, e = _identity_net(perm, 3)
    m = rng.integers(-127, 128, size=(5, 80)).astype(np.int32)
    out = oracle.guide_forward(W, sh, e, m)
    want = 2.0 * np.maximum(m[:, perm[:48]], 0) / 8.0
    assert np.array_equal(out, want)


def test_integer_network_rounding_and_clamp():
    """Requantisation is round-half-even of z / 2^shift, clamped to [0, 255]."""
    W = np.zeros(20480, dtype=np.int32)
    off = [0, 5120, 9216, 13312, 17408]
    weights = [1, 3, 5, -1, 2, 4]
    for o, w in enumerate(weights):
        W[off[0] + o * 80 + 78] = w            # the constant feature 127
        for l in (1, 2, 3):
            W[off[l] + o * 64 + o] = 1
        W[off[4] + o * 64 + o] = 1
    m = np.zeros((1, 80), dtype=np.int32); m[0, 78] = 127
    out = oracle.guide_forward(W, [1, 0, 0, 0], 0, m)[0]
    # 127 / 2 = 63.5 -> 64; 381 / 2 = 190.5 -> 190; 635 / 2 = 317.5 -> 318 -> 255;
    # -127 -> 0 (ReLU); 254 / 2 = 127; 508 / 2 = 254
    assert list(out[:6]) == [64, 190, 255, 0, 127, 254]


def _rand_batch(rows, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(rows, 80)); x[:, 78] = 127 / 128; x[:, 79] = 0
    om = rng.normal(size=(rows, 3)); om /= np.linalg.norm(om, axis=1, keepdims=True)
    wt = rng.uniform(0.1, 2.0, size=rows)
    return x, om, wt


def test_float_network_gradient_matches_finite_differences():
    W = scenes.random_float_guide(5, gain=0.9)
    x, om, wt = _rand_batch(6, 11)
    loss, g = oracle.mlp_loss_grad(W, x, om, wt)
    rng = np.random.default_rng(2)
    offs = [0, 5120, 9216, 13312, 17408, 20480]
    idx = np.concatenate([rng.integers(offs[l], offs[l + 1], size=10) for l in range(5)])
    h = 1e-6
    for i in idx:
        Wp = W.copy(); Wp[i] += h
        Wm = W.copy(); Wm[i] -= h
        fd = (oracle.mlp_loss_grad(Wp, x, om, wt, grad=False)
              - oracle.mlp_loss_grad(Wm, x, om, wt, grad=False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, g[i])


def test_float_network_matches_integer_network_on_exact_grid():
    """With two +-1 weights per row, inputs in {0, 1, 2} and zero shifts no
    activation leaves [0, 255] and nothing is rounded: the integer network
    and the float network (the training path) must agree exactly."""
    rng = np.random.default_rng(4)
    W = np.zeros(20480, dtype=np.int32)
    offs = [0, 5120, 9216, 13312, 17408]
    dims = [(64, 80), (64, 64), (64, 64), (64, 64), (48, 64)]
    for l, (o, i) in enumerate(dims):
        for r in range(o):
            cols = rng.choice(i, size=2, replace=False)
            W[offs[l] + r * i + cols] = rng.choice([-1, 1], size=2)
    m = rng.integers(0, 3, size=(16, 80)).astype(np.int32)
    out_i = oracle.guide_forward(W, [0, 0, 0, 0], 0, m)
    out_f = oracle.mlp_forward(W.astype(np.float64), m.astype(np.float64))
    assert np.array_equal(out_i, out_f)
    assert np.any(out_i != 0)


GUIDED_CASES = [
    ("cfg1_box_sphere", {"width": 8, "height": 8, "max_depth": 6}),      # motion: mapping on
    ("cfg2_box_blob", {"width": 8, "height": 8, "max_depth": 5, "blob_level": 2}),  # material
]


@pytest.mark.parametrize("builder,kw", GUIDED_CASES)
def test_guided_residual_matches_correlated_path_tracing(builder, kw):
    """Any proposal network keeps the residual estimator unbiased: guided
    technique (3) with the other techniques against correlated path
    tracing."""
    K = 24
    corr = H.run_many("corr", builder, kw, range(1000, 1000 + K), 1024)
    res = H.run_many("res", builder, kw, range(5000, 5000 + K), 128, guide=(3, {}))
    z, zs = H.zscores(res, corr)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
    assert np.abs(z).max() < 6.0


def test_guided_technique_three_alone_is_unbiased():
    """Technique (3) alone estimates its own domain; the guided and the
    cosine-sampled versions are two estimators of the same image."""
    kw = {"width": 8, "height": 8, "max_depth": 6}
    K = 24
    plain = H.run_many("res", "cfg1_box_sphere", kw, range(7000, 7000 + K), 256, mask=4)
    guided = H.run_many("res", "cfg1_box_sphere", kw, range(8000, 8000 + K), 256, mask=4,
                        guide=(5, {}))
    z, zs = H.zscores(guided, plain)
    assert abs(zs) < 4.0, zs
    assert np.sqrt((z ** 2).mean()) < 1.4
