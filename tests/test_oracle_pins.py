"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each pin is one of: a hand-worked closed form (tests/hand_cases.py), brute
force on tiny inputs, a library routine, or an invariant the paper states
(Eq. 5 order independence, Table 4, the empty set of Eq. 5).  The mutation
tests at the end plant plausible mistakes in a copy of the oracle and check
that some pin catches each one.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.special import expit

import oracle
from oracle import glassnet_oracle as O
from gen import synth
from tests import hand_cases as hc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_weights(seed, bias="uniform", H=4, Z=3):
    """Random model with small widths but the real channel counts."""
    rng = np.random.default_rng(seed)
    shapes = {
        "F1": (Z, synth.SCENE_DIM), "F2": (Z, Z), "phi1": (H, synth.TBUF_CHANNELS + Z),
        "phi2": (H, H), "rho": (H, 2 * H), "B1": (H, synth.GBUF_CHANNELS + H + Z),
        "B2": (H, H), "R1": (H, H), "R2": (3, H),
    }
    w = {}
    for k, (o, i) in shapes.items():
        W = rng.standard_normal((o, i)).astype(np.float32)
        b = (rng.uniform(-0.5, 0.5, o) if bias == "uniform" else np.zeros(o)).astype(np.float32)
        w[k] = (W, b)
    return w


# ---------------------------------------------------------------- primitives

def test_linear_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    for (n, i, o) in [(1, 1, 1), (3, 5, 2), (4, 7, 6)]:
        x = rng.standard_normal((n, i))
        W = rng.standard_normal((o, i))
        b = rng.standard_normal(o)
        got = O.linear(x, W, b)
        for r in range(n):
            for j in range(o):
                acc = float(b[j])
                for k in range(i):
                    acc += float(W[j, k]) * float(x[r, k])
                assert abs(got[r, j] - acc) < 1e-12


def test_relu_special_values():
    np.testing.assert_array_equal(O.relu([-2.0, -0.0, 0.0, 3.5]), [0.0, 0.0, 0.0, 3.5])


def test_sigmoid_closed_forms_and_library():
    assert O.sigmoid(0.0) == 0.5
    assert abs(O.sigmoid(math.log(3.0)) - 0.75) < 1e-15
    x = np.linspace(-30, 30, 601)
    np.testing.assert_allclose(O.sigmoid(x) + O.sigmoid(-x), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.sigmoid(x), expit(x), rtol=1e-14, atol=0)
    assert O.sigmoid(-1000.0) == 0.0 and O.sigmoid(1000.0) == 1.0


# ------------------------------------------------------------ hand-worked cases

def test_hand_scene_encoder():
    np.testing.assert_array_equal(O.scene_encoder(hc.W, hc.SCENE), hc.SIGMA)


def test_hand_per_layer_network():
    np.testing.assert_array_equal(O.per_layer_h(hc.W, hc.LAYER_A, hc.SIGMA), [5.0, 0.0])
    np.testing.assert_array_equal(O.per_layer_h(hc.W, hc.LAYER_B, hc.SIGMA), [5.0, 2.0])


def test_hand_pool_two_layers():
    V = np.stack([O.per_layer_h(hc.W, hc.LAYER_A, hc.SIGMA),
                  O.per_layer_h(hc.W, hc.LAYER_B, hc.SIGMA)])
    np.testing.assert_array_equal(O.set_pool(V), hc.POOL_TWO_LAYERS)
    assert O.set_pool(np.zeros((0, 2))) is None


@pytest.mark.parametrize("layers,logits", [
    ([hc.LAYER_A], hc.LOGITS_ONE_LAYER),
    ([hc.LAYER_A, hc.LAYER_B], hc.LOGITS_TWO_LAYERS),
    ([hc.LAYER_B, hc.LAYER_A], hc.LOGITS_TWO_LAYERS),
    ([], hc.LOGITS_NO_LAYER),
])
def test_hand_render_pixel(layers, logits):
    sigma = O.scene_encoder(hc.W, hc.SCENE)
    L = np.array(layers, np.float32).reshape(len(layers), 2)
    got = O.render_pixel(hc.W, sigma, hc.G, L)
    np.testing.assert_allclose(got, expit(logits), rtol=1e-15, atol=0)


@pytest.mark.parametrize("K", [2, 3, 5])
def test_hand_render_frame_matches_closed_forms(K):
    """2x2 frame through the vectorised path; K > c checks the mean divides by c."""
    counts = np.array([[1, 2], [0, 2]], np.uint8)
    gbuf = np.broadcast_to(hc.G[:, None, None], (2, 2, 2)).copy()
    tbuf = np.full((K, 2, 2, 2), np.nan, np.float32)
    tbuf[0, :, 0, 0] = hc.LAYER_A
    tbuf[0, :, 0, 1] = hc.LAYER_A
    tbuf[1, :, 0, 1] = hc.LAYER_B
    tbuf[0, :, 1, 1] = hc.LAYER_B
    tbuf[1, :, 1, 1] = hc.LAYER_A
    rgb = O.render_frame(hc.W, hc.SCENE, gbuf, tbuf, counts)
    np.testing.assert_allclose(rgb[:, 0, 0], expit(hc.LOGITS_ONE_LAYER), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 0, 1], expit(hc.LOGITS_TWO_LAYERS), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 1, 0], expit(hc.LOGITS_NO_LAYER), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 1, 1], expit(hc.LOGITS_TWO_LAYERS), rtol=1e-15)


# ------------------------------------------------------------------- invariants

def _table4_bound():
    with open(os.path.join(GOLDEN, "table4_order_invariance.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return max(float(r[3]) for r in rows)


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5])
def test_permutation_invariance_every_order(c):
    """Eq. 5 / Table 4: every order of the valid layers gives the same output."""
    bound = _table4_bound()
    assert bound == 0.0
    w = _tiny_weights(10 + c)
    rng = np.random.default_rng(c)
    sigma = O.scene_encoder(w, rng.standard_normal(synth.SCENE_DIM))
    g = rng.standard_normal(synth.GBUF_CHANNELS)
    L = rng.standard_normal((c, synth.TBUF_CHANNELS))
    ref = O.render_pixel(w, sigma, g, L)
    for perm in itertools.permutations(range(c)):
        got = O.render_pixel(w, sigma, g, L[list(perm)])
        assert np.max(np.abs(got - ref)) <= bound


def test_canonical_sum_agrees_with_plain_sum():
    rng = np.random.default_rng(7)
    V = rng.standard_normal((6, 9)) * 10
    pool = O.set_pool(V)
    np.testing.assert_allclose(pool[9:], V.sum(axis=0) / 6, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(pool[:9], V.max(axis=0))


def test_duplication_invariance_of_max_mean():
    """max and mean of {a, b} equal those of {a, a, b, b}."""
    rng = np.random.default_rng(3)
    w = _tiny_weights(3)
    sigma = O.scene_encoder(w, rng.standard_normal(synth.SCENE_DIM))
    g = rng.standard_normal(synth.GBUF_CHANNELS)
    a, b = rng.standard_normal((2, synth.TBUF_CHANNELS))
    one = O.render_pixel(w, sigma, g, np.stack([a, b]))
    two = O.render_pixel(w, sigma, g, np.stack([a, a, b, b]))
    np.testing.assert_allclose(one, two, rtol=0, atol=1e-14)


def test_empty_set_equals_independent_opaque_only_path():
    rng = np.random.default_rng(4)
    w = _tiny_weights(4)
    s = rng.standard_normal(synth.SCENE_DIM)
    sigma = O.scene_encoder(w, s)
    gb = rng.standard_normal((5, synth.GBUF_CHANNELS))
    ref = O.render_opaque_only(w, sigma, gb)
    for i in range(5):
        got = O.render_pixel(w, sigma, gb[i], np.zeros((0, synth.TBUF_CHANNELS)))
        np.testing.assert_allclose(got, ref[i], rtol=0, atol=1e-14)


def test_invalid_slots_never_read():
    w = _tiny_weights(5)
    f = synth.make_frame(6, 5, 4, counts="uniform", seed=5)
    a = O.render_frame(w, synth.make_scene(5), f.gbuf, f.tbuf, f.counts)
    t2 = f.tbuf.copy()
    c = f.counts.reshape(-1)
    t2r = t2.reshape(4, synth.TBUF_CHANNELS, -1)
    for k in range(4):
        t2r[k][:, c <= k] = np.float32(3.0e38)
    b = O.render_frame(w, synth.make_scene(5), f.gbuf, t2, f.counts)
    assert np.all(np.isfinite(a))
    np.testing.assert_array_equal(a, b)


def test_frame_matches_per_pixel_definition():
    """Vectorised frame path equals the per-pixel definition (SoA indexing p = y*w + x)."""
    w = _tiny_weights(6)
    f = synth.make_frame(3, 4, 3, counts="uniform", seed=6)
    s = synth.make_scene(6)
    rgb = O.render_frame(w, s, f.gbuf, f.tbuf, f.counts)
    sigma = O.scene_encoder(w, s)
    for y in range(3):
        for x in range(4):
            c = int(f.counts[y, x])
            L = f.tbuf[:c, :, y, x]
            ref = O.render_pixel(w, sigma, f.gbuf[:, y, x], L)
            np.testing.assert_allclose(rgb[:, y, x], ref, rtol=0, atol=1e-13)


def test_frame_permutation_bit_identical():
    w = _tiny_weights(8)
    f = synth.make_frame(8, 8, 5, counts="uniform", seed=8)
    s = synth.make_scene(8)
    ref = O.render_frame(w, s, f.gbuf, f.tbuf, f.counts)
    for seed in range(1, 4):
        fp = synth.permute_layers(f, seed)
        assert not np.array_equal(np.nan_to_num(fp.tbuf), np.nan_to_num(f.tbuf))
        np.testing.assert_array_equal(O.render_frame(w, s, fp.gbuf, fp.tbuf, fp.counts), ref)


def test_fold_identity():
    """Splitting phi1 and B1 into a sigma-independent part plus a folded bias is exact
    algebra: W [b ; sigma] + c = W_b b + (W_sigma sigma + c)."""
    w = _tiny_weights(9)
    rng = np.random.default_rng(9)
    sigma = O.scene_encoder(w, rng.standard_normal(synth.SCENE_DIM))
    t = rng.standard_normal((7, synth.TBUF_CHANNELS))
    W1, b1 = (np.float64(a) for a in w["phi1"])
    n_t = synth.TBUF_CHANNELS
    folded = t @ W1[:, :n_t].T + (W1[:, n_t:] @ sigma + b1)
    concat = O.linear(np.concatenate([t, np.broadcast_to(sigma, (7, sigma.size))], 1), W1, b1)
    np.testing.assert_allclose(folded, concat, rtol=0, atol=1e-12)


def test_alpha_blending_is_order_dependent_negative_control():
    """Eq. 3-4 changes when the layers are reordered; the network's pool does not."""
    C = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    a = np.array([0.5, 0.25, 0.75])
    fwd = O.alpha_blend(C, a)
    rev = O.alpha_blend(C[::-1], a[::-1])
    assert np.max(np.abs(fwd - rev)) > 0.1
    # one layer: alpha * C
    np.testing.assert_allclose(O.alpha_blend(C[:1], a[:1]), [0.5, 0, 0])


# --------------------------------------------------------------- mutation tests

def _pins_pass(mod):
    """Run the hand-case pins against a (possibly mutated) oracle module."""
    try:
        sigma = mod.scene_encoder(hc.W, hc.SCENE)
        cases = [([hc.LAYER_A], hc.LOGITS_ONE_LAYER),
                 ([hc.LAYER_A, hc.LAYER_B], hc.LOGITS_TWO_LAYERS),
                 ([], hc.LOGITS_NO_LAYER)]
        for layers, logits in cases:
            L = np.array(layers, np.float32).reshape(len(layers), 2)
            got = mod.render_pixel(hc.W, sigma, hc.G, L)
            if not np.allclose(got, expit(logits), rtol=1e-12, atol=0):
                return False
        counts = np.array([[2]], np.uint8)
        tbuf = np.full((3, 2, 1, 1), np.nan, np.float32)
        tbuf[0, :, 0, 0] = hc.LAYER_A
        tbuf[1, :, 0, 0] = hc.LAYER_B
        gbuf = hc.G.reshape(2, 1, 1)
        rgb = mod.render_frame(hc.W, hc.SCENE, gbuf, tbuf, counts)
        return bool(np.allclose(rgb[:, 0, 0], expit(hc.LOGITS_TWO_LAYERS), rtol=1e-12, atol=0))
    except Exception:
        return False


def _mutant(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)
    return O


def test_unmutated_oracle_passes_pins():
    assert _pins_pass(O)


MUTATIONS = {
    "pool order [mean; max]": ("set_pool", lambda V: (lambda p: None if p is None else
                                np.concatenate([p[len(p) // 2:], p[:len(p) // 2]]))(
                                    _ORIG["set_pool"](V))),
    "drop phi1 bias": ("per_layer_h", lambda w, b, s: _ORIG["per_layer_h"](
        {**w, "phi1": (w["phi1"][0], 0 * w["phi1"][1])}, b, s)),
    "sigma before layer channels": ("per_layer_h", lambda w, b, s: O.relu(O.linear(O.relu(O.linear(
        np.concatenate([np.broadcast_to(np.float64(s), np.shape(b)[:-1] + (np.shape(s)[-1],)),
                        np.float64(b)], -1), *w["phi1"])), *w["phi2"]))),
    "transposed phi2": ("per_layer_h", lambda w, b, s: _ORIG["per_layer_h"](
        {**w, "phi2": (w["phi2"][0].T, w["phi2"][1])}, b, s)),
    "no ReLU after phi2": ("per_layer_h", lambda w, b, s: O.linear(O.relu(O.linear(
        np.concatenate([np.float64(b), np.broadcast_to(np.float64(s), np.shape(b)[:-1] + (np.shape(s)[-1],))], -1),
        *w["phi1"])), *w["phi2"])),
    "B input [r; g; sigma]": ("final_blend_B", lambda w, g, r, s: _ORIG["final_blend_B"](w, r, g, s)),
    "wrong sign B2 bias": ("final_blend_B", lambda w, g, r, s: _ORIG["final_blend_B"](
        {**w, "B2": (w["B2"][0], -w["B2"][1])}, g, r, s)),
    "transposed F1": ("scene_encoder", lambda w, s: _ORIG["scene_encoder"](
        {**w, "F1": (w["F1"][0].T, w["F1"][1])}, s)),
    "rho drops bias": ("post_pool_rho", lambda w, p: O.relu(np.float64(p) @ np.float64(w["rho"][0]).T)),
    "R1 transposed": ("render_R", lambda w, y: _ORIG["render_R"](
        {**w, "R1": (w["R1"][0].T, w["R1"][1])}, y)),
    "sigmoid(-x)": ("sigmoid", lambda x: 1.0 / (1.0 + np.exp(np.float64(x)))),
}
_ORIG = {n: getattr(O, n) for n in ("set_pool", "per_layer_h", "final_blend_B",
                                     "scene_encoder", "post_pool_rho", "render_R", "sigmoid")}


@pytest.mark.parametrize("label", sorted(MUTATIONS))
def test_planted_mistake_is_caught(monkeypatch, label):
    name, fn = MUTATIONS[label]
    assert not _pins_pass(_mutant(monkeypatch, name, fn)), label


def test_mean_over_slots_instead_of_valid_layers_is_caught():
    """A mean that divides by K instead of the valid count fails the K=3 frame pin."""
    counts = np.array([[2]], np.uint8)
    tbuf = np.full((3, 2, 1, 1), 0.0, np.float32)
    tbuf[0, :, 0, 0] = hc.LAYER_A
    tbuf[1, :, 0, 0] = hc.LAYER_B
    sigma = O.scene_encoder(hc.W, hc.SCENE)
    V = np.stack([O.per_layer_h(hc.W, tbuf[k, :, 0, 0], sigma) for k in range(3)])
    wrong = np.concatenate([V[:2].max(0), V[:2].sum(0) / 3])
    right = O.set_pool(V[:2])
    assert not np.allclose(wrong, right)
    np.testing.assert_array_equal(right, hc.POOL_TWO_LAYERS)


# ------------------------------------------------------ sum pooling (Eq. 5 form)

def test_hand_set_sum_two_layers():
    V = np.stack([O.per_layer_h(hc.W, hc.LAYER_A, hc.SIGMA),
                  O.per_layer_h(hc.W, hc.LAYER_B, hc.SIGMA)])
    np.testing.assert_array_equal(O.set_sum(V), hc.TAU_TWO_LAYERS)
    np.testing.assert_array_equal(O.set_sum(np.zeros((0, 2))), np.zeros(2))


@pytest.mark.parametrize("layers,logits", [
    ([hc.LAYER_A], hc.LOGITS_SUM_ONE_LAYER),
    ([hc.LAYER_A, hc.LAYER_B], hc.LOGITS_SUM_TWO_LAYERS),
    ([hc.LAYER_B, hc.LAYER_A], hc.LOGITS_SUM_TWO_LAYERS),
    ([], hc.LOGITS_NO_LAYER),
])
def test_hand_render_pixel_sum(layers, logits):
    sigma = O.scene_encoder(hc.W, hc.SCENE)
    L = np.array(layers, np.float32).reshape(len(layers), 2)
    np.testing.assert_allclose(O.render_pixel_sum(hc.W, sigma, hc.G, L), expit(logits),
                               rtol=1e-15, atol=0)


def test_hand_render_frame_sum_matches_closed_forms():
    counts = np.array([[1, 2], [0, 2]], np.uint8)
    gbuf = np.broadcast_to(hc.G[:, None, None], (2, 2, 2)).copy()
    tbuf = np.full((3, 2, 2, 2), np.nan, np.float32)
    tbuf[0, :, 0, 0] = hc.LAYER_A
    tbuf[0, :, 0, 1] = hc.LAYER_A
    tbuf[1, :, 0, 1] = hc.LAYER_B
    tbuf[0, :, 1, 1] = hc.LAYER_B
    tbuf[1, :, 1, 1] = hc.LAYER_A
    rgb = O.render_frame(hc.W, hc.SCENE, gbuf, tbuf, counts, pooling="sum")
    np.testing.assert_allclose(rgb[:, 0, 0], expit(hc.LOGITS_SUM_ONE_LAYER), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 0, 1], expit(hc.LOGITS_SUM_TWO_LAYERS), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 1, 0], expit(hc.LOGITS_NO_LAYER), rtol=1e-15)
    np.testing.assert_allclose(rgb[:, 1, 1], expit(hc.LOGITS_SUM_TWO_LAYERS), rtol=1e-15)


def test_sum_pooling_is_not_duplication_invariant():
    """Unlike [max ; mean], the sum of {a, a, b, b} is twice that of {a, b}."""
    rng = np.random.default_rng(11)
    a, b = rng.random(4), rng.random(4)
    np.testing.assert_allclose(O.set_sum(np.stack([a, a, b, b])), 2 * O.set_sum(np.stack([a, b])),
                               rtol=1e-15)
    p1, p2 = O.set_pool(np.stack([a, b])), O.set_pool(np.stack([a, a, b, b]))
    np.testing.assert_array_equal(p1, p2)


def test_sum_pooling_permutation_invariant_and_empty_is_opaque_only():
    w = synth.make_weights(synth.Widths(hidden=8, latent=6), seed=3, bias="uniform")
    sigma = O.scene_encoder(w, synth.make_scene(2))
    rng = np.random.default_rng(5)
    g = rng.standard_normal(14)
    L = rng.standard_normal((4, 12))
    ref = O.render_pixel_sum(w, sigma, g, L)
    for perm in itertools.permutations(range(4)):
        np.testing.assert_array_equal(O.render_pixel_sum(w, sigma, g, L[list(perm)]), ref)
    np.testing.assert_allclose(O.render_pixel_sum(w, sigma, g, np.zeros((0, 12))),
                               O.render_opaque_only(w, sigma, g[None, :])[0], rtol=1e-14)


def test_sum_frame_matches_per_pixel_definition():
    w = synth.make_weights(synth.Widths(hidden=8, latent=6), seed=4, bias="uniform")
    scene = synth.make_scene(1)
    f = synth.make_frame(5, 3, 4, counts="uniform", seed=6)
    rgb = O.render_frame(w, scene, f.gbuf, f.tbuf, f.counts, pooling="sum")
    sigma = O.scene_encoder(w, scene)
    for y in range(5):
        for x in range(3):
            c = int(f.counts[y, x])
            exp = O.render_pixel_sum(w, sigma, f.gbuf[:, y, x], f.tbuf[:c, :, y, x])
            np.testing.assert_allclose(rgb[:, y, x], exp, rtol=1e-13, atol=1e-15)


def _sum_pins_pass(mod):
    """The sum-pooling hand pins, per pixel and through the frame path."""
    try:
        sigma = mod.scene_encoder(hc.W, hc.SCENE)
        for layers, logits in [([hc.LAYER_A], hc.LOGITS_SUM_ONE_LAYER),
                               ([hc.LAYER_A, hc.LAYER_B], hc.LOGITS_SUM_TWO_LAYERS),
                               ([], hc.LOGITS_NO_LAYER)]:
            L = np.array(layers, np.float32).reshape(len(layers), 2)
            if not np.allclose(mod.render_pixel_sum(hc.W, sigma, hc.G, L), expit(logits),
                               rtol=1e-12, atol=0):
                return False
        tbuf = np.full((3, 2, 1, 1), np.nan, np.float32)
        tbuf[0, :, 0, 0] = hc.LAYER_A
        tbuf[1, :, 0, 0] = hc.LAYER_B
        rgb = mod.render_frame(hc.W, hc.SCENE, hc.G.reshape(2, 1, 1), tbuf,
                               np.array([[2]], np.uint8), pooling="sum")
        return bool(np.allclose(rgb[:, 0, 0], expit(hc.LOGITS_SUM_TWO_LAYERS), rtol=1e-12, atol=0))
    except Exception:
        return False


SUM_MUTATIONS = {
    "sum drops the last layer": ("set_sum", lambda V: _ORIG_SUM(np.asarray(V)[:-1])
                                 if len(V) else _ORIG_SUM(V)),
    "sum is the mean": ("set_sum", lambda V: _ORIG_SUM(V) / max(len(V), 1)),
    "sum is the max": ("set_sum", lambda V: np.max(V, axis=0) if len(V) else _ORIG_SUM(V)),
    "tau through rho": ("final_blend_B", lambda w, g, r, s: _ORIG["final_blend_B"](
        w, g, O.relu(O.linear(np.concatenate([r, r], -1), *w["rho"])) if np.shape(r)[-1] ==
        np.shape(w["rho"][0])[0] else r, s)),
    "B input [tau; g; sigma]": ("final_blend_B", lambda w, g, r, s: _ORIG["final_blend_B"](w, r, g, s)),
}
_ORIG_SUM = O.set_sum


def test_unmutated_oracle_passes_sum_pins():
    assert _sum_pins_pass(O)


@pytest.mark.parametrize("label", sorted(SUM_MUTATIONS))
def test_planted_sum_mistake_is_caught(monkeypatch, label):
    name, fn = SUM_MUTATIONS[label]
    monkeypatch.setattr(O, name, fn)
    assert not _sum_pins_pass(O), label


# ------------------------------------------ positional encoding (Sec. 3.4)

def test_pe_of_zero_frequencies_is_the_input():
    x = np.random.default_rng(0).standard_normal((5, 3))
    np.testing.assert_array_equal(O.positional_encoding(x, 0), x)


def test_pe_known_values_and_block_layout():
    """Blocks [x ; sin(pi x) ; cos(pi x) ; sin(2 pi x) ; cos(2 pi x) ; ...],
    each over all channels; values at x = 0, 1/6, 1/2 fixed by trigonometry."""
    x = np.array([0.0, 1 / 6, 0.5])
    e = O.positional_encoding(x, 3)
    assert e.shape == (3 * 7,)
    r3 = np.sqrt(3) / 2
    want = np.array([0, 1 / 6, 0.5,        # x
                     0, 0.5, 1,            # sin(pi x)
                     1, r3, 0,             # cos(pi x)
                     0, r3, 0,             # sin(2 pi x)
                     1, 0.5, -1,           # cos(2 pi x)
                     0, r3, 0,             # sin(4 pi x) = sin(2 pi / 3)
                     1, -0.5, 1])          # cos(4 pi x)
    np.testing.assert_allclose(e, want, atol=1e-15)


def test_pe_blocks_obey_pythagoras_and_double_angle():
    x = np.random.default_rng(1).uniform(-3, 3, 7)
    e = O.positional_encoding(x, 5).reshape(11, 7)
    sn, cs = e[1::2], e[2::2]
    np.testing.assert_allclose(sn ** 2 + cs ** 2, 1.0, atol=1e-14)
    np.testing.assert_allclose(sn[1:], 2 * sn[:-1] * cs[:-1], atol=1e-12)
    np.testing.assert_allclose(cs[1:], 1 - 2 * sn[:-1] ** 2, atol=1e-12)


@pytest.mark.parametrize("layers,logits,sum_logits", [
    ([hc.LAYER_PA], hc.LOGITS_PE_ONE_LAYER, hc.LOGITS_PE_SUM_ONE_LAYER),
    ([hc.LAYER_PA, hc.LAYER_PB], hc.LOGITS_PE_TWO_LAYERS, hc.LOGITS_PE_SUM_TWO_LAYERS),
    ([hc.LAYER_PB, hc.LAYER_PA], hc.LOGITS_PE_TWO_LAYERS, hc.LOGITS_PE_SUM_TWO_LAYERS),
    ([], hc.LOGITS_PE_NO_LAYER, hc.LOGITS_PE_NO_LAYER),
])
def test_hand_pe_network(layers, logits, sum_logits):
    sigma = O.scene_encoder(hc.W_PE, hc.SCENE_PE)
    np.testing.assert_allclose(sigma, hc.SIGMA_PE, atol=1e-14)
    L = np.array(layers, np.float32).reshape(len(layers), 2)
    np.testing.assert_allclose(O.render_pixel(hc.W_PE, sigma, hc.G_PE, L), expit(logits), rtol=1e-12)
    np.testing.assert_allclose(O.render_pixel_sum(hc.W_PE, sigma, hc.G_PE, L), expit(sum_logits),
                               rtol=1e-12)


def test_hand_pe_frame_and_opaque_only():
    counts = np.array([[1, 2], [0, 2]], np.uint8)
    gbuf = np.broadcast_to(hc.G_PE[:, None, None], (2, 2, 2)).copy()
    tbuf = np.full((2, 2, 2, 2), np.nan, np.float32)
    tbuf[0, :, 0, 0] = hc.LAYER_PA
    tbuf[0, :, 0, 1] = hc.LAYER_PA
    tbuf[1, :, 0, 1] = hc.LAYER_PB
    tbuf[0, :, 1, 1] = hc.LAYER_PB
    tbuf[1, :, 1, 1] = hc.LAYER_PA
    for pooling, one, two in [("max_mean", hc.LOGITS_PE_ONE_LAYER, hc.LOGITS_PE_TWO_LAYERS),
                              ("sum", hc.LOGITS_PE_SUM_ONE_LAYER, hc.LOGITS_PE_SUM_TWO_LAYERS)]:
        rgb = O.render_frame(hc.W_PE, hc.SCENE_PE, gbuf, tbuf, counts, pooling=pooling)
        np.testing.assert_allclose(rgb[:, 0, 0], expit(one), rtol=1e-12)
        np.testing.assert_allclose(rgb[:, 0, 1], expit(two), rtol=1e-12)
        np.testing.assert_allclose(rgb[:, 1, 0], expit(hc.LOGITS_PE_NO_LAYER), rtol=1e-12)
        np.testing.assert_allclose(rgb[:, 1, 1], expit(two), rtol=1e-12)
    sigma = O.scene_encoder(hc.W_PE, hc.SCENE_PE)
    np.testing.assert_allclose(O.render_opaque_only(hc.W_PE, sigma, hc.G_PE[None, :])[0],
                               expit(hc.LOGITS_PE_NO_LAYER), rtol=1e-12)


def test_pe_network_with_zero_encoding_columns_is_the_plain_network():
    """Embed a plain weight set into L = 2 shapes with zeros in every sin / cos
    column: the raw block comes first in each input, so the outputs agree."""
    L = 2
    plain = synth.make_weights(synth.Widths(hidden=8, latent=6), seed=7, bias="uniform")
    pe = dict(plain)
    for name, n_raw in (("F1", synth.SCENE_DIM), ("phi1", 12), ("B1", 14)):
        W, b = plain[name]
        Wz = np.zeros((W.shape[0], W.shape[1] + 2 * L * n_raw), np.float32)
        Wz[:, :n_raw] = W[:, :n_raw]
        Wz[:, n_raw * (1 + 2 * L):] = W[:, n_raw:]
        pe[name] = (Wz, b)
    pe["pe_freqs"] = L
    scene = synth.make_scene(3)
    f = synth.make_frame(4, 5, 3, counts="uniform", seed=8)
    for pooling in ("max_mean", "sum"):
        np.testing.assert_allclose(O.render_frame(pe, scene, f.gbuf, f.tbuf, f.counts, pooling=pooling),
                                   O.render_frame(plain, scene, f.gbuf, f.tbuf, f.counts, pooling=pooling),
                                   rtol=1e-13, atol=1e-15)


def test_pe_frame_matches_per_pixel_definition():
    w = synth.make_weights(synth.Widths(hidden=8, latent=6, pe_freqs=3), seed=4, bias="uniform")
    scene = synth.make_scene(1)
    f = synth.make_frame(4, 3, 4, counts="uniform", seed=6)
    rgb = O.render_frame(w, scene, f.gbuf, f.tbuf, f.counts)
    sigma = O.scene_encoder(w, scene)
    for y in range(4):
        for x in range(3):
            c = int(f.counts[y, x])
            exp = O.render_pixel(w, sigma, f.gbuf[:, y, x], f.tbuf[:c, :, y, x])
            np.testing.assert_allclose(rgb[:, y, x], exp, rtol=1e-13, atol=1e-15)


def _pe_pins_pass(mod):
    try:
        sigma = mod.scene_encoder(hc.W_PE, hc.SCENE_PE)
        for layers, logits in [([hc.LAYER_PA], hc.LOGITS_PE_ONE_LAYER),
                               ([hc.LAYER_PA, hc.LAYER_PB], hc.LOGITS_PE_TWO_LAYERS),
                               ([], hc.LOGITS_PE_NO_LAYER)]:
            L = np.array(layers, np.float32).reshape(len(layers), 2)
            if not np.allclose(mod.render_pixel(hc.W_PE, sigma, hc.G_PE, L), expit(logits),
                               rtol=1e-12, atol=0):
                return False
        return True
    except Exception:
        return False


def _pe_interleaved(x, L):
    x = np.float64(x)
    cols = []
    for c in range(x.shape[-1]):
        cols.append(x[..., c:c + 1])
        for f in range(L):
            cols += [np.sin(np.pi * 2.0 ** f * x[..., c:c + 1]), np.cos(np.pi * 2.0 ** f * x[..., c:c + 1])]
    return np.concatenate(cols, axis=-1)


PE_MUTATIONS = {
    "sin and cos swapped": lambda x, L: (lambda e: np.concatenate(
        [e[..., :x.shape[-1]]] + [e[..., (2 * f + 2 - j) * x.shape[-1]:(2 * f + 3 - j) * x.shape[-1]]
                                  for f in range(L) for j in (0, 1)], axis=-1))(_ORIG_PE(x, L)),
    "no pi": lambda x, L: np.concatenate([np.float64(x)] + [fn(2.0 ** f * np.float64(x)) for f in range(L)
                                                            for fn in (np.sin, np.cos)], axis=-1),
    "frequencies from 2^1": lambda x, L: np.concatenate(
        [np.float64(x)] + [fn(np.pi * 2.0 ** (f + 1) * np.float64(x)) for f in range(L)
                           for fn in (np.sin, np.cos)], axis=-1),
    "interleaved per channel": _pe_interleaved,
    "raw input dropped": lambda x, L: _ORIG_PE(x, L)[..., x.shape[-1]:] if L else _ORIG_PE(x, L),
}
_ORIG_PE = O.positional_encoding


def test_unmutated_oracle_passes_pe_pins():
    assert _pe_pins_pass(O)


@pytest.mark.parametrize("label", sorted(PE_MUTATIONS))
def test_planted_pe_mistake_is_caught(monkeypatch, label):
    monkeypatch.setattr(O, "positional_encoding", PE_MUTATIONS[label])
    assert not _pe_pins_pass(O), label


# -------------------------------------------- spatial R (3x3 first layer)

def _r3_frame():
    counts = np.array([[1, 2], [0, 2]], np.uint8)
    gbuf = np.broadcast_to(hc.G[:, None, None], (2, 2, 2)).copy()
    tbuf = np.full((2, 2, 2, 2), np.nan, np.float32)
    tbuf[0, :, 0, 0] = hc.LAYER_A
    tbuf[0, :, 0, 1] = hc.LAYER_A
    tbuf[1, :, 0, 1] = hc.LAYER_B
    tbuf[0, :, 1, 1] = hc.LAYER_B
    tbuf[1, :, 1, 1] = hc.LAYER_A
    return gbuf, tbuf, counts


def test_hand_r3_frame():
    gbuf, tbuf, counts = _r3_frame()
    rgb = O.render_frame(hc.W_R3, hc.SCENE, gbuf, tbuf, counts)
    np.testing.assert_allclose(rgb, expit(hc.LOGITS_R3), rtol=1e-13)


def test_r3_per_pixel_paths_refuse():
    with pytest.raises(ValueError):
        O.render_pixel(hc.W_R3, hc.SIGMA, hc.G, np.zeros((0, 2)))


def _r3_weights(seed=7, H=8, Z=6, center_only=False):
    w = synth.make_weights(synth.Widths(hidden=H, latent=Z), seed=seed, bias="uniform")
    rng = np.random.default_rng(seed + 100)
    if center_only:
        K = np.zeros((H, H, 3, 3), np.float32)
        K[:, :, 1, 1] = w["R1"][0]
    else:
        K = (rng.standard_normal((H, H, 3, 3)) * 0.3).astype(np.float32)
    w3 = dict(w)
    w3["R1"] = (K.reshape(H, H * 9), w["R1"][1])
    w3["r_kernel"] = 3
    return w, w3, K


def test_r3_with_centre_tap_only_is_the_1x1_network():
    w, w3, _ = _r3_weights(center_only=True)
    scene = synth.make_scene(2)
    f = synth.make_frame(5, 7, 3, counts="uniform", seed=3)
    np.testing.assert_allclose(O.render_frame(w3, scene, f.gbuf, f.tbuf, f.counts),
                               O.render_frame(w, scene, f.gbuf, f.tbuf, f.counts), rtol=1e-13, atol=1e-15)


def test_r3_matches_torch_conv2d_cross_correlation():
    """torch's conv2d (cross-correlation, zero padding 1), FP64 on the CPU."""
    torch = pytest.importorskip("torch")
    _, w3, K = _r3_weights()
    rng = np.random.default_rng(4)
    Y = rng.random((6, 9, 8))
    b = np.float64(w3["R1"][1])
    ref = torch.nn.functional.conv2d(torch.from_numpy(Y.transpose(2, 0, 1)[None]),
                                     torch.from_numpy(np.float64(K)), torch.from_numpy(b), padding=1)
    q = np.maximum(ref[0].numpy().transpose(1, 2, 0), 0)
    W2, b2 = (np.float64(a) for a in w3["R2"])
    exp = (1 / (1 + np.exp(-(q @ W2.T + b2)))).transpose(2, 0, 1)
    np.testing.assert_allclose(O.render_R_frame(w3, Y), exp, rtol=1e-12, atol=1e-15)


def test_r3_brute_force_loops():
    _, w3, K = _r3_weights(seed=9, H=4)
    rng = np.random.default_rng(5)
    h, wd, H = 3, 4, 4
    Y = rng.standard_normal((h, wd, H))
    b = np.float64(w3["R1"][1])
    W2, b2 = (np.float64(a) for a in w3["R2"])
    out = np.zeros((3, h, wd))
    for y in range(h):
        for x in range(wd):
            q = [float(b[o]) for o in range(H)]
            for o in range(H):
                for i in range(H):
                    for ky in range(3):
                        for kx in range(3):
                            yy, xx = y + ky - 1, x + kx - 1
                            if 0 <= yy < h and 0 <= xx < wd:
                                q[o] += float(K[o, i, ky, kx]) * Y[yy, xx, i]
            q = [max(v, 0.0) for v in q]
            for c in range(3):
                z = float(b2[c]) + sum(float(W2[c, i]) * q[i] for i in range(H))
                out[c, y, x] = 1 / (1 + math.exp(-z))
    np.testing.assert_allclose(O.render_R_frame(w3, Y), out, rtol=1e-12)


def _r3_pins_pass(mod):
    try:
        gbuf, tbuf, counts = _r3_frame()
        rgb = mod.render_frame(hc.W_R3, hc.SCENE, gbuf, tbuf, counts)
        return bool(np.allclose(rgb, expit(hc.LOGITS_R3), rtol=1e-12, atol=0))
    except Exception:
        return False


def _r3_variant(kind):
    def f(weights, Y):
        Y = np.float64(Y)
        h, wd, H = Y.shape
        if O.r_kernel(weights) == 1:
            return O.render_R(weights, Y).transpose(2, 0, 1)
        flat = np.float64(weights["R1"][0])
        W = flat.reshape(-1, 9, H).transpose(0, 2, 1).reshape(-1, H, 3, 3) if kind == "tap_major" \
            else flat.reshape(-1, H, 3, 3)
        if kind == "flipped":
            W = W[:, :, ::-1, ::-1]
        if kind == "transposed":
            W = W.transpose(0, 1, 3, 2)
        Yp = np.pad(Y, ((1, 1), (1, 1), (0, 0)), mode="edge" if kind == "edge" else "constant")
        acc = np.broadcast_to(np.float64(weights["R1"][1]), (h, wd, W.shape[0])).copy()
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc = acc + Yp[1 + dy:1 + dy + h, 1 + dx:1 + dx + wd, :] @ W[:, :, dy + 1, dx + 1].T
        return O.sigmoid(O.linear(O.relu(acc), *weights["R2"])).transpose(2, 0, 1)
    return f


R3_MUTATIONS = ["flipped", "edge", "transposed", "tap_major"]


def test_unmutated_oracle_passes_r3_pins():
    assert _r3_pins_pass(O)
    # the reference re-implementation used for the mutations agrees when unmutated
    Y = np.random.default_rng(1).random((3, 4, 2))
    np.testing.assert_allclose(_r3_variant("none")(hc.W_R3, Y), O.render_R_frame(hc.W_R3, Y), rtol=1e-14)


@pytest.mark.parametrize("kind", R3_MUTATIONS)
def test_planted_r3_mistake_is_caught(monkeypatch, kind):
    monkeypatch.setattr(O, "render_R_frame", _r3_variant(kind))
    assert not _r3_pins_pass(O), kind


def test_mean_instead_of_sum_is_caught():
    """A tau that divides by the count (the mean) fails the two-layer hand pin."""
    sigma = O.scene_encoder(hc.W, hc.SCENE)
    V = np.stack([O.per_layer_h(hc.W, hc.LAYER_A, sigma), O.per_layer_h(hc.W, hc.LAYER_B, sigma)])
    wrong = O.render_R(hc.W, O.final_blend_B(hc.W, hc.G, O.set_sum(V) / 2, sigma))
    assert not np.allclose(wrong, expit(hc.LOGITS_SUM_TWO_LAYERS), rtol=1e-12)


def test_oracle_package_exports():
    for n in oracle.__all__ if hasattr(oracle, "__all__") else []:
        assert hasattr(oracle, n)
    assert callable(oracle.render_frame)
