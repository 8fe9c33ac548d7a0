"""Pins of the oracle's model-level operations (Sec. 3.2 simplification passes,
density control with phi reweighting and the LOD inheritance of Sec. 3.3)."""
import itertools
import math

import numpy as np
import pytest

from paper_2605_13794_gb300 import synth


def test_successive_sampling_probabilities_closed_forms(oracle_mod):
    s = np.array([1.0, 2.0, 3.0, 4.0])
    p1 = oracle_mod.successive_sampling_probs(s, 1)
    np.testing.assert_allclose(p1, s / s.sum(), atol=1e-15)        # one draw: proportional to s
    p2 = oracle_mod.successive_sampling_probs(s, 2)
    assert abs(p2.sum() - 2.0) < 1e-12                              # k items drawn
    # two draws by hand: P(i) = s_i/S + sum_{j != i} s_j/S * s_i/(S - s_j)
    S = s.sum()
    hand = [s[i] / S + sum(s[j] / S * s[i] / (S - s[j]) for j in range(4) if j != i) for i in range(4)]
    np.testing.assert_allclose(p2, hand, atol=1e-15)
    assert np.allclose(oracle_mod.successive_sampling_probs(s, 4), 1.0)


def test_exponential_clocks_sample_without_replacement_proportional_to_s(oracle_mod):
    # inclusion frequencies of Pass 1 over many draws against the exact
    # successive-sampling probabilities (5 sigma of a binomial frequency)
    s = np.array([1.0, 2.0, 3.0, 4.0, 0.5, 6.0], np.float32)
    k, draws = 3, 20000
    rng = np.random.default_rng(7)
    counts = np.zeros(len(s))
    for _ in range(draws):
        counts += oracle_mod.prune_sample(s, rng.exponential(size=len(s)).astype(np.float32), k)
    exact = oracle_mod.successive_sampling_probs(s.astype(np.float64), k)
    freq = counts / draws
    sd = np.sqrt(exact * (1 - exact) / draws)
    assert np.all(np.abs(freq - exact) <= 5 * sd + 1e-12), (freq, exact)


def test_sampling_keeps_exactly_k_and_never_zero_scores_first(oracle_mod):
    rng = np.random.default_rng(8)
    s = rng.uniform(0, 1, 200).astype(np.float32)
    s[::7] = 0
    keep = oracle_mod.prune_sample(s, rng.exponential(size=200).astype(np.float32), 150)
    assert keep.sum() == 150 and keep[s > 0].all() == ((s > 0).sum() <= 150)
    keep = oracle_mod.prune_sample(s, rng.exponential(size=200).astype(np.float32), 100)
    assert keep.sum() == 100 and not keep[s == 0].any()


def test_mass_cut_is_minimal_by_exhaustion(oracle_mod):
    rng = np.random.default_rng(9)
    s = rng.uniform(0, 1, 9)
    s[2] = 0.0
    keep = oracle_mod.prune_mass(s, 0.9)
    need = 0.9 * s.sum()
    assert s[keep].sum() >= need
    best = min(len(c) for r in range(1, 10) for c in itertools.combinations(range(9), r) if s[list(c)].sum() >= need)
    assert keep.sum() == best and not keep[2]


def _rows(g):
    rows = dict(mean=g.mean, log_scale=g.log_scale, quat=g.quat, opacity_logit=g.opacity_logit, sh=g.sh, lod=g.lod)
    rng = np.random.default_rng(3)
    rows["m"] = {k: rng.standard_normal(np.shape(v)) for k, v in rows.items() if k != "lod"}
    rows["v"] = {k: np.abs(rng.standard_normal(np.shape(v))) for k, v in rows.items() if k not in ("lod", "m")}
    return rows


def test_densify_by_hand(oracle_mod):
    O = oracle_mod
    g = synth.plain_scene(5, seed=10)
    g.quat[:] = np.array([1, 0, 0, 0], np.float32)
    g.log_scale[:] = np.log(np.float32(0.005))
    g.log_scale[3] = np.log(np.array([0.05, 0.02, 0.01], np.float32))   # large: split
    g.opacity_logit[:] = 0.0                                           # opacity 0.5
    g.opacity_logit[4] = np.float32(math.log(0.001 / 0.999))          # below min_opacity
    g.lod[:] = np.array([0, 1, 2, 5, 0], np.uint8)
    rows = _rows(g)
    P = O.DensifyParams(grad_threshold=1e-3, dense_scale=0.01, n_levels=6)
    absgrad = np.array([5e-4, 4e-3, 4e-3, 8e-3, 1.0])   # averaged: 2.5e-4, 2e-3, 2e-3, 4e-3
    denom = np.array([2, 2, 2, 2, 1])
    cvis = np.array([2, 2, 0, 2, 2])                      # Gaussian 2 never contributes: phi = 0
    crad = np.array([2, 2, 2, 2, 2])
    noise = np.random.default_rng(11).standard_normal((5, 2, 3))
    out, m, v, kind = O.densify(rows, absgrad, denom, cvis, crad, noise, P)
    assert list(kind) == [1, 2, 1, 3, 0]
    # 0 kept, 1 and its clone, 2 kept (phi = 0), 3's two children, 4 removed
    assert len(out["opacity_logit"]) == 6
    np.testing.assert_array_equal(out["mean"][0], g.mean[0])
    np.testing.assert_array_equal(out["mean"][1], g.mean[1])
    np.testing.assert_array_equal(out["mean"][2], g.mean[1])
    assert list(out["lod"]) == [0, 1, 1, 2, 5, 5]           # clone keeps the level; split +1, capped at 5
    np.testing.assert_allclose(m["mean"][1], rows["m"]["mean"][1])  # the parent keeps its moments
    assert not m["mean"][2].any() and not v["sh"][2].any()       # the clone starts from zero
    for c in range(2):                                           # identity rotation: mu + s * z
        mu, ls = g.mean[3].astype(np.float64), g.log_scale[3].astype(np.float64)
        np.testing.assert_allclose(out["mean"][4 + c], mu + np.exp(ls) * noise[3, c], rtol=1e-12)
        np.testing.assert_allclose(out["log_scale"][4 + c], ls - math.log(1.6), rtol=1e-12)
        assert not m["quat"][4 + c].any()


def test_split_children_follow_the_parent_rotation(oracle_mod):
    O = oracle_mod
    g = synth.plain_scene(1, seed=12)
    g.log_scale[:] = np.log(np.array([[0.2, 0.05, 0.01]], np.float32))
    g.opacity_logit[:] = 0.0
    rows = _rows(g)
    noise = np.array([[[1.0, 0, 0], [0, 0, 1.0]]])
    out, _, _, kind = O.densify(rows, [1.0], [1], [1], [1], noise, O.DensifyParams(dense_scale=0.01))
    assert kind[0] == 3
    q = g.quat[0] / np.linalg.norm(g.quat[0])
    w, x, y, z = q
    # the first column of R(q) is the local x axis
    axis_x = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    np.testing.assert_allclose(out["mean"][0] - g.mean[0], 0.2 * axis_x, atol=1e-6)
    assert abs(np.linalg.norm(out["mean"][1] - g.mean[0]) - 0.01) < 1e-7
