"""The seeded input generators follow the stated recipe (CPU only)."""
import math

import numpy as np

import synth


def test_same_seed_same_arrays_and_different_seeds_differ():
    a, b = synth.ragged_survey(200), synth.ragged_survey(200)
    assert np.array_equal(a.t, b.t) and np.array_equal(a.y, b.y) and np.array_equal(a.offsets, b.offsets)
    c = synth.ragged_survey(200, seed=synth.SEEDS["ragged_survey"] + 1)
    assert not np.array_equal(a.y[:50], c.y[:50])
    tr, inf = synth.learned_set(100, "learned_train"), synth.learned_set(100, "learned_infer")
    assert not np.array_equal(tr.t[:50], inf.t[:50])
    assert not np.array_equal(synth.learned_set(100, part=0).t[:50], synth.learned_set(100, part=1).t[:50])


def test_survey_cadence_and_ranges():
    b = synth.ragged_survey(2000)
    n_t = b.n_t
    assert n_t.min() >= 50 and n_t.max() <= 500 and abs(n_t.mean() - 275) < 10
    phase = np.mod(b.t - synth.T_START, synth.YEAR)
    assert phase.min() >= 0.0 and phase.max() < synth.SEASON          # six-month seasonal gap
    assert b.t.min() >= synth.T_START and b.t.max() < synth.T_START + 10 * synth.YEAR
    for o in range(0, b.n_obj, 97):                                    # sorted within each object
        seg = b.t[b.offsets[o]:b.offsets[o + 1]]
        assert np.all(np.diff(seg) >= 0)
    p_h = 24.0 / b.f_true
    assert p_h.min() >= 2.0 and p_h.max() <= 100.0
    assert b.sigma.min() >= 0.02 and b.sigma.max() <= 0.3
    g = synth.GRIDS["ragged_survey"]
    assert (g.f_min, g.f_max, g.n_f) == (0.24, 12.0, 100_000)


def test_lognormal_lengths_are_log_uniform():
    b = synth.ragged_lognormal(20000)
    n_t = b.n_t
    assert n_t.min() >= 10 and n_t.max() <= 2000
    assert abs(np.median(n_t) - math.sqrt(10 * 2000)) < 10            # log-uniform median
    assert synth.GRIDS["ragged_lognormal"].n_f == 50_000


def test_single_objects():
    s = synth.single_small()
    assert s.n_obj == 1 and s.t.size == 1000 and np.all(np.diff(s.t) >= 0)
    assert s.t.min() >= 60000.0 and s.t.max() <= 63650.0 and 0.2 <= s.f_true[0] <= 5.0
    big = synth.single_large()
    assert big.t.size == 100_000 and big.t.max() - big.t.min() <= 10 * synth.YEAR
    assert 0.1 <= big.f_true[0] <= 20.0 and synth.GRIDS["single_large"].n_f == 1_000_000


def test_subset_keeps_objects_whole():
    b = synth.ragged_survey(50)
    sub = b.subset([3, 7, 11])
    assert sub.n_obj == 3
    for i, o in enumerate([3, 7, 11]):
        assert np.array_equal(sub.t[sub.offsets[i]:sub.offsets[i + 1]], b.t[b.offsets[o]:b.offsets[o + 1]])
        assert sub.f_true[i] == b.f_true[o]
