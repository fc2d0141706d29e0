"""Host logic of the learned interval predictor (no GPU): the network's
inputs leave out the size, the sweep settings and labels, the fallback rule
for a rejected prediction, and the training set's size range."""
import numpy as np

from paper_2208_01339_gb300 import learn as L


def test_model_inputs_drop_only_the_size():
    f = np.arange(24, dtype=np.float64).reshape(3, 8) + 1.0
    g = L.model_inputs(f)
    assert g.shape == f.shape
    assert not g[:, 0].any()                       # log10 n held at zero
    np.testing.assert_array_equal(g[:, 1:], f[:, 1:])
    np.testing.assert_array_equal(f[:, 0], [1.0, 9.0, 17.0])  # the caller's array is not changed


def test_sweep_settings_and_labels():
    assert len(L.SETTINGS) == 32 and len(set(L.SETTINGS)) == 32
    assert L.FIXED_BEST in L.SETTINGS
    it = np.full((3, 32), 50.0)
    it[0, 5], it[1, 20], it[2, 7] = 10, 9, 8
    it[2, 3] = 8  # a tie goes to the first setting
    y, best = L.labels(it)
    np.testing.assert_array_equal(best, [5, 20, 3])
    np.testing.assert_allclose(10.0 ** y[1], L.SETTINGS[20])
    assert L.most_frequent_setting(np.vstack([it, it[1:2], it[1:2]])) == L.SETTINGS[20]


def test_auto_xi_is_the_clipped_ten_over_kappa_rule():
    assert L.auto_xi(1.0, 1e3) == 1e-2
    assert L.auto_xi(1.0, 1e5) == 1e-4
    assert L.auto_xi(1.0, 1e9) == 1e-6


def test_training_sizes_cover_the_requested_range():
    specs = L.training_specs(400)
    ns = np.array([s.N for s in specs])
    assert ns.min() >= 12 and ns.max() <= 64
    assert ns.max() > 56 and ns.min() < 16
    assert all(s.nrhs == 8 for s in specs)
