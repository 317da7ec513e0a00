"""Pins of the oracle's evaluation variants (quantisation, efficiency)."""
import numpy as np

from oracle import dos_oracle as O


def test_one_bit_keeps_the_two_end_levels():
    h = np.array([0.0, 0.2, 0.49, 0.51, 0.9, 1.0, 1.7, -0.3]) * 664.5e-9
    q = O.quantize_thickness(h, 664.5e-9, 1)
    assert set(np.round(q / 664.5e-9, 6)) <= {0.0, 1.0}
    assert q[0] == 0 and q[2] == 0 and q[3] > 0 and q[6] == q[5]


def test_quantisation_error_is_at_most_half_a_step_and_idempotent():
    rng = np.random.default_rng(0)
    hmax = 664.5e-9
    h = rng.uniform(0, hmax, 10000)
    for bits in (4, 6, 8, 16):
        q = O.quantize_thickness(h, hmax, bits)
        step = hmax / (2 ** bits - 1)
        # half a step, up to the FP64 rounding of h (2^B - 1) / h_max
        assert np.max(np.abs(q - h)) <= 0.5 * step * (1 + 1e-9)
        assert np.array_equal(O.quantize_thickness(q, hmax, bits), q)
        assert len(np.unique(q)) <= 2 ** bits


def test_quantisation_is_the_nearest_level_by_brute_force():
    """Fig. 7's B-bit design: each thickness goes to the closest of the 2^B
    levels k h_max / (2^B - 1); checked against an exhaustive search over all
    levels (thicknesses outside [0, h_max] go to the end levels)."""
    rng = np.random.default_rng(7)
    hmax = 664.5e-9
    for bits in (1, 2, 3, 5, 8):
        levels = np.arange(2 ** bits) * (hmax / (2 ** bits - 1))
        h = rng.uniform(-0.3 * hmax, 1.3 * hmax, 4000)
        nearest = levels[np.argmin(np.abs(h[:, None] - levels[None, :]), axis=1)]
        assert np.array_equal(O.quantize_thickness(h, hmax, bits), nearest)


def test_quantisation_hand_cases():
    """Two bits, h_max = 3: levels 0, 1, 2, 3; a thickness midway between two
    levels goes to the even level index (round half to even)."""
    h = np.array([-1.0, 0.0, 0.49, 0.5, 0.51, 1.5, 2.5, 2.51, 3.0, 7.0])
    assert O.quantize_level(h, 3.0, 2).tolist() == [0, 0, 0, 0, 1, 2, 2, 3, 3, 3]
    assert O.quantize_thickness(h, 3.0, 2).tolist() == [0.0, 0.0, 0.0, 0.0, 1.0, 2.0, 2.0, 3.0, 3.0, 3.0]


def test_efficiency_of_an_unobstructed_zero_gap_system():
    """With zero gaps and lossless flat layers the output equals the input
    aperture, so the efficiency is the fraction of the aperture the FOV sees."""
    n, a, f = 16, 10, 6
    out = O.forward(np.zeros((1, n, n)), [600e-9], [0.0, 0.0], 0.3e-6, 32, f, a, 1.5, 0.0)
    eta = O.diffraction_efficiency(out["I"], a)
    assert abs(eta[0] - f * f / (a * a)) < 1e-14
    out2 = O.forward(np.zeros((1, n, n)), [600e-9], [0.0, 0.0], 0.3e-6, 32, 12, 8, 1.5, 0.0)
    assert abs(O.diffraction_efficiency(out2["I"], 8)[0] - 1.0) < 1e-14


def test_efficiency_never_exceeds_one_for_lossless_propagation():
    rng = np.random.default_rng(1)
    h = rng.uniform(0, 600e-9, (2, 24, 24))
    out = O.forward(h, [500e-9, 700e-9], [5e-6, 7e-6, 6e-6], 0.3e-6, 48, 24, 12, 1.6, 0.0)
    eta = O.diffraction_efficiency(out["I"], 12)
    assert np.all(eta <= 1 + 1e-12) and np.all(eta > 0)
