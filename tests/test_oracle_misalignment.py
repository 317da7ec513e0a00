"""Pins of the misaligned-layer model (Section 3, "vaccination")."""
import numpy as np

from oracle import dos_oracle as O


def test_integer_lateral_shift_moves_the_layer():
    """Zero gaps: the output is the transmission; displacing the layer by whole
    pixels (+dx columns, +dy rows) moves its map by that amount."""
    rng = np.random.default_rng(3)
    n, a, pitch = 16, 8, 0.25e-6
    h = rng.uniform(0, 600e-9, (1, n, n))
    kap = 0.05
    disp = np.array([[2 * pitch, -1 * pitch, 0.0]])
    out = O.forward(h, [600e-9], [0.0, 0.0], pitch, 64, n, a, 1.5, kap, displacements=disp)
    moved = np.roll(np.roll(h[0], 2, axis=1), -1, axis=0)
    expect = np.exp(-4 * np.pi * kap * moved / 600e-9) * O.aperture_field(n, a).real
    assert np.max(np.abs(out["I"][0] - expect)) < 1e-12


def test_axial_shift_of_a_flat_layer_changes_nothing_in_a_periodic_window():
    """A flat lossless layer moved along z leaves the total path unchanged:
    gaps z0 + dz and z1 - dz compose to z0 + z1 (no cropping when M = N)."""
    n = 16
    lam = [550e-9, 650e-9]
    base = dict(gaps=[9e-6, 11e-6], pitch=0.35e-6, m=n, fov=n, aperture=10, n_index=1.5, kappa=0.0)
    a = O.forward(np.zeros((1, n, n)), lam, **base)["o"]
    b = O.forward(np.zeros((1, n, n)), lam, displacements=np.array([[0.0, 0.0, 0.7e-6]]), **base)["o"]
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_lateral_shift_of_a_flat_layer_is_invisible_in_a_periodic_window():
    n = 16
    base = dict(gaps=[9e-6, 11e-6], pitch=0.35e-6, m=n, fov=n, aperture=10, n_index=1.5, kappa=0.0)
    a = O.forward(np.zeros((1, n, n)), [600e-9], **base)["o"]
    b = O.forward(np.zeros((1, n, n)), [600e-9], displacements=np.array([[37e-9, -21e-9, 0.0]]), **base)["o"]
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_gradient_with_displacements_matches_central_differences():
    rng = np.random.default_rng(4)
    lam = np.array([480e-9, 650e-9])
    model = dict(lambdas=lam, gaps=np.array([5e-6, 4e-6, 6e-6]), pitch=0.3e-6, m=32, fov=8, aperture=8,
                 n_index=1.6, kappa=0.01, displacements=np.array([[31e-9, -17e-9, 90e-9], [-12e-9, 44e-9, -150e-9]]))
    h = rng.uniform(0, 550e-9, (2, 16, 16))
    T = rng.uniform(0, 1, (2, 8, 8))
    _, _, g, _ = O.loss_and_grad(h, T, **model)
    pixels = [(0, 8, 8), (1, 6, 10), (0, 3, 12)]
    fd = O.finite_difference(h, T, pixels, 1e-4 * 550e-9, **model)
    ad = np.array([g[p] for p in pixels])
    assert np.max(np.abs(ad - fd)) < 1e-6 * np.max(np.abs(ad))
