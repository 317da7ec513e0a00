"""Pins of the oracle's detector pixels (Section 4: the output FOV is divided
into 25 x 25 pixels, each covering several diffractive features; a detector
pixel integrates the intensity of the b x b simulation pixels under it)."""
import numpy as np
import pytest

from oracle import dos_oracle as O


def test_detector_of_blockwise_constant_intensity():
    """I constant c on every b x b block -> D = b^2 c (closed form)."""
    rng = np.random.default_rng(21)
    for b in (1, 2, 5):
        C = rng.uniform(0, 1, size=(3, 4, 4))
        I = np.stack([np.kron(C[w], np.ones((b, b))) for w in range(3)])
        assert np.allclose(O.detector_intensity(I, b), b * b * C, rtol=1e-14, atol=0)


def test_detector_keeps_total_power_and_single_pixel_sees_everything():
    rng = np.random.default_rng(22)
    I = rng.uniform(0, 1, size=(2, 12, 12))
    for b in (1, 2, 3, 4, 6, 12):
        D = O.detector_intensity(I, b)
        assert D.shape == (2, 12 // b, 12 // b)
        assert np.allclose(D.sum(axis=(1, 2)), I.sum(axis=(1, 2)), rtol=1e-14)
    assert np.allclose(O.detector_intensity(I, 12)[:, 0, 0], I.sum(axis=(1, 2)), rtol=1e-14)
    with pytest.raises(ValueError):
        O.detector_intensity(I, 5)


@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("b", [1, 2, 3])
def test_binned_loss_gradient_matches_central_differences_in_I(scaled, b):
    """dL/dI of the binned loss against central differences of L with respect
    to single simulation pixels (the plain loss is quadratic in I, so its
    central difference is exact up to rounding; the scaled loss's gradient
    holds sigma fixed, exact to first order by the envelope theorem)."""
    rng = np.random.default_rng(23 + b)
    I = rng.uniform(0.1, 1, size=(2, 6, 6))
    T = rng.uniform(0, 1, size=(2, 6 // b, 6 // b)) * b * b
    L, psnr, dLdI = O.mse_loss(I, T, scaled=scaled, detector_bin=b)
    assert dLdI.shape == I.shape
    d = 1e-6
    for idx in [(0, 0, 0), (0, 5, 4), (1, 2, 3), (1, 3, 1), (0, 4, 5)]:
        Ip = I.copy()
        Im = I.copy()
        Ip[idx] += d
        Im[idx] -= d
        fd = (O.mse_loss(Ip, T, scaled, b)[0] - O.mse_loss(Im, T, scaled, b)[0]) / (2 * d)
        assert abs(fd - dLdI[idx]) <= 1e-7 * np.max(np.abs(dLdI)), (idx, fd, dLdI[idx])


def test_binned_psnr_hand_computed():
    """2 x 2 simulation pixels under one detector pixel: D = sum I = 2,
    T = 1 -> sigma = 1/2, residual 0, PSNR infinite; plain MSE (2 - 1)^2 = 1."""
    I = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    T = np.array([[[1.0]]])
    L, psnr, dLdI = O.mse_loss(I, T, detector_bin=2)
    assert L == 1.0 and np.isinf(psnr[0])
    assert np.array_equal(dLdI, np.full((1, 2, 2), 2.0))


def test_binned_thickness_gradient_matches_central_differences():
    """The adjoint with a binned loss seed against central differences of the
    whole binned model (FP64)."""
    rng = np.random.default_rng(24)
    lam = np.array([480e-9, 560e-9, 690e-9])
    model = dict(lambdas=lam, gaps=np.array([6e-6, 5e-6, 7e-6]), pitch=0.29e-6, m=32,
                 fov=8, aperture=8, n_index=np.array([1.72, 1.70, 1.68]),
                 kappa=np.array([0.01, 0.02, 0.0]), n_medium=1.0, h_base=30e-9)
    h = rng.uniform(0, 550e-9, size=(2, 16, 16))
    T = rng.uniform(0, 4, size=(3, 4, 4))
    for scaled in (False, True):
        L, psnr, grad, _ = O.loss_and_grad(h, T, scaled=scaled, detector_bin=2, **model)
        pixels = [(0, 8, 8), (1, 5, 11), (0, 2, 14), (1, 9, 7)]
        fd = O.finite_difference(h, T, pixels, 1e-4 * 550e-9, scaled=scaled, detector_bin=2, **model)
        ad = np.array([grad[p] for p in pixels])
        assert np.max(np.abs(ad - fd)) < 1e-6 * np.max(np.abs(ad)), (ad, fd)
