"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against mathematics or textbook physics chosen so
that a plausible slip in it (a wrong sign, a transposed axis, a dropped
normalisation, a wrong frequency grid, an off-by-one crop) fails at least one
of them:

* brute-force DFT sums on tiny grids           -> FFT convention, 1/M^2, pad/crop
* z = 0 identity                                -> normalisation and alignment
* z1 + z2 composition (periodic)                -> phase linear in z
* plane waves with kz from |k| = 2 pi n/lambda  -> frequency grid, axis order, sign
* Parseval with every bin propagating           -> unitarity of the propagator
* Talbot self-imaging and half-period shift     -> non-paraxial dispersion
* Gaussian beam: exact Hankel quadrature and
  the paraxial closed form                      -> H as physics, pitch scaling
* direct Rayleigh-Sommerfeld sum (Eq. 4)        -> realisation of Eq. 4 by ASM
* transmission closed forms (Eq. 1)             -> Eq. 1 and layout of h
* dot-product test and central differences      -> adjoint and gradient
* hand-computed loss / PSNR                      -> objective and metric
"""
import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

from oracle import dos_oracle as O

LAM = 600e-9


def _rand_field(rng, n):
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


# --------------------------------------------------------------------------
# Propagator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(5, 8), (4, 9), (6, 6), (3, 10)])
def test_propagate_equals_bruteforce_dft_sums(n, m):
    """P_z written out with explicit DFT double sums (no FFT library)."""
    rng = np.random.default_rng(3)
    u = _rand_field(rng, n)
    pitch = 0.4 * LAM
    H = O.transfer_function(LAM, 3.0 * LAM, m, pitch, 1.0, "decay")
    o = (m - n) // 2
    big = np.zeros((m, m), complex)
    big[o:o + n, o:o + n] = u
    # forward DFT: U[k,l] = sum_{y,x} big[y,x] exp(-2 pi j (k y + l x)/m)
    U = np.zeros((m, m), complex)
    for k in range(m):
        for l in range(m):
            acc = 0j
            for y in range(m):
                for x in range(m):
                    acc += big[y, x] * np.exp(-2j * np.pi * (k * y + l * x) / m)
            U[k, l] = acc
    V = H * U
    out = np.zeros((m, m), complex)
    for y in range(m):
        for x in range(m):
            acc = 0j
            for k in range(m):
                for l in range(m):
                    acc += V[k, l] * np.exp(2j * np.pi * (k * y + l * x) / m)
            out[y, x] = acc / (m * m)
    ref = out[o:o + n, o:o + n]
    got = O.propagate(u, H)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("evan", ["decay", "zero"])
def test_zero_distance_is_identity(evan):
    rng = np.random.default_rng(1)
    u = _rand_field(rng, 12)
    H = O.transfer_function(LAM, 0.0, 24, 0.3 * LAM, 1.0, "decay")
    assert np.allclose(H, 1.0)
    assert np.max(np.abs(O.propagate(u, H) - u)) < 1e-14 * 12
    Hz = O.transfer_function(LAM, 0.0, 24, 0.3 * LAM, 1.0, evan)
    if evan == "zero":
        # only propagating bins survive: |Hz| is an indicator, idempotent
        assert set(np.unique(np.round(np.abs(Hz), 12))) <= {0.0, 1.0}


@pytest.mark.parametrize("evan", ["decay", "zero"])
def test_composition_periodic(evan):
    """Without padding (M = N) propagation is a semigroup in z."""
    rng = np.random.default_rng(2)
    n = 16
    u = _rand_field(rng, n)
    pitch = 0.45 * LAM
    z1, z2 = 7.3 * LAM, 11.9 * LAM
    H1 = O.transfer_function(LAM, z1, n, pitch, 1.3, evan)
    H2 = O.transfer_function(LAM, z2, n, pitch, 1.3, evan)
    H12 = O.transfer_function(LAM, z1 + z2, n, pitch, 1.3, evan)
    a = O.propagate(O.propagate(u, H1), H2)
    b = O.propagate(u, H12)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("a,b", [(3, 1), (1, 5), (13, 2), (8, 8), (0, 0)])
def test_plane_wave_picks_up_kz_phase(a, b):
    """A plane wave exp(j(kx x + ky y)) in a periodic window is an eigenmode of
    free space; travelling a distance z in +z it gains exp(+j kz z) with
    kx^2 + ky^2 + kz^2 = (2 pi n / lambda)^2 (outgoing sign of Eq. 4)."""
    m = 16
    pitch = 0.7 * LAM
    n_med = 1.2
    z = 5.5 * LAM
    y, x = np.mgrid[0:m, 0:m]
    u = np.exp(2j * np.pi * (a * x + b * y) / m)
    # wave-vector components of the bin (negative frequencies past m/2)
    fa = a if a < m / 2 else a - m
    fb = b if b < m / 2 else b - m
    kx = 2 * np.pi * fa / (m * pitch)
    ky = 2 * np.pi * fb / (m * pitch)
    k0 = 2 * np.pi * n_med / LAM
    kz2 = k0 ** 2 - kx ** 2 - ky ** 2
    expected = np.exp(1j * np.sqrt(kz2) * z) if kz2 >= 0 else np.exp(-np.sqrt(-kz2) * z)
    H = O.transfer_function(LAM, z, m, pitch, n_med, "decay")
    out = O.propagate(u, H)
    assert np.max(np.abs(out - expected * u)) < 1e-12


def test_parseval_when_every_bin_propagates():
    """With pitch >= lambda/(n sqrt 2) no bin is evanescent and the periodic
    propagator is unitary; with padding and cropping energy cannot grow."""
    rng = np.random.default_rng(4)
    n = 20
    u = _rand_field(rng, n)
    pitch = LAM / np.sqrt(2) * 1.01
    H = O.transfer_function(LAM, 37.0 * LAM, n, pitch, 1.0, "decay")
    assert np.all(np.abs(np.abs(H) - 1) < 1e-14)
    v = O.propagate(u, H)
    assert abs(np.linalg.norm(v) / np.linalg.norm(u) - 1) < 1e-13
    Hp = O.transfer_function(LAM, 37.0 * LAM, 2 * n, pitch, 1.0, "decay")
    assert np.linalg.norm(O.propagate(u, Hp)) <= np.linalg.norm(u) * (1 + 1e-13)


def test_talbot_self_imaging():
    """u = 1 + cos(2 pi x / d) reproduces itself (times the on-axis phase)
    after the non-paraxial Talbot length z_T = lambda' / (1 - sqrt(1 - (lambda'/d)^2)),
    lambda' = lambda / n, and shows the half-period shifted copy at z_T / 2."""
    m = 32
    pitch = 0.5 * LAM
    d_px = 8
    d = d_px * pitch
    n_med = 1.0
    lam_med = LAM / n_med
    zt = lam_med / (1 - np.sqrt(1 - (lam_med / d) ** 2))
    y, x = np.mgrid[0:m, 0:m]
    u = 1 + np.cos(2 * np.pi * x / d_px)
    on_axis = np.exp(2j * np.pi * n_med * zt / LAM)
    v = O.propagate(u, O.transfer_function(LAM, zt, m, pitch, n_med))
    assert np.max(np.abs(v - on_axis * u)) < 1e-11
    vh = O.propagate(u, O.transfer_function(LAM, zt / 2, m, pitch, n_med))
    shifted = 1 - np.cos(2 * np.pi * x / d_px)
    assert np.max(np.abs(vh - np.exp(1j * np.pi * n_med * zt / LAM) * shifted)) < 1e-11


def _gaussian_setup():
    n, m = 128, 256
    pitch = 0.5 * LAM
    w0 = 6 * LAM         # window edge at 5.3 w0: truncation below 1e-12
    c = (np.arange(n) - n // 2) * pitch        # pixel n//2 is the beam axis
    X, Y = np.meshgrid(c, c)
    u0 = np.exp(-(X ** 2 + Y ** 2) / w0 ** 2)
    return n, m, pitch, w0, X, Y, u0


@pytest.mark.parametrize("n_med", [1.0, 1.33])
def test_gaussian_beam_exact_hankel(n_med):
    """Exact scalar propagation of a Gaussian: its angular spectrum
    A(f) = pi w0^2 exp(-(pi w0 f)^2), each component advanced by
    exp(j 2 pi z sqrt((n/lambda)^2 - f^2)), summed back by a Hankel (J0) integral."""
    n, m, pitch, w0, X, Y, u0 = _gaussian_setup()
    z = 25 * LAM
    v = O.propagate(u0, O.transfer_function(LAM, z, m, pitch, n_med))
    f = np.linspace(0.0, 9.0 / (np.pi * w0), 40001)
    A = np.pi * w0 ** 2 * np.exp(-(np.pi * w0 * f) ** 2)
    kz = np.sqrt(np.maximum((n_med / LAM) ** 2 - f ** 2, 0.0))
    for (iy, ix) in [(64, 64), (64, 76), (56, 71), (46, 64), (64, 36)]:
        r = np.hypot(X[iy, ix], Y[iy, ix])
        ref = integrate.simpson(2 * np.pi * f * A * sp.j0(2 * np.pi * f * r)
                                * np.exp(2j * np.pi * z * kz), x=f)
        assert abs(v[iy, ix] - ref) < 1e-9, (iy, ix, v[iy, ix], ref)


def test_gaussian_beam_paraxial_closed_form():
    """Textbook paraxial Gaussian beam (outgoing convention exp(+jkz)):
    u = w0/w exp(-r^2/w^2) exp(j(kz + k r^2/(2R) - psi)); agreement is limited
    by the paraxial approximation, (lambda / (pi w0))^2 ~ 2.8e-3 here."""
    n, m, pitch, w0, X, Y, u0 = _gaussian_setup()
    z = 25 * LAM
    v = O.propagate(u0, O.transfer_function(LAM, z, m, pitch, 1.0))
    k = 2 * np.pi / LAM
    zr = np.pi * w0 ** 2 / LAM
    w = w0 * np.sqrt(1 + (z / zr) ** 2)
    R = z * (1 + (zr / z) ** 2)
    psi = np.arctan(z / zr)
    r2 = X ** 2 + Y ** 2
    ref = w0 / w * np.exp(-r2 / w ** 2) * np.exp(1j * (k * z + k * r2 / (2 * R) - psi))
    err = np.max(np.abs(v - ref)) / np.max(np.abs(ref))
    assert err < 5e-3
    # the conjugate (wrong-direction) propagation is far off
    assert np.max(np.abs(np.conj(v) * np.exp(2j * k * z) - ref)) > 0.1


def test_angular_spectrum_matches_rayleigh_sommerfeld_sum():
    """Eq. 4-5 summed literally (with the pitch^2 area element) agree with the
    angular-spectrum realisation up to sampling error (a few 1e-2 on a 24x24
    grid at half-wavelength pitch)."""
    n = 24
    pitch = 0.5 * LAM
    z = 10 * LAM
    u = O.aperture_field(n, 8).astype(complex)
    rs = O.rayleigh_sommerfeld_direct(u, LAM, z, pitch, 1.0)
    # large padding so the circular convolution equals the linear one
    asm = O.propagate(u, O.transfer_function(LAM, z, 4 * n, pitch, 1.0))
    rel = np.linalg.norm(asm - rs) / np.linalg.norm(rs)
    assert rel < 0.05, rel
    # a sign slip in the propagation phase would be O(1) off
    asm_conj = O.propagate(u, np.conj(O.transfer_function(LAM, z, 4 * n, pitch, 1.0)))
    assert np.linalg.norm(asm_conj - rs) / np.linalg.norm(rs) > 0.5


# --------------------------------------------------------------------------
# Transmission (Eq. 1, Eq. 2)
# --------------------------------------------------------------------------
def test_transmission_closed_forms():
    lam, n_idx = 550e-9, 1.62
    assert O.transmission(np.zeros((2, 2)), lam, n_idx, 0.3)[0, 0] == 1.0
    full_wave = lam / (n_idx - 1.0)     # one full 2 pi phase delay, no loss
    assert abs(O.transmission(np.array([full_wave]), lam, n_idx, 0.0)[0] - 1) < 1e-14
    half_wave = 0.5 * full_wave          # pi phase -> -1
    assert abs(O.transmission(np.array([half_wave]), lam, n_idx, 0.0)[0] + 1) < 1e-14
    quarter = 0.25 * full_wave           # exp(-j pi/2) = -j (Eq. 1 sign)
    assert abs(O.transmission(np.array([quarter]), lam, n_idx, 0.0)[0] + 1j) < 1e-14
    h = np.array([123e-9])
    kap = 0.02
    assert abs(abs(O.transmission(h, lam, n_idx, kap)[0])
               - np.exp(-2 * np.pi * kap * 123e-9 / lam)) < 1e-15
    # base thickness simply adds (Eq. 2)
    t1 = O.transmission(h, lam, n_idx, kap, 1.0, 50e-9)
    t2 = O.transmission(h + 50e-9, lam, n_idx, kap, 1.0, 0.0)
    assert abs(t1[0] - t2[0]) < 1e-15


def test_layer_layout_with_zero_gaps():
    """With zero gaps the output is the transmission itself, pixel by pixel, so
    the (layer, y, x) layout of h must show up unchanged (and untransposed) in I."""
    rng = np.random.default_rng(5)
    n, fov = 10, 6
    h = rng.uniform(0, 500e-9, size=(2, n, n))
    lam = np.array([520e-9, 610e-9])
    kap = np.array([0.05, 0.02])
    out = O.forward(h, lam, [0.0, 0.0, 0.0], 0.3e-6, 16, fov, fov, 1.5, kap)
    of = (n - fov) // 2
    for w in range(2):
        expect = np.exp(-4 * np.pi * kap[w] * (h[0] + h[1]) / lam[w])[of:of + fov, of:of + fov]
        assert np.max(np.abs(out["I"][w] - expect)) < 1e-14


def test_mirror_symmetry_of_the_cascade():
    """Free space and centred apertures are mirror symmetric: flipping every
    layer left-right flips every output left-right (an off-by-one in any of
    the centred pad / crop / FOV offsets breaks this)."""
    rng = np.random.default_rng(6)
    n, m, fov = 12, 24, 6
    h = rng.uniform(0, 600e-9, size=(2, n, n))
    lam = np.array([500e-9, 700e-9])
    kw = dict(gaps=[4e-6, 3e-6, 5e-6], pitch=0.3e-6, m=m, fov=fov, aperture=8,
              n_index=1.7, kappa=0.01)
    a = O.forward(h, lam, **kw)["I"]
    b = O.forward(h[:, :, ::-1], lam, **kw)["I"]
    assert np.max(np.abs(a[:, :, ::-1] - b)) < 1e-13 * np.max(a)
    c = O.forward(h[:, ::-1, :], lam, **kw)["I"]
    assert np.max(np.abs(a[:, ::-1, :] - c)) < 1e-13 * np.max(a)


# --------------------------------------------------------------------------
# Adjoint and gradient
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,evan", [(9, 16, "decay"), (8, 8, "decay"), (7, 20, "zero")])
def test_adjoint_dot_product(n, m, evan):
    rng = np.random.default_rng(7)
    x = _rand_field(rng, n)
    y = _rand_field(rng, n)
    H = O.transfer_function(LAM, 4.2 * LAM, m, 0.35 * LAM, 1.0, evan)
    lhs = np.vdot(y, O.propagate(x, H))
    rhs = np.vdot(O.propagate_adjoint(y, H), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _small_model():
    lam = np.array([480e-9, 560e-9, 690e-9])
    return dict(lambdas=lam, gaps=np.array([6e-6, 5e-6, 7e-6]), pitch=0.29e-6, m=32,
                fov=8, aperture=8, n_index=np.array([1.72, 1.70, 1.68]),
                kappa=np.array([0.01, 0.02, 0.0]), n_medium=1.0, h_base=30e-9)


@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("evan", ["decay", "zero"])
def test_gradient_matches_central_differences(scaled, evan):
    rng = np.random.default_rng(8)
    model = _small_model()
    model["evanescent"] = evan
    h = rng.uniform(0, 550e-9, size=(2, 16, 16))
    T = rng.uniform(0, 1, size=(3, 8, 8))
    L, psnr, grad, _ = O.loss_and_grad(h, T, scaled=scaled, **model)
    pixels = [(0, 8, 8), (1, 5, 11), (0, 2, 14), (1, 9, 7), (0, 15, 0)]
    fd = O.finite_difference(h, T, pixels, 1e-4 * 550e-9, scaled=scaled, **model)
    ad = np.array([grad[p] for p in pixels])
    assert np.max(np.abs(ad - fd)) < 1e-6 * np.max(np.abs(ad)), (ad, fd)


def test_gradient_tiny_workload_central_differences():
    from paper_2604_02624_gb300 import workloads as W
    w = W.workload("tiny")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    model = dict(lambdas=w.lambdas, gaps=w.gaps, pitch=w.pitch, m=w.m, fov=w.fov,
                 aperture=w.aperture, n_index=w.n_index, kappa=w.kappa)
    L, psnr, grad, _ = O.loss_and_grad(h, T, **model)
    pixels = [(0, 32, 32), (0, 20, 40), (0, 47, 17)]
    fd = O.finite_difference(h, T, pixels, 1e-4 * w.lambda_mean, **model)
    ad = np.array([grad[p] for p in pixels])
    assert np.max(np.abs(ad - fd) / np.abs(ad)) < 1e-6, (ad, fd)


# --------------------------------------------------------------------------
# Objective and metric
# --------------------------------------------------------------------------
def test_loss_zero_when_output_equals_target():
    rng = np.random.default_rng(9)
    I = rng.uniform(0, 1, size=(3, 5, 5))
    L, psnr, dLdI = O.mse_loss(I, I)
    assert L == 0.0 and np.all(dLdI == 0.0) and np.all(np.isinf(psnr))


def test_loss_hand_computed_2x2():
    """I = [[1,0],[0,1]], T = [[0.5,0],[0,0]]:
    plain MSE = (0.25 + 1)/4 = 0.3125;
    sigma = sum IT / sum I^2 = 0.5/2 = 0.25, residual [[-0.25,0],[0,0.25]],
    scaled MSE = 0.125/4 = 0.03125, PSNR = 10 log10(32) dB."""
    I = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    T = np.array([[[0.5, 0.0], [0.0, 0.0]]])
    L, psnr, dLdI = O.mse_loss(I, T)
    assert abs(L - 0.3125) < 1e-16
    assert abs(psnr[0] - 15.051499783199060) < 1e-12
    assert np.allclose(dLdI, 2 * (I - T) / 4)
    Ls, psnr_s, dLdI_s = O.mse_loss(I, T, scaled=True)
    assert abs(Ls - 0.03125) < 1e-16
    assert np.allclose(dLdI_s, 2 * 0.25 * np.array([[[-0.25, 0], [0, 0.25]]]) / 4)
