"""FP64 CPU oracle of the wavelength-multiplexed diffractive storage model.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path and
imports nothing from the product package; its inputs are plain numpy arrays.

It is written to be checked by eye against Section 4 of the paper
("Optical forward model of wavelength-multiplexed diffractive systems"):

* Eq. 1   thin-element transmission t = exp(-2 pi kappa h / lambda)
                                        * exp(-j 2 pi (n - n_air) h / lambda)
* Eq. 2   h = h_learnable + h_base
* Eq. 4   Rayleigh-Sommerfeld secondary wave; realised here by its exact
          Fourier transform, the angular-spectrum transfer function
          H(fx, fy; z) = exp(j 2 pi z sqrt((n/lambda)^2 - fx^2 - fy^2)),
          applied between zero-padded 2D DFTs (library FFT as a step)
* Eq. 5   layer cascade u^{l+1} = t * (sum_s u^l_s w^l_s)
* Section 2: output intensity O_w = |o_w|^2 scored by an MSE against its target,
          the reconstruction quality reported as a PSNR, and the design trained
          by error back-propagation (here: the adjoint of Eq. 1-5, in FP64).

Readings where the paper is silent (listed with reasons in the design notes):
the evanescent branch decays as exp(-2 pi z sqrt(-q)) unless "zero" is chosen;
the layer grid of N x N sits centred in the M x M padded grid and the output
is cropped back to N x N after every gap; the reference index of Eq. 1 is the
surrounding medium's index (air = 1 in every workload); the MSE is the plain
mean over channels and FOV pixels; the PSNR uses the least-squares scaled
output (sigma_w = sum I T / sum I^2) with peak value 1.

All functions take and return float64 / complex128 numpy arrays.  Lengths are
in metres.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# --------------------------------------------------------------------------
# Sampling grid (Section 4: spatial sampling period = feature size)
# --------------------------------------------------------------------------
def spatial_frequencies(m: int, pitch: float) -> np.ndarray:
    """Frequencies of the M DFT bins for samples spaced ``pitch`` apart."""
    return np.fft.fftfreq(m, d=pitch)


def centred_offset(outer: int, inner: int) -> int:
    return (outer - inner) // 2


def pad(u: np.ndarray, m: int) -> np.ndarray:
    """Zero-pad an N x N field into the centre of an M x M grid."""
    n = u.shape[-1]
    o = centred_offset(m, n)
    out = np.zeros((m, m), dtype=np.complex128)
    out[o:o + n, o:o + n] = u
    return out


def crop(big: np.ndarray, n: int) -> np.ndarray:
    """Central N x N window of an M x M grid (the layer aperture)."""
    m = big.shape[-1]
    o = centred_offset(m, n)
    return big[o:o + n, o:o + n].copy()


# --------------------------------------------------------------------------
# Free-space propagation (Eq. 4 -> angular spectrum, Eq. 5 convolution)
# --------------------------------------------------------------------------
def transfer_function(lam: float, z: float, m: int, pitch: float,
                      n_medium: float = 1.0, evanescent: str = "decay") -> np.ndarray:
    """H(fx_k, fy_l; z) for the M x M DFT grid, rows = fy, columns = fx.

    With q = (n/lambda)^2 - fx^2 - fy^2: exp(+j 2 pi z sqrt(q)) for q >= 0
    (the outgoing-wave sign of Eq. 4), exp(-2 pi z sqrt(-q)) for q < 0, or 0
    for q < 0 when ``evanescent == "zero"``.
    """
    f = spatial_frequencies(m, pitch)
    q = (n_medium / lam) ** 2 - f[:, None] ** 2 - f[None, :] ** 2
    H = np.zeros((m, m), dtype=np.complex128)
    prop = q >= 0.0
    H[prop] = np.exp(1j * TWO_PI * z * np.sqrt(q[prop]))
    if evanescent == "decay":
        H[~prop] = np.exp(-TWO_PI * z * np.sqrt(-q[~prop]))
    elif evanescent != "zero":
        raise ValueError(evanescent)
    return H


def gap_transfer(lam, gaps, g, m, pitch, n_medium=1.0, evanescent="decay", displacements=None):
    """Transfer function of gap g (from plane g to plane g+1; plane 0 is the
    input aperture, plane K+1 the detector, both fixed).

    ``displacements`` (K x 3: dx, dy, dz of layers 1..K [m]) describe
    misaligned layers (Section 3, "vaccination").  A layer displaced by D
    modulates with t(r - D); because free space is shift invariant this equals
    shifting the field by -D before the modulation and by +D after it, so gap g
    carries the lateral shift D_g - D_{g+1}, i.e. the factor
    exp(-2 pi j (fx a_x + fy a_y)), and its length becomes z_g + dz_{g+1} - dz_g.
    """
    z = gaps[g]
    if displacements is None:
        return transfer_function(lam, z, m, pitch, n_medium, evanescent)
    d = np.asarray(displacements, np.float64)
    k = d.shape[0]
    pad = np.zeros((k + 2, 3))
    pad[1:k + 1] = d
    a = pad[g] - pad[g + 1]
    H = transfer_function(lam, z + pad[g + 1, 2] - pad[g, 2], m, pitch, n_medium, evanescent)
    f = spatial_frequencies(m, pitch)
    ramp = np.exp(-1j * TWO_PI * (f[None, :] * a[0] + f[:, None] * a[1]))
    return H * ramp


def propagate(u: np.ndarray, H: np.ndarray) -> np.ndarray:
    """P_z(u) = crop_N( IDFT( H * DFT( pad_M(u) ) ) ).

    DFT = unnormalised, kernel exp(-j 2 pi k n / M); IDFT carries 1/M^2.
    With M = N (no padding) this is the periodic propagator.
    """
    n = u.shape[-1]
    m = H.shape[-1]
    return crop(np.fft.ifft2(H * np.fft.fft2(pad(u, m))), n)


def propagate_adjoint(g: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Hermitian adjoint of ``propagate``: the same chain with conj(H)."""
    n = g.shape[-1]
    m = H.shape[-1]
    return crop(np.fft.ifft2(np.conj(H) * np.fft.fft2(pad(g, m))), n)


# --------------------------------------------------------------------------
# Layers (Eq. 1, Eq. 2)
# --------------------------------------------------------------------------
def transmission(h: np.ndarray, lam: float, n_index: float, kappa: float,
                 n_medium: float = 1.0, h_base: float = 0.0) -> np.ndarray:
    """Eq. 1 with h = h_learnable + h_base (Eq. 2)."""
    hh = h + h_base
    amp = np.exp(-TWO_PI * kappa * hh / lam)
    phase = np.exp(-1j * TWO_PI * (n_index - n_medium) * hh / lam)
    return amp * phase


def dtransmission_dh_factor(lam: float, n_index: float, kappa: float,
                            n_medium: float = 1.0) -> complex:
    """c with dt/dh = c * t, from differentiating Eq. 1 in h."""
    return -TWO_PI * (kappa + 1j * (n_index - n_medium)) / lam


def aperture_field(n: int, a: int) -> np.ndarray:
    """Uniform unit-amplitude input field on the centred a x a aperture."""
    u = np.zeros((n, n), dtype=np.complex128)
    o = centred_offset(n, a)
    u[o:o + a, o:o + a] = 1.0
    return u


# --------------------------------------------------------------------------
# Forward model of one design (all channels)
# --------------------------------------------------------------------------
def forward(h, lambdas, gaps, pitch, m, fov, aperture, n_index, kappa,
            n_medium=1.0, h_base=0.0, evanescent="decay", keep_fields=True, displacements=None):
    """Run every channel through the K-layer cascade.

    h: (K, N, N) thicknesses.  Returns a dict with
      ``o``  (N_w, F, F) complex output fields on the FOV,
      ``I``  (N_w, F, F) intensities |o|^2,
      ``v``  (N_w, K, N, N) incoming fields of each layer (before modulation)
             when ``keep_fields``.
    """
    h = np.asarray(h, dtype=np.float64)
    k_layers, n, _ = h.shape
    lambdas = np.asarray(lambdas, dtype=np.float64)
    nw = lambdas.shape[0]
    n_index = np.broadcast_to(np.asarray(n_index, np.float64), (nw,))
    kappa = np.broadcast_to(np.asarray(kappa, np.float64), (nw,))
    gaps = np.asarray(gaps, dtype=np.float64)
    assert gaps.shape[0] == k_layers + 1
    of = centred_offset(n, fov)
    o_all = np.zeros((nw, fov, fov), dtype=np.complex128)
    v_all = np.zeros((nw, k_layers, n, n), dtype=np.complex128) if keep_fields else None
    for w in range(nw):
        lam = lambdas[w]
        v = propagate(aperture_field(n, aperture),
                      gap_transfer(lam, gaps, 0, m, pitch, n_medium, evanescent, displacements))
        for l in range(k_layers):
            if keep_fields:
                v_all[w, l] = v
            u = transmission(h[l], lam, n_index[w], kappa[w], n_medium, h_base) * v
            v = propagate(u, gap_transfer(lam, gaps, l + 1, m, pitch, n_medium, evanescent,
                                          displacements))
        o_all[w] = v[of:of + fov, of:of + fov]
    return {"o": o_all, "I": np.abs(o_all) ** 2, "v": v_all}


# --------------------------------------------------------------------------
# Objective (Section 2) and quality metric
# --------------------------------------------------------------------------
def detector_intensity(I, b):
    """Output pixels of the detector (Section 4: the output FOV is divided into
    25 x 25 pixels, each spanning several diffractive features): pixel (y, x)
    integrates the b x b simulation pixels it covers,
    D[w, y, x] = sum_{i, j < b} I[w, b y + i, b x + j].  b = 1 is the identity."""
    I = np.asarray(I, np.float64)
    nw, f, _ = I.shape
    if f % b:
        raise ValueError("the FOV side must be a multiple of the detector bin")
    fd = f // b
    D = np.zeros((nw, fd, fd))
    for i in range(b):
        for j in range(b):
            D += I[:, i::b, j::b]
    return D


def mse_loss(I, T, scaled=False, detector_bin=1):
    """Loss over all channels and detector pixels; returns (L, psnr[N_w], dL/dI).

    The detector reads D = detector_intensity(I, detector_bin) and T has its
    shape; with detector_bin = 1, D = I.
    plain:  L = mean_{w,p} (D - T)^2
    scaled: L = mean_{w,p} (sigma_w D - T)^2, sigma_w = sum_p D T / sum_p D^2;
            dL/dD holds sigma_w fixed, which is exact because sigma_w minimises
            the per-channel error.
    PSNR_w = 10 log10(1 / mean_p (sigma_w D - T)^2) (peak value 1).
    dL/dI of a simulation pixel is dL/dD of the detector pixel that covers it.
    """
    b = int(detector_bin)
    I = detector_intensity(I, b)
    T = np.asarray(T, np.float64)
    nw = I.shape[0]
    cnt = I[0].size
    sigma = np.array([np.sum(I[w] * T[w]) / np.sum(I[w] * I[w]) for w in range(nw)])
    mse_scaled = np.array([np.mean((sigma[w] * I[w] - T[w]) ** 2) for w in range(nw)])
    with np.errstate(divide="ignore"):
        psnr = 10.0 * np.log10(1.0 / mse_scaled)
    if scaled:
        L = np.sum(mse_scaled) / nw
        dLdI = np.stack([2.0 * sigma[w] * (sigma[w] * I[w] - T[w]) for w in range(nw)])
    else:
        L = np.sum((I - T) ** 2) / (nw * cnt)
        dLdI = 2.0 * (I - T)
    dLdI = np.repeat(np.repeat(dLdI, b, axis=1), b, axis=2)
    return L, psnr, dLdI / (nw * cnt)


# --------------------------------------------------------------------------
# Gradient by the adjoint of the cascade
# --------------------------------------------------------------------------
def backward(h, fwd, dLdI, lambdas, gaps, pitch, m, fov, n_index, kappa,
             n_medium=1.0, h_base=0.0, evanescent="decay", displacements=None):
    """dL/dh (K, N, N) for a real loss with gradient ``dLdI`` w.r.t. I = |o|^2.

    Convention: for complex z, grad_z L = dL/dRe z + j dL/dIm z.
      I = |o|^2          -> grad_o = 2 dL/dI o
      o = FOV crop of v  -> grad_v = zero-pad of grad_o
      v' = P_z u         -> grad_u = P_z^H grad_v'
      u = t v            -> grad_v = conj(t) grad_u,
                            dL/dh = Re(conj(grad_u) * c * u), c = dt/dh / t
    summed over the channels (the thickness is shared by every wavelength).
    """
    h = np.asarray(h, dtype=np.float64)
    k_layers, n, _ = h.shape
    lambdas = np.asarray(lambdas, dtype=np.float64)
    nw = lambdas.shape[0]
    n_index = np.broadcast_to(np.asarray(n_index, np.float64), (nw,))
    kappa = np.broadcast_to(np.asarray(kappa, np.float64), (nw,))
    of = centred_offset(n, fov)
    grad = np.zeros_like(h)
    for w in range(nw):
        lam = lambdas[w]
        g = np.zeros((n, n), dtype=np.complex128)
        g[of:of + fov, of:of + fov] = 2.0 * dLdI[w] * fwd["o"][w]
        for l in reversed(range(k_layers)):
            H = gap_transfer(lam, gaps, l + 1, m, pitch, n_medium, evanescent, displacements)
            a_u = propagate_adjoint(g, H)
            t = transmission(h[l], lam, n_index[w], kappa[w], n_medium, h_base)
            u = t * fwd["v"][w, l]
            c = dtransmission_dh_factor(lam, n_index[w], kappa[w], n_medium)
            grad[l] += np.real(np.conj(a_u) * c * u)
            g = np.conj(t) * a_u
    return grad


def loss_and_grad(h, T, lambdas, gaps, pitch, m, fov, aperture, n_index, kappa,
                  n_medium=1.0, h_base=0.0, evanescent="decay", scaled=False, displacements=None,
                  detector_bin=1):
    fwd = forward(h, lambdas, gaps, pitch, m, fov, aperture, n_index, kappa,
                  n_medium, h_base, evanescent, displacements=displacements)
    L, psnr, dLdI = mse_loss(fwd["I"], T, scaled, detector_bin)
    grad = backward(h, fwd, dLdI, lambdas, gaps, pitch, m, fov, n_index, kappa,
                    n_medium, h_base, evanescent, displacements=displacements)
    return L, psnr, grad, fwd


def loss_only(h, T, lambdas, gaps, pitch, m, fov, aperture, n_index, kappa,
              n_medium=1.0, h_base=0.0, evanescent="decay", scaled=False, displacements=None,
              detector_bin=1):
    fwd = forward(h, lambdas, gaps, pitch, m, fov, aperture, n_index, kappa,
                  n_medium, h_base, evanescent, keep_fields=False, displacements=displacements)
    return mse_loss(fwd["I"], T, scaled, detector_bin)[0]


def finite_difference(h, T, pixels, delta, **model):
    """Central differences of the loss at the listed (layer, y, x) pixels."""
    out = []
    for (l, y, x) in pixels:
        hp = np.array(h, dtype=np.float64, copy=True)
        hm = hp.copy()
        hp[l, y, x] += delta
        hm[l, y, x] -= delta
        out.append((loss_only(hp, T, **model) - loss_only(hm, T, **model)) / (2 * delta))
    return np.array(out)


# --------------------------------------------------------------------------
# Direct Rayleigh-Sommerfeld sum of Eq. 4-5 (cross-check of the realisation)
# --------------------------------------------------------------------------
def rayleigh_sommerfeld_direct(u: np.ndarray, lam: float, z: float, pitch: float,
                               n_medium: float = 1.0) -> np.ndarray:
    """Field on an N x N plane at distance z from the N x N source plane by the
    literal superposition of the secondary waves of Eq. 4, times the area
    element pitch^2 that turns Eq. 5's sum into a Riemann sum."""
    n = u.shape[-1]
    c = (np.arange(n) - (n - 1) / 2.0) * pitch
    X, Y = np.meshgrid(c, c)
    xs = X.ravel()
    ys = Y.ravel()
    us = u.ravel()
    out = np.zeros(n * n, dtype=np.complex128)
    for p in range(n * n):
        r = np.sqrt((xs[p] - xs) ** 2 + (ys[p] - ys) ** 2 + z ** 2)
        w = z / r ** 2 * (1.0 / (TWO_PI * r) + n_medium / (1j * lam)) \
            * np.exp(1j * TWO_PI * n_medium * r / lam)
        out[p] = np.sum(us * w) * pitch ** 2
    return out.reshape(n, n)


# --------------------------------------------------------------------------
# Evaluation variants of a trained design (Section 2 Fig. 5-7, Section 3)
# --------------------------------------------------------------------------
def quantize_level(h, h_max, bits):
    """Level index of the phase bit depth B (Fig. 7): the learnable thickness,
    limited to [0, h_max], is sent to the nearest of the 2^B evenly spaced
    levels k h_max / (2^B - 1), k = 0 .. 2^B - 1.  Nearest level by the
    definition, in FP64: k = rint(clip(h, 0, h_max) (2^B - 1) / h_max)
    (an exact half step goes to the even level)."""
    levels = 2 ** bits - 1
    hc = np.clip(np.asarray(h, np.float64), 0.0, float(h_max))
    return np.rint(hc * (levels / float(h_max))).astype(np.int64)


def quantize_thickness(h, h_max, bits):
    """Thickness of the nearest level (Fig. 7): k h_max / (2^B - 1), in FP64."""
    levels = 2 ** bits - 1
    return quantize_level(h, h_max, bits).astype(np.float64) * (float(h_max) / levels)


def channel_swap(psnr, lambdas):
    """Dynamic channel swapping (Section 2, the Fig. 2B text): after a first
    training run the images are ranked by their PSNR, best first, and handed
    out again to the wavelengths from the longest one down.  Returns perm with
    new_targets[c] = targets[perm[c]]; equal PSNRs (or wavelengths) keep their
    index order."""
    n = len(psnr)
    images = sorted(range(n), key=lambda i: (-float(psnr[i]), i))        # best image first
    channels = sorted(range(n), key=lambda c: (-float(lambdas[c]), c))   # longest wavelength first
    perm = np.empty(n, dtype=np.int64)
    for rank in range(n):
        perm[channels[rank]] = images[rank]
    return perm


def diffraction_efficiency(I, aperture):
    """Output diffraction efficiency (Section 2, Fig. 5): power on the output
    FOV over the power of the unit-amplitude input aperture (A^2 pixels)."""
    I = np.asarray(I, np.float64)
    return I.reshape(I.shape[0], -1).sum(axis=1) / float(aperture * aperture)
