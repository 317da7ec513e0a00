"""Seeded synthetic workloads for the diffractive-storage forward/adjoint path.

This module only *draws inputs*: geometry of the five workload families, seeded
thickness maps and seeded target patterns.  It holds none of the method's
arithmetic (no transmission, no propagation, no loss), so that both the CUDA
path and the FP64 CPU oracle can be fed the very same arrays without sharing
any computation.

Workload families (sizes follow the paper's storage designs, scaled to what a
test or a single GPU step can hold):

* ``tiny``      1 layer, 64x64 pixels padded to 128, 4 wavelengths 500-740 nm,
                n = 1.7, no loss, 32x32 FOV, binary 8x8 targets upsampled x4.
* ``small``     2 layers, 200x200 padded to 400, 6 wavelengths 500..740 nm
                (the experimental set of Section 2), n = 1.7, kappa = 0.01,
                50x50 FOV, grey 28x28 targets box-smoothed and upsampled.
* ``batched``   5 layers of 200x200 padded to 400, gaps of 210 mean
                wavelengths (axial span ~1260 lambda_m, Fig. 1), 256
                wavelengths 450-750 nm, n = 1.7, no loss.
* ``massive``   as ``batched`` with 4096 wavelengths and kappa = 0.01.
* ``precision`` 8 layers of 256x256 padded to 512, gaps 160 lambda_m,
                4096 wavelengths 450-750 nm, 64x64 FOV, grey 32x32 targets.

All lengths are in metres.  The pitch is half the mean wavelength of the
list; the aperture equals the FOV and both are centred in the layer.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

NM = 1e-9


@dataclasses.dataclass
class Workload:
    name: str
    n: int                      # thickness pixels per side (layer grid N)
    m: int                      # zero-padded FFT size M
    n_layers: int               # K
    lambdas: np.ndarray         # (N_w,) vacuum wavelengths [m]
    gaps: np.ndarray            # (K+1,) distances [m]: input->L1, L1->L2, ..., LK->output
    pitch: float                # sampling period [m]
    n_index: np.ndarray         # (N_w,) real part of the layer index
    kappa: np.ndarray           # (N_w,) extinction coefficient of the layer
    fov: int                    # output field-of-view side F (pixels)
    aperture: int               # input aperture side A (pixels)
    n_medium: float = 1.0
    h_base: float = 0.0
    target_kind: str = "gray"   # "gray" | "binary"
    target_src: int = 28        # low-resolution target side before upsampling
    h_fp64: bool = False        # thickness drawn and kept in FP64 (tiny case only)

    @property
    def n_lambda(self) -> int:
        return int(self.lambdas.shape[0])

    @property
    def lambda_mean(self) -> float:
        return float(np.mean(self.lambdas))

    def subset(self, idx: Sequence[int]) -> "Workload":
        """Same design restricted to the listed wavelength channels."""
        idx = np.asarray(idx, dtype=np.int64)
        return dataclasses.replace(
            self,
            name=f"{self.name}[{len(idx)}ch]",
            lambdas=self.lambdas[idx].copy(),
            n_index=self.n_index[idx].copy(),
            kappa=self.kappa[idx].copy(),
        )


def _family(name, n, m, k, lam_nm, gap_in_lm, n_idx, kappa, fov, kind, src,
            h_fp64=False) -> Workload:
    lam = np.asarray(lam_nm, dtype=np.float64) * NM
    lam_m = float(np.mean(lam))
    nw = lam.shape[0]
    return Workload(
        name=name, n=n, m=m, n_layers=k, lambdas=lam,
        gaps=np.full(k + 1, gap_in_lm * lam_m), pitch=0.5 * lam_m,
        n_index=np.full(nw, n_idx), kappa=np.full(nw, kappa),
        fov=fov, aperture=fov, target_kind=kind, target_src=src, h_fp64=h_fp64)


def workload(name: str, n_lambda: Optional[int] = None) -> Workload:
    """Build one of the named workload families.

    ``n_lambda`` overrides the channel count of the 450-750 nm families (used by
    tests that need the same geometry with fewer channels).
    """
    if name == "tiny":
        return _family("tiny", 64, 128, 1, [500, 580, 660, 740], 40, 1.7, 0.0,
                       32, "binary", 8, h_fp64=True)
    if name == "small":
        return _family("small", 200, 400, 2, np.linspace(500, 740, 6), 100, 1.7,
                       0.01, 50, "gray", 28)
    if name in ("batched", "massive"):
        nw = n_lambda or (256 if name == "batched" else 4096)
        kap = 0.0 if name == "batched" else 0.01
        return _family(name, 200, 400, 5, np.linspace(450, 750, nw), 210, 1.7,
                       kap, 50, "gray", 28)
    if name == "precision":
        nw = n_lambda or 4096
        return _family("precision", 256, 512, 8, np.linspace(450, 750, nw), 160,
                       1.7, 0.01, 64, "gray", 32)
    raise KeyError(name)


WORKLOADS = ("tiny", "small", "batched", "massive", "precision")


def thickness(w: Workload, seed: int = 0) -> np.ndarray:
    """h_l[y, x] ~ U[0, lambda_m) per pixel, shape (K, N, N).

    Drawn in FP64 from PCG64(seed); rounded to FP32 unless the workload keeps
    FP64 thickness.  Returned as float64 holding exactly the values both sides use.
    """
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.0, w.lambda_mean, size=(w.n_layers, w.n, w.n))
    if not w.h_fp64:
        h = h.astype(np.float32).astype(np.float64)
    return h


def _box3_inbounds(img: np.ndarray) -> np.ndarray:
    """3x3 mean over the in-bounds neighbours of each pixel (last two axes)."""
    s = img.shape[-1]
    pad = np.zeros(img.shape[:-2] + (s + 2, s + 2))
    pad[..., 1:-1, 1:-1] = img
    ones = np.zeros((s + 2, s + 2))
    ones[1:-1, 1:-1] = 1.0
    acc = np.zeros_like(img)
    cnt = np.zeros((s, s))
    for dy in range(3):
        for dx in range(3):
            acc += pad[..., dy:dy + s, dx:dx + s]
            cnt += ones[dy:dy + s, dx:dx + s]
    return acc / cnt


def _upsample_nearest(img: np.ndarray, out: int) -> np.ndarray:
    src = img.shape[-1]
    idx = (np.arange(out) * src) // out
    return img[..., idx[:, None], idx[None, :]]


def targets(w: Workload, seed: int = 1) -> np.ndarray:
    """Target patterns T_w in [0, 1], shape (N_w, F, F), float32 values in float64.

    Grey: i.i.d. U[0,1] on a src x src grid, 3x3 box-smoothed (in-bounds mean),
    nearest-upsampled to F x F.  Binary: {0,1} on src x src, nearest-upsampled.
    They stand in for the paper's CIFAR100 / MNIST targets, which are absent.
    """
    rng = np.random.default_rng(seed)
    s = w.target_src
    if w.target_kind == "binary":
        low = rng.integers(0, 2, size=(w.n_lambda, s, s)).astype(np.float64)
    else:
        low = _box3_inbounds(rng.uniform(0.0, 1.0, size=(w.n_lambda, s, s)))
    t = _upsample_nearest(low, w.fov)
    return np.ascontiguousarray(t.astype(np.float32).astype(np.float64))


def subset_indices(n_lambda: int, count: int) -> np.ndarray:
    """``count`` channel indices evenly spread over ``n_lambda`` (ends included)."""
    count = min(count, n_lambda)
    return np.unique(np.round(np.linspace(0, n_lambda - 1, count)).astype(np.int64))
