"""Shared helpers of the GPU parity tests: build the CUDA context and the
oracle call for the same design and the same seeded inputs."""
import dataclasses

import numpy as np

from paper_2604_02624_gb300 import workloads as W

# Tolerances (spec: FP32 field relative L2 <= 1e-5, intensity <= 1e-4,
# gradient vs finite differences <= 1e-3 relative).  The gradient against the
# FP64 oracle gradient is held to 1e-4 relative L2: it is a product of a
# forward and an adjoint field (each <= 1e-5) summed over channels in FP32.
TOL_FIELD = 1e-5
TOL_INTENSITY = 1e-4
TOL_GRAD_ORACLE = 1e-4
TOL_GRAD_FD = 1e-3
TOL_LOSS = 1e-4
# Split-BF16 DFT-GEMM path.  Spec target: 1e-4.  Bound derived from the
# arithmetic: a value held as bf16 hi + lo is exact to ~2^-18 relative and the
# dropped lo*lo product is of the same order, so one GEMM adds ~3 * 2^-18 ~ 1.1e-5
# relative L2 error; G chained GEMMs give ~1.1e-5 sqrt(G) on the field (twice that
# on |o|^2).  Tests allow 4x that estimate.
SPLIT_GEMM_EPS = 3 * 2.0 ** -18
# Spec target of the split-BF16 form.  The tensor core's FP32
# accumulation loses a little of every partial sum, so the GEMMs accumulate the
# small products first; then two parts per operand meet the target on every
# geometry (36 chained GEMMs at K = 8) and three parts add little.
SPLIT_TARGET = 1e-4


def split_bound(n_gemms: int, intensity: bool = False) -> float:
    return 4 * SPLIT_GEMM_EPS * n_gemms ** 0.5 * (2 if intensity else 1)


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_model(w: W.Workload, evanescent="decay"):
    return dict(lambdas=w.lambdas, gaps=w.gaps, pitch=w.pitch, m=w.m, fov=w.fov,
                aperture=w.aperture, n_index=w.n_index, kappa=w.kappa,
                n_medium=w.n_medium, h_base=w.h_base, evanescent=evanescent)


def custom(n, m, k, lambdas_nm, gap_lm, fov, aperture=None, n_index=1.7, kappa=0.0,
           n_medium=1.0, h_base=0.0, pitch_lm=0.5, name="custom"):
    lam = np.asarray(lambdas_nm, dtype=np.float64) * 1e-9
    lm = float(lam.mean())
    nw = lam.shape[0]
    gaps = np.broadcast_to(np.asarray(gap_lm, dtype=np.float64), (k + 1,)) * lm
    return W.Workload(name=name, n=n, m=m, n_layers=k, lambdas=lam, gaps=np.array(gaps),
                      pitch=pitch_lm * lm, n_index=np.broadcast_to(np.asarray(n_index, float), (nw,)).copy(),
                      kappa=np.broadcast_to(np.asarray(kappa, float), (nw,)).copy(), fov=fov,
                      aperture=aperture if aperture else fov, n_medium=n_medium, h_base=h_base,
                      target_kind="gray", target_src=min(8, fov))


def replace(w, **kw):
    return dataclasses.replace(w, **kw)
