"""PyTorch-facing API of the diffractive-storage engine.

PyTorch supplies device memory and the CUDA stream; every step of the forward
model, the objective and the adjoint runs in libdos.so kernels through the C
ABI (see ``_lib``).  Tensors passed in must be contiguous CUDA tensors of the
documented dtype on the context's device.

* :class:`DiffractiveStack` - one design (geometry, wavelength list, material)
  bound to a device; ``forward``, ``loss``, ``backward``, ``propagate``.
* :class:`DosFunction` - ``torch.autograd.Function`` whose forward is
  ``dos_forward`` and whose backward is ``dos_backward`` (the hand-written
  adjoint), so any torch objective of the intensities composes with it.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _need(t: torch.Tensor, dtype, shape, name: str, device) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name} must live on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class DiffractiveStack:
    """A K-layer thickness-coded diffractive design evaluated at N_w wavelengths.

    Lengths in metres.  ``gaps`` has K+1 entries (input->L1, ..., LK->output).
    """

    def __init__(self, *, n: int, m: int, n_layers: int, lambdas: Sequence[float],
                 gaps: Sequence[float], pitch: float, n_index, kappa=None, fov: int,
                 aperture: int = 0, n_medium: float = 1.0, h_base: float = 0.0,
                 evanescent: str = "decay", loss: str = "mse", n_lambda_total: int = 0,
                 path: str = "auto", detector_bin: int = 1, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        nw = lam.shape[0]
        self._lam = lam
        self._gaps = np.ascontiguousarray(gaps, dtype=np.float64)
        self._nidx = np.ascontiguousarray(np.broadcast_to(np.asarray(n_index, np.float64), (nw,)))
        self._kap = None if kappa is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(kappa, np.float64), (nw,)))
        if self._gaps.shape[0] != n_layers + 1:
            raise ValueError("gaps must have n_layers + 1 entries")
        self.n, self.m, self.n_layers, self.n_lambda, self.fov = n, m, n_layers, nw, fov
        self.detector_bin = max(1, int(detector_bin))
        self.det = fov // self.detector_bin  # detector pixels per side (targets, PSNR)
        cfg = L.DosConfig()
        cfg.n, cfg.m, cfg.n_layers, cfg.n_lambda = n, m, n_layers, nw
        cfg.n_lambda_total = n_lambda_total
        cfg.fov, cfg.aperture, cfg.pitch = fov, aperture, pitch
        cfg.gaps = L._dptr(self._gaps)
        cfg.lambda_ = L._dptr(self._lam)
        cfg.n_index = L._dptr(self._nidx)
        cfg.kappa = L._dptr(self._kap)
        cfg.n_medium, cfg.h_base = n_medium, h_base
        cfg.evanescent = {"decay": L.DOS_EVAN_DECAY, "zero": L.DOS_EVAN_ZERO}[evanescent]
        cfg.loss = {"mse": L.DOS_LOSS_MSE, "mse_scaled": L.DOS_LOSS_MSE_SCALED}[loss]
        cfg.detector_bin = int(detector_bin)
        cfg.path = {"auto": L.DOS_PATH_AUTO, "multipass": L.DOS_PATH_MULTIPASS,
                    "multipass_bulk": L.DOS_PATH_MULTIPASS_BULK,
                    "fused": L.DOS_PATH_FUSED, "dft_gemm": L.DOS_PATH_DFT_GEMM,
                    "dft_gemm_x3": L.DOS_PATH_DFT_GEMM_X3}[path]
        self._ctx = None
        with torch.cuda.device(self.device):
            self._ctx = L.dos_create(cfg, torch.cuda.current_stream(self.device).cuda_stream)

    @classmethod
    def from_workload(cls, w, **kw) -> "DiffractiveStack":
        return cls(n=w.n, m=w.m, n_layers=w.n_layers, lambdas=w.lambdas, gaps=w.gaps,
                   pitch=w.pitch, n_index=w.n_index, kappa=w.kappa, fov=w.fov,
                   aperture=w.aperture, n_medium=w.n_medium, h_base=w.h_base, **kw)

    # ------------------------------------------------------------------ plumbing
    def _bind(self) -> None:
        L.dos_set_stream(self._ctx, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self) -> None:
        if self._ctx:
            L.dos_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._ctx

    @property
    def workspace_bytes(self) -> int:
        return L.dos_workspace_bytes(self._ctx)

    @property
    def last_launch_count(self) -> int:
        return L.dos_last_launch_count(self._ctx)

    @property
    def path(self) -> str:
        return {1: "multipass", 2: "fused", 3: "dft_gemm", 4: "multipass_bulk",
                5: "dft_gemm_x3"}[L.dos_path(self._ctx)]

    # ------------------------------------------------------------------ compute
    def forward(self, h: torch.Tensor, save_for_backward: bool = True,
                out: Optional[torch.Tensor] = None, want_intensity: bool = True):
        h = h.contiguous()
        _need(h, torch.float32, (self.n_layers, self.n, self.n), "h", self.device)
        I = None
        if want_intensity:
            I = out if out is not None else torch.empty(
                (self.n_lambda, self.fov, self.fov), dtype=torch.float32, device=self.device)
            _need(I, torch.float32, (self.n_lambda, self.fov, self.fov), "out", self.device)
        self._bind()
        L.dos_forward(self._ctx, h.data_ptr(), I.data_ptr() if I is not None else 0, save_for_backward)
        return I

    def loss(self, T: torch.Tensor, read: bool = True, psnr: bool = True, grad: bool = True):
        """Returns (loss or None, psnr[N_w] or None, dL/dI or None).  T holds the
        targets of the detector pixels, [N_w][F/b][F/b]; dL/dI is [N_w][F][F]."""
        T = T.contiguous()
        _need(T, torch.float32, (self.n_lambda, self.det, self.det), "T", self.device)
        p = torch.empty(self.n_lambda, dtype=torch.float32, device=self.device) if psnr else None
        g = torch.empty((self.n_lambda, self.fov, self.fov), dtype=torch.float32,
                        device=self.device) if grad else None
        self._bind()
        val = L.dos_loss(self._ctx, T.data_ptr(), read, p.data_ptr() if p is not None else 0,
                         g.data_ptr() if g is not None else 0)
        return val, p, g

    def read_loss(self) -> float:
        self._bind()
        return L.dos_read_loss(self._ctx)

    def backward(self, dLdI: torch.Tensor, out: Optional[torch.Tensor] = None):
        """dL/dh of the last forward that saved its fields (the context kept
        that forward's thickness)."""
        dLdI = dLdI.contiguous()
        _need(dLdI, torch.float32, (self.n_lambda, self.fov, self.fov), "dLdI", self.device)
        g = out if out is not None else torch.empty((self.n_layers, self.n, self.n), dtype=torch.float32,
                                                    device=self.device)
        _need(g, torch.float32, (self.n_layers, self.n, self.n), "out", self.device)
        self._bind()
        L.dos_backward(self._ctx, dLdI.data_ptr(), g.data_ptr())
        return g

    def step(self, h: torch.Tensor, T: torch.Tensor, grad_out: Optional[torch.Tensor] = None,
             intensity_out: Optional[torch.Tensor] = None, psnr_out: Optional[torch.Tensor] = None,
             read: bool = False):
        """Forward + loss + backward in one call, replayed as a CUDA graph.
        Returns (loss or None, dL/dh).  Reusing the same tensors reuses the graph."""
        _need(h, torch.float32, (self.n_layers, self.n, self.n), "h", self.device)
        _need(T, torch.float32, (self.n_lambda, self.det, self.det), "T", self.device)
        g = grad_out if grad_out is not None else torch.empty_like(h)
        _need(g, torch.float32, (self.n_layers, self.n, self.n), "grad_out", self.device)
        if intensity_out is not None:
            _need(intensity_out, torch.float32, (self.n_lambda, self.fov, self.fov), "intensity_out", self.device)
        if psnr_out is not None:
            _need(psnr_out, torch.float32, (self.n_lambda,), "psnr_out", self.device)
        self._bind()
        val = L.dos_step(self._ctx, h.data_ptr(), T.data_ptr(), g.data_ptr(),
                         intensity_out.data_ptr() if intensity_out is not None else 0,
                         psnr_out.data_ptr() if psnr_out is not None else 0, read)
        return val, g

    def set_misalignment(self, displacements=None) -> None:
        """Displace layers 1..K by (dx, dy, dz) [m] (a (K, 3) array), or None."""
        if displacements is not None:
            displacements = np.asarray(displacements, dtype=np.float64)
            if displacements.shape != (self.n_layers, 3):
                raise ValueError("displacements must have shape (n_layers, 3)")
        L.dos_set_misalignment(self._ctx, displacements)

    def efficiency(self) -> torch.Tensor:
        """Output diffraction efficiency of every channel of the last forward."""
        eta = torch.empty(self.n_lambda, dtype=torch.float32, device=self.device)
        self._bind()
        L.dos_efficiency(self._ctx, eta.data_ptr())
        return eta

    def output_field(self) -> torch.Tensor:
        o = torch.empty((self.n_lambda, self.fov, self.fov), dtype=torch.complex64, device=self.device)
        self._bind()
        L.dos_output_field(self._ctx, o.data_ptr())
        return o

    def layer_field(self, layer: int) -> torch.Tensor:
        v = torch.empty((self.n_lambda, self.n, self.n), dtype=torch.complex64, device=self.device)
        self._bind()
        L.dos_layer_field(self._ctx, layer, v.data_ptr())
        return v

    def propagate(self, field: torch.Tensor, gap: int, adjoint: bool = False) -> torch.Tensor:
        field = field.contiguous()
        _need(field, torch.complex64, (self.n_lambda, self.n, self.n), "field", self.device)
        out = torch.empty_like(field)
        self._bind()
        L.dos_propagate(self._ctx, gap, field.data_ptr(), out.data_ptr(), adjoint)
        return out


class DosFunction(torch.autograd.Function):
    """I = DosFunction.apply(h, stack): intensities of every channel; the
    backward is the hand-written adjoint of the cascade (dos_backward)."""

    @staticmethod
    def forward(ctx, h: torch.Tensor, stack: DiffractiveStack):
        h = h.contiguous()
        I = stack.forward(h, save_for_backward=True)
        ctx.stack = stack
        return I

    @staticmethod
    def backward(ctx, gI: torch.Tensor):
        g = ctx.stack.backward(gI.contiguous().to(torch.float32))
        return g, None


def quantize_thickness(h: torch.Tensor, h_max: float, bits: int) -> torch.Tensor:
    """Thickness limited to [0, h_max] and rounded to 2^bits levels (phase bit depth)."""
    if not h.is_cuda or h.dtype != torch.float32:
        raise TypeError("h must be a float32 CUDA tensor")
    h = h.contiguous()
    out = torch.empty_like(h)
    L.dos_quantize_thickness(h.data_ptr(), out.data_ptr(), h.numel(), float(h_max), int(bits),
                             torch.cuda.current_stream(h.device).cuda_stream)
    return out


def detuning_psnr(design: dict, h: torch.Tensor, T: torch.Tensor, offsets, path: str = "auto",
                  device=None) -> torch.Tensor:
    """PSNR of every channel when it is probed at lambda_w + delta for each
    delta in ``offsets`` [m] (Section 3: robustness to probe-wavelength drift).

    ``design`` holds the DiffractiveStack keyword arguments of the trained
    design; the probe design evaluates all N_w x len(offsets) wavelengths in one
    context (material index and loss of the nominal channel).  Returns a
    [N_w, len(offsets)] tensor."""
    offsets = np.asarray(offsets, dtype=np.float64)
    lam = np.asarray(design["lambdas"], dtype=np.float64)
    nw, npr = lam.shape[0], offsets.shape[0]
    probe = dict(design)
    probe["lambdas"] = (lam[:, None] + offsets[None, :]).ravel()
    for key in ("n_index", "kappa"):
        if probe.get(key) is not None:
            probe[key] = np.repeat(np.broadcast_to(np.asarray(probe[key], np.float64), (nw,)), npr)
    st = DiffractiveStack(path=path, device=device or h.device, **probe)
    try:
        st.forward(h, save_for_backward=False, want_intensity=False)
        Tp = T.repeat_interleave(npr, dim=0).contiguous()
        _, psnr, _ = st.loss(Tp, read=False, psnr=True, grad=False)
        return psnr.view(nw, npr).clone()
    finally:
        st.close()
