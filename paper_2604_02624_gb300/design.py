"""Design-level drivers built on the engine: dynamic channel swapping and the
fine-tuning loop that follows it (Section 2, Fig. 2B).

The optimiser is the user's choice (the paper uses Adam, learning rate 1e-3);
every forward, objective and gradient evaluation runs in libdos through
``DiffractiveStack.step`` (one CUDA graph per step).
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np
import torch


def channel_swap(psnr, lambdas) -> np.ndarray:
    """Reassign images to wavelengths by reconstruction quality.

    The images are ranked by PSNR in descending order and handed out to the
    wavelengths starting from the longest one (Section 2): the best-projected
    image goes to the longest wavelength, the hardest image to the shortest.
    Returns ``perm`` with ``new_targets[c] = targets[perm[c]]``; ties keep the
    original order.
    """
    psnr = np.asarray(psnr, dtype=np.float64)
    lam = np.asarray(lambdas, dtype=np.float64)
    if psnr.shape != lam.shape:
        raise ValueError("psnr and lambdas must have one entry per channel")
    images = np.argsort(-psnr, kind="stable")     # best first
    channels = np.argsort(-lam, kind="stable")    # longest wavelength first
    perm = np.empty(psnr.shape[0], dtype=np.int64)
    perm[channels] = images
    return perm


def fine_tune(stack, h: torch.Tensor, T: torch.Tensor, steps: int, lr: float = 1e-3,
              h_scale: float = 1e-6, h_max: Optional[float] = None,
              callback: Optional[Callable[[int, float], None]] = None):
    """Adam on the thickness (in units of ``h_scale`` metres, so that the
    paper's learning rate applies to an O(1) parameter), with the learnable
    thickness kept in [0, h_max] after every step (Eq. 2).  Returns the final
    thickness and the loss of every step."""
    p = (h.detach().clone() / h_scale).requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr)
    grad = torch.empty_like(h)
    hcur = torch.empty_like(h)
    losses = []
    for it in range(steps):
        with torch.no_grad():
            hcur.copy_(p * h_scale)
        loss, _ = stack.step(hcur, T, grad_out=grad, read=True)
        losses.append(loss)
        if callback:
            callback(it, loss)
        opt.zero_grad(set_to_none=False)
        p.grad = grad * h_scale
        opt.step()
        if h_max is not None:
            with torch.no_grad():
                p.clamp_(0.0, h_max / h_scale)
    with torch.no_grad():
        hcur.copy_(p * h_scale)
    return hcur, losses
