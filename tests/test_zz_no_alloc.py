"""dos_loss_noalloc: scoring for callers that cannot allocate device memory.

Such callers (a framework that owns all device memory through its own pool,
a fixed start-up budget, a path where cudaMalloc would stall the device)
cannot create a context, whose workspace dos_create allocates.  The entry
point computes what dos_loss computes from caller intensities, with its
scratch in a fixed-size array inside the library.  This file is collected
last so that a stop at its first failure has already run every other test.
"""
import os

import numpy as np
import pytest
import torch

from paper_2604_02624_gb300 import _lib as L
from paper_2604_02624_gb300 import workloads as W
from paper_2604_02624_gb300.api import DiffractiveStack

from gpu_cases import TOL_INTENSITY, TOL_LOSS, assert_close

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not os.path.exists(L.LIB_PATH):
        from paper_2604_02624_gb300 import build
        build.build()
    L.load()
    torch.cuda.set_device(DEV)


@pytest.mark.parametrize("loss,mode", [("mse", L.DOS_LOSS_MSE), ("mse_scaled", L.DOS_LOSS_MSE_SCALED)])
def test_noalloc_scoring_matches_dos_loss_on_two_calls_in_a_row(loss, mode):
    w = W.workload("small")
    h = torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=DEV)
    T = torch.tensor(W.targets(w, 1), dtype=torch.float32, device=DEV)
    st = DiffractiveStack.from_workload(w, device=DEV, loss=loss)
    I = st.forward(h)
    L_ref, psnr_ref, g_ref = st.loss(T)
    psnr_ref = psnr_ref.cpu().numpy()
    g_ref = g_ref.cpu().numpy().astype(np.float64)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for call in range(2):
        psnr = torch.full((w.n_lambda,), float("nan"), device=DEV)
        g = torch.full_like(T, float("nan"))
        val = L.dos_loss_noalloc(I.data_ptr(), T.data_ptr(), w.n_lambda, w.fov, 0, mode, True,
                                 psnr.data_ptr(), g.data_ptr(), stream)
        torch.cuda.synchronize()
        assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref), (call, val, L_ref)
        assert np.max(np.abs(psnr.cpu().numpy() - psnr_ref)) <= 1e-3, call
        assert_close(g.cpu().numpy().astype(np.float64), g_ref, TOL_INTENSITY, call)
    st.close()


def test_noalloc_sharded_normalisation_and_no_loss_readback():
    """A shard of a larger design (n_lambda_total = 2 n_lambda) scores like
    dos_loss of a context created with the same n_lambda_total; with h_loss
    NULL the loss is not read back but PSNR and dL/dI are still written.
    Around the calls neither torch's allocator nor the device's free memory
    changes: the entry point allocates nothing."""
    w = W.workload("small")
    h = torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=DEV)
    T = torch.tensor(W.targets(w, 1), dtype=torch.float32, device=DEV)
    total = 2 * w.n_lambda
    st = DiffractiveStack.from_workload(w, device=DEV, n_lambda_total=total)
    I = st.forward(h)
    L_ref, psnr_ref, g_ref = st.loss(T)
    psnr_ref = psnr_ref.cpu().numpy()
    g_ref = g_ref.cpu().numpy().astype(np.float64)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    psnr = torch.full((w.n_lambda,), float("nan"), device=DEV)
    g = torch.full_like(T, float("nan"))
    val = L.dos_loss_noalloc(I.data_ptr(), T.data_ptr(), w.n_lambda, w.fov, total, L.DOS_LOSS_MSE, True,
                             psnr.data_ptr(), g.data_ptr(), stream)
    torch.cuda.synchronize()
    assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref), (val, L_ref)
    assert_close(g.cpu().numpy().astype(np.float64), g_ref, TOL_INTENSITY)
    psnr.fill_(float("nan"))
    g.fill_(float("nan"))
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated(DEV)
    free0, _ = torch.cuda.mem_get_info(DEV)
    assert L.dos_loss_noalloc(I.data_ptr(), T.data_ptr(), w.n_lambda, w.fov, total, L.DOS_LOSS_MSE, False,
                              psnr.data_ptr(), g.data_ptr(), stream) is None
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(DEV) == alloc0
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0
    assert np.max(np.abs(psnr.cpu().numpy() - psnr_ref)) <= 1e-3
    assert_close(g.cpu().numpy().astype(np.float64), g_ref, TOL_INTENSITY)
    st.close()


def test_noalloc_rejects_more_channels_than_its_scratch_holds():
    dummy = torch.zeros(4, device=DEV)
    with pytest.raises(L.DosError) as e:
        L.dos_loss_noalloc(dummy.data_ptr(), dummy.data_ptr(), L.DOS_NOALLOC_MAX_LAMBDA + 1, 1, 0,
                           L.DOS_LOSS_MSE, True, 0, 0, 0)
    assert e.value.code == L.DOS_ERR_ARG
    assert "fixed size" in str(e.value)
