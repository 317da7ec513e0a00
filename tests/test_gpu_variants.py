"""GPU parity of the evaluation variants (NEXT-2): phase bit depth,
diffraction efficiency and probe-wavelength detuning, against the oracle."""
import os

import numpy as np
import pytest
import torch

from oracle import dos_oracle as O
from paper_2604_02624_gb300 import _lib as L
from paper_2604_02624_gb300 import workloads as W
from paper_2604_02624_gb300.api import DiffractiveStack, detuning_psnr, quantize_thickness

from gpu_cases import TOL_INTENSITY, oracle_model, rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not os.path.exists(L.LIB_PATH):
        from paper_2604_02624_gb300 import build
        build.build()
    L.load()
    torch.cuda.set_device(DEV)


@pytest.mark.parametrize("bits", [1, 4, 6, 8, 16])
def test_quantisation_is_bit_exact(bits):
    rng = np.random.default_rng(bits)
    hmax = 664.5e-9
    h = rng.uniform(-0.2 * hmax, 1.2 * hmax, 100003).astype(np.float32)
    q = quantize_thickness(torch.tensor(h, device=DEV), hmax, bits).cpu().numpy()
    assert np.array_equal(q, O.quantize_thickness(h, hmax, bits))


def test_quantised_design_forward_matches_oracle():
    w = W.workload("small")
    h = W.thickness(w, 0)
    hq = quantize_thickness(torch.tensor(h, dtype=torch.float32, device=DEV), 664.5e-9, 4)
    st = DiffractiveStack.from_workload(w, device=DEV)
    I = st.forward(hq)
    ref = O.forward(hq.cpu().numpy().astype(np.float64), **oracle_model(w))
    assert rel_l2(I.cpu().numpy().astype(np.float64), ref["I"]) <= TOL_INTENSITY
    st.close()


@pytest.mark.parametrize("path", ["multipass", "fused"])
def test_efficiency_matches_oracle(path):
    w = W.workload("small")
    h = W.thickness(w, 0)
    st = DiffractiveStack.from_workload(w, device=DEV, path=path)
    st.forward(torch.tensor(h, dtype=torch.float32, device=DEV))
    eta = st.efficiency().cpu().numpy().astype(np.float64)
    ref = O.diffraction_efficiency(O.forward(h, keep_fields=False, **oracle_model(w))["I"], w.aperture)
    assert rel_l2(eta, ref) <= TOL_INTENSITY
    st.close()


def test_detuning_psnr():
    w = W.workload("tiny")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    design = dict(n=w.n, m=w.m, n_layers=w.n_layers, lambdas=w.lambdas, gaps=w.gaps, pitch=w.pitch,
                  n_index=w.n_index, kappa=w.kappa, fov=w.fov, aperture=w.aperture)
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    offsets = np.array([-2e-9, 0.0, 2e-9])
    p = detuning_psnr(design, hd, Td, offsets, path="multipass").cpu().numpy()
    st = DiffractiveStack(path="multipass", device=DEV, **design)
    st.forward(hd)
    _, nominal, _ = st.loss(Td)
    assert np.array_equal(p[:, 1], nominal.cpu().numpy())
    ws = w.subset(np.arange(w.n_lambda))
    ws.lambdas = w.lambdas + offsets[2]
    ref = O.mse_loss(O.forward(h, keep_fields=False, **oracle_model(ws))["I"], T)[1]
    assert np.max(np.abs(p[:, 2] - ref)) <= 1e-3
    st.close()


def test_fine_tune_after_channel_swap_lowers_the_loss():
    """The fine-tuning driver (Adam on h through the graph-captured step) lowers
    the swapped design's loss."""
    from paper_2604_02624_gb300.design import channel_swap, fine_tune
    w = W.workload("small")
    h = torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=DEV)
    T = torch.tensor(W.targets(w, 1), dtype=torch.float32, device=DEV)
    st = DiffractiveStack.from_workload(w, device=DEV, loss="mse_scaled")
    st.forward(h)
    _, psnr, _ = st.loss(T)
    perm = channel_swap(psnr.cpu().numpy(), w.lambdas)
    Ts = T[torch.tensor(perm, device=DEV)].contiguous()
    _, losses = fine_tune(st, h, Ts, steps=30, lr=1e-2, h_max=664.5e-9)
    assert losses[-1] < 0.9 * losses[0], losses
    st.close()


# ------------------------------------------------------------ misaligned layers (NEXT-4)
DISP = np.array([[31e-9, -17e-9, 90e-9], [-12e-9, 44e-9, -150e-9]])


@pytest.mark.parametrize("path", ["multipass", "multipass_bulk", "fused", "dft_gemm"])
def test_misaligned_layers_match_oracle(path):
    from gpu_cases import TOL_FIELD, TOL_GRAD_ORACLE, split_bound, TOL_GRAD_FD
    w = W.workload("small")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = DiffractiveStack.from_workload(w, device=DEV, path=path)
    st.set_misalignment(DISP)
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    I = st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(torch.tensor(T, dtype=torch.float32, device=DEV))
    g = st.backward(hd, dl).cpu().numpy().astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, displacements=DISP, **oracle_model(w))
    e_o = rel_l2(o.cpu().numpy().astype(np.complex128), fwd["o"])
    if path == "dft_gemm":
        assert e_o <= split_bound(4 * (w.n_layers + 1))
        assert rel_l2(g, g_ref) <= TOL_GRAD_FD
    else:
        assert e_o <= TOL_FIELD
        assert rel_l2(g, g_ref) <= TOL_GRAD_ORACLE
    # back to the aligned design
    st.set_misalignment(None)
    I0 = st.forward(hd).cpu().numpy().astype(np.float64)
    ref0 = O.forward(h, keep_fields=False, **oracle_model(w))["I"]
    assert rel_l2(I0, ref0) <= (split_bound(12, True) if path == "dft_gemm" else TOL_INTENSITY)
    st.close()


def test_graph_step_follows_misalignment_changes():
    w = W.workload("small")
    h = torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=DEV)
    T = torch.tensor(W.targets(w, 1), dtype=torch.float32, device=DEV)
    st = DiffractiveStack.from_workload(w, device=DEV, path="fused")
    g = torch.empty_like(h)
    rng = np.random.default_rng(5)
    for _ in range(3):
        disp = rng.uniform(-40e-9, 40e-9, (w.n_layers, 3))
        st.set_misalignment(disp)
        val, _ = st.step(h, T, grad_out=g, read=True)
        st.forward(h)
        L_ref, _, dl = st.loss(T)
        assert val == L_ref
        assert torch.equal(g, st.backward(h, dl))
    st.close()


# ------------------------------------------------------------ detector pixels (Section 4)
@pytest.mark.parametrize("path", ["multipass", "fused"])
@pytest.mark.parametrize("b,loss", [(2, "mse"), (5, "mse_scaled")])
def test_detector_pixels_loss_psnr_and_gradient(path, b, loss):
    """Detector pixels of b x b simulation pixels (b = 2: the 25 x 25 output
    pixels of a 50-pixel FOV): loss, PSNR, dL/dI and the thickness gradient
    against the FP64 oracle; the graph step gives the same values."""
    from gpu_cases import TOL_GRAD_ORACLE, TOL_LOSS
    w = W.workload("small")
    h = W.thickness(w, 0)
    fd = w.fov // b
    rng = np.random.default_rng(40 + b)
    T = (rng.uniform(0, 1, (w.n_lambda, fd, fd)) * 1e-4 * b * b).astype(np.float32)
    st = DiffractiveStack.from_workload(w, device=DEV, path=path, loss=loss, detector_bin=b)
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, device=DEV)
    st.forward(hd)
    val, psnr, dl = st.loss(Td)
    g = st.backward(hd, dl).clone()
    scaled = loss == "mse_scaled"
    L_ref, psnr_ref, g_ref, fwd = O.loss_and_grad(h, T, scaled=scaled, detector_bin=b, **oracle_model(w))
    _, _, dl_ref = O.mse_loss(fwd["I"], T, scaled, b)
    assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref)
    assert np.max(np.abs(psnr.cpu().numpy() - psnr_ref)) <= 1e-3
    assert rel_l2(dl.cpu().numpy().astype(np.float64), dl_ref) <= TOL_INTENSITY
    assert rel_l2(g.cpu().numpy().astype(np.float64), g_ref) <= TOL_GRAD_ORACLE
    gs = torch.empty_like(g)
    val2, _ = st.step(hd, Td, grad_out=gs, read=True)
    assert val2 == val and torch.equal(gs, g)
    with pytest.raises(ValueError):
        st.loss(torch.zeros((w.n_lambda, w.fov, w.fov), device=DEV))
    st.close()
