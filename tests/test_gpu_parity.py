"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Same seeded inputs on both sides; element-by-element comparisons at sizes the
oracle finishes in seconds (several tiles, ragged tails), and sampled
channels / subset designs at the full workload sizes.
"""
import numpy as np
import pytest
import torch

from oracle import dos_oracle as O
from paper_2604_02624_gb300 import workloads as W
from paper_2604_02624_gb300 import _lib as L
from paper_2604_02624_gb300.api import DiffractiveStack, DosFunction

from gpu_cases import (SPLIT_TARGET, TOL_FIELD, TOL_GRAD_FD, TOL_GRAD_ORACLE, TOL_INTENSITY, TOL_LOSS,
                       assert_close, custom, oracle_model, replace)

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import os
    if not os.path.exists(L.LIB_PATH):
        from paper_2604_02624_gb300 import build
        build.build()
    L.load()
    torch.cuda.set_device(DEV)


PATHS = ["multipass", "multipass_bulk", "fused"]
MULTIPASS = ["multipass", "multipass_bulk"]


def _stack(w, **kw):
    return DiffractiveStack.from_workload(w, device=DEV, **kw)


def _t(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def _np(x):
    return x.detach().cpu().numpy()


def _rand_fields(rng, nw, n):
    return rng.standard_normal((nw, n, n)) + 1j * rng.standard_normal((nw, n, n))


# ------------------------------------------------------------ single propagation
@pytest.mark.parametrize("n,m,adj,evan", [
    (64, 128, False, "decay"), (64, 128, True, "decay"), (200, 400, False, "decay"),
    (200, 400, True, "zero"), (256, 512, False, "decay"), (256, 512, True, "decay"),
    (50, 128, True, "decay"), (100, 200, False, "zero"), (1, 16, False, "decay"),
    (64, 64, False, "decay"), (7, 16, True, "decay"), (30, 32, False, "decay"),
])
def test_propagate_matches_oracle(n, m, adj, evan):
    w = custom(n, m, 1, [500, 587, 740], 40, n, name="prop")
    rng = np.random.default_rng(n * 1000 + m)
    f = _rand_fields(rng, w.n_lambda, n).astype(np.complex64)
    st = _stack(w, evanescent=evan)
    got = _np(st.propagate(torch.tensor(f, device=DEV), 0, adj)).astype(np.complex128)
    ref = np.stack([(O.propagate_adjoint if adj else O.propagate)(
        f[i].astype(np.complex128), O.transfer_function(w.lambdas[i], w.gaps[0], m, w.pitch, 1.0, evan))
        for i in range(w.n_lambda)])
    assert_close(got, ref, TOL_FIELD)
    st.close()


# ------------------------------------------------------------ forward model
def _forward_case(w, evan="decay", loss="mse", path="multipass"):
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, evanescent=evan, loss=loss, path=path)
    hd = _t(h)
    I = st.forward(hd)
    o = st.output_field()
    ref = O.forward(h, **{k: v for k, v in oracle_model(w, evan).items()})
    return st, h, T, hd, I, o, ref


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name", ["tiny", "small"])
def test_forward_fields_and_intensity(name, path):
    w = W.workload(name)
    st, h, T, hd, I, o, ref = _forward_case(w, path=path)
    assert st.path == path
    assert_close(_np(o).astype(np.complex128), ref["o"], TOL_FIELD)
    assert_close(_np(I).astype(np.float64), ref["I"], TOL_INTENSITY)
    for l in range(1, w.n_layers + 1):
        v = _np(st.layer_field(l)).astype(np.complex128)
        assert_close(v, ref["v"][:, l - 1], TOL_FIELD, l)
    # multi-pass: K row + K column passes and the output pass (gap 0 is the create-time input field)
    assert st.last_launch_count == (2 * w.n_layers + 1 if path in MULTIPASS else 1)
    st.close()


@pytest.mark.parametrize("path", MULTIPASS)
def test_forward_ragged_and_options(path):
    """N = 100 in M = 200 (ragged row blocks and column tiles), three layers with
    unequal gaps, a medium of index 1.33, base thickness, per-channel
    dispersion and loss, zeroed evanescent bins, full-window aperture."""
    lam = [455, 530, 610, 700, 745]
    w = custom(100, 200, 3, lam, [30, 55, 30, 80], 40, aperture=100,
               n_index=[1.52, 1.51, 1.50, 1.495, 1.49], kappa=[0.02, 0.0, 0.01, 0.03, 0.0],
               n_medium=1.33, h_base=120e-9, name="ragged")
    st, h, T, hd, I, o, ref = _forward_case(w, evan="zero", path=path)
    assert_close(_np(o).astype(np.complex128), ref["o"], TOL_FIELD)
    assert_close(_np(I).astype(np.float64), ref["I"], TOL_INTENSITY)
    st.close()


@pytest.mark.parametrize("path", MULTIPASS)
def test_forward_single_pixel_layer(path):
    w = custom(1, 16, 2, [500, 700], 3, 1, name="one-pixel")
    st, h, T, hd, I, o, ref = _forward_case(w, path=path)
    assert_close(_np(o).astype(np.complex128), ref["o"], TOL_FIELD)
    st.close()


# ------------------------------------------------------------ objective
@pytest.mark.parametrize("loss", ["mse", "mse_scaled"])
def test_loss_psnr_and_dldi(loss):
    w = W.workload("small")
    st, h, T, hd, I, o, ref = _forward_case(w, loss=loss, path="fused")
    val, psnr, dLdI = st.loss(_t(T))
    L_ref, psnr_ref, dLdI_ref = O.mse_loss(ref["I"], T, scaled=(loss == "mse_scaled"))
    assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref)
    assert np.max(np.abs(_np(psnr) - psnr_ref)) <= 1e-3
    assert_close(_np(dLdI).astype(np.float64), dLdI_ref, TOL_INTENSITY)
    st.close()


# ------------------------------------------------------------ gradient
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name,loss", [("tiny", "mse"), ("small", "mse"), ("small", "mse_scaled")])
def test_gradient_matches_oracle_and_finite_differences(name, loss, path):
    w = W.workload(name)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, loss=loss, path=path)
    hd = _t(h)
    st.forward(hd)
    _, _, dLdI = st.loss(_t(T))
    g = _np(st.backward(dLdI)).astype(np.float64)
    model = oracle_model(w)
    L_ref, _, g_ref, _ = O.loss_and_grad(h, T, scaled=(loss == "mse_scaled"), **model)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    c = w.n // 2
    pixels = [(0, c, c), (w.n_layers - 1, c - 7, c + 11), (0, c + 5, c - 9)]
    fd = O.finite_difference(h, T, pixels, 1e-4 * w.lambda_mean, scaled=(loss == "mse_scaled"), **model)
    got = np.array([g[p] for p in pixels])
    assert np.max(np.abs(got - fd) / np.abs(fd)) <= TOL_GRAD_FD, (got, fd)
    st.close()


@pytest.mark.parametrize("path", PATHS)
def test_autograd_function_composes_with_torch_loss(path):
    """A torch objective of the intensities back-propagates through DosFunction
    (dos_backward) to the FP64 oracle gradient of the same objective."""
    w = W.workload("tiny")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, path=path)
    hd = _t(h).requires_grad_(True)
    I = DosFunction.apply(hd, st)
    Td = _t(T)
    loss = ((I - Td) ** 2).mean()
    loss.backward()
    L_ref, _, g_ref, _ = O.loss_and_grad(h, T, **oracle_model(w))
    assert abs(loss.item() - L_ref) <= TOL_LOSS * L_ref
    assert_close(_np(hd.grad).astype(np.float64), g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("path", PATHS)
def test_backward_is_bitwise_deterministic(path):
    w = W.workload("small")
    h = _t(W.thickness(w, 0))
    st = _stack(w, path=path)
    st.forward(h)
    _, _, g = st.loss(_t(W.targets(w, 1)))
    a = st.backward(g).clone()
    b = st.backward(g).clone()
    assert torch.equal(a, b)
    st.close()


@pytest.mark.parametrize("path", PATHS)
def test_backward_uses_the_thickness_of_the_saved_forward(path):
    """dos_backward takes no thickness: the context keeps the one of the
    forward that saved its fields, so changing the caller's buffer between
    the two calls does not change the gradient."""
    w = W.workload("tiny")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, path=path)
    hd = _t(h)
    st.forward(hd)
    _, _, dl = st.loss(_t(T))
    hd.mul_(0.5)  # the caller's buffer changes after the forward
    g = _np(st.backward(dl)).astype(np.float64)
    _, _, g_ref, _ = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


def test_state_errors():
    w = W.workload("tiny")
    st = _stack(w)
    h = _t(W.thickness(w, 0))
    with pytest.raises(L.DosError) as e:
        st.backward(torch.zeros((w.n_lambda, w.fov, w.fov), device=DEV))
    assert e.value.code == L.DOS_ERR_STATE
    with pytest.raises(L.DosError) as e:
        st.loss(_t(W.targets(w, 1)))
    assert e.value.code == L.DOS_ERR_STATE
    st.forward(h, save_for_backward=False)
    with pytest.raises(L.DosError) as e:
        st.backward(torch.zeros((w.n_lambda, w.fov, w.fov), device=DEV))
    assert e.value.code == L.DOS_ERR_STATE
    st.close()


# ------------------------------------------------------------ full workload sizes
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name,count", [("massive", 5), ("precision", 3), ("batched", 4)])
def test_full_size_forward_on_sampled_channels(name, count, path):
    """All channels on the GPU in the bench's launch configuration; the oracle
    checks evenly spread channels (every channel is independent)."""
    w = W.workload(name)
    h = W.thickness(w, 0)
    st = _stack(w, path=path)
    I = st.forward(_t(h), save_for_backward=False)
    o = st.output_field()
    idx = W.subset_indices(w.n_lambda, count)
    ws = w.subset(idx)
    ref = O.forward(h, keep_fields=False, **oracle_model(ws))
    assert_close(_np(o[idx]).astype(np.complex128), ref["o"], TOL_FIELD)
    assert_close(_np(I[idx]).astype(np.float64), ref["I"], TOL_INTENSITY)
    st.close()


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name", ["massive", "precision"])
def test_full_geometry_gradient_on_channel_subset(name, path):
    """Gradient of the full geometry on a 16-channel subset design (the same
    layers, gaps and grid), against the FP64 oracle."""
    w = W.workload(name)
    ws = w.subset(W.subset_indices(w.n_lambda, 16))
    h = W.thickness(w, 0)
    T = W.targets(w, 1)[W.subset_indices(w.n_lambda, 16)]
    st = _stack(ws, path=path)
    hd = _t(h)
    st.forward(hd)
    _, _, dLdI = st.loss(_t(T))
    g = _np(st.backward(dLdI)).astype(np.float64)
    _, _, g_ref, _ = O.loss_and_grad(h, T, **oracle_model(ws))
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("path", PATHS)
def test_full_size_gradient_is_the_sum_of_channel_shards(path):
    """At 4096 channels the gradient equals the sum of the gradients of two
    channel shards that share the loss normalisation (the property that makes
    wavelength sharding across GPUs exact)."""
    w = W.workload("massive")
    h = _t(W.thickness(w, 0))
    T = W.targets(w, 1)
    st = _stack(w, path=path)
    st.forward(h)
    L_full, _, dLdI = st.loss(_t(T))
    g_full = st.backward(dLdI).clone()
    st.close()
    half = w.n_lambda // 2
    g_sum = torch.zeros_like(g_full)
    L_sum = 0.0
    for lo, hi in ((0, half), (half, w.n_lambda)):
        ws = w.subset(np.arange(lo, hi))
        s = _stack(ws, n_lambda_total=w.n_lambda, path=path)
        s.forward(h)
        Ls, _, dl = s.loss(_t(T[lo:hi]))
        g_sum += s.backward(dl)
        L_sum += Ls
        s.close()
    assert abs(L_sum - L_full) <= 1e-9 * abs(L_full)
    assert_close(_np(g_sum).astype(np.float64), _np(g_full).astype(np.float64), 1e-5)


def test_paths_agree_at_full_size():
    """The cluster-resident and the multi-pass implementations of the massive
    step give the same intensities and gradient (both FP32, different orders);
    the bulk-prefetch multi-pass passes do the plain passes' arithmetic in the
    same order."""
    w = W.workload("massive")
    h = _t(W.thickness(w, 0))
    T = _t(W.targets(w, 1))
    out = {}
    for path in PATHS:
        st = _stack(w, path=path)
        I = st.forward(h).clone()
        _, _, g = st.loss(T)
        out[path] = (I, st.backward(g).clone())
        st.close()
    ref = [_np(x).astype(np.float64) for x in out["multipass"]]
    assert_close(_np(out["fused"][0]).astype(np.float64), ref[0], 1e-5)
    assert_close(_np(out["fused"][1]).astype(np.float64), ref[1], 1e-4)
    assert_close(_np(out["multipass_bulk"][0]).astype(np.float64), ref[0], 1e-6)
    assert_close(_np(out["multipass_bulk"][1]).astype(np.float64), ref[1], 1e-6)


def test_auto_path_is_tuned_and_described():
    w = W.workload("batched")
    st = _stack(w, path="auto")
    d = L.dos_describe(st.handle)
    assert d.startswith("path=") and "tuned" in d, d
    assert st.path in PATHS
    st.close()


def test_fused_path_refuses_layers_wider_than_half_the_grid():
    w = custom(64, 64, 1, [500, 600], 10, 64, name="no-pad")
    with pytest.raises(L.DosError) as e:
        _stack(w, path="fused")
    assert e.value.code == L.DOS_ERR_UNSUPPORTED


@pytest.mark.parametrize("path", PATHS)
def test_graph_step_matches_separate_calls(path):
    """dos_step (captured once as a CUDA graph, then replayed) gives the same
    loss, intensities, PSNR and gradient as forward + loss + backward."""
    w = W.workload("small")
    h = _t(W.thickness(w, 0))
    T = _t(W.targets(w, 1))
    st = _stack(w, path=path)
    I_ref = st.forward(h).clone()
    L_ref, p_ref, dl = st.loss(T)
    g_ref = st.backward(dl).clone()
    I = torch.empty_like(I_ref)
    p = torch.empty_like(p_ref)
    g = torch.empty_like(g_ref)
    for _ in range(3):  # capture, then two replays
        val, _ = st.step(h, T, grad_out=g, intensity_out=I, psnr_out=p, read=True)
        torch.cuda.synchronize()
        assert val == L_ref
        assert torch.equal(I, I_ref) and torch.equal(p, p_ref) and torch.equal(g, g_ref)
    h2 = h * 0.5
    val2, g2 = st.step(h2, T, grad_out=g, read=True)   # new pointers: re-capture
    st.forward(h2)
    L2, _, dl2 = st.loss(T)
    assert val2 == L2
    assert torch.equal(g2, st.backward(dl2))
    st.close()


# ------------------------------------------------------------ split-BF16 DFT-GEMM form
@pytest.mark.parametrize("name,sub", [("tiny", None), ("small", None), ("massive", 16), ("precision", 16)])
def test_split_bf16_dft_gemm_against_oracle(name, sub):
    """The 2D DFTs as split-BF16 tcgen05 GEMMs (two bf16 parts, three
    products: the 3-term form) on every geometry, including the 8-layer
    precision design (4 GEMMs per gap, 36 chained GEMMs forward): field,
    intensity and gradient against the FP64 oracle within the split-BF16
    target of 1e-4, in relative L2 and element by element."""
    w = W.workload(name)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    if sub:
        idx = W.subset_indices(w.n_lambda, sub)
        w, T = w.subset(idx), T[idx]
    st = _stack(w, path="dft_gemm")
    assert st.path == "dft_gemm"
    hd = _t(h)
    I = st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(_t(T))
    g = _np(st.backward(dl)).astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(_np(o).astype(np.complex128), fwd["o"], SPLIT_TARGET, "field")
    assert_close(_np(I).astype(np.float64), fwd["I"], SPLIT_TARGET, "intensity")
    assert_close(g, g_ref, SPLIT_TARGET, "gradient")
    st.close()


@pytest.mark.parametrize("name,sub", [("tiny", None), ("small", None), ("massive", 16), ("precision", 16)])
def test_split_bf16_three_parts_meets_the_split_target(name, sub):
    """Three bf16 parts per operand and six products per GEMM: field,
    intensity and gradient within 1e-4 of the FP64 oracle (the split-BF16
    target) on every geometry, including the 8-layer precision design (36
    chained GEMMs, where two parts miss it); the short cascades meet the FP32
    paths' field tolerance.  What remains is the tensor core's FP32
    accumulation of the (0,0) product, ~1e-6 per GEMM at K = 1024."""
    w = W.workload(name)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    if sub:
        idx = W.subset_indices(w.n_lambda, sub)
        w, T = w.subset(idx), T[idx]
    st = _stack(w, path="dft_gemm_x3")
    assert st.path == "dft_gemm_x3"
    hd = _t(h)
    I = st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(_t(T))
    g = _np(st.backward(dl)).astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(_np(o).astype(np.complex128), fwd["o"], TOL_FIELD if name in ("tiny", "small") else SPLIT_TARGET,
                 "field")
    assert_close(_np(I).astype(np.float64), fwd["I"], SPLIT_TARGET, "intensity")
    assert_close(g, g_ref, SPLIT_TARGET, "gradient")
    st.close()


@pytest.mark.parametrize("n,m,k", [(51, 128, 2), (300, 512, 1), (7, 16, 3)])
def test_bulk_path_fallbacks_match_oracle(n, m, k):
    """Shapes where the bulk-prefetch passes fall back: odd N (checkpoint rows
    are not 16-byte multiples, the adjoint stages spectra instead), N > 256
    (one TMA box holds at most 256 rows, the column pass runs the plain
    kernel), and a single-tile M = 16."""
    fov = n if n < 16 else (n // 2 if (n - n // 2) % 2 == 0 else n // 2 + 1)  # N - F even
    w = custom(n, m, k, [480, 610, 720], 30, fov, name="bulk-fallback")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, path="multipass_bulk")
    assert st.path == "multipass_bulk"
    hd = _t(h)
    st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(_t(T))
    g = _np(st.backward(dl)).astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(_np(o).astype(np.complex128), fwd["o"], TOL_FIELD)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


def test_forced_configuration_and_tuning_cache(tmp_path, monkeypatch):
    """DOS_FORCE_CONFIG selects a named configuration without timing;
    DOS_TUNE_CACHE stores the tuned choice and a second context reuses it."""
    w = W.workload("batched")
    monkeypatch.setenv("DOS_FORCE_CONFIG", "multipass:bulk")
    st = _stack(w, path="auto")
    assert st.path == "multipass_bulk" and "DOS_FORCE_CONFIG" in L.dos_describe(st.handle)
    st.close()
    monkeypatch.delenv("DOS_FORCE_CONFIG")
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("DOS_TUNE_CACHE", str(cache))
    st = _stack(w, path="auto")
    first = st.path
    assert "tuned" in L.dos_describe(st.handle)
    st.close()
    assert cache.read_text().strip()
    st = _stack(w, path="auto")
    assert st.path == first and "tuning cache" in L.dos_describe(st.handle)
    st.close()


@pytest.mark.parametrize("mix", ["col", "row_fwd", "row_adj", "col+row_fwd", "col+row_adj", "row_fwd+row_adj"])
def test_mixed_multipass_kernels_match_oracle(monkeypatch, mix):
    """Under auto the tuner may run plain kernels for some pass kinds and the
    bulk-prefetching ones for the others; each mix is reachable by name and
    computes the oracle's field and gradient."""
    w = custom(100, 200, 3, [480, 610, 720], 30, 50, name="mixed")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_FORCE_CONFIG", f"multipass:bulk[{mix}]")
    st = _stack(w, path="auto")
    assert st.path == "multipass_bulk" and f"bulk[{mix}]" in L.dos_describe(st.handle)
    hd = _t(h)
    st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(_t(T))
    g = _np(st.backward(dl)).astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(_np(o).astype(np.complex128), fwd["o"], TOL_FIELD)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("path", ["dft_gemm", "dft_gemm_x3"])
@pytest.mark.parametrize("n,m,k", [(50, 128, 2), (7, 16, 1), (100, 200, 3)])
def test_split_bf16_ragged_shapes(path, n, m, k):
    """Shapes off the tile grid: N not a multiple of 8 (the row-DFT epilogue
    stores element by element), K padding (2N, 2M not multiples of 64), a
    data operand that is not a whole number of 256-row tiles, M = 16."""
    fov = n if n < 16 else (n // 2 if (n - n // 2) % 2 == 0 else n // 2 + 1)
    w = custom(n, m, k, [480, 610, 720], 30, fov, kappa=0.01, name="gemm-ragged")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    st = _stack(w, path=path)
    hd = _t(h)
    I = st.forward(hd)
    o = st.output_field()
    _, _, dl = st.loss(_t(T))
    g = _np(st.backward(dl)).astype(np.float64)
    L_ref, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(_np(o).astype(np.complex128), fwd["o"], SPLIT_TARGET)
    assert_close(_np(I).astype(np.float64), fwd["I"], SPLIT_TARGET)
    assert_close(g, g_ref, TOL_GRAD_FD)
    st.close()
