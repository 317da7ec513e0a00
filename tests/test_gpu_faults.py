"""Bounded device waits: an injected stall makes the bulk-prefetch passes'
waits expire, the host reads DOS_ERR_TIMEOUT, and the context stays usable.

The fault is made on the host (DOS_INJECT_WAIT_TIMEOUT at dos_create): the
first bulk pass announces bytes to its mbarrier without copying them, so the
wait of every block runs into its one-second limit; nothing traps or hangs.
"""
import os
import time

import numpy as np
import pytest
import torch

from oracle import dos_oracle as O
from paper_2604_02624_gb300 import _lib as L
from paper_2604_02624_gb300 import workloads as W
from paper_2604_02624_gb300.api import DiffractiveStack

from gpu_cases import TOL_GRAD_ORACLE, TOL_INTENSITY, TOL_LOSS, assert_close, custom, oracle_model

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _geometry(name):
    """tiny: M = 128, the column pass with one shared H tile; m512: N = 256 in
    M = 512, the column pass whose groups stage their H rows in their stage
    slots."""
    if name == "m512":
        return custom(256, 512, 1, [520, 610], 30, 64, name="m512")
    return W.workload(name)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not os.path.exists(L.LIB_PATH):
        from paper_2604_02624_gb300 import build
        build.build()
    L.load()
    torch.cuda.set_device(DEV)


def test_expired_bulk_wait_is_reported_and_context_recovers(monkeypatch):
    w = W.workload("tiny")
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_INJECT_WAIT_TIMEOUT", "1")
    st = DiffractiveStack.from_workload(w, device=DEV, path="multipass_bulk")
    monkeypatch.delenv("DOS_INJECT_WAIT_TIMEOUT")
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    t0 = time.time()
    st.forward(hd)
    with pytest.raises(L.DosError) as e:
        st.loss(Td)
    assert e.value.code == L.DOS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    # the same context, next call: normal results
    I = st.forward(hd).cpu().numpy().astype(np.float64)
    val, _, _ = st.loss(Td)
    L_ref, _, _, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(I, fwd["I"], TOL_INTENSITY)
    assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref)
    st.close()


@pytest.mark.parametrize("geometry", ["tiny", "m512"])
def test_expired_wait_in_the_staged_adjoint_row_pass(monkeypatch, geometry):
    """With only the adjoint row pass on its bulk kernel (both inputs staged by
    bulk copies), the injected stall reaches that pass: its blocks give up
    after the bounded waits, let their other copy land, and the next call that
    reads the device flag reports DOS_ERR_TIMEOUT; the context then computes
    the oracle's gradient.  At M = 512 the two inputs take turns in one
    stage."""
    w = _geometry(geometry)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_INJECT_WAIT_TIMEOUT", "1")
    monkeypatch.setenv("DOS_FORCE_CONFIG", "multipass:bulk[row_adj]")
    st = DiffractiveStack.from_workload(w, device=DEV, path="auto")
    monkeypatch.delenv("DOS_INJECT_WAIT_TIMEOUT")
    monkeypatch.delenv("DOS_FORCE_CONFIG")
    assert "bulk[row_adj]" in L.dos_describe(st.handle)
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    t0 = time.time()
    st.forward(hd)
    _, _, dl = st.loss(Td)          # the forward passes are plain: no stall yet
    st.backward(dl)             # the first bulk pass: its waits expire
    st.forward(hd)
    with pytest.raises(L.DosError) as e:
        st.loss(Td)
    assert e.value.code == L.DOS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    st.forward(hd)
    _, _, dl = st.loss(Td)
    g = st.backward(dl).cpu().numpy().astype(np.float64)
    _, _, g_ref, _ = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("geometry", ["tiny", "m512"])
def test_expired_wait_in_the_column_pass(monkeypatch, geometry):
    """With only the column pass on its TMA kernel, the injected stall reaches
    that pass (its first forward gap): every block's wait for its input rows
    expires, the host reads DOS_ERR_TIMEOUT, and the context then computes
    the oracle's intensities and gradient, at M = 128 and at M = 512 (where
    the H rows share the stage slots with the input rows)."""
    w = _geometry(geometry)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_INJECT_WAIT_TIMEOUT", "1")
    monkeypatch.setenv("DOS_FORCE_CONFIG", "multipass:bulk[col]")
    st = DiffractiveStack.from_workload(w, device=DEV, path="auto")
    monkeypatch.delenv("DOS_INJECT_WAIT_TIMEOUT")
    monkeypatch.delenv("DOS_FORCE_CONFIG")
    assert "bulk[col]" in L.dos_describe(st.handle)
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    t0 = time.time()
    st.forward(hd)
    with pytest.raises(L.DosError) as e:
        st.loss(Td)
    assert e.value.code == L.DOS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    I = st.forward(hd).cpu().numpy().astype(np.float64)
    _, _, dl = st.loss(Td)
    g = st.backward(dl).cpu().numpy().astype(np.float64)
    _, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(I, fwd["I"], TOL_INTENSITY)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("geometry", ["tiny", "m512"])
def test_expired_transfer_table_wait_in_a_blocks_last_item_is_reported(monkeypatch, geometry):
    """DOS_INJECT_WAIT_TIMEOUT=3: the column pass's copies land, but every
    thread gives up its wait for the transfer-table tile of its block's last
    item.  No later item's verdict reads that, so the block takes it after
    its loop, lets the tile land and sets the error flag: the host reads
    DOS_ERR_TIMEOUT instead of results computed from a tile that had not
    landed.  The context then computes the oracle's results."""
    w = _geometry(geometry)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_INJECT_WAIT_TIMEOUT", "3")
    monkeypatch.setenv("DOS_FORCE_CONFIG", "multipass:bulk[col]")
    st = DiffractiveStack.from_workload(w, device=DEV, path="auto")
    monkeypatch.delenv("DOS_INJECT_WAIT_TIMEOUT")
    monkeypatch.delenv("DOS_FORCE_CONFIG")
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    t0 = time.time()
    st.forward(hd)
    with pytest.raises(L.DosError) as e:
        st.loss(Td)
    assert e.value.code == L.DOS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    I = st.forward(hd).cpu().numpy().astype(np.float64)
    _, _, dl = st.loss(Td)
    g = st.backward(dl).cpu().numpy().astype(np.float64)
    _, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(I, fwd["I"], TOL_INTENSITY)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


@pytest.mark.parametrize("geometry,force", [
    ("tiny", "multipass:bulk"), ("tiny", "multipass:bulk[row_adj]"), ("tiny", "multipass:bulk[row_fwd]"),
    ("tiny", "multipass:bulk[col]"), ("m512", "multipass:bulk[col]"), ("m512", "multipass:bulk[row_adj]"),
])
def test_split_wait_verdict_is_taken_by_the_whole_block(monkeypatch, geometry, force):
    """Each thread times its own bounded wait.  DOS_INJECT_WAIT_TIMEOUT=2 lets
    the copies of the next bulk pass land but makes the odd threads of every
    block give up their first wait: the block must take one verdict (all of
    its threads leave the item, none writes partial results) and the host
    must read DOS_ERR_TIMEOUT, not silently skipped items.  The context then
    computes the oracle's intensities and gradient."""
    w = _geometry(geometry)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    monkeypatch.setenv("DOS_INJECT_WAIT_TIMEOUT", "2")
    monkeypatch.setenv("DOS_FORCE_CONFIG", force)
    st = DiffractiveStack.from_workload(w, device=DEV, path="auto")
    monkeypatch.delenv("DOS_INJECT_WAIT_TIMEOUT")
    monkeypatch.delenv("DOS_FORCE_CONFIG")
    hd = torch.tensor(h, dtype=torch.float32, device=DEV)
    Td = torch.tensor(T, dtype=torch.float32, device=DEV)
    t0 = time.time()
    st.forward(hd)
    if force.endswith("[row_adj]"):
        _, _, dl = st.loss(Td)       # forward passes plain: nothing injected yet
        st.backward(dl)          # the first bulk pass of this configuration
        st.forward(hd)
    with pytest.raises(L.DosError) as e:
        st.loss(Td)
    assert e.value.code == L.DOS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    I = st.forward(hd).cpu().numpy().astype(np.float64)
    _, _, dl = st.loss(Td)
    g = st.backward(dl).cpu().numpy().astype(np.float64)
    _, _, g_ref, fwd = O.loss_and_grad(h, T, **oracle_model(w))
    assert_close(I, fwd["I"], TOL_INTENSITY)
    assert_close(g, g_ref, TOL_GRAD_ORACLE)
    st.close()


def test_out_of_memory_is_reported_and_nothing_leaks():
    """A design whose checkpoints cannot fit (64 layers of 256 x 256 for 16384
    channels: 550 GB, after 26 GB of tables and spectra were allocated) fails in
    dos_create with DOS_ERR_OOM and a message; the device memory in use
    afterwards is what it was before."""
    free0, _ = torch.cuda.mem_get_info(DEV)
    lam = np.linspace(450e-9, 750e-9, 16384)
    with pytest.raises(L.DosError) as e:
        DiffractiveStack(n=256, m=512, n_layers=64, lambdas=lam, gaps=np.full(65, 1e-4), pitch=3e-7,
                         n_index=1.7, fov=64, path="multipass", device=DEV)
    assert e.value.code == L.DOS_ERR_OOM
    assert "cudaMalloc" in str(e.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert abs(free1 - free0) < 64 << 20
    # the library is still usable
    w = W.workload("tiny")
    st = DiffractiveStack.from_workload(w, device=DEV, path="multipass")
    st.forward(torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=DEV))
    st.close()


def test_non_finite_thickness_propagates_without_a_fault():
    """A NaN thickness pixel gives non-finite outputs (the caller's check finds
    them); no kernel traps and the context stays usable."""
    w = W.workload("tiny")
    h = W.thickness(w, 0).copy()
    st = DiffractiveStack.from_workload(w, device=DEV, path="multipass")
    hb = h.copy()
    hb[0, w.n // 2, w.n // 2] = np.nan
    I = st.forward(torch.tensor(hb, dtype=torch.float32, device=DEV))
    torch.cuda.synchronize()
    assert not torch.isfinite(I).all()
    I2 = st.forward(torch.tensor(h, dtype=torch.float32, device=DEV)).cpu().numpy().astype(np.float64)
    ref = O.forward(h, keep_fields=False, **oracle_model(w))["I"]
    assert_close(I2, ref, TOL_INTENSITY)
    st.close()
