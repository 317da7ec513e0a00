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

from gpu_cases import TOL_INTENSITY, TOL_LOSS, oracle_model, rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


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
    assert rel_l2(I, fwd["I"]) <= TOL_INTENSITY
    assert abs(val - L_ref) <= TOL_LOSS * abs(L_ref)
    st.close()
