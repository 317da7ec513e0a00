"""Host logic of bench.py: which column kernel a configuration name runs, and
that every stored DRAM-traffic figure names a committed ncu summary."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_family_from_configuration_name():
    kf = bench.kernel_family
    assert kf("path=multipass:bulk | tuned (fwd+bwd ms): ...", "column_forward") == "column_bulk"
    assert kf("path=multipass:bulk[col+row_fwd] | tuned", "column_adjoint") == "column_bulk"
    assert kf("path=multipass:bulk[row_fwd+row_adj] | tuned", "column_forward") == "column_plain"
    assert kf("path=multipass (DOS_FORCE_CONFIG)", "column_adjoint") == "column_plain"
    assert kf("path=multipass:bulk[col] (DOS_FORCE_CONFIG)", "row_forward") == "row_plain"
    assert kf("path=multipass:bulk[row_fwd+row_adj] | tuned", "row_adjoint") == "row_bulk"
    assert kf("path=multipass:bulk | tuned", "row_forward") == "row_bulk"
    assert kf("path=multipass:bulk[col+row_fwd] | tuned", "row_adjoint") == "row_plain"
    assert kf("path=multipass:bulk", "loss") is None
    assert kf("path=fused:C5:L16 threads=320 clusters=28 smem=1", "column_forward") is None


def test_traffic_entries_cite_committed_profiles():
    for key, (bytes_per_channel, src) in bench.TRAFFIC_PER_CHANNEL.items():
        assert bytes_per_channel > 0
        assert os.path.isfile(os.path.join(ROOT, src)), (key, src)


def test_step_bytes_structure():
    """Each extra layer adds one forward and one adjoint row pass (spectra in
    and out, checkpoint) and one forward and one adjoint column pass (spectra
    in and out, a transfer-table quadrant); the ideal count is 40 N^2 bytes
    per layer-propagation; both scale with the channels."""
    n, m, F = 200, 400, 50
    hs = m // 2 + 1
    b2, b3 = bench.step_bytes(n, m, 2, F, 7), bench.step_bytes(n, m, 3, F, 7)
    per_layer = 2 * (16 * n * m + 8 * n * n) + 2 * (16 * n * m + 8 * hs * hs)
    assert b3["design"] - b2["design"] == 7 * per_layer
    assert b3["ideal"] == 7 * 4 * 40 * n * n
    assert bench.step_bytes(n, m, 5, F, 14)["design"] == 2 * bench.step_bytes(n, m, 5, F, 7)["design"]


def test_roofline_bytes_are_the_methods():
    """roofline.frac's numerator can be recomputed from the method's bytes
    alone: 16 N^2 bytes per forward and 24 N^2 per adjoint layer-propagation, times
    the channels a launch advances; the whole step is (K + 1) * 40 N^2 per
    channel, which is step_bytes' "ideal"."""
    mb = bench.method_bytes_per_launch
    n, K, nw = 200, 5, 4096
    assert mb("column_forward", nw, n, K) == 16 * n * n * nw == 2_621_440_000
    assert mb("column_adjoint", nw, n, K) == 24 * n * n * nw
    assert mb("row_forward", nw, n, K) == mb("column_forward", nw, n, K)
    assert mb("fused_forward", nw, n, K) + mb("fused_adjoint", nw, n, K) == \
        nw * (K * 40 + 16) * n * n
    # forward and adjoint launches of a multi-pass step add up to the step's
    # algorithmic bytes once the adjoint's missing gap 0 is accounted for
    per_step = (K + 1) * mb("column_forward", nw, n, K) + K * mb("column_adjoint", nw, n, K)
    assert per_step + mb("column_adjoint", nw, n, K) == bench.step_bytes(n, 400, K, 50, nw)["ideal"]
    assert mb("loss", nw, n, K) is None
