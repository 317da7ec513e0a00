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
    assert kf("path=multipass:bulk[col] (DOS_FORCE_CONFIG)", "row_forward") is None
    assert kf("path=fused:C5:L16 threads=320 clusters=28 smem=1", "column_forward") is None


def test_traffic_entries_cite_committed_profiles():
    for key, (bytes_per_channel, src) in bench.TRAFFIC_PER_CHANNEL.items():
        assert bytes_per_channel > 0
        assert os.path.isfile(os.path.join(ROOT, src)), (key, src)
