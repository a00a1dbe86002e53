"""Host-side accounting of the benchmark (CPU only): the in-image tap count
behind GRay/s and the roofline's algorithmic bytes equals the number of non-zero
entries of the Joseph system matrix that the oracle builds column by column; the
instruction-issue view is the stated arithmetic; the committed ncu figures are
only used while the kernel source they were taken on is unchanged."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1903_10088_gb300 import phantom as ph  # noqa: E402


@pytest.mark.parametrize("geom,n_subsets", [
    (ph.Geometry(n=16, n_views=24, n_channels=20), 4),
    (ph.Geometry(n=12, n_views=18, n_channels=15, channel_offset=0.3, view0_rad=0.1), 3),
])
def test_tap_counts_equal_nonzeros_of_the_oracle_matrix(geom, n_subsets):
    n = geom.n
    cols = []
    for k in range(n * n):
        e = np.zeros((n, n))
        e.flat[k] = 1.0
        cols.append(oracle.forward(geom, e).ravel())     # column k of A, rays [V][C]
    A = np.stack(cols, axis=1)
    nz_per_view = (A != 0).reshape(geom.n_views, geom.n_channels, n * n).sum(axis=(1, 2))
    expected = np.array([nz_per_view[s::n_subsets].sum() for s in range(n_subsets)])
    taps = bench._tap_counts(geom, n_subsets)
    assert taps.tolist() == expected.tolist()


def test_issue_roofline_arithmetic():
    r = bench.issue_roofline(1.0e12, 1.0, 152, 2000.0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(4 * 152 * 2.0e9 / 1e9)
    assert r["achieved"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(1.0e12 / (4 * 152 * 2.0e9))
    assert bench.issue_roofline(None, 1.0, 152, 2000.0) is None
    assert bench.issue_roofline(1.0e12, 1.0, 152, None) is None


def test_ncu_record_only_for_the_source_it_was_taken_on(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "k_recon_traffic.json")) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["kernel_source_sha256_16"])
    assert bench.ncu_record() == rec
    assert bench.ncu_traffic() == rec["dram_bytes_per_launch_full_workload"]
    assert rec["dram_bytes_per_launch_full_workload"] == (rec["dram_bytes_read_per_launch"]
                                                          + rec["dram_bytes_write_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_record() is None and bench.ncu_traffic() is None
