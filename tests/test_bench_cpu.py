"""Host-side pieces of bench.py that need no GPU: the algorithmic-byte count
behind the roofline numerator and the options of its profiling entry."""
import os
import subprocess
import sys
from types import SimpleNamespace

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_of_the_rmat18_squaring():
    # R-MAT scale 18: m = 2^18 rows, nnz(A) = 7,613,374, nnz(C) = 2,958,724,919,
    # int32 columns and f64 values.  Symbolic: rowptr + col of A and of B (B = A)
    # plus rowptr(C); numeric: rowptr + col + val of A and of B, rowptr(C), and
    # 4 + 8 bytes written per C entry.
    m, nnz_a, nnz_c = 1 << 18, 7613374, 2958724919
    A = SimpleNamespace(nrows=m, nnz=nnz_a, col=np.empty(0, np.int32))
    sym, num = bench.algorithmic_bytes(A, nnz_c)
    a = 8 * (m + 1) + 4 * nnz_a
    assert sym == 2 * a + 8 * (m + 1)
    assert num == 2 * (a + 8 * nnz_a) + 8 * (m + 1) + 12 * nnz_c
    assert num == 35693711484          # the bench's roofline.algorithmic_bytes


def test_int64_columns_count_eight_bytes_per_index():
    A = SimpleNamespace(nrows=10, nnz=30, col=np.empty(0, np.int64))
    sym, num = bench.algorithmic_bytes(A, 50)
    a = 8 * 11 + 8 * 30
    assert sym == 2 * a + 8 * 11
    assert num == 2 * (a + 8 * 30) + 8 * 11 + 16 * 50


def test_profile_leg_options_are_listed():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert "--profile-leg" in out.stdout and "--products" in out.stdout
    for leg in ("product", "kslice", "batched", "batched-chain", "amg", "amg-chain", "mis2",
                "learned"):
        assert leg in out.stdout


def test_stage_report_sums_by_stage_and_product():
    stages = [(-1, "clear", 0.5), (0, "analysis", 1.0), (0, "numeric", 2.0),
              (1, "analysis", 3.0), (1, "numeric", 4.0)]
    r = bench._stage_report(stages)
    assert r["by_stage"] == {"clear": 0.5, "analysis": 4.0, "numeric": 6.0}
    assert r["by_product"] == {"0": 3.0, "1": 7.0}


def test_dense_kernel_digest_is_stored_with_the_traffic_figure():
    # the profile's traffic figure is used only while the kernel source
    # matches the digest recorded with it
    digest = bench.dense_kernel_digest()
    assert len(digest) == 16
    text = open(os.path.join(ROOT, "profiles", "numeric_dense_rmat18.md")).read()
    assert (f"`{digest}`" in text) == (bench.profiled_traffic() is not None)
