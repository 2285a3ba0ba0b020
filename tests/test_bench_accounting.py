"""The bench's accounting, on the CPU: the algorithmic flops behind every roofline
fraction against the per-k-point counts of the method's steps (complex multiply-add
= 8 real flops; eigensolve 16/3 n^3 + 8 n^2 p, overlap 8 n p^2, loop product 8 p^3),
the whole-job throughput formula, and the reading of committed ncu traffic lines."""
import os

import pytest

import bench


def _per_k(n, p):
    return {"eigh": 16.0 / 3.0 * n ** 3 + 8.0 * n * n * p, "overlap": 8.0 * n * p * p,
            "product": 8.0 * p ** 3}


@pytest.mark.parametrize("n, p, eigh, overlap, product", [
    (4, 2, 597.3, 128.0, 64.0),            # four-band models (spin Hall, BBH)
    (256, 64, 1.23e8, 8.39e6, 2.10e6),     # many-band model
    (400, 200, 5.97e8, 1.28e8, 6.40e7),    # disordered supercell L = 10
])
def test_per_k_counts(n, p, eigh, overlap, product):
    c = _per_k(n, p)
    assert c["eigh"] == pytest.approx(eigh, rel=2e-3)
    assert c["overlap"] == pytest.approx(overlap, rel=2e-3)
    assert c["product"] == pytest.approx(product, rel=2e-3)


def test_headline_kernel_flops():
    """BBH 60 x 60 nested (n = 4, p = 2, m = 1): states per k-point, overlaps per
    k-point, N products and one 2 x 2 eigen-decomposition (10 p^3) plus the transport
    per loop, and the nested products per base point."""
    n, p, N, Nt, m, nhop = 4, 2, 60, 60, 1, 12
    fl = bench.algorithmic_flops(n, p, N, Nt, m, nhop)
    K = N * Nt
    c = _per_k(n, p)
    assert fl["states"] == pytest.approx(K * (c["eigh"] + 8.0 * nhop))
    assert fl["overlaps"] == pytest.approx(K * c["overlap"])
    assert fl["loops"] == pytest.approx(Nt * (N * c["product"] + 10.0 * p ** 3
                                              + N * (8.0 * n * p * m + 8.0 * p * p * m)))
    assert fl["nested"] == pytest.approx(N * (Nt * (8.0 * n * m * m + 8.0 * m ** 3) + 10.0 * m ** 3))


def test_many_band_stage_flops():
    n, p, N, Nt = 256, 64, 101, 101
    K = N * Nt
    fl = bench.manyband_stage_flops(n, p, N, Nt, nnz_groups=1000, mixed=True, n_ent=n * n)
    assert fl["lg_tridiag"] == pytest.approx(K * 16.0 / 3.0 * n ** 3)
    assert fl["lg_backtransform"] == pytest.approx(K * 8.0 * n * n * (p + 1))  # p + 1 vectors (gap)
    assert fl["overlaps"] == pytest.approx(K * 8.0 * n * p * p)
    assert fl["lg_refine"] == pytest.approx(K * (8.0 * n * n * p + 16.0 * n * (n - p) * p + 16.0 * n * p * p))
    fp64 = bench.manyband_stage_flops(n, p, N, Nt, nnz_groups=1000, mixed=False)
    assert "lg_refine" not in fp64
    assert fp64["lg_backtransform"] == pytest.approx(K * 8.0 * n * n * p)


def test_weak_scaling_value():
    # all ranks' units over the slowest rank's seconds
    assert bench.weak_scaling_value(3600, 20, 4, 0.5) == pytest.approx(3600 * 20 * 4 / 0.5)


def test_committed_traffic_reads_only_a_matching_capture(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    names = ["loops.cu", "launch.h"]
    sha = bench.sources_sha256(names)
    (tmp_path / "a.md").write_text(
        "x\ntraffic: kernel=kfoo workload=w1 dram_bytes_per_launch=12345 "
        f"sources={','.join(names)} sha256={sha}\n")
    assert bench.committed_traffic("kfoo", "w1") == (12345, "a.md")
    got, why = bench.committed_traffic("kfoo", "w2")
    assert got is None and why
    (tmp_path / "a.md").write_text(
        "traffic: kernel=kfoo workload=w1 dram_bytes_per_launch=12345 "
        f"sources={','.join(names)} sha256={'0' * 64}\n")
    got, why = bench.committed_traffic("kfoo", "w1")
    assert got is None and "changed" in why
