"""CPU checks of the benchmark's roofline bookkeeping: the algorithmic work
of each stage's dominant kernel at the 703,026 x 1,000, k = 40 workload
against the figures worked out by hand from the data layout (read I in
fp32, the transformed cube as two bf16 terms padded to 64 spectra x 256
channels, P in fp32, Im in fp32; LAPACK's 4/3 m^3 for the Householder
tridiagonalisation; three bf16 products over the upper triangle of the
Gram matrix), and the rule that a stored DRAM-traffic figure is reported
only for the kernel sources it was captured on."""
import json

import pytest

import bench

N, M, K = 703_026, 1_000, 40
N_PAD, M_PAD = 703_040, 1_024  # 64-spectrum and 256-channel padding


@pytest.mark.parametrize("stage,want", [
    ("transform", 4 * N * M + 2 * 2 * N_PAD * M_PAD),   # 2.812 GB in + 2.880 GB out
    ("gram", 3 * M * M * N),                            # 2.109e12 flops
    ("eig", 4 * M ** 3 / 3),                            # 1.333e9 double-word flops
    ("project", 2 * 2 * N_PAD * M_PAD + 4 * N * K),     # 2.880 GB in + 0.112 GB out
    ("recon", 4 * N * M + 4 * N * K),                   # 2.812 GB out + 0.112 GB in
])
def test_work_model(stage, want):
    assert bench.algorithmic_work(stage, N, M, K) == pytest.approx(want, rel=1e-12)


def test_work_model_figures_in_gigabytes():
    gb = lambda s: bench.algorithmic_work(s, N, M, K) / 1e9  # noqa: E731
    assert round(gb("transform"), 2) == 5.69
    assert round(gb("project"), 2) == 2.99
    assert round(gb("recon"), 2) == 2.92
    assert bench.algorithmic_work("gram", N, M, K) == pytest.approx(2.109078e12)


def test_randomised_svd_work():
    # 2q + 2 passes over the padded bf16 hi + lo cube, q = 2: 17.3 GB
    want = (2 * bench.RSVD_POWER_ITERS + 2) * 2 * 2 * N_PAD * M_PAD
    assert bench.algorithmic_work("eig", N, M, K, svd="randomized") == pytest.approx(want)
    assert round(want / 1e9, 1) == 17.3
    assert bench.algorithmic_work("gram", N, M, K, svd="randomized") is None


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(
        {"k1": {"dram_bytes_per_launch": 100.0, "scale": 2.5, "source_hash": "abc"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k1", "abc") == pytest.approx(250.0)
    assert bench.traffic_from_profiles("k1", "abd") is None
    assert bench.traffic_from_profiles("k2", "abc") is None


def test_stage_kernels_have_sources():
    import os
    for stage, (kernel, srcs, bound) in bench.STAGE_KERNEL.items():
        assert bound in ("hbm", "tensor", "alu"), stage
        for f in srcs:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2005_07132_gb300", "csrc", f)), f
        assert len(bench.source_hash(srcs)) == 16
