"""Host rules of bench.py that shape its JSON line, without a GPU: the roofline's DRAM traffic is
taken from a committed capture only while the captured kernel's source is unchanged (else null),
scaled by the launch's algorithmic work; the L2 note compares the FP64 space-time iterate with the
129 MB L2."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from sfde_workloads import WORKLOADS  # noqa: E402


def test_traffic_needs_the_captured_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    csrc = tmp_path / "paper_1805_06688_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for files in bench.KERNEL_SOURCES.values():
        for f in files:
            (csrc / f).write_text("// kernel source " + f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_sha("k_digit_gemm_int")
    (prof / "traffic.json").write_text(json.dumps({
        "k_digit_gemm_int": {"source_sha": sha, "dram_bytes_per_alg_byte": 0.5},
        "k_fused_step": {"source_sha": "stale", "dram_bytes_per_flop": 1.0}}))
    assert bench.traffic_from_profile("k_digit_gemm_int", 1e12, 2e8) == 1e8
    assert bench.traffic_from_profile("k_fused_step", 1e12, 2e8) is None     # source changed
    assert bench.traffic_from_profile("k_tc_slice_gemm", 1e12, 2e8) is None  # never captured
    (csrc / "ozaki.cu").write_text("// kernel source changed")
    assert bench.traffic_from_profile("k_digit_gemm_int", 1e12, 2e8) is None


def test_l2_note_against_the_iterate_size():
    assert "larger than the 129 MB L2" in bench.l2_note(WORKLOADS["bump_N511_Nt2048"])
    assert "4.28 GB" in bench.l2_note(WORKLOADS["bump_N511_Nt2048"])   # 2049 x 511^2 x 8 B
    assert "fits in L2" in bench.l2_note(WORKLOADS["manufactured_N31_Nt64"])
