"""Host logic of bench.py that needs no GPU: the serving stream's request
recipe, the workload configs, the DFT report arithmetic and the gating of
profiled DRAM traffic on the kernel source."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_serving_requests_are_seeded_and_follow_the_recipe():
    a = bench.serve_requests(0, 64, 7)
    assert a == bench.serve_requests(0, 64, 7)          # same seed, same stream
    assert a != bench.serve_requests(1, 64, 7)
    for r in a:
        assert r["K"] in (16, 32, 64, 128, 256)
        assert 4 <= r["level"] <= 7
        assert 1e-6 <= r["beta"] <= 1e-2
        if r["oseen"]:
            assert r["nu"] in (1 / 50, 1 / 100)
            assert r["omega_conv"] == (0.5 if r["beta"] > 1e-4 else 0.0)
        else:
            assert r["nu"] == 1e-2 and r["omega_conv"] == 0.0
    assert any(r["oseen"] and r["beta"] > 1e-3 for r in a)  # the full beta range, Oseen included
    assert any(r["oseen"] and r["level"] == 4 for r in a)   # and the full grid range
    kinds = [r["oseen"] for r in a]
    assert 16 < sum(kinds) < 48                           # 50/50 draw
    assert all(r["level"] <= 5 for r in bench.serve_requests(0, 64, 5))


def test_workload_configs():
    c = bench.workload_config("stokes64_nt256", 2)
    assert (c["grid"], c["n_t"], c["betas"], c["parallelism"]) == ("64x64 Q2-Q1", 256, [1e-2, 1e-4, 1e-6], "replicas x2")
    assert c["l2"].startswith("inputs larger than L2")
    assert bench.workload_config("oseen256_nt128", 1)["outer"] == "FGMRES(20), tol 1e-8"


class _Sizes:
    n_t, J, n_blk = 256, 129, 75014


def test_dft_report_arithmetic():
    rep = bench.dft_report(_Sizes, {"dft_fwd": {"launches": 2, "timed": 2, "ms": 0.4}}, (1000.0, "x"))
    nbytes = 256 * 75014 * 8 + 129 * 75014 * 8
    assert rep["bytes_per_launch"] == nbytes
    assert abs(rep["dft_fwd"]["GBps"] - nbytes / 2e-4 / 1e9) < 1.0
    flops = 6 * 2 * 128 * 256 * 256 * ((75014 + 127) // 128)
    assert abs(rep["dft_fwd"]["tensor_tflops_issued"] - flops / 2e-4 / 1e12) < 0.1


def test_profiled_traffic_needs_matching_source():
    t = bench.profiled_traffic("mg_q2b_kernel_stokes64_nt256.md", "k_mg.cu")
    assert t is None or t > 1e9                              # None once the kernel source changed
    assert bench.profiled_traffic("mg_q2b_kernel_stokes64_nt256.md", "k_fields.cu") is None


def test_profiled_traffic_region_gate(tmp_path, monkeypatch):
    """With a kernel_source_end line only the text before it is hashed: edits
    after it keep the traffic figure, edits before it drop it."""
    import hashlib
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2405_18964_gb300" / "csrc"
    csrc.mkdir(parents=True)
    head, marker = b"__global__ void k() {}\n", "// other kernels"
    (csrc / "k.cu").write_bytes(head + marker.encode() + b"\nvoid f() {}\n")
    (tmp_path / "profiles" / "k.md").write_text(
        f"kernel_source_sha1: {hashlib.sha1(head).hexdigest()} (k.cu)\n"
        f"kernel_source_end: {marker}\ntraffic_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", "k.cu") == 1234
    (csrc / "k.cu").write_bytes(head + marker.encode() + b"\nvoid f() { g(); }\n")
    assert bench.profiled_traffic("k.md", "k.cu") == 1234
    (csrc / "k.cu").write_bytes(b"__global__ void k() { x(); }\n" + marker.encode() + b"\n")
    assert bench.profiled_traffic("k.md", "k.cu") is None
