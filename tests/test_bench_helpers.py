"""Host-side pieces of the benchmark: the code digest that keys recorded
profiles ignores comments but not code, and the recorded trace traffic is
reported only for the kernel source it was captured on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_digest_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("// header\nint f() { return 1; }\n\n   // note\nint g();\n")
    b = tmp_path / "b.cu"
    b.write_text("// another header\nint f() { return 1; }\nint g();   \n")
    c = tmp_path / "c.cu"
    c.write_text("int f() { return 2; }\nint g();\n")
    assert bench.kernel_code_digest(a) == bench.kernel_code_digest(b)
    assert bench.kernel_code_digest(a) != bench.kernel_code_digest(c)


def test_digest_can_leave_out_a_marked_section(tmp_path):
    first, stop = "// section A", "// section B"
    a = tmp_path / "a.cu"
    a.write_text(f"int f();\n{first}\nint g() {{ return 1; }}\n{stop}\nint h();\n")
    b = tmp_path / "b.cu"
    b.write_text(f"int f();\n{first}\nint g() {{ return 2; }}\n{stop}\nint h();\n")
    c = tmp_path / "c.cu"
    c.write_text(f"int f();\n{first}\nint g() {{ return 2; }}\n{stop}\nint h2();\n")
    skip = (first, stop)
    assert bench.kernel_code_digest(a, skip) == bench.kernel_code_digest(b, skip)
    assert bench.kernel_code_digest(a) != bench.kernel_code_digest(b)
    assert bench.kernel_code_digest(b, skip) != bench.kernel_code_digest(c, skip)
    # a marker that is missing or repeated: nothing is left out
    d = tmp_path / "d.cu"
    d.write_text(f"int f();\n{first}\nint g() {{ return 1; }}\nint h();\n")
    assert bench.kernel_code_digest(d, skip) == bench.kernel_code_digest(d)


def test_psf_section_markers_occur_once_in_the_kernel_source():
    src = os.path.join(ROOT, "paper_1505_07674_gb300", "csrc", "lensed_kernels.cu")
    lines = [line.rstrip() for line in open(src, encoding="utf-8")]
    first, stop = bench.PSF_SECTION
    assert lines.count(first) == 1 and lines.count(stop) == 1
    assert lines.index(first) < lines.index(stop)
    inside = "\n".join(lines[lines.index(first):lines.index(stop)])
    assert "k_psf(" in inside and "k_psf_sep(" in inside and "k_trace_rows" not in inside


def test_recorded_traffic_is_reported_only_for_the_captured_kernel_code():
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_trace_rows_traffic.txt")))
    src = os.path.join(ROOT, "paper_1505_07674_gb300", "csrc", "lensed_kernels.cu")
    if rec["code_sha256"] != bench.trace_code_digest(src):
        # the kernels changed since the capture: no traffic figure
        assert bench.trace_traffic(rec["points"]) is None
        return
    full = bench.trace_traffic(rec["points"])
    assert abs(full - rec["dram_bytes"]) <= 1e-6 * rec["dram_bytes"]
    assert abs(bench.trace_traffic(512) - rec["dram_bytes_per_point"] * 512) < 1.0
