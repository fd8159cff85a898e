"""Resource use of the benchmark's trace kernels, from the compiler (no GPU).

The trace kernels are bound by their instruction issue rate, so a register
spill in their ray loop, or a register count that halves the resident
warps, costs time that only a GPU run would otherwise reveal.  This test
compiles lensed_kernels.cu for sm_103a with the library's own flags and
reads ptxas's resource report (-Xptxas -v) for the instantiations that the
200x200 benchmark's autotuner chooses from: 5 x 5 Gauss-Legendre rows
(G = 5), FP32/MIXED and MIXED_FF, one CTA per item and persistent, and the
MIXED_FF second pass's pixel refinement.
"""
import os
import re
import subprocess
import tempfile

import pytest

from paper_1505_07674_gb300 import _build as B

# mangled-name fragments: k_trace_rows<MODE, 5, true, GQ> (MODE 0 = FP32, the
# first pass of MIXED too; 3 = MIXED_FF) in both launch forms, and
# k_refine_ff<5>
KERNELS = ("k_trace_rowsILi0ELi5ELb1ELb0E", "k_trace_rowsILi3ELi5ELb1ELb0E",
           "k_trace_rowsILi3ELi5ELb1ELb1E", "k_trace_rows_pqILi0ELi5ELb1ELb0E",
           "k_trace_rows_pqILi3ELi5ELb1ELb0E", "k_trace_rows_pqILi3ELi5ELb1ELb1E",
           "k_refine_ffILi5E")


@pytest.fixture(scope="module")
def report():
    try:
        exe = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    src = os.path.join(B.CSRC, "lensed_kernels.cu")
    with tempfile.TemporaryDirectory() as tmp:
        r = subprocess.run([exe, *B.ARCH, *B.NVCC_FLAGS, "-Xptxas", "-v", "-c", src, "-o",
                            os.path.join(tmp, "k.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, cur = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"(?:Compiling entry function|Function properties for) '?(\S+?)'?(?: for|$)",
                      line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            out.setdefault(cur, {})["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            out.setdefault(cur, {})["regs"] = int(m.group(1))
    return out


@pytest.mark.parametrize("frag", KERNELS)
def test_benchmark_trace_kernels_do_not_spill(report, frag):
    found = {k: v for k, v in report.items() if frag in k}
    assert found, (frag, sorted(report)[:5])
    for name, v in found.items():
        assert v.get("spill", 0) == 0, (name, v)
        # at most 80 registers: 64-thread CTAs then still fit 12 per SM
        assert v.get("regs", 0) <= 80 or "refine" in name, (name, v)
