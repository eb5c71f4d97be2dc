"""The algorithmic operation counts bench.py uses for its roofline are the ones the kernels'
own element templates produce on a counting scalar (tests/flop_count.cu)."""
import json
import os
import subprocess
import tempfile

import pytest

from paper_2606_04206_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bench_flop_constants_match_the_count():
    import bench
    exe = os.path.join(tempfile.mkdtemp(), "flop_count")
    r = subprocess.run([build.nvcc(), "-O0", "-std=c++17", "--expt-relaxed-constexpr", "-I", build.CSRC,
                        os.path.join(HERE, "flop_count.cu"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    assert bench.FLOPS_FWD_PER_VS == pytest.approx(out["forward_per_vertex_substep"], abs=0.05)
    assert bench.FLOPS_BWD_PER_VS == pytest.approx(out["backward_per_vertex_substep"], abs=0.05)
    # the hinge (the dominant element) is several hundred operations each way
    assert out["hinge_forward"] > 200 and out["hinge_reverse"] > 400
