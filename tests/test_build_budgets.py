"""Register and spill budgets of the hot kernels (no GPU): the CUDA translation unit is
compiled for sm_103a with ptxas's resource report, and the kernels whose occupancy the
design relies on are held to it:

* the default stencil form fits eight 256-thread blocks per SM (at most 32 registers)
  without spilling;
* the tensor-core GEMM configurations and the one-orbital tiled contraction spill
  nothing;
* the node-major transforms with a cell split between four lanes fit six 128-thread
  blocks per SM (at most 80 registers; the back transform spills at most 16 bytes), the
  forward transforms of the other node-major forms spill nothing at their default caps;
* the density pass and the column scales stay small."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1908_02456_gb300", "csrc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("ptxas") / "api.o"
    p = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v", "-Xcompiler", "-fPIC",
                        "-c", os.path.join(CSRC, "api.cu"), "-o", str(out)],
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    res, cur = {}, None
    for line in p.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            cur = m.group(1)
            res[cur] = {"regs": None, "spill": 0}
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            res[cur]["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            res[cur]["regs"] = int(m.group(1))
    return res


def pick(report, *parts):
    hits = {k: v for k, v in report.items() if all(s in k for s in parts)}
    assert hits, parts
    return hits


def test_stencil_fits_eight_blocks_per_sm(report):
    for v in pick(report, "stencil_stage_x2_lb", "ILi8E").values():
        assert v["regs"] <= 32 and v["spill"] == 0, v


def test_contractions_do_not_spill(report):
    gemm = pick(report, "gemm_tc")
    assert len(gemm) == 6                                  # {TF32, FP16} x {96-wide, 64 x 2, Karatsuba}
    for k, v in gemm.items():
        assert v["spill"] == 0, (k, v)
    for v in pick(report, "sym_gemv_tiles").values():
        assert v["spill"] == 0, v


def test_four_lane_transforms_fit_six_blocks_per_sm(report):
    for v in pick(report, "bnd_forward_quadsILi6E").values():
        assert v["regs"] <= 80 and v["spill"] == 0, v
    for v in pick(report, "bnd_back_quads_xILi6E").values():
        assert v["regs"] <= 80 and v["spill"] <= 16, v
    for part in ("bnd_forward_pairsILi4E", "bnd_forward_lanes", "bnd_back_lanesENS"):
        for v in pick(report, part).values():
            assert v["spill"] == 0, (part, v)


def test_small_kernels_stay_small(report):
    for part in ("density_potentialIfE", "tc_colexp_nm", "tc_colexpENS"):
        for v in pick(report, part).values():
            assert v["regs"] <= 40 and v["spill"] == 0, (part, v)
