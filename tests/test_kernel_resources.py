"""Resources of the hot kernels as ptxas reports them (CPU only: nvcc
cross-compiles for sm_103a without a GPU).

  - no transform, scan or quantiser kernel has a stack frame or spills: a
    run-time index into a by-value parameter array (the base pointers of a
    launch) or into a local array makes the compiler copy it to the stack,
    and every thread then reads it back from local memory;
  - the tile kernels keep the residency their shared-memory budgets are
    designed for on a 228 KB SM (1 KB reserved per block): 8 blocks of
    128 threads of `k_dfb_b` (4 taps), 4 of `k_dfb_a` (4 taps) and 4 of
    `k_lp_ff` (the float-float LP tiles of the forward transform and the
    inverse).
"""
import functools
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_00561_b300", "csrc")
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

HOT = ("k_dfb_a", "k_dfb_b", "k_lp_level", "k_lp_ff", "k_pyr_tail", "k_scan_reduce", "k_scan_sums", "k_scan_apply",
       "k_quant_b", "k_unquant_b", "k_colour_fwd_b", "k_colour_inv_b", "k_rle_count_b", "k_rle_write_b")


@functools.lru_cache(maxsize=None)
def _ptxas(src):
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c",
           os.path.join(CSRC, src), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            name = m.group(1)
            out[name] = {}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[name].update(stack=int(m.group(1)), spill=int(m.group(2)) + int(m.group(3)))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out[name]["regs"] = int(m.group(1))
            s = re.search(r"(\d+) bytes smem", line)
            out[name]["smem"] = int(s.group(1)) if s else 0
    return out


def _hot(mangled):
    return next((k for k in HOT if k in mangled), None)


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
@pytest.mark.parametrize("src", ["k_dfb.cu", "k_lp.cu", "k_codec.cu", "k_tail.cu"])
def test_hot_kernels_have_no_stack_frame(src):
    res = _ptxas(src)
    seen = [k for k in res if _hot(k)]
    assert seen, "no hot kernel found in " + src
    for k in seen:
        assert res[k].get("stack") == 0 and res[k].get("spill") == 0, (k, res[k])


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_tile_kernels_keep_their_residency():
    per_sm, reserved = 228 * 1024, 1024

    def blocks(smem_bytes, regs, threads=256):
        by_smem = per_sm // (smem_bytes + reserved)
        by_regs = 65536 // (regs * threads)
        return min(by_smem, by_regs)

    dfb = _ptxas("k_dfb.cu")
    # 128-thread blocks (the launches of a wave or more), both first-target parities and directions
    b4 = [v for k, v in dfb.items() if "k_dfb_b" in k and "Li4ELb" in k and "Li128EE" in k]
    assert len(b4) == 4 and all(blocks(v["smem"], v["regs"], threads=128) >= 8 for v in b4), b4
    # k_dfb_a: 4 polyphase planes and 2 scratch planes of 44 x 45 floats, dynamic
    a4 = [v for k, v in dfb.items() if "k_dfb_a" in k and "Li4EE" in k]
    assert len(a4) == 2 and all(blocks(v["smem"] + 6 * 44 * 45 * 4, v["regs"]) >= 4 for v in a4), a4
    lp = _ptxas("k_lp.cu")
    # k_lp_ff<4, 3, *> (analysis and synthesis): 77 x 78 main tile, two 2,696-float and two 35 x 35
    # float-float arrays, dynamic
    ff = [v for k, v in lp.items() if "k_lp_ff" in k and "ILi4ELi3E" in k]
    assert len(ff) == 2 and all(blocks(v["smem"] + 4 * (6008 + 2 * 2696 + 2 * 35 * 35), v["regs"]) >= 4 for v in ff), ff
