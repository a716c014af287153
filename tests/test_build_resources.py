"""Resources of the default launch of the pruned tile search, read from ptxas
(-Xptxas -v) for sm_103a: four blocks of kTileThreads threads must fit on one
SM.  Registers: at most 65,536 per SM.  Shared memory: static plus dynamic
(pruned_smem_bytes of the default staging capacity) plus the 1 KiB the runtime
reserves per block, at most a quarter of the SM's 228 KiB.  Both the launch
bounds and the default staging capacity are chosen for that occupancy, and a
change that breaks it would cost speed without failing any result check."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1210_8084_gb300", "csrc")
SM_SHARED_BYTES = 228 * 1024       # shared memory of one SM (sm_100 family)
BLOCK_RESERVED_BYTES = 1024        # reserved by the runtime per resident block
SM_REGISTERS = 65536


def _constant(text, name):
    m = re.search(r"constexpr int %s = (\d+);" % name, text)
    assert m, name
    return int(m.group(1))


def _entry_resources(ptxas_log, mangled_part):
    """(registers, static shared bytes, spill store bytes) of the entry whose
    mangled name contains mangled_part."""
    blocks = ptxas_log.split("Compiling entry function")
    for blk in blocks[1:]:
        if mangled_part not in blk.split("\n", 1)[0]:
            continue
        regs = int(re.search(r"Used (\d+) registers", blk).group(1))
        smem = re.search(r"(\d+) bytes smem", blk)
        spill = re.search(r"(\d+) bytes spill stores", blk)
        return regs, int(smem.group(1)) if smem else 0, int(spill.group(1)) if spill else 0
    raise AssertionError("entry not found: " + mangled_part)


def test_default_pruned_tile_launch_fits_four_blocks_per_sm(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    kernels = open(os.path.join(CSRC, "kmc_kernels.cuh")).read()
    internal = open(os.path.join(CSRC, "kmc_internal.h")).read()
    cap = _constant(internal, "kPrunedCap")
    threads = _constant(kernels, "kTileThreads")
    cluster = _constant(kernels, "kCluster")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-c",
                        os.path.join(CSRC, "kmc_f32.cu"), "-o", str(tmp_path / "kmc_f32.o"), "-Xptxas", "-v"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    log = r.stdout + r.stderr
    for dim in (3, 2):
        regs, static, _ = _entry_resources(log, "tile_pruned_kernelILi%dELi%dE" % (dim, cap))
        dynamic = (24 + 16 // cluster) * (cap & ~15)   # six floats per staged slot, one box record per cluster
        assert 4 * regs * threads <= SM_REGISTERS, (dim, regs)
        assert 4 * (static + dynamic + BLOCK_RESERVED_BYTES) <= SM_SHARED_BYTES, (dim, static, dynamic)
