"""The C-ABI library loads, exports every entry point include/kmc.h declares,
and the ctypes mirrors of its structs have the C layout.  CPU only: no call
here reaches the device."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kmc.h")


def header_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"KMC_API\s+[\w\s\*]+?\b(kmc_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__ as g
    g.build()
    return os.path.join(ROOT, "paper_1210_8084_gb300", "libkmc.so")


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("kmc_init", "kmc_step", "kmc_moments", "kmc_free"):
        assert required in names
    assert len(names) >= 10


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(kmc_\w+)", out))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(built_lib):
    import paper_1210_8084_gb300 as k
    for f in header_functions():
        assert hasattr(k.lib, f), f
        assert hasattr(k, f), f
    assert set(k.ABI_FUNCTIONS) == set(header_functions())


def test_struct_layouts_match_c(built_lib):
    import ctypes
    import paper_1210_8084_gb300 as k
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "kmc.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(kmc_config), sizeof(kmc_instance), sizeof(kmc_info));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(kmc_config, stream), offsetof(kmc_config, flags),
         offsetof(kmc_info, vmax), offsetof(kmc_info, bytes_device), offsetof(kmc_info, stage_cap),
         offsetof(kmc_info, time));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [ctypes.sizeof(k.KmcConfig), ctypes.sizeof(k.KmcInstance), ctypes.sizeof(k.KmcInfo)]
    assert offs == [k.KmcConfig.stream.offset, k.KmcConfig.flags.offset, k.KmcInfo.vmax.offset,
                    k.KmcInfo.bytes_device.offset, k.KmcInfo.stage_cap.offset, k.KmcInfo.time.offset]


def test_invalid_config_is_rejected_without_device(built_lib):
    """Argument validation happens on the host before any CUDA call."""
    import numpy as np
    import paper_1210_8084_gb300 as k
    pos = np.zeros((4, 3), np.float32)
    vel = np.zeros((4, 3), np.float32)
    bad = [
        k.make_config(dim_pos=4),
        k.make_config(precision=16),
        k.make_config(n_cells=(0, 1, 1)),
        k.make_config(lo=(1, 0, 0), hi=(0, 1, 1)),
        k.make_config(bc=(3, 0, 0)),
        k.make_config(dim_pos=3, flags=k.KMC_FLAG_VELOCITY_2D),
        k.make_config(dt=0.0),
        k.make_config(lam=0.0, sigma=0.0),
        k.make_config(flags=1 << 9),
        k.make_config(tile_threads=100),
        k.make_config(tile_threads=288),
        k.make_config(tile_cap=63),
        k.make_config(tile_split=9),
    ]
    for cfg in bad:
        with pytest.raises(k.KmcError) as e:
            k.kmc_init(cfg, 4, pos, vel)
        assert e.value.code == k.KMC_EINVAL
        assert k.kmc_last_error(None)
    with pytest.raises(k.KmcError):
        k.kmc_init(k.make_config(instances=[dict(n=3, lam=1e-3, dt=1e-3)] * 2), 4, pos, vel)
