"""CPU checks of the C-ABI library: it builds, loads, exports every declared symbol and its
structs match the header.  No compute calls (no GPU here)."""
import ctypes
import re
import subprocess

import pytest

import paper_1604_01093_b300 as bf
from paper_1604_01093_b300 import build as bfbuild
from paper_1604_01093_b300 import _lib

HEADER = bfbuild.INCLUDE / "bf.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_loads():
    path = bfbuild.build()
    assert path.exists()
    bf.lib()


def test_every_declared_symbol_is_exported():
    L = bf.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(_lib.EXPORTS) == names


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bf.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(bf_config), sizeof(bf_solve_params),'
                   ' sizeof(bf_solve_stats), offsetof(bf_solve_stats, r_max), offsetof(bf_solve_params, tile_px));}')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", str(bfbuild.INCLUDE), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(_lib.Config)
    assert int(out[1]) == ctypes.sizeof(_lib.SolveParams)
    assert int(out[2]) == ctypes.sizeof(_lib.SolveStats)
    assert int(out[3]) == _lib.SolveStats.r_max.offset
    assert int(out[4]) == _lib.SolveParams.tile_px.offset


def test_defaults_follow_the_paper():
    p = bf.default_params()
    assert p.tau_dist == 0.15 and p.tau_normal == 0.9 and p.max_angle_deg == 60.0
    cfg = _lib.Config()
    bf.lib().bf_default_config(ctypes.byref(cfg))
    assert (cfg.width, cfg.height) == (80, 60)


def test_status_strings():
    L = bf.lib()
    for s in range(8):
        assert L.bf_status_string(s)


def test_null_context_is_rejected_without_gpu():
    L = bf.lib()
    assert L.bf_destroy(None) == 0
    assert L.bf_solve_local(None, 0, None, 0, None, None) == 1
    assert L.bf_add_frames(None, 0, 0, None, None, 0, None) == 1
