"""CPU checks of the C-ABI library: it builds, loads, exports every declared symbol and its
structs match the header.  No compute calls (no GPU here)."""
import ctypes
import re
import subprocess

import numpy as np
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


def test_noalloc_rejects_bad_arguments_before_touching_the_gpu():
    """bf_dense_pair_noalloc checks its arguments before any CUDA call, so this runs without a GPU:
    frame sizes outside 8..160 x 8..120, a depth range that is empty, and non-finite gates or weights
    are BF_ERR_INVALID_ARG.  (The device pointers are never dereferenced on the host.)"""
    import ctypes
    import math

    from paper_1604_01093_b300 import _lib

    L = _lib.lib()
    fake = ctypes.c_void_p(256)
    eye = np.eye(4).ravel().copy()

    def call(W=80, H=60, dmin=0.1, dmax=10.0, **kw):
        p = _lib.default_params(**kw)
        return L.bf_dense_pair_noalloc(W, H, 65.625, 65.625, (W - 1) / 2, (H - 1) / 2, dmin, dmax, fake, fake, fake,
                                       fake, eye.ctypes.data, eye.ctypes.data, ctypes.byref(p), fake, None)

    bad = [dict(W=320, H=240), dict(W=161), dict(H=121), dict(W=4), dict(dmin=2.0, dmax=1.0), dict(dmin=1.0, dmax=1.0),
           dict(tau_dist=0.0), dict(tau_dist=math.nan), dict(tau_normal=math.nan), dict(w_dense=math.inf),
           dict(w_photo=math.nan), dict(w_geo=-math.inf)]
    for kw in bad:
        assert call(**kw) == 1, kw  # BF_ERR_INVALID_ARG
