"""The C-ABI library builds, loads and exports every entry point declared in include/*.h
(no compute calls: this runs without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

from paper_2511_08498_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(dex_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "dex_formal_solve_dense" in names and "dex_ctx_create" in names


def test_library_exports_every_declared_symbol():
    L = _native.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_prototypes_cover_header():
    assert set(declared_functions()) <= set(_native.PROTOTYPES)


def test_version_and_status_strings():
    L = _native.lib()
    assert L.dex_version() == 100
    assert L.dex_status_string(0) == b"ok"
    assert L.dex_status_string(1) == b"invalid argument"


def test_planes_size_arithmetic():
    L = _native.lib()
    assert L.dex_planes_floats(10, 11, 4) == 3 * 10 * 8
    assert L.dex_planes_floats(10, 0, 8) == 0
    assert L.dex_planes_floats(10, 3, 3) == 0  # unsupported batch width


def test_context_creation_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert _native.lib().dex_ctx_create(0, None, ctypes.byref(h)) == 2  # DEX_ERR_CUDA
    assert not h.value


def test_3d_size_arithmetic():
    # 8^3 blocks with levels 0..3: 512 + 64 + 8 + 1 = 585 records (1.14x MIP 0, Section 2.1);
    # states: 3 bits, 21 per 64-bit word (Section 2.3.1), so a 512^3 grid's 262144
    # blocks take ceil(262144 / 21) = 12484 words.
    L = _native.lib()
    assert [L.dex_chain_voxels3(m) for m in range(4)] == [512, 576, 584, 585]
    assert L.dex_chain_voxels3(4) == 0
    assert L.dex_state_words3(512, 512, 512) == -(-262144 // 21) == 12484
    assert L.dex_state_words3(8, 8, 8) == 1
    assert L.dex_brick3_floats(10, 9, 8, 3, 0) == 2 * 10 * 585 * 16
    assert L.dex_brick3_floats(10, 9, 8, 3, 1) == 2 * 10 * 585 * 8
    assert L.dex_brick3_floats(10, 9, 8, 4, 0) == 0
