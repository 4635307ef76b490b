"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/*.h declares, the ctypes table mirrors the header, and
argument validation rejects bad calls before touching the device."""
import ctypes
import glob
import os
import re

import pytest

import paper_1804_10694_gb300 as pkg
from paper_1804_10694_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gemm_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_ctypes_table_mirrors_header():
    assert _declared_functions() == set(_native.SIGNATURES)


def test_config_table():
    n = pkg.config_count("bf16x3")
    assert n == pkg.config_count("tf32x3") > 0
    assert pkg.config_count("simt") == 0
    seen = set()
    for i in range(n):
        c = pkg.config_get("bf16x3", i)
        assert c["block_n"] in ((64, 128) if c["cluster"] == 1 else (128, 256))
        assert c["cluster"] in (1, 2) and not (c["cluster"] == 2 and c["fused"])
        assert c["split_k"] >= 1 and 1 <= c["kb"] <= 8 and c["group_m"] >= 1
        key = tuple(sorted(c.items()))
        assert key not in seen
        seen.add(key)
    with pytest.raises(pkg.GemmError):
        pkg.config_get("bf16x3", n)
    # the six-product mode has the packed two thirds of the table (single
    # CTAs and pairs), two stages deep
    assert pkg.config_count("bf16x6") == n * 2 // 3
    for i in range(n * 2 // 3):
        c6, c3 = pkg.config_get("bf16x6", i), pkg.config_get("bf16x3", i)
        assert c6["fused"] == 0 and c6["stages"] == 2
        assert {k: v for k, v in c6.items() if k != "stages"} == \
            {k: v for k, v in c3.items() if k != "stages"}
    with pytest.raises(pkg.GemmError):
        pkg.config_get("bf16x6", n * 2 // 3)


def test_invalid_arguments_rejected_before_launch():
    lib = pkg.load()
    # negative size, ld below row length, null pointers: no device needed
    assert lib.gemm_f32(-1, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == 1
    assert lib.gemm_f32(4, 4, 8, 1.0, None, 7, None, 4, 0.0, None, 4) == 1
    assert b"lda" in lib.gemm_last_error()
    assert lib.gemm_f32(4, 4, 4, 1.0, None, 4, None, 3, 0.0, None, 4) == 1
    assert lib.gemm_f32(4, 5, 4, 1.0, None, 4, None, 5, 0.0, None, 4) == 1
    assert lib.gemm_f32(4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == 1   # null C
    h = ctypes.c_void_p()
    assert lib.gemm_plan_create(-3, 4, 4, 4, 4, 4, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_plan_create(4, 4, 4, 4, 4, 4, 2, 0, None) == 1
    assert lib.gemm_plan_execute(None, 1.0, None, None, 0.0, None, None) == 1
    assert lib.gemm_plan_create_config(4, 4, 4, 4, 4, 4, 2, -1, ctypes.byref(h)) == 1
    # empty problems are no-ops even without a device
    assert lib.gemm_f32(0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == 0
    assert lib.gemm_f32(4, 0, 4, 1.0, None, 4, None, 1, 0.0, None, 1) == 0


def test_split_pack_argument_checks():
    lib = pkg.load()
    assert lib.gemm_split_pack(1, 0, 4, 4, None, 4, None, 8, None, None) == 1   # SIMT mode
    assert lib.gemm_split_pack(2, 0, 4, 4, None, 3, None, 8, None, None) == 1   # ld < cols
    assert lib.gemm_split_pack(2, 0, 0, 4, None, 4, None, 8, None, None) == 0   # empty


def test_build_flags_target_sm103a():
    from paper_1804_10694_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_conv3x3_plan_argument_validation():
    """Rejected before any device work: channels not a multiple of 4,
    non-positive sizes, a SIMT mode, a packed configuration id where the
    packed convolution does not apply (C not a multiple of 16)."""
    import ctypes
    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.gemm_conv3x3_plan_create(1, 4, 4, 3, 8, 2, -1, ctypes.byref(h)) == 1
    assert lib.gemm_conv3x3_plan_create(0, 4, 4, 4, 8, 2, -1, ctypes.byref(h)) == 1
    assert lib.gemm_conv3x3_plan_create(1, 4, 4, 4, 8, 1, -1, ctypes.byref(h)) == 1
    packed = next(i for i in range(pkg.config_count("bf16x3")) if not pkg.config_get("bf16x3", i)["fused"])
    assert lib.gemm_conv3x3_plan_create(1, 4, 4, 4, 8, 2, packed, ctypes.byref(h)) == 1
    packed_tf32 = next(i for i in range(pkg.config_count("tf32x3")) if not pkg.config_get("tf32x3", i)["fused"])
    assert lib.gemm_conv3x3_plan_create(1, 4, 4, 24, 8, 3, packed_tf32, ctypes.byref(h)) == 1
    assert b"packed" in lib.gemm_last_error()
    # R x S filters: odd sizes 1..11 only; BF16X6 runs packed only (C % 16 == 0)
    for R, S in [(2, 3), (3, 4), (13, 3), (3, 13), (0, 1), (-1, 3)]:
        assert lib.gemm_conv_plan_create(1, 4, 4, 4, 8, R, S, 2, -1, ctypes.byref(h)) == 1, (R, S)
        assert b"filter" in lib.gemm_last_error()
    assert lib.gemm_conv_plan_create(1, 4, 4, 4, 8, 5, 5, 4, -1, ctypes.byref(h)) == 1


def test_transposed_arguments_validated_before_launch():
    import ctypes
    lib = pkg.load()
    h = ctypes.c_void_p()
    # transA: lda must cover M; transB: ldb must cover K (every mode, SIMT included)
    assert lib.gemm_plan_create_t(1, 0, 100, 50, 40, 99, 50, 50, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_plan_create_t(0, 1, 100, 50, 40, 40, 39, 50, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_plan_create_t(1, 1, 100, 50, 40, 99, 40, 50, 1, 0, ctypes.byref(h)) == 1
    assert lib.gemm_plan_create_t(1, 1, 100, 50, 40, 100, 39, 50, 1, 0, ctypes.byref(h)) == 1


def test_plan_options_validated_before_launch():
    """gemm_plan_create_opts: unknown option bits and bad shapes are rejected
    before any device work."""
    import ctypes
    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.gemm_plan_create_opts(64, 64, 64, 64, 64, 64, 2, 0, -1, 2, ctypes.byref(h)) == 1
    assert b"option" in lib.gemm_last_error()
    assert lib.gemm_plan_create_opts(64, 64, 64, 63, 64, 64, 2, 0, -1, 1, ctypes.byref(h)) == 1
    assert lib.gemm_plan_create_opts(64, 64, 64, 64, 64, 64, 2, 0, -1, 1, None) == 1
