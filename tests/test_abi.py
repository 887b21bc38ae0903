"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
entry point that include/countgauss.h declares, and validates arguments on the
host before launching anything."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1606_05732_gb300 import _lib
from paper_1606_05732_gb300 import build as cgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_symbols():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"^CG_API\s+[\w\s\*]+?\b(cg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    cgbuild.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ["cg_plan_create", "cg_plan_destroy", "cg_apply_csr", "cg_apply_dense", "cg_apply_adjoint",
                     "cg_plain_gaussian_apply", "cg_workspace_size", "cg_plan_check", "cg_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    bound = set(_lib.SIGNATURES) | {"cg_status_string"}
    assert set(declared_symbols()) <= bound | set(getattr(_lib, "EXTRA_SYMBOLS", ())), \
        set(declared_symbols()) - bound


def test_library_is_built_for_sm103a():
    obj = os.path.join(cgbuild.BUILD, "cg_sketch.o")
    assert "-gencode" in cgbuild.ARCH and "arch=compute_103a,code=sm_103a" in cgbuild.ARCH
    assert os.path.exists(obj)


def _plan(lib, n=100, d=4, m=8, B=16, seed=1):
    h = ctypes.c_void_p()
    st = lib.cg_plan_create(n, d, m, B, seed, ctypes.byref(h))
    return st, h


def test_plan_validation(lib):
    st, h = _plan(lib)
    assert st == 0 and h.value
    assert lib.cg_plan_destroy(h) == 0
    for bad in [(-1, 4, 8, 16), (10, 0, 8, 16), (10, 4, 0, 16), (10, 4, 8, 0), (10, 4, 8, 1 << 31),
                (10, 70000, 8, 16), ((1 << 31) - (1 << 20) + 1, 4, 8, 16)]:
        st, h = _plan(lib, *bad)
        assert st == 1 and not h.value


def test_options_and_workspace(lib):
    st, h = _plan(lib)
    val = ctypes.c_int64()
    assert lib.cg_plan_set_option(h, 1, 2) == 0
    assert lib.cg_plan_get_option(h, 1, ctypes.byref(val)) == 0 and val.value == 2
    assert lib.cg_plan_set_option(h, 1, 9) == 1
    assert lib.cg_plan_set_option(h, 99, 0) == 1
    assert lib.cg_plan_set_option(h, 3, 12345) == 0
    assert lib.cg_plan_get_option(h, 3, ctypes.byref(val)) == 0 and val.value == 12345
    for opt, good, bad in [(8, (0, 1, 16), (-1, 17)), (9, (0, 1, 32, 64, 128, 256), (2, 16, 33, 512, -32)),
                           (11, (0, 1, 2), (-1, 3)), (12, (0, 1), (-1, 2))]:
        for x in good:
            assert lib.cg_plan_set_option(h, opt, x) == 0
            assert lib.cg_plan_get_option(h, opt, ctypes.byref(val)) == 0 and val.value == x
        for x in bad:
            assert lib.cg_plan_set_option(h, opt, x) == 1
    sz = ctypes.c_size_t()
    for op in range(11):
        assert lib.cg_workspace_size(h, op, 1000, ctypes.byref(sz)) == 0
        assert sz.value >= 256 and sz.value % 256 == 0
    assert lib.cg_workspace_size(h, 42, 0, ctypes.byref(sz)) == 1
    lib.cg_plan_destroy(h)


def test_host_side_argument_errors_launch_nothing(lib):
    """Every one of these fails validation on the host, before any CUDA call."""
    st, h = _plan(lib)
    P = ctypes.c_void_p
    fake = P(1 << 20)  # never dereferenced: validation rejects the call first
    # null workspace
    assert lib.cg_apply_csr(h, fake, fake, fake, 10, fake, P(0), 0, P(0)) == 1
    # misaligned workspace
    assert lib.cg_apply_csr(h, fake, fake, fake, 10, fake, P((1 << 20) + 8), 1 << 20, P(0)) == 1
    # workspace too small
    assert lib.cg_apply_csr(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3
    # negative nnz, nnz >= 2^31
    assert lib.cg_apply_csr(h, fake, fake, fake, -1, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr(h, fake, fake, fake, 1 << 31, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr(h, fake, fake, fake, (1 << 31) - (1 << 20) + 1, fake, fake, 1 << 30, P(0)) == 1
    # null outputs / inputs
    assert lib.cg_apply_csr(h, fake, fake, fake, 10, P(0), fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr(h, P(0), fake, fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_dense(h, fake, 2, fake, fake, 1 << 30, P(0)) == 1  # ldx < d
    assert lib.cg_generate_words(1, 0, 0, -5, fake, P(0)) == 1
    assert lib.cg_generate_gaussian(1, 1, 8, 4, 2, 0, 3, fake, P(0)) == 1
    assert lib.cg_plan_check(None, fake, P(0)) == 1
    # the right projection: null Z, bad nnz, small workspace; deterministic mode unsupported
    assert lib.cg_apply_right_csr(h, fake, fake, fake, 10, P(0), fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_right_csr(h, fake, fake, fake, -3, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_right_csr(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3
    assert lib.cg_plan_set_option(h, 2, 1) == 0
    assert lib.cg_apply_right_csr(h, fake, fake, fake, 10, fake, fake, 1 << 30, P(0)) == 2
    # accumulating into SX is not offered with the deterministic (fixed-point) scatter
    assert lib.cg_plan_set_option(h, 12, 1) == 0
    assert lib.cg_sketch_csr(h, fake, fake, fake, 10, fake, fake, 1 << 30, P(0)) == 2
    lib.cg_plan_destroy(h)


def test_wide_offsets_argument_errors_launch_nothing(lib):
    """cg_apply_csr_i64 (64-bit row offsets): its host-side checks, before any CUDA call."""
    st, h = _plan(lib)
    P = ctypes.c_void_p
    fake = P(1 << 20)
    sz = ctypes.c_size_t()
    assert lib.cg_apply_csr_i64(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3  # workspace too small
    assert lib.cg_apply_csr_i64(h, fake, fake, fake, -1, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr_i64(h, fake, fake, fake, (1 << 40) + 1, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr_i64(h, P(0), fake, fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr_i64(h, P((1 << 20) + 4), fake, fake, 10, fake, fake, 1 << 30, P(0)) == 1  # 4-aligned
    assert lib.cg_apply_csr_i64(h, fake, P(0), fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_csr_i64(h, fake, fake, fake, 10, P(0), fake, 1 << 30, P(0)) == 1
    # the deterministic, partitioned and binned scatters take 32-bit offsets only
    for opt, val in ((2, 1), (7, 2), (7, 4)):
        assert lib.cg_plan_set_option(h, opt, val) == 0
        assert lib.cg_apply_csr_i64(h, fake, fake, fake, 10, fake, fake, 1 << 30, P(0)) == 2
        assert lib.cg_plan_set_option(h, opt, 0) == 0
    # the sketch alone: SX on a 16-byte boundary, the same option limits, a status word
    assert lib.cg_sketch_csr_i64(h, fake, fake, fake, 10, P((1 << 20) + 4), fake, 1 << 30, P(0)) == 1
    assert lib.cg_sketch_csr_i64(h, fake, fake, fake, 10, P(0), fake, 1 << 30, P(0)) == 1
    assert lib.cg_sketch_csr_i64(h, fake, fake, fake, -2, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_sketch_csr_i64(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3
    assert lib.cg_plan_set_option(h, 2, 1) == 0
    assert lib.cg_sketch_csr_i64(h, fake, fake, fake, 10, fake, fake, 1 << 30, P(0)) == 2
    assert lib.cg_plan_set_option(h, 2, 0) == 0
    assert lib.cg_workspace_size(h, 10, 1 << 35, ctypes.byref(sz)) == 0 and sz.value == 256
    # the adjoint at the stored entries: nnz range, null / misaligned pointers
    assert lib.cg_apply_adjoint_i64(h, fake, fake, fake, -1, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, fake, fake, fake, (1 << 40) + 1, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, fake, P(0), fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, fake, P((1 << 20) + 4), fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, fake, fake, fake, 10, P(0), fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, P(0), fake, fake, 10, fake, fake, 1 << 30, P(0)) == 1
    assert lib.cg_apply_adjoint_i64(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3
    # workspace: SX and the split-K partials, no scatter scratch (one-pass scatter), whatever nnz
    sz2 = ctypes.c_size_t()
    assert lib.cg_workspace_size(h, 9, 10, ctypes.byref(sz)) == 0
    assert lib.cg_workspace_size(h, 9, 1 << 33, ctypes.byref(sz2)) == 0
    assert sz.value == sz2.value >= 256 + 16 * 4 * 4
    # the deferred scatter (CG_OPT_SCATTER = 3) adds its 8-byte records, one slot per nonzero
    assert lib.cg_plan_set_option(h, 7, 3) == 0
    sz3, sz4 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.cg_workspace_size(h, 9, 1 << 33, ctypes.byref(sz3)) == 0
    assert lib.cg_workspace_size(h, 10, 1 << 33, ctypes.byref(sz4)) == 0
    assert sz3.value - sz2.value >= 8 << 33 and sz3.value - sz2.value < (8 << 33) + (1 << 20)
    assert sz4.value >= 256 + (8 << 33)
    assert lib.cg_apply_csr_i64(h, fake, fake, fake, 10, fake, fake, 16, P(0)) == 3
    assert lib.cg_plan_set_option(h, 7, 0) == 0
    lib.cg_plan_destroy(h)


def test_right_projection_workspace_holds_column_table(lib):
    """The right projection's workspace adds 4 bytes per column of A once the nonzeros
    hash every column more than four times on average (the per-column code table)."""
    n = 1000
    st, h = _plan(lib, n=n, d=300, m=128, B=640)
    sz = ctypes.c_size_t()
    sizes = {}
    for nnz in (0, 4 * n, 4 * n + 1):
        assert lib.cg_workspace_size(h, 8, nnz, ctypes.byref(sz)) == 0
        sizes[nnz] = sz.value
    assert sizes[0] == sizes[4 * n]
    assert sizes[4 * n + 1] - sizes[4 * n] >= 4 * n
    assert sizes[0] >= 256 + 640 * 300 * 4
    lib.cg_plan_destroy(h)


def test_status_strings(lib):
    for code in range(8):
        s = lib.cg_status_string(code).decode()
        assert s.startswith("CG_")


def test_c_program_uses_the_abi(lib, tmp_path):
    """A C99 program (tests/abi_smoke.c) compiles against include/countgauss.h with
    warnings as errors, links libcountgauss.so and runs its host-side calls."""
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = tmp_path / "abi_smoke"
    so_dir, so_name = os.path.split(_lib.library_path())
    assert so_name.startswith("lib") and so_name.endswith(".so")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_smoke.c"), "-L", so_dir, "-l" + so_name[3:-3],
                    "-Wl,-rpath," + so_dir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
