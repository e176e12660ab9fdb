"""CPU-only checks of the C ABI library: it loads, exports every function that
include/gsvd.h declares, and rejects bad arguments before any launch."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_00101_gb300.build import build
    build()
    import paper_1909_00101_gb300 as hz
    return hz.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsvd_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gsvd_create", "gsvd_destroy", "gsvd_solve", "gsvd_solve_batched", "gsvd_submit", "gsvd_poll"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1909_00101_gb300 as hz
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(hz.ENTRY_POINTS) <= set(declared_functions())


def test_config_defaults(lib):
    import paper_1909_00101_gb300 as hz
    c = hz.Config()
    lib.gsvd_config_default(ctypes.byref(c))
    assert c.max_sweeps == 30 and c.inner_max_sweeps == 30 and c.criterion == 1 and c.sort == 1
    assert c.hbm_budget_bytes == 60 << 30 and c.precision == 0
    assert c.shorten == 1 and c.fp32_params == 1 and c.inner_max_sweeps_fp32 == 1
    assert c.fp64_gemm == 1 and c.fp32_stop_permille == 50 and c.variant == 0
    # the binding's Config mirrors the C struct: variant is its last field
    # (the struct is padded to 8 bytes by its uint64 member)
    assert ctypes.sizeof(hz.Config) == (hz.Config.variant.offset + 4 + 7) // 8 * 8


def test_strerror(lib):
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.gsvd_strerror(s)
    assert lib.gsvd_strerror(-99) == b"unknown status"


def test_invalid_problems_rejected_before_any_launch(lib):
    import paper_1909_00101_gb300 as hz
    h = ctypes.c_void_p()
    cfg = hz.make_config()
    assert lib.gsvd_create(ctypes.byref(h), ctypes.byref(cfg), None) == 0
    F = np.zeros((3, 4), order="F")
    G = np.zeros((5, 4), order="F")
    Z = np.zeros((4, 4), order="F")
    v = np.zeros(4)
    p = hz._problem(F, G, Z, v, v, v, False)        # m_F < n
    info = hz.Info()
    assert lib.gsvd_solve(h, ctypes.byref(p), ctypes.byref(info)) == hz.EINVAL
    p.m_f = 6
    p.ldf = 2                                        # ld < m
    assert lib.gsvd_solve(h, ctypes.byref(p), ctypes.byref(info)) == hz.EINVAL
    p.ldf = 6
    p.dtype = 7                                      # bad dtype
    assert lib.gsvd_solve(h, ctypes.byref(p), ctypes.byref(info)) == hz.EINVAL
    assert lib.gsvd_solve(h, None, ctypes.byref(info)) == hz.EINVAL
    p.dtype = 0
    p.n = 0                                          # empty problem
    assert lib.gsvd_solve(h, ctypes.byref(p), ctypes.byref(info)) == hz.EINVAL
    p.n = 4
    assert lib.gsvd_solve_batched(h, None, -1, None) == hz.EINVAL
    # the autotuner checks its arguments before touching the GPU
    w = ctypes.c_int32(-1)
    assert lib.gsvd_autotune(h, 0, ctypes.c_int64(100), ctypes.c_int64(100), ctypes.c_int64(0), ctypes.byref(w)) == hz.EINVAL
    assert lib.gsvd_autotune(h, 0, ctypes.c_int64(10), ctypes.c_int64(100), ctypes.c_int64(64), ctypes.byref(w)) == hz.EINVAL
    assert lib.gsvd_autotune(h, 5, ctypes.c_int64(100), ctypes.c_int64(100), ctypes.c_int64(64), ctypes.byref(w)) == hz.EINVAL
    assert lib.gsvd_autotune(h, 0, ctypes.c_int64(100), ctypes.c_int64(100), ctypes.c_int64(64), None) == hz.EINVAL
    # a class that runs on the pointwise kernel has nothing to tune
    assert lib.gsvd_autotune(h, 0, ctypes.c_int64(100), ctypes.c_int64(100), ctypes.c_int64(32), ctypes.byref(w)) == 0
    assert w.value == 0
    # right vectors: ld >= n
    X = np.zeros((4, 4), order="F")
    p.X, p.ldx = X.ctypes.data, 3
    assert lib.gsvd_solve(h, ctypes.byref(p), ctypes.byref(info)) == hz.EINVAL
    assert info.status == hz.EINVAL
    assert lib.gsvd_destroy(h) == 0
    # a negative timeout is refused at creation
    c = hz.Config()
    lib.gsvd_config_default(ctypes.byref(c))
    c.timeout_ms = -1
    h2 = ctypes.c_void_p()
    assert lib.gsvd_create(ctypes.byref(h2), ctypes.byref(c), None) == hz.EINVAL


def test_bad_config_rejected(lib):
    import paper_1909_00101_gb300 as hz
    h = ctypes.c_void_p()
    for field, val in (("criterion", 3), ("max_sweeps", 0), ("inner_max_sweeps", 0), ("precision", 5),
                       ("variant", 4), ("variant", -1)):
        cfg = hz.make_config()
        setattr(cfg, field, val)
        assert lib.gsvd_create(ctypes.byref(h), ctypes.byref(cfg), None) == hz.EINVAL


def test_workspace_bytes_grows_with_size(lib):
    import paper_1909_00101_gb300 as hz
    cfg = hz.make_config(path="blocked", shorten=0)
    a = lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 512, 512, 256)
    b = lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 4096, 4096, 2048)
    c = lib.gsvd_workspace_bytes(ctypes.byref(cfg), 1, 4096, 4096, 2048)
    assert 0 < a < b < c
    mixed = hz.make_config(path="blocked", precision="mixed", shorten=0)
    assert lib.gsvd_workspace_bytes(ctypes.byref(mixed), 0, 4096, 4096, 2048) > b
    # QR shortening (real, tall): the n x n sub-problem's workspace plus
    # R_F, R_G, R1_F, R1_G (n^2 each) and a max(m_F, m_G) x n product buffer,
    # plus (fp64_gemm = 1) the BF16 digit planes of the largest product:
    # 8 digits x 2 bytes for both n x m operands of the Gram F^T F
    sh = hz.make_config(path="blocked", shorten=1, fp64_gemm=0)
    n, m = 2048, 4096
    sub = lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, n, n, n)
    got = lib.gsvd_workspace_bytes(ctypes.byref(sh), 0, m, m, n)
    assert got >= sub + 8 * (4 * n * n + m * n) and got <= sub + 8 * (4 * n * n + m * n) + 1024
    shoz = hz.make_config(path="blocked", shorten=1, fp64_gemm=1)
    got_oz = lib.gsvd_workspace_bytes(ctypes.byref(shoz), 0, m, m, n)
    planes = 2 * 8 * 2 * n * m
    assert planes <= got_oz - got <= planes + 65536  # + the per-row scale exponents
    # complex problems are not shortened
    assert lib.gsvd_workspace_bytes(ctypes.byref(sh), 1, m, m, n) == c
    # very tall pairs: the Grams are summed in pieces of at most 65536 rows,
    # so the planes are those of the m x n x n products (8 digits x 2 bytes
    # of the m x n operand and of the n x n one), not of the m-row Gram
    # (+ one scale exponent per row of both operands)
    n, m = 256, 200000
    base = lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, n, n, n) + 8 * (4 * n * n + m * n)
    extra = lib.gsvd_workspace_bytes(ctypes.byref(shoz), 0, m, m, n) - base
    prod = 16 * m * n + 16 * n * n
    assert prod <= extra <= prod + 4 * (m + n) + 2048 and extra < 2 * 8 * 2 * n * m


def test_size_limits_of_the_header(lib):
    """gsvd.h: n < 4 runs on the pointwise kernel, whose shared memory holds
    the whole problem; a tall problem with n < 4 has no plan (workspace 0,
    the solve returns EINVAL), a short one does."""
    import paper_1909_00101_gb300 as hz
    cfg = hz.make_config()
    assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 100, 100, 2) > 0
    assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 100000, 100000, 2) == 0
    assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 100000, 100000, 4) > 0
    assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 40000, 40000, 32769) == 0


def test_variants_plan_where_the_pivot_step_has_them(lib):
    """Variants 1-3 of Sec. 2.6 (enhanced dots, D-hat rescaling) have a plan on
    the pointwise kernel and on the blocked path with real-view width V <= 32
    (the two-CTA FP64 pivot step); none with V = 64 (w = 32, real)."""
    import paper_1909_00101_gb300 as hz
    for v in (1, 2, 3):
        cfg = hz.make_config(variant=v)
        assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 64, 48, 32) > 0
        assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 1, 48, 40, 24) > 0
        assert lib.gsvd_workspace_bytes(ctypes.byref(cfg), 0, 4096, 4096, 2048) > 0
        blk = hz.make_config(variant=v, path="blocked")
        assert lib.gsvd_workspace_bytes(ctypes.byref(blk), 0, 64, 48, 32) > 0
        wide = hz.make_config(variant=v, path="blocked", block_w=32)
        assert lib.gsvd_workspace_bytes(ctypes.byref(wide), 0, 300, 300, 128) == 0


def test_binding_structs_match_the_header(tmp_path):
    """Sizes and field offsets of gsvd_config, gsvd_problem and gsvd_info as
    compiled from include/gsvd.h equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    import paper_1909_00101_gb300 as hz
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsvd.h"', "int main(void) {"]
    checks = []
    for cname, cls in (("gsvd_config", hz.Config), ("gsvd_problem", hz.Problem), ("gsvd_info", hz.Info)):
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        checks.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            checks.append(getattr(cls, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.check_call(["gcc", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == checks
