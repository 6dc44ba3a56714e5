"""The C-ABI library loads on a machine without a GPU and exports every
function its headers declare (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1703_00186_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_headers_declare_the_core_calls():
    names = declared_functions()
    for n in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_adjoint_step",
              "lbm_propagate_bc", "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_no_undeclared_entry_point(lib):
    # every exported lbm_* function is declared (and so documented) in include/
    import shutil
    import subprocess
    from paper_1703_00186_gb300 import _lib as L
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if ln.split() and ln.split()[-1].startswith("lbm_")}
    assert exported, "no lbm_* symbols found"
    assert exported <= declared_functions(), sorted(exported - declared_functions())


def test_state_bytes_and_argument_checks_need_no_gpu(lib):
    from paper_1703_00186_gb300 import _lib as L
    p = L.LbmParams(64, 128, L.LBM_FP64, 0, 0.8, 1e-4, 0.5, 1.5, 1.0)
    assert lib.lbm_state_bytes(ctypes.byref(p)) == 37 * 134 * 64 * 8
    p32 = L.LbmParams(64, 128, L.LBM_FP32_SHIFTED, 0, 0.8, 1e-4, 0.5, 1.5, 1.0)
    assert lib.lbm_state_bytes(ctypes.byref(p32)) == 37 * 134 * 64 * 4
    bad = L.LbmParams(2, 128, L.LBM_FP64, 0, 0.8, 0.0, 1.0, 1.0, 1.0)
    assert lib.lbm_state_bytes(ctypes.byref(bad)) == 0
    ctx = ctypes.c_void_p()
    # rejected before any device work: too small, tau <= 0.5, NULL buffers, size mismatch
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(bad), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          0, None) == L.LBM_ERR_INVALID
    badtau = L.LbmParams(64, 128, L.LBM_FP64, 0, 0.5, 0.0, 1.0, 1.0, 1.0)
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(badtau), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          37 * 134 * 64 * 8, None) == L.LBM_ERR_INVALID
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(p), None, None, 0, None) == L.LBM_ERR_INVALID
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(p), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          12345, None) == L.LBM_ERR_SIZE
    assert not ctx.value
    assert lib.lbm_step(None, 1) == L.LBM_ERR_INVALID
    assert lib.lbm_step_path(None) == L.LBM_ERR_INVALID


def test_regularized_flag_only_with_fp64(lib):
    from paper_1703_00186_gb300 import _lib as L
    ctx = ctypes.c_void_p()
    p = L.LbmParams(64, 128, L.LBM_FP32_SHIFTED, L.LBM_FLAG_REGULARIZED, 0.8, 0.0, 1.0, 1.0, 1.0)
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(p), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          lib.lbm_state_bytes(ctypes.byref(p)), None) == L.LBM_ERR_INVALID
    bad = L.LbmParams(64, 128, L.LBM_FP64, 32, 0.8, 0.0, 1.0, 1.0, 1.0)   # unknown flag bit
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(bad), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          lib.lbm_state_bytes(ctypes.byref(bad)), None) == L.LBM_ERR_INVALID


def test_fp32_arith_flags_one_at_a_time_and_fp32_only(lib):
    from paper_1703_00186_gb300 import _lib as L
    terms, coll = L.LBM_FLAG_FP32_F64_TERMS, L.LBM_FLAG_FP32_F64_COLLIDE
    for prec, flags, rc in ((L.LBM_FP32_SHIFTED, terms, L.LBM_OK), (L.LBM_FP32_SHIFTED, coll, L.LBM_OK),
                            (L.LBM_FP32_SHIFTED, terms | coll, L.LBM_ERR_INVALID),
                            (L.LBM_FP64, terms, L.LBM_ERR_INVALID), (L.LBM_FP64_DF, coll, L.LBM_ERR_INVALID)):
        p = L.LbmParams(64, 128, prec, flags, 0.8, 1e-5, 0.9, 1.1, 1.0)
        assert lib.lbm_model_constants(ctypes.byref(p), None, None, None, None) == rc, (prec, flags)


def test_oversized_lattices_are_refused(lib):
    from paper_1703_00186_gb300 import _lib as L
    ctx = ctypes.c_void_p()
    tall = L.LbmParams(8, 4 * 65535 + 1, L.LBM_FP64, 0, 0.8, 0.0, 1.0, 1.0, 1.0)
    assert lib.lbm_create(ctypes.byref(ctx), ctypes.byref(tall), ctypes.c_void_p(8), ctypes.c_void_p(16),
                          lib.lbm_state_bytes(ctypes.byref(tall)), None) == L.LBM_ERR_INVALID


def test_host_constants_match_the_oracle_bit_for_bit(lib):
    # The library's host-side derivations (the quadrature solved by Newton in
    # double-double, the wall ratios) against the oracle's 60-digit solve,
    # rounded once to float64 on both sides: equal bit for bit.
    import numpy as np
    from oracle import lattice, model as M
    from paper_1703_00186_gb300 import _lib as L
    K = lattice.constants()
    for t_top, t_bottom in ((0.5, 1.5), (1.0, 1.0), (0.75, 1.25), (1.3, 0.6)):
        p = L.LbmParams(16, 12, L.LBM_FP64, 0, 0.8, 1e-4, t_top, t_bottom, 1.0)
        r = ctypes.c_double()
        w, qb, qt = [(ctypes.c_double * 37)() for _ in range(3)]
        assert lib.lbm_model_constants(ctypes.byref(p), ctypes.byref(r), w, qb, qt) == L.LBM_OK
        assert r.value == K["r"]
        np.testing.assert_array_equal(np.array(w[:]), K["w"])
        np.testing.assert_array_equal(np.array(qb[:]), M.wall_q(t_bottom, "bottom"))
        np.testing.assert_array_equal(np.array(qt[:]), M.wall_q(t_top, "top"))
    bad = L.LbmParams(16, 12, L.LBM_FP64, 0, 0.5, 0.0, 1.0, 1.0, 1.0)
    assert lib.lbm_model_constants(ctypes.byref(bad), None, None, None, None) == L.LBM_ERR_INVALID
    assert lib.lbm_model_constants(None, None, None, None, None) == L.LBM_ERR_INVALID
