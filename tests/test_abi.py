"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/seg.h declares, sizes its buffers, and
rejects bad arguments before touching the device."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_11534_gb300 import seg
    return seg.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "seg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(seg_[a-z_]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "seg_solve" in names and "seg_build_domain" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1807_11534_gb300 import seg
    assert set(declared_symbols()) <= set(seg.SIGNATURES)


def test_sizes(lib):
    from paper_1807_11534_gb300 import seg
    assert seg.seg_version() >= 100
    small = seg.seg_workspace_bytes(64, 64, 64, 16)
    big = seg.seg_workspace_bytes(4096, 4096, 4096, 4)
    assert 0 < small < big
    assert seg.seg_state_bytes(100, 128, 0, seg.SEG_MODE_DENSE, 0) >= 6 * 4 * 100 * 128
    dense = seg.seg_state_bytes(100, 128, 0, seg.SEG_MODE_DENSE, 0)
    tiled = seg.seg_state_bytes(100, 128, 0, seg.SEG_MODE_TILED, 0)
    assert dense < tiled < dense + 8 * 100 * 128 + 65536
    s32 = seg.seg_state_bytes(100, 128, 5000, seg.SEG_MODE_COMPACT, seg.SEG_STORE_F32)
    s16 = seg.seg_state_bytes(100, 128, 5000, seg.SEG_MODE_COMPACT, seg.SEG_STORE_BF16)
    assert s32 >= 5000 * (6 * 4 + 8) and s16 >= 5000 * (6 * 2 + 8) and s16 < s32


def _err(lib):
    return lib.seg_last_error().decode()


def test_host_side_argument_errors(lib):
    """Bad sizes, pitches, parameters and NULLs fail before any device work."""
    from paper_1807_11534_gb300 import seg
    fake = 1 << 20          # never dereferenced: validation fails first
    ws_ok = 1 << 30
    st = lib.seg_make_fitting(None, 8, 8, 32, 0.3, 0.7, None, None, 0, 0.0, fake, None,
                              fake, ws_ok, None)
    assert st == seg.SEG_ERR_INVALID_ARG and "non-NULL" in _err(lib)
    st = lib.seg_make_fitting(fake, 8, 8, 33, 0.3, 0.7, None, None, 0, 0.0, fake, None,
                              fake, ws_ok, None)
    assert st == seg.SEG_ERR_ALIGN
    st = lib.seg_make_fitting(fake, 8, 40, 32, 0.3, 0.7, None, None, 0, 0.0, fake, None,
                              fake, ws_ok, None)
    assert st == seg.SEG_ERR_INVALID_ARG
    st = lib.seg_make_fitting(fake, 8, 8, 32, 0.3, 0.7, None, None, 3, 0.0, fake, None,
                              fake, ws_ok, None)
    assert st == seg.SEG_ERR_INVALID_ARG and "markers" in _err(lib)
    st = lib.seg_make_fitting(fake, 8, 8, 32, 0.3, 0.7, None, None, 0, 0.0, fake, None,
                              None, 0, None)
    assert st == seg.SEG_ERR_WORKSPACE
    # domain: tile height, q, workspace size
    args = [fake, 8, 8, 32, 0.1, -1.0, 12, fake, fake, fake, fake, 10, None, 0, fake, None,
            fake, ws_ok, None]
    assert lib.seg_build_domain(*args) == seg.SEG_ERR_INVALID_ARG
    args[6] = 16
    args[5] = 1.5
    assert lib.seg_build_domain(*args) == seg.SEG_ERR_INVALID_ARG
    args[5] = -1.0
    args[4] = math.nan
    assert lib.seg_build_domain(*args) == seg.SEG_ERR_INVALID_ARG
    args[4] = 0.1
    args[17] = 10
    assert lib.seg_build_domain(*args) == seg.SEG_ERR_WORKSPACE
    # solve: parameter checks
    prm = seg.make_params(1.0, iters=10, tile_h=16)
    sargs = [fake, 8, 8, 32, fake, fake, fake, fake, fake, ctypes.byref(prm), fake, fake, fake,
             fake, fake, 1 << 20, fake, fake, ws_ok, None]
    for field, bad in (("theta", 0.0), ("tau", -1.0), ("n_inner", 0), ("check_every", 0),
                       ("tile_h", 5), ("mode", 7), ("storage", 9)):
        p2 = seg.make_params(1.0, iters=10, tile_h=16)
        setattr(p2, field, bad)
        sargs[9] = ctypes.byref(p2)
        assert lib.seg_solve(*sargs) == seg.SEG_ERR_INVALID_ARG, field
    p3 = seg.make_params(1.0, iters=10, tile_h=16, mode="dense", storage="bf16")
    sargs[9] = ctypes.byref(p3)
    assert lib.seg_solve(*sargs) == seg.SEG_ERR_INVALID_ARG
    # temporally blocked mode: float32 only, sweep * n_inner <= 8, sweep >= 0
    for kw in (dict(storage="f16"), dict(sweep=9), dict(sweep=3, n_inner=3), dict(sweep=-1)):
        p4 = seg.make_params(1.0, iters=10, tile_h=16, mode="tiled", **kw)
        sargs[9] = ctypes.byref(p4)
        assert lib.seg_solve(*sargs) == seg.SEG_ERR_INVALID_ARG, kw
    sargs[9] = None
    assert lib.seg_solve(*sargs) == seg.SEG_ERR_INVALID_ARG
    # energy / errors
    assert lib.seg_energy(fake, 8, 8, 32, fake, fake, fake, fake, 1.0, 0.0, fake, fake, ws_ok,
                          None) == seg.SEG_ERR_INVALID_ARG
    assert lib.seg_errors(fake, None, 8, 8, 32, 0.5, fake, fake, ws_ok, None) == seg.SEG_ERR_INVALID_ARG


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes,
    imports or links the other."""
    bad_pkg = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#include\s+\"seg_oracle)|liboracle|seg_oracle\.",
                         re.M)
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_1807_11534_gb300")):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                assert not bad_pkg.search(open(os.path.join(dirpath, fn)).read()), fn
    bad_orc = re.compile(r"paper_1807_11534_gb300|#include\s+\"(seg|seg_internal)\.(h|cuh)\"|libseg")
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            assert not bad_orc.search(open(os.path.join(ROOT, "oracle", fn)).read()), fn


def test_host_side_argument_errors_of_the_next_rows(lib):
    """The robust restriction, the primal-dual solver, the volume solver and
    the Chan-Vese update reject bad arguments before any device work."""
    from paper_1807_11534_gb300 import seg
    fake = 1 << 20
    ws_ok = 1 << 30
    # robust domain: radius range, then the checks of seg_build_domain
    rargs = [fake, None, 8, 8, 32, 0.1, -1.0, 0, 16, fake, fake, fake, fake, 10, None, 0, fake, None,
             fake, ws_ok, None]
    for r in (-1, 33):
        rargs[7] = r
        assert lib.seg_build_domain_robust(*rargs) == seg.SEG_ERR_INVALID_ARG
    rargs[7] = 2
    rargs[8] = 12
    assert lib.seg_build_domain_robust(*rargs) == seg.SEG_ERR_INVALID_ARG
    # box mean: radius, aliasing, NULL, pitch
    assert lib.seg_box_mean(fake, 8, 8, 32, 17, fake + 4096, None) == seg.SEG_ERR_INVALID_ARG
    assert lib.seg_box_mean(fake, 8, 8, 32, 1, fake, None) == seg.SEG_ERR_INVALID_ARG
    assert lib.seg_box_mean(None, 8, 8, 32, 1, fake, None) == seg.SEG_ERR_INVALID_ARG
    assert lib.seg_box_mean(fake, 8, 8, 33, 1, fake + 4096, None) == seg.SEG_ERR_ALIGN
    # primal-dual parameters
    base = dict(sigma=seg.PD_STEP, tau=seg.PD_STEP, tol=0.0, iters=10, check_every=10, warm_start=0,
                tile_h=16)
    pargs = [fake, 8, 8, 32, fake, fake, fake, fake, None, fake, fake, fake, fake, 1 << 20, fake, fake,
             ws_ok, None]
    assert lib.seg_solve_pd(*pargs) == seg.SEG_ERR_INVALID_ARG
    for field, bad in (("sigma", 0.0), ("tau", -1.0), ("sigma", math.inf), ("check_every", 0),
                       ("iters", -1), ("tile_h", 5)):
        kw = dict(base)
        kw[field] = bad
        prm = seg.seg_pd_params(1.0, kw["sigma"], kw["tau"], kw["tol"], kw["iters"], kw["check_every"],
                                kw["warm_start"], kw["tile_h"])
        pargs[8] = ctypes.byref(prm)
        assert lib.seg_solve_pd(*pargs) == seg.SEG_ERR_INVALID_ARG, field
    prm = seg.seg_pd_params(1.0, seg.PD_STEP, seg.PD_STEP, 0.0, 10, 10, 0, 16)
    pargs[8] = ctypes.byref(prm)
    pargs[3] = 33
    assert lib.seg_solve_pd(*pargs) == seg.SEG_ERR_ALIGN
    # volumes: parameters, sizes, state alignment
    vargs = [fake, 4, 8, 8, 32, fake, fake, fake, fake, fake, None, fake, fake, fake, fake, fake, fake,
             1 << 20, fake, fake, ws_ok, None]
    for kw in (dict(n_inner=2), dict(storage="bf16"), dict(check_every=0), dict(tile_h=5)):
        p = dict(lam=1.0, theta=0.2, tau=0.125, iters=10, tol=0.0, n_inner=1, check_every=10,
                 warm_start=False, mode="compact", storage="f32", tile_h=16)
        p.update(kw)
        prm3 = seg.make_params(*p.values())
        vargs[10] = ctypes.byref(prm3)
        assert lib.seg_solve3d(*vargs) == seg.SEG_ERR_INVALID_ARG, kw
    prm3 = seg.make_params(1.0, iters=10, tile_h=16)
    vargs[10] = ctypes.byref(prm3)
    vargs[1] = 0
    assert lib.seg_solve3d(*vargs) == seg.SEG_ERR_INVALID_ARG
    vargs[1] = 4
    vargs[16] = fake + 16   # the state
    assert lib.seg_solve3d(*vargs) == seg.SEG_ERR_ALIGN
    # Chan-Vese update
    assert lib.seg_update_means(fake, fake, 8, 8, 32, math.nan, None, fake, ws_ok, None) == \
        seg.SEG_ERR_INVALID_ARG
    assert lib.seg_update_means(fake, None, 8, 8, 32, 0.5, None, fake, ws_ok, None) == seg.SEG_ERR_INVALID_ARG


def test_state_sizes_of_the_next_rows(lib):
    from paper_1807_11534_gb300 import seg
    a, b = seg.seg_state_bytes3d(1000), seg.seg_state_bytes3d(100000)
    assert a < b and b >= 100000 * 92
