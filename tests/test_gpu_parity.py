"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer / bit / index outputs are compared bit-exactly; floating point within
the tolerances the target sets: u within 1e-4 with float32 storage of the
iteration state, 1e-2 with 16-bit storage.  Sizes span several tiles with
ragged tails (H, W not multiples of the tile), plus the degenerate domains
(empty, full), and the full-size workloads through sampled crops.
"""
import math

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import bits_to_mask, require_gpu, run_gpu, seg_mod

pytestmark = pytest.mark.gpu

TOL_U32 = 1e-4
TOL_P32 = 2e-4
TOL_U16 = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _fitting_gpu(z, c1=0.3, c2=0.7, label=None, markers=None, gamma=0.0):
    seg = seg_mod()
    H, W = z.shape
    S = seg.Solver(H, W)
    zt = seg.upload(z)
    lt = seg.upload(label) if label is not None else None
    mt = torch.from_numpy(np.ascontiguousarray(markers, np.int32)).cuda() if markers is not None else None
    S.fitting(zt, c1, c2, lt, mt, gamma)
    torch.cuda.synchronize()
    return seg.download(S.f), S.c.cpu().numpy()


# ----------------------------------------------------------------- fitting

@pytest.mark.parametrize("shape", [(37, 70), (64, 64), (129, 97), (1, 33)])
def test_fitting_cv_bit_exact(orc, shape):
    rng = np.random.default_rng(sum(shape))
    z = rng.uniform(-0.5, 1.5, shape).astype(np.float32)
    f, _ = _fitting_gpu(z, 0.3, 0.7)
    _, f_o = orc.fitting(z, 0.3, 0.7)
    np.testing.assert_array_equal(f, f_o)


@pytest.mark.parametrize("m", [1, 20, 1500])
def test_fitting_ds_bit_exact(orc, m):
    rng = np.random.default_rng(m)
    H, W = 77, 150
    z = rng.uniform(0, 1, (H, W)).astype(np.float32)
    mk = np.stack([rng.integers(0, H, m), rng.integers(0, W, m)], 1).astype(np.int32)
    f, _ = _fitting_gpu(z, 0.25, 0.75, markers=mk, gamma=0.5)
    _, f_o = orc.fitting(z, 0.25, 0.75, mk, 0.5)
    np.testing.assert_array_equal(f, f_o)


@pytest.mark.parametrize("where", ["inside", "outside", "far"])
def test_fitting_ds_markers_in_and_out_of_the_image(orc, where):
    """Marker distances are exact integers: 32-bit with every marker inside
    the image (each pixel's nearest distance computed once and reused),
    64-bit when one lies outside, however far (the distance then exceeds
    2^31); bit-exact against the oracle either way."""
    rng = np.random.default_rng(7)
    H, W = 120, 257
    z = rng.uniform(0, 1, (H, W)).astype(np.float32)
    mk = np.stack([rng.integers(0, H, 12), rng.integers(0, W, 12)], 1).astype(np.int32)
    if where == "outside":
        mk[3] = (-5, W + 40)
    elif where == "far":
        mk[0] = (-2_000_000_000, 2_000_000_000)
    f, _ = _fitting_gpu(z, 0.25, 0.75, markers=mk, gamma=0.5)
    _, f_o = orc.fitting(z, 0.25, 0.75, mk, 0.5)
    np.testing.assert_array_equal(f, f_o)


def test_fitting_label_means(orc):
    P = synth.ellipses_ds(seed=3, H=300, W=333)
    f, c = _fitting_gpu(P.z, label=P.label, markers=P.markers, gamma=P.gamma)
    c1, c2 = orc.class_means(P.z, P.label)
    assert abs(c[0] - c1) <= 1e-12 * abs(c1) and abs(c[1] - c2) <= 1e-12 * abs(c2)
    _, f_o = orc.fitting(P.z, c[0], c[1], P.markers, P.gamma)   # same c: bit-exact
    np.testing.assert_array_equal(f, f_o)


# ------------------------------------------------------------------ domain

def _domain_gpu(f, delta=math.inf, q=-1.0, tile_h=16, tiles_cap=None):
    seg = seg_mod()
    H, W = f.shape
    S = seg.Solver(H, W, tile_h=tile_h)
    S.f[:, :W].copy_(torch.from_numpy(f))
    if tiles_cap is None:
        d = S.domain(delta=delta, q=q)
    else:
        d = seg.build_domain(S.f, delta, q, tile_h, S.ws)
        d.tiles = d.tiles[:tiles_cap].clone()
        seg.seg_build_domain(S.f, delta, q, tile_h, d.act, d.fg, d.wstart, d.tiles, d.pixels,
                             d.counts, d.delta, S.ws)
    torch.cuda.synchronize()
    return S, d


@pytest.mark.parametrize("shape,tile_h", [((37, 70), 8), ((64, 64), 16), ((129, 97), 4),
                                          ((200, 301), 32), ((5, 1), 16)])
@pytest.mark.parametrize("delta", [0.0, 0.05, 0.2, math.inf])
def test_domain_lists_bit_exact(orc, shape, tile_h, delta):
    rng = np.random.default_rng(shape[0] * 7 + tile_h)
    f = rng.normal(0, 0.2, shape).astype(np.float32)
    f[0, 0] = 0.0
    S, d = _domain_gpu(f, delta=delta, tile_h=tile_h)
    S.check_status()
    H, W = shape
    reg = orc.domain(f, delta)
    np.testing.assert_array_equal(bits_to_mask(d.act, W), reg == 2)
    np.testing.assert_array_equal(bits_to_mask(d.fg, W), f < 0)
    tl = orc.tile_list(reg, tile_h, 32)
    pl = orc.pixel_list_tiled(reg, tile_h, 32)
    cnt = d.counts.cpu().numpy()
    assert cnt[0] == len(tl) and cnt[1] == len(pl)
    assert cnt[2] == int(np.sum(reg == 1))
    np.testing.assert_array_equal(d.tiles.cpu().numpy()[:len(tl)], tl)
    np.testing.assert_array_equal(d.pixels.cpu().numpy()[:len(pl)], pl)
    # compact index of every RD pixel = its position in the tile-major list
    ws = d.wstart.cpu().numpy()
    act = d.act.cpu().numpy().view(np.uint32)
    ii, jj = pl // W, pl % W
    below = act[ii, jj // 32] & ((np.uint32(1) << (jj % 32).astype(np.uint32)) - np.uint32(1))
    popc = np.array([bin(int(x)).count("1") for x in below], np.int64)
    np.testing.assert_array_equal(ws[ii, jj // 32] + popc, np.arange(len(pl)))


@pytest.mark.parametrize("q", [0.0, 0.02, 0.17, 0.4, 0.999, 1.0])
def test_quantile_delta_bit_exact(orc, q):
    rng = np.random.default_rng(17)
    f = rng.normal(0, 0.3, (123, 257)).astype(np.float32)
    f[5, :40] = f[7, 7]   # ties
    S, d = _domain_gpu(f, q=q, tile_h=8)
    dl = float(d.delta.cpu().numpy()[0])
    assert np.float32(dl) == np.float32(orc.quantile_delta(f, q))
    reg = orc.domain(f, dl)
    assert d.counts.cpu().numpy()[1] == int(np.sum(reg == 2)) >= math.ceil(q * f.size)
    assert d.counts.cpu().numpy()[3] == min(math.ceil(q * f.size), f.size)


def test_domain_nonfinite_and_capacity():
    seg = seg_mod()
    f = np.random.default_rng(0).normal(0, 0.2, (40, 64)).astype(np.float32)
    f[3, 5] = np.nan
    S, d = _domain_gpu(f, delta=0.1)
    with pytest.raises(seg.SegError) as e:
        S.check_status()
    assert e.value.status == seg.SEG_ERR_NONFINITE
    f[3, 5] = 0.0
    S, d = _domain_gpu(f, delta=0.3, tile_h=8, tiles_cap=2)
    with pytest.raises(seg.SegError) as e:
        S.check_status()
    assert e.value.status == seg.SEG_ERR_CAPACITY


# ------------------------------------------------------------------- solve

def _cmp_state(out, st, tol_u, tol_p):
    du = np.max(np.abs(out["u"] - st.u))
    dv = np.max(np.abs(out["v"] - st.v))
    dp = max(np.max(np.abs(out["p1"] - st.p1)), np.max(np.abs(out["p2"] - st.p2)))
    assert du <= tol_u and dv <= tol_u and dp <= tol_p, (du, dv, dp)


def _problem(shape, seed=0):
    P = synth.small_example(seed=seed, H=shape[0], W=shape[1])
    return P


@pytest.mark.parametrize("mode", ["dense", "compact", "tiled"])
@pytest.mark.parametrize("delta", [0.05, 0.15, 0.25, math.inf])
@pytest.mark.parametrize("shape,tile_h", [((67, 131), 8), ((256, 256), 16), ((90, 45), 32),
                                          ((33, 200), 4), ((300, 29), 8), ((1, 97), 4)])
def test_solve_matches_oracle(orc, mode, delta, shape, tile_h):
    P = _problem(shape, seed=shape[1])
    _, f = orc.fitting(P.z, 0.3, 0.7)
    iters = 120
    out = run_gpu(f, delta=delta, lam=1.0, iters=iters, mode=mode, tile_h=tile_h)
    st = orc.solve(f, orc.domain(f, delta), 1.0, 0.2, 0.125, iters)
    _cmp_state(out, st, TOL_U32, TOL_P32)
    assert out["stats"][0] == iters
    # last stopping-test norms agree with the oracle's increments
    np.testing.assert_allclose(out["stats"][1:3], st.hist[-1], rtol=2e-3, atol=1e-5)


@pytest.mark.parametrize("mode", ["dense", "compact", "tiled"])
def test_solve_stops_like_the_oracle(orc, mode):
    P = _problem((96, 160), seed=4)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    tol = 1e-2
    out = run_gpu(f, delta=0.2, lam=1.0, iters=2000, tol=tol, check_every=1, mode=mode)
    st = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=2000, tol=tol)
    l_gpu, l_o = int(out["stats"][0]), st.iters_done
    crit = np.max(st.hist, axis=1) if st.hist.size else np.zeros(0)
    if l_gpu != l_o:
        # only a criterion within float32 rounding of tol may flip
        full = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=max(l_gpu, l_o))
        c = np.max(full.hist, axis=1)
        assert abs(l_gpu - l_o) == 1 and abs(c[min(l_gpu, l_o) - 1] - tol) < 1e-5 * tol
    else:
        _cmp_state(out, st, TOL_U32, TOL_P32)
    assert l_o < 2000 and crit[-1] <= tol


@pytest.mark.parametrize("mode", ["dense", "compact", "tiled"])
def test_inner_sweeps_and_warm_start(orc, mode):
    P = _problem((70, 100), seed=6)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, 0.2)
    out = run_gpu(f, delta=0.2, lam=2.0, iters=30, n_inner=3, mode=mode, tile_h=8,
                  sweep=2 if mode == "tiled" else 0)
    st = orc.solve(f, reg, 2.0, iters=30, n_inner=3)
    _cmp_state(out, st, TOL_U32, TOL_P32)
    # continue from the oracle state on the GPU: 25 more iterations
    out2 = run_gpu(f, delta=0.2, lam=2.0, iters=25, mode=mode, tile_h=8, warm=st)
    st2 = orc.solve(f, reg, 2.0, iters=25, state=st)
    _cmp_state(out2, st2, TOL_U32, TOL_P32)


@pytest.mark.parametrize("sweep,n_inner,check_every", [(1, 1, 7), (2, 1, 5), (3, 2, 10), (4, 1, 6),
                                                      (8, 1, 8), (5, 1, 100)])
@pytest.mark.parametrize("shape", [(200, 301), (61, 69), (123, 57)])
def test_tiled_sweeps_and_windows(orc, sweep, n_inner, check_every, shape):
    """Temporally blocked solve: several window rows and columns with ragged
    last windows, sweeps of 1 to 8 iterations, inner fixed-point sweeps, and
    stopping tests that split sweeps (check_every not a multiple of sweep)."""
    P = _problem(shape, seed=sum(shape))
    _, f = orc.fitting(P.z, 0.3, 0.7)
    iters = 47
    for delta in (0.2, math.inf):
        out = run_gpu(f, delta=delta, lam=1.2, iters=iters, n_inner=n_inner,
                      check_every=check_every, mode="tiled", sweep=sweep)
        st = orc.solve(f, orc.domain(f, delta), 1.2, 0.2, 0.125, iters, n_inner=n_inner)
        _cmp_state(out, st, TOL_U32, TOL_P32)
        assert out["stats"][0] == iters
        np.testing.assert_allclose(out["stats"][1:3], st.hist[-1], rtol=2e-3, atol=1e-5)


def test_tiled_rejects_bad_sweeps():
    seg = seg_mod()
    f = np.random.default_rng(3).normal(0, 0.2, (40, 40)).astype(np.float32)
    S = seg.Solver(40, 40, mode="tiled")
    S.f[:, :40].copy_(torch.from_numpy(f))
    S.domain(delta=0.2)
    for sweep, n_inner in ((9, 1), (3, 3)):
        with pytest.raises(seg.SegError) as e:
            S.solve(1.0, iters=5, n_inner=n_inner, sweep=sweep)
        assert e.value.status == seg.SEG_ERR_INVALID_ARG


def test_empty_and_full_domain_edges(orc):
    P = _problem((50, 70), seed=7)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    for mode in ("dense", "compact", "tiled"):
        out = run_gpu(f, delta=0.0, iters=10, tol=1e-9, check_every=1, mode=mode)
        h = (f < 0).astype(np.float64)
        np.testing.assert_array_equal(out["u"], h)
        np.testing.assert_array_equal(out["v"], h)
        assert not out["p1"].any() and not out["p2"].any()
        assert out["counts"][0] == 0 and out["stats"][0] == 1   # stops at the first check
    # a 1-row and a 1-column image, full domain
    for shape in ((1, 40), (40, 1)):
        rng = np.random.default_rng(1)
        f1 = rng.normal(0, 0.3, shape).astype(np.float32)
        for mode in ("dense", "compact", "tiled"):
            out = run_gpu(f1, iters=50, mode=mode, tile_h=4)
            st = orc.solve(f1, orc.domain(f1, math.inf), 1.0, iters=50)
            _cmp_state(out, st, TOL_U32, TOL_P32)


@pytest.mark.parametrize("q", [0.0005, 0.0015])
def test_fused_iteration_on_a_very_sparse_domain(orc, q):
    """At most one RD pixel per block (33 and 99 RD pixels of a 256 x 256
    image, 128 blocks): the compact solver takes its fused iteration (one
    phase per iteration, the dual steps of x - e1 and x - e2 redone by the
    thread of x), neither shared-memory path (stats[6] = stats[7] = 0)."""
    P = _problem((256, 256), seed=12)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = run_gpu(f, q=q, iters=80, mode="compact", tile_h=16)
    n = int(out["counts"][1])
    assert 0 < n <= 128
    assert out["stats"][6] == 0 and out["stats"][7] == 0
    st = orc.solve(f, orc.domain(f, out["delta"]), 1.0, iters=80)
    _cmp_state(out, st, TOL_U32, TOL_P32)


def test_compact_capacity_overflow_is_reported():
    seg = seg_mod()
    f = np.random.default_rng(2).normal(0, 0.2, (64, 64)).astype(np.float32)
    S = seg.Solver(64, 64, tile_h=16, mode="compact", capacity=10)
    S.f[:, :64].copy_(torch.from_numpy(f))
    S.domain(delta=0.2)
    S.solve(1.0, iters=5)
    with pytest.raises(seg.SegError) as e:
        S.check_status()
    assert e.value.status == seg.SEG_ERR_CAPACITY


BF16_FAILS = ("bf16 storage of p and v does not meet the 1e-2 bound on u in the max norm: "
              "8 significant bits, and its unbiased rounding noise accumulates in the slowly "
              "contracting modes of the iteration (max |u - u_oracle| about 2e-2 here)")


@pytest.mark.parametrize("storage", ["f16", pytest.param("bf16", marks=pytest.mark.xfail(
    strict=True, reason=BF16_FAILS))])
def test_16bit_storage(orc, storage):
    """p and v in 16 bits (stochastic rounding), float32 arithmetic, against
    the FP64 oracle: max |u - u_oracle| <= 1e-2 and the masks at 0.5 agree.
    fp16 (11 significant bits) meets it; bf16 does not (an expected failure,
    strict: the day it passes, the mark must go)."""
    P = _problem((128, 160), seed=8)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = run_gpu(f, delta=0.2, lam=1.0, iters=200, mode="compact", storage=storage)
    st = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=200)
    assert np.mean((out["u"] > 0.5) != (st.u > 0.5)) < 1e-3
    err = np.abs(out["u"] - st.u)
    assert err.max() <= TOL_U16, err.max()


def test_bf16_storage_mean_error_and_mask(orc):
    """What bf16 storage does meet against the oracle on the same problem:
    a small mean error and the same mask at 0.5 (its max-norm failure is the
    expected failure above)."""
    P = _problem((128, 160), seed=8)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = run_gpu(f, delta=0.2, lam=1.0, iters=200, mode="compact", storage="bf16")
    st = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=200)
    err = np.abs(out["u"] - st.u)
    assert err.mean() <= 1e-3, err.mean()
    assert np.mean((out["u"] > 0.5) != (st.u > 0.5)) < 1e-3
    assert out["v"].min() >= 0 and out["v"].max() <= 1


# ----------------------------------------------------------------- energies

def test_energy_and_errors_match_oracle(orc):
    seg = seg_mod()
    P = _problem((77, 101), seed=9)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = run_gpu(f, delta=0.2, lam=1.5, iters=80, mode="compact")
    S = out["solver"]
    e = S.energy(1.5, 0.2).cpu().numpy()
    eo = orc.energy(out["u"], out["v"], out["p1"], out["p2"], f, 1.5, 0.2)
    exp = np.array([eo["tv"], eo["ecr_u"], eo["ecr_v"], eo["edf"], eo["dual"], eo["gap"]])
    np.testing.assert_allclose(e, exp, rtol=1e-10, atol=1e-9)
    gt = run_gpu(f, lam=1.5, iters=300, mode="dense")
    S.errors(S.u, gt["solver"].u)
    got = S.err_out.cpu().numpy()
    e1, e2 = orc.errors(out["u"], gt["u"])
    assert got[0] == pytest.approx(e1, abs=1e-15) and got[1] == pytest.approx(e2, rel=1e-10)


# ------------------------------------------------------- full-size workloads

def _crop_check(orc, f_full, out_u, delta, lam, K, centres):
    H, W = f_full.shape
    R = 2 * K + 4
    worst = 0.0
    for (i, j) in centres:
        a, b = max(0, i - R), min(H, i + R + 1)
        c, d = max(0, j - R), min(W, j + R + 1)
        fc = np.ascontiguousarray(f_full[a:b, c:d])
        st = orc.solve(fc, orc.domain(fc, delta), lam, iters=K)
        worst = max(worst, abs(st.u[i - a, j - c] - out_u[i, j]))
    return worst


@pytest.mark.slow
@pytest.mark.parametrize("mode,delta", [("compact", 0.1), ("compact", 0.2), ("dense", 0.1), ("tiled", 0.1),
                                        ("tiled", 0.2)])
def test_full_size_2048_ds_sampled(orc, mode, delta):
    """2048x2048 distance-selective workload in the benchmark's launch
    configuration: K iterations on the GPU, then the oracle on crops of
    radius 2K+4 around sampled pixels (the iteration's domain of dependence
    grows by 2 pixels per iteration, so the crop centre is exact).  At
    delta = 0.1 (237K RD pixels) and 0.2 (863K, the benchmark's delta) the
    compact solver takes its one-barrier iteration with shared-memory state,
    a ring of recomputed border pixels, ghost words and the final write-back
    of pixels no other block reads."""
    seg = seg_mod()
    P = synth.ellipses_ds(seed=0, H=2048, W=2048)
    c1, c2 = orc.class_means(P.z, P.label)
    _, f = orc.fitting(P.z, c1, c2, P.markers, P.gamma)
    K, lam = 30, 2.0
    out = run_gpu(f, delta=delta, lam=lam, iters=K, mode=mode, tile_h=16)
    reg = orc.domain(f, delta)
    rng = np.random.default_rng(0)
    act = np.argwhere(reg == 2)
    pick = act[rng.choice(len(act), 32, replace=False)]
    centres = [tuple(x) for x in pick] + [(0, 0), (2047, 2047), (0, 1500), (2047, 3)]
    assert _crop_check(orc, f, out["u"], delta, lam, K, centres) <= TOL_U32
    # invariants over the whole image
    assert np.all(np.sqrt(out["p1"] ** 2 + out["p2"] ** 2) <= 1 + 1e-6)
    assert out["v"].min() >= 0 and out["v"].max() <= 1
    fixed = reg != 2
    np.testing.assert_array_equal(out["u"][fixed], (reg[fixed] == 1).astype(np.float64))


@pytest.mark.slow
@pytest.mark.parametrize("delta", [0.1, 0.2, 0.3, 0.5, math.inf])
def test_compact_matches_dense_on_the_whole_image(orc, delta):
    """Every pixel of the 2048x2048 workload: the compact solver (the
    one-barrier shared-memory iteration at delta = 0.1 and 0.2; the row-major
    solve beyond, with each block's neighbourhoods and theta lambda f in
    shared memory at 0.3, its neighbourhoods alone at 0.5 and on the full
    domain) against the dense solver run on the same restricted domain,
    itself checked against the oracle above; both are float32 iterations of
    the same steps."""
    P = synth.ellipses_ds(seed=0, H=2048, W=2048)
    c1, c2 = orc.class_means(P.z, P.label)
    _, f = orc.fitting(P.z, c1, c2, P.markers, P.gamma)
    K, lam = 40, 2.0
    oc = run_gpu(f, delta=delta, lam=lam, iters=K, mode="compact", tile_h=16)
    od = run_gpu(f, delta=delta, lam=lam, iters=K, mode="dense", tile_h=16)
    for k in ("u", "v", "p1", "p2"):
        assert np.max(np.abs(oc[k] - od[k])) <= TOL_U32, k
    np.testing.assert_allclose(oc["stats"][1:3], od["stats"][1:3], rtol=1e-3)


@pytest.mark.slow
@pytest.mark.parametrize("storage", ["f16", pytest.param("bf16", marks=pytest.mark.xfail(
    strict=True, reason=BF16_FAILS))])
def test_16bit_storage_on_the_shared_memory_path(orc, storage):
    """16-bit p, v on the benchmark image at its delta (0.2, the one-barrier
    iteration with shared-memory state) against the FP64 oracle on the whole
    image (OpenMP build when present)."""
    P = synth.ellipses_ds(seed=0, H=2048, W=2048)
    c1, c2 = orc.class_means(P.z, P.label)
    _, f = orc.fitting(P.z, c1, c2, P.markers, P.gamma)
    K, lam = 200, 2.0
    o16 = run_gpu(f, delta=0.2, lam=lam, iters=K, mode="compact", tile_h=16, storage=storage)
    st = orc.solve(f, orc.domain(f, 0.2), lam, iters=K, parallel=orc.has_omp())
    d = np.abs(o16["u"] - st.u)
    assert np.mean((o16["u"] > 0.5) != (st.u > 0.5)) <= 1e-3
    assert o16["v"].min() >= 0 and o16["v"].max() <= 1
    assert d.max() <= TOL_U16, d.max()


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["compact", "tiled"])
def test_largest_image_sampled(orc, mode):
    """A 16384 x 16384 image (268 M pixels; H * ld must stay below 2^31):
    random fitting term, delta = 0.1, 20 iterations, oracle crops around
    sampled RD pixels and the four corners."""
    seg = seg_mod()
    rng = np.random.default_rng(21)
    H = W = 16384
    f = rng.normal(0.0, 0.3, (H, W)).astype(np.float32)
    K, delta, lam = 20, 0.1, 1.0
    S = seg.Solver(H, W, tile_h=16, mode=mode)
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=delta)
    S.solve(lam, iters=K, check_every=K)
    torch.cuda.synchronize()
    S.check_status()
    inrd = np.abs(f) < np.float32(delta)
    assert int(S.dom.counts[1].item()) == int(np.count_nonzero(inrd))
    u = S.u[:, :W].cpu().numpy()      # float32, 1 GB
    del S
    act = np.argwhere(inrd)
    pick = act[rng.choice(len(act), 12, replace=False)]
    centres = [tuple(x) for x in pick] + [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0)]
    assert _crop_check(orc, f, u, delta, lam, K, centres) <= TOL_U32


@pytest.mark.slow
def test_full_size_4096_sampled(orc):
    """4096x4096 polygons at float32 storage, 20 iterations, against the
    oracle on crops (the 2000-iteration whole-image comparison is in
    test_gpu_fullsize.py)."""
    P = synth.polygons(seed=0)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    K, delta = 20, 0.1
    o32 = run_gpu(f, delta=delta, iters=K, mode="compact", storage="f32", tile_h=16)
    reg = orc.domain(f, delta)
    rng = np.random.default_rng(1)
    act = np.argwhere(reg == 2)
    centres = [tuple(x) for x in act[rng.choice(len(act), 8, replace=False)]]
    assert _crop_check(orc, f, o32["u"], delta, 1.0, K, centres) <= TOL_U32
