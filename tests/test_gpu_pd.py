"""Restricted primal-dual (Chambolle-Pock) solver of Eq. CR (seg_solve_pd)
against the FP64 oracle's solve_pd: small ragged images, restricted and full
domains, early stop, warm start, the full-size image through oracle crops,
and the argument and capacity errors."""
import math

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, seg_mod

pytestmark = pytest.mark.gpu

TOL_U, TOL_P = 1e-4, 2e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _run(f, lam, iters, delta=math.inf, q=-1.0, tile_h=16, tol=0.0, check_every=10, warm=None,
         mode="compact"):
    seg = seg_mod()
    H, W = f.shape
    S = seg.Solver(H, W, tile_h=tile_h, mode=mode)
    S.f[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(f)))
    S.domain(delta=delta, q=q)
    if warm is not None:
        for name in ("u", "p1", "p2"):
            getattr(S, name)[:, :W].copy_(torch.from_numpy(np.asarray(getattr(warm, name), np.float32)))
    S.solve_pd(lam, iters=iters, tol=tol, check_every=check_every, warm_start=warm is not None)
    torch.cuda.synchronize()
    S.check_status()
    out = {k: seg.download(getattr(S, k)).astype(np.float64) for k in ("u", "p1", "p2")}
    out["stats"] = S.stats.cpu().numpy()
    out["delta"] = float(S.dom.delta.cpu().numpy()[0])
    return out


def _cmp(out, st):
    du = np.max(np.abs(out["u"] - st.u))
    dp = max(np.max(np.abs(out["p1"] - st.p1)), np.max(np.abs(out["p2"] - st.p2)))
    assert du <= TOL_U and dp <= TOL_P, (du, dp)


@pytest.mark.parametrize("shape,tile_h", [((67, 131), 8), ((90, 45), 16), ((1, 97), 4), ((40, 1), 32),
                                          ((200, 301), 16)])
@pytest.mark.parametrize("dq", [dict(delta=math.inf), dict(delta=0.2), dict(q=0.3)])
def test_pd_matches_oracle(orc, shape, tile_h, dq):
    P = synth.small_example(seed=shape[0] + tile_h, H=shape[0], W=shape[1])
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = _run(f, 1.0, 150, tile_h=tile_h, **dq)
    st = orc.solve_pd(f, orc.domain(f, out["delta"]), 1.0, iters=150)
    _cmp(out, st)
    assert out["stats"][0] == 150


@pytest.mark.parametrize("lam", [0.7, 2.0])
def test_pd_noisy_image_matches_oracle(orc, lam):
    P = synth.noisy_example(seed=3, H=120, W=140)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = _run(f, lam, 300, q=0.4, tile_h=8)
    st = orc.solve_pd(f, orc.domain(f, out["delta"]), lam, iters=300)
    _cmp(out, st)


def test_pd_early_stop_and_warm_start(orc):
    P = synth.small_example(seed=9, H=96, W=120)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, 0.25)
    full = orc.solve_pd(f, reg, 1.0, iters=400)
    # the Section 4 test every 5 iterations; tol is put between the norms of
    # a check past iteration 100 that sets a new low by more than 5 % and
    # the lowest before it, so the stop iteration is far from a tie
    checks = np.max(full.hist, axis=1)[4::5]
    k = next(k for k in range(20, len(checks)) if checks[:k].min() > 1.05 * checks[k])
    tol = math.sqrt(checks[:k].min() * checks[k])
    stop = 5 * (k + 1)
    out = _run(f, 1.0, 400, delta=0.25, tol=tol, check_every=5)
    assert int(out["stats"][0]) == stop
    _cmp(out, orc.solve_pd(f, reg, 1.0, iters=stop))
    # warm start from the oracle's 60th iterate (ubar restarts at u, so this
    # is not the 120th cold iterate)
    a = orc.solve_pd(f, reg, 1.0, iters=60)
    out = _run(f, 1.0, 60, delta=0.25, warm=a)
    _cmp(out, orc.solve_pd(f, reg, 1.0, iters=60, state=a))


def test_pd_empty_domain_and_dense_solver_buffers(orc):
    f = np.random.default_rng(2).normal(0, 0.3, (33, 70)).astype(np.float32)
    out = _run(f, 1.0, 20, delta=0.0, mode="dense")   # the solver keeps its own compact state
    np.testing.assert_array_equal(out["u"], (f < 0).astype(np.float64))
    assert not out["p1"].any() and not out["p2"].any()


def test_pd_full_size_sampled(orc):
    """2048x2048 distance-selective image at delta = 0.2 (863K RD pixels):
    K iterations on the GPU, the oracle on crops of radius 2K+4 around
    sampled pixels (the domain of dependence grows by at most 2 pixels per
    iteration)."""
    P = synth.ellipses_ds(seed=0, H=2048, W=2048)
    c1, c2 = orc.class_means(P.z, P.label)
    _, f = orc.fitting(P.z, c1, c2, P.markers, P.gamma)
    K, lam, delta = 30, 2.0, 0.2
    out = _run(f, lam, K, delta=delta, tile_h=32)
    reg = orc.domain(f, delta)
    rng = np.random.default_rng(1)
    act = np.argwhere(reg == 2)
    centres = [tuple(x) for x in act[rng.choice(len(act), 24, replace=False)]] + [(0, 0), (2047, 2047)]
    R = 2 * K + 4
    worst = 0.0
    for (i, j) in centres:
        a, b = max(0, i - R), min(2048, i + R + 1)
        c, d = max(0, j - R), min(2048, j + R + 1)
        fc = np.ascontiguousarray(f[a:b, c:d])
        st = orc.solve_pd(fc, orc.domain(fc, delta), lam, iters=K)
        worst = max(worst, abs(st.u[i - a, j - c] - out["u"][i, j]))
    assert worst <= TOL_U
    assert np.all(np.hypot(out["p1"], out["p2"]) <= 1 + 1e-6)
    assert out["u"].min() >= 0 and out["u"].max() <= 1
    assert out["stats"][7] > 0   # the shared-memory, one-barrier iteration ran


def test_pd_argument_and_capacity_errors():
    seg = seg_mod()
    f = np.random.default_rng(0).normal(0, 0.3, (30, 40)).astype(np.float32)
    S = seg.Solver(30, 40, capacity=100)
    S.f[:, :40].copy_(torch.from_numpy(f))
    S.domain(delta=math.inf)
    for kw in (dict(sigma=0.0), dict(tau=-1.0), dict(sigma=math.inf), dict(check_every=0), dict(iters=-1)):
        with pytest.raises(seg.SegError) as e:
            S.solve_pd(1.0, **kw)
        assert e.value.status == seg.SEG_ERR_INVALID_ARG
    S.solve_pd(1.0, iters=10)   # 1200 RD pixels in a state for 100
    with pytest.raises(seg.SegError) as e:
        S.check_status()
    assert e.value.status == seg.SEG_ERR_CAPACITY


@pytest.mark.slow
def test_pd_largest_image_sampled(orc):
    """A 16384 x 16384 image (268 M pixels, H * ld just below 2^31) with the
    primal-dual solver: random fitting term, delta = 0.1, 12 iterations,
    oracle crops around sampled RD pixels and the corners."""
    seg = seg_mod()
    rng = np.random.default_rng(31)
    H = W = 16384
    f = rng.normal(0.0, 0.3, (H, W)).astype(np.float32)
    K, delta, lam = 12, 0.1, 1.0
    S = seg.Solver(H, W, tile_h=16, mode="compact")
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=delta)
    S.solve_pd(lam, iters=K, check_every=K)
    torch.cuda.synchronize()
    S.check_status()
    inrd = np.abs(f) < np.float32(delta)
    assert int(S.dom.counts[1].item()) == int(np.count_nonzero(inrd))
    u = S.u[:, :W].cpu().numpy()
    del S
    act = np.argwhere(inrd)
    centres = [tuple(x) for x in act[rng.choice(len(act), 10, replace=False)]]
    centres += [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0)]
    R = 2 * K + 4
    worst = 0.0
    for (i, j) in centres:
        a, b = max(0, i - R), min(H, i + R + 1)
        c, d = max(0, j - R), min(W, j + R + 1)
        fc = np.ascontiguousarray(f[a:b, c:d])
        st = orc.solve_pd(fc, orc.domain(fc, delta), lam, iters=K)
        worst = max(worst, abs(st.u[i - a, j - c] - u[i, j]))
    assert worst <= TOL_U
