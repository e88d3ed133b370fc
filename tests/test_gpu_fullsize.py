"""Parity at the benchmarked configurations, every pixel, at their own
iteration counts, against the FP64 oracle (its OpenMP build when the compiler
has one: the same bits as the serial build, on all cores):

 * the 2048 x 2048 distance-selective image (40 ellipses, 20 markers,
   gamma 0.5), lambda 2, 1000 iterations: the restricted solve at delta 0.2
   in the benchmark's launch configuration (compact, tile height 32) and
   the full-domain solve (dense, delta = inf) timed beside it;
 * the 4096 x 4096 polygon image (200 polygons, CV term), lambda 1, 2000
   iterations, delta 0.1 and inf, at float32 and 16-bit storage.

Bounds: u and v within 1e-4 at float32 storage, and theta div p (the part
of p that enters u = v - theta div p) within 2e-4; p itself is determined by
the method only up to divergence-free fields (they leave u unchanged, and
the iteration does not contract along them), so over thousands of float32
iterations its rounding drifts along them: p is compared element-wise in the
shorter parity tests, and here only its divergence plus |p| <= 1.  At 16-bit
storage, u within 1e-2: fp16 meets it on the restricted domain; fp16 on the
full domain and bf16 everywhere are expected failures of the max-norm bound
(measured: fp16 full domain 0.046 over the 16.7 M pixels), with their mean
error and mask agreement checked."""
import functools
import math

import numpy as np
import pytest

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, run_gpu, seg_mod

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_U32, TOL_P32, TOL_U16 = 1e-4, 2e-4, 1e-2
BF16_FAILS = ("bf16 storage does not meet the 1e-2 max-norm bound on u (8 significant bits; "
              "the rounding noise accumulates in slowly contracting modes)")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


@functools.lru_cache(maxsize=None)
def _ds2048():
    import oracle
    P = synth.ellipses_ds(seed=0, H=2048, W=2048)
    c1, c2 = oracle.class_means(P.z, P.label)
    _, f = oracle.fitting(P.z, c1, c2, P.markers, P.gamma)
    return f


@functools.lru_cache(maxsize=None)
def _poly4096():
    import oracle
    P = synth.polygons(seed=0)
    _, f = oracle.fitting(P.z, 0.3, 0.7)
    return f


@functools.lru_cache(maxsize=None)
def _oracle_solve(which, delta, lam, iters):
    import oracle
    f = _ds2048() if which == "ds2048" else _poly4096()
    st = oracle.solve(f, oracle.domain(f, delta), lam, iters=iters, parallel=oracle.has_omp())
    return st


def _div(p1, p2):
    """Chambolle's divergence (minus the adjoint of the forward difference)."""
    d = np.zeros_like(p1)
    d[:-1, :] += p1[:-1, :]; d[1:, :] -= p1[:-1, :]
    d[:, :-1] += p2[:, :-1]; d[:, 1:] -= p2[:, :-1]
    return d


def _cmp32(out, st, theta=0.2):
    for k in ("u", "v"):
        d = np.max(np.abs(out[k] - getattr(st, k)))
        assert d <= TOL_U32, (k, d)
    d = theta * np.max(np.abs(_div(out["p1"], out["p2"]) - _div(st.p1, st.p2)))
    assert d <= TOL_P32, ("theta div p", d)
    # |p| <= 1 holds exactly in exact arithmetic; each float32 step (hardware
    # reciprocal square root and fast divide, a few ulp) can leave |p| a few
    # ulp above 1, and where |g| is near 0 the step barely contracts that
    # excess, so it random-walks: about sqrt(K) x 1e-7 after K iterations
    assert np.sqrt(np.max(out["p1"] ** 2 + out["p2"] ** 2)) <= 1 + 1e-4


@pytest.mark.parametrize("mode,delta,tile_h", [("compact", 0.2, 32), ("dense", math.inf, 32)])
def test_benchmark_image_at_1000_iterations(orc, mode, delta, tile_h):
    f = _ds2048()
    out = run_gpu(f, delta=delta, lam=2.0, iters=1000, mode=mode, tile_h=tile_h)
    st = _oracle_solve("ds2048", delta, 2.0, 1000)
    _cmp32(out, st)
    assert out["stats"][0] == 1000


@pytest.mark.parametrize("delta", [0.1, math.inf])
def test_polygons_4096_at_2000_iterations_float32(orc, delta):
    f = _poly4096()
    out = run_gpu(f, delta=delta, lam=1.0, iters=2000, mode="compact", tile_h=16)
    _cmp32(out, _oracle_solve("poly4096", delta, 1.0, 2000))


F16_FULL_FAILS = ("fp16 storage on the full 4096^2 domain does not meet the 1e-2 max-norm bound on u "
                  "after 2000 iterations (measured 0.046 at the worst of 16.7 M pixels)")


@pytest.mark.parametrize("delta,storage", [
    (0.1, "f16"),
    pytest.param(math.inf, "f16", marks=pytest.mark.xfail(strict=True, reason=F16_FULL_FAILS)),
    pytest.param(0.1, "bf16", marks=pytest.mark.xfail(strict=True, reason=BF16_FAILS)),
    pytest.param(math.inf, "bf16", marks=pytest.mark.xfail(strict=True, reason=BF16_FAILS))])
def test_polygons_4096_at_2000_iterations_16bit(orc, delta, storage):
    f = _poly4096()
    out = run_gpu(f, delta=delta, lam=1.0, iters=2000, mode="compact", tile_h=16, storage=storage)
    st = _oracle_solve("poly4096", delta, 1.0, 2000)
    assert np.mean((out["u"] > 0.5) != (st.u > 0.5)) <= 1e-4
    d = np.abs(out["u"] - st.u)
    assert d.max() <= TOL_U16, d.max()


@pytest.mark.parametrize("delta,storage", [(math.inf, "f16"), (0.1, "bf16"), (math.inf, "bf16")])
def test_polygons_4096_16bit_mean_error_and_mask(orc, delta, storage):
    f = _poly4096()
    out = run_gpu(f, delta=delta, lam=1.0, iters=2000, mode="compact", tile_h=16, storage=storage)
    st = _oracle_solve("poly4096", delta, 1.0, 2000)
    d = np.abs(out["u"] - st.u)
    assert d.mean() <= 1e-3, d.mean()
    assert np.mean((out["u"] > 0.5) != (st.u > 0.5)) <= 1e-4


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_polygons_4096_stopping_test_on_the_row_major_path(orc, storage):
    """The 4096^2 image at delta 0.1 (an RD beyond the shared-memory paths:
    the row-major solve, whose barriers are split around each block's
    interior pixels) with the Section 4 stopping test: a solve stopped by
    tol gives the bits of the same solve run for exactly that many
    iterations without a test, and the test's rule holds at the stop."""
    f = _poly4096()
    base = run_gpu(f, delta=0.1, lam=1.0, iters=300, check_every=10, storage=storage)
    # a tolerance the increments cross between iterations 10 and 300
    tol = 1.5 * max(base["stats"][1], base["stats"][2])
    a = run_gpu(f, delta=0.1, lam=1.0, iters=300, tol=tol, check_every=10, storage=storage)
    n = int(a["stats"][0])
    assert 10 <= n < 300 and n % 10 == 0, n
    assert max(a["stats"][1], a["stats"][2]) <= tol
    b = run_gpu(f, delta=0.1, lam=1.0, iters=n, check_every=10, storage=storage)
    for k in ("u", "v", "p1", "p2"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("which,delta", [("ds2048", 0.3), ("ds2048", 0.5), ("poly4096", math.inf)])
def test_warm_start_on_the_row_major_path(orc, which, delta):
    """Warm start on the row-major solve (the 2048^2 image at delta 0.3: each
    block's neighbourhoods and theta lambda f in shared memory; at 0.5: its
    neighbourhoods alone; the 4096^2 full domain: the launch without shared
    memory): 20 iterations, then 20 more from the returned state, against 40
    cold iterations."""
    import torch
    seg = seg_mod()
    f = _ds2048() if which == "ds2048" else _poly4096()
    H, W = f.shape
    S = seg.Solver(H, W, tile_h=32 if which == "ds2048" else 16, mode="compact")
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=delta)
    lam = 2.0 if which == "ds2048" else 1.0

    def state():
        torch.cuda.synchronize()
        S.check_status()
        return {k: seg.download(getattr(S, k)).astype(np.float64) for k in ("u", "v", "p1", "p2")}

    S.solve(lam, iters=40)
    cold = state()
    S.solve(lam, iters=20)
    S.solve(lam, iters=20, warm_start=True)
    warm = state()
    for k in cold:
        assert np.max(np.abs(warm[k] - cold[k])) <= 1e-5, k
