"""Parity of the batched compact solve (seg_solve_batch: many images of uneven
size and per-image lambda / restricted fraction in one persistent launch)
with the FP64 oracle run on each image on its own."""
import math

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, seg_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _batch(orc, shapes, lams, qs, iters, storage="f32", tile_h=16, capacity=None, tol=0.0,
           check_every=10):
    seg = seg_mod()
    B = seg.BatchSolver(shapes, tile_h=tile_h, storage=storage, capacity=capacity)
    fs = []
    for k, ((H, W), S) in enumerate(zip(shapes, B.solvers)):
        P = synth.small_example(seed=100 + k, H=H, W=W)
        _, f = orc.fitting(P.z, 0.3, 0.7)
        fs.append(f)
        S.f[:, :W].copy_(torch.from_numpy(f))
        S.domain(q=qs[k])
    B.solve(lams, iters=iters, tol=tol, check_every=check_every)
    torch.cuda.synchronize()
    return B, fs


def test_batch_matches_oracle_per_image(orc):
    shapes = [(67, 131), (90, 45), (33, 200), (128, 128), (1, 97), (200, 61)]
    lams = [1.0, 0.5, 2.0, 1.5, 1.0, 3.0]
    qs = [0.1, 0.3, 0.05, 0.4, 0.5, 0.2]
    iters = 100
    B, fs = _batch(orc, shapes, lams, qs, iters)
    B.check_status()
    seg = seg_mod()
    total = 0
    for k, S in enumerate(B.solvers):
        delta = float(S.dom.delta.cpu().numpy()[0])
        assert np.float32(delta) == np.float32(orc.quantile_delta(fs[k], qs[k]))
        reg = orc.domain(fs[k], delta)
        total += int(np.sum(reg == 2))
        st = orc.solve(fs[k], reg, lams[k], 0.2, 0.125, iters)
        for name, ref in (("u", st.u), ("v", st.v), ("p1", st.p1), ("p2", st.p2)):
            got = seg.download(getattr(S, name)).astype(np.float64)
            err = np.max(np.abs(got - ref))
            assert err <= (1e-4 if name in ("u", "v") else 2e-4), (k, name, err)
    stats = B.stats.cpu().numpy()
    assert stats[0] == iters and stats[3] == total


def test_batch_of_one_is_the_single_image_solve(orc):
    seg = seg_mod()
    B, fs = _batch(orc, [(111, 93)], [1.3], [0.25], 80)
    f = fs[0]
    S = seg.Solver(111, 93, tile_h=16, mode="compact")
    S.f[:, :93].copy_(torch.from_numpy(f))
    S.domain(q=0.25)
    S.solve(1.3, iters=80)
    torch.cuda.synchronize()
    for name in ("u", "v", "p1", "p2"):
        np.testing.assert_array_equal(seg.download(getattr(S, name)),
                                      seg.download(getattr(B.solvers[0], name)))


def test_batch_stopping_test_over_the_whole_batch(orc):
    """Section 4's criterion on the concatenated images: the batch stops at the
    first check where max(||du||, ||dv||) over all images is <= tol."""
    shapes = [(64, 64), (48, 80)]
    lams, qs = [1.0, 2.0], [0.3, 0.3]
    B, fs = _batch(orc, shapes, lams, qs, 3000, tol=1e-2, check_every=1)
    l = int(B.stats[0].item())
    hist = []
    for k, S in enumerate(B.solvers):
        reg = orc.domain(fs[k], float(S.dom.delta.cpu().numpy()[0]))
        hist.append(orc.solve(fs[k], reg, lams[k], iters=l + 1).hist)
    du = np.sqrt(sum(h[:, 0] ** 2 for h in hist))
    dv = np.sqrt(sum(h[:, 1] ** 2 for h in hist))
    crit = np.maximum(du, dv)
    first = int(np.argmax(crit <= 1e-2)) + 1
    assert l < 3000 and abs(first - l) <= 1 and (first == l or abs(crit[min(first, l) - 1] - 1e-2) < 1e-5)


def test_batch_capacity_overflow_is_reported(orc):
    seg = seg_mod()
    B, _ = _batch(orc, [(64, 64), (64, 64)], [1.0, 1.0], [0.5, 0.5], 5, capacity=100)
    with pytest.raises(seg.SegError) as e:
        B.check_status()
    assert e.value.status == seg.SEG_ERR_CAPACITY


@pytest.mark.slow
def test_full_size_batch_of_64(orc):
    """The 64-image workload (sides U{128..1024}, q ~ U[0.02, 0.4]) in one
    persistent launch: exact active counts per image, invariants everywhere,
    and the oracle on crops around sampled RD pixels of three images."""
    seg = seg_mod()
    probs = synth.batch(seed=0)
    shapes = [p.z.shape for p in probs]
    B = seg.BatchSolver(shapes, tile_h=16)
    fs = []
    for P, S in zip(probs, B.solvers):
        _, f = orc.fitting(P.z, 0.3, 0.7)
        fs.append(f)
        S.f[:, :f.shape[1]].copy_(torch.from_numpy(f))
        S.domain(q=P.q)
    K = 25
    B.solve([P.lam for P in probs], iters=K)
    torch.cuda.synchronize()
    B.check_status()
    rng = np.random.default_rng(3)
    for k in (0, 17, 63):
        S, f = B.solvers[k], fs[k]
        delta = float(S.dom.delta.cpu().numpy()[0])
        reg = orc.domain(f, delta)
        assert int(S.dom.counts[1].item()) == int(np.sum(reg == 2)) >= math.ceil(probs[k].q * f.size)
        u = seg.download(S.u).astype(np.float64)
        p1, p2 = seg.download(S.p1), seg.download(S.p2)
        v = seg.download(S.v)
        assert np.all(np.sqrt(p1.astype(np.float64) ** 2 + p2 ** 2) <= 1 + 1e-6)
        assert v.min() >= 0 and v.max() <= 1
        H, W = f.shape
        R = 2 * K + 4
        act = np.argwhere(reg == 2)
        for (i, j) in act[rng.choice(len(act), 4, replace=False)]:
            a, b = max(0, i - R), min(H, i + R + 1)
            c, d = max(0, j - R), min(W, j + R + 1)
            fc = np.ascontiguousarray(f[a:b, c:d])
            st = orc.solve(fc, orc.domain(fc, delta), probs[k].lam, iters=K)
            assert abs(st.u[i - a, j - c] - u[i, j]) <= 1e-4


def test_largest_batch_and_one_more(orc):
    """128 images (the most one launch takes) of sizes 1x1 .. 48x48, each
    against the oracle; 129 images are refused before any device work."""
    seg = seg_mod()
    rng = np.random.default_rng(12)
    shapes = [(int(rng.integers(1, 49)), int(rng.integers(1, 49))) for _ in range(128)]
    lams = [float(x) for x in rng.uniform(0.5, 3.0, 128)]
    qs = [float(x) for x in rng.uniform(0.0, 1.0, 128)]
    B, fs = _batch(orc, shapes, lams, qs, 40)
    B.check_status()
    for k, S in enumerate(B.solvers):
        delta = float(S.dom.delta.cpu().numpy()[0])
        st = orc.solve(fs[k], orc.domain(fs[k], delta), lams[k], 0.2, 0.125, 40)
        assert np.max(np.abs(seg.download(S.u).astype(np.float64) - st.u)) <= 1e-4, k
    B129 = seg.BatchSolver(shapes + [(8, 8)], tile_h=16)
    for S in B129.solvers:
        S.f.zero_()
        S.domain(delta=0.1)
    with pytest.raises(seg.SegError) as e:
        B129.solve([1.0] * 129, iters=5)
    assert e.value.status == seg.SEG_ERR_INVALID_ARG


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batch_waves_give_the_same_iterates(orc, storage):
    """A batch with a fixed iteration count larger than one wave (5,000
    pixels per block) runs in waves of whole images; with a stopping test
    (never met) it runs as one range.  The images are independent and every
    path rounds alike, so both give the same bits."""
    seg = seg_mod()
    shapes = [(600, 640), (512, 700), (640, 480), (700, 600), (480, 512), (620, 600), (500, 500)]
    lams = [1.0, 1.5, 2.0, 0.7, 1.2, 1.8, 1.1]
    qs = [0.4, 0.35, 0.4, 0.3, 0.4, 0.38, 0.4]
    outs = []
    for tol in (0.0, 1e-30):
        B, _ = _batch(orc, shapes, lams, qs, 40, storage=storage, tol=tol)
        B.check_status()
        assert int(B.stats[3].item()) > 152 * 5000   # more than one wave
        outs.append([{k: seg.download(getattr(S, k)) for k in ("u", "v", "p1", "p2")} for S in B.solvers])
        outs[-1].append(B.stats.cpu().numpy().copy())
    for a, b in zip(outs[0][:-1], outs[1][:-1]):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])
    sa, sb = outs[0][-1], outs[1][-1]
    assert sa[0] == sb[0] == 40 and sa[3] == sb[3]
    # the last test's norms: summed over the waves vs over the one range
    assert sa[1] == pytest.approx(sb[1], rel=1e-5) and sa[2] == pytest.approx(sb[2], rel=1e-5)
