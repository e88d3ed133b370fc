"""Robust restriction (the Conclusion's noisy-f case): the local mean of f,
the partition thresholded on it with the sign disagreements, the square
dilation of RD, and solves on that domain, against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import bits_to_mask, require_gpu, run_gpu, seg_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _field(shape, seed, sigma=0.3):
    f = np.random.default_rng(seed).normal(0, sigma, shape).astype(np.float32)
    f.flat[:: 17] = 0.0
    return f


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (33, 1), (37, 70), (64, 64), (129, 97)])
@pytest.mark.parametrize("r", [0, 1, 3, 16])
def test_box_mean_bit_exact(orc, shape, r):
    seg = seg_mod()
    f = _field(shape, shape[0] + r)
    fd = seg.upload(f)
    out = seg.image(*shape)
    seg.seg_box_mean(fd, r, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(seg.download(out), orc.box_mean(f, r))


@pytest.mark.parametrize("shape,tile_h", [((37, 70), 8), ((64, 64), 16), ((129, 97), 4),
                                          ((1, 33), 32), ((50, 31), 16), ((200, 301), 32)])
@pytest.mark.parametrize("kw", [dict(delta=0.05, radius=1), dict(delta=0.02, radius=5),
                                dict(q=0.1, radius=31), dict(q=0.03, radius=32),
                                dict(delta=0.05, smooth=1), dict(q=0.05, smooth=2),
                                dict(q=0.05, smooth=1, radius=2), dict(delta=0.0, smooth=3)])
def test_robust_domain_bit_exact(orc, shape, tile_h, kw):
    """Bit planes, counts, tile and pixel lists and compact starts of the
    robust partition equal the oracle's lists of the same partition."""
    seg = seg_mod()
    H, W = shape
    f = _field(shape, H * 3 + tile_h)
    S = seg.Solver(H, W, tile_h=tile_h)
    S.f[:, :W].copy_(torch.from_numpy(f))
    d = S.domain(delta=kw.get("delta", math.inf), q=kw.get("q", -1.0), radius=kw.get("radius", 0),
                 smooth=kw.get("smooth", 0))
    torch.cuda.synchronize()
    S.check_status()
    reg = orc.robust_region(f, kw.get("delta"), kw.get("q", -1.0), kw.get("smooth", 0),
                            kw.get("radius", 0))
    np.testing.assert_array_equal(bits_to_mask(d.act, W), reg == 2)
    np.testing.assert_array_equal(bits_to_mask(d.fg, W), f < 0)
    # padding bits beyond W stay clear
    act = d.act.cpu().numpy().view(np.uint32)
    assert int(bits_to_mask(d.act, act.shape[1] * 32)[:, W:].sum()) == 0
    tl = orc.tile_list(reg, tile_h, 32)
    pl = orc.pixel_list_tiled(reg, tile_h, 32)
    cnt = d.counts.cpu().numpy()
    assert cnt[0] == len(tl) and cnt[1] == len(pl) and cnt[2] == int(np.sum(reg == 1))
    np.testing.assert_array_equal(d.tiles.cpu().numpy()[:len(tl)], tl)
    np.testing.assert_array_equal(d.pixels.cpu().numpy()[:len(pl)], pl)
    ws = d.wstart.cpu().numpy()
    ii, jj = pl // W, pl % W
    below = act[ii, jj // 32] & ((np.uint32(1) << (jj % 32).astype(np.uint32)) - np.uint32(1))
    popc = np.array([bin(int(x)).count("1") for x in below], np.int64)
    np.testing.assert_array_equal(ws[ii, jj // 32] + popc, np.arange(len(pl)))


@pytest.mark.parametrize("mode", ["compact", "dense", "tiled"])
@pytest.mark.parametrize("kw", [dict(q=0.05, smooth=1), dict(q=0.1, radius=1)])
def test_solve_on_the_robust_domain(orc, mode, kw):
    P = synth.noisy_example(seed=1, H=90, W=110)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    out = run_gpu(f, q=kw["q"], lam=2.0, iters=150, mode=mode, tile_h=8,
                  radius=kw.get("radius", 0), smooth=kw.get("smooth", 0))
    reg = orc.robust_region(f, None, kw["q"], kw.get("smooth", 0), kw.get("radius", 0))
    st = orc.solve(f, reg, 2.0, iters=150)
    for k, tol in (("u", 1e-4), ("v", 1e-4), ("p1", 2e-4), ("p2", 2e-4)):
        assert np.max(np.abs(out[k] - getattr(st, k))) <= tol, k


def test_robust_arguments_are_checked():
    seg = seg_mod()
    S = seg.Solver(20, 40)
    for r in (-1, 33):
        with pytest.raises(seg.SegError) as e:
            S.domain(delta=0.1, radius=r)
        assert e.value.status == seg.SEG_ERR_INVALID_ARG
    with pytest.raises(seg.SegError) as e:
        seg.seg_box_mean(S.f, 17, seg.image(20, 40))
    assert e.value.status == seg.SEG_ERR_INVALID_ARG
    with pytest.raises(seg.SegError) as e:
        seg.seg_box_mean(S.f, 1, S.f)
    assert e.value.status == seg.SEG_ERR_INVALID_ARG
    f = np.zeros((20, 40), np.float32)
    f[4, 4] = np.inf
    S.f[:, :40].copy_(torch.from_numpy(f))
    S.domain(q=0.1, smooth=1)
    with pytest.raises(seg.SegError) as e:
        S.check_status()
    assert e.value.status == seg.SEG_ERR_NONFINITE
