"""Helpers for the GPU parity tests: run the CUDA path through the C ABI
binding on numpy inputs, and decode its outputs for comparison with the oracle."""
import math

import numpy as np
import pytest
import torch


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU: the CUDA path has no CPU fallback")


def seg_mod():
    from paper_1807_11534_gb300 import seg
    seg.load()
    return seg


def bits_to_mask(words, W):
    """uint32 bit plane [H][nw] (as int32 tensor) -> bool [H][W]."""
    w = words.cpu().numpy().view(np.uint32)
    H, nw = w.shape
    b = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool)
    return b.reshape(H, nw * 32)[:, :W]


def run_gpu(f32, delta=math.inf, q=-1.0, lam=1.0, theta=0.2, tau=0.125, iters=100, tol=0.0,
            n_inner=1, check_every=10, mode="compact", storage="f32", tile_h=16, warm=None, sweep=0,
            radius=0, smooth=0):
    """Domain + solve for a float32 fitting term; returns a dict of numpy
    outputs (u, v, p1, p2 as float64) and the solver."""
    seg = seg_mod()
    H, W = f32.shape
    S = seg.Solver(H, W, tile_h=tile_h, mode=mode, storage=storage)
    S.f[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(f32)))
    S.domain(delta=delta, q=q, radius=radius, smooth=smooth)
    if warm is not None:
        for name in ("u", "v", "p1", "p2"):
            getattr(S, name)[:, :W].copy_(torch.from_numpy(np.asarray(getattr(warm, name), np.float32)))
    S.solve(lam, theta, tau, iters, tol, n_inner, check_every, warm_start=warm is not None,
            sweep=sweep)
    torch.cuda.synchronize()
    S.check_status()
    out = {k: seg.download(getattr(S, k)).astype(np.float64) for k in ("u", "v", "p1", "p2")}
    out["stats"] = S.stats.cpu().numpy()
    out["counts"] = S.dom.counts.cpu().numpy()
    out["delta"] = float(S.dom.delta.cpu().numpy()[0])
    out["solver"] = S
    return out
