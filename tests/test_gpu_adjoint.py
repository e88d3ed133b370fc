"""The hand-written adjoint (seg_solve_diff + seg_backward, and the
torch.autograd.Function around them) against the FP64 oracle's reverse mode
(itself pinned by central finite differences) and against finite
differences of the CUDA forward."""
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


def _gpu_grad(f, delta, lam, gu, gv, iters, ckpt_every, z=None, c=None):
    seg = seg_mod()
    H, W = f.shape
    S = seg.DiffSolver(H, W, iters, ckpt_every)
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=delta)
    S.solve_diff(lam)
    g = seg.upload(gu.astype(np.float32))
    gvt = seg.upload(gv.astype(np.float32)) if gv is not None else None
    zt = seg.upload(z) if z is not None else None
    ct = torch.tensor(c, dtype=torch.float64, device="cuda") if c is not None else None
    gf, gout = S.backward(g, gvt, zt, ct)
    torch.cuda.synchronize()
    S.check_status()
    return seg.download(gf).astype(np.float64), gout.cpu().numpy(), S


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12))


@pytest.mark.parametrize("shape,delta,iters,ce", [((40, 50), np.inf, 30, 7), ((64, 64), 0.25, 60, 20),
                                                  ((33, 70), 0.12, 25, 25), ((20, 31), 0.3, 9, 1)])
def test_backward_matches_oracle_reverse_mode(orc, shape, delta, iters, ce):
    rng = np.random.default_rng(sum(shape))
    P = synth.small_example(seed=shape[0], H=shape[0], W=shape[1])
    _, f = orc.fitting(P.z, 0.3, 0.7)
    gu = rng.normal(size=shape)
    gv = rng.normal(size=shape)
    lam = 1.3
    gf, gout, _ = _gpu_grad(f, delta, lam, gu, gv, iters, ce)
    reg = orc.domain(f, delta)
    gf_o, gl_o = orc.solve_grad(f, reg, lam, gu, gv, iters=iters)
    assert np.all(gf[reg != 2] == 0)
    assert _rel(gf, gf_o) <= 1e-3, _rel(gf, gf_o)
    assert abs(gout[0] - gl_o) <= 1e-3 * max(1.0, abs(gl_o)), (gout[0], gl_o)


def test_c_gradients_through_the_fitting_term(orc):
    """dL/dc1 = sum dL/df (-2)(z - c1), dL/dc2 = sum dL/df 2(z - c2) (Eq. CV)."""
    rng = np.random.default_rng(5)
    P = synth.small_example(seed=9, H=48, W=64)
    c1, c2 = 0.32, 0.69
    _, f = orc.fitting(P.z, c1, c2)
    gu = rng.normal(size=f.shape)
    gf, gout, _ = _gpu_grad(f, 0.2, 1.0, gu, None, 40, 10, z=P.z, c=[c1, c2])
    reg = orc.domain(f, 0.2)
    gf_o, _ = orc.solve_grad(f, reg, 1.0, gu, None, iters=40)
    z = P.z.astype(np.float64)
    e1 = float(np.sum(gf_o * (-2.0) * (z - c1)))
    e2 = float(np.sum(gf_o * 2.0 * (z - c2)))
    assert abs(gout[1] - e1) <= 1e-3 * max(1.0, abs(e1)) and abs(gout[2] - e2) <= 1e-3 * max(1.0, abs(e2))


@pytest.mark.slow
def test_crops_of_the_differentiation_workload(orc):
    """1024x1024 random-shape images with generator masks, BCE(u_K, mask) on
    clip(u_K, 1e-4, 1 - 1e-4), K = 200 unrolled iterations, checkpoints every
    20; the gradient of 64x64 crops (each an independent problem) against the
    oracle's reverse mode, and against central differences of the CUDA
    forward with h = 1e-3 along a random direction."""
    rng = np.random.default_rng(11)
    probs = synth.training_batch(seed=0, n_images=2, side=1024)
    for P in probs:
        _, f_full = orc.fitting(P.z, 0.3, 0.7)
        i0, j0 = rng.integers(0, 1024 - 64, 2)
        f = np.ascontiguousarray(f_full[i0:i0 + 64, j0:j0 + 64])
        m = P.label[i0:i0 + 64, j0:j0 + 64].astype(np.float64)
        K, lam, delta = 200, 1.0, 0.2
        # BCE gradient at the oracle's u_K
        reg = orc.domain(f, delta)
        u = orc.solve(f, reg, lam, iters=K).u
        uc = np.clip(u, 1e-4, 1 - 1e-4)
        gu = np.where((u > 1e-4) & (u < 1 - 1e-4), (uc - m) / (uc * (1 - uc)), 0.0) / u.size
        gf, gout, S = _gpu_grad(f, delta, lam, gu, None, K, 20)
        gf_o, gl_o = orc.solve_grad(f, reg, lam, gu, None, iters=K)
        assert _rel(gf, gf_o) <= 1e-3, _rel(gf, gf_o)
        assert abs(gout[0] - gl_o) <= 1e-3 * max(1e-3, abs(gl_o))
        # finite differences of the CUDA forward (linear loss <gu, u_K>)
        seg = seg_mod()
        d = np.where(reg == 2, rng.normal(size=f.shape), 0.0)
        h = 1e-3

        def loss(ff):
            T = seg.DiffSolver(64, 64, K, 20)
            T.f[:, :64].copy_(torch.from_numpy(ff.astype(np.float32)))
            T.dom = S.dom     # the partition of the unperturbed f stays fixed
            T.solve_diff(lam)
            return float(np.sum(gu * seg.download(T.u)))

        fd = (loss(f + h * d) - loss(f - h * d)) / (2 * h)
        an = float(np.sum(gf * d))
        assert abs(fd - an) <= 2e-2 * max(abs(an), 1e-3), (fd, an)


def test_autograd_function(orc):
    seg = seg_mod()
    rng = np.random.default_rng(3)
    P = synth.small_example(seed=3, H=50, W=70)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    S = seg.DiffSolver(50, 70, 40, 10)
    S.f[:, :70].copy_(torch.from_numpy(f))
    S.domain(delta=0.2)
    ft = S.f.clone().requires_grad_(True)
    lam = torch.tensor(1.2, dtype=torch.float64, device="cuda", requires_grad=True)
    wgt = torch.zeros_like(S.f)
    wgt[:, :70] = torch.from_numpy(rng.normal(size=(50, 70)).astype(np.float32))
    u = seg.SegSolveFn.apply(ft, lam, S)
    (u * wgt).sum().backward()
    reg = orc.domain(f, 0.2)
    gf_o, gl_o = orc.solve_grad(f, reg, 1.2, wgt[:, :70].cpu().numpy().astype(np.float64), None, iters=40)
    assert _rel(ft.grad[:, :70].cpu().numpy().astype(np.float64), gf_o) <= 1e-3
    assert abs(lam.grad.item() - gl_o) <= 1e-3 * max(1.0, abs(gl_o))
    # c1, c2 through the fitting term
    z = seg.upload(P.z)
    c1 = torch.tensor(0.3, dtype=torch.float64, device="cuda", requires_grad=True)
    c2 = torch.tensor(0.7, dtype=torch.float64, device="cuda", requires_grad=True)
    lam2 = torch.tensor(1.2, dtype=torch.float64, device="cuda", requires_grad=True)
    u2 = seg.SegFitSolveFn.apply(z, c1, c2, lam2, S, 0.2)
    (u2 * wgt).sum().backward()
    zz = P.z.astype(np.float64)
    assert abs(c1.grad.item() - np.sum(gf_o * -2 * (zz - 0.3))) <= 1e-3 * max(1.0, abs(c1.grad.item()))
    assert abs(c2.grad.item() - np.sum(gf_o * 2 * (zz - 0.7))) <= 1e-3 * max(1.0, abs(c2.grad.item()))
    assert abs(lam2.grad.item() - gl_o) <= 1e-3 * max(1.0, abs(gl_o))


def _batch_vs_single(orc, shapes, lams, delta, iters, ce, with_c):
    seg = seg_mod()
    rng = np.random.default_rng(len(shapes) + iters)
    probs = [synth.small_example(seed=10 + k, H=h, W=w) for k, (h, w) in enumerate(shapes)]
    fs = [orc.fitting(P.z, 0.3, 0.7)[1] for P in probs]
    gus = [rng.normal(size=s).astype(np.float32) for s in shapes]
    gvs = [rng.normal(size=s).astype(np.float32) for s in shapes]
    B = seg.BatchDiffSolver(shapes, iters, ce)
    for S, f in zip(B.solvers, fs):
        S.f[:, :f.shape[1]].copy_(torch.from_numpy(f))
        S.domain(delta=delta)
    B.solve_diff(lams)
    g_u = [seg.upload(g) for g in gus]
    g_v = [seg.upload(g) for g in gvs]
    zs = [seg.upload(P.z) for P in probs] if with_c else None
    cs = [torch.tensor([0.3, 0.7], dtype=torch.float64, device="cuda") for _ in probs] if with_c else None
    out = B.backward(g_u, g_v, zs, cs)
    torch.cuda.synchronize()
    B.check_status()
    for k, (f, P) in enumerate(zip(fs, probs)):
        gf1, gout1, S1 = _gpu_grad(f, delta, lams[k], gus[k], gvs[k], iters, ce,
                                   z=P.z if with_c else None, c=[0.3, 0.7] if with_c else None)
        Sb = B.solvers[k]
        np.testing.assert_array_equal(seg.download(Sb.u), seg.download(S1.u))
        np.testing.assert_array_equal(seg.download(out[k][0]).astype(np.float64), gf1)
        np.testing.assert_array_equal(out[k][1].cpu().numpy(), gout1)


@pytest.mark.parametrize("delta,iters,ce,with_c", [(0.2, 40, 20, True), (np.inf, 25, 7, False),
                                                   (0.12, 30, 30, False)])
def test_batched_adjoint_equals_the_per_image_adjoint(orc, delta, iters, ce, with_c):
    """seg_solve_diff_batch + seg_backward_batch on images of uneven size and
    lambda give, image by image, the same bits as seg_solve_diff +
    seg_backward on that image alone: the forward iterates (u), dL/df and the
    FP64 sums for lambda, c1, c2 (the images are independent problems, the
    reverse sweep's arithmetic is per pixel, and the sums run per image in
    the same fixed order)."""
    _batch_vs_single(orc, [(67, 131), (90, 45), (33, 200), (128, 96)], [1.0, 1.7, 0.6, 2.5], delta, iters, ce,
                     with_c)


@pytest.mark.slow
def test_batched_adjoint_on_the_differentiation_workload(orc):
    """The differentiation workload's shape (8 images of 1024 x 1024, K = 200,
    checkpoints every 20, delta = 0.2; the global-memory paths of the forward
    and the reverse sweep): the batch against the per-image adjoint on two
    of its images, bit for bit, and the per-image adjoint against the
    oracle's reverse mode is covered above."""
    seg = seg_mod()
    probs = synth.training_batch(seed=0, n_images=8, side=1024, iters=200)
    fs = [orc.fitting(P.z, 0.3, 0.7)[1] for P in probs]
    B = seg.BatchDiffSolver([(1024, 1024)] * 8, 200, 20)
    for S, f in zip(B.solvers, fs):
        S.f[:, :1024].copy_(torch.from_numpy(f))
        S.domain(delta=0.2)
    B.solve_diff([1.0] * 8)
    rng = np.random.default_rng(3)
    gus = [rng.normal(size=(1024, 1024)).astype(np.float32) for _ in probs]
    out = B.backward([seg.upload(g) for g in gus])
    torch.cuda.synchronize()
    B.check_status()
    for k in (0, 5):
        gf1, gout1, _ = _gpu_grad(fs[k], 0.2, 1.0, gus[k], None, 200, 20)
        np.testing.assert_array_equal(seg.download(out[k][0]).astype(np.float64), gf1)
        np.testing.assert_array_equal(out[k][1].cpu().numpy(), gout1)




def _clip_pattern(orc, f, reg, lam, iters):
    """Where v = clip(u - theta lambda f, 0, 1) sits on a bound, iteration by
    iteration (-1 at 1, +1 at 0, 0 inside): the loss is a smooth function of
    f and lambda wherever this pattern does not change."""
    st = orc.solve(f, reg, lam, iters=1)
    pats = np.empty((iters,) + f.shape, np.int8)
    for k in range(iters):
        if k:
            st = orc.solve(f, reg, lam, iters=1, state=st)
        pats[k] = (st.v <= 0.0).astype(np.int8) - (st.v >= 1.0).astype(np.int8)
    return st, pats


@pytest.mark.slow
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_backward_matches_fp64_finite_differences(orc, seed):
    """The GPU backward against central finite differences directly, to 1e-3
    relative, on the differentiation workload's configuration: a 64x64 crop
    (across a shape boundary) of a 1024x1024 training image, CV fitting term
    from z with c1 = 0.3, c2 = 0.7, delta = 0.2, K = 200 unrolled iterations,
    checkpoints every 20, L = <g, u_K> with g the BCE gradient at u_K.

    The differences are taken on the FP64 oracle forward with the partition
    held fixed (the adjoint's convention), along three random directions on
    RD, along df/dc1 = -2(z - c1) and df/dc2 = 2(z - c2) (so the c
    derivatives are the f derivative along those directions), and in lambda.
    The unrolled map is piecewise smooth: it has a kink wherever an iterate
    of v meets a bound of the clip, so each difference uses the largest step
    h in {1e-5, 1e-6, 1e-7, 1e-8} at which the oracle's clip pattern over all K
    iterations is the same at both ends as at the centre.  The oracle reads f
    as float32, so the GPU's directional derivative is formed along the steps
    actually taken.  A derivative that is a sum with more than hundredfold
    cancellation is compared at 1e-3 of a hundredth of its sum of absolute
    terms (float32 resolves each term to about 1e-6), which applies only to
    dL/dc2 on some crops."""
    rng = np.random.default_rng(40 + seed)
    P = synth.training_batch(seed=seed, n_images=1, side=1024)[0]
    K, lam, delta = 200, 1.0, 0.2
    c1, c2 = 0.3, 0.7
    for _ in range(400):
        i0, j0 = rng.integers(0, 1024 - 64, 2)
        z = np.ascontiguousarray(P.z[i0:i0 + 64, j0:j0 + 64])
        _, f = orc.fitting(z, c1, c2)
        reg = orc.domain(f, delta)
        rd = reg == 2
        # a boundary in the crop, and no RD pixel whose f a step could move across 0 (u0 = H(-f))
        if 0.2 < P.label[i0:i0 + 64, j0:j0 + 64].mean() < 0.8 and np.abs(f[rd]).min() > 1e-4:
            break
    else:
        pytest.skip("no crop across a boundary")
    m = P.label[i0:i0 + 64, j0:j0 + 64].astype(np.float64)
    st, pat0 = _clip_pattern(orc, f, reg, lam, K)
    u = st.u
    uc = np.clip(u, 1e-4, 1 - 1e-4)
    gu = np.where((u > 1e-4) & (u < 1 - 1e-4), (uc - m) / (uc * (1 - uc)), 0.0) / u.size
    gf, gout, _ = _gpu_grad(f, delta, lam, gu, None, K, 20, z=z, c=[c1, c2])

    def loss(ff, ll=lam):
        return float(np.sum(gu * orc.solve(ff, reg, ll, iters=K).u))

    zz = z.astype(np.float64)
    dirs = {f"f{k}": np.where(rd, np.clip(rng.normal(size=f.shape), -3, 3), 0.0) for k in range(3)}
    dirs["c1"] = np.where(rd, -2 * (zz - c1), 0.0)
    dirs["c2"] = np.where(rd, 2 * (zz - c2), 0.0)
    results = {}
    for name, d in dirs.items():
        for h in (1e-5, 1e-6, 1e-7, 1e-8):
            fp = (f.astype(np.float64) + h * d).astype(np.float32)
            fm = (f.astype(np.float64) - h * d).astype(np.float32)
            if np.array_equal(_clip_pattern(orc, fp, reg, lam, K)[1], pat0) and \
                    np.array_equal(_clip_pattern(orc, fm, reg, lam, K)[1], pat0):
                terms = gf * (fp.astype(np.float64) - fm) / (2 * h)
                results[name] = ((loss(fp) - loss(fm)) / (2 * h), float(np.sum(terms)),
                                 float(np.sum(np.abs(terms))), h)
                break
    for h in (1e-5, 1e-6, 1e-7, 1e-8):
        if np.array_equal(_clip_pattern(orc, f, reg, lam + h, K)[1], pat0) and \
                np.array_equal(_clip_pattern(orc, f, reg, lam - h, K)[1], pat0):
            results["lambda"] = ((loss(f, lam + h) - loss(f, lam - h)) / (2 * h), float(gout[0]), 0.0, h)
            break
    assert set(results) == set(dirs) | {"lambda"}, sorted(results)   # a smooth step was found for each
    for name, (fd, an, absum, h) in results.items():
        scale = max(abs(fd), absum / 100)
        assert abs(fd - an) <= 1e-3 * scale, (name, h, fd, an, absum)
    # the c gradients are the f gradient's sums along df/dc (FP64 on both sides)
    for k, name in ((1, "c1"), (2, "c2")):
        e = float(np.sum(gf * dirs[name]))
        assert abs(gout[k] - e) <= 1e-9 * float(np.sum(np.abs(gf * dirs[name]))), (name, gout[k], e)
