"""The bounded device-side waits of the persistent solvers, driven to run out
from the host (no GPU fault involved): seg_set_wait_limit makes every grid
barrier of a workspace wait for one arrival more than its launch has blocks,
with a bound of a few thousand cycles.  Every block must give up, the solve
must return, seg_read_status must report SEG_ERR_TIMEOUT, and solves
afterwards (the same workspace with the limit reset, and a fresh solver)
must run normally and still match the oracle."""
import math

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, run_gpu, seg_mod

pytestmark = pytest.mark.gpu

SHORT = 20000   # cycles: about 10 us at the SM clock


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _expect_timeout(check_status):
    seg = seg_mod()
    with pytest.raises(seg.SegError) as e:
        check_status()
    assert e.value.status == seg.SEG_ERR_TIMEOUT


def _f(H, W, seed):
    P = synth.small_example(seed=seed, H=H, W=W)
    return (0.8 * P.z - 0.4).astype(np.float32)


@pytest.mark.parametrize("shape,delta", [((96, 130), 0.15), ((2048, 1024), math.inf), ((4096, 2048), math.inf)])
def test_compact_solve_times_out_and_recovers(orc, shape, delta):
    """(96 x 130, delta 0.15): the shared-memory one-barrier path; (2048 x
    1024, full domain, 2.1 M RD pixels): the row-major solve with its
    neighbourhoods in shared memory; (4096 x 2048, full domain, 8.4 M RD
    pixels): the row-major solve launched without shared memory."""
    seg = seg_mod()
    H, W = shape
    f = _f(H, W, 3)
    S = seg.Solver(H, W, tile_h=16, mode="compact")
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=delta)
    seg.seg_set_wait_limit(S.ws, SHORT, 1, S.stream)
    S.solve(1.0, iters=50)
    torch.cuda.synchronize()
    _expect_timeout(S.check_status)
    # the same workspace with the default limit again: a normal solve
    seg.seg_set_wait_limit(S.ws, 0, 0, S.stream)
    S.solve(1.0, iters=50)
    torch.cuda.synchronize()
    S.check_status()
    if H * W <= 20000:
        st = orc.solve(f, orc.domain(f, delta), 1.0, iters=50)
        assert np.max(np.abs(seg.download(S.u) - st.u)) <= 1e-4
    # a fresh solver in the same process
    out = run_gpu(f[:64, :80], delta=delta, iters=40)
    st = orc.solve(f[:64, :80], orc.domain(f[:64, :80], delta), 1.0, iters=40)
    assert np.max(np.abs(out["u"] - st.u)) <= 1e-4


def test_primal_dual_and_volume_solves_time_out(orc):
    seg = seg_mod()
    f = _f(80, 96, 4)
    S = seg.Solver(80, 96, tile_h=16, mode="compact")
    S.f[:, :96].copy_(torch.from_numpy(f))
    S.domain(delta=0.2)
    seg.seg_set_wait_limit(S.ws, SHORT, 1, S.stream)
    S.solve_pd(1.0, iters=30)
    torch.cuda.synchronize()
    _expect_timeout(S.check_status)
    seg.seg_set_wait_limit(S.ws, 0, 0, S.stream)
    S.solve_pd(1.0, iters=30)
    torch.cuda.synchronize()
    S.check_status()
    st = orc.solve_pd(f, orc.domain(f, 0.2), 1.0, iters=30)
    assert np.max(np.abs(seg.download(S.u) - st.u)) <= 1e-4

    V = synth.spheres_volume(seed=1, D=12, H=20, W=24)
    VS = seg.VolumeSolver(12, 20, 24)
    VS.fitting(VS.upload(V.z), 0.3, 0.7)
    VS.domain(delta=0.2)
    seg.seg_set_wait_limit(VS.ws, SHORT, 2, VS.stream)
    VS.solve(2.0, iters=20)
    torch.cuda.synchronize()
    _expect_timeout(VS.check_status)
    seg.seg_set_wait_limit(VS.ws, 0, 0, VS.stream)
    VS.solve(2.0, iters=20)
    torch.cuda.synchronize()
    VS.check_status()
    # the full volume: the one-voxel kernel (RD above half the volume)
    VS.domain(delta=math.inf)
    seg.seg_set_wait_limit(VS.ws, SHORT, 2, VS.stream)
    VS.solve(2.0, iters=20)
    torch.cuda.synchronize()
    _expect_timeout(VS.check_status)
    seg.seg_set_wait_limit(VS.ws, 0, 0, VS.stream)
    VS.solve(2.0, iters=20)
    torch.cuda.synchronize()
    VS.check_status()


def test_reverse_sweep_times_out_and_recovers(orc):
    """The adjoint's persistent sweep (its shared-memory kernel at this
    size): the barrier wait runs out, the status says so, and a second
    backward on the same forward state matches the oracle's reverse mode."""
    seg = seg_mod()
    rng = np.random.default_rng(8)
    H, W, K, C = 48, 64, 30, 10
    f = _f(H, W, 6)
    gu = rng.normal(size=(H, W))
    S = seg.DiffSolver(H, W, K, C)
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=0.2)
    S.solve_diff(1.0)
    g = seg.upload(gu.astype(np.float32))
    seg.seg_set_wait_limit(S.ws, SHORT, 1, S.stream)
    S.backward(g)
    torch.cuda.synchronize()
    _expect_timeout(S.check_status)
    seg.seg_set_wait_limit(S.ws, 0, 0, S.stream)
    gf, gout = S.backward(g)
    torch.cuda.synchronize()
    S.check_status()
    gf_o, gl_o = orc.solve_grad(f, orc.domain(f, 0.2), 1.0, gu, None, iters=K)
    gf = seg.download(gf).astype(np.float64)
    assert np.linalg.norm(gf - gf_o) <= 1e-3 * np.linalg.norm(gf_o)
    assert abs(gout.cpu().numpy()[0] - gl_o) <= 1e-3 * max(1.0, abs(gl_o))


def test_batch_solve_times_out_and_recovers(orc):
    seg = seg_mod()
    shapes = [(70, 90), (128, 40), (33, 200)]
    B = seg.BatchSolver(shapes, tile_h=16)
    fs = []
    for k, ((H, W), S) in enumerate(zip(shapes, B.solvers)):
        f = _f(H, W, 10 + k)
        fs.append(f)
        S.f[:, :W].copy_(torch.from_numpy(f))
        S.domain(delta=0.2)
    seg.seg_set_wait_limit(B.ws, SHORT, 1, B.stream)
    B.solve([1.0] * 3, iters=40)
    torch.cuda.synchronize()
    _expect_timeout(B.check_status)
    seg.seg_set_wait_limit(B.ws, 0, 0, B.stream)
    B.solve([1.0] * 3, iters=40)
    torch.cuda.synchronize()
    B.check_status()
    for f, S in zip(fs, B.solvers):
        st = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=40)
        assert np.max(np.abs(seg.download(S.u) - st.u)) <= 1e-4


def test_wait_limit_arguments_are_checked():
    seg = seg_mod()
    ws = seg.workspace(32, 32)
    with pytest.raises(seg.SegError) as e:
        seg.seg_set_wait_limit(ws, -1, 0)
    assert e.value.status == seg.SEG_ERR_INVALID_ARG
    with pytest.raises(seg.SegError):
        seg.seg_set_wait_limit(ws, 100, -2)
