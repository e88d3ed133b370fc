"""The compact solver's one-barrier iteration, which the 2048x2048
distance-selective image takes at its benchmark delta (0.2, 863K RD pixels):
each block keeps its pixels' state in shared memory and also runs the dual
step of the ring of pixels other blocks own directly above or left of its
own, so one grid barrier ends an iteration.  Covered here: that every block
ran it, the Section 4 stopping test (decided in every block), warm start, and
the checkpoints of the differentiable forward (through the adjoint, against
the oracle's reverse mode on a crop), and the primal-dual solver's
shared-memory iteration built the same way.  Parity against the oracle on
sampled crops and against the dense solver on the whole image is in
test_gpu_parity.py (test_gpu_pd.py for the primal-dual solver)."""
import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, seg_mod

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

H = W = 2048
DELTA, LAM = 0.2, 2.0


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


@pytest.fixture(scope="module")
def f_ds(orc):
    P = synth.ellipses_ds(seed=0, H=H, W=W)
    c1, c2 = orc.class_means(P.z, P.label)
    return orc.fitting(P.z, c1, c2, P.markers, P.gamma)[1]


def _solver(f):
    seg = seg_mod()
    S = seg.Solver(H, W, tile_h=16)
    S.f[:, :W].copy_(torch.from_numpy(f))
    S.domain(delta=DELTA)
    return S


def _state(S):
    seg = seg_mod()
    torch.cuda.synchronize()
    S.check_status()
    return {k: seg.download(getattr(S, k)).copy() for k in ("u", "v", "p1", "p2")}


def test_every_block_runs_one_barrier_and_stops_at_a_check(f_ds):
    S = _solver(f_ds)
    # ||du||, ||dv|| at the checks l = 5, 10, ..., 150 (a cold solve of l
    # iterations ends with the test of iteration l, as the long run does)
    norms = []
    for l in range(5, 155, 5):
        st = S.solve(LAM, iters=l, check_every=5).cpu().numpy()
        norms.append(max(st[1], st[2]))
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        # shared-memory state and one barrier in every block of the grid
        # (a whole number of blocks per SM)
        assert st[6] == st[7] and st[6] >= sms and st[6] % sms == 0, st
    norms = np.array(norms)
    # tol between a check that sets a new low by more than 5 % and the lowest before it
    k = next(k for k in range(6, len(norms)) if norms[:k].min() > 1.05 * norms[k])
    tol = float(np.sqrt(norms[:k].min() * norms[k]))
    stop = 5 * (k + 1)
    S.solve(LAM, iters=stop, check_every=5)
    ref = _state(S)
    st = S.solve(LAM, iters=600, tol=tol, check_every=5).cpu().numpy()
    got = _state(S)
    assert int(st[0]) == stop and int(st[5]) == stop
    for name in ref:   # the stopped iterate is the cold iterate of that many iterations
        np.testing.assert_array_equal(got[name], ref[name], err_msg=name)


def test_warm_start_continues_the_iteration(f_ds):
    S = _solver(f_ds)
    S.solve(LAM, iters=40)
    cold = _state(S)
    S.solve(LAM, iters=20)
    S.solve(LAM, iters=20, warm_start=True)
    warm = _state(S)
    for name in cold:
        assert np.max(np.abs(warm[name].astype(np.float64) - cold[name])) <= 1e-5, name


def test_checkpoints_through_the_adjoint_on_a_crop(orc, f_ds):
    """seg_solve_diff on the whole image (one-barrier iteration, checkpoints
    every 10 of K = 20 iterations), a loss on a 16x16 window around an RD
    pixel; dL/df against the oracle's reverse mode on a crop of radius
    8 + 4K + 4 (dL/df is nonzero within 2K + 8 of the window's centre, and
    the forward iterate there depends on f within 2K more)."""
    seg = seg_mod()
    K, ce = 20, 10
    S = seg.DiffSolver(H, W, K, ce)
    S.f[:, :W].copy_(torch.from_numpy(f_ds))
    S.domain(delta=DELTA)
    S.solve_diff(LAM)
    torch.cuda.synchronize()
    assert S.stats.cpu().numpy()[7] > 0   # the one-barrier iteration wrote the checkpoints
    reg_full = orc.domain(f_ds, DELTA)
    rng = np.random.default_rng(4)
    act = np.argwhere(reg_full == 2)
    act = act[(act[:, 0] > 200) & (act[:, 0] < H - 200) & (act[:, 1] > 200) & (act[:, 1] < W - 200)]
    ci, cj = act[rng.integers(len(act))]
    gu = np.zeros((H, W))
    gu[ci - 8:ci + 8, cj - 8:cj + 8] = rng.normal(size=(16, 16))
    gf, gout = S.backward(seg.upload(gu.astype(np.float32)))
    torch.cuda.synchronize()
    S.check_status()
    gf = seg.download(gf).astype(np.float64)
    R = 8 + 4 * K + 4
    sl = (slice(ci - R, ci + R), slice(cj - R, cj + R))
    f_c = np.ascontiguousarray(f_ds[sl])
    reg = orc.domain(f_c, DELTA)
    gf_o, _ = orc.solve_grad(f_c, reg, LAM, gu[sl], None, iters=K)
    inner = np.zeros_like(gf, dtype=bool)
    inner[sl] = True
    assert np.all(gf[~inner] == 0)
    d = gf[sl] - gf_o
    assert np.linalg.norm(d) <= 1e-3 * np.linalg.norm(gf_o), (np.linalg.norm(d), np.linalg.norm(gf_o))


def test_primal_dual_stops_at_a_check_with_the_cold_iterate(f_ds):
    """The primal-dual solver's shared-memory iteration on the same image:
    a tolerance between two checks stops it at the right check, with the
    bits of a cold solve of that many iterations."""
    seg = seg_mod()
    S = _solver(f_ds)
    norms = []
    for l in range(5, 155, 5):
        st = S.solve_pd(LAM, iters=l, check_every=5).cpu().numpy()
        norms.append(max(st[1], st[2]))
        assert st[7] > 0, st
    norms = np.array(norms)
    k = next(k for k in range(6, len(norms)) if norms[:k].min() > 1.05 * norms[k])
    tol = float(np.sqrt(norms[:k].min() * norms[k]))
    stop = 5 * (k + 1)
    S.solve_pd(LAM, iters=stop, check_every=5)
    torch.cuda.synchronize()
    ref = {n: seg.download(getattr(S, n)).copy() for n in ("u", "p1", "p2")}
    st = S.solve_pd(LAM, iters=600, tol=tol, check_every=5).cpu().numpy()
    torch.cuda.synchronize()
    S.check_status()
    assert int(st[0]) == stop and int(st[5]) == stop
    for n in ref:
        np.testing.assert_array_equal(seg.download(getattr(S, n)), ref[n], err_msg=n)


def test_two_barrier_shared_memory_path_when_the_ring_does_not_fit(orc, f_ds):
    """At |RD|/N = 0.225 (3,105 pixels per 512-thread block at tile height
    16) the blocks' state fits in shared memory without the ring but not
    with it:
    the grid vote sends every block to the two-barrier shared-memory
    iteration.  Every pixel against the dense solver on the same domain."""
    seg = seg_mod()
    K, q = 40, 0.225
    out = {}
    for mode in ("compact", "dense"):
        S = seg.Solver(H, W, tile_h=16, mode=mode)
        S.f[:, :W].copy_(torch.from_numpy(f_ds))
        S.domain(q=q)
        st = S.solve(LAM, iters=K).cpu().numpy()
        out[mode] = (_state(S), st)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    st = out["compact"][1]
    assert st[7] == 0 and st[6] >= sms and st[6] % sms == 0, st
    for k in ("u", "v", "p1", "p2"):
        d = np.abs(out["compact"][0][k].astype(np.float64) - out["dense"][0][k])
        assert d.max() <= 1e-4, (k, d.max())
