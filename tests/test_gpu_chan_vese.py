"""The Chan-Vese loop on the restricted solve (seg_update_means between
solves, seg_make_fitting with the means kept on the device) against the
FP64 oracle's loop."""
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


def test_update_means_on_the_solvers_u(orc):
    """The class means of z over the GPU's own u (the decision u > 0.5 is the
    same in float32 and FP64 for a float32 u), and an empty class keeping the
    value the workspace held."""
    seg = seg_mod()
    P = synth.small_example(seed=2, H=70, W=90)
    S = seg.Solver(70, 90, mode="compact")
    z = seg.upload(P.z)
    S.fitting(z, 0.3, 0.7)
    S.domain(delta=0.2)
    S.solve(1.0, iters=50)
    S.update_means(z)
    torch.cuda.synchronize()
    u = seg.download(S.u).astype(np.float64)
    c1, c2 = orc.update_means(P.z, u, 0.5, 0.3, 0.7)
    got = S.c.cpu().numpy()
    assert got[0] == pytest.approx(c1, rel=1e-12) and got[1] == pytest.approx(c2, rel=1e-12)
    # all of u below the threshold: c1 keeps its value
    S.u.zero_()
    S.fitting(z, 0.25, 0.75)
    S.update_means(z)
    got = S.c.cpu().numpy()
    assert got[0] == 0.25 and got[1] == pytest.approx(float(np.mean(P.z.astype(np.float64))), rel=1e-12)


def test_fitting_with_the_stored_means_is_bit_exact(orc):
    seg = seg_mod()
    P = synth.small_example(seed=3, H=40, W=50)
    S = seg.Solver(40, 50, mode="compact")
    z = seg.upload(P.z)
    S.fitting(z, 0.31, 0.68)
    S.fitting(z, math.nan, math.nan)
    _, f = orc.fitting(P.z, 0.31, 0.68)
    np.testing.assert_array_equal(seg.download(S.f), f)
    assert S.c.cpu().numpy().tolist() == [0.31, 0.68]


@pytest.mark.parametrize("mode,kw", [("compact", dict(delta=0.2)), ("compact", dict(q=0.3)),
                                     ("dense", dict(delta=math.inf)), ("tiled", dict(delta=0.15))])
def test_chan_vese_loop_matches_the_oracle(orc, mode, kw):
    seg = seg_mod()
    P = synth.small_example(seed=7, H=96, W=128)
    outer, iters, lam = 4, 80, 1.0
    S = seg.Solver(96, 128, mode=mode)
    z = seg.upload(P.z)
    S.chan_vese(z, lam, 0.35, 0.62, outer=outer, iters=iters, **kw)
    torch.cuda.synchronize()
    S.check_status()
    st, used, hist = orc.chan_vese(P.z, 0.35, 0.62, lam, outer, iters, delta=kw.get("delta", math.inf),
                                   q=kw.get("q", -1.0))
    got_c = S.c.cpu().numpy()
    assert got_c[0] == pytest.approx(used[0], rel=1e-6) and got_c[1] == pytest.approx(used[1], rel=1e-6)
    u = seg.download(S.u).astype(np.float64)
    assert np.max(np.abs(u - st.u)) <= 1e-4
    assert np.array_equal(u > 0.5, st.u > 0.5)
