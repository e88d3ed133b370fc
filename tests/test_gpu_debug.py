"""Debugging aids of the library, on the GPU: the synchronous debug mode
(SEG_DEBUG=1 in the environment: every launch of a public call is followed by
a stream synchronisation and a read of the workspace's status word, so the
call that raised a device-side error returns it and names the launch), and
poisoned padding (NaN in the columns W..ld-1 of every image must neither
reach the results nor be overwritten)."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_1807_11534_gb300 import synth
from tests.gpu_helpers import require_gpu, seg_mod

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_1807_11534_gb300 import seg, synth
seg.load()
out = {}
f = np.random.default_rng(2).normal(0, 0.2, (64, 64)).astype(np.float32)
# a capacity overflow, recorded on the device by the compact gather
S = seg.Solver(64, 64, tile_h=16, mode="compact", capacity=10)
S.f[:, :64].copy_(torch.from_numpy(f))
S.domain(delta=0.2)
try:
    S.solve(1.0, iters=5)
    out["overflow"] = None
except seg.SegError as e:
    out["overflow"] = [e.status, str(e)]
# a normal solve: same bits as without the debug mode
P = synth.small_example(seed=3, H=70, W=90)
T = seg.Solver(70, 90, tile_h=16, mode="compact")
T.fitting(seg.upload(P.z), 0.3, 0.7)
T.domain(delta=0.15)
T.solve(1.0, iters=40, check_every=10)
torch.cuda.synchronize()
T.check_status()
out["u"] = seg.download(T.u).astype(np.float64).tolist()
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    seg_mod()


def _run_child(debug):
    env = dict(os.environ)
    if debug:
        env["SEG_DEBUG"] = "1"
    else:
        env.pop("SEG_DEBUG", None)
    r = subprocess.run([sys.executable, "-c", _CHILD.replace("ROOT", repr(ROOT))], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_mode_reports_a_device_error_at_the_call_that_raised_it():
    seg = seg_mod()
    dbg = _run_child(True)
    assert dbg["overflow"] is not None, "the solve itself must fail in debug mode"
    status, msg = dbg["overflow"]
    assert status == seg.SEG_ERR_CAPACITY
    assert "k_batch_bases" in msg and "debug check" in msg
    plain = _run_child(False)
    assert plain["overflow"] is None          # reported only at the next status read
    np.testing.assert_array_equal(np.array(dbg["u"]), np.array(plain["u"]))


def _poison(t, W):
    if t.shape[1] > W:
        t[:, W:] = float("nan")


@pytest.mark.parametrize("mode,delta", [("compact", 0.15), ("dense", 0.15), ("tiled", math.inf),
                                        ("compact", math.inf)])
def test_poisoned_padding_is_neither_read_nor_written(orc, mode, delta):
    """W = 75 (ld = 96): NaN in columns 75..95 of z, f, u, v, p1, p2 before the
    fitting term, the domain and the solve; the results equal those of the
    clean run bit for bit and the padding is still NaN afterwards."""
    seg = seg_mod()
    H, W = 61, 75
    P = synth.small_example(seed=7, H=H, W=W)
    outs = []
    for poison in (False, True):
        S = seg.Solver(H, W, tile_h=16, mode=mode)
        z = seg.upload(P.z)
        if poison:
            for t in (z, S.f, S.u, S.v, S.p1, S.p2):
                _poison(t, W)
        S.fitting(z, 0.3, 0.7)
        S.domain(delta=delta)
        S.solve(1.0, iters=30, check_every=10)
        S.energy(1.0)
        torch.cuda.synchronize()
        S.check_status()
        outs.append({k: getattr(S, k).cpu().numpy().copy() for k in ("f", "u", "v", "p1", "p2")} |
                    {"e": S.energy_out.cpu().numpy().copy()})
    clean, dirty = outs
    for k in ("f", "u", "v", "p1", "p2"):
        np.testing.assert_array_equal(dirty[k][:, :W], clean[k][:, :W])
        assert np.all(np.isnan(dirty[k][:, W:])), k
    np.testing.assert_array_equal(dirty["e"], clean["e"])
