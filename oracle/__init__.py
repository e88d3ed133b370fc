"""FP64 CPU oracle for the restricted-domain dual TV segmentation (arXiv 1807.11534).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its binding) never imports it, and it shares no code with them.

The arithmetic lives in plain C (``seg_oracle.c``, compiled with FMA
contraction off so every FP64 operation is one IEEE rounding); this module
only compiles it and marshals numpy arrays in and out.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_OMP_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc).

    SEG_ORACLE_LIB names a prebuilt copy instead (used to check that the pins
    fail on a deliberately mutated oracle)."""
    if os.environ.get("SEG_ORACLE_LIB"):
        return os.environ["SEG_ORACLE_LIB"]
    os.makedirs(_OUT_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "seg_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_omp(force: bool = False) -> str | None:
    """The same source compiled with -fopenmp into liboracle_omp.so: the
    row and pixel loops of the solve run on all cores; every output element
    is computed by the same operations as in the serial build and the
    increments are summed per row, then over rows in order, so both builds
    give identical bits.  Returns None when the compiler has no OpenMP."""
    if os.environ.get("SEG_ORACLE_LIB"):
        return None
    os.makedirs(_OUT_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "seg_oracle.h")
    if (not force and os.path.exists(_OMP_PATH)
            and os.path.getmtime(_OMP_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _OMP_PATH
    tmp = _OMP_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                              stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        return None
    os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def threads() -> int:
    """Cores the OpenMP build uses (the process's CPU affinity, unless
    OMP_NUM_THREADS says otherwise)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit():
        return int(env)
    return len(os.sched_getaffinity(0))


def has_omp() -> bool:
    return build_omp() is not None


def _load(omp: bool = False):
    global _lib, _omp_lib
    with _lock:
        if omp:
            if _omp_lib is not None:
                return _omp_lib
            path = build_omp()
            if path is None:
                raise RuntimeError("the OpenMP build of the oracle is not available")
        elif _lib is not None:
            return _lib
        else:
            path = build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I, L, D, F = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        lib.oracle_fitting.argtypes = [P, I, I, D, D, P, I, D, P, P]
        lib.oracle_fitting.restype = None
        lib.oracle_class_means.argtypes = [P, P, L, P, P]
        lib.oracle_class_means.restype = None
        lib.oracle_update_means.argtypes = [P, P, L, D, P, P]
        lib.oracle_update_means.restype = None
        lib.oracle_quantile_delta.argtypes = [P, L, D]
        lib.oracle_quantile_delta.restype = F
        lib.oracle_domain.argtypes = [P, L, F, P]
        lib.oracle_domain.restype = None
        lib.oracle_box_mean.argtypes = [P, I, I, I, P]
        lib.oracle_box_mean.restype = None
        lib.oracle_domain_robust.argtypes = [P, P, L, F, P]
        lib.oracle_domain_robust.restype = None
        lib.oracle_dilate.argtypes = [P, I, I, I, P]
        lib.oracle_dilate.restype = None
        lib.oracle_pixel_list.argtypes = [P, L, P]
        lib.oracle_pixel_list.restype = L
        lib.oracle_tile_list.argtypes = [P, I, I, I, I, P]
        lib.oracle_tile_list.restype = L
        lib.oracle_pixel_list_tiled.argtypes = [P, I, I, I, I, P]
        lib.oracle_pixel_list_tiled.restype = L
        lib.oracle_grad.argtypes = [P, I, I, P, P]
        lib.oracle_grad.restype = None
        lib.oracle_div.argtypes = [P, P, I, I, P]
        lib.oracle_div.restype = None
        lib.oracle_solve.argtypes = [P, I, I, P, D, D, D, I, I, D, I, P, P, P, P, P]
        lib.oracle_solve.restype = I
        lib.oracle_solve_grad.argtypes = [P, I, I, P, D, D, D, I, P, P, P, P]
        lib.oracle_grad3.argtypes = [P, I, I, I, P, P, P]
        lib.oracle_grad3.restype = None
        lib.oracle_div3.argtypes = [P, P, P, I, I, I, P]
        lib.oracle_div3.restype = None
        lib.oracle_solve3.argtypes = [P, I, I, I, P, D, D, D, I, D, I, P, P, P, P, P, P]
        lib.oracle_solve3.restype = ctypes.c_int
        lib.oracle_solve_pd.argtypes = [P, I, I, P, D, D, D, I, D, I, P, P, P, P]
        lib.oracle_solve_pd.restype = ctypes.c_int
        lib.oracle_solve_grad.restype = None
        lib.oracle_energy.argtypes = [P, P, P, P, P, I, I, D, D, P]
        lib.oracle_energy.restype = None
        lib.oracle_errors.argtypes = [P, P, L, D, P]
        lib.oracle_errors.restype = None
        if omp:
            _omp_lib = lib
        else:
            _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ------------------------------------------------------------------ wrappers

def fitting(z, c1, c2, markers=None, gamma=0.0):
    """Eq. CV / Eq. DS in FP64; returns (f64, f32) with f32 = round(f64)."""
    lib = _load()
    z = _c(z, np.float32)
    H, W = z.shape
    m = _c(markers if markers is not None else np.zeros((0, 2)), np.int32).reshape(-1, 2)
    f64 = np.empty((H, W), np.float64)
    f32 = np.empty((H, W), np.float32)
    lib.oracle_fitting(_ptr(z), H, W, float(c1), float(c2), _ptr(m) if len(m) else None,
                       len(m), float(gamma), _ptr(f64), _ptr(f32))
    return f64, f32


def class_means(z, label):
    lib = _load()
    z = _c(z, np.float32)
    lab = _c(label, np.uint8)
    c1, c2 = ctypes.c_double(), ctypes.c_double()
    lib.oracle_class_means(_ptr(z), _ptr(lab), z.size, ctypes.byref(c1), ctypes.byref(c2))
    return c1.value, c2.value


def update_means(z, u, thresh, c1, c2):
    """Chan-Vese intensity update: (mean of z over u > thresh, mean over
    u <= thresh); a class without pixels keeps c1 resp. c2."""
    lib = _load()
    z = _c(z, np.float32)
    uu = _c(u, np.float64)
    a, b = ctypes.c_double(c1), ctypes.c_double(c2)
    lib.oracle_update_means(_ptr(z), _ptr(uu), z.size, float(thresh), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def chan_vese(z, c1, c2, lam, outer, iters, delta=float("inf"), q=-1.0, thresh=0.5, theta=0.2,
              tau=0.125):
    """Chan-Vese loop on the restricted solve: for t = 0 .. outer-1, the
    fitting term of Eq. CV with (c1, c2), its domain (delta, or quantile q),
    `iters` iterations warm-started from the previous solve, then the
    intensity update from u.  Returns (state of the last solve, the (c1, c2)
    that solve used, the list of (c1, c2) per outer step)."""
    st, used = None, []
    for t in range(outer):
        if t > 0:
            c1, c2 = update_means(z, st.u, thresh, c1, c2)
        used.append((c1, c2))
        _, f = fitting(z, c1, c2)
        d = quantile_delta(f, q) if q >= 0 else delta
        st = solve(f, domain(f, d), lam, theta, tau, iters, state=st)
    return st, (c1, c2), used


def quantile_delta(f32, q):
    lib = _load()
    f = _c(f32, np.float32)
    return float(np.float32(lib.oracle_quantile_delta(_ptr(f), f.size, float(q))))


def domain(f32, delta):
    """Region codes (0 Bg, 1 Fg, 2 RD) for threshold `delta` (float32)."""
    lib = _load()
    f = _c(f32, np.float32)
    reg = np.empty(f.shape, np.uint8)
    lib.oracle_domain(_ptr(f), f.size, float(np.float32(delta)), _ptr(reg))
    return reg


def box_mean(f32, r):
    """Local mean of f over (2r+1)^2 squares clipped to the image (float32)."""
    lib = _load()
    f = _c(f32, np.float32)
    H, W = f.shape
    out = np.empty_like(f)
    lib.oracle_box_mean(_ptr(f), H, W, int(r), _ptr(out))
    return out


def domain_robust(f32, fbar, delta):
    """Robust partition: RD = {|fbar| < delta} plus sign disagreements of f and fbar."""
    lib = _load()
    f = _c(f32, np.float32)
    m = _c(fbar, np.float32)
    reg = np.empty(f.shape, np.uint8)
    lib.oracle_domain_robust(_ptr(f), _ptr(m), f.size, float(np.float32(delta)), _ptr(reg))
    return reg


def robust_region(f32, delta=None, q=-1.0, smooth=0, radius=0):
    """The partition seg_build_domain_robust builds: threshold on the local mean
    (smooth > 0) or on f, delta from q's quantile when q >= 0, then dilation."""
    fbar = box_mean(f32, smooth) if smooth else _c(f32, np.float32)
    d = quantile_delta(fbar, q) if q >= 0 else delta
    reg = domain_robust(f32, fbar, d) if smooth else domain(f32, d)
    return dilate(reg, radius) if radius else reg


def dilate(region, r):
    """RD grown by Chebyshev distance r (robust restriction, Conclusion)."""
    lib = _load()
    reg = _c(region, np.uint8)
    H, W = reg.shape
    out = np.empty_like(reg)
    lib.oracle_dilate(_ptr(reg), H, W, int(r), _ptr(out))
    return out


def pixel_list(region):
    lib = _load()
    r = _c(region, np.uint8)
    n = lib.oracle_pixel_list(_ptr(r), r.size, None)
    out = np.empty(max(n, 1), np.int32)
    lib.oracle_pixel_list(_ptr(r), r.size, _ptr(out))
    return out[:n]


def tile_list(region, th, tw):
    lib = _load()
    r = _c(region, np.uint8)
    H, W = r.shape
    n = lib.oracle_tile_list(_ptr(r), H, W, th, tw, None)
    out = np.empty(max(n, 1), np.int32)
    lib.oracle_tile_list(_ptr(r), H, W, th, tw, _ptr(out))
    return out[:n]


def pixel_list_tiled(region, th, tw=32):
    lib = _load()
    r = _c(region, np.uint8)
    H, W = r.shape
    n = lib.oracle_pixel_list_tiled(_ptr(r), H, W, th, tw, None)
    out = np.empty(max(n, 1), np.int32)
    lib.oracle_pixel_list_tiled(_ptr(r), H, W, th, tw, _ptr(out))
    return out[:n]


def grad(w):
    lib = _load()
    w = _c(w, np.float64)
    H, W = w.shape
    g1, g2 = np.empty_like(w), np.empty_like(w)
    lib.oracle_grad(_ptr(w), H, W, _ptr(g1), _ptr(g2))
    return g1, g2


def div(p1, p2):
    lib = _load()
    p1, p2 = _c(p1, np.float64), _c(p2, np.float64)
    H, W = p1.shape
    d = np.empty_like(p1)
    lib.oracle_div(_ptr(p1), _ptr(p2), H, W, _ptr(d))
    return d


class State:
    """Oracle iterate (u, v, p1, p2) in FP64 plus the per-iteration increments."""

    def __init__(self, u, v, p1, p2, iters_done, hist):
        self.u, self.v, self.p1, self.p2 = u, v, p1, p2
        self.iters_done = iters_done
        self.hist = hist

    def copy(self):
        return State(self.u.copy(), self.v.copy(), self.p1.copy(), self.p2.copy(),
                     self.iters_done, self.hist.copy())


def solve(f32, region, lam, theta=0.2, tau=0.125, iters=100, n_inner=1, tol=0.0,
          state: State | None = None, parallel: bool = False) -> State:
    """Run the restricted dual iteration (Section 3); warm-starts from `state`.
    parallel: use the OpenMP build (same results, all cores)."""
    lib = _load(omp=parallel)
    f = _c(f32, np.float32)
    reg = _c(region, np.uint8)
    H, W = f.shape
    if state is None:
        u = np.zeros((H, W)); v = np.zeros((H, W)); p1 = np.zeros((H, W)); p2 = np.zeros((H, W))
        warm = 0
    else:
        u, v, p1, p2 = (_c(a, np.float64).copy() for a in (state.u, state.v, state.p1, state.p2))
        warm = 1
    hist = np.zeros((max(iters, 1), 2))
    done = lib.oracle_solve(_ptr(f), H, W, _ptr(reg), float(lam), float(theta), float(tau),
                            int(iters), int(n_inner), float(tol), warm,
                            _ptr(u), _ptr(v), _ptr(p1), _ptr(p2), _ptr(hist))
    return State(u, v, p1, p2, done, hist[:done])


def grad3(w):
    lib = _load()
    w = _c(w, np.float64)
    D, H, W = w.shape
    g = [np.empty_like(w) for _ in range(3)]
    lib.oracle_grad3(_ptr(w), D, H, W, *(_ptr(x) for x in g))
    return tuple(g)


def div3(p1, p2, p3):
    lib = _load()
    ps = [_c(x, np.float64) for x in (p1, p2, p3)]
    D, H, W = ps[0].shape
    d = np.empty_like(ps[0])
    lib.oracle_div3(*(_ptr(x) for x in ps), D, H, W, _ptr(d))
    return d


class State3:
    """Oracle iterate of a volume: u, v, p1, p2, p3 (FP64) and the increments."""

    def __init__(self, u, v, p1, p2, p3, iters_done, hist):
        self.u, self.v, self.p1, self.p2, self.p3 = u, v, p1, p2, p3
        self.iters_done = iters_done
        self.hist = hist


def solve3(f32, region, lam, theta=0.2, tau=0.125, iters=100, tol=0.0,
           state: State3 | None = None) -> State3:
    """Section 3's iteration on a [D][H][W] volume (region codes per voxel)."""
    lib = _load()
    f = _c(f32, np.float32)
    reg = _c(region, np.uint8)
    D, H, W = f.shape
    if state is None:
        arrs = [np.zeros((D, H, W)) for _ in range(5)]
        warm = 0
    else:
        arrs = [_c(a, np.float64).copy() for a in (state.u, state.v, state.p1, state.p2, state.p3)]
        warm = 1
    hist = np.zeros((max(iters, 1), 2))
    done = lib.oracle_solve3(_ptr(f), D, H, W, _ptr(reg), float(lam), float(theta), float(tau),
                             int(iters), float(tol), warm, *(_ptr(a) for a in arrs), _ptr(hist))
    return State3(*arrs, done, hist[:done])


PD_STEP = 1.0 / math.sqrt(8.0)   # sigma = tau = 1/sqrt(8): sigma tau ||grad||^2 <= 1


def solve_pd(f32, region, lam, sigma=PD_STEP, tau=PD_STEP, iters=100, tol=0.0,
             state: State | None = None) -> State:
    """Restricted primal-dual (Chambolle-Pock) solve of Eq. CR on the same
    partition; v of the returned state is u (the method has no v)."""
    lib = _load()
    f = _c(f32, np.float32)
    reg = _c(region, np.uint8)
    H, W = f.shape
    if state is None:
        u = np.zeros((H, W)); p1 = np.zeros((H, W)); p2 = np.zeros((H, W))
        warm = 0
    else:
        u, p1, p2 = (_c(a, np.float64).copy() for a in (state.u, state.p1, state.p2))
        warm = 1
    hist = np.zeros((max(iters, 1), 2))
    done = lib.oracle_solve_pd(_ptr(f), H, W, _ptr(reg), float(lam), float(sigma), float(tau),
                               int(iters), float(tol), warm, _ptr(u), _ptr(p1), _ptr(p2), _ptr(hist))
    return State(u, u, p1, p2, done, hist[:done])


def solve_grad(f32, region, lam, gu, gv=None, theta=0.2, tau=0.125, iters=20):
    """(dL/df, dL/dlambda) for L = <gu, u^K> + <gv, v^K> (reverse mode)."""
    lib = _load()
    f = _c(f32, np.float32)
    reg = _c(region, np.uint8)
    H, W = f.shape
    gu = _c(gu, np.float64)
    gvv = _c(gv, np.float64) if gv is not None else None
    gf = np.zeros((H, W))
    glam = ctypes.c_double()
    lib.oracle_solve_grad(_ptr(f), H, W, _ptr(reg), float(lam), float(theta), float(tau), int(iters),
                          _ptr(gu), _ptr(gvv), _ptr(gf), ctypes.byref(glam))
    return gf, glam.value


def energy(u, v, p1, p2, f32, lam, theta=0.2):
    """dict with TV(u), E_CR(u), E_CR(v), E_DF, dual bound D(p) and gap."""
    lib = _load()
    f = _c(f32, np.float32)
    H, W = f.shape
    arrs = [_c(a, np.float64) for a in (u, v, p1, p2)]
    out = np.zeros(6)
    lib.oracle_energy(*(_ptr(a) for a in arrs), _ptr(f), H, W, float(lam), float(theta), _ptr(out))
    return dict(tv=out[0], ecr_u=out[1], ecr_v=out[2], edf=out[3], dual=out[4], gap=out[5])


def errors(u_star, u_gt, eps=0.5):
    """(E1, E2) of Section 4."""
    lib = _load()
    a, b = _c(u_star, np.float64), _c(u_gt, np.float64)
    out = np.zeros(2)
    lib.oracle_errors(_ptr(a), _ptr(b), a.size, float(eps), _ptr(out))
    return float(out[0]), float(out[1])


def pipeline(problem, delta=None, q=None, iters=None, n_inner=1, tol=0.0):
    """Fitting -> domain -> solve for a synthetic problem; returns a dict."""
    import math
    c1, c2 = problem.c1, problem.c2
    if math.isnan(c1) or math.isnan(c2):
        c1, c2 = class_means(problem.z, problem.label)
    _, f32 = fitting(problem.z, c1, c2, problem.markers if problem.gamma else None,
                     problem.gamma)
    if q is None and delta is None:
        q = problem.q if problem.q >= 0 else None
        delta = problem.delta
    if q is not None and q >= 0:
        delta = quantile_delta(f32, q)
    reg = domain(f32, np.float32(delta) if np.isfinite(delta) else np.float32(np.inf))
    st = solve(f32, reg, problem.lam, problem.theta, problem.tau,
               problem.iters if iters is None else iters, n_inner, tol)
    return dict(c1=c1, c2=c2, f32=f32, delta=delta, region=reg, state=st)
