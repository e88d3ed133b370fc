"""Python binding of libseg (include/seg.h): the same entry points, argument
marshalling only.

Every ``seg_*`` function here forwards to the C ABI with raw device pointers
taken from torch tensors and the current torch CUDA stream; all arithmetic runs
in the CUDA kernels of libseg.  There is no CPU fallback: if the library cannot
be loaded the import raises.

Higher up, ``Solver`` (one image), ``BatchSolver``, ``DiffSolver`` (with
the adjoint), ``VolumeSolver`` (3-D) and ``capture_graph`` only allocate
buffers (through torch), chain the entry points and record their launches.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import torch

from . import build as _build

SEG_OK = 0
SEG_ERR_INVALID_ARG = 1
SEG_ERR_ALIGN = 2
SEG_ERR_CUDA = 3
SEG_ERR_CAPACITY = 4
SEG_ERR_TIMEOUT = 5
SEG_ERR_NONFINITE = 6
SEG_ERR_WORKSPACE = 7

SEG_MODE_DENSE = 0
SEG_MODE_COMPACT = 1
SEG_MODE_TILED = 2
_MODE_BY_NAME = {"dense": SEG_MODE_DENSE, "compact": SEG_MODE_COMPACT, "tiled": SEG_MODE_TILED}
SEG_STORE_F32 = 0
SEG_STORE_BF16 = 1
SEG_STORE_F16 = 2

_STORE_BY_NAME = {"f32": SEG_STORE_F32, "fp32": SEG_STORE_F32, "bf16": SEG_STORE_BF16,
                  "f16": SEG_STORE_F16, "fp16": SEG_STORE_F16}


class SegError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libseg status {status}: {msg}")
        self.status = status


class seg_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("theta", ctypes.c_double),
                ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("iters", ctypes.c_int), ("n_inner", ctypes.c_int),
                ("check_every", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("mode", ctypes.c_int), ("storage", ctypes.c_int),
                ("tile_h", ctypes.c_int), ("sweep", ctypes.c_int)]


class seg_pd_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("tile_h", ctypes.c_int)]


PD_STEP = 1.0 / math.sqrt(8.0)   # sigma = tau = 1/sqrt(8): sigma tau ||grad||^2 <= 1


class seg_image(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("ld", ctypes.c_int), ("act", ctypes.c_void_p), ("fg", ctypes.c_void_p),
                ("wstart", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("p1", ctypes.c_void_p), ("p2", ctypes.c_void_p),
                ("lambda_", ctypes.c_double)]


class seg_adj_image(ctypes.Structure):
    _fields_ = [("grad_u", ctypes.c_void_p), ("grad_v", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("grad_f", ctypes.c_void_p), ("grad_out", ctypes.c_void_p)]


_lib = None

# exported entry points and their C signatures (include/seg.h)
_P, _I, _L, _D, _F, _Z = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                          ctypes.c_float, ctypes.c_size_t)
SIGNATURES = {
    "seg_version": ([], _I),
    "seg_last_error": ([], ctypes.c_char_p),
    "seg_launch_count": ([], ctypes.c_ulonglong),
    "seg_workspace_bytes": ([_I, _I, _I, _I], _Z),
    "seg_state_bytes": ([_I, _I, _L, _I, _I], _Z),
    "seg_read_status": ([_P, _Z, _P], _I),
    "seg_make_fitting": ([_P, _I, _I, _I, _D, _D, _P, _P, _I, _D, _P, _P, _P, _Z, _P], _I),
    "seg_build_domain": ([_P, _I, _I, _I, _D, _D, _I, _P, _P, _P, _P, _I, _P, _L, _P, _P, _P, _Z, _P], _I),
    "seg_build_domain_robust": ([_P, _P, _I, _I, _I, _D, _D, _I, _I, _P, _P, _P, _P, _I, _P, _L, _P,
                                 _P, _P, _Z, _P], _I),
    "seg_box_mean": ([_P, _I, _I, _I, _I, _P, _P], _I),
    "seg_update_means": ([_P, _P, _I, _I, _I, _D, _P, _P, _Z, _P], _I),
    "seg_solve": ([_P, _I, _I, _I, _P, _P, _P, _P, _P, ctypes.POINTER(seg_params),
                   _P, _P, _P, _P, _P, _Z, _P, _P, _Z, _P], _I),
    "seg_energy": ([_P, _I, _I, _I, _P, _P, _P, _P, _D, _D, _P, _P, _Z, _P], _I),
    "seg_errors": ([_P, _P, _I, _I, _I, _D, _P, _P, _Z, _P], _I),
    "seg_energy_noalloc": ([_P, _I, _I, _I, _P, _P, _P, _P, _D, _D, _P, _P], _I),
    "seg_batch_workspace_bytes": ([_I, _L], _Z),
    "seg_ckpt_bytes": ([_L, _I, _I], _Z),
    "seg_backward_scratch_bytes": ([_L, _I], _Z),
    "seg_solve_diff": ([_P, _I, _I, _I, _P, _P, _P, _P, _P, ctypes.POINTER(seg_params), _P, _P, _P, _P,
                        _P, _Z, _I, _P, _Z, _P, _P, _Z, _P], _I),
    "seg_backward": ([_P, _I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(seg_params), _P, _Z, _P, _Z, _I,
                      _P, _P, _P, _P, _P, _P, _P, _Z, _P, _Z, _P], _I),
    "seg_solve_pd": ([_P, _I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(seg_pd_params), _P, _P, _P, _P,
                      _Z, _P, _P, _Z, _P], _I),
    "seg_state_bytes3d": ([_L], _Z),
    "seg_solve3d": ([_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, ctypes.POINTER(seg_params), _P, _P, _P, _P,
                     _P, _P, _Z, _P, _P, _Z, _P], _I),
    "seg_solve_batch": ([ctypes.POINTER(seg_image), _I, ctypes.POINTER(seg_params), _P, _Z, _P, _P, _Z,
                         _P], _I),
    "seg_solve_diff_batch": ([ctypes.POINTER(seg_image), _I, ctypes.POINTER(seg_params), _P, _Z, _I, _P, _Z,
                              _P, _P, _Z, _P], _I),
    "seg_backward_batch": ([ctypes.POINTER(seg_image), ctypes.POINTER(seg_adj_image), _I,
                            ctypes.POINTER(seg_params), _P, _Z, _P, _Z, _I, _P, _Z, _P, _Z, _P], _I),
    "seg_set_wait_limit": ([_P, _Z, ctypes.c_longlong, _I, _P], _I),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libseg.so (building it first if needed).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"libseg not built at {path}")
        _build.build()
    if torch.cuda.is_available():
        torch.cuda.init()   # share torch's CUDA runtime / primary context
    lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(st):
    if st != SEG_OK:
        msg = _lib.seg_last_error().decode(errors="replace")
        raise SegError(st, msg)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("libseg takes device tensors only")
    return t.data_ptr()


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ----------------------------------------------------------- thin wrappers

def seg_version():
    return load().seg_version()


def seg_launch_count():
    return load().seg_launch_count()


def seg_workspace_bytes(H, W, ld, tile_h):
    return load().seg_workspace_bytes(H, W, ld, tile_h)


def seg_state_bytes(H, ld, capacity, mode, storage):
    return load().seg_state_bytes(H, ld, capacity, mode, storage)


def seg_read_status(ws, stream=None):
    lib = load()
    _check(lib.seg_read_status(_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def seg_set_wait_limit(ws, wait_cycles, extra_arrivals=0, stream=None):
    _check(load().seg_set_wait_limit(_ptr(ws), _nbytes(ws), int(wait_cycles), int(extra_arrivals),
                                     _stream(stream)))


def seg_make_fitting(z, c1, c2, label, markers, gamma, f, c_out, ws, stream=None):
    lib = load()
    n_markers = 0 if markers is None else markers.shape[0]
    _check(lib.seg_make_fitting(_ptr(z), z.shape[0], _W(z), z.stride(0), float(c1), float(c2), _ptr(label),
                                _ptr(markers), n_markers, float(gamma), _ptr(f), _ptr(c_out),
                                _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_update_means(z, u, thresh, c_out, ws, stream=None):
    _check(load().seg_update_means(_ptr(z), _ptr(u), z.shape[0], _W(z), z.stride(0), float(thresh),
                                   _ptr(c_out), _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_build_domain(f, delta, q, tile_h, act, fg, wstart, tiles, pixels, counts, delta_out, ws,
                     stream=None):
    lib = load()
    _check(lib.seg_build_domain(_ptr(f), f.shape[0], _W(f), f.stride(0), float(delta), float(q),
                                int(tile_h), _ptr(act), _ptr(fg), _ptr(wstart), _ptr(tiles),
                                tiles.numel(), _ptr(pixels),
                                0 if pixels is None else pixels.numel(), _ptr(counts),
                                _ptr(delta_out), _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_solve_pd(f, act, fg, wstart, counts, params: seg_pd_params, u, p1, p2, state, stats, ws,
                 stream=None):
    lib = load()
    _check(lib.seg_solve_pd(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(act), _ptr(fg), _ptr(wstart),
                            _ptr(counts), ctypes.byref(params), _ptr(u), _ptr(p1), _ptr(p2), _ptr(state),
                            _nbytes(state), _ptr(stats), _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_state_bytes3d(capacity):
    return load().seg_state_bytes3d(int(capacity))


def seg_solve3d(f, D, H, act, fg, wstart, voxels, counts, params: seg_params, u, v, p1, p2, p3, state,
                stats, ws, stream=None):
    """f, u, v, p1, p2, p3: [D*H][ld] stacked volume images; wstart, voxels:
    seg_build_domain's compact starts and RD voxel list for the stacked image."""
    lib = load()
    _check(lib.seg_solve3d(_ptr(f), int(D), int(H), _W(f), f.stride(0), _ptr(act), _ptr(fg), _ptr(wstart),
                           _ptr(voxels),
                           _ptr(counts), ctypes.byref(params), _ptr(u), _ptr(v), _ptr(p1), _ptr(p2),
                           _ptr(p3), _ptr(state), _nbytes(state), _ptr(stats), _ptr(ws), _nbytes(ws),
                           _stream(stream)))


def seg_build_domain_robust(f, fbar, delta, q, radius, tile_h, act, fg, wstart, tiles, pixels,
                            counts, delta_out, ws, stream=None):
    lib = load()
    _check(lib.seg_build_domain_robust(_ptr(f), _ptr(fbar), f.shape[0], _W(f), f.stride(0),
                                       float(delta), float(q), int(radius), int(tile_h), _ptr(act),
                                       _ptr(fg), _ptr(wstart), _ptr(tiles), tiles.numel(),
                                       _ptr(pixels), 0 if pixels is None else pixels.numel(),
                                       _ptr(counts), _ptr(delta_out), _ptr(ws), _nbytes(ws),
                                       _stream(stream)))


def seg_box_mean(f, radius, out, stream=None):
    _check(load().seg_box_mean(_ptr(f), f.shape[0], _W(f), f.stride(0), int(radius), _ptr(out),
                               _stream(stream)))


def _build_into(f, delta, q, radius, tile_h, d, ws, stream, fbar=None):
    if radius or fbar is not None:
        seg_build_domain_robust(f, fbar, delta, q, radius, tile_h, d.act, d.fg, d.wstart, d.tiles,
                                d.pixels, d.counts, d.delta, ws, stream)
    else:
        seg_build_domain(f, delta, q, tile_h, d.act, d.fg, d.wstart, d.tiles, d.pixels, d.counts,
                         d.delta, ws, stream)


def seg_solve(f, act, fg, wstart, tiles, counts, params: seg_params, u, v, p1, p2, state, stats,
              ws, stream=None):
    lib = load()
    _check(lib.seg_solve(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(act), _ptr(fg), _ptr(wstart),
                         _ptr(tiles), _ptr(counts), ctypes.byref(params), _ptr(u), _ptr(v), _ptr(p1),
                         _ptr(p2), _ptr(state), _nbytes(state), _ptr(stats), _ptr(ws), _nbytes(ws),
                         _stream(stream)))


def seg_energy(f, u, v, p1, p2, lam, theta, out, ws, stream=None):
    lib = load()
    _check(lib.seg_energy(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(u), _ptr(v), _ptr(p1),
                          _ptr(p2), float(lam), float(theta), _ptr(out), _ptr(ws), _nbytes(ws),
                          _stream(stream)))


def seg_energy_noalloc(f, u, v, p1, p2, lam, theta, out, stream=None):
    """seg_energy for callers that cannot allocate: no workspace argument; the
    library's fixed device scratch array is used instead (see include/seg.h)."""
    lib = load()
    _check(lib.seg_energy_noalloc(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(u), _ptr(v),
                                  _ptr(p1), _ptr(p2), float(lam), float(theta), _ptr(out),
                                  _stream(stream)))


def seg_batch_workspace_bytes(n_images, max_pixels=0):
    return load().seg_batch_workspace_bytes(int(n_images), int(max_pixels))


def seg_solve_batch(images, params: seg_params, state, stats, ws, stream=None):
    """`images`: a ctypes array of seg_image (device pointers)."""
    lib = load()
    _check(lib.seg_solve_batch(images, len(images), ctypes.byref(params), _ptr(state),
                               _nbytes(state), _ptr(stats), _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_ckpt_bytes(capacity, iters, ckpt_every):
    return load().seg_ckpt_bytes(int(capacity), int(iters), int(ckpt_every))


def seg_backward_scratch_bytes(capacity, ckpt_every):
    return load().seg_backward_scratch_bytes(int(capacity), int(ckpt_every))


def seg_solve_diff(f, act, fg, wstart, tiles, counts, params: seg_params, u, v, p1, p2, state,
                   ckpt_every, ckpt, stats, ws, stream=None):
    lib = load()
    _check(lib.seg_solve_diff(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(act), _ptr(fg),
                              _ptr(wstart), _ptr(tiles), _ptr(counts), ctypes.byref(params), _ptr(u),
                              _ptr(v), _ptr(p1), _ptr(p2), _ptr(state), _nbytes(state),
                              int(ckpt_every), _ptr(ckpt), _nbytes(ckpt), _ptr(stats), _ptr(ws),
                              _nbytes(ws), _stream(stream)))


def seg_backward(f, act, fg, wstart, counts, params: seg_params, state, ckpt, ckpt_every, grad_u,
                 grad_v, z, c, grad_f, grad_out, scratch, ws, stream=None):
    lib = load()
    _check(lib.seg_backward(_ptr(f), f.shape[0], _W(f), f.stride(0), _ptr(act), _ptr(fg),
                            _ptr(wstart), _ptr(counts), ctypes.byref(params), _ptr(state),
                            _nbytes(state), _ptr(ckpt), _nbytes(ckpt), int(ckpt_every),
                            _ptr(grad_u), _ptr(grad_v), _ptr(z), _ptr(c), _ptr(grad_f),
                            _ptr(grad_out), _ptr(scratch), _nbytes(scratch), _ptr(ws), _nbytes(ws),
                            _stream(stream)))


def seg_solve_diff_batch(images, params: seg_params, state, ckpt_every, ckpt, stats, ws, stream=None):
    """`images`: a ctypes array of seg_image (device pointers)."""
    _check(load().seg_solve_diff_batch(images, len(images), ctypes.byref(params), _ptr(state), _nbytes(state),
                                       int(ckpt_every), _ptr(ckpt), _nbytes(ckpt), _ptr(stats), _ptr(ws),
                                       _nbytes(ws), _stream(stream)))


def seg_backward_batch(images, adj, params: seg_params, state, ckpt, ckpt_every, scratch, ws, stream=None):
    """`images`, `adj`: ctypes arrays of seg_image and seg_adj_image."""
    _check(load().seg_backward_batch(images, adj, len(images), ctypes.byref(params), _ptr(state),
                                     _nbytes(state), _ptr(ckpt), _nbytes(ckpt), int(ckpt_every), _ptr(scratch),
                                     _nbytes(scratch), _ptr(ws), _nbytes(ws), _stream(stream)))


def seg_errors(u_star, u_gt, eps, out, ws, stream=None):
    lib = load()
    _check(lib.seg_errors(_ptr(u_star), _ptr(u_gt), u_star.shape[0], _W(u_star), u_star.stride(0),
                          float(eps), _ptr(out), _ptr(ws), _nbytes(ws), _stream(stream)))


def _nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


# Images are passed as [H][ld] views whose logical width is kept in an
# attribute set by `image()`; a plain [H][W] contiguous tensor is fine too
# when W is a multiple of 32.
def _W(t):
    return getattr(t, "_seg_w", t.shape[1])


# ------------------------------------------------------------ allocation

def pitch(W: int) -> int:
    return (W + 31) // 32 * 32


def image(H, W, dtype=torch.float32, device="cuda", fill=0):
    """[H][ld] device buffer with ld = W rounded up to 32; returns a tensor of
    shape [H, ld] tagged with its logical width W."""
    ld = pitch(W)
    t = torch.full((H, ld), fill, dtype=dtype, device=device)
    t._seg_w = W
    return t


def upload(a, device="cuda"):
    """Host array [H, W] -> pitched device image [H, ld]."""
    a = torch.as_tensor(a)
    H, W = a.shape
    t = image(H, W, dtype=a.dtype, device=device)
    t[:, :W].copy_(a)
    return t


def download(t):
    return t[:, :_W(t)].cpu().numpy()


def workspace(H, W, tile_h=16, device="cuda"):
    nb = seg_workspace_bytes(H, W, pitch(W), tile_h)
    return torch.zeros((nb + 15) // 16 * 16, dtype=torch.uint8, device=device)


@dataclass
class Domain:
    """Outputs of seg_build_domain for one image."""

    H: int
    W: int
    tile_h: int
    act: torch.Tensor
    fg: torch.Tensor
    wstart: torch.Tensor
    tiles: torch.Tensor
    pixels: torch.Tensor | None
    counts: torch.Tensor
    delta: torch.Tensor

    @property
    def n_tiles_total(self):
        return -(-self.H // self.tile_h) * -(-self.W // 32)


def build_domain(f, delta=math.inf, q=-1.0, tile_h=16, ws=None, with_pixels=True, stream=None,
                 radius=0, fbar=None):
    H, W = f.shape[0], _W(f)
    ld = f.stride(0)
    dev = f.device
    nw = ld // 32
    ntiles = -(-H // tile_h) * -(-W // 32)
    dom = Domain(H, W, tile_h,
                 act=torch.zeros((H, nw), dtype=torch.int32, device=dev),
                 fg=torch.zeros((H, nw), dtype=torch.int32, device=dev),
                 wstart=torch.zeros((H, nw), dtype=torch.int32, device=dev),
                 tiles=torch.zeros(max(ntiles, 1), dtype=torch.int32, device=dev),
                 pixels=torch.zeros(max(H * W, 1), dtype=torch.int32, device=dev) if with_pixels else None,
                 counts=torch.zeros(4, dtype=torch.int32, device=dev),
                 delta=torch.zeros(1, dtype=torch.float32, device=dev))
    if ws is None:
        ws = workspace(H, W, tile_h, dev)
    _build_into(f, delta, q, radius, tile_h, dom, ws, stream, fbar)
    return dom


def _mode(mode):
    return _MODE_BY_NAME[mode] if isinstance(mode, str) else int(mode)


def make_params(lam, theta=0.2, tau=0.125, iters=100, tol=0.0, n_inner=1, check_every=10,
                warm_start=False, mode="compact", storage="f32", tile_h=16, sweep=0) -> seg_params:
    return seg_params(float(lam), float(theta), float(tau), float(tol), int(iters), int(n_inner),
                      int(check_every), int(bool(warm_start)), _mode(mode),
                      _STORE_BY_NAME[storage] if isinstance(storage, str) else int(storage),
                      int(tile_h), int(sweep))


def state_buffer(H, W, capacity, mode="compact", storage="f32", device="cuda"):
    m = _mode(mode)
    s = _STORE_BY_NAME[storage] if isinstance(storage, str) else int(storage)
    nb = seg_state_bytes(H, pitch(W), int(capacity), m, s)
    return torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=device)


def capture_graph(fn, warmup=1):
    """Record the libseg launches that `fn()` issues on the current stream into
    a CUDA graph (torch's capture API); returns the graph, to be replayed with
    ``g.replay()``.  The buffers `fn` uses must stay alive and in place."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


class Solver:
    """Buffers for one H x W image and the chain fitting -> domain -> solve ->
    energy through the C ABI.  Allocation only (torch); every step runs in
    libseg's kernels on the current (or given) stream."""

    def __init__(self, H, W, tile_h=16, mode="compact", storage="f32", capacity=None,
                 device="cuda", stream=None):
        self.H, self.W, self.tile_h = H, W, tile_h
        self.mode, self.storage = mode, storage
        self.device = torch.device(device)
        self.stream = stream
        self.ws = workspace(H, W, tile_h, self.device)
        self.capacity = H * W if capacity is None else int(capacity)
        self.state = state_buffer(H, W, self.capacity, mode, storage, self.device)
        self.f = image(H, W, device=self.device)
        self.u = image(H, W, device=self.device)
        self.v = image(H, W, device=self.device)
        self.p1 = image(H, W, device=self.device)
        self.p2 = image(H, W, device=self.device)
        self.stats = torch.zeros(8, dtype=torch.float64, device=self.device)
        self.c = torch.zeros(2, dtype=torch.float64, device=self.device)
        self.energy_out = torch.zeros(6, dtype=torch.float64, device=self.device)
        self.err_out = torch.zeros(2, dtype=torch.float64, device=self.device)
        self.dom = None

    def fitting(self, z, c1=0.3, c2=0.7, label=None, markers=None, gamma=0.0):
        seg_make_fitting(z, c1, c2, label, markers, gamma, self.f, self.c, self.ws, self.stream)
        return self.f

    def domain(self, f=None, delta=math.inf, q=-1.0, with_pixels=True, radius=0, smooth=0):
        """RD = {|f| < delta} (or q's quantile).  smooth > 0: the robust
        restriction on the local mean of f over (2 smooth + 1)^2 squares;
        radius > 0: RD grown by that many pixels (seg_build_domain_robust)."""
        f = self.f if f is None else f
        fbar = None
        if smooth:
            if getattr(self, "fbar", None) is None:
                self.fbar = image(self.H, self.W, device=self.device)
            seg_box_mean(f, smooth, self.fbar, self.stream)
            fbar = self.fbar
        if self.dom is None or (self.dom.pixels is None) == with_pixels:
            self.dom = build_domain(f, delta, q, self.tile_h, self.ws, with_pixels, self.stream,
                                    radius, fbar)
        else:
            _build_into(f, delta, q, radius, self.tile_h, self.dom, self.ws, self.stream, fbar)
        return self.dom

    def solve(self, lam, theta=0.2, tau=0.125, iters=100, tol=0.0, n_inner=1, check_every=10,
              warm_start=False, f=None, sweep=0):
        f = self.f if f is None else f
        d = self.dom
        prm = make_params(lam, theta, tau, iters, tol, n_inner, check_every, warm_start,
                          self.mode, self.storage, self.tile_h, sweep)
        seg_solve(f, d.act, d.fg, d.wstart, d.tiles, d.counts, prm, self.u, self.v, self.p1,
                  self.p2, self.state, self.stats, self.ws, self.stream)
        return self.stats

    def solve_pd(self, lam, sigma=PD_STEP, tau=PD_STEP, iters=100, tol=0.0, check_every=10,
                 warm_start=False, f=None):
        """Restricted primal-dual (Chambolle-Pock) solve of Eq. CR on the
        current domain (seg_solve_pd); writes self.u, self.p1, self.p2 (v is
        not part of this method and is left as it was)."""
        f = self.f if f is None else f
        d = self.dom
        if self.mode == "compact" and self.storage == "f32":
            state = self.state
        else:   # the primal-dual solver keeps a float32 compact state
            if getattr(self, "_pd_state", None) is None:
                self._pd_state = state_buffer(self.H, self.W, self.capacity, "compact", "f32",
                                              self.device)
            state = self._pd_state
        prm = seg_pd_params(float(lam), float(sigma), float(tau), float(tol), int(iters),
                            int(check_every), int(bool(warm_start)), int(self.tile_h))
        seg_solve_pd(f, d.act, d.fg, d.wstart, d.counts, prm, self.u, self.p1, self.p2, state,
                     self.stats, self.ws, self.stream)
        return self.stats

    def update_means(self, z, thresh=0.5):
        """Chan-Vese intensity update from this solver's u (into self.c and
        the workspace, for fitting with c1 = c2 = NaN)."""
        seg_update_means(z, self.u, thresh, self.c, self.ws, self.stream)
        return self.c

    def chan_vese(self, z, lam, c1=0.3, c2=0.7, outer=5, iters=100, delta=math.inf, q=-1.0,
                  thresh=0.5, theta=0.2, tau=0.125, check_every=None):
        """Chan-Vese loop on the restricted solve, all on the device: for
        t = 0 .. outer-1 the fitting term of Eq. CV with the current (c1, c2)
        (the given ones, then the class means of z over u > thresh and
        u <= thresh), its domain, and `iters` iterations warm-started from the
        previous solve.  Returns self.c, the (c1, c2) of the last solve."""
        for t in range(outer):
            if t == 0:
                self.fitting(z, c1, c2)
            else:
                self.update_means(z, thresh)
                self.fitting(z, math.nan, math.nan)
            self.domain(delta=delta, q=q)
            self.solve(lam, theta, tau, iters, 0.0, 1, check_every or iters, warm_start=t > 0)
        return self.c

    def energy(self, lam, theta=0.2, f=None):
        f = self.f if f is None else f
        seg_energy(f, self.u, self.v, self.p1, self.p2, lam, theta, self.energy_out, self.ws,
                   self.stream)
        return self.energy_out

    def errors(self, u_star, u_gt, eps=0.5):
        seg_errors(u_star, u_gt, eps, self.err_out, self.ws, self.stream)
        return self.err_out

    def check_status(self):
        seg_read_status(self.ws, self.stream)


class VolumeSolver:
    """Buffers for one D x H x W volume, stored as its slices stacked into a
    (D*H) x W image ([D][H][ld] float32), and the chain fitting -> domain ->
    solve through the C ABI (seg_make_fitting and seg_build_domain on the
    stacked image, seg_solve3d for the iteration)."""

    def __init__(self, D, H, W, tile_h=16, capacity=None, device="cuda", stream=None):
        self.D, self.H, self.W, self.tile_h = D, H, W, tile_h
        self.device = torch.device(device)
        self.stream = stream
        R = D * H
        self.ws = workspace(R, W, tile_h, self.device)
        self.f = image(R, W, device=self.device)
        self.u = image(R, W, device=self.device)
        self.v = image(R, W, device=self.device)
        self.p1 = image(R, W, device=self.device)
        self.p2 = image(R, W, device=self.device)
        self.p3 = image(R, W, device=self.device)
        self.capacity = D * H * W if capacity is None else int(capacity)
        nb = seg_state_bytes3d(self.capacity)
        self.state = torch.empty((nb + 255) // 256 * 256, dtype=torch.uint8, device=self.device)
        self.stats = torch.zeros(8, dtype=torch.float64, device=self.device)
        self.c = torch.zeros(2, dtype=torch.float64, device=self.device)
        self.dom = None

    def upload(self, a):
        """Host volume [D, H, W] -> stacked device image."""
        a = torch.as_tensor(a, dtype=torch.float32).reshape(self.D * self.H, self.W)
        return upload(a, self.device)

    def download(self, t):
        """Stacked device image -> host volume [D, H, W]."""
        return download(t).reshape(self.D, self.H, self.W)

    def fitting(self, z, c1=0.3, c2=0.7, label=None):
        seg_make_fitting(z, c1, c2, label, None, 0.0, self.f, self.c, self.ws, self.stream)
        return self.f

    def domain(self, delta=math.inf, q=-1.0):
        if self.dom is None:
            self.dom = build_domain(self.f, delta, q, self.tile_h, self.ws, True, self.stream)
        else:
            d = self.dom
            seg_build_domain(self.f, delta, q, self.tile_h, d.act, d.fg, d.wstart, d.tiles, d.pixels,
                             d.counts, d.delta, self.ws, self.stream)
        return self.dom

    def solve(self, lam, theta=0.2, tau=0.125, iters=100, tol=0.0, check_every=10, warm_start=False):
        d = self.dom
        prm = make_params(lam, theta, tau, iters, tol, 1, check_every, warm_start, "compact", "f32",
                          self.tile_h)
        seg_solve3d(self.f, self.D, self.H, d.act, d.fg, d.wstart, d.pixels, d.counts, prm, self.u, self.v,
                    self.p1, self.p2, self.p3, self.state, self.stats, self.ws, self.stream)
        return self.stats

    def check_status(self):
        seg_read_status(self.ws, self.stream)


class BatchSolver:
    """Buffers for a batch of images (one Solver per image for the fitting
    term and the domain) and one shared compact state: the iteration of all
    images runs in one persistent launch (seg_solve_batch)."""

    def __init__(self, shapes, tile_h=16, storage="f32", capacity=None, device="cuda", stream=None):
        self.device = torch.device(device)
        self.stream = stream
        self.tile_h, self.storage = tile_h, storage
        Hm = max(h for h, _ in shapes)
        Wm = max(w for _, w in shapes)
        # one workspace large enough for the largest image serves every image
        self.ws_img = workspace(Hm, Wm, tile_h, self.device)
        self.solvers = []
        for (H, W) in shapes:
            S = Solver.__new__(Solver)
            S.H, S.W, S.tile_h, S.mode, S.storage = H, W, tile_h, "compact", storage
            S.device, S.stream, S.ws = self.device, stream, self.ws_img
            S.capacity, S.state = 0, None
            S.f = image(H, W, device=self.device)
            S.u = image(H, W, device=self.device)
            S.v = image(H, W, device=self.device)
            S.p1 = image(H, W, device=self.device)
            S.p2 = image(H, W, device=self.device)
            S.stats = torch.zeros(8, dtype=torch.float64, device=self.device)
            S.c = torch.zeros(2, dtype=torch.float64, device=self.device)
            S.energy_out = torch.zeros(6, dtype=torch.float64, device=self.device)
            S.err_out = torch.zeros(2, dtype=torch.float64, device=self.device)
            S.dom = None
            self.solvers.append(S)
        total = sum(h * w for h, w in shapes)
        self.capacity = total if capacity is None else int(capacity)
        self.state = state_buffer(0, 32, self.capacity, "compact", storage, self.device)
        nb = seg_batch_workspace_bytes(len(shapes), total)
        self.ws = torch.zeros((nb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        self.stats = torch.zeros(8, dtype=torch.float64, device=self.device)

    def images(self, lams):
        arr = (seg_image * len(self.solvers))()
        for k, (S, lam) in enumerate(zip(self.solvers, lams)):
            d = S.dom
            arr[k] = seg_image(S.f.data_ptr(), S.H, S.W, S.f.stride(0), d.act.data_ptr(),
                               d.fg.data_ptr(), d.wstart.data_ptr(), d.counts.data_ptr(),
                               S.u.data_ptr(), S.v.data_ptr(), S.p1.data_ptr(), S.p2.data_ptr(),
                               float(lam))
        return arr

    def solve(self, lams, theta=0.2, tau=0.125, iters=100, tol=0.0, n_inner=1, check_every=10,
              warm_start=False):
        prm = make_params(1.0, theta, tau, iters, tol, n_inner, check_every, warm_start, "compact",
                          self.storage, self.tile_h)
        seg_solve_batch(self.images(lams), prm, self.state, self.stats, self.ws, self.stream)
        return self.stats

    def check_status(self):
        seg_read_status(self.ws, self.stream)
        seg_read_status(self.ws_img, self.stream)


class DiffSolver(Solver):
    """A compact float32 Solver whose solve can be differentiated: the forward
    (seg_solve_diff) keeps checkpoints every `ckpt_every` iterations and
    `backward` runs the adjoint (seg_backward)."""

    def __init__(self, H, W, iters, ckpt_every=20, tile_h=16, capacity=None, device="cuda",
                 stream=None):
        super().__init__(H, W, tile_h=tile_h, mode="compact", storage="f32", capacity=capacity,
                         device=device, stream=stream)
        self.iters, self.ckpt_every = int(iters), int(ckpt_every)
        cap = self.capacity
        nb = seg_ckpt_bytes(cap, self.iters, self.ckpt_every)
        self.ckpt = torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        nb = seg_backward_scratch_bytes(cap, self.ckpt_every)
        self.scratch = torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        self.grad_f = image(H, W, device=self.device)
        self.grad_out = torch.zeros(3, dtype=torch.float64, device=self.device)
        self._prm = None

    def solve_diff(self, lam, theta=0.2, tau=0.125, f=None):
        f = self.f if f is None else f
        d = self.dom
        self._prm = make_params(lam, theta, tau, self.iters, 0.0, 1, self.iters, False, "compact",
                                "f32", self.tile_h)
        seg_solve_diff(f, d.act, d.fg, d.wstart, d.tiles, d.counts, self._prm, self.u, self.v,
                       self.p1, self.p2, self.state, self.ckpt_every, self.ckpt, self.stats, self.ws,
                       self.stream)
        return self.u

    def backward(self, grad_u, grad_v=None, z=None, c=None, f=None):
        f = self.f if f is None else f
        d = self.dom
        seg_backward(f, d.act, d.fg, d.wstart, d.counts, self._prm, self.state, self.ckpt,
                     self.ckpt_every, grad_u, grad_v, z, c, self.grad_f, self.grad_out,
                     self.scratch, self.ws, self.stream)
        return self.grad_f, self.grad_out


class BatchDiffSolver(BatchSolver):
    """A float32 BatchSolver whose batched solve can be differentiated: the
    forward (seg_solve_diff_batch) keeps checkpoints every `ckpt_every`
    iterations and `backward` runs the adjoint of every image in one
    persistent sweep (seg_backward_batch)."""

    def __init__(self, shapes, iters, ckpt_every=20, tile_h=16, capacity=None, device="cuda", stream=None):
        super().__init__(shapes, tile_h=tile_h, storage="f32", capacity=capacity, device=device,
                         stream=stream)
        self.iters, self.ckpt_every = int(iters), int(ckpt_every)
        nb = seg_ckpt_bytes(self.capacity, self.iters, self.ckpt_every)
        self.ckpt = torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        nb = seg_backward_scratch_bytes(self.capacity, self.ckpt_every)
        self.scratch = torch.empty((nb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        for S in self.solvers:
            S.grad_f = image(S.H, S.W, device=self.device)
            S.grad_out = torch.zeros(3, dtype=torch.float64, device=self.device)
        self._prm = None
        self._lams = None

    def solve_diff(self, lams, theta=0.2, tau=0.125):
        self._lams = list(lams)
        self._prm = make_params(1.0, theta, tau, self.iters, 0.0, 1, self.iters, False, "compact", "f32",
                                self.tile_h)
        seg_solve_diff_batch(self.images(self._lams), self._prm, self.state, self.ckpt_every, self.ckpt,
                             self.stats, self.ws, self.stream)

    def backward(self, grads_u, grads_v=None, zs=None, cs=None):
        n = len(self.solvers)
        adj = (seg_adj_image * n)()
        for k, S in enumerate(self.solvers):
            gv = grads_v[k] if grads_v is not None else None
            z = zs[k] if zs is not None else None
            c = cs[k] if cs is not None else None
            adj[k] = seg_adj_image(_ptr(grads_u[k]), _ptr(gv), _ptr(z), _ptr(c), _ptr(S.grad_f),
                                   _ptr(S.grad_out))
        seg_backward_batch(self.images(self._lams), adj, self._prm, self.state, self.ckpt, self.ckpt_every,
                           self.scratch, self.ws, self.stream)
        return [(S.grad_f, S.grad_out) for S in self.solvers]


class SegSolveFn(torch.autograd.Function):
    """u^K = solve(f, lambda) through the unrolled restricted iteration, with
    the hand-written adjoint as its backward.  f is a [H, ld] image tensor
    (its domain must already be built in `solver` with solver.domain), lam a
    0-d float64 tensor; returns u^K ([H, ld])."""

    @staticmethod
    def forward(ctx, f, lam, solver: DiffSolver, theta=0.2, tau=0.125):
        solver.f.copy_(f)
        solver.solve_diff(float(lam.item()), theta, tau)
        ctx.solver = solver
        return solver.u.clone()

    @staticmethod
    def backward(ctx, grad_u):
        S = ctx.solver
        g = image(S.H, S.W, device=S.device)
        g.copy_(grad_u)
        gf, gout = S.backward(g)
        return gf.clone(), gout[0].clone(), None, None, None


class SegFitSolveFn(torch.autograd.Function):
    """u^K = solve(f(z; c1, c2), lambda) with f the piecewise-constant fitting
    term (Eq. CV); gradients for c1, c2 and lambda.  z: [H, ld] image tensor;
    c1, c2, lam: 0-d float64 tensors.  The domain is built from f at delta
    (and held fixed in the backward)."""

    @staticmethod
    def forward(ctx, z, c1, c2, lam, solver: DiffSolver, delta, theta=0.2, tau=0.125):
        seg_make_fitting(z, float(c1.item()), float(c2.item()), None, None, 0.0, solver.f, solver.c,
                         solver.ws, solver.stream)
        solver.domain(delta=delta)
        solver.solve_diff(float(lam.item()), theta, tau)
        ctx.solver, ctx.z = solver, z
        return solver.u.clone()

    @staticmethod
    def backward(ctx, grad_u):
        S = ctx.solver
        g = image(S.H, S.W, device=S.device)
        g.copy_(grad_u)
        _, gout = S.backward(g, z=ctx.z, c=S.c)
        return None, gout[1].clone(), gout[2].clone(), gout[0].clone(), None, None, None, None


_TUNE_CACHE = {}


def autotune(key, make_run, candidates, reps=3):
    """Project autotuner: `make_run(c)` prepares the work for candidate c (for
    example a solver whose domain uses tile height c) and returns a callable
    that runs a short solve on the current stream; each candidate is timed
    with CUDA events (best of `reps` after one warm-up) and the fastest is
    returned and cached under `key`."""
    if key in _TUNE_CACHE:
        return _TUNE_CACHE[key]
    best, best_t = None, None
    for c in candidates:
        run = make_run(c)
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = None
        for _ in range(reps):
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1)
            t = dt if t is None else min(t, dt)
        if best_t is None or t < best_t:
            best, best_t = c, t
    _TUNE_CACHE[key] = best
    return best
