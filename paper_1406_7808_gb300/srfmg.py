"""Thin Python binding of the C ABI in include/srfmg.h (ctypes; argument
marshalling only -- every step of the solve runs in the CUDA library).

Device arrays are torch float64 CUDA tensors of shape (n, n, n) -- or
(n l2, n l1, n l0) on the domain [0, l0] x [0, l1] x [0, l2] -- contiguous,
index order [z][y][x]; work is queued on torch's current CUDA stream.  The
library is loaded on first use; a missing or unloadable library raises
RuntimeError (there is no fallback path).
"""
import ctypes
import os

import numpy as np

from . import build as _build

MAXK = 12

SR_OK = 0
SR_ERR_INVALID = -1
SR_ERR_UNSUPPORTED_SIZE = -2
SR_ERR_OOM = -3
SR_ERR_CUDA = -4
SR_ERR_TIMEOUT = -5
SR_ERR_NONFINITE = -6
SR_ERR_NO_DEVICE = -7

SR_FP64 = 0
SR_MIXED = 1


class SRFMGError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Config(ctypes.Structure):
    """Mirror of sr_fmg_config."""
    _fields_ = [
        ("n", ctypes.c_int),
        ("n_coarse", ctypes.c_int),
        ("seg", ctypes.c_int),
        ("K", ctypes.c_int),
        ("A", ctypes.c_int),
        ("B", ctypes.c_int),
        ("use_J", ctypes.c_int),
        ("J", ctypes.c_int * MAXK),
        ("alpha", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("n_outer", ctypes.c_int),
        ("mbs", ctypes.c_int),
        ("len", ctypes.c_int * 3),
        ("stencil", ctypes.c_int),
        ("w", ctypes.c_double * 3),
        ("graph", ctypes.c_int),
        ("seg_first", ctypes.c_int),
        ("seg_count", ctypes.c_int),
    ]


_LIB = None
_VP = ctypes.c_void_p


def library_path():
    return _build.LIBRARY


def load():
    """Load the CUDA library (raises RuntimeError if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    lib.sr_fmg_default_config.argtypes = [ctypes.POINTER(Config), ctypes.c_int]
    lib.sr_fmg_default_config.restype = None
    lib.sr_fmg_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Config)]
    lib.sr_fmg_destroy.argtypes = [_VP]
    lib.sr_fmg_workspace_bytes.argtypes = [_VP, ctypes.POINTER(ctypes.c_size_t)]
    for name in ("sr_fmg_solve", "sr_fmg_solve_async", "sr_fmg_solve_host"):
        getattr(lib, name).argtypes = [_VP, _VP, _VP, _VP]
    lib.sr_fmg_check.argtypes = [_VP, _VP]
    lib.sr_fmg_solve_host_async.argtypes = [_VP, _VP, _VP, _VP]
    lib.sr_fmg_check_host.argtypes = [_VP]
    lib.sr_fmg_status_string.argtypes = [ctypes.c_int]
    lib.sr_fmg_status_string.restype = ctypes.c_char_p
    lib.sr_fmg_launches_per_solve.argtypes = [_VP, ctypes.POINTER(ctypes.c_int)]
    lib.sr_fmg_vsolve.argtypes = [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                  _VP]
    lib.sr_fmg_profile.argtypes = [_VP, ctypes.c_int]
    lib.sr_fmg_profile_kinds.argtypes = []
    lib.sr_fmg_profile_read.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
    lib.sr_fmg_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int]
    lib.sr_fmg_batch_destroy.argtypes = [_VP]
    for name in ("sr_fmg_batch_solve", "sr_fmg_batch_solve_async"):
        getattr(lib, name).argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]
    lib.sr_fmg_batch_check.argtypes = [_VP, _VP]
    lib.sr_fmg_batch_autotune.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP,
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_float)]
    lib.sr_fmg_batch_set_streams.argtypes = [_VP, ctypes.c_int]
    lib.sr_fmg_solve_batched.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                         ctypes.POINTER(_VP), ctypes.c_int, _VP]
    lib.sr_op_apply.argtypes = [ctypes.c_int, _VP, _VP, _VP]
    lib.sr_op_residual.argtypes = [ctypes.c_int, _VP, _VP, _VP, _VP]
    lib.sr_op_smooth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 _VP, _VP, _VP]
    lib.sr_op_smooth_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, _VP, _VP, _VP]
    lib.sr_op_restrict.argtypes = [ctypes.c_int, _VP, _VP, _VP]
    lib.sr_op_prolong.argtypes = [ctypes.c_int, _VP, _VP, _VP]
    lib.sr_op_coarse_solve.argtypes = [ctypes.c_int, _VP, _VP, _VP]
    lib.sr_op_vcycle.argtypes = [ctypes.POINTER(Config), _VP, _VP, _VP]
    PC = ctypes.POINTER(Config)
    for name in ("sr_op_apply_ex", "sr_op_restrict_ex", "sr_op_prolong_ex",
                 "sr_op_coarse_solve_ex"):
        getattr(lib, name).argtypes = [PC, _VP, _VP, _VP]
    lib.sr_op_residual_ex.argtypes = [PC, _VP, _VP, _VP, _VP]
    lib.sr_op_smooth_ex.argtypes = [PC, ctypes.c_int, _VP, _VP, _VP]
    lib.sr_probe_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]
    lib.sr_debug_fail_alloc.argtypes = [ctypes.c_int]
    lib.sr_debug_alloc_count.argtypes = []
    lib.sr_debug_alloc_count.restype = ctypes.c_longlong
    lib.sr_debug_live_bytes.argtypes = []
    lib.sr_debug_live_bytes.restype = ctypes.c_longlong
    lib.sr_debug_last_stage_trim.argtypes = [_VP, ctypes.c_int]
    lib.sr_debug_narrow.argtypes = [_VP, _VP, ctypes.c_longlong, _VP]
    lib.sr_debug_segment_legs.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.sr_debug_force_wait_timeout.argtypes = [_VP, ctypes.c_int]
    lib.sr_debug_persistent_vcycle.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.sr_fmg_set_launch_shape.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
    lib.sr_fmg_launch_shape.argtypes = [_VP, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
    lib.sr_fmg_stage_down.argtypes = [_VP, _VP, ctypes.c_int, _VP]
    lib.sr_fmg_stage_buffers.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                         ctypes.POINTER(ctypes.c_size_t)]
    lib.sr_fmg_stage_up.argtypes = [_VP, _VP, ctypes.c_int, _VP, _VP]
    _LIB = lib
    return lib


def status_string(status):
    try:
        return load().sr_fmg_status_string(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status, what):
    if status != SR_OK:
        raise SRFMGError(status, what)


def probe_fma_rate(bits=64):
    """Measured peak FMA rate of the current device in lane operations per
    second (bits = 64: float64, 32: float32); sr_probe_fma_rate."""
    rate = ctypes.c_double(0.0)
    _check(load().sr_probe_fma_rate(int(bits), ctypes.byref(rate), _stream()), "sr_probe_fma_rate")
    return rate.value


def debug_fail_alloc(nth):
    """Make the nth device allocation of the library from now fail as out of
    memory (0: off); for testing the error paths."""
    _check(load().sr_debug_fail_alloc(int(nth)), "sr_debug_fail_alloc")


def debug_narrow(x):
    """float64 CUDA tensor -> float32 through the library's integer-pipe
    rounding (sr_debug_narrow)."""
    import torch
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    _check(load().sr_debug_narrow(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  x.numel(), _stream()), "sr_debug_narrow")
    return out


def debug_alloc_count():
    """Device allocations the library has attempted since it was loaded."""
    return int(load().sr_debug_alloc_count())


def debug_live_bytes():
    """Bytes of device memory the library's handles hold now."""
    return int(load().sr_debug_live_bytes())


def mbs_schedule(J1, K):
    """Maximum buffer schedule (Sec. 5.2.1): J_k = 2^(k-1) J_1, k = 1..K."""
    return [J1 << (k - 1) for k in range(1, K + 1)]


def buffer_schedule(A, B, K):
    """J_k = 2 floor((A + B (K - k)) / 2), k = 1..K (Eq. eq:nb)."""
    return [2 * ((A + B * (K - k)) // 2) for k in range(1, K + 1)]


def make_config(n, *, seg=0, K=0, A=8, B=0, J=None, n_coarse=0, alpha=1, nu1=2, nu2=2,
                cheb_lo=1.0 / 6.0, cheb_hi=1.0, precision=SR_FP64, n_outer=2, mixed=False,
                mbs=False, lengths=(1, 1, 1), stencil=7, weights=None, graph=False,
                segments=None):
    """sr_fmg_config with n cells per unit length (mixed=True selects SR_MIXED;
    mbs=True the maximum buffer schedule J_k = 2^(k-1) A; lengths the domain
    [0, l0] x [0, l1] x [0, l2]; stencil 7 or 27 with weights (faces, edges,
    corners); graph=True queues each solve as one captured CUDA graph;
    segments=(first, count) a segment range, solved stage by stage)."""
    c = Config()
    load().sr_fmg_default_config(ctypes.byref(c), int(n))
    c.n_coarse, c.seg, c.K, c.A, c.B = n_coarse, seg, K, A, B
    if J is not None:
        if len(J) != K:
            raise ValueError("J must have K entries")
        c.use_J = 1
        for i, v in enumerate(J):
            c.J[i] = int(v)
    c.alpha, c.nu1, c.nu2 = alpha, nu1, nu2
    c.cheb_lo, c.cheb_hi = cheb_lo, cheb_hi
    c.precision, c.n_outer = (SR_MIXED if mixed else precision), n_outer
    c.mbs = int(bool(mbs))
    for d in range(3):
        c.len[d] = int(lengths[d])
    c.stencil = int(stencil)
    c.graph = int(bool(graph))
    if segments is not None:
        c.seg_first, c.seg_count = int(segments[0]), int(segments[1])
    if weights is None and int(stencil) == 27:
        weights = W27_DEFAULT
    if weights is not None:
        for d in range(3):
            c.w[d] = float(weights[d])
    return c


# the 27-point reading used when no weights are given: (14, 3, 1)/30 for the
# face, edge and corner neighbours (centre 128/30)
W27_DEFAULT = (14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)


def grid_shape(n, lengths=(1, 1, 1)):
    """Array shape (z, y, x) of the grid with n cells per unit length."""
    return (n * int(lengths[2]), n * int(lengths[1]), n * int(lengths[0]))


GEO_KEYS = ("lengths", "stencil", "weights")


def _per_unit(t, lengths):
    n = t.shape[2] // int(lengths[0])
    if n < 1 or tuple(t.shape) != grid_shape(n, lengths):
        raise ValueError(f"shape {tuple(t.shape)} does not match the domain lengths {lengths}")
    return n


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, shape=None, name="array"):
    """shape None: any cube; else the exact (z, y, x) shape"""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dim() != 3:
        raise ValueError(f"{name} must be a 3D tensor")
    if shape is None and len(set(t.shape)) != 1:
        raise ValueError(f"{name} must have shape (n, n, n)")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One sr_fmg_t handle: plan and device workspace for one configuration."""

    def __init__(self, n, **kw):
        self.config = make_config(n, **kw)
        self.n = int(n)
        self.shape = grid_shape(self.n, kw.get("lengths", (1, 1, 1)))
        h = _VP()
        _check(load().sr_fmg_create(ctypes.byref(h), ctypes.byref(self.config)), "sr_fmg_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().sr_fmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- stage-by-stage solve (segment ranges shared among handles) ----

    @property
    def K(self):
        return int(self.config.K) if self.config.seg else 0

    def stage_down(self, f, k):
        """SR stage k up to the transition level (k = 1 also runs the f
        hierarchy and the global FMG); the handle's genuine transition-level
        cells land in the exchange arrays, zeros elsewhere."""
        _check(load().sr_fmg_stage_down(self._h, _dev(f, self.shape, "f"), int(k), _stream()),
               "sr_fmg_stage_down")

    def stage_buffers(self):
        """The two exchange arrays (\\hat I u_1 and the restricted residual
        on the transition level) as torch float64 CUDA tensors that alias the
        handle's memory: the caller sums them over all handles in place."""
        import torch
        a, b, count = _VP(), _VP(), ctypes.c_size_t()
        _check(load().sr_fmg_stage_buffers(self._h, ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(count)), "sr_fmg_stage_buffers")
        return tuple(torch.as_tensor(_DeviceArray(p.value, count.value), device="cuda")
                     for p in (a, b))

    def stage_up(self, f, k, out):
        """Transition level, global V-cycle and the up-leg of stage k; after
        the last stage the handle's genuine finest cells go to out."""
        _check(load().sr_fmg_stage_up(self._h, _dev(f, self.shape, "f"), int(k),
                                      _dev(out, self.shape, "out"), _stream()),
               "sr_fmg_stage_up")
        return out

    @property
    def launch_shape(self):
        """(zchunk, cells_per_thread) of the handle's kernels."""
        z, c = ctypes.c_int(), ctypes.c_int()
        _check(load().sr_fmg_launch_shape(self._h, ctypes.byref(z), ctypes.byref(c)),
               "sr_fmg_launch_shape")
        return z.value, c.value

    def set_launch_shape(self, zchunk, cells_per_thread):
        """Cells in z per thread of the column kernels and cells per thread of
        the per-cell kernels (results do not depend on them)."""
        _check(load().sr_fmg_set_launch_shape(self._h, int(zchunk), int(cells_per_thread)),
               "sr_fmg_set_launch_shape")

    def debug_segment_legs(self, enable):
        """Segment-resident legs on or off (default: off, the separate kernels
        are faster on GB300); returns the levels that have one (a list of j)."""
        levels = ctypes.c_int(0)
        _check(load().sr_debug_segment_legs(self._h, int(bool(enable)), ctypes.byref(levels)),
               "sr_debug_segment_legs")
        return [j for j in range(1, 31) if levels.value >> j & 1]

    def debug_persistent_vcycle(self, enable):
        """The global V-cycle as one persistent launch (default) or as separate
        kernels; returns whether the handle can use the persistent one."""
        avail = ctypes.c_int(0)
        _check(load().sr_debug_persistent_vcycle(self._h, int(bool(enable)), ctypes.byref(avail)),
               "sr_debug_persistent_vcycle")
        return bool(avail.value)

    def debug_force_wait_timeout(self, enable):
        """Make the legs' bounded waits run out (the solve reports
        SR_ERR_TIMEOUT); for testing."""
        _check(load().sr_debug_force_wait_timeout(self._h, int(bool(enable))),
               "sr_debug_force_wait_timeout")

    def debug_last_stage_trim(self, enable):
        """Turn the last stage's trimming on (default) or off (same result)."""
        _check(load().sr_debug_last_stage_trim(self._h, int(bool(enable))),
               "sr_debug_last_stage_trim")

    @property
    def workspace_bytes(self):
        b = ctypes.c_size_t()
        _check(load().sr_fmg_workspace_bytes(self._h, ctypes.byref(b)), "workspace_bytes")
        return b.value

    @property
    def launches_per_solve(self):
        v = ctypes.c_int()
        _check(load().sr_fmg_launches_per_solve(self._h, ctypes.byref(v)), "launches_per_solve")
        return v.value

    def profile(self, enable):
        """Start (True, clears counters) or stop per-kernel event timing."""
        _check(load().sr_fmg_profile(self._h, int(bool(enable))), "sr_fmg_profile")

    def profile_read(self):
        """{kernel: dict(launches, ms, ops, bytes)} for kernels that ran; ops are
        the algorithmic floating-point operations (float32 for kinds ending in
        _f32, float64 otherwise)."""
        lib = load()
        out = {}
        for k in range(lib.sr_fmg_profile_kinds()):
            name = ctypes.c_char_p()
            launches = ctypes.c_longlong()
            ms, ops, nbytes = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(lib.sr_fmg_profile_read(self._h, k, ctypes.byref(name), ctypes.byref(launches),
                                           ctypes.byref(ms), ctypes.byref(ops),
                                           ctypes.byref(nbytes)), "sr_fmg_profile_read")
            if launches.value:
                out[name.value.decode()] = dict(launches=launches.value, ms=ms.value,
                                                ops=ops.value, bytes=nbytes.value)
        return out

    def solve(self, f, out=None):
        """u = solver(f) for a float64 CUDA tensor f; waits and checks status."""
        import torch
        if out is None:
            out = torch.empty_like(f)
        _check(load().sr_fmg_solve(self._h, _dev(f, self.shape, "f"), _dev(out, self.shape, "u"),
                                   _stream()), "sr_fmg_solve")
        return out

    def vsolve(self, f, u=None, rtol=1e-4, max_cycles=100):
        """Iterative V-cycle solve (plain float64 handle): V-cycles on u (zero
        if None, else updated in place) until ||f - A u||_inf <= rtol ||f||_inf.
        Returns (u, cycles, relative residual)."""
        import torch
        if u is None:
            u = torch.zeros_like(f)
        cycles, rel = ctypes.c_int(), ctypes.c_double()
        _check(load().sr_fmg_vsolve(self._h, _dev(f, self.shape, "f"), _dev(u, self.shape, "u"),
                                    float(rtol), int(max_cycles), ctypes.byref(cycles),
                                    ctypes.byref(rel), _stream()), "sr_fmg_vsolve")
        return u, cycles.value, rel.value

    def solve_async(self, f, out):
        _check(load().sr_fmg_solve_async(self._h, _dev(f, self.shape, "f"), _dev(out, self.shape, "u"),
                                         _stream()), "sr_fmg_solve_async")
        return out

    def check(self):
        _check(load().sr_fmg_check(self._h, _stream()), "sr_fmg_check")

    def solve_host_async(self, f, out):
        """Queue a pipelined end-to-end solve of host f into host out (both
        stay owned by the caller and must not change until check_host());
        consecutive calls overlap their copies with each other's solves."""
        _check(load().sr_fmg_solve_host_async(self._h, _host_ptr(f, self.shape, "f"),
                                              _host_ptr(out, self.shape, "out"), _stream()),
               "sr_fmg_solve_host_async")
        return out

    def check_host(self):
        """Wait for every queued pipelined solve's result to reach the host."""
        _check(load().sr_fmg_check_host(self._h), "sr_fmg_check_host")

    def solve_host(self, f, out=None):
        """End-to-end solve of a host array (numpy float64 (n, n, n) or a CPU
        tensor); the copies to and from the device run inside the library."""
        if hasattr(f, "numpy"):
            f = f.numpy()
        f = np.ascontiguousarray(f, dtype=np.float64)
        if tuple(f.shape) != self.shape:
            raise ValueError(f"f must have shape {self.shape}")
        if out is None:
            out = np.empty_like(f)
        fp = ctypes.c_void_p(f.ctypes.data)
        up = ctypes.c_void_p(out.ctypes.data) if isinstance(out, np.ndarray) else \
            ctypes.c_void_p(out.data_ptr())
        _check(load().sr_fmg_solve_host(self._h, fp, up, _stream()), "sr_fmg_solve_host")
        return out


class _DeviceArray:
    """A float64 vector in device memory the library owns, exposed through
    the CUDA array interface (torch.as_tensor wraps it without a copy)."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def segment_range(nsegs, rank, world):
    """(first, count) of the contiguous share of nsegs segments that rank
    `rank` of `world` owns (shares differ by at most one segment)."""
    first = rank * nsegs // world
    return first, (rank + 1) * nsegs // world - first


def segment_count(n, seg, lengths=(1, 1, 1)):
    """Segments of an SR configuration: (n l0 / seg)(n l1 / seg)(n l2 / seg)."""
    out = 1
    for l in lengths:
        out *= n * int(l) // seg
    return out


def solve_staged(solvers, f, out, reduce_sum=None):
    """SR-FMG of one problem through the stage entry points.  solvers: the
    handles this process drives (segment ranges of the same problem, or one
    handle with all segments); f: each handle's copy of the whole right-hand
    side (one tensor, or one per handle); out: the output tensor(s), each
    handle writing its own segments' genuine cells.  reduce_sum(tensors)
    sums the exchange arrays in place over all handles of the problem that
    other processes drive (None: this process drives them all); the arrays
    of the local handles are summed here first.  Every step of the solve
    runs in the library; this loop only moves the two transition-level
    arrays between handles (Sec. 4: the transition level is the one
    exchange of the method)."""
    solvers = list(solvers)
    fs = f if isinstance(f, (list, tuple)) else [f] * len(solvers)
    outs = out if isinstance(out, (list, tuple)) else [out] * len(solvers)
    K = solvers[0].K
    for k in range(1, K + 1):
        for s, fk in zip(solvers, fs):
            s.stage_down(fk, k)
        bufs = [s.stage_buffers() for s in solvers]
        exchange_sum(bufs, reduce_sum)
        for s, fk, o in zip(solvers, fs, outs):
            s.stage_up(fk, k, o)
    return outs


def exchange_sum(bufs, reduce_sum=None):
    """bufs: per local handle, a tuple of arrays; afterwards every handle's
    arrays hold the sum over all handles (the local ones, then reduce_sum
    across processes).  Works on any torch tensors (CUDA or CPU).  Every
    cell has one owner, so the sum is exact whatever its order."""
    total = [t.clone() for t in bufs[0]]
    for b in bufs[1:]:
        for acc, x in zip(total, b):
            acc.add_(x)
    if reduce_sum is not None:
        reduce_sum(total)
    for b in bufs:
        for dst, src in zip(b, total):
            dst.copy_(src)
    return total


def _host_ptr(a, shape, name):
    """address of a host float64 array (numpy, or a CPU tensor) of the given shape"""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous() or tuple(a.shape) != shape:
            raise ValueError(f"{name} must be a contiguous float64 CPU tensor of shape {shape}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous \
            or a.shape != shape:
        raise ValueError(f"{name} must be a contiguous float64 array of shape {shape}")
    return ctypes.c_void_p(a.ctypes.data)


class Batch:
    """Many solves (grids of any sizes) run as one CUDA graph launch.

    solvers: Solver objects, one per problem (kept alive by the batch).
    solve(fs, us): fs, us lists of float64 CUDA tensors, problem i solved by
    solvers[i]; the graph is captured on the first call for a pointer set and
    relaunched afterwards."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        hs = (_VP * len(self.solvers))(*[s._h for s in self.solvers])
        b = _VP()
        _check(load().sr_fmg_batch_create(ctypes.byref(b), hs, len(self.solvers)),
               "sr_fmg_batch_create")
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            load().sr_fmg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ptrs(self, fs, us):
        if len(fs) != len(self.solvers) or len(us) != len(self.solvers):
            raise ValueError("one f and one u per problem")
        fp = (_VP * len(fs))(*[_dev(f, s.shape, "f").value for f, s in zip(fs, self.solvers)])
        up = (_VP * len(us))(*[_dev(u, s.shape, "u").value for u, s in zip(us, self.solvers)])
        return fp, up

    def solve(self, fs, us):
        fp, up = self._ptrs(fs, us)
        _check(load().sr_fmg_batch_solve(self._b, fp, up, _stream()), "sr_fmg_batch_solve")
        return us

    def solve_async(self, fs, us):
        fp, up = self._ptrs(fs, us)
        _check(load().sr_fmg_batch_solve_async(self._b, fp, up, _stream()),
               "sr_fmg_batch_solve_async")
        return us

    def check(self):
        _check(load().sr_fmg_batch_check(self._b, _stream()), "sr_fmg_batch_check")

    def autotune(self, fs, us):
        """Time the graph with 1, 2, 4, ... branches and keep the fastest;
        returns (branches, ms per batch)."""
        fp, up = self._ptrs(fs, us)
        best, ms = ctypes.c_int(), ctypes.c_float()
        _check(load().sr_fmg_batch_autotune(self._b, fp, up, _stream(), ctypes.byref(best),
                                            ctypes.byref(ms)), "sr_fmg_batch_autotune")
        return best.value, ms.value

    def set_streams(self, streams):
        _check(load().sr_fmg_batch_set_streams(self._b, int(streams)), "sr_fmg_batch_set_streams")


def solve_batched(solvers, fs, us):
    """One-shot batched solve through sr_fmg_solve_batched."""
    hs = (_VP * len(solvers))(*[s._h for s in solvers])
    fp = (_VP * len(fs))(*[_dev(f, s.shape, "f").value for f, s in zip(fs, solvers)])
    up = (_VP * len(us))(*[_dev(u, s.shape, "u").value for u, s in zip(us, solvers)])
    _check(load().sr_fmg_solve_batched(hs, fp, up, len(solvers), _stream()),
           "sr_fmg_solve_batched")
    return us


# ---- single components on whole grids (for parity tests) ----

def _geo_cfg(t, geo, **extra):
    return make_config(_per_unit(t, geo.get("lengths", (1, 1, 1))), **geo, **extra)


def op_apply(u, **geo):
    """A u; geo: lengths, stencil, weights (default: unit cube, 7-point)."""
    import torch
    out = torch.empty_like(u)
    if geo:
        c = _geo_cfg(u, geo)
        _check(load().sr_op_apply_ex(ctypes.byref(c), _dev(u, u.shape), _dev(out, u.shape),
                                     _stream()), "sr_op_apply_ex")
    else:
        _check(load().sr_op_apply(u.shape[0], _dev(u), _dev(out), _stream()), "sr_op_apply")
    return out


def op_residual(u, f, **geo):
    import torch
    r = torch.empty_like(u)
    if geo:
        c = _geo_cfg(u, geo)
        _check(load().sr_op_residual_ex(ctypes.byref(c), _dev(f, u.shape), _dev(u, u.shape),
                                        _dev(r, u.shape), _stream()), "sr_op_residual_ex")
    else:
        _check(load().sr_op_residual(u.shape[0], _dev(f), _dev(u), _dev(r), _stream()),
               "sr_op_residual")
    return r


def op_smooth(u, f, nu, cheb_lo=1.0 / 6.0, cheb_hi=1.0, **geo):
    """Chebyshev smoother; returns a new tensor (u is not modified)."""
    u = u.clone()
    if geo:
        c = _geo_cfg(u, geo, cheb_lo=cheb_lo, cheb_hi=cheb_hi)
        _check(load().sr_op_smooth_ex(ctypes.byref(c), nu, _dev(f, u.shape), _dev(u, u.shape),
                                      _stream()), "sr_op_smooth_ex")
    else:
        _check(load().sr_op_smooth(u.shape[0], nu, cheb_lo, cheb_hi, _dev(f), _dev(u),
                                   _stream()), "sr_op_smooth")
    return u


NOALLOC_MAX_N = 64


def op_smooth_noalloc(u, f, nu, cheb_lo=1.0 / 6.0, cheb_hi=1.0):
    """Chebyshev smoother whose scratch lives in a fixed device array of the
    library (no device allocation; n <= NOALLOC_MAX_N).  For callers that
    cannot allocate device memory where they smooth.  Calls that overlap on
    the GPU share that scratch and race.  Returns a new tensor."""
    u = u.clone()
    _check(load().sr_op_smooth_noalloc(u.shape[0], nu, cheb_lo, cheb_hi, _dev(f), _dev(u),
                                       _stream()), "sr_op_smooth_noalloc")
    return u


def op_restrict(a, **geo):
    import torch
    out = torch.empty(tuple(v // 2 for v in a.shape), dtype=a.dtype, device=a.device)
    if geo:
        c = _geo_cfg(a, geo)
        _check(load().sr_op_restrict_ex(ctypes.byref(c), _dev(a, a.shape), _dev(out, out.shape),
                                        _stream()), "sr_op_restrict_ex")
    else:
        _check(load().sr_op_restrict(a.shape[0], _dev(a), _dev(out), _stream()),
               "sr_op_restrict")
    return out


def op_prolong(ac, **geo):
    import torch
    out = torch.empty(tuple(2 * v for v in ac.shape), dtype=ac.dtype, device=ac.device)
    if geo:
        c = _geo_cfg(ac, geo)
        _check(load().sr_op_prolong_ex(ctypes.byref(c), _dev(ac, ac.shape),
                                       _dev(out, out.shape), _stream()), "sr_op_prolong_ex")
    else:
        _check(load().sr_op_prolong(ac.shape[0], _dev(ac), _dev(out), _stream()),
               "sr_op_prolong")
    return out


def op_coarse_solve(f, **geo):
    import torch
    u = torch.empty_like(f)
    if geo:
        c = _geo_cfg(f, geo)
        _check(load().sr_op_coarse_solve_ex(ctypes.byref(c), _dev(f, f.shape), _dev(u, f.shape),
                                            _stream()), "sr_op_coarse_solve_ex")
    else:
        _check(load().sr_op_coarse_solve(f.shape[0], _dev(f), _dev(u), _stream()),
               "sr_op_coarse_solve")
    return u


def op_vcycle(f, u, **kw):
    """One FAS V-cycle; returns a new tensor."""
    u = u.clone()
    c = make_config(_per_unit(f, kw.get("lengths", (1, 1, 1))), **kw)
    _check(load().sr_op_vcycle(ctypes.byref(c), _dev(f, f.shape), _dev(u, f.shape), _stream()),
           "sr_op_vcycle")
    return u


def _autograd_function():
    import torch

    class SRFMGFunction(torch.autograd.Function):
        """u = S(f) with S the (SR-)FMG solve; backward returns S(dL/du).

        A is symmetric, so the derivative of the exact discrete solution
        A^-1 f is A^-1 g; the backward pass approximates it with a second
        solve on g.  S itself is linear but not symmetric (the cycle is not),
        so S(g) differs from the exact derivative of the algorithm, S^T g, by
        the order of the algebraic error."""

        @staticmethod
        def forward(ctx, f, solver):
            ctx.solver = solver
            return solver.solve(f.contiguous())

        @staticmethod
        def backward(ctx, g):
            return ctx.solver.solve(g.contiguous()), None

    return SRFMGFunction


_FN = None


def solve_autograd(f, solver):
    """Differentiable solve: u = S(f), with dL/df = S(dL/du)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(f, solver)
