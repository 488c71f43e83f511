"""Python binding of libspectra_gb (argument marshalling only).

Every computation runs in the CUDA library behind the C ABI declared in
``include/spectra_gb.h``; this module only converts torch tensors to device
pointers and return codes to exceptions.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspectra_gb.so")

OK, EINVAL, ENOTPD, EUNBOUNDED, ENOCONV, ECUDA, ENOMEM = range(7)
ST_OK, ST_NOT_PD, ST_UNBOUNDED, ST_NOCONV, ST_RHO, ST_DEGENERATE, ST_INVALID = range(7)
MODE_FP64, MODE_MIXED, MODE_LEARNED = 0, 1, 2
# solver-path flags of a segment record (sp_record_segments)
SEG_SHIFT_RETRY, SEG_FALLBACK, SEG_LEARNED_OK, SEG_LEARNED_MISS, SEG_NOCONV, SEG_REFINED = (
    1, 2, 4, 8, 16, 32)
MODES = {"fp64": MODE_FP64, "mixed": MODE_MIXED, "learned": MODE_LEARNED}
STAT_NAMES = ["segments", "reflections", "bad_steps", "lanczos_iters", "shift_retries",
              "noconv", "fp64_fallbacks", "power_iters", "learned_ok", "learned_miss"]
NUM_STATS = 12

_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class SpectraError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("spectra_gb error %d: %s" % (code, msg))
        self.code = code


def _bind(L):
    def f(name, args, res=ctypes.c_int):
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    f("sp_last_error", [], ctypes.c_char_p)
    f("sp_version", [], ctypes.c_char_p)
    f("sp_create_spectrahedron", [_i, _i, _vp, ctypes.c_uint32, ctypes.POINTER(_vp)])
    f("sp_destroy_spectrahedron", [_vp])
    f("sp_spec_dims", [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)])
    f("sp_set_solver", [_vp, _i, _d, _d])
    f("sp_membership", [_vp, _i, _vp, _vp, _vp])
    f("sp_set_mixed_solver", [_vp, _d, _d, _d, _i])
    f("sp_volume_estimate", [_vp, _d, _d, _d, _i, _i, _i, _i, _i, ctypes.c_uint64, _vp, _vp,
                             _vp])
    f("sp_intersect", [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp])
    f("sp_reflect", [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp])
    f("sp_init_chains", [_vp, _i, _vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(_vp),
                         _vp])
    f("sp_destroy_chains", [_vp])
    f("sp_step_billiard", [_vp, _i, _d, _i, _d, _i, _vp])
    f("sp_step_hnr", [_vp, _i, _i, _vp])
    f("sp_step_cdhr", [_vp, _i, _i, _vp])
    f("sp_get_state", [_vp, _vp, ctypes.POINTER(ctypes.c_uint32), _vp])
    f("sp_set_state", [_vp, _vp, ctypes.c_uint32, _vp])
    f("sp_chain_status", [_vp, _vp, ctypes.POINTER(ctypes.c_longlong), _vp])
    f("sp_intersect_noalloc", [_i, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp])
    f("sp_form_pencil", [_vp, _i, _vp, _vp, _vp, _vp, _i, _vp])
    f("sp_set_stage_timers", [_vp, _vp])
    f("sp_attach_mlp", [_vp, _vp, _d, _d, _d, _i])
    f("sp_record_tuples", [_vp, _vp, _vp, _i, _vp])
    f("sp_kernel_timing", [_vp, _i, _vp])
    f("sp_record_segments", [_vp, _vp, _i, _i, _vp])
    f("sp_learned_counts", [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)])
    f("sp_selftest_recip", [_i, _vp, _vp, _vp])
    f("sp_halfspace_fraction", [_vp, _vp, _d, _d, _i, _vp, _vp])
    f("sp_curve_reflect", [_vp, _i, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp])
    f("sp_step_hmc", [_vp, _i, _vp, _d, _d, _i, _d, _vp])
    f("sp_create_batch", [_i, _vp, _vp, ctypes.c_uint64, ctypes.POINTER(_vp), _vp])
    f("sp_destroy_batch", [_vp])
    f("sp_batch_billiard", [_vp, _i, _vp, _i, _d, _vp])
    f("sp_batch_dims", [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                        ctypes.POINTER(_i)])
    f("sp_batch_state", [_vp, _i, _vp, ctypes.POINTER(ctypes.c_uint32), _vp])
    f("sp_batch_stats", [_vp, _vp, _vp])
    f("sp_batch_panels", [_vp, _vp, _vp])
    f("sp_batch_tune", [_vp, ctypes.c_char_p, _vp, _vp])
    f("sp_mlp_create", [_i, _i, _i, ctypes.c_uint64, ctypes.POINTER(_vp)])
    f("sp_mlp_destroy", [_vp])
    f("sp_mlp_dims", [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                      ctypes.POINTER(ctypes.c_longlong)])
    f("sp_mlp_params", [_vp, _vp, _vp])
    f("sp_mlp_forward", [_vp, _i, _vp, _vp, _vp])
    f("sp_mlp_gradients", [_vp, _i, _vp, _vp, _vp, _vp, _vp])
    f("sp_mlp_train", [_vp, _i, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp])
    f("sp_mlp_save", [_vp, ctypes.c_char_p])
    f("sp_mlp_load", [ctypes.c_char_p, ctypes.c_uint64, ctypes.POINTER(_vp)])


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libspectra_gb.so is not built (run paper_2010_03817_gb300/"
                                   "build.py or __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            _bind(L)
            _lib = L
    return _lib


def _check(code: int):
    if code != OK:
        raise SpectraError(code, lib().sp_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev(t, dtype=None, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, shape, tuple(t.shape)))
    return _vp(t.data_ptr())


def pack_lmi(A) -> np.ndarray:
    """(n+1, m, m) stack -> (n+1, m(m+1)/2): lower triangles packed row by row."""
    A = np.asarray(A, dtype=np.float64)
    il = np.tril_indices(A.shape[1])
    return np.ascontiguousarray(A[:, il[0], il[1]])


def intersect_noalloc(A_packed, n: int, m: int, x, v, t_minus, t_plus, status, stream=None):
    """sp_intersect_noalloc: every buffer is the caller's (CUDA tensors); the
    library allocates nothing."""
    import torch
    C = x.shape[0]
    _check(lib().sp_intersect_noalloc(
        n, m, _dev(A_packed, torch.float64, (n + 1, m * (m + 1) // 2), "A_packed"), C,
        _dev(x, torch.float64, (C, n), "x"), _dev(v, torch.float64, (C, n), "v"),
        _dev(t_minus, torch.float64, (C,), "t_minus"), _dev(t_plus, torch.float64, (C,), "t_plus"),
        _dev(status, torch.int32, (C,), "status"), _stream(stream)))


def decode_segments(buf, count: int, every: int, n: int) -> dict:
    """Split the filled slots of a segment record (sp_record_segments) into
    host arrays p, v, w_hat (K x n), t_plus, t_minus, status, reflected,
    chain, step, k (the segment's index in its step) and flags (the solver
    path: SEG_* bits) (K each)."""
    filled = min(buf.shape[0], (int(count) + every - 1) // every)
    R = buf[:filled].cpu().numpy()
    return {"p": R[:, :n], "v": R[:, n:2 * n], "w_hat": R[:, 2 * n:3 * n],
            "t_plus": R[:, 3 * n], "t_minus": R[:, 3 * n + 1],
            "status": R[:, 3 * n + 2].astype(np.int32), "reflected": R[:, 3 * n + 3] > 0.5,
            "chain": R[:, 3 * n + 4].astype(np.int64), "step": R[:, 3 * n + 5].astype(np.int64),
            "k": R[:, 3 * n + 6].astype(np.int64), "flags": R[:, 3 * n + 7].astype(np.int64)}


def selftest_recip(x, stream=None):
    """The dense kernels' 1/sqrt(x) and 1/x routines on a CUDA float64 vector
    x: (count, 4) = FP64 rsqrt, FP64 reciprocal, double-float rsqrt,
    double-float reciprocal (sp_selftest_recip)."""
    import torch
    C = x.shape[0]
    out = torch.empty((C, 4), dtype=torch.float64, device=x.device)
    _check(lib().sp_selftest_recip(C, _dev(x, torch.float64, (C,), "x"), _dev(out),
                                   _stream(stream)))
    return out


def version() -> str:
    return lib().sp_version().decode()


class Spectrahedron:
    """Device-resident LMI F(x) = A_0 + sum_i x_i A_i (Eq. 1).

    A: (n+1, m, m) float64 array-like on the host; fp64_only skips the mixed
    path's precomputed operands (SP_FLAG_FP64_ONLY)."""

    def __init__(self, A, fp64_only: bool = False):
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        if A.ndim != 3 or A.shape[1] != A.shape[2]:
            raise ValueError("A must be (n+1) x m x m")
        self.n = A.shape[0] - 1
        self.m = A.shape[1]
        h = _vp()
        _check(lib().sp_create_spectrahedron(self.n, self.m, A.ctypes.data_as(_vp),
                                             1 if fp64_only else 0, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().sp_destroy_spectrahedron(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def attach_mlp(self, net, x_scale: float = 1.0, t_scale: float = 1.0, margin: float = 0.05,
                   iters: int = 12):
        """Warm-start network for SP_MODE_LEARNED walks (None detaches)."""
        self._mlp = net
        _check(lib().sp_attach_mlp(self._h, net.handle if net is not None else None, x_scale,
                                   t_scale, margin, iters))

    def learned_counts(self):
        """(accepted, rejected) warm starts of the last learned reflect call."""
        a, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().sp_learned_counts(self._h, ctypes.byref(a), ctypes.byref(r)))
        return a.value, r.value

    def set_stage_timers(self, timers=None):
        """Mixed-path stage timers: an int64 CUDA tensor (SMs x 16), or None."""
        import torch
        _check(lib().sp_set_stage_timers(self._h, _dev(timers, torch.int64) if timers is not None
                                         else None))

    def set_solver(self, kmax: int = 96, tol: float = 1e-13, sigma_frac: float = 0.1):
        _check(lib().sp_set_solver(self._h, kmax, tol, sigma_frac))

    def set_mixed_solver(self, tol32: float = 1e-4, tol64: float = 1e-10, delta1: float = 2e-4,
                         power_iters: int = 8):
        """Stage-1 / stage-2 parameters of the mixed path (sp_set_mixed_solver)."""
        _check(lib().sp_set_mixed_solver(self._h, tol32, tol64, delta1, power_iters))

    # -- primitives ---------------------------------------------------------
    def form_pencil(self, x=None, v=None, mode: str = "fp64", stream=None):
        """(F(x_c), V_c) as packed lower triangles (count x m(m+1)/2); either
        argument may be None."""
        import torch
        ref = x if x is not None else v
        C = ref.shape[0]
        P = self.m * (self.m + 1) // 2
        F = torch.empty((C, P), dtype=torch.float64, device=ref.device) if x is not None else None
        V = torch.empty((C, P), dtype=torch.float64, device=ref.device) if v is not None else None
        _check(lib().sp_form_pencil(
            self._h, C, _dev(x, torch.float64, (C, self.n), "x") if x is not None else None,
            _dev(v, torch.float64, (C, self.n), "v") if v is not None else None,
            _dev(F) if F is not None else None, _dev(V) if V is not None else None, MODES[mode],
            _stream(stream)))
        return F, V

    def volume(self, r_inner: float, r_outer: float, ratio: float = 0.5, chains: int = 4096,
               burn_in: int = 10, steps: int = 20, walk: str = "billiard", mode: str = "fp64",
               seed: int = 1, stream=None):
        """Multiphase Monte Carlo volume over a sequence of balls (sp_volume_estimate):
        (volume, {"phases", "samples_per_phase", "rel_std_err", "seconds"})."""
        vol = ctypes.c_double(0.0)
        info = (ctypes.c_double * 4)()
        _check(lib().sp_volume_estimate(self._h, r_inner, r_outer, ratio, chains, burn_in, steps,
                                        {"billiard": 0, "hnr": 1}[walk], MODES[mode], seed,
                                        ctypes.byref(vol), info, _stream(stream)))
        return vol.value, {"phases": int(info[0]), "samples_per_phase": int(info[1]),
                           "rel_std_err": info[2], "seconds": info[3]}

    def membership(self, x, stream=None):
        import torch
        C = x.shape[0]
        inside = torch.empty(C, dtype=torch.int32, device=x.device)
        _check(lib().sp_membership(self._h, C, _dev(x, torch.float64, (C, self.n), "x"),
                                   _dev(inside), _stream(stream)))
        return inside

    def intersect(self, x, v, want_u: bool = False, mode: str = "fp64", stream=None):
        """Alg. 2 for the lines x_c + t v_c: (t_minus, t_plus, u or None, status)."""
        import torch
        C = x.shape[0]
        dev = x.device
        tm = torch.empty(C, dtype=torch.float64, device=dev)
        tp = torch.empty(C, dtype=torch.float64, device=dev)
        st = torch.empty(C, dtype=torch.int32, device=dev)
        u = torch.empty((C, self.m), dtype=torch.float64, device=dev) if want_u else None
        _check(lib().sp_intersect(self._h, C, _dev(x, torch.float64, (C, self.n), "x"),
                                  _dev(v, torch.float64, (C, self.n), "v"), _dev(tm), _dev(tp),
                                  _dev(u) if want_u else None, _dev(st), MODES[mode],
                                  _stream(stream)))
        return tm, tp, u, st

    def reflect(self, x, v, mode: str = "fp64", stream=None):
        """Alg. 3 for the lines x_c + t v_c: (t_plus, w_hat, s, status)."""
        import torch
        C = x.shape[0]
        dev = x.device
        tp = torch.empty(C, dtype=torch.float64, device=dev)
        wh = torch.empty((C, self.n), dtype=torch.float64, device=dev)
        s = torch.empty((C, self.n), dtype=torch.float64, device=dev)
        st = torch.empty(C, dtype=torch.int32, device=dev)
        _check(lib().sp_reflect(self._h, C, _dev(x, torch.float64, (C, self.n), "x"),
                                _dev(v, torch.float64, (C, self.n), "v"), _dev(tp), _dev(wh),
                                _dev(s), _dev(st), MODES[mode], _stream(stream)))
        return tp, wh, s, st

    def curve_reflect(self, x, v, c, T: float, stream=None):
        """REFLECTION of the HMC trajectories x_c + v_c t - (c / (2T)) t^2 of
        the Boltzmann density exp(-c.x / T) (Sec. 3.3; m <= 64):
        (t_plus, w_hat, s, status), s the reflected velocity at the hit point;
        c: host array (n)."""
        import torch
        C = x.shape[0]
        dev = x.device
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
        if c.shape != (self.n,):
            raise ValueError("c must have n entries")
        tp = torch.empty(C, dtype=torch.float64, device=dev)
        wh = torch.empty((C, self.n), dtype=torch.float64, device=dev)
        s = torch.empty((C, self.n), dtype=torch.float64, device=dev)
        st = torch.empty(C, dtype=torch.int32, device=dev)
        _check(lib().sp_curve_reflect(self._h, C, _dev(x, torch.float64, (C, self.n), "x"),
                                      _dev(v, torch.float64, (C, self.n), "v"),
                                      c.ctypes.data_as(_vp), T, _dev(tp), _dev(wh), _dev(s),
                                      _dev(st), _stream(stream)))
        return tp, wh, s, st


class Chains:
    """C independent walkers on a Spectrahedron (state on the device)."""

    def __init__(self, spec: Spectrahedron, C: int, x0=None, seed: int = 0, chain0: int = 0,
                 stream=None):
        import torch
        self.spec = spec
        self.C = C
        h = _vp()
        if x0 is None:
            ptr = None
        elif isinstance(x0, torch.Tensor) and x0.is_cuda:
            ptr = _dev(x0, torch.float64, (C, spec.n), "x0")
        else:
            x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64))
            if x0.shape != (C, spec.n):
                raise ValueError("x0 must be (C, n)")
            self._x0_host = x0
            ptr = x0.ctypes.data_as(_vp)
        _check(lib().sp_init_chains(spec.handle, C, ptr, seed, chain0, ctypes.byref(h),
                                    _stream(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().sp_destroy_chains(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def billiard(self, steps: int, tau: float, rho: int = 100, kappa: float = 1e-6,
                 mode: str = "fp64", stream=None):
        _check(lib().sp_step_billiard(self._h, steps, tau, rho, kappa, MODES[mode],
                                      _stream(stream)))

    def hnr(self, steps: int, mode: str = "fp64", stream=None):
        _check(lib().sp_step_hnr(self._h, steps, MODES[mode], _stream(stream)))

    def cdhr(self, steps: int, mode: str = "fp64", stream=None):
        _check(lib().sp_step_cdhr(self._h, steps, MODES[mode], _stream(stream)))

    def hmc(self, steps: int, c, T: float, tau: float, rho: int = 100, kappa: float = 1e-6,
            stream=None):
        """HMC with reflections for exp(-c.x / T) (Alg. 6, sp_step_hmc); c: host array (n)."""
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
        if c.shape != (self.spec.n,):
            raise ValueError("c must have n entries")
        _check(lib().sp_step_hmc(self._h, steps, c.ctypes.data_as(_vp), T, tau, rho, kappa,
                                 _stream(stream)))

    def state(self, stream=None):
        """(x as a CUDA float64 tensor (C, n), next step number)."""
        import torch
        x = torch.empty((self.C, self.spec.n), dtype=torch.float64, device="cuda")
        step = ctypes.c_uint32(0)
        _check(lib().sp_get_state(self._h, _dev(x), ctypes.byref(step), _stream(stream)))
        return x, step.value

    def state_host(self, out: np.ndarray | None = None, stream=None):
        """Copy the points into a host array (synchronises the stream)."""
        if out is None:
            out = np.empty((self.C, self.spec.n), dtype=np.float64)
        step = ctypes.c_uint32(0)
        _check(lib().sp_get_state(self._h, out.ctypes.data_as(_vp), ctypes.byref(step),
                                  _stream(stream)))
        return out, step.value

    def set_state(self, x, step: int, stream=None):
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            ptr = _dev(x, torch.float64, (self.C, self.spec.n), "x")
        else:
            x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
            ptr = x.ctypes.data_as(_vp)
        _check(lib().sp_set_state(self._h, ptr, step, _stream(stream)))

    def kernel_timing(self, enable: int = -1):
        """Per-kernel CUDA-event timing of walk calls (see sp_kernel_timing)."""
        out = (ctypes.c_double * 13)()
        _check(lib().sp_kernel_timing(self._h, enable, out))
        k = ["fp64_ms", "fp64_launches", "form_ms", "form_launches", "wave_ms", "wave_launches",
             "mlp_ms", "mlp_launches", "other_launches", "contract_ms", "contract_launches",
             "finish_ms", "finish_launches"]
        return {name: out[i] for i, name in enumerate(k)}

    def record(self, x_out=None, y_out=None, count=None):
        """Record (features, targets) tuples of later mixed / learned Billiard
        walks into CUDA tensors (x_out: cap x 2n, y_out: cap x (1+m) float32,
        count: int32 scalar tensor, zeroed by the caller); no arguments stop."""
        import torch
        if x_out is None:
            _check(lib().sp_record_tuples(self._h, None, None, 0, None))
            return
        cap = x_out.shape[0]
        _check(lib().sp_record_tuples(self._h, _dev(x_out, torch.float32), _dev(y_out, torch.float32),
                                      cap, _dev(count, torch.int32)))

    def halfspace_fraction(self, c, b1: float, b2: float, groups: int = 1, stream=None):
        """Per group of C / groups chains, the fraction of points with
        c.x <= b1 or c.x >= b2 (sp_halfspace_fraction); c: host array (n)."""
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
        if c.shape != (self.spec.n,):
            raise ValueError("c must have n entries")
        out = np.zeros(groups, dtype=np.float64)
        _check(lib().sp_halfspace_fraction(self._h, c.ctypes.data_as(_vp), b1, b2, groups,
                                           out.ctypes.data_as(_vp), _stream(stream)))
        return out

    def record_segments(self, buf=None, count=None, every: int = 1):
        """Record every `every`-th boundary-oracle call of later walks into buf
        (CUDA float64 tensor, capacity x (3n + 8)) with the int32 ticket
        counter `count` (zeroed by the caller); no arguments stop."""
        import torch
        if buf is None:
            _check(lib().sp_record_segments(self._h, None, 0, 1, None))
            return
        n = self.spec.n
        if buf.dim() != 2 or buf.shape[1] != 3 * n + 8:
            raise ValueError("buf must be (capacity, 3n + 8)")
        _check(lib().sp_record_segments(self._h, _dev(buf, torch.float64), buf.shape[0], every,
                                        _dev(count, torch.int32)))

    def status(self, stream=None):
        """(per-chain status tensor, dict of summed statistics)."""
        import torch
        st = torch.empty(self.C, dtype=torch.int32, device="cuda")
        stats = (ctypes.c_longlong * NUM_STATS)()
        _check(lib().sp_chain_status(self._h, _dev(st), stats, _stream(stream)))
        return st, {k: int(stats[i]) for i, k in enumerate(STAT_NAMES)}


class Batch:
    """Spectrahedra of uneven sizes walked together in one persistent launch
    (sp_create_batch / sp_batch_*; FP64 path).  specs: Spectrahedron objects
    (kept alive by the batch); chains: chains per body (start: the origin)."""

    def __init__(self, specs, chains, seed: int = 0, stream=None):
        self.specs = list(specs)
        self.B = len(self.specs)
        hs = (_vp * self.B)(*[sp.handle for sp in self.specs])
        cs = np.ascontiguousarray(np.asarray(chains, dtype=np.int32))
        h = _vp()
        _check(lib().sp_create_batch(self.B, ctypes.cast(hs, _vp), cs.ctypes.data_as(_vp), seed,
                                     ctypes.byref(h), _stream(stream)))
        self._h = h
        self.chains = cs.tolist()

    def close(self):
        if getattr(self, "_h", None):
            lib().sp_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def billiard(self, steps: int, tau, rho: int = 100, kappa: float = 1e-6, stream=None):
        t = np.ascontiguousarray(np.asarray(tau, dtype=np.float64).reshape(-1))
        if t.size == 1:
            t = np.full(self.B, float(t[0]))
        _check(lib().sp_batch_billiard(self._h, steps, t.ctypes.data_as(_vp), rho, kappa,
                                       _stream(stream)))

    def dims(self, body: int):
        n, m, c, c0 = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().sp_batch_dims(self._h, body, ctypes.byref(n), ctypes.byref(m),
                                   ctypes.byref(c), ctypes.byref(c0)))
        return n.value, m.value, c.value, c0.value

    def state(self, body: int, stream=None) -> np.ndarray:
        n, _, c, _ = self.dims(body)
        out = np.empty((c, n), dtype=np.float64)
        _check(lib().sp_batch_state(self._h, body, out.ctypes.data_as(_vp), None,
                                    _stream(stream)))
        return out

    def stats(self, stream=None):
        out = np.zeros((self.B, NUM_STATS), dtype=np.int64)
        _check(lib().sp_batch_stats(self._h, out.ctypes.data_as(_vp), _stream(stream)))
        return [{k: int(out[b, i]) for i, k in enumerate(STAT_NAMES)} for b in range(self.B)]

    def panels(self, new=None):
        out = np.zeros(self.B, dtype=np.int32)
        p_in = None
        if new is not None:
            p_in = np.ascontiguousarray(np.asarray(new, dtype=np.int32))
        _check(lib().sp_batch_panels(self._h, out.ctypes.data_as(_vp),
                                     p_in.ctypes.data_as(_vp) if p_in is not None else None))
        return out

    def tune(self, cache_path=None, stream=None):
        """Autotune the Cholesky panel width per body (sp_batch_tune);
        returns (panels, calibration ms per width 4/8/16)."""
        times = np.zeros((self.B, 3), dtype=np.float64)
        _check(lib().sp_batch_tune(self._h, os.fsencode(cache_path) if cache_path else None,
                                   times.ctypes.data_as(_vp), _stream(stream)))
        return self.panels(), times


class MLP:
    """The warm-start network din -> dh -> dh -> dout on the GPU (sp_mlp_*)."""

    def __init__(self, din: int, dh: int, dout: int, seed: int = 0):
        h = _vp()
        _check(lib().sp_mlp_create(din, dh, dout, seed, ctypes.byref(h)))
        self._h = h
        self.din, self.dh, self.dout = din, dh, dout
        npar = ctypes.c_longlong(0)
        _check(lib().sp_mlp_dims(h, None, None, None, ctypes.byref(npar)))
        self.nparams = npar.value

    @classmethod
    def load(cls, path: str, seed: int = 0) -> "MLP":
        """A network saved by save() (sp_mlp_load)."""
        h = _vp()
        _check(lib().sp_mlp_load(os.fsencode(path), seed, ctypes.byref(h)))
        q = cls.__new__(cls)
        q._h = h
        din, dh, dout = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        npar = ctypes.c_longlong(0)
        _check(lib().sp_mlp_dims(h, ctypes.byref(din), ctypes.byref(dh), ctypes.byref(dout),
                                 ctypes.byref(npar)))
        q.din, q.dh, q.dout, q.nparams = din.value, dh.value, dout.value, npar.value
        return q

    def save(self, path: str) -> None:
        """Write the network to a file (sp_mlp_save)."""
        _check(lib().sp_mlp_save(self._h, os.fsencode(path)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().sp_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """[(name, shape)] of the flat parameter vector."""
        doutp = (self.dout + 15) // 16 * 16
        dinp = (self.din + 7) // 8 * 8
        return [("W1", (self.dh, dinp)), ("b1", (self.dh,)), ("W2", (self.dh, self.dh)),
                ("b2", (self.dh,)), ("W3", (doutp, self.dh)), ("b3", (doutp,))]

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        _check(lib().sp_mlp_params(self._h, out.ctypes.data_as(_vp), None))
        return out

    def set_params(self, flat) -> None:
        flat = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        assert flat.size == self.nparams
        _check(lib().sp_mlp_params(self._h, None, flat.ctypes.data_as(_vp)))

    def unflatten(self, flat):
        out, o = [], 0
        for _, shp in self.layout():
            k = int(np.prod(shp))
            out.append(np.asarray(flat[o:o + k]).reshape(shp))
            o += k
        return out

    def forward(self, X, stream=None):
        import torch
        B = X.shape[0]
        Y = torch.empty((B, self.dout), dtype=torch.float32, device=X.device)
        _check(lib().sp_mlp_forward(self._h, B, _dev(X, torch.float32, (B, self.din), "X"),
                                    _dev(Y), _stream(stream)))
        return Y

    def gradients(self, X, T, stream=None):
        """(loss, flat gradient) for one batch (B a multiple of 8)."""
        import torch
        B = X.shape[0]
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().sp_mlp_gradients(self._h, B, _dev(X, torch.float32, (B, self.din), "X"),
                                      _dev(T, torch.float32, (B, self.dout), "T"),
                                      g.ctypes.data_as(_vp), ctypes.byref(loss), _stream(stream)))
        return float(loss.value), g

    def train(self, X, T, epochs: int, batch: int, lr: float, stream=None):
        import torch
        B = X.shape[0]
        losses = np.zeros(epochs, dtype=np.float32)
        _check(lib().sp_mlp_train(self._h, B, _dev(X, torch.float32, (B, self.din), "X"),
                                  _dev(T, torch.float32, (B, self.dout), "T"), epochs, batch,
                                  ctypes.c_float(lr), losses.ctypes.data_as(_vp), _stream(stream)))
        return losses
