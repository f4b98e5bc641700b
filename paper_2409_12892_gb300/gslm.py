"""Thin Python binding of libgslm (include/gslm.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module turns torch
CUDA tensors into device pointers, cameras into ``gslm_camera`` structs, and
status codes into exceptions. PyTorch supplies device memory and the stream.

Names follow the C ABI without the ``gslm_`` prefix: ``render``,
``build_cache``, ``apply_J``, ``apply_JT``, ``jacobi_diag``, ``pcg_solve``,
``combine_accumulate``, ``combine_finish``, ``lm_step``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

try:
    import torch
except ImportError:   # pragma: no cover - torch is part of the image
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgslm.so")
N_PARAMS = 59

c_float, c_double, c_int32, c_int64, c_void_p, c_size_t = (
    ctypes.c_float, ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t)

STATUS = {0: "GSLM_OK", -1: "GSLM_E_INVALID", -2: "GSLM_E_OOM", -3: "GSLM_E_CUDA",
          -4: "GSLM_E_CACHE_OVERFLOW", -5: "GSLM_E_TIMEOUT", -6: "GSLM_E_NUMERIC", 1: "GSLM_W_PCG_BREAKDOWN"}
CACHE_FMT = {"fp32": 0, "bf16": 1, "fp16s": 2, "thin": 3}
OBJECTIVE = {"l2": 0, "l1ssim": 1}


class GslmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("width", c_int32), ("height", c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("cache_fmt", c_int32), ("n_iters", c_int32), ("break_rel2", c_float),
                ("lambda_min", c_float), ("lambda_max", c_float), ("smooth", c_int32),
                ("mem_budget", c_size_t), ("group", c_int32), ("profile", c_int32), ("autotune", c_int32),
                ("batch", c_int32), ("graph", c_int32), ("batch_ctas", c_int32), ("apply_variant", c_int32),
                ("line_search", c_int32), ("pad", c_int32), ("batch_mem", c_size_t), ("objective", c_int32),
                ("lambda_l1", c_float), ("lambda_ssim", c_float), ("res_eps", c_float)]


class CacheInfo(ctypes.Structure):
    _fields_ = [("entries", c_int64), ("segments", c_int64), ("splats", c_int64), ("active_splats", c_int64),
                ("keys", c_int64), ("bytes", c_int64), ("pixels", c_int64), ("views", c_int32),
                ("cache_fmt", c_int32)]


class PcgStats(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("breakdown", c_int32), ("rr", c_double), ("bb", c_double)]


class LMState(ctypes.Structure):
    _fields_ = [("lambda_", c_float), ("step", c_int32)]


class LMStats(ctypes.Structure):
    _fields_ = [("cost", c_double), ("cost_new", c_double), ("predicted", c_double), ("rho", c_double),
                ("accepted", c_int32), ("pcg_iters", c_int32), ("cache_entries", c_int64),
                ("cache_bytes", c_int64), ("ms_total", c_double), ("ms_phase", c_double * 8),
                ("n_pairs", c_int32), ("trial_overflows", c_int32), ("pair_bytes", c_double), ("cache_segments", c_int64),
                ("active_splats", c_int64), ("gamma", c_double), ("ls_evals", c_int32), ("seq_groups", c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgslm.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgslm.so not found at {path}: build it with "
                           "`python -m paper_2409_12892_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "gslm_default_options": (None, [P]),
        "gslm_create": (c_int32, [P, P, P]),
        "gslm_destroy": (None, [P]),
        "gslm_last_error": (ctypes.c_char_p, [P]),
        "gslm_set_options": (c_int32, [P, P]),
        "gslm_render": (c_int32, [P, P, c_int64, c_int64, P, c_int32, P, P, P]),
        "gslm_build_cache": (c_int32, [P, P, c_int64, c_int64, P, c_int32, P, P, P, P, P]),
        "gslm_cache_stats": (c_int32, [P, P]),
        "gslm_cache_free": (None, [P]),
        "gslm_apply_J": (c_int32, [P, P, P, P]),
        "gslm_apply_JT": (c_int32, [P, P, P, P]),
        "gslm_jacobi_diag": (c_int32, [P, P, P]),
        "gslm_pcg_solve": (c_int32, [P, P, P, P, P, c_float, P, P]),
        "gslm_pcg_solve_batch": (c_int32, [P, P, c_int32, P, P, P, c_float, P, P]),
        "gslm_combine_accumulate": (c_int32, [P, c_int64, c_int64, P, P, P, P]),
        "gslm_combine_finish": (c_int32, [P, c_int64, c_int64, P, P, P]),
        "gslm_lm_step": (c_int32, [P, P, c_int64, c_int64, P, c_int32, P, P, P, c_int32, P, P, P]),
        "gslm_version": (ctypes.c_char_p, []),
        "gslm_kernel_launches": (c_int64, []),
        "gslm_memory_usage": (c_int32, [P, c_int32, P]),
        "gslm_cache_weights": (c_int32, [P, P]),
        "gslm_autotune_info": (c_int32, [P, P, P]),
        "gslm_apply_JT_noalloc": (c_int32, [P, P, P, P]),
        "gslm_precond_weight_count": (c_int32, []),
        "gslm_precond_create": (c_int32, [P, P, P, P, ctypes.c_uint64, P]),
        "gslm_precond_free": (None, [P]),
        "gslm_precond_get": (c_int32, [P, P, P, P]),
        "gslm_precond_set": (c_int32, [P, P, P, P]),
        "gslm_precond_features": (c_int32, [P, P, P, P]),
        "gslm_precond_fit_standardizer": (c_int32, [P, P, c_int64]),
        "gslm_precond_apply": (c_int32, [P, P, c_int64, c_int64, P, P]),
        "gslm_precond_backward": (c_int32, [P, P, c_int64, c_int64, P, P, P, c_int32]),
        "gslm_precond_unrolled_grad": (c_int32, [P, P, P, P, c_float, P, c_int32, P, P]),
        "gslm_precond_accumulate": (c_int32, [P, P, P, P, P, c_float, c_int32, c_float, P]),
        "gslm_precond_adam": (c_int32, [P, c_float]),
        "gslm_set_precond": (c_int32, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def kernel_launches() -> int:
    return int(load_library().gslm_kernel_launches())


def exported_symbols() -> list:
    return ["gslm_default_options", "gslm_create", "gslm_destroy", "gslm_last_error", "gslm_set_options",
            "gslm_render", "gslm_build_cache", "gslm_cache_stats", "gslm_cache_free", "gslm_apply_J",
            "gslm_apply_JT", "gslm_jacobi_diag", "gslm_pcg_solve", "gslm_pcg_solve_batch", "gslm_combine_accumulate",
            "gslm_combine_finish", "gslm_lm_step", "gslm_version", "gslm_kernel_launches", "gslm_memory_usage",
            "gslm_cache_weights", "gslm_autotune_info",
            "gslm_apply_JT_noalloc", "gslm_precond_weight_count", "gslm_precond_create", "gslm_precond_free",
            "gslm_precond_get", "gslm_precond_set", "gslm_precond_features", "gslm_precond_fit_standardizer",
            "gslm_precond_apply", "gslm_precond_backward", "gslm_precond_unrolled_grad",
            "gslm_precond_accumulate", "gslm_precond_adam", "gslm_set_precond"]


# ----------------------------------------------------------------------------- marshalling helpers
def padded_ld(n: int, multiple: int = 128) -> int:
    return ((n + multiple - 1) // multiple) * multiple


def to_soa(params_aos, device="cuda", ld: int | None = None):
    """(N, 59) host array -> torch float32 [59, ld] on `device` (zero padding)."""
    a = np.asarray(params_aos, np.float32)
    n = a.shape[0]
    ld = ld or padded_ld(n)
    out = np.zeros((N_PARAMS, ld), np.float32)
    out[:, :n] = a.T
    return torch.from_numpy(out).to(device)


def from_soa(t, n: int) -> np.ndarray:
    """torch [59, ld] -> (N, 59) float64 numpy."""
    return t[:, :n].double().cpu().numpy().T.copy()


def make_cameras(cams) -> ctypes.Array:
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        R = np.asarray(c.R, np.float32).ravel()
        t = np.asarray(c.t, np.float32).ravel()
        arr[i].R[:] = [float(v) for v in R]
        arr[i].t[:] = [float(v) for v in t]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def n_pixels(cams) -> int:
    return int(sum(int(c.width) * int(c.height) for c in cams))


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


@dataclass
class Cache:
    handle: int
    ctx: "Context"
    n: int
    ld: int
    cams: list
    F: object
    b: object
    cost: float

    def info(self) -> CacheInfo:
        ci = CacheInfo()
        self.ctx._check(self.ctx.lib.gslm_cache_stats(ctypes.c_void_p(self.handle), ctypes.byref(ci)))
        return ci

    def weights(self):
        """Residual-to-pixel weights (dr/dc)^2 per pixel channel, [pixels][3] (1 for L2)."""
        w = torch.empty((n_pixels(self.cams), 3), dtype=torch.float32, device=self.b.device if self.b is not None
                        else "cuda")
        self.ctx._check(self.ctx.lib.gslm_cache_weights(ctypes.c_void_p(self.handle), _ptr(w)))
        return w

    def free(self):
        if self.handle:
            self.ctx.lib.gslm_cache_free(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A libgslm context on the current CUDA device and torch's current stream."""

    def __init__(self, cache_fmt="fp32", n_iters=8, break_rel2=0.01, lambda_min=1e-4, lambda_max=1e4,
                 smooth=False, mem_budget=0, group=32, profile=False, autotune=True, batch=True, graph=True,
                 batch_ctas=0, apply_variant=0, line_search=8, batch_mem=0, objective="l2", lambda_l1=0.8,
                 lambda_ssim=0.2, res_eps=1e-4, stream=None):
        self.lib = load_library()
        opt = Options()
        self.lib.gslm_default_options(ctypes.byref(opt))
        opt.cache_fmt = CACHE_FMT[cache_fmt] if isinstance(cache_fmt, str) else int(cache_fmt)
        opt.n_iters, opt.break_rel2 = int(n_iters), float(break_rel2)
        opt.lambda_min, opt.lambda_max = float(lambda_min), float(lambda_max)
        opt.smooth, opt.mem_budget, opt.group = int(bool(smooth)), int(mem_budget), int(group)
        opt.profile = int(bool(profile))
        opt.autotune = int(bool(autotune))
        opt.batch, opt.graph, opt.batch_ctas = int(bool(batch)), int(bool(graph)), int(batch_ctas)
        opt.apply_variant = int(apply_variant)
        opt.line_search = int(line_search)
        opt.batch_mem = int(batch_mem)
        opt.objective = OBJECTIVE[objective] if isinstance(objective, str) else int(objective)
        opt.lambda_l1, opt.lambda_ssim, opt.res_eps = float(lambda_l1), float(lambda_ssim), float(res_eps)
        self.opt = opt
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = ctypes.c_void_p()
        s = self.lib.gslm_create(ctypes.byref(opt), ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
        if s != 0:
            raise GslmError(s, "gslm_create failed")
        self.h = h

    def close(self):
        if self.h:
            self.lib.gslm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int) -> int:
        if s < 0:
            msg = self.lib.gslm_last_error(self.h).decode(errors="replace") if self.h else ""
            raise GslmError(s, msg)
        return s

    def autotune_info(self) -> dict:
        """Kernel variants the autotuner chose: {'apply_J': [fp32, bf16, fp16s], 'apply_JT': [...]}."""
        out = (c_int32 * 6)()
        ms = (c_float * 6)()
        self._check(self.lib.gslm_autotune_info(self.h, out, ms))
        return {"apply_J": list(out[0:3]), "apply_JT": list(out[3:6]), "ms_J": list(ms[0:3]), "ms_JT": list(ms[3:6])}

    def memory_usage(self, reset_peak=False) -> dict:
        """Bytes of the library's memory pool: in use, held (in use + kept for reuse), peak in use."""
        out = (c_int64 * 3)()
        self._check(self.lib.gslm_memory_usage(self.h, int(bool(reset_peak)), out))
        return {"used": out[0], "reserved": out[1], "peak": out[2]}

    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "cache_fmt" and isinstance(v, str):
                v = CACHE_FMT[v]
            setattr(self.opt, k, v)
        self._check(self.lib.gslm_set_options(self.h, ctypes.byref(self.opt)))

    # ------------------------------------------------------------------ calls
    def render(self, params, n: int, cams, targets=None, img=None):
        P = n_pixels(cams)
        if img is None:
            img = torch.empty((P, 3), dtype=torch.float32, device=params.device)
        cost = c_double(0.0)
        ca = make_cameras(cams)
        self._check(self.lib.gslm_render(self.h, _ptr(params), n, params.shape[1], ca, len(cams), _ptr(img),
                                         _ptr(targets), ctypes.byref(cost) if targets is not None else None))
        return img, (cost.value if targets is not None else None)

    def build_cache(self, params, n: int, cams, targets, want_F=True, want_b=True) -> Cache:
        P = n_pixels(cams)
        ld = params.shape[1]
        F = torch.empty((P, 3), dtype=torch.float32, device=params.device) if want_F else None
        b = torch.empty((N_PARAMS, ld), dtype=torch.float32, device=params.device) if want_b else None
        if b is not None:
            b.zero_()
        h = ctypes.c_void_p()
        cost = c_double(0.0)
        ca = make_cameras(cams)
        self._check(self.lib.gslm_build_cache(self.h, _ptr(params), n, ld, ca, len(cams), _ptr(targets),
                                              ctypes.byref(h), _ptr(F), _ptr(b), ctypes.byref(cost)))
        return Cache(h.value, self, n, ld, list(cams), F, b, cost.value)

    def apply_J(self, cache: Cache, p, u=None):
        if u is None:
            u = torch.empty((n_pixels(cache.cams), 3), dtype=torch.float32, device=p.device)
        self._check(self.lib.gslm_apply_J(self.h, ctypes.c_void_p(cache.handle), _ptr(p), _ptr(u)))
        return u

    def apply_JT(self, cache: Cache, u, g=None):
        if g is None:
            g = torch.zeros((N_PARAMS, cache.ld), dtype=torch.float32, device=u.device)
        self._check(self.lib.gslm_apply_JT(self.h, ctypes.c_void_p(cache.handle), _ptr(u), _ptr(g)))
        return g

    def jacobi_diag(self, cache: Cache, diag=None):
        if diag is None:
            diag = torch.zeros((N_PARAMS, cache.ld), dtype=torch.float32, device="cuda")
        self._check(self.lib.gslm_jacobi_diag(self.h, ctypes.c_void_p(cache.handle), _ptr(diag)))
        return diag

    def pcg_solve(self, cache: Cache, b, diag, lam: float, precond=None, x=None, stats=True):
        if x is None:
            x = torch.zeros((N_PARAMS, cache.ld), dtype=torch.float32, device=b.device)
        st = PcgStats()
        s = self._check(self.lib.gslm_pcg_solve(self.h, ctypes.c_void_p(cache.handle), _ptr(b), _ptr(diag),
                                                _ptr(precond), float(lam), _ptr(x),
                                                ctypes.byref(st) if stats else None))
        return x, st, s

    def pcg_solve_batch(self, caches, bs, diags, lam: float, precond=None, xs=None):
        """Algorithm 1 for several subsets in lock step. Returns (xs, [PcgStats], status)."""
        n = len(caches)
        if xs is None:
            xs = [torch.zeros((N_PARAMS, c.ld), dtype=torch.float32, device=b.device) for c, b in zip(caches, bs)]
        arr = lambda vals: (c_void_p * n)(*vals)
        st = (PcgStats * n)()
        pre = arr([_ptr(t) for t in precond]) if precond is not None else None
        s = self._check(self.lib.gslm_pcg_solve_batch(self.h, arr([c.handle for c in caches]), n,
                                                      arr([_ptr(b) for b in bs]), arr([_ptr(d) for d in diags]), pre,
                                                      float(lam), arr([_ptr(x) for x in xs]), st))
        return xs, list(st), s

    def combine_accumulate(self, n: int, delta, diag, num, den):
        self._check(self.lib.gslm_combine_accumulate(self.h, n, delta.shape[1], _ptr(delta), _ptr(diag),
                                                     _ptr(num), _ptr(den)))

    def combine_finish(self, n: int, num, den, delta):
        self._check(self.lib.gslm_combine_finish(self.h, n, num.shape[1], _ptr(num), _ptr(den), _ptr(delta)))

    def precond_features(self, cache: Cache, diag, phi=None):
        """Features [N][64] of the learned preconditioner for a cache's system."""
        if phi is None:
            phi = torch.empty((cache.n, 64), dtype=torch.float32, device=diag.device)
        self._check(self.lib.gslm_precond_features(self.h, ctypes.c_void_p(cache.handle), _ptr(diag), _ptr(phi)))
        return phi

    def unrolled_grad(self, cache: Cache, b, diag, lam: float, D, K: int, want_grad=True):
        """(L, dL/dD) of the K-iteration unrolled PCG residual for the diagonal D."""
        loss = c_double(0.0)
        dD = torch.zeros_like(D) if want_grad else None
        self._check(self.lib.gslm_precond_unrolled_grad(self.h, ctypes.c_void_p(cache.handle), _ptr(b), _ptr(diag),
                                                        float(lam), _ptr(D), int(K), ctypes.byref(loss), _ptr(dD)))
        return loss.value, dD

    def set_precond(self, pc: "Precond | None"):
        """lm_step uses the network for subsets without an explicit preconditioner (None: Jacobi)."""
        self._check(self.lib.gslm_set_precond(self.h, ctypes.c_void_p(pc.h if pc is not None else None)))

    def lm_step(self, params, n: int, cams, targets, subsets, lam: float, step: int = 0, precond=None):
        """One LM step. subsets: list of lists of camera indices. Returns (LMState, LMStats)."""
        ca = make_cameras(cams)
        flat = [int(v) for s in subsets for v in s]
        off = np.cumsum([0] + [len(s) for s in subsets]).astype(np.int32)
        views = (c_int32 * len(flat))(*flat)
        offs = (c_int32 * len(off))(*[int(v) for v in off])
        pre = None
        if precond is not None:
            pre = (c_void_p * len(precond))(*[_ptr(t) for t in precond])
        state = LMState(float(lam), int(step))
        stats = LMStats()
        self._check(self.lib.gslm_lm_step(self.h, _ptr(params), n, params.shape[1], ca, len(cams), _ptr(targets),
                                          views, offs, len(subsets), pre, ctypes.byref(state),
                                          ctypes.byref(stats)))
        return state, stats


def _host_f32(a, n: int):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, np.float32).ravel())
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class Precond:
    """The learned diagonal preconditioner (gslm_precond_*) on a context's device and stream."""

    def __init__(self, ctx: Context, weights=None, mean=None, std=None, seed: int = 0):
        self.ctx, self.lib = ctx, ctx.lib
        self.n_weights = int(self.lib.gslm_precond_weight_count())
        w, m, s = _host_f32(weights, self.n_weights), _host_f32(mean, 64), _host_f32(std, 64)
        h = ctypes.c_void_p()
        f = lambda a: a.ctypes.data_as(c_void_p) if a is not None else None
        ctx._check(self.lib.gslm_precond_create(ctx.h, f(w), f(m), f(s), ctypes.c_uint64(seed), ctypes.byref(h)))
        self.h = h.value

    def free(self):
        if self.h:
            self.lib.gslm_precond_free(ctypes.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def get(self):
        """(weights, mean, std) as float32 numpy arrays."""
        w, m, s = np.empty(self.n_weights, np.float32), np.empty(64, np.float32), np.empty(64, np.float32)
        self.ctx._check(self.lib.gslm_precond_get(ctypes.c_void_p(self.h), w.ctypes.data_as(c_void_p),
                                                  m.ctypes.data_as(c_void_p), s.ctypes.data_as(c_void_p)))
        return w, m, s

    def set(self, weights=None, mean=None, std=None):
        w, m, s = _host_f32(weights, self.n_weights), _host_f32(mean, 64), _host_f32(std, 64)
        f = lambda a: a.ctypes.data_as(c_void_p) if a is not None else None
        self.ctx._check(self.lib.gslm_precond_set(ctypes.c_void_p(self.h), f(w), f(m), f(s)))

    def fit_standardizer(self, phi):
        self.ctx._check(self.lib.gslm_precond_fit_standardizer(ctypes.c_void_p(self.h), _ptr(phi), phi.shape[0]))

    def apply(self, phi, diag, D=None):
        """D [59][ld] = softplus(net(phi)) / clamp(diag)."""
        if D is None:
            D = torch.zeros_like(diag)
        self.ctx._check(self.lib.gslm_precond_apply(ctypes.c_void_p(self.h), _ptr(phi), phi.shape[0], diag.shape[1],
                                                    _ptr(diag), _ptr(D)))
        return D

    def backward(self, phi, diag, dD, grad=None, accumulate=False):
        """Weight gradient for the upstream dL/dD."""
        if grad is None:
            grad = torch.zeros(self.n_weights, dtype=torch.float32, device=diag.device)
        self.ctx._check(self.lib.gslm_precond_backward(ctypes.c_void_p(self.h), _ptr(phi), phi.shape[0],
                                                       diag.shape[1], _ptr(diag), _ptr(dD), _ptr(grad),
                                                       int(bool(accumulate))))
        return grad

    def accumulate(self, cache: Cache, phi, b, diag, lam: float, K: int, weight: float = 1.0) -> float:
        """Adds weight * dL/dweights of the unrolled loss on one system; returns L."""
        loss = c_double(0.0)
        self.ctx._check(self.lib.gslm_precond_accumulate(ctypes.c_void_p(self.h), ctypes.c_void_p(cache.handle),
                                                         _ptr(phi), _ptr(b), _ptr(diag), float(lam), int(K),
                                                         float(weight), ctypes.byref(loss)))
        return loss.value

    def adam(self, lr: float):
        self.ctx._check(self.lib.gslm_precond_adam(ctypes.c_void_p(self.h), float(lr)))
