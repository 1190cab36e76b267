"""Thin Python binding of libatkm (include/atkm.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts torch
tensors to device pointers, fills the C structs and checks return codes.  It
raises if the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libatkm.so")

ATKM_OK = 0
ATKM_ERR_ARG = 1
ATKM_ERR_UNSUPPORTED_SIZE = 2
ATKM_ERR_OOM = 3
ATKM_ERR_CUDA = 4
ATKM_NOT_CONVERGED = 5
ATKM_STAGNATED = 6
ATKM_ERR_NAN = 7
ATKM_ERR_TIMEOUT = 8
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_UNSUPPORTED_SIZE", 3: "ERR_OOM", 4: "ERR_CUDA",
                5: "NOT_CONVERGED", 6: "STAGNATED", 7: "ERR_NAN", 8: "ERR_TIMEOUT"}
ATKM_PLAN_F32 = 1
ATKM_PLAN_DF32 = 2
ATKM_PLAN_GENERIC_FFT = 4
ATKM_PLAN_AUTOTUNE = 8
PRECISION_F64 = 0
PRECISION_F32_F64 = 1
PRECISION_F32_SPLIT = 2
PRECISION_DF32_SPLIT = 3
ATKM_GEMM_TCGEN05 = 0
ATKM_GEMM_MMA_SYNC = 1
ATKM_GEMM_TCGEN05_WAIT_TEST = 2


class AtkmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double * 3), ("beta", C.c_double), ("lam", C.c_double), ("Omega", C.c_double)]


class Energy(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("E", "E_kin", "E_pot", "E_int", "E_dip", "E_rot", "mu", "virial", "norm2")]


class PcgOpts(C.Structure):
    _fields_ = [("tol_residual", C.c_double), ("tol_linf", C.c_double), ("max_iter", C.c_int),
                ("max_halvings", C.c_int), ("precision_mode", C.c_int), ("switch_tol", C.c_double),
                ("log_capacity", C.c_int), ("resume", C.c_int), ("no_graphs", C.c_int), ("time_limit_s", C.c_double),
                ("f32_window", C.c_int), ("f32_gain", C.c_double), ("mg_f64_levels", C.c_int)]


class IterLog(C.Structure):
    _fields_ = [("n", C.c_int), ("halvings", C.c_int), ("reset_to_sd", C.c_int), ("accepted", C.c_int),
                ("f32_phase", C.c_int), ("pad_", C.c_int)] + \
               [(k, C.c_double) for k in ("E", "mu", "residual", "linf_step", "alpha", "beta_cg", "d1",
                                          "curvature", "t0", "t")]


class TuneInfo(C.Structure):
    _fields_ = [("precision", C.c_int), ("length", C.c_int), ("line_major", C.c_int), ("engine", C.c_int),
                ("tile_shift", C.c_int), ("pad_", C.c_int), ("ms_default", C.c_double), ("ms_best", C.c_double)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int), ("pad_", C.c_int), ("ms_total", C.c_double),
                ("bytes_total", C.c_double), ("flops_total", C.c_double)]


class Result(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("E", "mu", "E_kin", "E_pot", "E_int", "E_dip", "E_rot", "virial",
                                          "residual", "linf_step")] + \
               [("iters", C.c_int), ("halvings", C.c_int), ("f32_iters", C.c_int), ("status", C.c_int),
                ("log", C.POINTER(IterLog)), ("log_count", C.c_int), ("device_loop", C.c_int),
                ("switch_residual", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libatkm.so (built by paper_2603_05194_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libatkm.so not found at {path}: run `python -m paper_2603_05194_gb300.build`")
    lib = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "atkm_plan_create": (ip, [C.POINTER(vp), C.POINTER(C.c_int), dp, dp, C.c_uint, vp]),
        "atkm_plan_destroy": (None, [vp]),
        "atkm_last_error_string": (C.c_char_p, [vp]),
        "atkm_plan_device_bytes": (C.c_ulonglong, [vp]),
        "atkm_plan_copy_U0": (ip, [vp, vp, vp]),
        "atkm_plan_copy_multiplier": (ip, [vp, vp, vp]),
        "dipolar_potential": (ip, [vp, vp, vp, vp]),
        "dipolar_potential_from_psi": (ip, [vp, vp, vp, vp]),
        "dipolar_potential_from_pair": (ip, [vp, vp, vp, vp, vp]),
        "dipolar_potential_from_psi_f32": (ip, [vp, vp, vp, vp]),
        "dipolar_potential_from_psi_df32": (ip, [vp, vp, vp, vp]),
        "apply_H": (ip, [vp, C.POINTER(Params), vp, vp, vp, vp, vp]),
        "atkm_energy_parts": (ip, [vp, C.POINTER(Params), vp, vp, C.POINTER(Energy), vp]),
        "apply_preconditioner": (ip, [vp, C.POINTER(Params), C.c_double, vp, vp, vp, vp, vp]),
        "pcg_ground_state": (ip, [vp, C.POINTER(Params), C.POINTER(PcgOpts), vp, C.POINTER(Result), vp]),
        "pcg_ground_state_batched": (ip, [C.c_int, C.POINTER(vp), C.POINTER(Params), C.POINTER(PcgOpts),
                                          C.POINTER(vp), C.POINTER(Result), vp]),
        "atkm_spectral_upsample": (ip, [vp, vp, vp, vp, vp]),
        "pcg_ground_state_mg": (ip, [C.c_int, C.POINTER(vp), C.POINTER(Params), C.POINTER(PcgOpts),
                                     C.POINTER(vp), C.POINTER(Result), vp]),
        "atkm_guess_net_num_params": (C.c_ulonglong, []),
        "atkm_guess_net_create": (ip, [C.POINTER(vp), C.c_ulonglong, vp]),
        "atkm_guess_net_destroy": (None, [vp]),
        "atkm_guess_net_get_params": (ip, [vp, vp, vp]),
        "atkm_guess_net_set_params": (ip, [vp, vp, vp]),
        "atkm_guess_net_forward": (ip, [vp, C.c_int, vp, vp, vp]),
        "atkm_guess_net_grad": (ip, [vp, C.c_int, vp, vp, vp, vp, vp]),
        "atkm_guess_net_train_step": (ip, [vp, C.c_int, vp, vp, C.c_float, vp, vp]),
        "atkm_guess_net_set_gemm_engine": (ip, [vp, C.c_int]),
        "atkm_guess_net_check": (ip, [vp, vp]),
        "atkm_guess_net_profile_step": (ip, [vp, C.c_int, vp, vp, C.c_float, vp, dp, dp, C.POINTER(C.c_int), dp,
                                             C.c_int, vp]),
        "atkm_plan_set_profiling": (ip, [vp, C.c_int]),
        "atkm_measure_fp64_fma": (ip, [C.c_int, C.c_int, C.c_int, dp, vp]),
        "atkm_launch_count": (C.c_ulonglong, []),
        "atkm_inner_products_noalloc": (ip, [C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_ulonglong, C.c_double, vp,
                                             vp]),
        "atkm_plan_kernel_stats": (ip, [vp, C.POINTER(KernelStat), C.c_int, C.POINTER(C.c_int)]),
        "atkm_plan_autotune": (ip, [vp, vp]),
        "atkm_plan_tuning": (ip, [vp, C.POINTER(TuneInfo), C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def pcg_ground_state_batched(plans, params, psis, tol_residual=1e-8, tol_linf=0.0, max_iter=10000, max_halvings=20,
                             precision=PRECISION_F64, switch_tol=1e-5, stream=None, graphs=True,
                             time_limit_s=0.0, f32_window=0, f32_gain=0.0) -> list:
    """Runs independent solves (one plan each, grids may differ) concurrently
    through pcg_ground_state_batched; returns one result dict per instance."""
    lib = load_library()
    n = len(plans)
    if not (n == len(params) == len(psis)) or n == 0:
        raise ValueError("plans, params and psis must have the same, non-zero length")
    for pl, ps in zip(plans, psis):
        _ptr(ps, torch.complex128, pl.shape, "psi")
    opts = PcgOpts(tol_residual, tol_linf, max_iter, max_halvings, precision, switch_tol, 0, 0, 0 if graphs else 1,
                   time_limit_s, f32_window, f32_gain, 0)
    ph = (C.c_void_p * n)(*[pl._h for pl in plans])
    pa = (Params * n)(*params)
    pp = (C.c_void_p * n)(*[C.c_void_p(t.data_ptr()) for t in psis])
    res = (Result * n)()
    code = lib.pcg_ground_state_batched(n, ph, pa, C.byref(opts), pp, res, _stream(stream))
    if code not in (ATKM_OK, ATKM_NOT_CONVERGED, ATKM_STAGNATED, ATKM_ERR_NAN, ATKM_ERR_TIMEOUT):
        raise AtkmError(code, lib.atkm_last_error_string(None).decode())
    outs = []
    for i in range(n):
        d = {k: getattr(res[i], k) for k, _ in Result._fields_ if k != "log"}
        d["status_name"] = STATUS_NAMES.get(res[i].status, str(res[i].status))
        outs.append(d)
    return outs


def pcg_ground_state_mg(plans, params, psis, tol_residual=1e-8, tol_linf=0.0, max_iter=10000, max_halvings=20,
                        precision=PRECISION_F64, switch_tol=1e-5, stream=None, graphs=True, time_limit_s=0.0,
                        f32_window=0, f32_gain=0.0, mg_f64_levels=0) -> list:
    """Cascadic multigrid PCG-ATKM-MG through pcg_ground_state_mg: plans and
    psis from the coarsest level to the finest, psis[0] the initial guess;
    with a precision form the mg_f64_levels coarsest levels run in FP64.
    Returns one result dict per level."""
    lib = load_library()
    n = len(plans)
    if n == 0 or len(psis) != n:
        raise ValueError("plans and psis must have the same, non-zero length")
    for pl, ps in zip(plans, psis):
        _ptr(ps, torch.complex128, pl.shape, "psi")
    opts = PcgOpts(tol_residual, tol_linf, max_iter, max_halvings, precision, switch_tol, 0, 0, 0 if graphs else 1,
                   time_limit_s, f32_window, f32_gain, mg_f64_levels)
    ph = (C.c_void_p * n)(*[pl._h for pl in plans])
    pp = (C.c_void_p * n)(*[C.c_void_p(t.data_ptr()) for t in psis])
    res = (Result * n)()
    code = lib.pcg_ground_state_mg(n, ph, C.byref(params), C.byref(opts), pp, res, _stream(stream))
    if code not in (ATKM_OK, ATKM_NOT_CONVERGED, ATKM_STAGNATED, ATKM_ERR_NAN, ATKM_ERR_TIMEOUT):
        raise AtkmError(code, lib.atkm_last_error_string(None).decode())
    outs = []
    for i in range(n):
        d = {k: getattr(res[i], k) for k, _ in Result._fields_ if k != "log"}
        d["status_name"] = STATUS_NAMES.get(res[i].status, str(res[i].status))
        outs.append(d)
    return outs


def inner_products_noalloc(us, vs, hvol: float, out: torch.Tensor, stream=None) -> torch.Tensor:
    """<u_i, v_i> = hvol Re(sum u_i conj v_i) into the device tensor `out`
    through the allocation-free entry point (see include/atkm.h)."""
    lib = load_library()
    n = len(us)
    if len(vs) != n:
        raise ValueError("us and vs differ in length")
    ua = (C.c_void_p * max(n, 1))(*[C.c_void_p(t.data_ptr()) for t in us])
    va = (C.c_void_p * max(n, 1))(*[C.c_void_p(t.data_ptr()) for t in vs])
    numel = us[0].numel() if n else 0
    for t in list(us) + list(vs):
        if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous() and t.numel() == numel):
            raise ValueError("vectors must be contiguous complex128 CUDA tensors of equal size")
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= n):
        raise ValueError("out must be a float64 CUDA tensor with npairs elements")
    code = lib.atkm_inner_products_noalloc(ua, va, n, numel, float(hvol), C.c_void_p(out.data_ptr()),
                                           _stream(stream))
    if code != ATKM_OK:
        raise AtkmError(code, lib.atkm_last_error_string(None).decode())
    return out


def spectral_upsample(coarse: "Plan", fine: "Plan", psi_c: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """Fourier interpolant of psi_c on the fine plan's grid (same box)."""
    lib = load_library()
    out = torch.empty(fine.shape, dtype=torch.complex128, device="cuda") if out is None else out
    code = lib.atkm_spectral_upsample(coarse._h, fine._h, _ptr(psi_c, torch.complex128, coarse.shape, "psi_c"),
                                      _ptr(out, torch.complex128, fine.shape, "psi_f"), _stream(stream))
    if code != ATKM_OK:
        raise AtkmError(code, lib.atkm_last_error_string(None).decode())
    return out


GUESS_SHAPE = (16, 64, 64)


class GuessNet:
    """Handle of the learned initial-guess network (see include/atkm.h)."""

    def __init__(self, seed: int = 0, stream=None):
        self._lib = load_library()
        self._h = C.c_void_p()
        code = self._lib.atkm_guess_net_create(C.byref(self._h), int(seed), _stream(stream))
        if code != ATKM_OK:
            raise AtkmError(code, self._lib.atkm_last_error_string(None).decode())
        self.num_params = int(self._lib.atkm_guess_net_num_params())

    def __del__(self):
        try:
            if self._h and self._h.value:
                self._lib.atkm_guess_net_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def _check(self, code):
        if code != ATKM_OK:
            raise AtkmError(code, self._lib.atkm_last_error_string(None).decode())

    def set_gemm_engine(self, engine: int):
        """ATKM_GEMM_TCGEN05 (default) or ATKM_GEMM_MMA_SYNC for the dense GEMMs."""
        self._check(self._lib.atkm_guess_net_set_gemm_engine(self._h, int(engine)))

    def check(self, stream=None):
        """Raises ATKM_ERR_TIMEOUT if a tensor-core GEMM gave up waiting (synchronises the stream)."""
        self._check(self._lib.atkm_guess_net_check(self._h, _stream(stream)))

    def get_params(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        self._check(self._lib.atkm_guess_net_get_params(self._h, C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def set_params(self, w: torch.Tensor, stream=None):
        _ptr(w, torch.float32, (self.num_params,), "params")
        self._check(self._lib.atkm_guess_net_set_params(self._h, C.c_void_p(w.data_ptr()), _stream(stream)))

    def forward(self, feats: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        B = feats.shape[0]
        _ptr(feats, torch.float32, (B, 8), "feats")
        out = torch.empty((B,) + GUESS_SHAPE, dtype=torch.complex128, device="cuda") if out is None else out
        _ptr(out, torch.complex128, (B,) + GUESS_SHAPE, "psi")
        self._check(self._lib.atkm_guess_net_forward(self._h, B, C.c_void_p(feats.data_ptr()),
                                                     C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def grad(self, feats: torch.Tensor, targets: torch.Tensor, stream=None):
        B = feats.shape[0]
        _ptr(feats, torch.float32, (B, 8), "feats")
        _ptr(targets, torch.complex128, (B,) + GUESS_SHAPE, "targets")
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self._lib.atkm_guess_net_grad(self._h, B, C.c_void_p(feats.data_ptr()),
                                                  C.c_void_p(targets.data_ptr()), C.c_void_p(g.data_ptr()),
                                                  C.c_void_p(loss.data_ptr()), _stream(stream)))
        return g, loss

    def train_step(self, feats: torch.Tensor, targets: torch.Tensor, lr: float, loss=None, stream=None):
        B = feats.shape[0]
        _ptr(feats, torch.float32, (B, 8), "feats")
        _ptr(targets, torch.complex128, (B,) + GUESS_SHAPE, "targets")
        loss = torch.empty(1, dtype=torch.float32, device="cuda") if loss is None else loss
        self._check(self._lib.atkm_guess_net_train_step(self._h, B, C.c_void_p(feats.data_ptr()),
                                                        C.c_void_p(targets.data_ptr()), C.c_float(lr),
                                                        C.c_void_p(loss.data_ptr()), _stream(stream)))
        return loss

    def profile_step(self, feats: torch.Tensor, targets: torch.Tensor, lr: float, stream=None) -> dict:
        """One training step with its GEMMs timed by CUDA events (see include/atkm.h)."""
        B = feats.shape[0]
        _ptr(feats, torch.float32, (B, 8), "feats")
        _ptr(targets, torch.complex128, (B,) + GUESS_SHAPE, "targets")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        g, t, n = C.c_double(0.0), C.c_double(0.0), C.c_int(0)
        each = (C.c_double * 16)()
        self._check(self._lib.atkm_guess_net_profile_step(self._h, B, C.c_void_p(feats.data_ptr()),
                                                          C.c_void_p(targets.data_ptr()), C.c_float(lr),
                                                          C.c_void_p(loss.data_ptr()), C.byref(g), C.byref(t),
                                                          C.byref(n), each, 16, _stream(stream)))
        return {"gemm_ms": g.value, "step_ms": t.value, "gemm_calls": n.value, "loss": float(loss.item()),
                "each_ms": [each[i] for i in range(min(n.value, 16))]}


def measure_fp64_fma(blocks_per_sm=8, iters=4096, repeats=5, stream=None) -> float:
    """Peak binary64 FMA rate of the current device in GFLOP/s (see include/atkm.h)."""
    lib = load_library()
    g = C.c_double(0.0)
    code = lib.atkm_measure_fp64_fma(blocks_per_sm, iters, repeats, C.byref(g), _stream(stream))
    if code != ATKM_OK:
        raise AtkmError(code, lib.atkm_last_error_string(None).decode())
    return g.value


def launch_count() -> int:
    """Kernels launched by libatkm in this process so far."""
    return int(load_library().atkm_launch_count())


def _ptr(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_params(gamma, beta, lam, Omega) -> Params:
    p = Params()
    p.gamma[:] = [float(g) for g in gamma]
    p.beta, p.lam, p.Omega = float(beta), float(lam), float(Omega)
    return p


class Plan:
    """Owning handle of an atkm_plan (grid, box, dipole axis, multiplier)."""

    def __init__(self, N, L, n, f32: bool = False, stream=None, df32: bool = False, generic_fft: bool = False,
                 autotune: bool = False):
        lib = load_library()
        self.N = tuple(int(v) for v in N)
        self.L = tuple(float(v) for v in L)
        self.n = tuple(float(v) for v in n)
        self.shape = (self.N[2], self.N[1], self.N[0])
        self._h = C.c_void_p()
        Na = (C.c_int * 3)(*self.N)
        La = (C.c_double * 3)(*self.L)
        na = (C.c_double * 3)(*self.n)
        flags = (ATKM_PLAN_F32 if f32 else 0) | (ATKM_PLAN_DF32 if df32 else 0) | \
            (ATKM_PLAN_GENERIC_FFT if generic_fft else 0) | (ATKM_PLAN_AUTOTUNE if autotune else 0)
        code = lib.atkm_plan_create(C.byref(self._h), Na, La, na, flags, _stream(stream))
        if code != ATKM_OK:
            raise AtkmError(code, lib.atkm_last_error_string(None).decode())
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.atkm_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        if code != ATKM_OK:
            raise AtkmError(code, self._lib.atkm_last_error_string(self._h).decode())

    @property
    def device_bytes(self) -> int:
        return int(self._lib.atkm_plan_device_bytes(self._h))

    # ---- FFT-tile autotuner
    def autotune(self, stream=None):
        self._check(self._lib.atkm_plan_autotune(self._h, _stream(stream)))

    def tuning(self) -> list:
        cap = 64
        arr = (TuneInfo * cap)()
        n = self._lib.atkm_plan_tuning(self._h, arr, cap)
        if n < 0:
            raise AtkmError(-n, "atkm_plan_tuning")
        return [{k: getattr(arr[i], k) for k, _ in TuneInfo._fields_ if k != "pad_"} for i in range(min(n, cap))]

    # ---- measurement support
    def set_profiling(self, on: bool):
        self._check(self._lib.atkm_plan_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self) -> list:
        cap = 64
        arr = (KernelStat * cap)()
        cnt = C.c_int(0)
        self._check(self._lib.atkm_plan_kernel_stats(self._h, arr, cap, C.byref(cnt)))
        return [dict(name=arr[i].name.decode(), launches=arr[i].launches, ms_total=arr[i].ms_total,
                     bytes_total=arr[i].bytes_total, flops_total=arr[i].flops_total)
                for i in range(min(cnt.value, cap))]

    # ---- multiplier
    def U0(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.N[2] + 1, self.N[1] + 1, self.N[0] + 1), dtype=torch.float64, device="cuda")
        self._check(self._lib.atkm_plan_copy_U0(self._h, C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def multiplier(self, stream=None) -> torch.Tensor:
        out = torch.empty((2 * self.N[2], 2 * self.N[1], 2 * self.N[0]), dtype=torch.float64, device="cuda")
        self._check(self._lib.atkm_plan_copy_multiplier(self._h, C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    # ---- dipolar potential
    def dipolar_potential(self, rho, out=None, stream=None):
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda") if out is None else out
        self._check(self._lib.dipolar_potential(self._h, _ptr(rho, torch.float64, self.shape, "rho"),
                                                _ptr(out, torch.float64, self.shape, "phi"), _stream(stream)))
        return out

    def dipolar_potential_from_psi(self, psi, out=None, stream=None, f32=False, df32=False):
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda") if out is None else out
        fn = (self._lib.dipolar_potential_from_psi_f32 if f32 else
              self._lib.dipolar_potential_from_psi_df32 if df32 else self._lib.dipolar_potential_from_psi)
        self._check(fn(self._h, _ptr(psi, torch.complex128, self.shape, "psi"),
                       _ptr(out, torch.float64, self.shape, "phi"), _stream(stream)))
        return out

    def dipolar_potential_from_pair(self, a, b, out=None, stream=None):
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda") if out is None else out
        self._check(self._lib.dipolar_potential_from_pair(
            self._h, _ptr(a, torch.complex128, self.shape, "a"), _ptr(b, torch.complex128, self.shape, "b"),
            _ptr(out, torch.float64, self.shape, "phi"), _stream(stream)))
        return out

    # ---- Hamiltonian, energy, preconditioner
    def apply_H(self, prm: Params, f, phi, Phi, out=None, stream=None):
        out = torch.empty(self.shape, dtype=torch.complex128, device="cuda") if out is None else out
        self._check(self._lib.apply_H(self._h, C.byref(prm), _ptr(f, torch.complex128, self.shape, "f"),
                                      _ptr(phi, torch.complex128, self.shape, "phi"),
                                      _ptr(Phi, torch.float64, self.shape, "Phi"),
                                      _ptr(out, torch.complex128, self.shape, "Hf"), _stream(stream)))
        return out

    def energy_parts(self, prm: Params, phi, Phi, stream=None) -> dict:
        e = Energy()
        self._check(self._lib.atkm_energy_parts(self._h, C.byref(prm), _ptr(phi, torch.complex128, self.shape, "phi"),
                                                _ptr(Phi, torch.float64, self.shape, "Phi"), C.byref(e),
                                                _stream(stream)))
        return {k: getattr(e, k) for k, _ in Energy._fields_}

    def apply_preconditioner(self, prm: Params, alpha: float, r, phi, Phi, out=None, stream=None):
        out = torch.empty(self.shape, dtype=torch.complex128, device="cuda") if out is None else out
        self._check(self._lib.apply_preconditioner(
            self._h, C.byref(prm), C.c_double(alpha), _ptr(r, torch.complex128, self.shape, "r"),
            _ptr(phi, torch.complex128, self.shape, "phi"), _ptr(Phi, torch.float64, self.shape, "Phi"),
            _ptr(out, torch.complex128, self.shape, "Pr"), _stream(stream)))
        return out

    # ---- Algorithm 1
    def pcg_ground_state(self, prm: Params, psi, tol_residual=1e-8, tol_linf=0.0, max_iter=10000,
                         max_halvings=20, precision=PRECISION_F64, switch_tol=1e-5, log_capacity=0,
                         stream=None, check=True, resume=False, graphs=True, time_limit_s=0.0,
                         f32_window=0, f32_gain=0.0) -> dict:
        opts = PcgOpts(tol_residual, tol_linf, max_iter, max_halvings, precision, switch_tol, log_capacity,
                       1 if resume else 0, 0 if graphs else 1, time_limit_s, f32_window, f32_gain, 0)
        res = Result()
        logs = (IterLog * max(1, log_capacity))()
        res.log = C.cast(logs, C.POINTER(IterLog)) if log_capacity > 0 else C.POINTER(IterLog)()
        code = self._lib.pcg_ground_state(self._h, C.byref(prm), C.byref(opts),
                                          _ptr(psi, torch.complex128, self.shape, "psi"), C.byref(res),
                                          _stream(stream))
        if check and code not in (ATKM_OK, ATKM_NOT_CONVERGED, ATKM_STAGNATED, ATKM_ERR_TIMEOUT):
            self._check(code)
        out = {k: getattr(res, k) for k, _ in Result._fields_ if k != "log"}
        out["status_name"] = STATUS_NAMES.get(res.status, str(res.status))
        out["log"] = [{k: getattr(logs[i], k) for k, _ in IterLog._fields_ if k != "pad_"}
                      for i in range(res.log_count)]
        return out
