"""The C++17 CPU oracle (oracle/cpp/atkm_oracle.cpp): TEST INFRASTRUCTURE ONLY.

A plain, slow binary64 restatement of PCG-ATKM with its own mixed-radix FFT
and its own Faddeeva function, compiled with g++ (OpenMP over independent FFT
lines and grid planes; every sum in a fixed order, so the result does not
depend on the thread count).  This module builds it in-tree and exposes it
with numpy arrays; it imports nothing from the product package.  Only
``tests/``, ``__graft_entry__`` and the CPU legs of ``bench.py`` use it.
"""
from __future__ import annotations

import ctypes as C
import fcntl
import os
import shutil
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "atkm_oracle.cpp")
LIB = os.path.join(HERE, "cpp", "libatkm_oracle.so")
# -ffp-contract=off: no fused multiply-adds, so x86 and Arm builds round alike
FLAGS = ["-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared"]

OK, NOT_CONVERGED, STAGNATED, ERR_NAN = 0, 5, 6, 7


def build(force: bool = False) -> str:
    """Compiles libatkm_oracle.so next to its source (a few seconds)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    with open(LIB + ".lock", "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
            return LIB
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([cxx, *FLAGS, "-o", tmp, SRC], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"building the C++ oracle failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


class LogEntry(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("n", "halvings", "reset", "accepted", "has_step", "pad_")] + \
               [(k, C.c_double) for k in ("E", "mu", "residual", "linf_step", "alpha", "beta_cg", "d1", "curv", "t0",
                                          "t", "wall")]


class Result(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("E", "mu", "E_kin", "E_pot", "E_int", "E_dip", "E_rot", "virial",
                                          "residual", "linf_step")] + \
               [(k, C.c_int) for k in ("iters", "halvings", "status", "log_count")]


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        sig = {
            "ora_max_threads": (ip, []),
            "ora_dft1": (ip, [dp, ip, ip]),
            "ora_fft3": (ip, [dp, ip, ip, ip, ip, ip]),
            "ora_faddeeva": (ip, [dp, dp, C.c_long]),
            "ora_plan_create": (vp, [C.POINTER(C.c_int), dp, dp, ip]),
            "ora_plan_destroy": (None, [vp]),
            "ora_plan_set_threads": (None, [vp, ip]),
            "ora_plan_U0": (None, [vp, dp]),
            "ora_plan_K": (None, [vp, dp]),
            "ora_dipolar_potential": (None, [vp, dp, dp]),
            "ora_apply_H": (None, [vp, dp, dp, dp, dp, dp]),
            "ora_energy_parts": (None, [vp, dp, dp, dp, dp]),
            "ora_inner": (C.c_double, [vp, dp, dp]),
            "ora_precond_shift": (C.c_double, [vp, dp, dp, dp]),
            "ora_apply_precond": (None, [vp, dp, dp, dp, dp, C.c_double, dp]),
            "ora_pcg": (ip, [vp, dp, dp, dp, dp, C.POINTER(Result), C.POINTER(LogEntry), ip]),
            "ora_spectral_upsample": (ip, [C.POINTER(C.c_int), dp, C.POINTER(C.c_int), dp, ip]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def max_threads() -> int:
    return int(load().ora_max_threads())


def dft1(x, sign=-1) -> np.ndarray:
    """Unscaled DFT of a complex vector, sum_j x_j e^{sign 2 pi i jk/n}."""
    a = np.array(x, dtype=np.complex128, copy=True)
    if load().ora_dft1(_d(a), a.size, sign) != OK:
        raise ValueError("bad length")
    return a


def fft3(a, sign=-1, threads=1) -> np.ndarray:
    """3D DFT of a (N_z, N_y, N_x) complex array; sign -1 scaled by 1/N."""
    b = np.array(a, dtype=np.complex128, copy=True, order="C")
    nz, ny, nx = b.shape
    load().ora_fft3(_d(b), nx, ny, nz, sign, threads)
    return b


def faddeeva(z) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).ravel())
    out = np.empty_like(z)
    load().ora_faddeeva(_d(z), _d(out), z.size)
    return out


def spectral_upsample(psi_c, Nf, threads=1) -> np.ndarray:
    """Fourier interpolant of a coarse grid function on a finer grid (same box)."""
    c = np.ascontiguousarray(psi_c, dtype=np.complex128)
    Nc = (C.c_int * 3)(c.shape[2], c.shape[1], c.shape[0])
    out = np.empty((Nf[2], Nf[1], Nf[0]), dtype=np.complex128)
    if load().ora_spectral_upsample(Nc, _d(c), (C.c_int * 3)(*Nf), _d(out), threads) != OK:
        raise ValueError("the fine grid must not be coarser")
    return out


@dataclass
class PcgOptions:
    tol_residual: float = 1e-8
    tol_linf: float = 0.0
    max_iter: int = 10000
    max_halvings: int = 20
    energy_tol_ulps: float = 32.0


@dataclass
class PcgResult:
    phi: np.ndarray
    Phi: np.ndarray
    status: int
    iters: int
    residual: float
    mu: float
    parts: dict
    halvings: int
    linf_step: float
    log: list = field(default_factory=list)


class Plan:
    """Grid, box and dipole axis with U0 and K precomputed (Algorithm 1,
    first step; §2.2: once per domain and mesh)."""

    def __init__(self, N, L, n, threads: int = 1):
        self.N = tuple(int(v) for v in N)
        self.L = tuple(float(v) for v in L)
        self.n = tuple(float(v) for v in n)
        self.shape = (self.N[2], self.N[1], self.N[0])
        self.hvol = float(np.prod([2 * self.L[i] / self.N[i] for i in range(3)]))
        self.threads = max(1, int(threads))
        lib = load()
        h = lib.ora_plan_create((C.c_int * 3)(*self.N), (C.c_double * 3)(*self.L), (C.c_double * 3)(*self.n),
                                self.threads)
        if not h:
            raise ValueError("bad plan arguments (odd or too small grid, non-positive box, |n| != 1)")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ora_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_threads(self, threads: int):
        self.threads = max(1, int(threads))
        self._lib.ora_plan_set_threads(self._h, self.threads)

    def _c(self, a):
        return np.ascontiguousarray(a, dtype=np.complex128).reshape(self.shape)

    def _r(self, a):
        return np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)

    @staticmethod
    def _prm(prm):
        return np.array([prm.gamma[0], prm.gamma[1], prm.gamma[2], prm.beta, prm.lam, prm.Omega], dtype=np.float64)

    def U0(self) -> np.ndarray:
        out = np.empty((self.N[2] + 1, self.N[1] + 1, self.N[0] + 1))
        self._lib.ora_plan_U0(self._h, _d(out))
        return out

    def K(self) -> np.ndarray:
        out = np.empty((2 * self.N[2], 2 * self.N[1], 2 * self.N[0]))
        self._lib.ora_plan_K(self._h, _d(out))
        return out

    def dipolar_potential(self, rho) -> np.ndarray:
        r = self._r(rho)
        out = np.empty(self.shape)
        self._lib.ora_dipolar_potential(self._h, _d(r), _d(out))
        return out

    def apply_H(self, prm, f, phi, Phi) -> np.ndarray:
        p = self._prm(prm)
        f, phi, Phi = self._c(f), self._c(phi), self._r(Phi)
        out = np.empty(self.shape, dtype=np.complex128)
        self._lib.ora_apply_H(self._h, _d(p), _d(f), _d(phi), _d(Phi), _d(out))
        return out

    def energy_parts(self, prm, phi, Phi) -> dict:
        p = self._prm(prm)
        phi, Phi = self._c(phi), self._r(Phi)
        out = np.empty(8)
        self._lib.ora_energy_parts(self._h, _d(p), _d(phi), _d(Phi), _d(out))
        return dict(zip(("E_kin", "E_pot", "E_int", "E_dip", "E_rot", "E", "virial", "mu"), out.tolist()))

    def inner(self, u, v) -> float:
        return float(self._lib.ora_inner(self._h, _d(self._c(u)), _d(self._c(v))))

    def precond_shift(self, prm, phi, Phi) -> float:
        return float(self._lib.ora_precond_shift(self._h, _d(self._prm(prm)), _d(self._c(phi)), _d(self._r(Phi))))

    def apply_precond(self, prm, r, phi, Phi, alpha) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        self._lib.ora_apply_precond(self._h, _d(self._prm(prm)), _d(self._c(r)), _d(self._c(phi)),
                                    _d(self._r(Phi)), float(alpha), _d(out))
        return out

    def pcg_ground_state(self, prm, phi0, opts: PcgOptions = PcgOptions(), log_capacity=None) -> PcgResult:
        """Algorithm 1 (PCG-ATKM) with the step control of §2.3 (i)-(iii)."""
        cap = opts.max_iter + 2 if log_capacity is None else log_capacity
        psi = self._c(phi0).copy()
        Phi = np.empty(self.shape)
        o = np.array([opts.tol_residual, opts.tol_linf, opts.max_iter, opts.max_halvings, opts.energy_tol_ulps],
                     dtype=np.float64)
        res = Result()
        logs = (LogEntry * max(1, cap))()
        self._lib.ora_pcg(self._h, _d(self._prm(prm)), _d(o), _d(psi), _d(Phi), C.byref(res), logs, cap)
        log = []
        for i in range(res.log_count):
            e = logs[i]
            d = dict(n=e.n, E=e.E, mu=e.mu, residual=e.residual, linf_step=e.linf_step, wall=e.wall)
            if e.has_step:
                d.update(alpha=e.alpha, beta_cg=e.beta_cg, reset=bool(e.reset), d1=e.d1, curv=e.curv, t0=e.t0,
                         t=e.t, halvings=e.halvings, accepted=bool(e.accepted))
            log.append(d)
        parts = dict(E_kin=res.E_kin, E_pot=res.E_pot, E_int=res.E_int, E_dip=res.E_dip, E_rot=res.E_rot, E=res.E,
                     virial=res.virial)
        return PcgResult(phi=psi, Phi=Phi, status=res.status, iters=res.iters, residual=res.residual, mu=res.mu,
                         parts=parts, halvings=res.halvings, linf_step=res.linf_step, log=log)
