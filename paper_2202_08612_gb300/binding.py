"""Thin ctypes binding of the MLCC3 C ABI (include/mlcc3.h).

Argument marshalling only: every array is passed as a raw pointer (a torch
CUDA tensor's device pointer, or a contiguous float64 numpy array's host
pointer) and all arithmetic happens in the CUDA library.  Loading fails
loudly when libmlcc3.so is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlcc3.so")

MLCC3_FP64 = 0
MLCC3_SPLIT_BF16X3 = 1

ERRORS = {-1: "MLCC3_ERR_ARG", -2: "MLCC3_ERR_CUDA", -3: "MLCC3_ERR_OOM",
          -4: "MLCC3_ERR_SINGULAR_DENOM", -5: "MLCC3_ERR_TIMEOUT", -6: "MLCC3_ERR_STATE"}

# Every symbol include/mlcc3.h declares.
EXPORTS = ("mlcc3_create", "mlcc3_destroy", "mlcc3_last_error", "mlcc3_build_integrals",
           "mlcc3_triples_omega", "mlcc3_jacobian_right", "mlcc3_jacobian_left",
           "mlcc3_transition_density", "mlcc3_oscillator_strength", "mlcc3_debug_fetch",
           "mlcc3_debug_nbatches", "mlcc3_debug_profile", "mlcc3_debug_kernel_stats",
           "mlcc3_triples_omega_static", "mlcc3_debug_tc_gemm", "mlcc3_set_param",
           "mlcc3_sweep_create", "mlcc3_sweep_set_system", "mlcc3_sweep_run", "mlcc3_sweep_info",
           "mlcc3_sweep_destroy", "mlcc3_rayleigh_quotient", "mlcc3_ground_density",
           "mlcc3_multiplier_transformation", "mlcc3_cnto_matrices", "mlcc3_shard_batches",
           "mlcc3_transition_densities", "mlcc3_fp64emu_gemm")


class MLCC3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Dims(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int64), ("n_vir", ctypes.c_int64),
                ("n_act_occ", ctypes.c_int64), ("n_act_vir", ctypes.c_int64),
                ("n_chol", ctypes.c_int64), ("core_mask", ctypes.POINTER(ctypes.c_uint8))]


_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2202_08612_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    lib.mlcc3_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_Dims), I, P]
    lib.mlcc3_destroy.argtypes = [P]
    lib.mlcc3_destroy.restype = None
    lib.mlcc3_last_error.restype = ctypes.c_char_p
    lib.mlcc3_build_integrals.argtypes = [P] * 6
    lib.mlcc3_triples_omega.argtypes = [P, P, P]
    lib.mlcc3_triples_omega_static.argtypes = [P, P, P]
    lib.mlcc3_jacobian_right.argtypes = [P, I, P, P, P, P, P]
    lib.mlcc3_jacobian_left.argtypes = [P, I, P, P, P, P, P]
    lib.mlcc3_transition_density.argtypes = [P, D] + [P] * 10
    lib.mlcc3_oscillator_strength.argtypes = [P, D, P, P, P, P]
    lib.mlcc3_debug_fetch.argtypes = [P, ctypes.c_char_p, P, ctypes.c_size_t]
    lib.mlcc3_debug_nbatches.argtypes = [P]
    lib.mlcc3_debug_nbatches.restype = ctypes.c_longlong
    lib.mlcc3_debug_profile.argtypes = [P, I]
    lib.mlcc3_debug_tc_gemm.argtypes = [P, P, P, I, I, I]
    lib.mlcc3_set_param.argtypes = [P, ctypes.c_char_p, ctypes.c_longlong]
    lib.mlcc3_sweep_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), I, I, P]
    lib.mlcc3_sweep_set_system.argtypes = [P, I, I, P, P, P, P]
    lib.mlcc3_sweep_run.argtypes = [P, P]
    lib.mlcc3_sweep_info.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    lib.mlcc3_sweep_destroy.argtypes = [P]
    lib.mlcc3_sweep_destroy.restype = None
    lib.mlcc3_rayleigh_quotient.argtypes = [P, D, P, P, P, P, D, P]
    lib.mlcc3_ground_density.argtypes = [P, P, P, P]
    lib.mlcc3_multiplier_transformation.argtypes = [P, P, P, P, P]
    lib.mlcc3_cnto_matrices.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]
    L = ctypes.c_longlong
    lib.mlcc3_fp64emu_gemm.argtypes = [P, L, P, L, P, L, I, I, I, I, P]
    lib.mlcc3_shard_batches.argtypes = [I, P, I, I, I, P, I]
    lib.mlcc3_transition_densities.argtypes = [P, I, P] + [P] * 10
    lib.mlcc3_debug_kernel_stats.argtypes = [P, I, ctypes.c_char_p, ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(D), ctypes.POINTER(D)]
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype
    _lib = lib
    return lib


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or a numpy float64 array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("numpy arrays must be contiguous float64")
        return x.ctypes.data
    # torch.Tensor
    if not x.is_contiguous() or str(x.dtype) != "torch.float64":
        raise ValueError("tensors must be contiguous float64")
    return x.data_ptr()


def cnto_matrices(R1, R2, M, N, stream=None):
    """mlcc3_cnto_matrices: M [N_O][N_O], N [N_V][N_V] of one state (device arrays)."""
    lib = load()
    NV, NO = R1.shape
    rc = lib.mlcc3_cnto_matrices(NO, NV, _ptr(R1), _ptr(R2), _ptr(M), _ptr(N), stream)
    if rc != 0:
        raise MLCC3Error(rc, lib.mlcc3_last_error().decode())


def shard_batches(n_act_occ, core_mask, cvs, shard_count, shard_index):
    """mlcc3_shard_batches: the unique batches (i, j, k) that shard
    `shard_index` of `shard_count` processes (host only, no GPU needed)."""
    lib = load()
    mask = None
    if core_mask is not None:
        mask = np.ascontiguousarray(core_mask, dtype=np.uint8)
    cap = n_act_occ ** 3 + 1
    buf = np.zeros(3 * cap, dtype=np.int32)
    n = lib.mlcc3_shard_batches(int(n_act_occ), None if mask is None else mask.ctypes.data,
                                int(bool(cvs)), int(shard_count), int(shard_index),
                                buf.ctypes.data, cap)
    if n < 0:
        raise MLCC3Error(n, lib.mlcc3_last_error().decode())
    return [tuple(int(v) for v in buf[3 * u:3 * u + 3]) for u in range(n)]


def tc_gemm(A, B, C):
    """C = A B^T (torch CUDA float64 tensors) on the split-precision tensor-core kernel."""
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    rc = lib.mlcc3_debug_tc_gemm(_ptr(A), _ptr(B), _ptr(C), M, N, K)
    if rc != 0:
        raise MLCC3Error(rc, lib.mlcc3_last_error().decode())


def fp64emu_gemm(A, B, C, slices=5, stream=None):
    """mlcc3_fp64emu_gemm: C = A B^T (torch CUDA float64 tensors, row-major,
    unit column stride) to FP64 accuracy on the BF16 tensor cores."""
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    # contiguous rows (_ptr checks): the leading dimensions are the row lengths
    rc = lib.mlcc3_fp64emu_gemm(_ptr(A), K, _ptr(B), K, _ptr(C), N, M, N, K, int(slices), stream)
    if rc != 0:
        raise MLCC3Error(rc, lib.mlcc3_last_error().decode())


class Context:
    """One library context (mlcc3_create .. mlcc3_destroy)."""

    def __init__(self, n_occ, n_vir, n_act_occ, n_act_vir, n_chol, precision=MLCC3_FP64,
                 core_mask=None, stream=None):
        self.lib = load()
        self._core = None
        if core_mask is not None:
            self._core = np.ascontiguousarray(core_mask, dtype=np.uint8)
        dims = _Dims(n_occ, n_vir, n_act_occ, n_act_vir, n_chol,
                     self._core.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                     if self._core is not None else None)
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream)
        self._check(self.lib.mlcc3_create(ctypes.byref(h), ctypes.byref(dims), precision, s))
        self.h = h
        self.dims = (n_occ, n_vir, n_act_occ, n_act_vir, n_chol)

    def _check(self, rc):
        if rc != 0:
            raise MLCC3Error(rc, self.lib.mlcc3_last_error().decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlcc3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_integrals(self, chol, t1, eps, t2c, t2x):
        self._check(self.lib.mlcc3_build_integrals(self.h, _ptr(chol), _ptr(t1), _ptr(eps),
                                                   _ptr(t2c), _ptr(t2x)))

    def triples_omega(self, omega1, omega2):
        self._check(self.lib.mlcc3_triples_omega(self.h, _ptr(omega1), _ptr(omega2)))

    def triples_omega_static(self, omega1, omega2):
        """mlcc3_triples_omega without allocating: scratch in a fixed device array."""
        self._check(self.lib.mlcc3_triples_omega_static(self.h, _ptr(omega1), _ptr(omega2)))

    def jacobian_right(self, omega, R1, R2, rho1, rho2):
        w = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        self._check(self.lib.mlcc3_jacobian_right(self.h, len(w), w.ctypes.data, _ptr(R1),
                                                  _ptr(R2), _ptr(rho1), _ptr(rho2)))

    def jacobian_left(self, omega, L1, L2, sigma1, sigma2):
        w = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        self._check(self.lib.mlcc3_jacobian_left(self.h, len(w), w.ctypes.data, _ptr(L1),
                                                 _ptr(L2), _ptr(sigma1), _ptr(sigma2)))

    def transition_density(self, omega, lam1, lam2, R1, R2, L1, L2, D00_in, D00_T, Dm0_T, D0m_T):
        self._check(self.lib.mlcc3_transition_density(
            self.h, float(omega), _ptr(lam1), _ptr(lam2), _ptr(R1), _ptr(R2), _ptr(L1), _ptr(L2),
            _ptr(D00_in), _ptr(D00_T), _ptr(Dm0_T), _ptr(D0m_T)))

    def transition_densities(self, omega, lam1, lam2, R1, R2, L1, L2, D00_in, D00_T, Dm0_T, D0m_T):
        """mlcc3_transition_densities: several states in one call (shared tau,
        lambda3 and D^{0-0}); R1, R2, L1, L2, Dm0_T, D0m_T hold len(omega) states."""
        w = np.ascontiguousarray(omega, dtype=np.float64)
        self._check(self.lib.mlcc3_transition_densities(
            self.h, len(w), w.ctypes.data, _ptr(lam1), _ptr(lam2), _ptr(R1), _ptr(R2), _ptr(L1),
            _ptr(L2), _ptr(D00_in), _ptr(D00_T), _ptr(Dm0_T), _ptr(D0m_T)))

    def ground_density(self, lam1, lam2, D00_T):
        """Triples part of D^{0-0} alone (mlcc3_ground_density)."""
        self._check(self.lib.mlcc3_ground_density(self.h, _ptr(lam1), _ptr(lam2), _ptr(D00_T)))

    def multiplier_transformation(self, lam1, lam2, eta1, eta2):
        """Triples part of lambda^T A at omega = 0 (mlcc3_multiplier_transformation)."""
        self._check(self.lib.mlcc3_multiplier_transformation(self.h, _ptr(lam1), _ptr(lam2),
                                                             _ptr(eta1), _ptr(eta2)))

    def oscillator_strength(self, omega, D0m, Dm0, mu) -> float:
        f = ctypes.c_double()
        self._check(self.lib.mlcc3_oscillator_strength(self.h, float(omega), _ptr(D0m), _ptr(Dm0),
                                                       _ptr(mu), ctypes.byref(f)))
        return f.value

    def debug_fetch(self, name: str, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float64)
        self._check(self.lib.mlcc3_debug_fetch(self.h, name.encode(), out.ctypes.data, n))
        return out

    def rayleigh_quotient(self, omega, R1, R2, L1, L2, sd_part=0.0) -> float:
        """(sd_part + <L, rho_T(omega)>) / <L, R> (mlcc3_rayleigh_quotient)."""
        out = ctypes.c_double()
        self._check(self.lib.mlcc3_rayleigh_quotient(self.h, float(omega), _ptr(R1), _ptr(R2),
                                                     _ptr(L1), _ptr(L2), float(sd_part),
                                                     ctypes.byref(out)))
        return out.value

    def set_param(self, name: str, value: int):
        """mlcc3_set_param (tuning knobs such as "tc_kcap")."""
        self._check(self.lib.mlcc3_set_param(self.h, name.encode(), int(value)))

    def profile(self, enable: bool):
        """Clear the launch counters; with enable, time every launch with CUDA events."""
        self._check(self.lib.mlcc3_debug_profile(self.h, 1 if enable else 0))

    def kernel_stats(self) -> dict:
        """{kernel name: (launches, summed ms, flops)} since the last profile() call."""
        out, i = {}, 0
        name = ctypes.create_string_buffer(128)
        n, ms, fl = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        while self.lib.mlcc3_debug_kernel_stats(self.h, i, name, 128, ctypes.byref(n),
                                                 ctypes.byref(ms), ctypes.byref(fl)) == 0:
            out[name.value.decode()] = (n.value, ms.value, fl.value)
            i += 1
        return out

    def nbatches(self) -> int:
        return int(self.lib.mlcc3_debug_nbatches(self.h))


class Sweep:
    """mlcc3_sweep_*: right Jacobian transformations of several systems in one
    captured CUDA graph (see the header).  Vectors must be device tensors; the
    sweep keeps references to them because the graph reads their addresses."""

    def __init__(self, contexts, tune=True, stream=None):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h for c in self.contexts])
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream)
        self._check(self.lib.mlcc3_sweep_create(ctypes.byref(h), arr, len(self.contexts),
                                                1 if tune else 0, s))
        self.h = h
        self._keep = {}

    def _check(self, rc):
        if rc != 0:
            raise MLCC3Error(rc, self.lib.mlcc3_last_error().decode())

    def set_system(self, q, R1, R2, rho1, rho2):
        n_vec = int(R1.shape[0])
        self._keep[q] = (R1, R2, rho1, rho2)
        self._check(self.lib.mlcc3_sweep_set_system(self.h, q, n_vec, _ptr(R1), _ptr(R2),
                                                    _ptr(rho1), _ptr(rho2)))

    def run(self, omega):
        w = np.ascontiguousarray(omega, dtype=np.float64)
        self._check(self.lib.mlcc3_sweep_run(self.h, w.ctypes.data))

    def info(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.lib.mlcc3_sweep_info(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlcc3_sweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
