"""Python binding of libnolsm.so (ctypes): the C ABI of include/nolsm.h, argument marshalling only.

Every step of the NOLSM path runs in the library's CUDA kernels.  When the library is missing
the import of this module raises: there is no CPU fallback.  Device buffers are torch CUDA
tensors (or raw pointers); the context works on the caller's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnolsm.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTPD, ENOCONV, EBRACKET, ETIMEOUT, ENOTBUILT, ENONFINITE = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTPD", "ENOCONV", "EBRACKET", "ETIMEOUT", "ENOTBUILT",
                "ENONFINITE"]
MEM_DEVICE, MEM_HOST = 0, 1
PREC_FP32, PREC_MIXED_FP16, PREC_MIXED_BF16 = 1, 2, 3
BOUNDS_GERSHGORIN, BOUNDS_LANCZOS, BOUNDS_LEARNED = 0, 1, 2
CHOL_FP64, CHOL_FP32, CHOL_FP64_INV64 = 0, 1, 2

FUNCTIONS = ["nolsm_default_options", "nolsm_create", "nolsm_build_submatrices", "nolsm_sign_batch", "nolsm_set_mu",
             "nolsm_density", "nolsm_band_energy", "nolsm_block_info", "nolsm_block_index_set", "nolsm_block_bounds",
             "nolsm_block_state", "nolsm_block_matrix", "nolsm_counters", "nolsm_band_energy_noalloc",
             "nolsm_last_error", "nolsm_destroy"]


class NolsmCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("memory", C.c_int32)]


class NolsmOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("bounds", C.c_int32), ("chol_precision", C.c_int32),
                ("scaled", C.c_int32), ("sign_tol", C.c_double), ("max_iter", C.c_int32),
                ("refine_iters", C.c_int32), ("spin_factor", C.c_double), ("lower_bound", C.c_double),
                ("alpha_margin", C.c_double), ("wait_budget", C.c_int64), ("mlp_path", C.c_char_p)]


class NolsmSignStats(C.Structure):
    _fields_ = [("mu", C.c_double), ("n_electrons", C.c_double), ("band_energy", C.c_double),
                ("max_residual", C.c_double), ("iters_avg", C.c_double), ("iters_min", C.c_int32),
                ("iters_max", C.c_int32), ("n_blocks", C.c_int32), ("n_restarted", C.c_int32),
                ("flops_paper", C.c_double), ("flops_executed", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NolsmError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libnolsm.so is not built ({path}); run python -m paper_2205_12182_gb300.build")
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
    pi32, pf64 = C.POINTER(C.c_int32), C.POINTER(C.c_double)
    sig = {
        "nolsm_default_options": (i32, [C.POINTER(NolsmOptions)]),
        "nolsm_create": (i32, [C.POINTER(P), C.POINTER(NolsmOptions), P]),
        "nolsm_build_submatrices": (i32, [P, C.POINTER(NolsmCsr), C.POINTER(NolsmCsr), i32, P, P, P, P]),
        "nolsm_sign_batch": (i32, [P, f64, C.POINTER(NolsmSignStats)]),
        "nolsm_set_mu": (i32, [P, f64, f64, f64, f64, i32, pf64, pf64, pi32]),
        "nolsm_density": (i32, [P, P, i32]),
        "nolsm_band_energy": (i32, [P, pf64]),
        "nolsm_block_info": (i32, [P, i32, pi32, pi32]),
        "nolsm_block_index_set": (i32, [P, i32, P]),
        "nolsm_block_bounds": (i32, [P, P, P]),
        "nolsm_block_state": (i32, [P, P, P, P]),
        "nolsm_block_matrix": (i32, [P, i32, i32, P]),
        "nolsm_counters": (i32, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), pf64, pf64, i32]),
        "nolsm_band_energy_noalloc": (i32, [i64, P, P, f64, P, P]),
        "nolsm_last_error": (C.c_char_p, [P]),
        "nolsm_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


def _ptr(x) -> int:
    """Raw address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _check(ctx, status):
    if status != OK:
        msg = _lib.nolsm_last_error(ctx).decode() if ctx else ""
        raise NolsmError(status, msg)


# ---------------------------------------------------------------- thin functions with the ABI's names

def nolsm_default_options() -> NolsmOptions:
    o = NolsmOptions()
    _check(None, _lib.nolsm_default_options(C.byref(o)))
    return o


def nolsm_create(options: NolsmOptions | None = None, stream: int | None = None):
    ctx = C.c_void_p()
    _check(None, _lib.nolsm_create(C.byref(ctx), C.byref(options) if options is not None else None, stream))
    return ctx


def nolsm_build_submatrices(ctx, H: NolsmCsr, S: NolsmCsr, n_blocks, blk_ptr, blk_cols, extra_ptr=None,
                            extra_idx=None):
    _check(ctx, _lib.nolsm_build_submatrices(ctx, C.byref(H), C.byref(S), int(n_blocks), _ptr(blk_ptr),
                                             _ptr(blk_cols), _ptr(extra_ptr), _ptr(extra_idx)))


def nolsm_sign_batch(ctx, mu: float) -> dict:
    s = NolsmSignStats()
    _check(ctx, _lib.nolsm_sign_batch(ctx, float(mu), C.byref(s)))
    return s.as_dict()


def nolsm_set_mu(ctx, n_electrons, mu_lo=0.0, mu_hi=0.0, tol_n=1e-3, max_steps=60):
    mu, n, st = C.c_double(), C.c_double(), C.c_int32()
    _check(ctx, _lib.nolsm_set_mu(ctx, float(n_electrons), float(mu_lo), float(mu_hi), float(tol_n), int(max_steps),
                                  C.byref(mu), C.byref(n), C.byref(st)))
    return mu.value, n.value, st.value


def nolsm_density(ctx, d_val=None, memory=MEM_DEVICE):
    _check(ctx, _lib.nolsm_density(ctx, _ptr(d_val), int(memory)))


def nolsm_band_energy(ctx) -> float:
    e = C.c_double()
    _check(ctx, _lib.nolsm_band_energy(ctx, C.byref(e)))
    return e.value


def nolsm_block_info(ctx, b):
    n, c = C.c_int32(), C.c_int32()
    _check(ctx, _lib.nolsm_block_info(ctx, int(b), C.byref(n), C.byref(c)))
    return n.value, c.value


def nolsm_block_index_set(ctx, b) -> np.ndarray:
    n, _ = nolsm_block_info(ctx, b)
    out = np.empty(n, np.int32)
    _check(ctx, _lib.nolsm_block_index_set(ctx, int(b), out.ctypes.data))
    return out


def nolsm_block_bounds(ctx, n_blocks):
    lo, hi = np.empty(n_blocks), np.empty(n_blocks)
    _check(ctx, _lib.nolsm_block_bounds(ctx, lo.ctypes.data, hi.ctypes.data))
    return lo, hi


def nolsm_block_state(ctx, n_blocks):
    it = np.empty(n_blocks, np.int32)
    res = np.empty(n_blocks)
    st = np.empty(n_blocks, np.int32)
    _check(ctx, _lib.nolsm_block_state(ctx, it.ctypes.data, res.ctypes.data, st.ctypes.data))
    return it, res, st


def nolsm_block_matrix(ctx, b, which=0) -> np.ndarray:
    n, _ = nolsm_block_info(ctx, b)
    out = np.empty((n, n), np.float32)
    _check(ctx, _lib.nolsm_block_matrix(ctx, int(b), int(which), out.ctypes.data))
    return out


def nolsm_counters(ctx, reset=False) -> dict:
    la, ga = C.c_int64(), C.c_int64()
    ms, fl = C.c_double(), C.c_double()
    _check(ctx, _lib.nolsm_counters(ctx, C.byref(la), C.byref(ga), C.byref(ms), C.byref(fl), int(bool(reset))))
    return {"launches": la.value, "gemm_launches": ga.value, "gemm_ms": ms.value, "gemm_flops": fl.value}


def nolsm_band_energy_noalloc(nnz, d_val, h_val, spin_factor, e_out, stream=None):
    """Band energy into the device double e_out without allocating (see include/nolsm.h)."""
    _check(None, _lib.nolsm_band_energy_noalloc(int(nnz), _ptr(d_val), _ptr(h_val), float(spin_factor),
                                                _ptr(e_out), stream))


def nolsm_last_error(ctx) -> str:
    return _lib.nolsm_last_error(ctx).decode()


def nolsm_destroy(ctx):
    _lib.nolsm_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper

def make_csr(n, nnz, row_ptr, col, val, memory) -> NolsmCsr:
    return NolsmCsr(int(n), int(nnz), _ptr(row_ptr), _ptr(col), _ptr(val), int(memory))


class Nolsm:
    """One context on the current CUDA device and stream.

    ``system`` is any object with row_ptr, col, h, s, blk_ptr, blk_cols, extra_ptr, extra_idx
    (numpy arrays).  ``memory='device'`` copies the CSR to torch CUDA tensors first (kept alive
    here); ``'host'`` hands pinned host arrays to the library, which copies them itself.
    """

    def __init__(self, precision=PREC_MIXED_FP16, stream=None, **opts):
        import torch
        o = nolsm_default_options()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.ctx = nolsm_create(o, stream)
        self._keep = []
        self._cache = {}

    def close(self):
        if self.ctx:
            nolsm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stage(self, system, memory="device"):
        """CSR arrays of `system` as torch tensors on the device or in pinned host memory (cached)."""
        import torch
        key = (id(system), memory)
        if key not in self._cache:
            arrs = [np.ascontiguousarray(system.row_ptr, np.int64), np.ascontiguousarray(system.col, np.int32),
                    np.ascontiguousarray(system.h, np.float64), np.ascontiguousarray(system.s, np.float64)]
            if memory == "device":
                ts = [torch.from_numpy(a).to(torch.device("cuda")) for a in arrs]
            else:
                ts = [torch.from_numpy(a).pin_memory() for a in arrs]
            self._cache[key] = (system, ts)
        return self._cache[key][1]

    def build(self, system, memory="device"):
        n, nnz = system.n_basis, system.nnz
        rp, cl, hv, sv = self.stage(system, memory)
        kind = MEM_DEVICE if memory == "device" else MEM_HOST
        self._keep = [rp, cl, hv, sv]
        H = make_csr(n, nnz, rp, cl, hv, kind)
        S = make_csr(n, nnz, rp, cl, sv, kind)
        bp = np.ascontiguousarray(system.blk_ptr, np.int32)
        bc = np.ascontiguousarray(system.blk_cols, np.int32)
        ep = None if system.extra_ptr is None else np.ascontiguousarray(system.extra_ptr, np.int32)
        ei = None if system.extra_idx is None else np.ascontiguousarray(system.extra_idx, np.int32)
        nolsm_build_submatrices(self.ctx, H, S, len(bp) - 1, bp, bc, ep, ei)
        self.n_blocks = len(bp) - 1
        self.nnz = nnz
        return self

    def sign_batch(self, mu):
        return nolsm_sign_batch(self.ctx, mu)

    def set_mu(self, n_electrons, mu_lo=0.0, mu_hi=0.0, tol_n=1e-3, max_steps=60):
        return nolsm_set_mu(self.ctx, n_electrons, mu_lo, mu_hi, tol_n, max_steps)

    def density(self, out=None, memory=MEM_DEVICE):
        import torch
        if out is None:
            out = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
            memory = MEM_DEVICE
        nolsm_density(self.ctx, out, memory)
        return out

    def band_energy(self):
        return nolsm_band_energy(self.ctx)

    def index_set(self, b):
        return nolsm_block_index_set(self.ctx, b)

    def bounds(self):
        return nolsm_block_bounds(self.ctx, self.n_blocks)

    def iters(self):
        return nolsm_block_state(self.ctx, self.n_blocks)[0]

    def block_state(self):
        return nolsm_block_state(self.ctx, self.n_blocks)

    def counters(self, reset=False):
        return nolsm_counters(self.ctx, reset)

    def block_matrix(self, b, which=0):
        return nolsm_block_matrix(self.ctx, b, which)
