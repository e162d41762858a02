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
BOUNDS_GERSHGORIN, BOUNDS_LANCZOS, BOUNDS_LEARNED, BOUNDS_GIVEN = 0, 1, 2, 3
CHOL_FP64, CHOL_FP32, CHOL_FP64_INV64, CHOL_DF64, CHOL_DF64_SIMT = 0, 1, 2, 3, 4
SCHEDULE_PERSISTENT, SCHEDULE_PER_PRODUCT, SCHEDULE_AUTO, SCHEDULE_PERSISTENT_INTERLEAVED = 0, 1, 2, 3
REFINE_TENSOR, REFINE_SIMT = 0, 1
MU_FIRST_AUFBAU, MU_FIRST_MIDPOINT = 0, 1
LOOP_GRAPH, LOOP_HOST = 0, 1
COMBINE_CUBIC, COMBINE_PERFORMANCE = 0, 1

FUNCTIONS = ["nolsm_default_options", "nolsm_create", "nolsm_build_submatrices", "nolsm_sign_batch", "nolsm_set_mu", "nolsm_solve_chunked",
             "nolsm_density", "nolsm_band_energy", "nolsm_block_info", "nolsm_block_index_set", "nolsm_block_bounds",
             "nolsm_block_state", "nolsm_block_traces", "nolsm_own_diagonal", "nolsm_block_matrix", "nolsm_block_factor", "nolsm_counters", "nolsm_phase_times", "nolsm_set_wait_budget",
             "nolsm_band_energy_noalloc",
             "nolsm_block_features", "nolsm_block_lanczos", "nolsm_mlp_create", "nolsm_mlp_get_params",
             "nolsm_mlp_gradient", "nolsm_mlp_adam", "nolsm_mlp_predict", "nolsm_mlp_destroy", "nolsm_set_predictor",
             "nolsm_keep_bounds", "nolsm_set_block_bounds", "nolsm_set_schedule_table", "nolsm_last_schedule", "nolsm_combine_blocks", "nolsm_last_error", "nolsm_destroy"]

PHASES = ("gather", "factor", "inverse", "congruence", "build_rest", "sign_setup", "products", "slab", "density",
          "energy", "factor_trsm", "factor_update")

N_PARAMS = 32 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3
N_FEATURES, N_OUTPUTS = 32, 3


class NolsmCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("memory", C.c_int32)]


class NolsmOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("bounds", C.c_int32), ("chol_precision", C.c_int32),
                ("scaled", C.c_int32), ("sign_tol", C.c_double), ("max_iter", C.c_int32),
                ("refine_iters", C.c_int32), ("spin_factor", C.c_double), ("lower_bound", C.c_double),
                ("alpha_margin", C.c_double), ("wait_budget", C.c_int64), ("lanczos_steps", C.c_int32),
                ("schedule", C.c_int32), ("refine_path", C.c_int32), ("fp8_iters", C.c_int32),
                ("mu_first", C.c_int32), ("loop", C.c_int32)]


class NolsmSignStats(C.Structure):
    _fields_ = [("mu", C.c_double), ("n_electrons", C.c_double), ("band_energy", C.c_double),
                ("max_residual", C.c_double), ("iters_avg", C.c_double), ("iters_min", C.c_int32),
                ("iters_max", C.c_int32), ("n_blocks", C.c_int32), ("n_restarted", C.c_int32),
                ("flops_paper", C.c_double), ("flops_executed", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NolsmChunkedStats(C.Structure):
    _fields_ = [("mu", C.c_double), ("n_electrons", C.c_double), ("band_energy", C.c_double),
                ("band_energy_traces", C.c_double), ("iters_avg", C.c_double), ("flops_paper", C.c_double),
                ("flops_executed", C.c_double), ("flops_useful", C.c_double), ("ms_total", C.c_double),
                ("ms_last_pass", C.c_double),
                ("iters_max", C.c_int32), ("passes", C.c_int32), ("chunks", C.c_int32), ("n_blocks", C.c_int32),
                ("max_chunk_blocks", C.c_int32), ("reserved", C.c_int32)]

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
        "nolsm_solve_chunked": (i32, [P, C.POINTER(NolsmCsr), C.POINTER(NolsmCsr), i32, P, P, P, P, i32, f64, f64,
                                      i32, P, P, P, C.POINTER(NolsmChunkedStats)]),
        "nolsm_density": (i32, [P, P, i32]),
        "nolsm_band_energy": (i32, [P, pf64]),
        "nolsm_block_info": (i32, [P, i32, pi32, pi32]),
        "nolsm_block_index_set": (i32, [P, i32, P]),
        "nolsm_block_bounds": (i32, [P, P, P]),
        "nolsm_block_state": (i32, [P, P, P, P]),
        "nolsm_block_traces": (i32, [P, P, P]),
        "nolsm_own_diagonal": (i32, [P, C.POINTER(C.c_int64), P]),
        "nolsm_block_matrix": (i32, [P, i32, i32, P]),
        "nolsm_block_factor": (i32, [P, i32, P]),
        "nolsm_counters": (i32, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), pf64, pf64, i32]),
        "nolsm_band_energy_noalloc": (i32, [i64, P, P, f64, P, P]),
        "nolsm_phase_times": (i32, [P, pf64, i32, i32]),
        "nolsm_set_wait_budget": (i32, [P, i64]),
        "nolsm_block_features": (i32, [P, f64, P]),
        "nolsm_block_lanczos": (i32, [P, i32, i32, P]),
        "nolsm_mlp_create": (i32, [C.POINTER(P), P, P, P]),
        "nolsm_mlp_get_params": (i32, [P, P]),
        "nolsm_mlp_gradient": (i32, [P, P, P, i32, P, P, pf64]),
        "nolsm_mlp_adam": (i32, [P, C.c_float, C.c_float, C.c_float, C.c_float]),
        "nolsm_mlp_predict": (i32, [P, P, i32, P]),
        "nolsm_mlp_destroy": (None, [P]),
        "nolsm_set_predictor": (i32, [P, P]),
        "nolsm_keep_bounds": (i32, [P, i32]),
        "nolsm_set_schedule_table": (i32, [P, i32, P, P, P]),
        "nolsm_last_schedule": (i32, [P, pi32, pi32]),
        "nolsm_set_block_bounds": (i32, [P, P, i32]),
        "nolsm_combine_blocks": (i32, [C.POINTER(NolsmCsr), i32, P, P, P, P, i32, i32, P, P, i32, pi32, P, P, P, P, P,
                                       P, P]),
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


def nolsm_solve_chunked(ctx, H: NolsmCsr, S: NolsmCsr, n_blocks, blk_ptr, blk_cols, extra_ptr, extra_idx,
                        chunk_blocks, n_electrons, tol_n, max_passes, d_val, block_n=None, block_e=None) -> dict:
    st = NolsmChunkedStats()
    _check(ctx, _lib.nolsm_solve_chunked(ctx, C.byref(H), C.byref(S), int(n_blocks), _ptr(blk_ptr), _ptr(blk_cols),
                                         _ptr(extra_ptr), _ptr(extra_idx), int(chunk_blocks), float(n_electrons),
                                         float(tol_n), int(max_passes), _ptr(d_val), _ptr(block_n), _ptr(block_e),
                                         C.byref(st)))
    return st.as_dict()


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


def nolsm_block_traces(ctx, n_blocks):
    """(electron count, band energy) terms of every block at the last sign evaluation (host)."""
    n = np.empty(n_blocks)
    e = np.empty(n_blocks)
    _check(ctx, _lib.nolsm_block_traces(ctx, n.ctypes.data, e.ctypes.data))
    return n, e


def nolsm_own_diagonal(ctx) -> np.ndarray:
    """Diagonal of A0 at every own column (host float32, block order)."""
    n = C.c_int64()
    _check(ctx, _lib.nolsm_own_diagonal(ctx, C.byref(n), None))
    out = np.empty(n.value, np.float32)
    _check(ctx, _lib.nolsm_own_diagonal(ctx, C.byref(n), out.ctypes.data))
    return out


def nolsm_block_matrix(ctx, b, which=0) -> np.ndarray:
    n, _ = nolsm_block_info(ctx, b)
    out = np.empty((n, n), np.float32)
    _check(ctx, _lib.nolsm_block_matrix(ctx, int(b), int(which), out.ctypes.data))
    return out


def nolsm_block_factor(ctx, b) -> np.ndarray:
    n, _ = nolsm_block_info(ctx, b)
    out = np.empty((n, n), np.float64)
    _check(ctx, _lib.nolsm_block_factor(ctx, int(b), out.ctypes.data))
    return out


def nolsm_set_wait_budget(ctx, budget):
    """Poll budget of every device-side wait for the calls that follow."""
    _check(ctx, _lib.nolsm_set_wait_budget(ctx, int(budget)))


def nolsm_phase_times(ctx, reset=False) -> dict:
    """Cumulative device milliseconds of every stage of the path (nolsm_phase order)."""
    ms = (C.c_double * len(PHASES))()
    _check(ctx, _lib.nolsm_phase_times(ctx, ms, len(PHASES), 1 if reset else 0))
    return dict(zip(PHASES, list(ms)))


def nolsm_counters(ctx, reset=False) -> dict:
    la, ga = C.c_int64(), C.c_int64()
    ms, fl = C.c_double(), C.c_double()
    _check(ctx, _lib.nolsm_counters(ctx, C.byref(la), C.byref(ga), C.byref(ms), C.byref(fl), int(bool(reset))))
    return {"launches": la.value, "gemm_launches": ga.value, "gemm_ms": ms.value, "gemm_flops": fl.value}


def nolsm_band_energy_noalloc(nnz, d_val, h_val, spin_factor, e_out, stream=None):
    """Band energy into the device double e_out without allocating (see include/nolsm.h)."""
    _check(None, _lib.nolsm_band_energy_noalloc(int(nnz), _ptr(d_val), _ptr(h_val), float(spin_factor),
                                                _ptr(e_out), stream))


def nolsm_block_features(ctx, mu, feat):
    _check(ctx, _lib.nolsm_block_features(ctx, float(mu), _ptr(feat)))


def nolsm_block_lanczos(ctx, steps, op, out):
    _check(ctx, _lib.nolsm_block_lanczos(ctx, int(steps), int(op), _ptr(out)))


def nolsm_mlp_create(params, norm, stream=None):
    m = C.c_void_p()
    p = None if params is None else np.ascontiguousarray(params, np.float32)
    nrm = np.ascontiguousarray(norm, np.float32)
    _check(None, _lib.nolsm_mlp_create(C.byref(m), None if p is None else p.ctypes.data, nrm.ctypes.data, stream))
    return m


def nolsm_mlp_get_params(mlp) -> np.ndarray:
    out = np.empty(N_PARAMS, np.float32)
    _check(None, _lib.nolsm_mlp_get_params(mlp, out.ctypes.data))
    return out


def nolsm_mlp_gradient(mlp, x, t, n, w, grad=None):
    ww = np.ascontiguousarray(w, np.float32)
    loss = C.c_double()
    _check(None, _lib.nolsm_mlp_gradient(mlp, _ptr(x), _ptr(t), int(n), ww.ctypes.data, _ptr(grad), C.byref(loss)))
    return loss.value


def nolsm_mlp_adam(mlp, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(None, _lib.nolsm_mlp_adam(mlp, lr, beta1, beta2, eps))


def nolsm_mlp_predict(mlp, x, n, y):
    _check(None, _lib.nolsm_mlp_predict(mlp, _ptr(x), int(n), _ptr(y)))


def nolsm_mlp_destroy(mlp):
    _lib.nolsm_mlp_destroy(mlp)


def nolsm_set_predictor(ctx, mlp):
    _check(ctx, _lib.nolsm_set_predictor(ctx, mlp))


def nolsm_combine_blocks(n, row_ptr, col, blk_ptr, blk_cols, extra_ptr=None, extra_idx=None,
                         criterion=COMBINE_CUBIC, pn_dim=None, pn_time=None, max_dim=4096) -> dict:
    """Host arrays in, host arrays out: the combined blocks (Eq. 9 / Eq. 10) and their dimensions."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    blk_ptr = np.ascontiguousarray(blk_ptr, np.int32)
    blk_cols = np.ascontiguousarray(blk_cols, np.int32)
    nb = blk_ptr.shape[0] - 1
    has_extra = extra_ptr is not None
    if has_extra:
        extra_ptr = np.ascontiguousarray(extra_ptr, np.int32)
        extra_idx = np.ascontiguousarray(extra_idx, np.int32)
    npts = 0
    if pn_dim is not None:
        pn_dim = np.ascontiguousarray(pn_dim, np.int32)
        pn_time = np.ascontiguousarray(pn_time, np.float64)
        npts = pn_dim.shape[0]
    pattern = make_csr(n, col.shape[0], row_ptr, col, None, MEM_HOST)
    n_out = C.c_int32(0)
    group = np.empty(nb, np.int32)
    o_ptr = np.empty(nb + 1, np.int32)
    o_cols = np.empty(max(blk_cols.shape[0], 1), np.int32)
    o_eptr = np.empty(nb + 1, np.int32) if has_extra else None
    o_eidx = np.empty(max(int(extra_ptr[-1]), 1), np.int32) if has_extra else None
    o_dim = np.empty(nb, np.int32)
    cost = np.zeros(2, np.float64)
    _check(None, _lib.nolsm_combine_blocks(C.byref(pattern), nb, _ptr(blk_ptr), _ptr(blk_cols), _ptr(extra_ptr),
                                           _ptr(extra_idx), int(criterion), npts, _ptr(pn_dim), _ptr(pn_time),
                                           int(max_dim), C.byref(n_out), _ptr(group), _ptr(o_ptr), _ptr(o_cols),
                                           _ptr(o_eptr), _ptr(o_eidx), _ptr(o_dim), _ptr(cost)))
    m = n_out.value
    out = {"n_blocks": m, "group": group, "blk_ptr": o_ptr[:m + 1].copy(), "blk_cols": o_cols[:o_ptr[m]].copy(),
           "dim": o_dim[:m].copy(), "cost_in": float(cost[0]), "cost_out": float(cost[1]),
           "extra_ptr": None, "extra_idx": None}
    if has_extra:
        out["extra_ptr"] = o_eptr[:m + 1].copy()
        out["extra_idx"] = o_eidx[:o_eptr[m]].copy()
    return out


PN_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "pn_gb300.json")
# the same measurement with the whole step's device time in the numerator (measure_pn --what step)
PN_STEP_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "pn_step_gb300.json")


def load_pn_table(path: str = PN_TABLE):
    """(sizes, time per flop) of the measured product throughput, for COMBINE_PERFORMANCE."""
    import json
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d["n"], np.int32), np.asarray(d["time_per_flop"], np.float64)


def combine_blocks(system, criterion=COMBINE_CUBIC, pn=None, max_dim=4096):
    """(copy of a dataclass system with the combined blocks, result of nolsm_combine_blocks)."""
    import dataclasses
    dims, times = pn if pn is not None else (None, None)
    r = nolsm_combine_blocks(len(system.row_ptr) - 1, system.row_ptr, system.col, system.blk_ptr, system.blk_cols,
                             system.extra_ptr, system.extra_idx, criterion, dims, times, max_dim)
    return dataclasses.replace(system, blk_ptr=r["blk_ptr"], blk_cols=r["blk_cols"], extra_ptr=r["extra_ptr"],
                               extra_idx=r["extra_idx"]), r


def nolsm_set_schedule_table(ctx, n_pad, schedule, ms_per_block=None):
    """Measured schedule per n_pad for SCHEDULE_AUTO (host arrays; empty removes the table); optional
    per-block times (n x 3: persistent, per-product, interleaved) for AUTO's prediction."""
    n_pad = np.ascontiguousarray(n_pad, np.int32)
    schedule = np.ascontiguousarray(schedule, np.int32)
    ms = None if ms_per_block is None else np.ascontiguousarray(ms_per_block, np.float64).reshape(-1)
    _check(ctx, _lib.nolsm_set_schedule_table(ctx, int(n_pad.shape[0]), _ptr(n_pad) if n_pad.size else None,
                                              _ptr(schedule) if schedule.size else None,
                                              _ptr(ms) if ms is not None and ms.size else None))


def nolsm_last_schedule(ctx):
    """(schedule of the last sign evaluation, or -2 for a split one; blocks of its persistent launch)."""
    sc, nq = C.c_int32(), C.c_int32()
    _check(ctx, _lib.nolsm_last_schedule(ctx, C.byref(sc), C.byref(nq)))
    return sc.value, nq.value


SCHEDULE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "schedule_gb300.json")


def load_schedule_table(path: str = SCHEDULE_TABLE):
    """(n_pad, schedule, ms per block of persistent / per-product / interleaved) of a table written by
    paper_2205_12182_gb300.autotune (the batch times divided by the batch's blocks)."""
    import json
    with open(path) as f:
        d = json.load(f)
    blocks = np.asarray(d["blocks"], np.float64)
    ms = np.stack([np.asarray(d["ms"][k], np.float64) / blocks for k in ("persistent", "per_product", "interleaved")],
                  axis=1)
    return np.asarray(d["n_pad"], np.int32), np.asarray(d["schedule"], np.int32), ms


def nolsm_keep_bounds(ctx, steps=64):
    _check(ctx, _lib.nolsm_keep_bounds(ctx, int(steps)))


def nolsm_set_block_bounds(ctx, bounds, memory=MEM_DEVICE):
    _check(ctx, _lib.nolsm_set_block_bounds(ctx, _ptr(bounds), int(memory)))


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
        if getattr(system, "on_device", False):
            if memory != "device":
                raise ValueError("a device-resident system can only be used with memory='device'")
            return [system.row_ptr, system.col, system.h, system.s]
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

    def solve_chunked(self, system, d_out, n_electrons=None, tol_n=1e-3, max_passes=60, chunk_blocks=0,
                      block_traces=False):
        """nolsm_solve_chunked on a system whose CSR is (or is copied) on the device; D into d_out
        (device float64, nnz).  Returns the statistics, plus per-block terms when block_traces."""
        rp, cl, hv, sv = self.stage(system, "device")
        self._keep = [rp, cl, hv, sv]
        H = make_csr(system.n_basis, system.nnz, rp, cl, hv, MEM_DEVICE)
        S = make_csr(system.n_basis, system.nnz, rp, cl, sv, MEM_DEVICE)
        bp = np.ascontiguousarray(system.blk_ptr, np.int32)
        bc = np.ascontiguousarray(system.blk_cols, np.int32)
        ep = None if system.extra_ptr is None else np.ascontiguousarray(system.extra_ptr, np.int32)
        ei = None if system.extra_idx is None else np.ascontiguousarray(system.extra_idx, np.int32)
        nb = len(bp) - 1
        bn = np.empty(nb) if block_traces else None
        be = np.empty(nb) if block_traces else None
        st = nolsm_solve_chunked(self.ctx, H, S, nb, bp, bc, ep, ei, chunk_blocks,
                                 system.n_electrons if n_electrons is None else n_electrons, tol_n, max_passes,
                                 d_out, bn, be)
        self.n_blocks = None      # the context now holds the last chunk's build
        if block_traces:
            st["block_n"], st["block_e"] = bn, be
        return st

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

    def block_traces(self):
        return nolsm_block_traces(self.ctx, self.n_blocks)

    def own_diagonal(self):
        return nolsm_own_diagonal(self.ctx)

    def features(self, mu):
        import torch
        f = torch.empty((self.n_blocks, N_FEATURES), dtype=torch.float32, device="cuda")
        nolsm_block_features(self.ctx, mu, f)
        return f

    def lanczos(self, steps, op=0):
        import torch
        out = torch.empty((self.n_blocks, 4), dtype=torch.float32, device="cuda")
        nolsm_block_lanczos(self.ctx, steps, op, out)
        return out

    def set_predictor(self, predictor):
        self._predictor = predictor
        nolsm_set_predictor(self.ctx, predictor.mlp if predictor is not None else None)

    def counters(self, reset=False):
        return nolsm_counters(self.ctx, reset)

    def phase_times(self, reset=False):
        return nolsm_phase_times(self.ctx, reset)

    def keep_bounds(self, steps=64):
        nolsm_keep_bounds(self.ctx, steps)

    def set_schedule_table(self, table=None):
        """The autotuner's table ((n_pad, schedule[, ms per block]) arrays, or the committed file when
        None)."""
        t = load_schedule_table() if table is None else table
        nolsm_set_schedule_table(self.ctx, *t)

    def last_schedule(self):
        return nolsm_last_schedule(self.ctx)

    def set_block_bounds(self, bounds):
        nolsm_set_block_bounds(self.ctx, bounds, MEM_HOST if isinstance(bounds, np.ndarray) else MEM_DEVICE)

    def set_wait_budget(self, budget):
        nolsm_set_wait_budget(self.ctx, budget)

    def block_matrix(self, b, which=0):
        return nolsm_block_matrix(self.ctx, b, which)

    def block_factor(self, b):
        return nolsm_block_factor(self.ctx, b)


class BoundPredictor:
    """The spectral-bound network on the GPU; weights live in a raw float32 file plus JSON metadata."""

    def __init__(self, params=None, norm=None, stream=None):
        if norm is None:
            norm = np.concatenate([np.zeros(N_FEATURES), np.ones(N_FEATURES), np.zeros(N_OUTPUTS), np.ones(N_OUTPUTS)])
        self.norm = np.asarray(norm, np.float32)
        self.mlp = nolsm_mlp_create(params, self.norm, stream)

    def close(self):
        if self.mlp:
            nolsm_mlp_destroy(self.mlp)
            self.mlp = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        return nolsm_mlp_get_params(self.mlp)

    def gradient(self, x, t, w=(1.0, 1.0, 1.0), grad=None):
        return nolsm_mlp_gradient(self.mlp, x, t, x.shape[0], w, grad)

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        nolsm_mlp_adam(self.mlp, lr, beta1, beta2, eps)

    def predict(self, x):
        import torch
        y = torch.empty((x.shape[0], N_OUTPUTS), dtype=torch.float32, device=x.device)
        nolsm_mlp_predict(self.mlp, x, x.shape[0], y)
        return y

    def save(self, path, meta=None):
        import json
        base = path[:-5] if path.endswith(".json") else path
        self.params().astype("<f4").tofile(base + ".bin")
        info = {"layers": [32, 128, 128, 3], "activation": "gelu", "n_params": N_PARAMS,
                "params_file": os.path.basename(base + ".bin"), "dtype": "float32 little-endian",
                "norm": [float(v) for v in self.norm], "outputs": ["lambda_min", "lambda_max", "log10_dist_mu"]}
        if meta:
            info.update(meta)
        with open(base + ".json", "w") as f:
            json.dump(info, f, indent=1)

    @classmethod
    def load(cls, path, stream=None):
        import json
        base = path[:-5] if path.endswith(".json") else path
        info = json.load(open(base + ".json"))
        params = np.fromfile(os.path.join(os.path.dirname(base + ".json"), info["params_file"]), dtype="<f4")
        return cls(params, np.asarray(info["norm"], np.float32), stream)
