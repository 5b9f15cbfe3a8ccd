"""Python binding of the QTT GB300 library (include/qtt.h) -- argument marshalling only.

Every computation happens in the CUDA library ``_build/libqtt.so``; this module never falls
back to host arithmetic.  If the library is missing, loading raises.  PyTorch provides the
device memory (caching allocator, through the library's allocator hooks) and the stream.

Function names follow the C ABI: ``qtt_encode``, ``mpo_apply_round``, ``mps_hadamard_round``,
``mps_axpby_round``, ``poisson_solve``, ``fractional_step`` (plus helpers).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqtt.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "qtt.h")

QTT_HOST, QTT_DEVICE = 0, 1
QTT_ORDER_SEQUENTIAL, QTT_ORDER_INTERLEAVED = 0, 1
ORDERING = {"sequential": QTT_ORDER_SEQUENTIAL, "interleaved": QTT_ORDER_INTERLEAVED}
ERRORS = {-1: "QTT_ERR_ARG", -2: "QTT_ERR_ALLOC", -3: "QTT_ERR_CUDA", -4: "QTT_ERR_NOT_CONVERGED",
          -5: "QTT_ERR_TIMEOUT", -6: "QTT_ERR_NONFINITE", -7: "QTT_ERR_UNSUPPORTED"}


class QttError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class qtt_trunc(C.Structure):
    _fields_ = [("chi_max", C.c_int), ("rel_tol", C.c_double), ("prec", C.c_int), ("apply", C.c_int)]


PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
APPLY = {"gram": 0, "sketch": 1}


class qtt_round_info(C.Structure):
    _fields_ = [("max_bond", C.c_int), ("norm", C.c_double), ("discarded_norm", C.c_double)]


class qtt_solve_opts(C.Structure):
    _fields_ = [("max_sweeps", C.c_int), ("rel_tol", C.c_double), ("cg_max_iter", C.c_int),
                ("cg_tol", C.c_double), ("stall", C.c_double)]


class qtt_solve_info(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("cg_iters", C.c_int), ("rel_residual", C.c_double), ("status", C.c_int)]


SOLVE_STATUS = {0: "converged", 1: "stalled", 2: "max_sweeps", 3: "nonfinite", 4: "timeout"}


class qtt_case_params(C.Structure):
    _fields_ = [("n_eta", C.c_int), ("n_xi", C.c_int), ("ordering", C.c_int), ("D", C.c_double),
                ("R", C.c_double), ("Re", C.c_double), ("dt", C.c_double), ("rot", C.c_double),
                ("u_inf", C.c_double), ("chi", C.c_int), ("fit_sweeps", C.c_int),
                ("mom", qtt_solve_opts), ("poi", qtt_solve_opts), ("poisson_warm", C.c_int), ("apply", C.c_int)]


class qtt_step_info(C.Structure):
    _fields_ = [("u", qtt_solve_info), ("v", qtt_solve_info), ("p", qtt_solve_info), ("finite", C.c_int),
                ("cd", C.c_double), ("cl", C.c_double)]


def _solve_dict(i: qtt_solve_info) -> dict:
    return dict(sweeps=i.sweeps, cg_iters=i.cg_iters, rel_residual=i.rel_residual, status=i.status)


def solve_opts(max_sweeps: int, rel_tol: float, cg_max_iter: int, cg_tol: float = 1e-2,
               stall: float = 0.1) -> qtt_solve_opts:
    """ALS options (stop rule of include/qtt.h): sweeps until the true relative residual is
    <= rel_tol, a sweep gains less than the fraction ``stall``, or max_sweeps; local CG to
    cg_tol x the current residual, at most cg_max_iter iterations."""
    return qtt_solve_opts(int(max_sweeps), float(rel_tol), int(cg_max_iter), float(cg_tol), float(stall))


# Step defaults (the oracle's StepOpts has the same): momentum and Poisson solve options.
MOM_DEFAULT = (6, 1e-8, 100, 1e-2, 0.1)
POI_DEFAULT = (12, 1e-10, 500, 1e-2, 0.1)


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
P = C.c_void_p
I, D, L, S = C.c_int, C.c_double, C.c_int64, C.c_size_t
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int)
FLP = C.POINTER(C.c_float)

_SIGS = {
    "qtt_ctx_create": (I, [C.POINTER(P), I, P, ALLOC_FN, FREE_FN, P]),
    "qtt_ctx_destroy": (None, [P]),
    "qtt_ctx_sync": (I, [P]),
    "qtt_last_error": (C.c_char_p, []),
    "qtt_ctx_kernel_launches": (L, [P]),
    "qtt_ctx_pool_bytes": (S, [P]),
    "qtt_ctx_profile": (I, [P, I, DP, DP, C.POINTER(C.c_int64)]),
    "qtt_ctx_profile_phases": (I, [P, DP, C.POINTER(C.c_int64)]),
    "qtt_qr": (I, [P, I, I, I, DP, DP, DP, I]),
    "qtt_ctx_set_cg_mode": (I, [P, I]),
    "qtt_ctx_set_wait_limit": (I, [P, D]),
    "qtt_check_recip": (I, [P, I, DP, DP]),
    "qtt_dgemm": (I, [P, I, I, I, DP, DP, DP, I]),
    "qtt_ctx_set_gemm_mode": (I, [P, I]),
    "qtt_profiler_range": (I, [I]),
    "qtt_mps_create": (I, [P, I, I, IP, DP, I, C.POINTER(P)]),
    "qtt_mps_free": (I, [P]),
    "qtt_mps_n": (I, [P]),
    "qtt_mps_d": (I, [P]),
    "qtt_mps_bonds": (I, [P, IP]),
    "qtt_mps_size": (L, [P]),
    "qtt_mps_get_cores": (I, [P, DP, I]),
    "qtt_mps_device_ptr": (P, [P]),
    "qtt_mps_copy": (I, [P, C.POINTER(P)]),
    "qtt_mpo_create": (I, [P, I, I, IP, DP, I, C.POINTER(P)]),
    "qtt_mpo_free": (I, [P]),
    "qtt_mpo_bonds": (I, [P, IP]),
    "qtt_mpo_get_cores": (I, [P, DP, I]),
    "qtt_encode": (I, [P, DP, I, I, I, qtt_trunc, C.POINTER(P), C.POINTER(qtt_round_info)]),
    "qtt_decode": (I, [P, P, DP, I]),
    "qtt_field_to_vector": (I, [P, DP, DP, I, I, I, I, I]),
    "qtt_round": (I, [P, P, qtt_trunc, C.POINTER(P), C.POINTER(qtt_round_info)]),
    "mps_axpby_round": (I, [P, D, P, D, P, qtt_trunc, C.POINTER(P), C.POINTER(qtt_round_info)]),
    "mpo_apply_round": (I, [P, P, P, qtt_trunc, C.POINTER(P), C.POINTER(qtt_round_info)]),
    "mps_hadamard_round": (I, [P, P, P, qtt_trunc, P, I, C.POINTER(P), C.POINTER(qtt_round_info)]),
    "mps_dot": (I, [P, P, P, DP]),
    "qtt_sym_eig": (I, [P, I, DP, DP, DP]),
    "mps_dot_noalloc": (I, [I, I, IP, P, IP, P, P, P]),
    "poisson_solve": (I, [P, P, P, P, C.POINTER(qtt_solve_opts), C.POINTER(qtt_solve_info)]),
    "qtt_case_create": (I, [P, C.POINTER(qtt_case_params), C.POINTER(P)]),
    "qtt_case_free": (I, [P]),
    "qtt_case_set_state": (I, [P, P, P, P]),
    "qtt_case_get_state": (I, [P, C.POINTER(P), C.POINTER(P), C.POINTER(P)]),
    "qtt_case_get_operator": (I, [P, I, C.POINTER(P)]),
    "qtt_case_get_vector": (I, [P, I, C.POINTER(P)]),
    "fractional_step": (I, [P, P, I, I, C.POINTER(qtt_step_info)]),
    "qtt_ctx_set_autotune": (I, [P, I]),
    "qtt_ctx_set_precision": (I, [P, I]),
    "qtt_ctx_autotune_table": (I, [P, I, C.POINTER(C.c_int64), IP]),
    "fractional_step_batch": (I, [P, I, C.POINTER(P), I, I, C.POINTER(qtt_step_info), IP]),
    "qtt_case_forces": (I, [P, P, DP, DP]),
    "qtt_case_use_graph": (I, [P, I]),
    "qtt_case_phase_ms": (I, [P, DP]),
    "qtt_strouhal": (I, [DP, DP, I, DP]),
    "qtt_nn_param_count": (L, [I, I, I]),
    "qtt_nn_create": (I, [P, I, I, I, FLP, C.POINTER(P)]),
    "qtt_nn_free": (I, [P]),
    "qtt_nn_get_params": (I, [P, FLP]),
    "qtt_nn_get_grad": (I, [P, FLP]),
    "qtt_nn_set_scaling": (I, [P, FLP, FLP, C.c_float]),
    "qtt_nn_predict": (I, [P, I, I, I, FLP, I, FLP, I]),
    "qtt_nn_train_step": (I, [P, I, I, I, FLP, FLP, I, C.c_float, FLP]),
    "qtt_grid_restrict": (I, [P, I, I, I, DP, I, FLP, I]),
    "qtt_grid_prolong": (I, [P, I, I, I, FLP, I, DP, I]),
    "qtt_field_moments": (I, [P, L, FLP, I, DP, DP]),
}


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions declared in include/qtt.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?!typedef)(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"QTT CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def _check(rc):
    if rc != 0:
        raise QttError(rc, lib().qtt_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(DP)


# ------------------------------------------------------------------ context

class Context:
    """One device, one stream (torch's current stream unless given), torch-backed device memory."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True, allocator=None):
        """allocator: optional (alloc(nbytes) -> int device pointer or 0, free(ptr)) pair of Python
        callables given to the library's allocator hooks instead of torch's caching allocator."""
        import torch
        self.device = device
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        sp = P(self.stream.cuda_stream)
        if allocator is not None:
            ua, uf = allocator
            self._alloc = ALLOC_FN(lambda nbytes, _user: ua(int(nbytes)) or None)
            self._free = FREE_FN(lambda ptr, _user: uf(int(ptr)))
        elif use_torch_allocator:
            dev, st = device, self.stream

            def _alloc(nbytes, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            def _free(ptr, _user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc = ALLOC_FN(_alloc)
            self._free = FREE_FN(_free)
        else:
            self._alloc = ALLOC_FN()
            self._free = FREE_FN()
        h = P()
        _check(lib().qtt_ctx_create(C.byref(h), device, sp, self._alloc, self._free, None))
        self.h = h

    def sync(self):
        _check(lib().qtt_ctx_sync(self.h))

    def kernel_launches(self) -> int:
        return int(lib().qtt_ctx_kernel_launches(self.h))

    def pool_bytes(self) -> int:
        return int(lib().qtt_ctx_pool_bytes(self.h))

    PROFILE_CLASSES = ("gemm_f64", "qr_f64", "eig_jacobi", "cg_update", "other",
                       "phase_apply", "phase_rhs_and_momentum", "phase_unused", "phase_poisson", "phase_projection")

    def profile(self, on: bool):
        """Read and reset the per-class kernel timing; switch recording on/off."""
        k = len(self.PROFILE_CLASSES)
        ms = np.zeros(k); fl = np.zeros(k); n = np.zeros(k, dtype=np.int64)
        _check(lib().qtt_ctx_profile(self.h, 1 if on else 0, _dp(ms), _dp(fl),
                                     n.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: dict(ms=float(ms[i]), flops=float(fl[i]), launches=int(n[i]))
                for i, k in enumerate(self.PROFILE_CLASSES)}

    def set_wait_limit(self, seconds: float):
        """Limit of every bounded device wait (grid barriers of the cooperative CG), default 2 s."""
        _check(lib().qtt_ctx_set_wait_limit(self.h, float(seconds)))

    def set_precision(self, prec: str):
        """Contraction precision of the steps and solves on this context: fp64, fp32, tf32, bf16."""
        _check(lib().qtt_ctx_set_precision(self.h, PREC[prec]))

    def set_autotune(self, on: int):
        """1: tune GEMM shapes met from now on; 0: stop tuning (picks stay in use); -1: clear."""
        _check(lib().qtt_ctx_set_autotune(self.h, int(on)))

    def autotune_table(self) -> list[dict]:
        n = C.c_int()
        _check(lib().qtt_ctx_autotune_table(self.h, 0, None, C.byref(n)))
        rows = np.zeros((max(n.value, 1), 9), dtype=np.int64)
        _check(lib().qtt_ctx_autotune_table(self.h, n.value, rows.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(n)))
        keys = ("batch", "M", "N", "K", "engine", "tile", "splits", "best_ns", "default_ns")
        return [dict(zip(keys, (int(v) for v in r))) for r in rows[:n.value]]

    def set_gemm_mode(self, mode: int):
        """0 (default): large products on the tensor cores (digit-split FP64); 1: FP64 pipe only."""
        _check(lib().qtt_ctx_set_gemm_mode(self.h, int(mode)))

    def set_cg_mode(self, mode: int):
        """ALS local CG solves: 0 (default) one cooperative kernel per solve, its contractions on
        the tensor cores at full-bond sites (bonds multiplying to >= 4096) and on the FP64 pipe
        elsewhere; 1 one kernel per stage; 2 the cooperative kernel on the FP64 pipe only; 3 the
        tensor-core contractions wherever the cooperative kernel fits."""
        _check(lib().qtt_ctx_set_cg_mode(self.h, int(mode)))

    def profile_phases(self):
        """Kernel-class ms and launch counts of the last profile() read-out, by step phase."""
        kc = self.PROFILE_CLASSES[:5]
        rows = ("apply", "rhs_and_momentum", "unused", "poisson", "projection", "outside")
        ms = np.zeros(len(rows) * len(kc)); n = np.zeros(len(rows), dtype=np.int64)
        _check(lib().qtt_ctx_profile_phases(self.h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64))))
        ms = ms.reshape(len(rows), len(kc))
        return {r: dict({k: float(ms[i, j]) for j, k in enumerate(kc)}, launches=int(n[i]))
                for i, r in enumerate(rows) if r != "unused"}

    def close(self):
        if getattr(self, "h", None):
            lib().qtt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPS:
    """Handle of a qtt_mps (cores live on the device)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    @classmethod
    def from_cores(cls, ctx: Context, cores) -> "MPS":
        n = len(cores)
        d = cores[0].shape[1]
        bonds = np.array([cores[0].shape[0]] + [c.shape[2] for c in cores], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in cores]))
        h = P()
        _check(lib().qtt_mps_create(ctx.h, n, d, bonds.ctypes.data_as(IP), _dp(flat), QTT_HOST, C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def from_flat(cls, ctx: Context, bonds, d: int, flat_ptr: int) -> "MPS":
        """New MPS whose cores are copied from host memory at ``flat_ptr`` (all cores
        concatenated, float64; may be pinned memory) -- no intermediate host copy."""
        b = np.asarray(bonds, dtype=np.int32)
        h = P()
        _check(lib().qtt_mps_create(ctx.h, len(b) - 1, d, b.ctypes.data_as(IP), C.cast(flat_ptr, DP), QTT_HOST,
                                    C.byref(h)))
        return cls(ctx, h)

    def get_flat(self, flat_ptr: int):
        """Copy all cores (concatenated) into host memory at ``flat_ptr``."""
        _check(lib().qtt_mps_get_cores(self.h, C.cast(flat_ptr, DP), QTT_HOST))

    @property
    def n(self) -> int:
        return lib().qtt_mps_n(self.h)

    @property
    def d(self) -> int:
        return lib().qtt_mps_d(self.h)

    def bonds(self) -> list[int]:
        b = np.zeros(self.n + 1, dtype=np.int32)
        _check(lib().qtt_mps_bonds(self.h, b.ctypes.data_as(IP)))
        return [int(v) for v in b]

    def cores(self) -> list[np.ndarray]:
        b = self.bonds()
        d = self.d
        flat = np.zeros(int(lib().qtt_mps_size(self.h)))
        _check(lib().qtt_mps_get_cores(self.h, _dp(flat), QTT_HOST))
        out, o = [], 0
        for k in range(self.n):
            sz = b[k] * d * b[k + 1]
            out.append(flat[o:o + sz].reshape(b[k], d, b[k + 1]).copy())
            o += sz
        return out

    def copy(self) -> "MPS":
        h = P()
        _check(lib().qtt_mps_copy(self.h, C.byref(h)))
        return MPS(self.ctx, h)

    def __del__(self):
        # Handles die with their context's pool: free only while the context is open.
        try:
            if self.h and self.ctx.h:
                lib().qtt_mps_free(self.h)
            self.h = None
        except Exception:
            pass


class MPO:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    @classmethod
    def from_cores(cls, ctx: Context, cores) -> "MPO":
        n = len(cores)
        d = cores[0].shape[1]
        bonds = np.array([cores[0].shape[0]] + [c.shape[3] for c in cores], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in cores]))
        h = P()
        _check(lib().qtt_mpo_create(ctx.h, n, d, bonds.ctypes.data_as(IP), _dp(flat), QTT_HOST, C.byref(h)))
        return cls(ctx, h)

    def bonds(self) -> list[int]:
        b = np.zeros(65, dtype=np.int32)
        _check(lib().qtt_mpo_bonds(self.h, b.ctypes.data_as(IP)))
        nz = int(np.nonzero(b)[0][-1]) + 1
        return [int(v) for v in b[:nz]]

    def cores(self) -> list[np.ndarray]:
        b = self.bonds()
        n = len(b) - 1
        tot = sum(b[k] * 4 * b[k + 1] for k in range(n))
        flat = np.zeros(tot)
        _check(lib().qtt_mpo_get_cores(self.h, _dp(flat), QTT_HOST))
        out, o = [], 0
        for k in range(n):
            sz = b[k] * 4 * b[k + 1]
            out.append(flat[o:o + sz].reshape(b[k], 2, 2, b[k + 1]).copy())
            o += sz
        return out

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib().qtt_mpo_free(self.h)
            self.h = None
        except Exception:
            pass


# ------------------------------------------------------------------ operations (C-ABI names)

def _trunc(chi, rel_tol, prec="fp64", apply="gram"):
    return qtt_trunc(int(chi), float(rel_tol), PREC[prec], APPLY[apply])


def _info_ptr(out_info):
    return C.byref(out_info[1]) if out_info is not None else None


def _round_info(out_info):
    """(dict to fill, struct) when the caller asked for the rounding record."""
    return None if out_info is None else (out_info, qtt_round_info())


def _fill_round(ri):
    if ri is not None:
        d, st = ri
        d.update(max_bond=st.max_bond, norm=st.norm, discarded_norm=st.discarded_norm)


def qtt_encode(ctx: Context, dense, n: int, chi: int, rel_tol: float = 0.0, d: int = 2, out_info=None) -> MPS:
    a = np.ascontiguousarray(np.asarray(dense, dtype=np.float64).ravel())
    h = P()
    ri = _round_info(out_info)
    _check(lib().qtt_encode(ctx.h, _dp(a), QTT_HOST, n, d, _trunc(chi, rel_tol), C.byref(h), _info_ptr(ri)))
    _fill_round(ri)
    return MPS(ctx, h)


def qtt_decode(ctx: Context, x: MPS) -> np.ndarray:
    out = np.zeros(x.d ** x.n)
    _check(lib().qtt_decode(ctx.h, x.h, _dp(out), QTT_HOST))
    return out


def qtt_field_to_vector(ctx: Context, field, ordering: str, inverse: bool = False) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(field, dtype=np.float64))
    if inverse:
        raise ValueError("use qtt_vector_to_field")
    ne, nx = int(np.log2(a.shape[0])), int(np.log2(a.shape[1]))
    out = np.zeros(a.size)
    _check(lib().qtt_field_to_vector(ctx.h, _dp(a), _dp(out), QTT_HOST, ne, nx, ORDERING[ordering], 0))
    return out


def qtt_vector_to_field(ctx: Context, vec, n_eta: int, n_xi: int, ordering: str) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(vec, dtype=np.float64).ravel())
    out = np.zeros(a.size)
    _check(lib().qtt_field_to_vector(ctx.h, _dp(a), _dp(out), QTT_HOST, n_eta, n_xi, ORDERING[ordering], 1))
    return out.reshape(2 ** n_eta, 2 ** n_xi)


def qtt_round(ctx: Context, x: MPS, chi: int, rel_tol: float = 0.0, out_info=None, prec: str = "fp64") -> MPS:
    """TT-rounding; ``out_info`` (a dict, optional) receives max_bond, norm, discarded_norm."""
    h = P()
    ri = _round_info(out_info)
    _check(lib().qtt_round(ctx.h, x.h, _trunc(chi, rel_tol, prec), C.byref(h), _info_ptr(ri)))
    _fill_round(ri)
    return MPS(ctx, h)


def mps_axpby_round(ctx: Context, alpha: float, x: MPS, beta: float, y: MPS, chi: int, rel_tol: float = 0.0,
                    out_info=None, prec: str = "fp64") -> MPS:
    h = P()
    ri = _round_info(out_info)
    _check(lib().mps_axpby_round(ctx.h, alpha, x.h, beta, y.h, _trunc(chi, rel_tol, prec), C.byref(h),
                                 _info_ptr(ri)))
    _fill_round(ri)
    return MPS(ctx, h)


def mpo_apply_round(ctx: Context, M: MPO, x: MPS, chi: int, rel_tol: float = 0.0, out_info=None,
                    prec: str = "fp64", apply: str = "gram") -> MPS:
    """apply: "gram" (Gram-environment rounding) or "sketch" (sketched orthogonalisation with
    factored eigenpair refinement), QTT_APPLY_* of include/qtt.h."""
    h = P()
    ri = _round_info(out_info)
    _check(lib().mpo_apply_round(ctx.h, M.h, x.h, _trunc(chi, rel_tol, prec, apply), C.byref(h), _info_ptr(ri)))
    _fill_round(ri)
    return MPS(ctx, h)


def mps_hadamard_round(ctx: Context, a: MPS, b: MPS, chi: int, sweeps: int = 2, init: MPS | None = None,
                       out_info=None, prec: str = "fp64") -> MPS:
    h = P()
    ri = _round_info(out_info)
    _check(lib().mps_hadamard_round(ctx.h, a.h, b.h, _trunc(chi, 0.0, prec), init.h if init is not None else None,
                                    sweeps, C.byref(h), _info_ptr(ri)))
    _fill_round(ri)
    return MPS(ctx, h)


def profiler_range(start: bool):
    """cudaProfilerStart / Stop (to bracket the launches an external profiler captures)."""
    _check(lib().qtt_profiler_range(1 if start else 0))


def mps_dot_noalloc(n: int, d: int, a_bonds, a_cores_dev: int, b_bonds, b_cores_dev: int, out_dev: int,
                    stream: int = 0):
    """<a, b> into the device double at ``out_dev`` without allocating device memory; cores are
    given as device pointers to unpadded concatenated cores (see include/qtt.h)."""
    ab = np.ascontiguousarray(np.asarray(a_bonds, dtype=np.int32))
    bb = np.ascontiguousarray(np.asarray(b_bonds, dtype=np.int32))
    _check(lib().mps_dot_noalloc(n, d, ab.ctypes.data_as(IP), a_cores_dev, bb.ctypes.data_as(IP), b_cores_dev,
                                 out_dev, stream))


def qtt_dgemm(ctx: Context, A, B, path: int = 0):
    """A @ B on the device (row-major FP64); path 0 context mode, 1 FP64 pipe, 2 tensor cores."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64))
    m, k = A.shape
    k2, n = B.shape
    if k2 != k:
        raise ValueError("inner dimensions differ")
    Cm = np.zeros((m, n))
    _check(lib().qtt_dgemm(ctx.h, m, n, k, _dp(A), _dp(B), _dp(Cm), int(path)))
    return Cm


def qtt_check_recip(ctx: Context, x):
    """Max relative errors (reciprocal, reciprocal square root) of the QR's Newton iterations."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    err = np.zeros(2)
    _check(lib().qtt_check_recip(ctx.h, x.size, _dp(x), _dp(err)))
    return float(err[0]), float(err[1])


def qtt_qr(ctx: Context, A, trans: bool = False, path: int = 0):
    """Householder QR of a small dense matrix on the device: A = Q R (LAPACK sign convention).

    With trans=True the argument is A^T (n x m) and Q^T is returned in place of Q.
    path: 0 automatic, 1 one CTA, 2 cluster kernel."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    if trans:
        n, m = A.shape
    else:
        m, n = A.shape
    kk = min(m, n)
    Q = np.zeros((kk, m) if trans else (m, kk))
    R = np.zeros((kk, n))
    _check(lib().qtt_qr(ctx.h, m, n, 1 if trans else 0, _dp(A), _dp(Q), _dp(R), int(path)))
    return Q, R


def qtt_sym_eig(ctx: Context, S):
    """(w descending, V with eigenvectors as columns) of a small symmetric matrix."""
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
    n = S.shape[0]
    w = np.zeros(n); V = np.zeros((n, n))
    _check(lib().qtt_sym_eig(ctx.h, n, _dp(S), _dp(w), _dp(V)))
    return w, V


def mps_dot(ctx: Context, a: MPS, b: MPS) -> float:
    out = C.c_double()
    _check(lib().mps_dot(ctx.h, a.h, b.h, C.byref(out)))
    return out.value


def poisson_solve(ctx: Context, A: MPO, b: MPS, x: MPS, max_sweeps: int, rel_tol: float, cg_max_iter: int,
                  cg_tol: float = 1e-2, stall: float = 0.1, check: bool = False) -> dict:
    """Solve A x = b in place on x (ALS under the stop rule of include/qtt.h).  Returns the solve
    record (sweeps, cg_iters, rel_residual, status) and the return code (``rc``); a stall or
    running out of sweeps raises only when ``check``; other errors always raise."""
    o = solve_opts(max_sweeps, rel_tol, cg_max_iter, cg_tol, stall)
    info = qtt_solve_info()
    rc = lib().poisson_solve(ctx.h, A.h, b.h, x.h, C.byref(o), C.byref(info))
    if rc != 0 and (check or rc != -4):
        _check(rc)
    return dict(_solve_dict(info), rc=rc)


# ------------------------------------------------------------------ cylinder case

class Case:
    def __init__(self, ctx: Context, n_eta: int, n_xi: int, R: float, Re: float, dt: float, chi: int,
                 ordering: str = "interleaved", D: float = 1.0, rot: float = 0.0, u_inf: float = 1.0,
                 fit_sweeps: int = 1, mom=MOM_DEFAULT, poi=POI_DEFAULT, poisson_warm: str = "previous",
                 apply: str = "gram"):
        """mom, poi: ALS options (max_sweeps, rel_tol, cg_max_iter[, cg_tol[, stall]]); poisson_warm:
        "previous" (p^m) or "extrapolated" (2 p^m - p^(m-1), fitted); apply: rounding of the
        step's MPO-MPS products, "gram" or "sketch"."""
        self.ctx = ctx
        self.params = qtt_case_params(n_eta, n_xi, ORDERING[ordering], D, R, Re, dt, rot, u_inf, chi, fit_sweeps,
                                      solve_opts(*mom), solve_opts(*poi),
                                      {"previous": 0, "extrapolated": 1}[poisson_warm], APPLY[apply])
        h = P()
        _check(lib().qtt_case_create(ctx.h, C.byref(self.params), C.byref(h)))
        self.h = h

    def set_state(self, u: MPS, v: MPS, p: MPS):
        _check(lib().qtt_case_set_state(self.h, u.h, v.h, p.h))

    def get_state(self):
        hu, hv, hp = P(), P(), P()
        _check(lib().qtt_case_get_state(self.h, C.byref(hu), C.byref(hv), C.byref(hp)))
        return MPS(self.ctx, hu), MPS(self.ctx, hv), MPS(self.ctx, hp)

    def operator(self, which: int) -> MPO:
        h = P()
        _check(lib().qtt_case_get_operator(self.h, which, C.byref(h)))
        return MPO(self.ctx, h)

    def vector(self, which: int):
        h = P()
        _check(lib().qtt_case_get_vector(self.h, which, C.byref(h)))
        return MPS(self.ctx, h) if h.value else None

    def fractional_step(self, nsteps: int = 1, with_forces: bool = False, check: bool = True):
        return fractional_step(self.ctx, self, nsteps, with_forces, check=check)

    def phase_ms(self):
        """Wall time (ms) of the last step's phases: apply, rhs+momentum, Poisson, projection."""
        out = np.zeros(4)
        _check(lib().qtt_case_phase_ms(self.h, _dp(out)))
        return dict(zip(("apply", "rhs_and_momentum", "poisson", "projection"), out.tolist()))

    def use_graph(self, enable: bool):
        _check(lib().qtt_case_use_graph(self.h, 1 if enable else 0))

    def forces(self):
        cd, cl = C.c_double(), C.c_double()
        _check(lib().qtt_case_forces(self.ctx.h, self.h, C.byref(cd), C.byref(cl)))
        return cd.value, cl.value

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib().qtt_case_free(self.h)
            self.h = None
        except Exception:
            pass


def fractional_step(ctx: Context, case: Case, nsteps: int = 1, with_forces: bool = False, info: bool = True,
                    check: bool = True):
    """Advance ``nsteps`` fractional steps; returns per-step dicts (the three solve records u, v,
    p, ``finite``, C_D, C_L; plus cg_u, cg_v, cg_p) or None.  A non-zero return code raises when
    ``check`` (the exception carries the records as ``.records``)."""
    if not info:
        rc = lib().fractional_step(ctx.h, case.h, nsteps, 0, None)
        if rc != 0 and check:
            raise QttError(rc, lib().qtt_last_error().decode())
        return None
    recs = (qtt_step_info * max(nsteps, 1))()
    rc = lib().fractional_step(ctx.h, case.h, nsteps, 1 if with_forces else 0, recs)
    out = [dict(u=_solve_dict(r.u), v=_solve_dict(r.v), p=_solve_dict(r.p), finite=r.finite, cd=r.cd, cl=r.cl,
                cg_u=r.u.cg_iters, cg_v=r.v.cg_iters, cg_p=r.p.cg_iters, rc=rc) for r in recs[:nsteps]]
    if rc != 0 and check:
        err = QttError(rc, lib().qtt_last_error().decode())
        err.records = out
        raise err
    return out


def fractional_step_batch(ctx: Context, cases, nsteps: int = 1, with_forces: bool = False, info: bool = True,
                          check: bool = True):
    """Advance every case of ``cases`` by ``nsteps`` fractional steps, their step graphs replayed
    concurrently.  Returns (records, statuses): records[i] is the list of per-step dicts of case
    i (as fractional_step returns them; None when ``info`` is false), statuses[i] its return code.
    The most severe non-zero code raises when ``check`` (the exception carries ``.records`` and
    ``.statuses``)."""
    n = len(cases)
    hs = (P * n)(*[cs.h for cs in cases])
    status = np.zeros(n, dtype=np.int32)
    recs = (qtt_step_info * max(n * nsteps, 1))() if info else None
    rc = lib().fractional_step_batch(ctx.h, n, hs, nsteps, 1 if (with_forces and info) else 0, recs,
                                     status.ctypes.data_as(IP))
    out = None
    if info:
        out = [[dict(u=_solve_dict(r.u), v=_solve_dict(r.v), p=_solve_dict(r.p), finite=r.finite, cd=r.cd,
                     cl=r.cl, cg_u=r.u.cg_iters, cg_v=r.v.cg_iters, cg_p=r.p.cg_iters, rc=int(status[i]))
                for r in recs[i * nsteps:(i + 1) * nsteps]] for i in range(n)]
    if rc != 0 and check:
        err = QttError(rc, lib().qtt_last_error().decode())
        err.records, err.statuses = out, [int(v) for v in status]
        raise err
    return out, [int(v) for v in status]


def _fp(a: np.ndarray):
    return a.ctypes.data_as(FLP)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class NN:
    """The learned warm start's network (FP32, on the context's device)."""

    def __init__(self, ctx: Context, c_in: int, width: int, depth: int, params):
        self.ctx, self.c_in, self.width, self.depth = ctx, c_in, width, depth
        p = _f32(params)
        if p.size != self.param_count(c_in, width, depth):
            raise ValueError("params: wrong size")
        h = P()
        _check(lib().qtt_nn_create(ctx.h, c_in, width, depth, _fp(p), C.byref(h)))
        self.h = h

    @staticmethod
    def param_count(c_in: int, width: int, depth: int) -> int:
        return int(lib().qtt_nn_param_count(c_in, width, depth))

    def params(self) -> np.ndarray:
        out = np.zeros(self.param_count(self.c_in, self.width, self.depth), dtype=np.float32)
        _check(lib().qtt_nn_get_params(self.h, _fp(out)))
        return out

    def grad(self) -> np.ndarray:
        out = np.zeros(self.param_count(self.c_in, self.width, self.depth), dtype=np.float32)
        _check(lib().qtt_nn_get_grad(self.h, _fp(out)))
        return out

    def set_scaling(self, shift, scale, out_scale: float):
        _check(lib().qtt_nn_set_scaling(self.h, _fp(_f32(shift)), _fp(_f32(scale)), float(out_scale)))

    def predict(self, x) -> np.ndarray:
        x = _f32(x)
        B, _, H, W = x.shape
        y = np.zeros((B, 1, H, W), dtype=np.float32)
        _check(lib().qtt_nn_predict(self.h, B, H, W, _fp(x), QTT_HOST, _fp(y), QTT_HOST))
        return y

    def train_step(self, x, y, lr: float) -> float:
        x, y = _f32(x), _f32(y)
        B, _, H, W = x.shape
        loss = C.c_float()
        _check(lib().qtt_nn_train_step(self.h, B, H, W, _fp(x), _fp(y), QTT_HOST, float(lr), C.byref(loss)))
        return float(loss.value)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib().qtt_nn_free(self.h)
            self.h = None
        except Exception:
            pass


def grid_restrict(ctx: Context, fine, levels: int) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(fine, dtype=np.float64))
    Hc, Wc = f.shape[0] >> levels, f.shape[1] >> levels
    out = np.zeros((Hc, Wc), dtype=np.float32)
    _check(lib().qtt_grid_restrict(ctx.h, Hc, Wc, levels, _dp(f), QTT_HOST, _fp(out), QTT_HOST))
    return out


def grid_prolong(ctx: Context, coarse, levels: int) -> np.ndarray:
    c = _f32(coarse)
    Hc, Wc = c.shape
    out = np.zeros((Hc << levels, Wc << levels))
    _check(lib().qtt_grid_prolong(ctx.h, Hc, Wc, levels, _fp(c), QTT_HOST, _dp(out), QTT_HOST))
    return out


def field_moments(ctx: Context, x) -> tuple[float, float]:
    a = _f32(x).ravel()
    m, r = C.c_double(), C.c_double()
    _check(lib().qtt_field_moments(ctx.h, a.size, _fp(a), QTT_HOST, C.byref(m), C.byref(r)))
    return m.value, r.value


def qtt_strouhal(t, cl) -> float:
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    c = np.ascontiguousarray(np.asarray(cl, dtype=np.float64))
    out = C.c_double()
    _check(lib().qtt_strouhal(_dp(t), _dp(c), len(t), C.byref(out)))
    return out.value
