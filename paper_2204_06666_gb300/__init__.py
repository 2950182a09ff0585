"""Python binding of libehyb.so, the GB300 EHYB SpMV library (C ABI in include/ehyb.h).

Argument marshalling only: every step of the SpMV runs in the library's CUDA kernels.
PyTorch supplies device memory and streams; numpy arrays carry host CSR data.  The
module-level functions carry the C names (``ehyb_plan_create_csr``, ``ehyb_spmv`` ...);
``Plan`` and ``CsrBaseline`` wrap them with exceptions and ownership.

There is no fallback: if libehyb.so is missing the import fails with instructions.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# EHYB_LIBRARY: path of another build of the same library (e.g. one compiled with different options)
_LIB_PATH = os.environ.get("EHYB_LIBRARY") or os.path.join(_PKG, "libehyb.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(or python paper_2204_06666_gb300/build.py) first")

_lib = ctypes.CDLL(_LIB_PATH)

STATUS = {0: "EHYB_OK", 1: "EHYB_ERR_INVALID_ARG", 2: "EHYB_ERR_NOT_SQUARE", 3: "EHYB_ERR_INDEX_RANGE",
          4: "EHYB_ERR_TOO_LARGE", 5: "EHYB_ERR_OOM", 6: "EHYB_ERR_CUDA", 7: "EHYB_ERR_UNSUPPORTED",
          8: "EHYB_ERR_NOT_CONVERGED", 9: "EHYB_ERR_TIMEOUT", 10: "EHYB_ERR_NO_DEVICE", 11: "EHYB_ERR_IO",
          12: "EHYB_ERR_BOUNDS"}
EHYB_OK, EHYB_ERR_TIMEOUT, EHYB_ERR_NOT_CONVERGED, EHYB_ERR_IO = 0, 9, 8, 11


class EhybError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = _lib.ehyb_status_string(self.status).decode()
        cuda = _lib.ehyb_last_cuda_error().decode()
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)} ({msg})" + (f" [{cuda}]" if cuda else ""))


class Options(ctypes.Structure):
    _fields_ = [("slice_rows", ctypes.c_int32), ("ell_width_cap", ctypes.c_int32), ("ell_tpr", ctypes.c_int32),
                ("er_tpr", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("lowp", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("num_sms", ctypes.c_int32), ("smem_budget", ctypes.c_int32),
                ("part_vec", ctypes.c_void_p), ("wait_timeout_ns", ctypes.c_int64),
                ("inject_wait_fault", ctypes.c_int32), ("keep_host", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("er_layout", ctypes.c_int32), ("part_nnz", ctypes.c_int32), ("tuner", ctypes.c_int32),
                ("host_threads", ctypes.c_int32), ("partitioner", ctypes.c_int32), ("lowp_group", ctypes.c_int32),
                ("spmm_rhs", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nparts", ctypes.c_int32),
                ("nslices", ctypes.c_int32), ("slice_rows", ctypes.c_int32), ("ell_tpr", ctypes.c_int32),
                ("er_tpr", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("lowp", ctypes.c_int32), ("ell_nnz", ctypes.c_int64), ("ell_stored", ctypes.c_int64),
                ("er_rows", ctypes.c_int64), ("er_nnz", ctypes.c_int64), ("bytes_effective", ctypes.c_int64),
                ("bytes_device", ctypes.c_int64), ("partition_ms", ctypes.c_double), ("reorder_ms", ctypes.c_double),
                ("upload_ms", ctypes.c_double), ("device_status", ctypes.c_int32), ("num_sms", ctypes.c_int32),
                ("er_layout", ctypes.c_int32), ("er_stored", ctypes.c_int64), ("tuner_path", ctypes.c_int32),
                ("ell_width_cap", ctypes.c_int32), ("lowp_group", ctypes.c_int32), ("max_stage_rows", ctypes.c_int32),
                ("n_halo", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanExport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nparts", ctypes.c_int32), ("nslices", ctypes.c_int32),
                ("tpr", ctypes.c_int32), ("ell_stored", ctypes.c_int64), ("er_rows", ctypes.c_int64),
                ("er_nnz", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in (
                    "new_to_old", "part_ptr", "slice_ptr", "slice_pos", "ell_col", "ell_val", "row_ell_count",
                    "er_part_ptr", "er_row", "er_ptr", "er_col", "er_val")] + [
                ("er_layout", ctypes.c_int32), ("er_stored", ctypes.c_int64), ("er_slice_pos", ctypes.c_void_p),
                ("er_scol", ctypes.c_void_p), ("er_sval", ctypes.c_void_p), ("row_er_count", ctypes.c_void_p),
                ("lowp", ctypes.c_int32), ("lowp_group", ctypes.c_int32), ("ell_val_low", ctypes.c_void_p),
                ("ell_col_low", ctypes.c_void_p), ("er_sval_low", ctypes.c_void_p), ("er_scol_low", ctypes.c_void_p),
                ("n_halo", ctypes.c_int64), ("halo_ptr", ctypes.c_void_p), ("halo_new", ctypes.c_void_p)]


class CgInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("flexible", ctypes.c_int32), ("relres", ctypes.c_double), ("relres_recursive", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneEntry(ctypes.Structure):
    _fields_ = [("slice_rows", ctypes.c_int32), ("ell_width_cap", ctypes.c_int32), ("ell_tpr", ctypes.c_int32),
                ("valid", ctypes.c_int32), ("ms", ctypes.c_double)]


_P, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("ehyb_status_string", [ctypes.c_int], ctypes.c_char_p)
_sig("ehyb_last_cuda_error", [], ctypes.c_char_p)
_sig("ehyb_options_default", [ctypes.POINTER(Options)], None)
_sig("ehyb_test_fail_allocs_after", [_I32], None)
_sig("ehyb_test_bounds_probe", [_I64, _I64])
_sig("ehyb_plan_create_csr", [_I64, _I64, _I64, _P, _P, _P, ctypes.POINTER(Options), _P, ctypes.POINTER(_P)])
_sig("ehyb_destroy", [_P])
_sig("ehyb_spmv", [_P, _P, _P, _P])
_sig("ehyb_spmv_permuted", [_P, _P, _P, _P])
_sig("ehyb_permute", [_P, _I32, _P, _P, _P])
_sig("ehyb_spmv_host", [_P, _P, _P, _P])
_sig("ehyb_spmv_host_many", [_P, _I32, _P, _P, _P])
_sig("ehyb_spmv_lowp", [_P, _P, _P, _P])
_sig("ehyb_spmv_noalloc", [_P, _P, _P, _P])
_sig("ehyb_spmm", [_P, _I32, _P, _P, _P])
_sig("ehyb_cg", [_P, _P, _P, _D, _I32, _I32, _D, ctypes.POINTER(CgInfo), _P])
_sig("ehyb_cg_history", [_P, _P, _I32, ctypes.POINTER(_I32)])
_sig("ehyb_batch_create", [_I32, _P, ctypes.POINTER(_P)])
_sig("ehyb_batch_spmv", [_P, _P, _P, _P])
_sig("ehyb_batch_info", [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)])
_sig("ehyb_batch_destroy", [_P])
_sig("ehyb_tune_grid_size", [], _I32)
_sig("ehyb_tune_grid", [_I64, _P, _I32, _I32, _P])
_sig("ehyb_features", [_I64, _P, _P, _P, _I32, _P])
_sig("ehyb_tune_sweep", [_I64, _I64, _P, _P, _P, _I32, _P, ctypes.POINTER(_I32), _P])
_sig("ehyb_tuner_set_model", [_P, _P, _P, _P, _P])
_sig("ehyb_tuner_predict", [_I64, _I64, _P, _P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                            ctypes.POINTER(_I32), ctypes.POINTER(_D)])
_sig("ehyb_mlp_param_count", [], _I32)
_sig("ehyb_mlp_workspace_bytes", [_I32], _I64)
_sig("ehyb_mlp_forward", [_P, _P, _I32, _P, _P, _P])
_sig("ehyb_mlp_loss_grad", [_P, _P, _P, _I32, _P, _P, _P, _P])
_sig("ehyb_mlp_adam", [_P, _P, _P, _P, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P])
_sig("ehyb_fp64_fma_peak", [_I32, _I32, ctypes.POINTER(_D), ctypes.POINTER(_D)])


class ShardInfo(ctypes.Structure):
    _fields_ = [("nranks", ctypes.c_int32), ("rank", ctypes.c_int32), ("part_begin", ctypes.c_int32),
                ("part_end", ctypes.c_int32), ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64),
                ("n_local", ctypes.c_int64), ("n_halo", ctypes.c_int64), ("send_total", ctypes.c_int64),
                ("slab_stored", ctypes.c_int64), ("er_stored", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32)
_sig("ehyb_shard_create", [_P, _I32, _I32, _P, ctypes.POINTER(_P)])
_sig("ehyb_shard_info", [_P, ctypes.POINTER(ShardInfo)])
_sig("ehyb_shard_lists", [_P, _P, _P, _P, _P])
_sig("ehyb_shard_export", [_P, ctypes.POINTER(PlanExport)])
_sig("ehyb_shard_pack", [_P, _P, _P, _P])
_sig("ehyb_shard_spmv", [_P, _P, _P, _P])
_sig("ehyb_shard_cg", [_P, _P, _P, _P, _P, _D, _I32, EXCHANGE_FN, ALLREDUCE_FN, _P, ctypes.POINTER(CgInfo), _P])
_sig("ehyb_shard_destroy", [_P])
_sig("ehyb_plan_info", [_P, ctypes.POINTER(PlanInfo)])
_sig("ehyb_plan_check", [_P])
_sig("ehyb_plan_export", [_P, ctypes.POINTER(PlanExport)])
_sig("ehyb_plan_save", [_P, ctypes.c_char_p])
_sig("ehyb_fsai_create", [_P, _I64, _I64, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)])
_sig("ehyb_precond_info", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D)])
_sig("ehyb_precond_export", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)])
_sig("ehyb_precond_destroy", [_P])
_sig("ehyb_pcg", [_P, _P, _P, _P, _D, _I32, ctypes.POINTER(CgInfo), _P])
_sig("ehyb_pcg_history", [_P, _P, _I32, ctypes.POINTER(_I32)])
_sig("ehyb_pcg_refined", [_P, _P, _P, _P, _D, _I32, _D, ctypes.POINTER(CgInfo), _P])
_sig("ehyb_plan_load", [ctypes.c_char_p, ctypes.POINTER(Options), _P, ctypes.POINTER(_P)])
_sig("ehyb_profile_enable", [_P, _I32])
_sig("ehyb_profile_read", [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)])
_sig("ehyb_csr_create", [_I64, _I64, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)])
_sig("ehyb_csr_spmv", [_P, _P, _P, _P])
_sig("ehyb_csr_set_tpr", [_P, _I32])
_sig("ehyb_csr_destroy", [_P])


def lib_path() -> str:
    return _LIB_PATH


def _check(st: int, where: str):
    if st != 0:
        raise EhybError(st, where)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype_name: str) -> int:
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch." + dtype_name):
        raise TypeError(f"expected a contiguous CUDA torch.{dtype_name} tensor, got {t.dtype} on {t.device}")
    return t.data_ptr()


def _host(a, dtype) -> int:
    if hasattr(a, "data_ptr") and not hasattr(a, "ctypes"):  # torch CPU tensor (possibly pinned)
        if a.is_cuda or not a.is_contiguous() or a.element_size() != np.dtype(dtype).itemsize:
            raise TypeError(f"expected a contiguous CPU tensor of {np.dtype(dtype)}")
        return a.data_ptr()
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a contiguous numpy {np.dtype(dtype)} array")
    return a.ctypes.data


def make_options(**kw) -> Options:
    o = Options()
    _lib.ehyb_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "part_vec":
            continue
        setattr(o, k, int(v))
    return o


# ---------------------------------------------------------------- C-named thin wrappers

def ehyb_plan_create_csr(n_rows, n_cols, nnz, row_ptr, col, val, opt: Options | None, stream, out: ctypes.c_void_p):
    return _lib.ehyb_plan_create_csr(n_rows, n_cols, nnz, row_ptr, col, val,
                                     ctypes.byref(opt) if opt is not None else None, stream, ctypes.byref(out))


def ehyb_destroy(plan):
    return _lib.ehyb_destroy(plan)


def ehyb_spmv(plan, x, y, stream):
    return _lib.ehyb_spmv(plan, x, y, stream)


def ehyb_spmv_permuted(plan, xp, yp, stream):
    return _lib.ehyb_spmv_permuted(plan, xp, yp, stream)


def ehyb_permute(plan, to_new, x, y, stream):
    return _lib.ehyb_permute(plan, to_new, x, y, stream)


def ehyb_spmv_host(plan, x, y, stream):
    return _lib.ehyb_spmv_host(plan, x, y, stream)


def ehyb_spmv_lowp(plan, x, y, stream):
    return _lib.ehyb_spmv_lowp(plan, x, y, stream)


def ehyb_spmv_noalloc(plan, x, y, stream):
    return _lib.ehyb_spmv_noalloc(plan, x, y, stream)


def ehyb_cg(plan, b, x, rtol, max_iter, refine, inner_rtol, info: CgInfo, stream):
    return _lib.ehyb_cg(plan, b, x, rtol, max_iter, refine, inner_rtol, ctypes.byref(info), stream)


def ehyb_plan_check(plan):
    return _lib.ehyb_plan_check(plan)


def ehyb_plan_save(plan, path: str):
    return _lib.ehyb_plan_save(plan, os.fsencode(path))


def ehyb_plan_load(path: str, opt: Options | None, stream, out: ctypes.c_void_p):
    return _lib.ehyb_plan_load(os.fsencode(path), ctypes.byref(opt) if opt is not None else None, stream,
                               ctypes.byref(out))


def fp64_fma_peak(iters: int = 2048, reps: int = 5) -> tuple[float, float]:
    """(TFLOP/s, best launch ms) of the current device's FP64 FMA pipe (ehyb_fp64_fma_peak)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ehyb_fp64_fma_peak(iters, reps, ctypes.byref(tf), ctypes.byref(ms)), "ehyb_fp64_fma_peak")
    return tf.value, ms.value


def ehyb_test_fail_allocs_after(count: int):
    _lib.ehyb_test_fail_allocs_after(count)


def ehyb_test_bounds_probe(i: int, lim: int) -> int:
    return int(_lib.ehyb_test_bounds_probe(int(i), int(lim)))


# ---------------------------------------------------------------- owning wrappers

class Plan:
    """An EHYB plan built from a host CSR matrix (anything with n, row_ptr, col, val)."""

    def __init__(self, A, stream=None, part_vec=None, **opts):
        self._h = ctypes.c_void_p()
        rp = np.ascontiguousarray(A.row_ptr, np.int64)
        c = np.ascontiguousarray(A.col, np.int32)
        v = np.ascontiguousarray(A.val, np.float64)
        n = int(A.n)
        n_cols = int(opts.pop("n_cols", n))
        o = make_options(**opts)
        pv = None
        if part_vec is not None:
            pv = np.ascontiguousarray(part_vec, np.int32)
            o.part_vec = pv.ctypes.data
        self.host_only = bool(opts.get("host_only", 0))
        s = None if self.host_only else _stream(stream)
        st = ehyb_plan_create_csr(n, n_cols, int(rp[-1]) if rp.size else 0, rp.ctypes.data, c.ctypes.data,
                                  v.ctypes.data, o, s, self._h)
        _check(st, "ehyb_plan_create_csr")
        self.n = n

    @classmethod
    def load(cls, path: str, stream=None, **opts):
        """A plan read from a file written by save() (no partitioning or encoding; opts: run-time choices)."""
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        o = make_options(**opts)
        self.host_only = bool(opts.get("host_only", 0))
        s = None if self.host_only else _stream(stream)
        _check(ehyb_plan_load(path, o, s, self._h), "ehyb_plan_load")
        self.n = int(self.info()["n"])
        return self

    def save(self, path: str):
        _check(ehyb_plan_save(self._h, path), "ehyb_plan_save")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()   # the handle is released whatever the status
            _check(_lib.ehyb_destroy(h), "ehyb_destroy")

    def __del__(self):
        try:
            if self._h:
                _lib.ehyb_destroy(self._h)
        except Exception:
            pass

    def spmv(self, x, y, stream=None):
        _check(ehyb_spmv(self._h, _dev(x, "float64"), _dev(y, "float64"), _stream(stream)), "ehyb_spmv")

    def spmv_permuted(self, xp, yp, stream=None):
        _check(ehyb_spmv_permuted(self._h, _dev(xp, "float64"), _dev(yp, "float64"), _stream(stream)),
               "ehyb_spmv_permuted")

    def permute(self, to_new: bool, x, y, stream=None):
        _check(ehyb_permute(self._h, int(bool(to_new)), _dev(x, "float64"), _dev(y, "float64"), _stream(stream)),
               "ehyb_permute")

    def spmv_host(self, x, y, stream=None):
        _check(ehyb_spmv_host(self._h, _host(x, np.float64), _host(y, np.float64), _stream(stream)),
               "ehyb_spmv_host")

    def spmv_host_many(self, xs, ys, stream=None):
        """y_i = A x_i for lists of CPU float64 tensors (pinned for overlap), copies and products pipelined."""
        if len(xs) != len(ys):
            raise ValueError("xs and ys differ in length")
        X = (ctypes.c_void_p * max(1, len(xs)))(*[_host(x, np.float64) for x in xs])
        Y = (ctypes.c_void_p * max(1, len(ys)))(*[_host(y, np.float64) for y in ys])
        _check(_lib.ehyb_spmv_host_many(self._h, len(xs), X, Y, _stream(stream)), "ehyb_spmv_host_many")

    def spmv_lowp(self, x, y, stream=None):
        _check(ehyb_spmv_lowp(self._h, _dev(x, "float32"), _dev(y, "float32"), _stream(stream)), "ehyb_spmv_lowp")

    def spmv_noalloc(self, x, y, stream=None):
        _check(ehyb_spmv_noalloc(self._h, _dev(x, "float64"), _dev(y, "float64"), _stream(stream)),
               "ehyb_spmv_noalloc")

    def spmm(self, X, Y, stream=None):
        """Y = A X for row-major (n, k) CUDA float64 tensors."""
        if X.dim() != 2 or X.shape != Y.shape or X.shape[0] != self.n:
            raise ValueError("X and Y must both be (n, k)")
        _check(_lib.ehyb_spmm(self._h, int(X.shape[1]), _dev(X, "float64"), _dev(Y, "float64"), _stream(stream)),
               "ehyb_spmm")

    def cg(self, b, x, rtol: float = 1e-10, max_iter: int = 10000, refine: int = 0, inner_rtol: float = 0.0,
           stream=None, raise_not_converged: bool = False):
        """Solve A x = b in place on x (CUDA float64 tensors, original numbering).  Returns (status, info)."""
        info = CgInfo()
        st = ehyb_cg(self._h, _dev(b, "float64"), _dev(x, "float64"), float(rtol), int(max_iter), int(refine),
                     float(inner_rtol), info, _stream(stream))
        if st != 0 and (st != EHYB_ERR_NOT_CONVERGED or raise_not_converged):
            raise EhybError(st, "ehyb_cg")
        return st, info.as_dict()

    def pcg(self, M: "Fsai", b, x, rtol: float = 1e-10, max_iter: int = 10000, stream=None,
            raise_not_converged: bool = False):
        """Preconditioned CG with M (an Fsai of this plan), in place on x (CUDA float64, original numbering)."""
        info = CgInfo()
        st = _lib.ehyb_pcg(self._h, M._h, _dev(b, "float64"), _dev(x, "float64"), float(rtol), int(max_iter),
                           ctypes.byref(info), _stream(stream))
        if st != 0 and (st != EHYB_ERR_NOT_CONVERGED or raise_not_converged):
            raise EhybError(st, "ehyb_pcg")
        return st, info.as_dict()

    def pcg_refined(self, M: "Fsai", b, x, rtol: float = 1e-10, max_iter: int = 10000, inner_rtol: float = 0.0,
                    stream=None, raise_not_converged: bool = False):
        """FP32 PCG with FP64 residual replacement (the plan and M need their low-precision values)."""
        info = CgInfo()
        st = _lib.ehyb_pcg_refined(self._h, M._h, _dev(b, "float64"), _dev(x, "float64"), float(rtol), int(max_iter),
                                   float(inner_rtol), ctypes.byref(info), _stream(stream))
        if st != 0 and (st != EHYB_ERR_NOT_CONVERGED or raise_not_converged):
            raise EhybError(st, "ehyb_pcg_refined")
        return st, info.as_dict()

    def cg_history(self, cap: int = 100000) -> np.ndarray:
        h = np.zeros(cap)
        cnt = ctypes.c_int32(0)
        _check(_lib.ehyb_cg_history(self._h, h.ctypes.data, cap, ctypes.byref(cnt)), "ehyb_cg_history")
        return h[:cnt.value]

    def check(self) -> int:
        return int(ehyb_plan_check(self._h))

    def info(self) -> dict:
        inf = PlanInfo()
        _check(_lib.ehyb_plan_info(self._h, ctypes.byref(inf)), "ehyb_plan_info")
        return inf.as_dict()

    def export(self) -> dict:
        ex = PlanExport()
        _check(_lib.ehyb_plan_export(self._h, ctypes.byref(ex)), "ehyb_plan_export")
        return _export_dict(ex)

    def profile_enable(self, on: bool = True):
        _check(_lib.ehyb_profile_enable(self._h, int(on)), "ehyb_profile_enable")

    def profile_read(self):
        ms, cnt = ctypes.c_double(0), ctypes.c_int64(0)
        _check(_lib.ehyb_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt)), "ehyb_profile_read")
        return ms.value, cnt.value


def _arr(ptr, count, dt):
    if count == 0 or not ptr:
        return np.zeros(count, dt)
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))), (count,)).copy()


def _export_dict(ex: PlanExport) -> dict:
    n, nparts, ns = ex.n, ex.nparts, ex.nslices
    arr = _arr
    low = 1 if (ex.lowp and ex.ell_val_low) else 0   # the lowp copies are exported by host-kept plans only
    return {"n": n, "tpr": ex.tpr, "nparts": nparts,
            "new_to_old": arr(ex.new_to_old, n, np.int32), "part_ptr": arr(ex.part_ptr, nparts + 1, np.int32),
            "slice_ptr": arr(ex.slice_ptr, nparts + 1, np.int32),
            "slice_pos": arr(ex.slice_pos, ns + 1, np.int64),
            "ell_col": arr(ex.ell_col, ex.ell_stored, np.uint16),
            "ell_val": arr(ex.ell_val, ex.ell_stored, np.float64),
            "row_ell_count": arr(ex.row_ell_count, n, np.int32),
            "er_part_ptr": arr(ex.er_part_ptr, nparts + 1, np.int32),
            "er_row": arr(ex.er_row, ex.er_rows, np.int32), "er_ptr": arr(ex.er_ptr, ex.er_rows + 1, np.int64),
            "er_col": arr(ex.er_col, ex.er_nnz, np.int32), "er_val": arr(ex.er_val, ex.er_nnz, np.float64),
            "er_layout": ex.er_layout, "er_slice_pos": arr(ex.er_slice_pos, ns + 1, np.int64),
            "er_scol": arr(ex.er_scol, ex.er_stored if ex.er_layout == 0 else 0, np.int32),
            "er_sval": arr(ex.er_sval, ex.er_stored if ex.er_layout == 0 else 0, np.float64),
            "row_er_count": arr(ex.row_er_count, n, np.int32),
            "lowp": ex.lowp, "lowp_group": ex.lowp_group,
            "ell_val_low": arr(ex.ell_val_low, low * ex.ell_stored, np.float32 if ex.lowp == 1 else np.uint16),
            "ell_col_low": arr(ex.ell_col_low, low * ex.ell_stored, np.uint16),
            "er_sval_low": arr(ex.er_sval_low, low * (ex.er_stored if ex.er_layout == 0 else 0),
                               np.float32 if ex.lowp == 1 else np.uint16),
            "er_scol_low": arr(ex.er_scol_low, low * (ex.er_stored if ex.er_layout == 0 else 0), np.int32),
            "halo_ptr": arr(ex.halo_ptr, nparts + 1, np.int64), "halo_new": arr(ex.halo_new, ex.n_halo, np.int32)}


class Shard:
    """Rank `rank`'s row shard of `plan` among `nranks` (ehyb_shard_*): its partitions, its halo list and the
    exchange lists.  Vectors are device float64 tensors in the plan's numbering: x_local / y_local hold the
    rank's rows, x_ext = [x_local | halo].  Communication is the caller's (see TorchComm)."""

    def __init__(self, plan: "Plan", nranks: int, rank: int, stream=None):
        self._h = ctypes.c_void_p()
        import torch
        # a host-only plan gives a host-only shard, which uploads nothing (no stream needed)
        st = _stream(stream) if (stream is not None or torch.cuda.is_available()) else None
        _check(_lib.ehyb_shard_create(plan.handle, int(nranks), int(rank), st, ctypes.byref(self._h)),
               "ehyb_shard_create")
        i = self.info()
        self.nranks, self.rank = nranks, rank
        self.n_local, self.n_halo, self.send_total = i["n_local"], i["n_halo"], i["send_total"]
        self.row_begin, self.row_end = i["row_begin"], i["row_end"]
        L = self.lists()
        self.send_counts = np.diff(L["send_ptr"]).tolist()
        self.recv_counts = np.diff(L["recv_ptr"]).tolist()

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = ShardInfo()
        _check(_lib.ehyb_shard_info(self._h, ctypes.byref(inf)), "ehyb_shard_info")
        return inf.as_dict()

    def lists(self) -> dict:
        inf = self.info()
        R = inf["nranks"]
        sp, rp = np.zeros(R + 1, np.int64), np.zeros(R + 1, np.int64)
        si, hr = np.zeros(inf["send_total"], np.int32), np.zeros(inf["n_halo"], np.int32)
        _check(_lib.ehyb_shard_lists(self._h, sp.ctypes.data, si.ctypes.data if si.size else None, rp.ctypes.data,
                                     hr.ctypes.data if hr.size else None), "ehyb_shard_lists")
        return {"send_ptr": sp, "send_idx": si, "recv_ptr": rp, "halo_rows": hr}

    def export(self) -> dict:
        ex = PlanExport()
        _check(_lib.ehyb_shard_export(self._h, ctypes.byref(ex)), "ehyb_shard_export")
        return _export_dict(ex)

    def pack(self, x_local, send_buf, stream=None):
        _check(_lib.ehyb_shard_pack(self._h, _dev(x_local, "float64") if self.n_local else None,
                                    _dev(send_buf, "float64") if self.send_total else None, _stream(stream)),
               "ehyb_shard_pack")

    def spmv(self, x_ext, y_local, stream=None):
        _check(_lib.ehyb_shard_spmv(self._h, _dev(x_ext, "float64"), _dev(y_local, "float64"), _stream(stream)),
               "ehyb_shard_spmv")

    def cg(self, b_local, x_local, comm, rtol: float = 1e-10, max_iter: int = 10000, stream=None):
        """Distributed FP64 CG (ehyb_shard_cg), called on every rank with its rows; `comm` supplies
        exchange(shard, send_buf, p_ext) and allreduce(list of floats) -> list.  Returns (status, info)."""
        import torch
        dev = x_local.device
        p_ext = torch.zeros(self.n_local + self.n_halo, dtype=torch.float64, device=dev)
        send = torch.zeros(max(self.send_total, 1), dtype=torch.float64, device=dev)

        def _exchange(ctx, send_ptr, halo_ptr, stream_ptr):
            try:
                comm.exchange(self, send, p_ext)
                return 0
            except Exception:   # noqa: BLE001 -- reported to the library as a failed step
                import traceback
                traceback.print_exc()
                return 1

        def _allreduce(ctx, vals, count):
            try:
                out = comm.allreduce([vals[i] for i in range(count)])
                for i in range(count):
                    vals[i] = float(out[i])
                return 0
            except Exception:   # noqa: BLE001
                import traceback
                traceback.print_exc()
                return 1
        ex_cb, ar_cb = EXCHANGE_FN(_exchange), ALLREDUCE_FN(_allreduce)
        info = CgInfo()
        st = _lib.ehyb_shard_cg(self._h, _dev(b_local, "float64") if self.n_local else None,
                                _dev(x_local, "float64") if self.n_local else None, p_ext.data_ptr(), send.data_ptr(),
                                float(rtol), int(max_iter), ex_cb, ar_cb, None, ctypes.byref(info), _stream(stream))
        if st not in (0, EHYB_ERR_NOT_CONVERGED):
            raise EhybError(st, "ehyb_shard_cg")
        return st, info.as_dict()

    def close(self):
        if self._h:
            _lib.ehyb_shard_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class TorchComm:
    """The two communication steps of the shard path on torch.distributed (NCCL for device tensors, gloo for
    host tensors): the halo exchange as one all_to_all_single with the shard's per-peer counts, and the sum of
    a few scalars as one all_reduce."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group

    def exchange(self, shard: "Shard", send_buf, x_ext):
        import torch
        halo = x_ext[shard.n_local:shard.n_local + shard.n_halo]
        self.dist.all_to_all_single(halo, send_buf[:shard.send_total], output_split_sizes=shard.recv_counts,
                                    input_split_sizes=shard.send_counts, group=self.group)
        if halo.is_cuda:
            torch.cuda.synchronize()

    def allreduce(self, values):
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor(values, dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().tolist()


class Fsai:
    """FSAI preconditioner (M^-1 = G^T G) of a plan's matrix A (the same host CSR the plan was built from)."""

    def __init__(self, plan: "Plan", A, lowp: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        self.plan = plan    # keeps the plan alive as long as the preconditioner
        rp = np.ascontiguousarray(A.row_ptr, np.int64)
        c = np.ascontiguousarray(A.col, np.int32)
        v = np.ascontiguousarray(A.val, np.float64)
        s = None if plan.host_only else _stream(stream)
        _check(_lib.ehyb_fsai_create(plan.handle, int(A.n), int(rp[-1]) if rp.size else 0, rp.ctypes.data,
                                     c.ctypes.data, v.ctypes.data, int(lowp), s, ctypes.byref(self._h)),
               "ehyb_fsai_create")

    def info(self) -> dict:
        nnz, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
        _check(_lib.ehyb_precond_info(self._h, ctypes.byref(nnz), ctypes.byref(ms)), "ehyb_precond_info")
        return {"nnz_g": nnz.value, "setup_ms": ms.value}

    def export(self):
        """G in the plan's numbering as (row_ptr, col, val) numpy copies."""
        n, rp, c, v = ctypes.c_int64(0), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(_lib.ehyb_precond_export(self._h, ctypes.byref(n), ctypes.byref(rp), ctypes.byref(c), ctypes.byref(v)),
               "ehyb_precond_export")
        row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_int64)), (n.value + 1,)).copy()
        nnz = int(row_ptr[-1])
        if nnz == 0:
            return row_ptr, np.zeros(0, np.int32), np.zeros(0)
        col = np.ctypeslib.as_array(ctypes.cast(c, ctypes.POINTER(ctypes.c_int32)), (nnz,)).copy()
        val = np.ctypeslib.as_array(ctypes.cast(v, ctypes.POINTER(ctypes.c_double)), (nnz,)).copy()
        return row_ptr, col, val

    def history(self, cap: int = 100000) -> np.ndarray:
        h = np.zeros(cap)
        cnt = ctypes.c_int32(0)
        _check(_lib.ehyb_pcg_history(self._h, h.ctypes.data, cap, ctypes.byref(cnt)), "ehyb_pcg_history")
        return h[:cnt.value]

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()   # the handle is released whatever the status
            _check(_lib.ehyb_precond_destroy(h), "ehyb_precond_destroy")

    def __del__(self):
        try:
            if self._h:
                _lib.ehyb_precond_destroy(self._h)
        except Exception:
            pass


class CsrBaseline:
    """The plain vector-CSR kernel on the same GPU (tpr lanes per row)."""

    def __init__(self, A, tpr: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        rp = np.ascontiguousarray(A.row_ptr, np.int64)
        c = np.ascontiguousarray(A.col, np.int32)
        v = np.ascontiguousarray(A.val, np.float64)
        _check(_lib.ehyb_csr_create(int(A.n), int(rp[-1]), rp.ctypes.data, c.ctypes.data, v.ctypes.data, tpr,
                                    _stream(stream), ctypes.byref(self._h)), "ehyb_csr_create")
        self.n = int(A.n)

    def set_tpr(self, tpr: int):
        _check(_lib.ehyb_csr_set_tpr(self._h, tpr), "ehyb_csr_set_tpr")

    def spmv(self, x, y, stream=None):
        _check(_lib.ehyb_csr_spmv(self._h, _dev(x, "float64"), _dev(y, "float64"), _stream(stream)),
               "ehyb_csr_spmv")

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()   # the handle is released whatever the status
            _check(_lib.ehyb_csr_destroy(h), "ehyb_csr_destroy")

    def __del__(self):
        try:
            if self._h:
                _lib.ehyb_csr_destroy(self._h)
        except Exception:
            pass


class Batch:
    """Several plans run by one persistent launch (ehyb_batch_*); keeps the plans alive."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        self._h = ctypes.c_void_p()
        _check(_lib.ehyb_batch_create(len(self.plans), arr, ctypes.byref(self._h)), "ehyb_batch_create")

    def spmv(self, xs, ys, stream=None):
        n = len(self.plans)
        xa = (ctypes.c_void_p * n)(*[_dev(x, "float64") for x in xs])
        ya = (ctypes.c_void_p * n)(*[_dev(y, "float64") for y in ys])
        _check(_lib.ehyb_batch_spmv(self._h, xa, ya, _stream(stream)), "ehyb_batch_spmv")

    def info(self) -> dict:
        t, g, th = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(_lib.ehyb_batch_info(self._h, ctypes.byref(t), ctypes.byref(g), ctypes.byref(th)), "ehyb_batch_info")
        return {"tiles": t.value, "grid": g.value, "threads": th.value}

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()   # the handle is released whatever the status
            _check(_lib.ehyb_batch_destroy(h), "ehyb_batch_destroy")

    def __del__(self):
        try:
            if self._h:
                _lib.ehyb_batch_destroy(self._h)
        except Exception:
            pass


# ---------------------------------------------------------------- tuner

def _csr_arrays(A):
    rp = np.ascontiguousarray(A.row_ptr, np.int64)
    c = np.ascontiguousarray(A.col, np.int32)
    v = np.ascontiguousarray(A.val, np.float64)
    return rp, c, v


def features(A, num_sms: int = 152) -> np.ndarray:
    """The tuner's 16 matrix features (ehyb_features)."""
    rp, c, v = _csr_arrays(A)
    out = np.zeros(16, np.float32)
    _check(_lib.ehyb_features(int(A.n), rp.ctypes.data, c.ctypes.data, v.ctypes.data, num_sms, out.ctypes.data),
           "ehyb_features")
    return out


def _table_dicts(tab):
    return [{"slice_rows": e.slice_rows, "ell_width_cap": e.ell_width_cap, "ell_tpr": e.ell_tpr,
             "valid": bool(e.valid), "ms": e.ms} for e in tab]


def tune_grid(A, num_sms: int = 152, smem_optin: int = 232448):
    """The knob configurations of the tuning grid for this matrix (no GPU use)."""
    g = _lib.ehyb_tune_grid_size()
    tab = (TuneEntry * g)()
    rp = np.ascontiguousarray(A.row_ptr, np.int64)
    _check(_lib.ehyb_tune_grid(int(A.n), rp.ctypes.data, num_sms, smem_optin, tab), "ehyb_tune_grid")
    return _table_dicts(tab)


def tune_sweep(A, reps: int = 10, stream=None):
    """Exhaustive sweep: (table of configurations with measured ms, index of the fastest)."""
    g = _lib.ehyb_tune_grid_size()
    tab = (TuneEntry * g)()
    best = ctypes.c_int32(-1)
    rp, c, v = _csr_arrays(A)
    _check(_lib.ehyb_tune_sweep(int(A.n), int(rp[-1]), rp.ctypes.data, c.ctypes.data, v.ctypes.data, reps, tab,
                                ctypes.byref(best), _stream(stream)), "ehyb_tune_sweep")
    return _table_dicts(tab), best.value


def tuner_set_model(params, feat_mean, feat_std, out_mean, out_std):
    """Load the tuner network (numpy float32 arrays) into the library; params=None unloads it."""
    if params is None:
        _check(_lib.ehyb_tuner_set_model(None, None, None, None, None), "ehyb_tuner_set_model")
        return
    arrs = [np.ascontiguousarray(a, np.float32) for a in (params, feat_mean, feat_std, out_mean, out_std)]
    _check(_lib.ehyb_tuner_set_model(*[a.ctypes.data for a in arrs]), "ehyb_tuner_set_model")


def tuner_predict(A):
    """(slice_rows, ell_width_cap, ell_tpr, predicted ns per entry) from the loaded model."""
    rp, c, v = _csr_arrays(A)
    sr, cap, tpr, ns = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
    _check(_lib.ehyb_tuner_predict(int(A.n), int(rp[-1]), rp.ctypes.data, c.ctypes.data, v.ctypes.data,
                                   ctypes.byref(sr), ctypes.byref(cap), ctypes.byref(tpr), ctypes.byref(ns)),
           "ehyb_tuner_predict")
    return sr.value, cap.value, tpr.value, ns.value


class Mlp:
    """Device-side training state of the tuner network, driven through the library's MLP kernels.
    All tensors are torch float32 CUDA tensors."""

    def __init__(self, params):
        import torch
        self.n = int(_lib.ehyb_mlp_param_count())
        self.params = params.to(device="cuda", dtype=torch.float32).contiguous().clone()
        assert self.params.numel() == self.n
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step_no = 0
        self._ws = None

    def _workspace(self, batch):
        import torch
        need = int(_lib.ehyb_mlp_workspace_bytes(batch))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 4), dtype=torch.uint8, device="cuda")
        return self._ws.data_ptr()

    def forward(self, X):
        import torch
        out = torch.empty((X.shape[0], 4), dtype=torch.float32, device="cuda")
        _check(_lib.ehyb_mlp_forward(self.params.data_ptr(), _dev(X, "float32"), X.shape[0], out.data_ptr(),
                                     self._workspace(X.shape[0]), _stream(None)), "ehyb_mlp_forward")
        return out

    def loss_grad(self, X, T):
        _check(_lib.ehyb_mlp_loss_grad(self.params.data_ptr(), _dev(X, "float32"), _dev(T, "float32"), X.shape[0],
                                       self.grad.data_ptr(), self.loss.data_ptr(), self._workspace(X.shape[0]),
                                       _stream(None)), "ehyb_mlp_loss_grad")
        return self.loss, self.grad

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_no += 1
        _check(_lib.ehyb_mlp_adam(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr(),
                                  self.step_no, lr, beta1, beta2, eps, _stream(None)), "ehyb_mlp_adam")
