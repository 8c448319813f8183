"""Thin ctypes binding of the engine's C ABI (``include/spmttkrp.h``).

Argument marshalling only: every step of the computation runs inside the
CUDA library.  Tensors are passed as raw pointers (``data_ptr()``), streams as
``torch.cuda.current_stream().cuda_stream``.  Importing this module never
falls back to anything: if the shared library is missing or fails to load,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

from . import _build

SPM_OK = 0
STATUS = {
    0: "SPM_OK", -1: "SPM_ERR_INVALID_ARG", -2: "SPM_ERR_INDEX_RANGE", -3: "SPM_ERR_DUPLICATE",
    -4: "SPM_ERR_OOM", -5: "SPM_ERR_CUDA", -6: "SPM_ERR_UNSUPPORTED", -7: "SPM_ERR_NOT_SPD",
    -8: "SPM_ERR_STATE", -9: "SPM_ERR_TIMEOUT",
}
DTYPES = {"f32": 0, "bf16": 1}
Q_INFO, Q_NEXT_POS, Q_BOUNDS, Q_SPLITS, Q_ELEMS, Q_VALS, Q_RAW = range(7)
SWEEP_GRAPH = 1

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "spmttkrp.h")


class SpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("factor_dtype", ctypes.c_int), ("partition", ctypes.c_int),
                ("nblk", ctypes.c_int), ("tile", ctypes.c_int),
                ("max_bytes", ctypes.c_size_t), ("checks", ctypes.c_int),
                ("host_only", ctypes.c_int), ("variant", ctypes.c_int),
                ("unroll", ctypes.c_int), ("stages", ctypes.c_int),
                ("element_bytes", ctypes.c_int),
                ("cache_hints", ctypes.c_int),
                ("stream", ctypes.c_void_p),
                ("keep_base", ctypes.c_int),
                ("plan_on_host", ctypes.c_int),
                ("wait_limit_ns", ctypes.c_int64),
                ("inject_wait_stall", ctypes.c_int)]


_LIB = None
P = ctypes.c_void_p
I64P = ctypes.POINTER(ctypes.c_int64)


def declared_functions():
    """Names of the functions ``include/spmttkrp.h`` declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", text, flags=re.M)))


def lib():
    """Loads the engine library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"engine library missing ({_build.LIB}); run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    L.spmttkrp_version.restype = ctypes.c_int
    L.spmttkrp_last_error.restype = ctypes.c_char_p
    L.spmttkrp_opts_init.argtypes = [ctypes.POINTER(Opts)]
    L.spmttkrp_plan_create.argtypes = [ctypes.POINTER(P), P, P, ctypes.c_int64, I64P,
                                       ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts)]
    L.spmttkrp_plan_destroy.argtypes = [P]
    L.spmttkrp_set_stream.argtypes = [P, P]
    L.spmttkrp_remap.argtypes = [P, ctypes.c_int]
    L.spmttkrp_compute.argtypes = [P, ctypes.c_int, P, P]
    L.spmttkrp_compute_ex.argtypes = [P, ctypes.c_int, P, P, ctypes.c_int]
    L.spmttkrp_sweep.argtypes = [P, P, P, ctypes.c_int]
    L.cp_als_iter.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double)]
    L.cp_als_run.argtypes = [P, P, P, ctypes.c_int, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.cp_loss_fwd.argtypes = [P, P, P]
    L.cp_loss_fwd_ex.argtypes = [P, P, P, ctypes.c_int]
    L.cp_loss_bwd.argtypes = [P, P, P, P]
    L.spmttkrp_autotune.argtypes = [P, P, P, ctypes.c_int]
    L.spmttkrp_plan_query.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t]
    L.spmttkrp_device_status.argtypes = [P]
    L.spmttkrp_check_elements.argtypes = [P, ctypes.c_int64, ctypes.c_int, I64P, ctypes.c_int,
                                          P, ctypes.c_int, P]
    L.spmttkrp_plan_check.argtypes = [P]
    L.spmttkrp_memprobe.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, ctypes.c_int, P]
    for name in declared_functions():
        getattr(L, name).restype = ctypes.c_char_p if name == "spmttkrp_last_error" \
            else ctypes.c_int
    _LIB = L
    return L


def check(status: int):
    if status != SPM_OK:
        raise SpmError(status, lib().spmttkrp_last_error().decode(errors="replace"))


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else ctypes.c_void_p(t.data_ptr())
    return arr


def _stream_ptr(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream) if hasattr(stream, "cuda_stream") \
        else ctypes.c_void_p(stream)


def memprobe(kind: int, src, dst, n: int, run: int = 1, stream=None):
    """Queues one memory-probe kernel (0 copy, 1 scatter, 2 gather of 32-byte
    records; see spmttkrp_memprobe) on `stream` (default: torch's current)."""
    check(lib().spmttkrp_memprobe(int(kind), ctypes.c_void_p(src.data_ptr()),
                                  ctypes.c_void_p(dst.data_ptr()), int(n), int(run),
                                  _stream_ptr(stream)))


def check_elements(elems, nnz: int, dims, elem_bytes: int, next_pos=None, alpha_word: int = 0,
                   stream=None):
    """Device check of a working copy held in a CUDA tensor `elems` (nnz records of
    elem_bytes: int32 indices, float value, padding).  `next_pos` is an int32 CUDA tensor
    or None; `alpha_word` the word index of a carried remap id (0 = none).  Raises
    SpmError (INDEX_RANGE or STATE) on a violation."""
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    check(lib().spmttkrp_check_elements(
        ctypes.c_void_p(elems.data_ptr()), int(nnz), len(d),
        d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(elem_bytes),
        None if next_pos is None else ctypes.c_void_p(next_pos.data_ptr()), int(alpha_word),
        _stream_ptr(stream)))


class Plan:
    """One COO tensor prepared for all-mode spMTTKRP on the current CUDA device."""

    def __init__(self, coo, vals, dims: Sequence[int], rank: int, dtype: str = "f32",
                 nblk: int = 0, tile: int = 0, max_bytes: int = 0, checks: bool = False,
                 host_only: bool = False, stream=None, variant: int = 0, unroll: int = 0,
                 cache_hints: int = 0, stages: int = 0, element_bytes: int = 0,
                 keep_base: bool = False, partition: int = 0, plan_on_host: bool = False,
                 wait_limit_ns: int = 0, inject_wait_stall: bool = False):
        L = lib()
        coo = np.ascontiguousarray(np.asarray(coo.cpu() if hasattr(coo, "cpu") else coo,
                                              dtype=np.int64))
        vals = np.ascontiguousarray(np.asarray(vals.cpu() if hasattr(vals, "cpu") else vals,
                                               dtype=np.float32))
        self.dims = tuple(int(d) for d in dims)
        self.nmodes = len(self.dims)
        self.rank = int(rank)
        self.nnz = int(vals.shape[0])
        self.dtype = dtype
        o = Opts()
        L.spmttkrp_opts_init(ctypes.byref(o))
        o.factor_dtype = DTYPES[dtype]
        o.nblk, o.tile, o.max_bytes = int(nblk), int(tile), int(max_bytes)
        o.checks, o.host_only = int(bool(checks)), int(bool(host_only))
        o.variant = int(variant)
        o.unroll, o.cache_hints, o.stages = int(unroll), int(cache_hints), int(stages)
        o.element_bytes = int(element_bytes)
        o.keep_base = int(bool(keep_base))
        o.partition = int(partition)
        o.plan_on_host = int(bool(plan_on_host))
        o.wait_limit_ns = int(wait_limit_ns)
        o.inject_wait_stall = int(bool(inject_wait_stall))
        # without an explicit stream the plan follows torch's current stream at
        # every call (so its work is ordered with the caller's tensors)
        self._follow = stream is None and not host_only
        o.stream = None if host_only else _stream_ptr(stream)
        self._stream = None if host_only else o.stream
        d = np.asarray(self.dims, dtype=np.int64)
        h = ctypes.c_void_p()
        st = L.spmttkrp_plan_create(ctypes.byref(h),
                                    coo.ctypes.data if coo.size else None,
                                    vals.ctypes.data if vals.size else None,
                                    self.nnz, d.ctypes.data_as(I64P), self.nmodes, self.rank,
                                    ctypes.byref(o))
        check(st)
        self._h = h
        self._device = None
        if not host_only:
            import torch
            if torch.cuda.is_available():
                self._device = torch.cuda.current_device()
        self.loss_generation = 0  # bumped by every cp_loss_fwd / cp_loss_bwd

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            check(lib().spmttkrp_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._follow = False
        self._stream = _stream_ptr(stream)
        check(lib().spmttkrp_set_stream(self._h, self._stream))

    # -- argument checks (before any pointer reaches the C ABI)
    def _sync_stream(self):
        if not self._follow:
            return
        import torch
        cur = torch.cuda.current_stream().cuda_stream
        if self._stream is None or self._stream.value != cur:
            self._stream = ctypes.c_void_p(cur)
            check(lib().spmttkrp_set_stream(self._h, self._stream))

    def _check_tensor(self, t, rows, what, dtype=None):
        import torch
        want = dtype or (torch.bfloat16 if self.dtype == "bf16" else torch.float32)
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{what}: expected a torch.Tensor")
        if not t.is_cuda or (self._device is not None and t.device.index != self._device):
            raise ValueError(f"{what}: must be on the plan's CUDA device")
        if t.dtype != want:
            raise ValueError(f"{what}: dtype {t.dtype}, the plan needs {want}")
        if tuple(t.shape) != (rows, self.rank):
            raise ValueError(f"{what}: shape {tuple(t.shape)}, expected {(rows, self.rank)}")
        if not t.is_contiguous():
            raise ValueError(f"{what}: must be contiguous (row-major I x R)")

    def _check_factors(self, factors, skip=-1):
        if len(factors) != self.nmodes:
            raise ValueError(f"expected {self.nmodes} factors, got {len(factors)}")
        for k, f in enumerate(factors):
            if k != skip:
                self._check_tensor(f, self.dims[k], f"factor {k}")

    def _check_outs(self, outs, what="output"):
        import torch
        if len(outs) != self.nmodes:
            raise ValueError(f"expected {self.nmodes} {what}s, got {len(outs)}")
        for k, o in enumerate(outs):
            self._check_tensor(o, self.dims[k], f"{what} {k}", torch.float32)

    # -- compute
    def remap(self, mode: int):
        self._sync_stream()
        check(lib().spmttkrp_remap(self._h, int(mode)))

    def compute(self, mode: int, factors, out, keep_order: bool = False):
        """Mode-n spMTTKRP into out; with keep_order the pass writes no remap and the
        working copy stays in mode-n order."""
        import torch
        self._check_factors(factors, skip=int(mode))
        self._check_tensor(out, self.dims[int(mode)], "out", torch.float32)
        self._sync_stream()
        if keep_order:
            check(lib().spmttkrp_compute_ex(self._h, int(mode), _ptrs(factors),
                                            ctypes.c_void_p(out.data_ptr()), 1))
            return
        check(lib().spmttkrp_compute(self._h, int(mode), _ptrs(factors),
                                     ctypes.c_void_p(out.data_ptr())))

    def sweep(self, factors, outs, graph: bool = False):
        self._check_factors(factors)
        self._check_outs(outs)
        self._sync_stream()
        check(lib().spmttkrp_sweep(self._h, _ptrs(factors), _ptrs(outs),
                                   SWEEP_GRAPH if graph else 0))

    def als_iter(self, factors, lam) -> float:
        import torch
        self._check_factors(factors)
        if lam.dtype != torch.float32 or lam.numel() != self.rank or not lam.is_contiguous():
            raise ValueError("lambda: contiguous float32 tensor of rank elements")
        self._sync_stream()
        fit = ctypes.c_double()
        check(lib().cp_als_iter(self._h, _ptrs(factors), ctypes.c_void_p(lam.data_ptr()),
                                ctypes.byref(fit)))
        return fit.value

    def als_run(self, factors, lam, max_iters: int, tol: float = 0.0) -> list:
        """Up to max_iters CP-ALS iterations in one graph launch, stopping on the
        device when the fit changes by less than tol; returns the fits."""
        import torch
        self._check_factors(factors)
        if lam.dtype != torch.float32 or lam.numel() != self.rank or not lam.is_contiguous():
            raise ValueError("lambda: contiguous float32 tensor of rank elements")
        self._sync_stream()
        fits = (ctypes.c_double * int(max_iters))()
        n = ctypes.c_int()
        check(lib().cp_als_run(self._h, _ptrs(factors), ctypes.c_void_p(lam.data_ptr()),
                               int(max_iters), float(tol), fits, ctypes.byref(n)))
        return [fits[i] for i in range(n.value)]

    def loss_fwd(self, factors, loss, forward_only: bool = False):
        """CP-loss forward; its residuals (and, for fused plans, the gradient of the
        current mode) stay in the plan for the next loss_bwd.  forward_only runs
        the plain forward pass.  Returns the plan's loss generation, which this
        call advances."""
        import torch
        self._check_factors(factors)
        if loss.dtype != torch.float32 or loss.numel() != 1:
            raise ValueError("loss: float32 scalar tensor")
        self._sync_stream()
        check(lib().cp_loss_fwd_ex(self._h, _ptrs(factors), ctypes.c_void_p(loss.data_ptr()),
                                   1 if forward_only else 0))
        self.loss_generation += 1
        return self.loss_generation

    def loss_bwd(self, factors, grad_out, grads):
        """CP-loss gradients from the residuals of the last loss_fwd (which this
        call consumes, advancing the loss generation)."""
        import torch
        self._check_factors(factors)
        self._check_outs(grads, "gradient")
        if grad_out.dtype != torch.float32 or grad_out.numel() != 1:
            raise ValueError("grad_out: float32 scalar tensor")
        self._sync_stream()
        try:
            check(lib().cp_loss_bwd(self._h, _ptrs(factors),
                                    ctypes.c_void_p(grad_out.data_ptr()), _ptrs(grads)))
        finally:
            self.loss_generation += 1

    def autotune(self, factors, scratch, ignore_cache: bool = False):
        self._check_factors(factors)
        self._check_outs(scratch, "scratch")
        self._sync_stream()
        check(lib().spmttkrp_autotune(self._h, _ptrs(factors), _ptrs(scratch),
                                      1 if ignore_cache else 0))

    def device_status(self):
        check(lib().spmttkrp_device_status(self._h))

    def check(self):
        """Device check of the working copy: indices in range, next_pos a permutation,
        carried remap ids equal to next_pos.  Raises SpmError on a violation."""
        check(lib().spmttkrp_plan_check(self._h))

    # -- queries
    def info(self, mode: int = 0) -> dict:
        buf = np.zeros(16, dtype=np.int64)
        check(lib().spmttkrp_plan_query(self._h, Q_INFO, int(mode), buf.ctypes.data, buf.nbytes))
        keys = ["nnz", "nmodes", "rank", "elem_bytes", "cur_mode", "dtype", "tile", "nblk",
                "nsplit", "launches_per_sweep", "device_bytes", "cur_buf", "host_only",
                "num_sms", "normx2", "lanes"]
        d = dict(zip(keys, buf.tolist()))
        d["normx2"] = float(buf[14:15].view(np.float64)[0])
        flags = d["host_only"]
        d["host_only"], d["variant"], d["keep_base"] = flags & 1, (flags >> 8) & 3, (flags >> 2) & 1
        d["write_orders"] = (flags >> 10) & 1
        d["hot_rows"] = (flags >> 11) & 0x1FFFFF
        d["stages"] = (flags >> 3) & 7
        d["partition"] = (flags >> 6) & 1
        d["remap_ids_in_elements"] = (flags >> 7) & 1
        return d

    def next_pos(self, mode: int) -> np.ndarray:
        out = np.zeros(self.nnz, dtype=np.int32)
        check(lib().spmttkrp_plan_query(self._h, Q_NEXT_POS, int(mode), out.ctypes.data,
                                        out.nbytes))
        return out

    def bounds(self, mode: int) -> np.ndarray:
        nblk = self.info(mode)["nblk"]
        out = np.zeros(nblk + 1, dtype=np.int64)
        check(lib().spmttkrp_plan_query(self._h, Q_BOUNDS, int(mode), out.ctypes.data,
                                        out.nbytes))
        return out

    def splits(self, mode: int) -> np.ndarray:
        ns = self.info(mode)["nsplit"]
        out = np.zeros((ns, 3), dtype=np.int64)
        check(lib().spmttkrp_plan_query(self._h, Q_SPLITS, int(mode),
                                        out.ctypes.data if ns else
                                        np.zeros(1, np.int64).ctypes.data, max(out.nbytes, 8)))
        return out

    def raw_elements(self) -> np.ndarray:
        """Stored nonzeros of the working copy as int32 words [nnz, elem_bytes / 4]."""
        es = self.info()["elem_bytes"]
        out = np.zeros((self.nnz, es // 4), dtype=np.int32)
        if self.nnz:
            check(lib().spmttkrp_plan_query(self._h, Q_RAW, 0, out.ctypes.data, out.nbytes))
        return out

    def elements(self):
        """Working copy (indices int32 [nnz, N], values float32 [nnz]) in its current order."""
        idx = np.zeros((self.nnz, self.nmodes), dtype=np.int32)
        val = np.zeros(self.nnz, dtype=np.float32)
        if self.nnz:
            check(lib().spmttkrp_plan_query(self._h, Q_ELEMS, 0, idx.ctypes.data, idx.nbytes))
            check(lib().spmttkrp_plan_query(self._h, Q_VALS, 0, val.ctypes.data, val.nbytes))
        return idx, val
