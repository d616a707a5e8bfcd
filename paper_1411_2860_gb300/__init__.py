"""Projection-based GEMM and 1-D cross-correlation on GB300 (sm_103a).

Python binding of ``libprojgemm.so`` (C ABI in ``include/projgemm.h``).  This
module only marshals arguments: torch supplies device memory and streams,
every step of the computation runs in the library's CUDA kernels.  There is
no CPU fallback: without the built library (``build()``) or without an
sm_103a GPU, calls raise.

The method follows Anam, Whatmough and Andreopoulos (IEEE TCSVT 2014):
inner-dimension blocks are projected group by group (groups of L values, an
invertible L x L matrix C and D = C^-1, Sec. III-A/B), only the first l+1
projections are kept (Eq. 8), and the reduced products are accumulated.
R = (l+1) * block / L components per block; R = block is exact.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

from . import _build

__all__ = [
    "build", "lib_path", "select_library", "library_variant", "ProjError", "proj_gemm", "proj_gemm_project",
    "proj_gemm_multiply", "proj_gemm_fused",
    "proj_conv", "proj_conv_project", "proj_conv_correlate", "gemm_workspace_size",
    "conv_workspace_size", "basis_build", "check", "exported_symbols", "proj_gemm_backward",
    "proj_gemm_backward_saved", "ProjGemmFn",
    "gemm_backward_workspace_size",
    "proj_matmul", "BatchPlan", "batch_gemm", "batch_conv", "autotune_cached_product", "proj_gemm_cached",
]

PJ_OK, PJ_EINVAL, PJ_EUNSUPPORTED, PJ_ENOMEM, PJ_ECUDA, PJ_ETIMEOUT = range(6)
PJ_F64, PJ_F32, PJ_BF16, PJ_E4M3 = range(4)
BASIS = {"dct2": 0, "haar": 1, "user": 2}
_DT = {torch.float64: PJ_F64, torch.float32: PJ_F32, torch.bfloat16: PJ_BF16}
_COMPUTE = {"f64": PJ_F64, "bf16": PJ_BF16, "e4m3": PJ_E4M3}
_STATUS = {PJ_EINVAL: "EINVAL", PJ_EUNSUPPORTED: "EUNSUPPORTED", PJ_ENOMEM: "ENOMEM", PJ_ECUDA: "ECUDA",
           PJ_ETIMEOUT: "ETIMEOUT"}

_lock = threading.Lock()
_lib = None


class ProjError(RuntimeError):
    """A library call returned a non-zero pj_status."""

    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Basis(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("L", ctypes.c_int32), ("user_C", ctypes.POINTER(ctypes.c_double))]


class _Prec(ctypes.Structure):
    _fields_ = [("compute", ctypes.c_int32), ("split_terms", ctypes.c_int32), ("split_lead", ctypes.c_int32),
                ("fp8_tier", ctypes.c_int32)]


class _BatchDesc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("in_dtype", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("ldb", ctypes.c_int64), ("ldy", ctypes.c_int64), ("block", ctypes.c_int64), ("R", ctypes.c_int64),
                ("basis", _Basis), ("prec", _Prec)]


class _Tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("max_split", ctypes.c_int32),
                ("solo", ctypes.c_int32), ("us_per_tile", ctypes.c_double), ("us_per_stage", ctypes.c_double),
                ("us_per_out_kb", ctypes.c_double)]


class _Report(ctypes.Structure):
    _fields_ = [("alg_flops", ctypes.c_double), ("alg_bytes", ctypes.c_double), ("norm_A", ctypes.c_double),
                ("norm_B", ctypes.c_double), ("trunc_bound", ctypes.c_double), ("round_bound", ctypes.c_double)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("gemm_tiles", ctypes.c_int32), ("mx_tiles", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("split_instances", ctypes.c_int32), ("model_makespan_us", ctypes.c_double),
                ("model_total_us", ctypes.c_double)]


TUNING_KEYS = ("schedule", "tile_rows", "max_split", "solo", "us_per_tile", "us_per_stage", "us_per_out_kb")


def _tuning(t):
    if t is None:
        return None
    unknown = set(t) - set(TUNING_KEYS)
    if unknown:
        raise ValueError(f"unknown tuning keys {sorted(unknown)}")
    return _Tuning(int(t.get("schedule", 0)), int(t.get("tile_rows", 0)), int(t.get("max_split", 0)),
                   int(t.get("solo", 0)),
                   float(t.get("us_per_tile", 0.0)), float(t.get("us_per_stage", 0.0)),
                   float(t.get("us_per_out_kb", 0.0)))


_variant = "pairs"


def select_library(variant: str) -> None:
    """Choose the library build this process loads, before its first call.

    "pairs" (default): the one-GPU build, whose reduced GEMMs may run on
    clusters of two CTAs sharing operand tiles by cluster multicast.
    "solo": the same library compiled without any multicast form; a process
    that runs one of several GPUs (one process per GPU) must load this one."""
    global _variant
    if variant not in _build.VARIANTS:
        raise ValueError(f"unknown library variant {variant!r} (one of {sorted(_build.VARIANTS)})")
    with _lock:
        if _lib is not None and variant != _variant:
            raise RuntimeError(f"library variant {_variant!r} is already loaded in this process")
        _variant = variant


def library_variant() -> str:
    return _variant


def build(force: bool = False) -> str:
    """Compile the selected variant of libprojgemm for sm_103a (in-tree) and return its path."""
    return _build.build(force=force, variant=_variant)


def lib_path() -> str:
    return _build.lib_path(_variant)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.lib_path(_variant)
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} is not built; call paper_1411_2860_gb300.build() first")
        lib = ctypes.CDLL(path)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
        B, P = ctypes.POINTER(_Basis), ctypes.POINTER(_Prec)
        sig = {
            "pj_last_error": ([], ctypes.c_char_p),
            "pj_version": ([], ctypes.c_char_p),
            "pj_check": ([vp, vp], ctypes.c_int),
            "pj_basis_build": ([B, i32, vp, vp, vp, sz, vp], ctypes.c_int),
            "proj_gemm_workspace_size": ([i64, i64, i64, i64, i64, B, P], sz),
            "proj_gemm": ([vp, i64, vp, i64, vp, i64, i64, i64, i64, i32, i32, i64, i64, B, P, vp, sz, vp],
                          ctypes.c_int),
            "proj_gemm_project": ([vp, i64, vp, i64, i64, i64, i64, i32, i64, i64, B, P, vp, sz, vp], ctypes.c_int),
            "proj_gemm_multiply": ([vp, i64, i64, i64, i64, i32, i64, i64, B, P, vp, sz, vp], ctypes.c_int),
            "proj_gemm_fused": ([vp, i64, vp, i64, i64, i64, i64, i32, i32, i64, i64, B, P, vp, sz, vp],
                                ctypes.c_int),
            "proj_gemm_backward_workspace_size": ([i64, i64, i64, i64, i64, B, P], sz),
            "proj_gemm_backward_saved": ([vp, sz, vp, i64, vp, i64, vp, i64, i64, i64, i64, i32, i32, i64, i64, B, P,
                                          vp, sz, vp], ctypes.c_int),
            "proj_gemm_backward": ([vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, i64, i64, i64, i32, i32, i64, i64,
                                    B, P, vp, sz, vp], ctypes.c_int),
            "proj_conv_workspace_size": ([i64, i64, i64, i64, i64, B, P], sz),
            "proj_conv": ([vp, i64, vp, i64, i64, vp, i32, i32, i64, i64, B, P, vp, sz, vp], ctypes.c_int),
            "proj_conv_interp": ([vp, i64, vp, i64, i64, vp, i32, i32, i64, i64, B, P, i32, vp, sz, vp],
                                 ctypes.c_int),
            "proj_conv_host_workspace_size": ([i64, i64, i64, i64, i64, B, P, i32], sz),
            "proj_conv_host": ([vp, i64, vp, i64, i64, vp, i32, i32, i64, i64, B, P, i32, vp, sz, vp],
                               ctypes.c_int),
            "proj_conv_project": ([vp, i64, vp, i64, i64, i32, i64, i64, B, P, vp, sz, vp], ctypes.c_int),
            "proj_conv_correlate": ([i64, i64, i64, vp, i32, i64, i64, B, P, vp, sz, vp], ctypes.c_int),
            "proj_batch_workspace_size": ([ctypes.POINTER(_BatchDesc), i32], sz),
            "proj_batch_plan_create": ([ctypes.POINTER(_BatchDesc), i32, vp, sz, vp, ctypes.POINTER(vp)],
                                       ctypes.c_int),
            "proj_batch_workspace_size_tuned": ([ctypes.POINTER(_BatchDesc), i32, ctypes.POINTER(_Tuning)], sz),
            "proj_batch_plan_create_tuned": ([ctypes.POINTER(_BatchDesc), i32, ctypes.POINTER(_Tuning), vp, sz, vp,
                                              ctypes.POINTER(vp)], ctypes.c_int),
            "proj_batch_plan_info": ([vp, ctypes.POINTER(_BatchInfo)], ctypes.c_int),
            "proj_batch_run": ([vp, vp], ctypes.c_int),
            "proj_batch_destroy": ([vp], None),
            "proj_gemm_report_workspace_size": ([i64, i64], sz),
            "proj_gemm_report": ([vp, i64, vp, i64, i64, i64, i64, i32, i32, i64, i64, B, P, vp, sz, vp,
                                  ctypes.POINTER(_Report)], ctypes.c_int),
            "pj_selftest_workspace_size": ([], sz),
            "pj_selftest_timeout": ([i32, vp, sz, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols() -> list:
    """Function names declared in include/*.h (the C ABI)."""
    inc = os.path.join(os.path.dirname(_build.HERE), "include")
    names = []
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z][a-z0-9_]*)\s*\(", txt, re.M)
    return sorted(set(names))


def last_error() -> str:
    return _load().pj_last_error().decode()


def version() -> str:
    return _load().pj_version().decode()


def _check(st: int, where: str):
    if st != PJ_OK:
        raise ProjError(st, where, last_error())


def _basis(kind: str, L: int, user_C=None, holder=None):
    """pj_basis for the C ABI.  A user matrix is copied to a host tensor that the
    library reads when the stream runs the call (at every replay of a captured
    graph), so it is kept alive on `holder` (the call's workspace) when given."""
    keep = None
    b = _Basis(BASIS[kind], int(L), None)
    if kind == "user":
        if user_C is None:
            raise ValueError("basis 'user' needs user_C")
        keep = torch.as_tensor(user_C, dtype=torch.float64).contiguous().cpu().clone()
        b.user_C = ctypes.cast(keep.data_ptr(), ctypes.POINTER(ctypes.c_double))
        if holder is not None:
            kept = getattr(holder, "_pj_user_bases", None)
            if kept is None:
                kept = []
                holder._pj_user_bases = kept
            kept.append(keep)
    return b, keep


def _prec(compute: str, split: int, split_lead: int = 0, fp8_tier: int = 0):
    return _Prec(_COMPUTE[compute], int(split), int(split_lead), int(fp8_tier))


def _stream(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _workspace(nbytes: int, device, workspace=None):
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError(f"workspace too small: {workspace.numel()} < {nbytes} bytes")
        return workspace
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def gemm_workspace_size(M, N, K, block_k, R, basis="dct2", L=8, compute="bf16", split=1, user_C=None,
                        split_lead: int = 0, fp8_tier: int = 0) -> int:
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, split, split_lead, fp8_tier)
    n = _load().proj_gemm_workspace_size(M, N, K, block_k, R, ctypes.byref(b), ctypes.byref(p))
    if n == 0:
        raise ProjError(PJ_EINVAL, "proj_gemm_workspace_size", last_error())
    return int(n)


def _rows(t):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit stride in its last dimension")
    return t.stride(0)


def gemm_backward_workspace_size(M, N, K, block_k, R, basis="dct2", L=8, compute="bf16", user_C=None) -> int:
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, 1)
    n = _load().proj_gemm_backward_workspace_size(M, N, K, block_k, R, ctypes.byref(b), ctypes.byref(p))
    if n == 0:
        raise ProjError(PJ_EINVAL, "proj_gemm_backward_workspace_size", last_error())
    return n


def proj_gemm(A, B, block_k: int, R: int, basis: str = "dct2", L: int = 8, compute: str | None = None,
              split: int = 1, out_dtype=None, user_C=None, out=None, workspace=None, stream=None,
              split_lead: int = 0, fp8_tier: int = 0):
    """Y = projected product of A (M x K) and B (K x N), R components per block of block_k.

    CUDA tensors run on their device; CPU tensors are copied to the current
    device (pinned when possible), computed there and copied back.
    compute: "f64" (float64 inputs), "bf16" or "e4m3" (float32 / bfloat16 inputs); None picks
    "f64" for float64 inputs and "bf16" otherwise.  split = 2 adds the lo terms (hi*lo + lo*hi);
    split_lead = t keeps them on the first t projections of every group only.
    fp8_tier = n adds the next n projections of every group (p = l+1 .. l+n) in E4M3 with
    per-32 block scales, on top of the BF16 product (FP32 output).
    """
    host = A.device.type == "cpu"
    if host:
        dev = torch.device("cuda", torch.cuda.current_device())
        A_d = A.to(dev, non_blocking=True)
        B_d = B.to(dev, non_blocking=True)
        Y = proj_gemm(A_d, B_d, block_k, R, basis, L, compute, split, out_dtype, user_C, None, workspace, stream,
                      split_lead, fp8_tier)
        return Y.to("cpu", non_blocking=False) if out is None else out.copy_(Y)
    if compute is None:
        compute = "f64" if A.dtype == torch.float64 else "bf16"
    if out_dtype is None:
        out_dtype = torch.float64 if compute == "f64" else torch.float32
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError(f"inner dimensions differ: {K} vs {K2}")
    if B.dtype != A.dtype:
        raise ValueError("A and B must share a dtype")
    lda, ldb = _rows(A), _rows(B)
    if out is None:
        out = torch.empty((M, N), dtype=out_dtype, device=A.device)
    ldy = _rows(out)
    b, _keep = _basis(basis, L, user_C, workspace)
    p = _prec(compute, split, split_lead, fp8_tier)
    lib = _load()
    nbytes = lib.proj_gemm_workspace_size(M, N, K, block_k, R, ctypes.byref(b), ctypes.byref(p))
    if nbytes == 0:
        raise ProjError(PJ_EINVAL, "proj_gemm", last_error())
    ws = _workspace(nbytes, A.device, workspace)
    with torch.cuda.device(A.device):
        st = lib.proj_gemm(_ptr(A), lda, _ptr(B), ldb, _ptr(out), ldy, M, N, K, _DT[A.dtype], _DT[out.dtype],
                           block_k, R, ctypes.byref(b), ctypes.byref(p), _ptr(ws), ws.numel(),
                           _stream(stream, A.device))
    _check(st, "proj_gemm")
    return out


def proj_gemm_project(A, B, block_k: int, R: int, workspace, basis="dct2", L=8, compute="bf16", split=1,
                      user_C=None, stream=None, M=None, N=None, K=None, split_lead: int = 0, fp8_tier: int = 0):
    """Stage 1 of proj_gemm: project A and/or B (None keeps the workspace copy)."""
    lib = _load()
    if A is not None:
        M, K = A.shape
    if B is not None:
        K, N = B.shape
    dtype = (A if A is not None else B).dtype
    dev = (A if A is not None else B).device
    b, _keep = _basis(basis, L, user_C, workspace)
    p = _prec(compute, split, split_lead, fp8_tier)
    st = lib.proj_gemm_project(_ptr(A), _rows(A) if A is not None else 0, _ptr(B), _rows(B) if B is not None else 0,
                               M, N, K, _DT[dtype], block_k, R, ctypes.byref(b), ctypes.byref(p), _ptr(workspace),
                               workspace.numel(), _stream(stream, dev))
    _check(st, "proj_gemm_project")


def proj_gemm_multiply(out, K: int, block_k: int, R: int, workspace, basis="dct2", L=8, compute="bf16", split=1,
                       user_C=None, stream=None, split_lead: int = 0, fp8_tier: int = 0):
    """Stage 2 of proj_gemm: Y from the projected operands in the workspace."""
    lib = _load()
    M, N = out.shape
    b, _keep = _basis(basis, L, user_C, workspace)
    p = _prec(compute, split, split_lead, fp8_tier)
    st = lib.proj_gemm_multiply(_ptr(out), _rows(out), M, N, K, _DT[out.dtype], block_k, R, ctypes.byref(b),
                                ctypes.byref(p), _ptr(workspace), workspace.numel(), _stream(stream, out.device))
    _check(st, "proj_gemm_multiply")
    return out


def proj_gemm_fused(A, out, block_k: int, R: int, workspace, basis="dct2", L=8, split=1, user_C=None,
                    stream=None):
    """out = (A projected inside the GEMM kernel) x B_d, with B_d already projected into
    `workspace` by proj_gemm_project(None, B, ...).  L = 8 and R = block_k only; plain or
    fully split BF16 components."""
    lib = _load()
    M, K = A.shape
    N = out.shape[1]
    b, _keep = _basis(basis, L, user_C, workspace)
    p = _prec("bf16", split)
    st = lib.proj_gemm_fused(_ptr(A), _rows(A), _ptr(out), _rows(out), M, N, K, _DT[A.dtype], _DT[out.dtype],
                             block_k, R, ctypes.byref(b), ctypes.byref(p), _ptr(workspace), workspace.numel(),
                             _stream(stream, A.device))
    _check(st, "proj_gemm_fused")
    return out


def proj_gemm_backward(A, B, dY, block_k: int, R: int, basis: str = "dct2", L: int = 8,
                       compute: str | None = None, out_dtype=None, user_C=None, workspace=None, stream=None,
                       dA=None, dB=None):
    """(dA, dB) of sum(dY * Y) for Y = proj_gemm(A, B): dA = expand_C(dY B_d^T), dB = expand_D(A_c^T dY).

    The projected operands are recomputed from A and B.  dY is taken in A's dtype.
    dA (M x K) and dB (K x N) may be given (any row pitch, unit column stride).
    """
    if compute is None:
        compute = "f64" if A.dtype == torch.float64 else "bf16"
    if out_dtype is None:
        out_dtype = A.dtype
    M, K = A.shape
    N = B.shape[1]
    dY = dY.to(A.dtype).contiguous()
    if dA is None:
        dA = torch.empty((M, K), dtype=out_dtype, device=A.device)
    if dB is None:
        dB = torch.empty((K, N), dtype=out_dtype, device=A.device)
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, 1)
    lib = _load()
    nbytes = lib.proj_gemm_backward_workspace_size(M, N, K, block_k, R, ctypes.byref(b), ctypes.byref(p))
    if nbytes == 0:
        raise ProjError(PJ_EINVAL, "proj_gemm_backward", last_error())
    ws = _workspace(nbytes, A.device, workspace)
    with torch.cuda.device(A.device):
        st = lib.proj_gemm_backward(_ptr(A), _rows(A), _ptr(B), _rows(B), _ptr(dY), _rows(dY), _ptr(dA), _rows(dA),
                                    _ptr(dB), _rows(dB), M, N, K, _DT[A.dtype], _DT[out_dtype], block_k, R,
                                    ctypes.byref(b), ctypes.byref(p), _ptr(ws), ws.numel(),
                                    _stream(stream, A.device))
    _check(st, "proj_gemm_backward")
    return dA, dB


def proj_gemm_backward_saved(fwd_workspace, dY, K: int, block_k: int, R: int, basis: str = "dct2", L: int = 8,
                             compute: str = "bf16", out_dtype=None, user_C=None, workspace=None, stream=None,
                             dA=None, dB=None):
    """(dA, dB) as proj_gemm_backward, from the A_c and B_d that a forward call
    (proj_gemm with split = 1, or proj_gemm_project of both operands) left in
    `fwd_workspace` for the same M = dY.shape[0], N = dY.shape[1], K, block_k, R,
    basis and compute; A and B are not needed."""
    M, N = dY.shape
    if out_dtype is None:
        out_dtype = dY.dtype
    if dA is None:
        dA = torch.empty((M, K), dtype=out_dtype, device=dY.device)
    if dB is None:
        dB = torch.empty((K, N), dtype=out_dtype, device=dY.device)
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, 1)
    lib = _load()
    nbytes = lib.proj_gemm_backward_workspace_size(M, N, K, block_k, R, ctypes.byref(b), ctypes.byref(p))
    if nbytes == 0:
        raise ProjError(PJ_EINVAL, "proj_gemm_backward_saved", last_error())
    ws = _workspace(nbytes, dY.device, workspace)
    with torch.cuda.device(dY.device):
        st = lib.proj_gemm_backward_saved(_ptr(fwd_workspace), fwd_workspace.numel(), _ptr(dY), _rows(dY), _ptr(dA),
                                          _rows(dA), _ptr(dB), _rows(dB), M, N, K, _DT[dY.dtype], _DT[out_dtype],
                                          block_k, R, ctypes.byref(b), ctypes.byref(p), _ptr(ws), ws.numel(),
                                          _stream(stream, dY.device))
    _check(st, "proj_gemm_backward_saved")
    return dA, dB


class ProjGemmFn(torch.autograd.Function):
    """Y = projected A B with hand-written adjoint kernels (basis held fixed).

    By default backward recomputes A_c and B_d from the saved inputs rather than
    storing them; with save_projections the forward's workspace (which holds A_c
    and B_d) is kept instead and backward reads them from it (split = 1 only).
    """

    @staticmethod
    def forward(ctx, A, B, block_k, R, basis="dct2", L=8, user_C=None, split=1, save_projections=False):
        ctx.cfg = (block_k, R, basis, L, user_C)
        out_dtype = torch.float64 if A.dtype == torch.float64 else torch.float32
        ctx.fwd_ws = None
        if save_projections:
            if split != 1:
                raise ValueError("save_projections needs split = 1")
            compute = "f64" if A.dtype == torch.float64 else "bf16"
            M, K = A.shape
            ws = torch.empty(gemm_workspace_size(M, B.shape[1], K, block_k, R, basis, L, compute, user_C=user_C),
                             dtype=torch.uint8, device=A.device)
            ctx.fwd_ws = ws
            ctx.shape = (K, A.dtype, B.dtype)
            ctx.save_for_backward()
            return proj_gemm(A.contiguous(), B.contiguous(), block_k, R, basis, L, split=1, out_dtype=out_dtype,
                             user_C=user_C, workspace=ws)
        ctx.save_for_backward(A, B)
        return proj_gemm(A.contiguous(), B.contiguous(), block_k, R, basis, L, split=split, out_dtype=out_dtype,
                         user_C=user_C)

    @staticmethod
    def backward(ctx, dY):
        block_k, R, basis, L, user_C = ctx.cfg
        if ctx.fwd_ws is not None:
            K, a_dtype, b_dtype = ctx.shape
            compute = "f64" if a_dtype == torch.float64 else "bf16"
            dA, dB = proj_gemm_backward_saved(ctx.fwd_ws, dY.to(a_dtype).contiguous(), K, block_k, R, basis, L,
                                              compute, out_dtype=a_dtype, user_C=user_C)
            ctx.fwd_ws = None
            dB = dB.to(b_dtype)
        else:
            A, B = ctx.saved_tensors
            dA, dB = proj_gemm_backward(A.contiguous(), B.contiguous(), dY, block_k, R, basis, L, user_C=user_C)
        return (dA if ctx.needs_input_grad[0] else None, dB if ctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None)


def proj_matmul(A, B, block_k: int, R: int, basis: str = "dct2", L: int = 8, user_C=None, split: int = 1,
                save_projections: bool = False):
    """Differentiable projected product (see ProjGemmFn)."""
    return ProjGemmFn.apply(A, B, block_k, R, basis, L, user_C, split, save_projections)


def conv_workspace_size(S, T, n_templates, R, basis="haar", L=64, compute="bf16", split=1, user_C=None) -> int:
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, split)
    n = _load().proj_conv_workspace_size(S, T, n_templates, T, R, ctypes.byref(b), ctypes.byref(p))
    if n == 0:
        raise ProjError(PJ_EINVAL, "proj_conv_workspace_size", last_error())
    return int(n)


def proj_conv(signal, templates, R: int, basis: str = "haar", L: int = 64, out=None, workspace=None,
              stream=None, pin_output: bool = True, step: int = 1, user_C=None, compute: str = "bf16"):
    """r[m, t] = projected valid cross-correlation of signal (S,) with templates (n_t, T).

    step > 1 (a power of two, at most T / R): only every step-th lag is computed and
    the lags between are interpolated from their two computed neighbours
    (proj_conv_interp; step = 2 is the paper's half-sample option).
    compute="e4m3": E4M3 components with per-32 block scales (Haar, R a multiple of
    64, CUDA tensors, step 1; planned in the workspace per call).
    CUDA tensors run on their device; CPU tensors are copied to the current
    device, computed there and the result copied back to host memory.
    """
    if compute != "bf16" and (signal.device.type == "cpu" or step != 1):
        raise ValueError("E4M3 correlation takes CUDA tensors and step 1")
    if signal.device.type == "cpu" and step == 1:
        # host buffers: proj_conv_host overlaps the copy of each lag range to the
        # host with the correlation of the next
        return proj_conv_host(signal, templates, R, basis, L, out, workspace, stream, pin_output, user_C=user_C)
    if signal.device.type == "cpu":
        dev = torch.device("cuda", torch.cuda.current_device())
        s_d = signal.to(dev, non_blocking=True)
        k_d = templates.to(dev, non_blocking=True)
        r = proj_conv(s_d, k_d, R, basis, L, None, workspace, stream, step=step, user_C=user_C)
        if out is None:
            out = torch.empty(r.shape, dtype=r.dtype, pin_memory=pin_output)
        out.copy_(r, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        return out
    S = signal.shape[0]
    nt, T = templates.shape
    if signal.dtype != torch.float32 or templates.dtype != torch.float32:
        raise ValueError("CONV takes float32 signal and templates")
    if not signal.is_contiguous() or not templates.is_contiguous():
        raise ValueError("signal and templates must be contiguous")
    if out is None:
        out = torch.empty((S - T + 1, nt), dtype=torch.float32, device=signal.device)
    b, _keep = _basis(basis, L, user_C)
    p = _prec(compute, 1)
    lib = _load()
    nbytes = lib.proj_conv_workspace_size(S, T, nt, T, R, ctypes.byref(b), ctypes.byref(p))
    if nbytes == 0:
        raise ProjError(PJ_EINVAL, "proj_conv", last_error())
    ws = _workspace(nbytes, signal.device, workspace)
    with torch.cuda.device(signal.device):
        if step == 1:
            st = lib.proj_conv(_ptr(signal), S, _ptr(templates), T, nt, _ptr(out), PJ_F32, PJ_F32, T, R,
                               ctypes.byref(b), ctypes.byref(p), _ptr(ws), ws.numel(),
                               _stream(stream, signal.device))
        else:
            st = lib.proj_conv_interp(_ptr(signal), S, _ptr(templates), T, nt, _ptr(out), PJ_F32, PJ_F32, T, R,
                                      ctypes.byref(b), ctypes.byref(p), int(step), _ptr(ws), ws.numel(),
                                      _stream(stream, signal.device))
    _check(st, "proj_conv_interp" if step != 1 else "proj_conv")
    return out


def conv_host_workspace_size(S, T, n_templates, R, basis="haar", L=64, chunks: int = 4, user_C=None) -> int:
    b, _keep = _basis(basis, L, user_C)
    p = _prec("bf16", 1)
    n = _load().proj_conv_host_workspace_size(S, T, n_templates, T, R, ctypes.byref(b), ctypes.byref(p), chunks)
    if n == 0:
        raise ProjError(PJ_EINVAL, "proj_conv_host_workspace_size", last_error())
    return int(n)


def proj_conv_host(signal, templates, R: int, basis: str = "haar", L: int = 64, out=None, workspace=None,
                   stream=None, pin_output: bool = True, chunks: int = 4, device=None, user_C=None):
    """proj_conv with signal, templates and result in host memory (proj_conv_host in the
    C ABI): the lags run in `chunks` ranges and each range's copy to the host overlaps
    the correlation of the next.  Returns when the result is in `out`."""
    if signal.dtype != torch.float32 or templates.dtype != torch.float32:
        raise ValueError("CONV takes float32 signal and templates")
    device = device or torch.device("cuda", torch.cuda.current_device())
    signal = signal.contiguous()
    templates = templates.contiguous()
    S = signal.shape[0]
    nt, T = templates.shape
    if out is None:
        out = torch.empty((S - T + 1, nt), dtype=torch.float32, pin_memory=pin_output)
    if out.device.type != "cpu" or not out.is_contiguous():
        raise ValueError("out must be a contiguous host tensor")
    b, _keep = _basis(basis, L, user_C)
    p = _prec("bf16", 1)
    lib = _load()
    nbytes = lib.proj_conv_host_workspace_size(S, T, nt, T, R, ctypes.byref(b), ctypes.byref(p), chunks)
    if nbytes == 0:
        raise ProjError(PJ_EINVAL, "proj_conv_host", last_error())
    if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
        workspace = _workspace(nbytes, device, None)
    with torch.cuda.device(device):
        st = lib.proj_conv_host(_ptr(signal), S, _ptr(templates), T, nt, _ptr(out), PJ_F32, PJ_F32, T, R,
                                ctypes.byref(b), ctypes.byref(p), int(chunks), _ptr(workspace), workspace.numel(),
                                _stream(stream, device))
        _check(st, "proj_conv_host")
        (stream or torch.cuda.current_stream(device)).synchronize()
    return out


def proj_conv_project(signal, templates, R: int, workspace, basis="haar", L=64, T=None, n_templates=None,
                      stream=None, user_C=None):
    """Stage 1 of proj_conv: projected signal and (unless None) templates into the workspace."""
    lib = _load()
    if templates is not None:
        n_templates, T = templates.shape
    b, _keep = _basis(basis, L, user_C)
    p = _prec("bf16", 1)
    st = lib.proj_conv_project(_ptr(signal), signal.shape[0], _ptr(templates), T, n_templates, PJ_F32, T, R,
                               ctypes.byref(b), ctypes.byref(p), _ptr(workspace), workspace.numel(),
                               _stream(stream, signal.device))
    _check(st, "proj_conv_project")


def proj_conv_correlate(S: int, T: int, n_templates: int, R: int, out, workspace, basis="haar", L=64,
                        stream=None, user_C=None):
    """Stage 2 of proj_conv: the reduced correlation from the workspace into out ((S-T+1) x n_t)."""
    lib = _load()
    b, _keep = _basis(basis, L, user_C)
    p = _prec("bf16", 1)
    st = lib.proj_conv_correlate(S, T, n_templates, _ptr(out), PJ_F32, T, R, ctypes.byref(b), ctypes.byref(p),
                                 _ptr(workspace), workspace.numel(), _stream(stream, out.device))
    _check(st, "proj_conv_correlate")
    return out


def basis_build(kind: str, L: int, lp1: int, user_C=None, device=None, stream=None):
    """(C_R, D_R): kept basis tables built on the GPU in FP64 (L x lp1 and lp1 x L)."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    lib = _load()
    C = torch.empty((L, lp1), dtype=torch.float64, device=device)
    D = torch.empty((lp1, L), dtype=torch.float64, device=device)
    ws = torch.empty(512 * 1024, dtype=torch.uint8, device=device)
    b, _keep = _basis(kind, L, user_C)
    st = lib.pj_basis_build(ctypes.byref(b), lp1, _ptr(C), _ptr(D), _ptr(ws), ws.numel(), _stream(stream, device))
    _check(st, "pj_basis_build")
    check(ws, stream)
    return C, D


def proj_gemm_report(A, B, block_k: int, R: int, basis: str = "dct2", L: int = 8, compute: str | None = None,
                     split: int = 1, split_lead: int = 0, out_dtype=None, user_C=None, stream=None) -> dict:
    """A-posteriori report of proj_gemm(A, B, ...): algorithmic flops and bytes, the
    Frobenius norms of A and B, a bound on the truncation error ||A B - Y_R||_F
    (-1 for a user basis) and one on the rounding error ||Y - Y_R||_F of the chosen
    arithmetic (-1 for E4M3).  Synchronizes the stream."""
    lib = _load()
    M, K = A.shape
    N = B.shape[1]
    if compute is None:
        compute = "f64" if A.dtype == torch.float64 else "bf16"
    if out_dtype is None:
        out_dtype = torch.float64 if compute == "f64" else torch.float32
    ws = torch.empty(lib.proj_gemm_report_workspace_size(K, block_k), dtype=torch.uint8, device=A.device)
    b, _keep = _basis(basis, L, user_C, ws)
    p = _prec(compute, split, split_lead)
    rep = _Report()
    st = lib.proj_gemm_report(_ptr(A), _rows(A), _ptr(B), _rows(B), M, N, K, _DT[A.dtype], _DT[out_dtype], block_k, R,
                              ctypes.byref(b), ctypes.byref(p), _ptr(ws), ws.numel(), _stream(stream, A.device),
                              ctypes.byref(rep))
    _check(st, "proj_gemm_report")
    return {name: getattr(rep, name) for name, _ in _Report._fields_}


def selftest_timeout(which: int, device=None, stream=None) -> int:
    """Failure-detection self-test: run a kernel whose bounded waits run out
    (which = 0: a lone wait; which = 1: a GEMM on a CTA pair whose copy producers
    stop early) and return pj_check's status, PJ_ETIMEOUT when the waits gave up
    as designed.  Takes about 2 s."""
    lib = _load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    ws = torch.empty(lib.pj_selftest_workspace_size(), dtype=torch.uint8, device=dev)
    st = _stream(stream, dev)
    _check(lib.pj_selftest_timeout(int(which), _ptr(ws), ws.numel(), st), "pj_selftest_timeout")
    return lib.pj_check(_ptr(ws), st)


def check(workspace, stream=None):
    """Synchronize and raise if a kernel recorded an error in the workspace's error word."""
    lib = _load()
    st = lib.pj_check(_ptr(workspace), _stream(stream, workspace.device))
    _check(st, "pj_check")


# ------------------------------------------------------------------ batch --

def batch_gemm(A, B, Y, block_k: int, R: int, basis: str = "dct2", L: int = 8, split: int = 1, user_C=None,
               compute: str = "bf16"):
    """Descriptor of one projected GEMM instance Y = proj(A) proj(B) for BatchPlan
    (compute "bf16" or "e4m3")."""
    M, K = A.shape
    N = B.shape[1]
    return dict(op=0, A=A, B=B, Y=Y, M=M, N=N, K=K, lda=_rows(A), ldb=_rows(B), ldy=_rows(Y), block=block_k, R=R,
                basis=basis, L=L, split=split, user_C=user_C, in_dtype=_DT[A.dtype], out_dtype=_DT[Y.dtype],
                compute=compute)


def batch_conv(signal, templates, out, R: int, basis: str = "haar", L: int = 64, split: int = 1,
               compute: str = "bf16"):
    """Descriptor of one projected cross-correlation instance for BatchPlan
    (split=2: hi + lo residual components, three reduced products; compute="e4m3":
    E4M3 components with per-32 block scales, split 1)."""
    nt, T = templates.shape
    return dict(op=1, A=signal, B=templates, Y=out, M=signal.shape[0], N=nt, K=T, lda=0, ldb=0, ldy=0, block=T,
                R=R, basis=basis, L=L, split=split, user_C=None, in_dtype=PJ_F32, out_dtype=PJ_F32,
                compute=compute)


class BatchPlan:
    """Plan of many uneven GEMM / CONV instances run as batched projections plus one
    persistent grouped tensor-core GEMM (proj_batch_* in the C ABI).

    The tensors named in the descriptors must stay alive while the plan is used;
    run() reads their current contents.
    """

    def __init__(self, descs, device=None, stream=None, tuning=None):
        """tuning: None (defaults) or a dict with any of TUNING_KEYS (pj_batch_tuning)."""
        self._lib = _load()
        self._keep = []
        arr = (_BatchDesc * len(descs))()
        for i, d in enumerate(descs):
            b, keep = _basis(d["basis"], d["L"], d.get("user_C"))
            self._keep.append((d, keep))
            arr[i] = _BatchDesc(d["op"], d["in_dtype"], d["out_dtype"], 0, d["A"].data_ptr(), d["B"].data_ptr(),
                                d["Y"].data_ptr(), d["M"], d["N"], d["K"], d["lda"], d["ldb"], d["ldy"], d["block"],
                                d["R"], b, _prec(d.get("compute", "bf16"), d["split"]))
        self._arr = arr
        self.tuning = dict(tuning) if tuning else None
        tun = _tuning(tuning)
        tp = ctypes.byref(tun) if tun is not None else None
        n = self._lib.proj_batch_workspace_size_tuned(arr, len(descs), tp)
        if n == 0:
            raise ProjError(PJ_EINVAL, "proj_batch_workspace_size", last_error())
        device = device or descs[0]["A"].device
        self.device = device
        self.workspace = torch.empty(int(n), dtype=torch.uint8, device=device)
        plan = ctypes.c_void_p()
        with torch.cuda.device(device):
            st = self._lib.proj_batch_plan_create_tuned(arr, len(descs), tp, _ptr(self.workspace),
                                                        self.workspace.numel(), _stream(stream, device),
                                                        ctypes.byref(plan))
        _check(st, "proj_batch_plan_create")
        self._plan = plan

    def info(self) -> dict:
        """The tuner's decisions: tiles per grouped launch, CTAs, split instances, model times (us)."""
        inf = _BatchInfo()
        _check(self._lib.proj_batch_plan_info(self._plan, ctypes.byref(inf)), "proj_batch_plan_info")
        return {k: getattr(inf, k) for k, _ in _BatchInfo._fields_}

    def run(self, stream=None):
        with torch.cuda.device(self.device):
            st = self._lib.proj_batch_run(self._plan, _stream(stream, self.device))
        _check(st, "proj_batch_run")

    def check(self, stream=None):
        check(self.workspace, stream)

    def __del__(self):
        plan = getattr(self, "_plan", None)
        if plan:
            self._lib.proj_batch_destroy(plan)
            self._plan = None


# --------------------------------------------------------------- autotuner --

DEFAULT_CANDIDATES = (
    None,                                            # cost-model splits, fitted heights, round-robin by K
    {"tile_rows": 256},                              # the same with full-height tiles
    {"schedule": 2},                                 # cost-model splits, least-loaded CTA first (LPT)
    {"schedule": 1},                                 # no model: round-robin by reduced K, fitted heights
    {"schedule": 1, "tile_rows": 256},               # no model, full-height tiles (the untuned plan)
    {"tile_rows": 128},                              # 128-row tiles
    {"solo": 1},                                     # every CTA loads its own A_c tiles (no CTA pairs)
)


def _batch_key(descs) -> str:
    import hashlib
    import json
    name = torch.cuda.get_device_name()
    shape = [(d["op"], d["M"], d["N"], d["K"], d["block"], d["R"], d["split"], d.get("compute", "bf16"),
              d["basis"], d["L"], d["in_dtype"], d["out_dtype"]) for d in descs]
    return hashlib.sha256(json.dumps([name, shape]).encode()).hexdigest()[:24]


TUNE_CACHE_VERSION = 2   # bump when the tuning knobs or the planner change meaning


def _entry_digest(entry) -> str:
    import hashlib
    import json
    body = {k: entry[k] for k in ("version", "library", "best", "trials")}
    return hashlib.sha256(json.dumps(body, sort_keys=True).encode()).hexdigest()


def _cache_load(cache, key):
    """The cached (best, trials) under `key`, or None when the file is missing or
    unreadable, the entry absent, written by another cache or library version, or
    its checksum does not match its contents."""
    import json
    if not cache or not os.path.exists(cache):
        return None
    try:
        with open(cache) as f:
            entry = json.load(f).get(key)
        if (entry is None or entry.get("version") != TUNE_CACHE_VERSION or entry.get("library") != version()
                or entry.get("sha256") != _entry_digest(entry)):
            return None
        return entry["best"], entry["trials"]
    except (OSError, ValueError, KeyError, TypeError, AttributeError):
        return None


def _cache_store(cache, key, best, trials):
    """Add the entry to the JSON cache file (written to a temporary file, then renamed)."""
    import json
    data = {}
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                data = json.load(f)
            if not isinstance(data, dict):
                data = {}
        except (OSError, ValueError):
            data = {}
    entry = {"version": TUNE_CACHE_VERSION, "library": version(), "best": best, "trials": trials}
    entry["sha256"] = _entry_digest(entry)
    data[key] = entry
    tmp = f"{cache}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, cache)


def _cached_product_key(A, out, block_k, R, basis, L, split, user_C) -> str:
    import hashlib
    import json
    uc = None
    if user_C is not None:
        uc = hashlib.sha256(torch.as_tensor(user_C, dtype=torch.float64).contiguous().numpy().tobytes()).hexdigest()
    body = [torch.cuda.get_device_name(A.device), "cached_product", list(A.shape), list(out.shape), block_k, R, basis,
            L, split, str(A.dtype), str(out.dtype), uc]
    return hashlib.sha256(json.dumps(body).encode()).hexdigest()[:24]


def autotune_cached_product(A, out, block_k: int, R: int, workspace, basis="dct2", L=8, split=1, user_C=None,
                            reps: int = 3, stream=None, cache=None):
    """Time the two ways of multiplying a new A by the B_d already projected into
    `workspace` (proj_gemm_project(None, B, ...)) and return (best, trials), best being
    "two_pass" (proj_gemm_project of A, then proj_gemm_multiply) or "fused"
    (proj_gemm_fused: A projected inside the GEMM).  A path the library refuses for
    these shapes is recorded with its error and not chosen.  Each path runs once,
    then `reps` times between CUDA events on `stream`; `out` holds the last result.
    With `cache` the answer is kept and looked up like autotune_batch's."""
    key = _cached_product_key(A, out, block_k, R, basis, L, split, user_C)
    hit = _cache_load(cache, key)
    if hit is not None:
        return hit
    stream = stream or torch.cuda.current_stream(A.device)
    M, K = A.shape
    N = out.shape[1]

    def two_pass():
        proj_gemm_project(A, None, block_k, R, workspace, basis, L, "bf16", split, user_C=user_C, stream=stream, N=N)
        proj_gemm_multiply(out, K, block_k, R, workspace, basis, L, "bf16", split, user_C=user_C, stream=stream)

    def fused():
        proj_gemm_fused(A, out, block_k, R, workspace, basis, L, split, user_C=user_C, stream=stream)

    trials = []
    for name, fn in (("two_pass", two_pass), ("fused", fused)):
        try:
            fn()
        except ProjError as e:
            trials.append({"path": name, "ms": None, "error": str(e)})
            continue
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        ev[1].synchronize()
        trials.append({"path": name, "ms": ev[0].elapsed_time(ev[1]) / reps})
    best = min((t for t in trials if t["ms"] is not None), key=lambda t: t["ms"])["path"]
    if cache:
        _cache_store(cache, key, best, trials)
    return best, trials


def proj_gemm_cached(A, out, block_k: int, R: int, workspace, basis="dct2", L=8, split=1, user_C=None, path=None,
                     stream=None, cache=None):
    """out = A_c B_d with B_d already in `workspace`, by `path` ("two_pass" or "fused"),
    or, with path None, by the one autotune_cached_product measures (and caches) for
    these shapes."""
    if path is None:
        path, _ = autotune_cached_product(A, out, block_k, R, workspace, basis, L, split, user_C, stream=stream,
                                          cache=cache)
    if path == "fused":
        return proj_gemm_fused(A, out, block_k, R, workspace, basis, L, split, user_C=user_C, stream=stream)
    if path != "two_pass":
        raise ValueError(f"unknown path {path!r}")
    proj_gemm_project(A, None, block_k, R, workspace, basis, L, "bf16", split, user_C=user_C, stream=stream,
                      N=out.shape[1])
    return proj_gemm_multiply(out, A.shape[1], block_k, R, workspace, basis, L, "bf16", split, user_C=user_C,
                              stream=stream)


def autotune_batch(descs, candidates=DEFAULT_CANDIDATES, reps: int = 3, device=None, stream=None, cache=None):
    """Measure candidate tunings of one batch on the GPU and return (best, trials).

    Each candidate (a pj_batch_tuning dict, None = defaults) is planned, run once,
    then timed over `reps` runs with CUDA events on `stream`; the fastest wins.
    trials lists {"tuning", "ms", "info"} per candidate.  With `cache` (a JSON file
    path) a result found under the key of this GPU, these shapes and these
    candidates is returned without measuring (entries carry the cache and library
    versions and a checksum; others are measured again), and new results are
    stored there.
    """
    import json
    key = _batch_key(descs) + ":" + json.dumps(list(candidates), sort_keys=True)
    hit = _cache_load(cache, key)
    if hit is not None:
        return hit
    device = device or descs[0]["A"].device
    stream = stream or torch.cuda.current_stream(device)
    trials = []
    for cand in candidates:
        plan = BatchPlan(descs, device=device, stream=stream, tuning=cand)
        plan.run(stream)
        plan.check(stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            plan.run(stream)
        ev[1].record(stream)
        ev[1].synchronize()
        trials.append({"tuning": cand, "ms": ev[0].elapsed_time(ev[1]) / reps, "info": plan.info()})
        del plan
        torch.cuda.empty_cache()
    best = min(trials, key=lambda t: t["ms"])["tuning"]
    if cache:
        _cache_store(cache, key, best, trials)
    return best, trials
