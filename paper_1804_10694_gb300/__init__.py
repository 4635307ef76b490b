"""GB300-native split-precision sgemm: C = alpha*A*B + beta*C in FP32 semantics
(the running example and sgemm benchmark of the Tiramisu paper, arXiv
1804.10694, Section I and Section VI-A).

Python binding of the C ABI in include/gemm.h.  It only marshals arguments:
every step of the computation runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams.  Matrices are row-major torch.float32 CUDA
tensors with unit inner stride; leading dimensions are read from the strides.
"""
from __future__ import annotations

import ctypes

from . import _native
from ._native import GemmConfig, GemmError, check, load  # noqa: F401

MODES = {"auto": 0, "simt": 1, "f32_simt": 1, "bf16x3": 2, "tf32x3": 3}
SELECTS = {"default": 0, "model": 1, "table": 2, "exhaustive": 3}


def _mode(m) -> int:
    return MODES[m] if isinstance(m, str) else int(m)


def _select(s) -> int:
    return SELECTS[s] if isinstance(s, str) else int(s)


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _matrix(t, name: str):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    rows, cols = t.shape
    if rows > 0 and cols > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must have unit inner stride (row-major)")
    ld = t.stride(0) if rows > 1 else max(cols, 1)
    return t.data_ptr(), rows, cols, max(ld, cols, 1)


def gemm(A, B, C, alpha: float = 1.0, beta: float = 0.0, mode="auto", select="default",
         stream=None):
    """C <- alpha*A@B + beta*C in place (C is returned)."""
    pa, M, K, lda = _matrix(A, "A")
    pb, K2, N, ldb = _matrix(B, "B")
    pc, M2, N2, ldc = _matrix(C, "C")
    if K2 != K or M2 != M or N2 != N:
        raise ValueError(f"shape mismatch: A {tuple(A.shape)}, B {tuple(B.shape)}, C {tuple(C.shape)}")
    lib = load()
    check(lib.gemm_f32_ex(M, N, K, alpha, pa, lda, pb, ldb, beta, pc, ldc, _mode(mode),
                          _select(select), _stream_handle(stream)))
    return C


def gemm_f32(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc):
    """Direct pass-through of gemm_f32 (device pointers as integers)."""
    check(load().gemm_f32(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc))


def gemm_f32_ex(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, mode, select, stream):
    check(load().gemm_f32_ex(M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc,
                             _mode(mode), _select(select), stream))


def gemm_host(A, B, C, alpha: float = 1.0, beta: float = 0.0, mode="auto", stream=None):
    """gemm_f32_host on numpy float32 arrays or pinned CPU torch tensors (C
    updated in place).  The copies to and from the device happen inside the
    call."""
    import numpy as np

    def host(x, name):
        if hasattr(x, "data_ptr"):
            if x.dtype.__repr__() != "torch.float32" or x.dim() != 2 or x.stride(1) != 1:
                raise TypeError(f"{name}: 2-D row-major float32 CPU tensor expected")
            return x.data_ptr(), x.shape[0], x.shape[1], max(x.stride(0), x.shape[1], 1)
        if not isinstance(x, np.ndarray) or x.dtype != np.float32 or not x.flags.c_contiguous:
            raise TypeError(f"{name}: C-contiguous float32 numpy array expected")
        return x.ctypes.data, x.shape[0], x.shape[1], max(x.shape[1], 1)

    pa, M, lda_cols, lda = host(A, "A")
    pb, K, ldb_cols, ldb = host(B, "B")
    pc, M2, ldc_cols, ldc = host(C, "C")
    N = ldb_cols
    K_ = lda_cols
    if K_ != K or M2 != M or ldc_cols != N:
        raise ValueError("shape mismatch")
    h = 0 if stream is None else _stream_handle(stream)
    check(load().gemm_f32_host(M, N, K, alpha, pa, lda, pb, ldb, beta, pc, ldc, _mode(mode), h))
    return C


class Plan:
    """A gemm plan for one shape (owns its workspace); see gemm_plan_create."""

    def __init__(self, M, N, K, lda=None, ldb=None, ldc=None, mode="auto", select="default",
                 config_id: int | None = None):
        lib = load()
        self._lib = lib
        self.M, self.N, self.K = M, N, K
        self.lda = lda if lda is not None else max(K, 1)
        self.ldb = ldb if ldb is not None else max(N, 1)
        self.ldc = ldc if ldc is not None else max(N, 1)
        h = ctypes.c_void_p()
        if config_id is None:
            check(lib.gemm_plan_create(M, N, K, self.lda, self.ldb, self.ldc, _mode(mode),
                                       _select(select), ctypes.byref(h)))
        else:
            check(lib.gemm_plan_create_config(M, N, K, self.lda, self.ldb, self.ldc, _mode(mode),
                                              int(config_id), ctypes.byref(h)))
        self._h = h

    def execute(self, A, B, C, alpha: float = 1.0, beta: float = 0.0, stream=None):
        pa, M, K, lda = _matrix(A, "A")
        pb, _, N, ldb = _matrix(B, "B")
        pc, _, _, ldc = _matrix(C, "C")
        if (M, N, K) != (self.M, self.N, self.K) or (lda, ldb, ldc) != (self.lda, self.ldb, self.ldc):
            raise ValueError("tensors do not match the plan's shape / leading dimensions")
        check(self._lib.gemm_plan_execute(self._h, alpha, pa, pb, beta, pc, _stream_handle(stream)))
        return C

    def execute_ptrs(self, alpha, A_ptr, B_ptr, beta, C_ptr, stream=None):
        check(self._lib.gemm_plan_execute(self._h, alpha, A_ptr, B_ptr, beta, C_ptr,
                                          _stream_handle(stream)))

    def info(self) -> dict:
        m, c, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        check(self._lib.gemm_plan_info(self._h, ctypes.byref(m), ctypes.byref(c), ctypes.byref(w)))
        return {"mode": m.value, "config_id": c.value, "workspace_bytes": w.value}

    def profile(self, max_records: int):
        """Record stage-timing events for the next max_records executions."""
        check(self._lib.gemm_plan_profile(self._h, int(max_records)))

    def profile_read(self) -> dict:
        n = ctypes.c_int()
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        check(self._lib.gemm_plan_profile_read(self._h, ctypes.byref(n), ctypes.byref(a),
                                               ctypes.byref(b), ctypes.byref(c)))
        return {"records": n.value, "pack_ms": a.value, "main_ms": b.value, "reduce_ms": c.value}

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(self._lib.gemm_plan_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def config_count(mode="bf16x3") -> int:
    return load().gemm_config_count(_mode(mode))


def config_get(mode, config_id: int) -> dict:
    c = GemmConfig()
    check(load().gemm_config_get(_mode(mode), config_id, ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in GemmConfig._fields_}


def config_default(mode, M, N, K) -> int:
    return load().gemm_config_default(_mode(mode), M, N, K)


def device_error() -> None:
    """Raise if a kernel abandoned a pipeline wait since the last check."""
    check(load().gemm_device_error())


def sm_count() -> int:
    return load().gemm_device_sm_count()


def packed_pitch(mode, K: int) -> int:
    q = 8 if _mode(mode) == 2 else 4
    return (K + q - 1) // q * q


def split_pack(X, mode="bf16x3", transpose: bool = False, stream=None):
    """Run the packing stage alone; returns (planes, amax) torch tensors.
    planes: [2][rows][pitch] (bf16 or float32 holding tf32 values); amax:
    int32 view of the per-block max |x| bit patterns."""
    import torch
    px, rows, cols, ld = _matrix(X, "X")
    m = _mode(mode)
    K = rows if transpose else cols
    prow = cols if transpose else rows
    pitch = packed_pitch(m, K)
    dt = torch.bfloat16 if m == 2 else torch.float32
    planes = torch.zeros((2, prow, pitch), dtype=dt, device=X.device)
    amax = torch.zeros(((prow + 127) // 128,), dtype=torch.int32, device=X.device)
    check(load().gemm_split_pack(m, 1 if transpose else 0, rows, cols, px, ld, planes.data_ptr(),
                                 pitch, amax.data_ptr(), _stream_handle(stream)))
    return planes, amax
