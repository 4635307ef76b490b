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

MODES = {"auto": 0, "simt": 1, "f32_simt": 1, "bf16x3": 2, "tf32x3": 3, "bf16x6": 4}
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


def gemm_f32_t(trans_a, trans_b, M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, mode,
               select, stream):
    check(load().gemm_f32_t(int(trans_a), int(trans_b), M, N, K, alpha, A_ptr, lda, B_ptr, ldb, beta,
                            C_ptr, ldc, _mode(mode), _select(select), stream))


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
                 config_id: int | None = None, trans_a: bool = False, trans_b: bool = False,
                 compensated: bool = False):
        lib = load()
        self._lib = lib
        self.M, self.N, self.K = M, N, K
        self.trans_a, self.trans_b = bool(trans_a), bool(trans_b)
        self.lda = lda if lda is not None else max(M if trans_a else K, 1)
        self.ldb = ldb if ldb is not None else max(K if trans_b else N, 1)
        self.ldc = ldc if ldc is not None else max(N, 1)
        h = ctypes.c_void_p()
        if compensated:
            if trans_a or trans_b:
                raise ValueError("the compensated epilogue is offered for untransposed plans")
            check(lib.gemm_plan_create_opts(M, N, K, self.lda, self.ldb, self.ldc, _mode(mode),
                                            _select(select), -1 if config_id is None else int(config_id),
                                            1, ctypes.byref(h)))
        elif trans_a or trans_b:
            if config_id is not None:
                raise ValueError("transposed plans choose their configuration by `select`")
            check(lib.gemm_plan_create_t(int(trans_a), int(trans_b), M, N, K, self.lda, self.ldb,
                                         self.ldc, _mode(mode), _select(select), ctypes.byref(h)))
        elif config_id is None:
            check(lib.gemm_plan_create(M, N, K, self.lda, self.ldb, self.ldc, _mode(mode),
                                       _select(select), ctypes.byref(h)))
        else:
            check(lib.gemm_plan_create_config(M, N, K, self.lda, self.ldb, self.ldc, _mode(mode),
                                              int(config_id), ctypes.byref(h)))
        self._h = h

    def execute(self, A, B, C, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """A, B as stored (K x M for a transposed A, N x K for a transposed B)."""
        pa, ra, ca, lda = _matrix(A, "A")
        pb, rb, cb, ldb = _matrix(B, "B")
        pc, M, N, ldc = _matrix(C, "C")
        K = ra if self.trans_a else ca
        ok = (ca, ra) == (M, K) if self.trans_a else (ra, ca) == (M, K)
        ok = ok and ((rb, cb) == (N, K) if self.trans_b else (rb, cb) == (K, N))
        if not ok or (M, N, K) != (self.M, self.N, self.K) or (lda, ldb, ldc) != (self.lda, self.ldb, self.ldc):
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
    q = 8 if _mode(mode) in (2, 4) else 4
    return (K + q - 1) // q * q


def split_pack(X, mode="bf16x3", transpose: bool = False, stream=None):
    """Run the packing stage alone; returns (planes, amax) torch tensors.
    planes: [2][rows][pitch] (bf16 or float32 holding tf32 values; [3][rows]
    [pitch] bf16 for bf16x6); amax: int32 view of the per-block max |x| bit
    patterns."""
    import torch
    px, rows, cols, ld = _matrix(X, "X")
    m = _mode(mode)
    K = rows if transpose else cols
    prow = cols if transpose else rows
    pitch = packed_pitch(m, K)
    dt = torch.bfloat16 if m in (2, 4) else torch.float32
    planes = torch.zeros((3 if m == 4 else 2, prow, pitch), dtype=dt, device=X.device)
    nblk = (prow + 127) // 128
    work = torch.zeros((2 * nblk,), dtype=torch.int32, device=X.device)   # maxima, then counters
    check(load().gemm_split_pack(m, 1 if transpose else 0, rows, cols, px, ld, planes.data_ptr(),
                                 pitch, work.data_ptr(), _stream_handle(stream)))
    return planes, work[:nblk]


# ------------------------------------------------------------- convolution
class ConvPlan(Plan):
    """Direct convolution with an odd R x S filter (stride 1, same zero
    padding) as an implicit gemm on NHWC images; see gemm_conv_plan_create."""

    def __init__(self, batch, H, W, C, K, R=3, S=3, mode="bf16x3", config_id: int | None = None):
        lib = load()
        self._lib = lib
        self.batch, self.H, self.W, self.C, self.K_out, self.R, self.S = batch, H, W, C, K, R, S
        self.M, self.N, self.K = batch * H * W, K, R * S * C
        self.lda, self.ldb, self.ldc = R * S * C, K, K
        h = ctypes.c_void_p()
        check(lib.gemm_conv_plan_create(batch, H, W, C, K, int(R), int(S), _mode(mode),
                                        -1 if config_id is None else int(config_id), ctypes.byref(h)))
        self._h = h

    def execute(self, x, f, out, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """x: [batch, H, W, C], f: [R, S, C, K], out: [batch, H, W, K], all
        contiguous float32 CUDA tensors."""
        import torch
        want = {"x": (x, (self.batch, self.H, self.W, self.C)),
                "f": (f, (self.R, self.S, self.C, self.K_out)),
                "out": (out, (self.batch, self.H, self.W, self.K_out))}
        for name, (t, shape) in want.items():
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError(f"{name} must be a float32 CUDA tensor")
            if tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous tensor of shape {shape}")
        check(self._lib.gemm_plan_execute(self._h, alpha, x.data_ptr(), f.data_ptr(), beta,
                                          out.data_ptr(), _stream_handle(stream)))
        return out


class Conv3x3Plan(ConvPlan):
    """ConvPlan with a 3x3 filter (zero padding 1); see gemm_conv3x3_plan_create."""

    def __init__(self, batch, H, W, C, K, mode="bf16x3", config_id: int | None = None):
        super().__init__(batch, H, W, C, K, 3, 3, mode, config_id)


# ------------------------------------------------------------------ grouped
def _i64_array(vals):
    arr = (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])
    return arr


class GroupedPlan:
    """Plan for G independent gemms run in one persistent launch (see
    gemm_grouped_plan_create).  shapes: list of (M, N, K); leading dimensions
    default to the row lengths."""

    def __init__(self, shapes, lds=None, mode="bf16x3", select="default", block_n=None, kb=None):
        lib = load()
        self._lib = lib
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        G = len(self.shapes)
        if lds is None:
            lds = [(max(k, 1), max(n, 1), max(n, 1)) for (m, n, k) in self.shapes]
        self.lds = [tuple(int(x) for x in l) for l in lds]
        arrs = [_i64_array([s[i] for s in self.shapes]) for i in range(3)]
        larrs = [_i64_array([l[i] for l in self.lds]) for i in range(3)]
        h = ctypes.c_void_p()
        if block_n is None:
            check(lib.gemm_grouped_plan_create(G, *arrs, *larrs, _mode(mode), _select(select),
                                               ctypes.byref(h)))
        else:
            check(lib.gemm_grouped_plan_create_config(G, *arrs, *larrs, _mode(mode), int(block_n),
                                                      int(kb if kb else 4), ctypes.byref(h)))
        self._h = h
        self.G = G

    def prepare(self, As, Bs, Cs, alphas, betas):
        """Marshal the per-problem arguments once (sequences of CUDA tensors
        or integer device pointers, and scalars); execute() without arguments
        then reuses them, so that a replay costs one C call."""
        G = self.G

        def ptr(x):
            return x if isinstance(x, int) else x.data_ptr()
        self._args = ((ctypes.c_float * G)(*[float(a) for a in alphas]),
                      (ctypes.c_void_p * G)(*[ptr(x) for x in As]),
                      (ctypes.c_void_p * G)(*[ptr(x) for x in Bs]),
                      (ctypes.c_float * G)(*[float(b) for b in betas]),
                      (ctypes.c_void_p * G)(*[ptr(x) for x in Cs]))
        return self

    def execute(self, As=None, Bs=None, Cs=None, alphas=None, betas=None, stream=None,
                graph: bool = True):
        """Run the group; with no tensors given, the prepared arguments are used."""
        if As is not None:
            self.prepare(As, Bs, Cs, alphas, betas)
        fn = self._lib.gemm_grouped_execute if graph else self._lib.gemm_grouped_execute_eager
        check(fn(self._h, *self._args, _stream_handle(stream)))

    def info(self) -> dict:
        bn, kb, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        w = ctypes.c_size_t()
        check(self._lib.gemm_grouped_plan_info(self._h, ctypes.byref(bn), ctypes.byref(kb),
                                               ctypes.byref(t), ctypes.byref(w)))
        return {"block_n": bn.value, "kb": kb.value, "tiles": t.value, "workspace_bytes": w.value}

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(self._lib.gemm_grouped_plan_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# --------------------------------------------------------- tuning and model
def _shape6(s):
    """(M, N, K) with tight leading dimensions, or (M, N, K, lda, ldb, ldc)."""
    s = [int(x) for x in s]
    if len(s) == 3:
        M, N, K = s
        return [M, N, K, max(K, 1), max(N, 1), max(N, 1)]
    if len(s) == 6:
        return s
    raise ValueError(f"a shape is (M, N, K) or (M, N, K, lda, ldb, ldc), got {s}")


def autotune(shapes, mode="bf16x3", reps: int = 5, out_path: str | None = None):
    """Time every distinct configuration of each shape ((M, N, K) with tight
    leading dimensions, or (M, N, K, lda, ldb, ldc)); rows are appended to
    out_path (CSV) and the best per shape enters the tuned table."""
    flat = [x for s in shapes for x in _shape6(s)]
    arr = _i64_array(flat) if flat else None
    check(load().gemm_autotune(arr, len(shapes), _mode(mode), int(reps),
                               out_path.encode() if out_path else None))


def autotune_load(path: str):
    check(load().gemm_autotune_load(path.encode()))


def autotune_best(M, N, K, mode="bf16x3", lda=None, ldb=None, ldc=None):
    M, N, K, lda_, ldb_, ldc_ = _shape6((M, N, K))
    cid, ms = ctypes.c_int(), ctypes.c_float()
    check(load().gemm_autotune_best(M, N, K, lda if lda is not None else lda_,
                                    ldb if ldb is not None else ldb_, ldc if ldc is not None else ldc_,
                                    _mode(mode), ctypes.byref(cid), ctypes.byref(ms)))
    return cid.value, ms.value


def select_config(M, N, K, mode="bf16x3", select="default", lda=None, ldb=None, ldc=None) -> int:
    """Configuration id a plan would get under a selection policy."""
    M, N, K, lda_, ldb_, ldc_ = _shape6((M, N, K))
    cid = ctypes.c_int()
    check(load().gemm_select_config(M, N, K, lda if lda is not None else lda_,
                                    ldb if ldb is not None else ldb_, ldc if ldc is not None else ldc_,
                                    _mode(mode), _select(select), ctypes.byref(cid)))
    return cid.value


def costmodel_feature_count() -> int:
    return load().gemm_costmodel_feature_count()


def costmodel_features(M, N, K, mode, config_id, sms=None):
    import numpy as np
    out = np.zeros(costmodel_feature_count(), dtype=np.float32)
    check(load().gemm_costmodel_features(M, N, K, _mode(mode), int(config_id),
                                         int(sms if sms else 152), out.ctypes.data))
    return out


def costmodel_train(timings_path: str, epochs: int = 2000, seed: int = 0,
                    out_model: str | None = None) -> float:
    loss = ctypes.c_float()
    check(load().gemm_costmodel_train(timings_path.encode(), int(epochs), int(seed),
                                      out_model.encode() if out_model else None,
                                      ctypes.byref(loss)))
    return loss.value


def costmodel_load(path: str):
    check(load().gemm_costmodel_load(path.encode()))


def costmodel_predict(M, N, K, mode="bf16x3"):
    cid, ms = ctypes.c_int(), ctypes.c_float()
    check(load().gemm_costmodel_predict(M, N, K, _mode(mode), ctypes.byref(cid), ctypes.byref(ms)))
    return cid.value, ms.value


def mlp_loss_grad(theta, X, t):
    """GPU loss and gradient of the cost model's MLP (float32 numpy in/out)."""
    import numpy as np
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    grad = np.zeros_like(theta)
    loss = ctypes.c_float()
    check(load().gemm_mlp_loss_grad(X.shape[0], theta.ctypes.data, X.ctypes.data, t.ctypes.data,
                                    ctypes.byref(loss), grad.ctypes.data))
    return loss.value, grad


def mlp_adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    import numpy as np
    theta = np.array(theta, dtype=np.float32)
    m = np.array(m, dtype=np.float32)
    v = np.array(v, dtype=np.float32)
    grad = np.ascontiguousarray(grad, dtype=np.float32)
    check(load().gemm_mlp_adam_step(theta.size, theta.ctypes.data, grad.ctypes.data, m.ctypes.data,
                                    v.ctypes.data, int(step), lr, beta1, beta2, eps))
    return theta, m, v
