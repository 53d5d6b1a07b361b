"""ctypes binding of libbst (include/bst.h) -- argument marshalling only.

Every ``bst_*`` function here has the name, arguments and meaning of the C entry point
of the same name; handles are ``ctypes.c_void_p``.  Device buffers are torch CUDA
tensors (passed as their data pointers); streams are torch streams (or raw
``cudaStream_t`` integers).  Every call raises :class:`BstError` when the library
returns an error status.

On top of the raw calls, :class:`Matrix`, :class:`Tensor` and :func:`multiply` keep a
handle together with the torch tensor that owns its data.  All compute happens in
the library's CUDA kernels; there is no CPU path here.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbst.so")
_lock = threading.Lock()
_lib = None

BST_FP64 = 0
BST_FP64_EMU_BF16 = 1
BST_TF32X3 = 2
PRECISIONS = {"fp64": BST_FP64, "emu_bf16": BST_FP64_EMU_BF16, "tf32x3": BST_TF32X3}


class BstError(RuntimeError):
    def __init__(self, code: int, name: str, msg: str, what: str):
        super().__init__(f"{what}: {name}: {msg}")
        self.code = code
        self.name = name


class bst_stats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_filtered", C.c_int64), ("n_stack", C.c_int64),
                ("n_c_blocks", C.c_int64), ("n_c_elements", C.c_int64),
                ("n_buckets", C.c_int32), ("split_k", C.c_int32),
                ("flops", C.c_double), ("bytes", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_VP = C.c_void_p
_SIGS = {
    "bst_last_error": ([], C.c_char_p),
    "bst_status_name": ([C.c_int32], C.c_char_p),
    "bst_version": ([], C.c_char_p),
    "bst_kernel_launches": ([], C.c_int64),
    "bst_context_create": ([C.POINTER(_VP), C.c_int32, ALLOC_FN, FREE_FN, _VP], C.c_int32),
    "bst_context_destroy": ([_VP], C.c_int32),
    "bst_matrix_create": ([_VP, C.POINTER(_VP), C.c_int32, _VP, C.c_int32, _VP, C.c_int64, _VP,
                           _VP, _VP, _VP], C.c_int32),
    "bst_matrix_info": ([_VP, _VP, _VP, _VP, _VP], C.c_int32),
    "bst_matrix_get_index": ([_VP, _VP, _VP, _VP], C.c_int32),
    "bst_matrix_bind_data": ([_VP, _VP], C.c_int32),
    "bst_matrix_destroy": ([_VP], C.c_int32),
    "bst_matrix_data_size": ([_VP, _VP], C.c_int32),
    "bst_multiply_adjoint": ([_VP, _VP, _VP, _VP, C.c_double, _VP], C.c_int32),
    "bst_matrix_filter": ([_VP, _VP, C.c_double, _VP, C.POINTER(_VP)], C.c_int32),
    "bst_matrix_filter_copy": ([_VP, _VP, _VP], C.c_int32),
    "bst_multiply_plan": ([_VP, C.c_char, C.c_char, _VP, _VP, _VP, C.c_double, _VP,
                           C.POINTER(_VP)], C.c_int32),
    "bst_plan_result": ([_VP, C.POINTER(_VP)], C.c_int32),
    "bst_plan_stats": ([_VP, C.POINTER(bst_stats)], C.c_int32),
    "bst_plan_get_stacks": ([_VP, _VP, _VP, _VP, _VP, _VP], C.c_int32),
    "bst_plan_split_histogram": ([_VP, _VP], C.c_int32),
    "bst_plan_schedule_info": ([_VP, _VP], C.c_int32),
    "bst_plan_emu_costs": ([_VP, _VP], C.c_int32),
    "bst_multiply_execute": ([_VP, C.c_double, C.c_double, C.c_int32, C.c_int32, _VP], C.c_int32),
    "bst_multiply_execute_static": ([_VP, C.c_double, C.c_double, C.c_int32, _VP], C.c_int32),
    "bst_static_scratch_doubles": ([], C.c_size_t),
    "bst_plan_adjoint": ([_VP, _VP, _VP, _VP, _VP, C.c_double, C.c_double, _VP], C.c_int32),
    "bst_plan_destroy": ([_VP], C.c_int32),
    "bst_tune_set": ([_VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32], C.c_int32),
    "bst_tune_get": ([_VP, C.c_int32, C.c_int32, C.c_int32, _VP], C.c_int32),
    "bst_tensor_create": ([_VP, C.POINTER(_VP), C.c_int32, _VP, _VP, C.c_int64, _VP, _VP, _VP],
                          C.c_int32),
    "bst_tensor_info": ([_VP, _VP, _VP, _VP], C.c_int32),
    "bst_tensor_get_index": ([_VP, _VP, _VP], C.c_int32),
    "bst_tensor_bind_data": ([_VP, _VP], C.c_int32),
    "bst_tensor_destroy": ([_VP], C.c_int32),
    "bst_contract_plan": ([_VP, _VP, _VP, C.c_int32, _VP, _VP, C.c_int32, _VP, C.c_int32, _VP,
                           _VP, _VP, C.c_double, _VP, C.POINTER(_VP)], C.c_int32),
    "bst_plan_result_tensor": ([_VP, C.POINTER(_VP)], C.c_int32),
    "bst_batch_create": ([_VP, C.c_int32, _VP, C.POINTER(_VP)], C.c_int32),
    "bst_batch_execute": ([_VP, _VP, _VP, C.c_int32, _VP], C.c_int32),
    "bst_batch_destroy": ([_VP], C.c_int32),
    "bst_sum_parts": ([_VP, C.c_int32, C.c_int64, _VP, _VP, _VP, _VP, _VP], C.c_int32),
    "bst_debug_wait_probe": ([_VP, C.c_int64, _VP], C.c_int32),
}


def load():
    """Load libbst.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1910_13555_gb300.build.build()")
            lib = C.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(st, what):
    if st:
        lib = load()
        raise BstError(st, lib.bst_status_name(st).decode(), lib.bst_last_error().decode(), what)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


# ---- raw calls (same names as the C ABI) ------------------------------------------


def bst_version() -> str:
    return load().bst_version().decode()


def bst_kernel_launches() -> int:
    return int(load().bst_kernel_launches())


def bst_context_create(device: int = 0, alloc=None, free=None, user=None):
    h = C.c_void_p()
    a = ALLOC_FN(alloc) if alloc else C.cast(None, ALLOC_FN)
    f = FREE_FN(free) if free else C.cast(None, FREE_FN)
    _check(load().bst_context_create(C.byref(h), device, a, f, user), "bst_context_create")
    h._keep = (a, f)
    return h


def bst_context_destroy(ctx):
    _check(load().bst_context_destroy(ctx), "bst_context_destroy")


def bst_matrix_create(ctx, row_sizes, col_sizes, rows, cols, data=None, stream=None):
    rs, cs, r, c = _i32(row_sizes), _i32(col_sizes), _i32(rows), _i32(cols)
    h = C.c_void_p()
    _check(load().bst_matrix_create(ctx, C.byref(h), len(rs), _ptr(rs), len(cs), _ptr(cs), len(r),
                                    _ptr(r), _ptr(c), _ptr(data), _stream(stream)),
           "bst_matrix_create")
    return h


def bst_matrix_info(m):
    nbr, nbc, nb, ne = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
    _check(load().bst_matrix_info(m, C.byref(nbr), C.byref(nbc), C.byref(nb), C.byref(ne)),
           "bst_matrix_info")
    return nbr.value, nbc.value, nb.value, ne.value


def bst_matrix_get_index(m):
    _, _, nb, _ = bst_matrix_info(m)
    r = np.empty(nb, np.int32)
    c = np.empty(nb, np.int32)
    o = np.empty(nb, np.int64)
    _check(load().bst_matrix_get_index(m, _ptr(r), _ptr(c), _ptr(o)), "bst_matrix_get_index")
    return r, c, o


def bst_matrix_bind_data(m, data):
    _check(load().bst_matrix_bind_data(m, _ptr(data)), "bst_matrix_bind_data")


def bst_matrix_destroy(m):
    _check(load().bst_matrix_destroy(m), "bst_matrix_destroy")


def bst_matrix_data_size(m) -> int:
    v = C.c_int64()
    _check(load().bst_matrix_data_size(m, C.byref(v)), "bst_matrix_data_size")
    return v.value


def bst_multiply_adjoint(plan, dC, dA, dB, alpha=1.0, stream=None):
    _check(load().bst_multiply_adjoint(plan, _ptr(dC), _ptr(dA), _ptr(dB), float(alpha),
                                       _stream(stream)), "bst_multiply_adjoint")


def bst_matrix_filter(ctx, X, eps, stream=None):
    h = C.c_void_p()
    _check(load().bst_matrix_filter(ctx, X, float(eps), _stream(stream), C.byref(h)),
           "bst_matrix_filter")
    return h


def bst_matrix_filter_copy(X, Y, stream=None):
    _check(load().bst_matrix_filter_copy(X, Y, _stream(stream)), "bst_matrix_filter_copy")


def bst_multiply_plan(ctx, transa, transb, A, B, C_in=None, eps=0.0, stream=None):
    h = C.c_void_p()
    _check(load().bst_multiply_plan(ctx, transa.encode(), transb.encode(), A, B, C_in, eps,
                                    _stream(stream), C.byref(h)), "bst_multiply_plan")
    return h


def bst_plan_result(plan):
    h = C.c_void_p()
    _check(load().bst_plan_result(plan, C.byref(h)), "bst_plan_result")
    return h


def bst_plan_stats(plan) -> dict:
    s = bst_stats()
    _check(load().bst_plan_stats(plan, C.byref(s)), "bst_plan_stats")
    return s.as_dict()


def bst_plan_split_histogram(plan) -> np.ndarray:
    """hist[s]: staged FP64 tiles split over s lane groups; hist[0]: direct-load blocks."""
    h = np.zeros(17, np.int64)
    _check(load().bst_plan_split_histogram(plan, _ptr(h)), "bst_plan_split_histogram")
    return h


def bst_plan_schedule_info(plan) -> dict:
    """How the plan's native-FP64 execute runs: staged kernel, strided staging, inner
    split, slab reading of A."""
    v = np.zeros(4, np.int32)
    _check(load().bst_plan_schedule_info(plan, _ptr(v)), "bst_plan_schedule_info")
    return dict(staged=bool(v[0]), strided=bool(v[1]), split=bool(v[2]), slab=bool(v[3]))


def bst_plan_emu_costs(plan) -> dict:
    out = np.zeros(4, np.float64)
    _check(load().bst_plan_emu_costs(plan, _ptr(out)), "bst_plan_emu_costs")
    return {"tensor_flops": float(out[0]), "bytes": float(out[1]),
            "intermediate_bytes": float(out[2]), "panel": bool(out[3])}


def bst_plan_get_stacks(plan):
    st = bst_plan_stats(plan)
    nb, ns = st["n_buckets"], st["n_stack"]
    mnk = np.empty((nb, 3), np.int32)
    bp = np.empty(nb + 1, np.int64)
    a = np.empty(ns, np.int32)
    b = np.empty(ns, np.int32)
    c = np.empty(ns, np.int32)
    _check(load().bst_plan_get_stacks(plan, _ptr(mnk), _ptr(bp), _ptr(a), _ptr(b), _ptr(c)),
           "bst_plan_get_stacks")
    return dict(mnk=mnk, bucket_ptr=bp, a_off=a, b_off=b, c_off=c)


def bst_multiply_execute(plan, alpha=1.0, beta=0.0, precision=BST_FP64, split_k=1, stream=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    _check(load().bst_multiply_execute(plan, alpha, beta, precision, split_k, _stream(stream)),
           "bst_multiply_execute")


def bst_multiply_execute_static(plan, alpha=1.0, beta=0.0, split_k=1, stream=None):
    _check(load().bst_multiply_execute_static(plan, alpha, beta, split_k, _stream(stream)),
           "bst_multiply_execute_static")


def bst_static_scratch_doubles() -> int:
    return int(load().bst_static_scratch_doubles())


def bst_plan_adjoint(plan, dC, dA, dB, dC_in=None, alpha=1.0, beta=0.0, stream=None):
    _check(load().bst_plan_adjoint(plan, _ptr(dC), _ptr(dA), _ptr(dB), _ptr(dC_in), alpha, beta,
                                   _stream(stream)), "bst_plan_adjoint")


def bst_plan_destroy(plan):
    _check(load().bst_plan_destroy(plan), "bst_plan_destroy")


BST_TUNE_EMU_ROW_SCALE = 0
BST_TUNE_EMU_SWAP = 1
BST_TUNE_F64_SPLIT = 2
BST_TUNE_CONTRACT_SLAB = 3
BST_TUNE_EMU_PANEL = 4


def bst_tune_set(ctx, key, value, m=0, n=0):
    _check(load().bst_tune_set(ctx, key, m, n, value), "bst_tune_set")


def bst_tune_get(ctx, key, m=0, n=0) -> int:
    v = C.c_int32()
    _check(load().bst_tune_get(ctx, key, m, n, C.byref(v)), "bst_tune_get")
    return v.value


def bst_tensor_create(ctx, block_sizes, index, data=None, stream=None):
    nblk = _i32([len(s) for s in block_sizes])
    bsz = _i32(np.concatenate([_i32(s) for s in block_sizes])) if len(block_sizes) else _i32([])
    idx = _i32(index).reshape(-1)
    rank = len(block_sizes)
    nb = idx.size // max(rank, 1)
    h = C.c_void_p()
    _check(load().bst_tensor_create(ctx, C.byref(h), rank, _ptr(nblk), _ptr(bsz), nb, _ptr(idx),
                                    _ptr(data), _stream(stream)), "bst_tensor_create")
    return h


def bst_tensor_info(t):
    r, nb, ne = C.c_int32(), C.c_int64(), C.c_int64()
    _check(load().bst_tensor_info(t, C.byref(r), C.byref(nb), C.byref(ne)), "bst_tensor_info")
    return r.value, nb.value, ne.value


def bst_tensor_get_index(t):
    rank, nb, _ = bst_tensor_info(t)
    idx = np.empty((nb, rank), np.int32)
    off = np.empty(nb, np.int64)
    _check(load().bst_tensor_get_index(t, _ptr(idx), _ptr(off)), "bst_tensor_get_index")
    return idx, off


def bst_tensor_bind_data(t, data):
    _check(load().bst_tensor_bind_data(t, _ptr(data)), "bst_tensor_bind_data")


def bst_tensor_destroy(t):
    _check(load().bst_tensor_destroy(t), "bst_tensor_destroy")


def bst_contract_plan(ctx, T1, T2, c1, c2, f1, f2, result_order=None, R_in=None, eps=0.0,
                      stream=None):
    c1, c2, f1, f2 = _i32(c1), _i32(c2), _i32(f1), _i32(f2)
    ro = _i32(result_order) if result_order is not None else None
    h = C.c_void_p()
    _check(load().bst_contract_plan(ctx, T1, T2, len(c1), _ptr(c1), _ptr(c2), len(f1), _ptr(f1),
                                    len(f2), _ptr(f2), _ptr(ro), R_in, eps, _stream(stream),
                                    C.byref(h)), "bst_contract_plan")
    return h


def bst_plan_result_tensor(plan):
    h = C.c_void_p()
    _check(load().bst_plan_result_tensor(plan, C.byref(h)), "bst_plan_result_tensor")
    return h


def bst_batch_create(ctx, plans):
    arr = (C.c_void_p * len(plans))(*[p.value for p in plans])
    h = C.c_void_p()
    _check(load().bst_batch_create(ctx, len(plans), arr, C.byref(h)), "bst_batch_create")
    return h


def bst_batch_execute(batch, alpha, beta, precision=BST_FP64, stream=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    a = np.ascontiguousarray(alpha, np.float64)
    b = np.ascontiguousarray(beta, np.float64)
    _check(load().bst_batch_execute(batch, _ptr(a), _ptr(b), precision, _stream(stream)),
           "bst_batch_execute")


def bst_batch_destroy(batch):
    _check(load().bst_batch_destroy(batch), "bst_batch_destroy")


def bst_debug_wait_probe(ctx, bound_ns, stream=None):
    _check(load().bst_debug_wait_probe(ctx, int(bound_ns), _stream(stream)),
           "bst_debug_wait_probe")


def bst_sum_parts(ctx, nparts, nblocks, dst_off, src_off, src, dst, stream=None):
    """dst_off (int64, nblocks + 1), src_off (int64, nparts * nblocks), src, dst: device
    tensors (FP64 for src and dst)."""
    _check(load().bst_sum_parts(ctx, int(nparts), int(nblocks), _ptr(dst_off), _ptr(src_off),
                                _ptr(src), _ptr(dst), _stream(stream)), "bst_sum_parts")


# ---- convenience wrappers -----------------------------------------------------------

_ctx_cache = {}


def context(device: int = 0):
    """A process-wide context per device (stream-ordered cudaMallocAsync allocator)."""
    if device not in _ctx_cache:
        _ctx_cache[device] = bst_context_create(device)
    return _ctx_cache[device]


class Matrix:
    """A library matrix handle with the torch tensor that owns its data."""

    def __init__(self, handle, data, owned=True):
        self.handle = handle
        self.data = data
        self.owned = owned

    @classmethod
    def from_host(cls, row_sizes, col_sizes, rows, cols, data, device=0, stream=None):
        import torch
        d = torch.as_tensor(np.ascontiguousarray(data, np.float64)).to(f"cuda:{device}")
        h = bst_matrix_create(context(device), row_sizes, col_sizes, rows, cols, d, stream)
        return cls(h, d)

    @property
    def info(self):
        return bst_matrix_info(self.handle)

    def index(self):
        return bst_matrix_get_index(self.handle)

    def __del__(self):
        if getattr(self, "owned", False) and self.handle:
            try:
                bst_matrix_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


class Plan:
    """A multiply or contraction plan; ``result`` is the C_out matrix (pattern + data)."""

    def __init__(self, handle, keep=()):
        self.handle = handle
        self._keep = keep
        self.result = None

    def stats(self):
        return bst_plan_stats(self.handle)

    def stacks(self):
        return bst_plan_get_stacks(self.handle)

    def split_histogram(self):
        return bst_plan_split_histogram(self.handle)

    def schedule_info(self):
        return bst_plan_schedule_info(self.handle)

    def alloc_result(self, device=0):
        import torch
        h = bst_plan_result(self.handle)
        _, _, _, ne = bst_matrix_info(h)
        d = torch.empty(max(ne, 1), dtype=torch.float64, device=f"cuda:{device}")
        bst_matrix_bind_data(h, d)
        self.result = Matrix(h, d, owned=False)
        return self.result

    def execute(self, alpha=1.0, beta=0.0, precision=BST_FP64, split_k=1, stream=None):
        bst_multiply_execute(self.handle, alpha, beta, precision, split_k, stream)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                bst_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


class Tensor:
    """A library tensor handle with the torch tensor that owns its data."""

    def __init__(self, handle, data, owned=True):
        self.handle = handle
        self.data = data
        self.owned = owned

    @classmethod
    def from_host(cls, block_sizes, index, data, device=0, stream=None):
        import torch
        d = torch.as_tensor(np.ascontiguousarray(data, np.float64)).to(f"cuda:{device}")
        h = bst_tensor_create(context(device), block_sizes, index, d, stream)
        return cls(h, d)

    @property
    def info(self):
        return bst_tensor_info(self.handle)

    def index(self):
        return bst_tensor_get_index(self.handle)

    def __del__(self):
        if getattr(self, "owned", False) and self.handle:
            try:
                bst_tensor_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


class ContractPlan(Plan):
    """A contraction plan; ``result`` is the result tensor (pattern + data)."""

    def alloc_result(self, device=0):
        import torch
        h = bst_plan_result_tensor(self.handle)
        _, _, ne = bst_tensor_info(h)
        d = torch.empty(max(ne, 1), dtype=torch.float64, device=f"cuda:{device}")
        bst_tensor_bind_data(h, d)
        self.result = Tensor(h, d, owned=False)
        return self.result


def contract_plan(T1: Tensor, T2: Tensor, c1, c2, f1, f2, result_order=None,
                  R_in: Tensor | None = None, eps=0.0, device=0, stream=None) -> ContractPlan:
    h = bst_contract_plan(context(device), T1.handle, T2.handle, c1, c2, f1, f2, result_order,
                          R_in.handle if R_in is not None else None, eps, stream)
    return ContractPlan(h, keep=(T1, T2, R_in))


def contract(T1: Tensor, T2: Tensor, c1, c2, f1, f2, result_order=None, R_in=None, alpha=1.0,
             beta=0.0, eps=0.0, precision=BST_FP64, split_k=1, device=0, stream=None):
    """Plan + allocate the result tensor + execute; returns the plan (``plan.result``)."""
    p = contract_plan(T1, T2, c1, c2, f1, f2, result_order, R_in, eps, device, stream)
    p.alloc_result(device)
    p.execute(alpha, beta, precision, split_k, stream)
    return p


def filter_blocks(X: Matrix, eps, device=0, stream=None) -> Matrix:
    """The blocks of X with Frobenius norm >= eps, as a new matrix with its own data."""
    import torch
    h = bst_matrix_filter(context(device), X.handle, eps, stream)
    _, _, _, ne = bst_matrix_info(h)
    d = torch.empty(max(ne, 1), dtype=torch.float64, device=f"cuda:{device}")
    bst_matrix_bind_data(h, d)
    bst_matrix_filter_copy(X.handle, h, stream)
    return Matrix(h, d)


def multiply_plan(A: Matrix, B: Matrix, C_in: Matrix | None = None, eps=0.0, transa="N",
                  transb="N", device=0, stream=None) -> Plan:
    h = bst_multiply_plan(context(device), transa, transb, A.handle, B.handle,
                          C_in.handle if C_in is not None else None, eps, stream)
    return Plan(h, keep=(A, B, C_in))


def multiply(A: Matrix, B: Matrix, C_in: Matrix | None = None, alpha=1.0, beta=0.0, eps=0.0,
             transa="N", transb="N", precision=BST_FP64, split_k=1, device=0, stream=None):
    """Plan + allocate C_out + execute; returns the plan (``plan.result`` is C_out)."""
    p = multiply_plan(A, B, C_in, eps, transa, transb, device, stream)
    p.alloc_result(device)
    p.execute(alpha, beta, precision, split_k, stream)
    return p
