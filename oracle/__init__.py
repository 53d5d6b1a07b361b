"""CPU oracle for the block-sparse multiply and tensor contraction (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the library's product path never does.
The oracle is plain C (``bst_oracle.c``, FP64 loops, ``-ffp-contract=off``) written from
the paper's definitions (Sec. 2 local multiply of small dense blocks, Sec. 3.1 the
transposed S_C << S_A,S_B product, Sec. 4 contraction over 1-3 index sets) and shares
no code with the CUDA library.

Every function here takes plain numpy arrays (block sizes, block index, packed data)
and returns plain numpy arrays.  All of them are pinned by ``tests/test_oracle_*.py``
against dense brute force, ``np.einsum`` and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bst_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {
    0: "OK",
    1: "INVALID_ARG",
    2: "OUT_OF_RANGE",
    3: "DUPLICATE_BLOCK",
    4: "SHAPE_MISMATCH",
    5: "OVERFLOW",
    6: "ALLOC",
}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {ERRORS.get(code, code)}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction) if needed."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                 "-std=c99", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Mat(C.Structure):
    _fields_ = [("nbr", C.c_int32), ("nbc", C.c_int32),
                ("rsz", C.c_void_p), ("csz", C.c_void_p),
                ("nblocks", C.c_int64), ("brow", C.c_void_p), ("bcol", C.c_void_p),
                ("data", C.c_void_p)]


class _Ten(C.Structure):
    _fields_ = [("rank", C.c_int32), ("nblk", C.c_void_p), ("bsz", C.c_void_p),
                ("nblocks", C.c_int64), ("idx", C.c_void_p), ("data", C.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        vp = C.c_void_p
        lib.or_block_norms.argtypes = [vp, vp]
        lib.or_multiply.argtypes = [C.c_char, C.c_char, vp, vp, vp, C.c_double, C.c_double,
                                    C.c_double, C.POINTER(vp)]
        lib.or_multiply_sample.argtypes = [C.c_char, C.c_char, vp, vp, vp, C.c_double,
                                           C.c_double, C.c_double, C.c_int64, vp, vp, vp, vp]
        lib.or_multiply_adjoint.argtypes = [C.c_char, C.c_char, vp, vp, vp, C.c_double,
                                            C.c_double, C.c_double, vp, vp, vp, vp]
        lib.or_result_sizes.argtypes = [vp, vp]
        lib.or_result_flops.argtypes = [vp]
        lib.or_result_flops.restype = C.c_double
        lib.or_result_get.argtypes = [vp] * 10
        lib.or_result_free.argtypes = [vp]
        lib.or_contract.argtypes = [vp, vp, C.c_int32, vp, vp, C.c_int32, vp, C.c_int32, vp, vp,
                                    vp, C.c_double, C.c_double, C.c_double, C.POINTER(vp)]
        lib.or_contract_adjoint.argtypes = [vp, vp, C.c_int32, vp, vp, C.c_int32, vp, C.c_int32,
                                            vp, vp, vp, C.c_double, C.c_double, C.c_double, vp,
                                            vp, vp, vp]
        lib.or_contract_sample.argtypes = [vp, vp, C.c_int32, vp, vp, C.c_int32, vp, C.c_int32,
                                           vp, vp, vp, C.c_double, C.c_double, C.c_double,
                                           C.c_int64, vp, vp, vp]
        lib.or_tresult_sizes.argtypes = [vp, vp]
        lib.or_tresult_flops.argtypes = [vp]
        lib.or_tresult_flops.restype = C.c_double
        lib.or_tresult_get.argtypes = [vp, vp, vp, vp]
        lib.or_tresult_free.argtypes = [vp]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class _MatArgs:
    """Holds the contiguous arrays alive for as long as the ctypes struct is used."""

    def __init__(self, row_sizes, col_sizes, rows, cols, data):
        self.rs = np.ascontiguousarray(row_sizes, dtype=np.int32)
        self.cs = np.ascontiguousarray(col_sizes, dtype=np.int32)
        self.r = np.ascontiguousarray(rows, dtype=np.int32)
        self.c = np.ascontiguousarray(cols, dtype=np.int32)
        self.d = np.ascontiguousarray(data, dtype=np.float64)
        self.s = _Mat(len(self.rs), len(self.cs), _p(self.rs), _p(self.cs), len(self.r),
                      _p(self.r), _p(self.c), _p(self.d))

    @property
    def ref(self):
        return C.byref(self.s)


def _mat(m):
    """Accepts any object with row_sizes, col_sizes, rows, cols, data attributes."""
    if m is None:
        return None
    return _MatArgs(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)


def block_norms(m) -> np.ndarray:
    """Frobenius norm of every block, in canonical (row, col) order."""
    lib = _load()
    a = _mat(m)
    out = np.empty(len(a.r), dtype=np.float64)
    st = lib.or_block_norms(a.ref, _p(out))
    if st:
        raise OracleError(st, "block_norms")
    return out


def multiply(A, B, C_in=None, alpha=1.0, beta=0.0, eps=0.0, transa="N", transb="N"):
    """C_out = alpha*op(A)*op(B) + beta*C_in with the block-norm filter eps.

    Returns a dict with the C_out pattern (rows, cols, offsets), its packed data, and
    the stacks: mnk (nbuckets x 3), bucket_ptr, a_off, b_off, c_off, plus counters.
    """
    lib = _load()
    a, b, c = _mat(A), _mat(B), _mat(C_in)
    res = C.c_void_p()
    st = lib.or_multiply(transa.encode(), transb.encode(), a.ref, b.ref,
                         c.ref if c else None, alpha, beta, eps, C.byref(res))
    if st:
        raise OracleError(st, "multiply")
    try:
        sz = np.zeros(6, dtype=np.int64)
        lib.or_result_sizes(res, _p(sz))
        nblk, nel, nst, nbk = (int(x) for x in sz[:4])
        out = dict(
            rows=np.empty(nblk, np.int32), cols=np.empty(nblk, np.int32),
            offsets=np.empty(nblk, np.int64), data=np.empty(nel, np.float64),
            mnk=np.empty((nbk, 3), np.int32), bucket_ptr=np.empty(nbk + 1, np.int64),
            a_off=np.empty(nst, np.int32), b_off=np.empty(nst, np.int32),
            c_off=np.empty(nst, np.int32))
        lib.or_result_get(res, *(_p(out[k]) for k in (
            "rows", "cols", "offsets", "data", "mnk", "bucket_ptr", "a_off", "b_off", "c_off")))
        out["ncandidates"] = int(sz[4])
        out["nfiltered"] = int(sz[5])
        out["flops"] = float(lib.or_result_flops(res))
        return out
    finally:
        lib.or_result_free(res)


def multiply_sample(A, B, C_in, alpha, beta, eps, bi, bj, transa="N", transb="N",
                    row_sizes=None, col_sizes=None):
    """Values of the requested C_out blocks (bi[e], bj[e]) only, same definition as
    :func:`multiply`.  Returns (packed values in request order, present flags)."""
    lib = _load()
    a, b, c = _mat(A), _mat(B), _mat(C_in)
    bi = np.ascontiguousarray(bi, np.int32)
    bj = np.ascontiguousarray(bj, np.int32)
    m = np.asarray(row_sizes)[bi].astype(np.int64)
    n = np.asarray(col_sizes)[bj].astype(np.int64)
    out = np.empty(int((m * n).sum()), np.float64)
    present = np.empty(len(bi), np.int8)
    st = lib.or_multiply_sample(transa.encode(), transb.encode(), a.ref, b.ref,
                                c.ref if c else None, alpha, beta, eps, len(bi), _p(bi), _p(bj),
                                _p(out), _p(present))
    if st:
        raise OracleError(st, "multiply_sample")
    return out, present.astype(bool)


def multiply_adjoint(A, B, C_in, alpha, beta, eps, dC, transa="N", transb="N"):
    """(dA, dB, dC_in) of the filtered product, in the stored packing of each input."""
    lib = _load()
    a, b, c = _mat(A), _mat(B), _mat(C_in)
    dC = np.ascontiguousarray(dC, np.float64)
    dA = np.empty(len(a.d), np.float64)
    dB = np.empty(len(b.d), np.float64)
    dCi = np.empty(len(c.d), np.float64) if c else None
    st = lib.or_multiply_adjoint(transa.encode(), transb.encode(), a.ref, b.ref,
                                 c.ref if c else None, alpha, beta, eps, _p(dC), _p(dA), _p(dB),
                                 _p(dCi))
    if st:
        raise OracleError(st, "multiply_adjoint")
    return dA, dB, dCi


class _TenArgs:
    def __init__(self, t):
        self.nblk = np.ascontiguousarray([len(s) for s in t.block_sizes], np.int32)
        self.bsz = np.ascontiguousarray(np.concatenate(
            [np.asarray(s, np.int32) for s in t.block_sizes]), np.int32)
        self.idx = np.ascontiguousarray(t.index, np.int32).reshape(-1)
        self.d = np.ascontiguousarray(t.data, np.float64)
        rank = len(t.block_sizes)
        self.s = _Ten(rank, _p(self.nblk), _p(self.bsz), len(self.idx) // max(rank, 1),
                      _p(self.idx), _p(self.d))

    @property
    def ref(self):
        return C.byref(self.s)


def _i32(x):
    return np.ascontiguousarray(x, np.int32)


def contract(T1, T2, c1, c2, f1, f2, result_order=None, R_in=None, alpha=1.0, beta=0.0,
             eps=0.0):
    """R = alpha * sum_{contracted} T1*T2 + beta*R_in over the kept block pairs.

    Tensors are objects with ``block_sizes`` (list of per-mode arrays), ``index``
    (nblocks x rank) and ``data``.  Returns dict(index, offsets, data, npairs,
    nfiltered, flops, block_sizes)."""
    lib = _load()
    t1, t2 = _TenArgs(T1), _TenArgs(T2)
    ri = _TenArgs(R_in) if R_in is not None else None
    c1, c2, f1, f2 = _i32(c1), _i32(c2), _i32(f1), _i32(f2)
    ro = _i32(result_order) if result_order is not None else None
    res = C.c_void_p()
    st = lib.or_contract(t1.ref, t2.ref, len(c1), _p(c1), _p(c2), len(f1), _p(f1), len(f2),
                         _p(f2), _p(ro), ri.ref if ri else None, alpha, beta, eps,
                         C.byref(res))
    if st:
        raise OracleError(st, "contract")
    try:
        sz = np.zeros(5, np.int64)
        lib.or_tresult_sizes(res, _p(sz))
        rank, nblk, nel = int(sz[0]), int(sz[1]), int(sz[2])
        out = dict(index=np.empty((nblk, rank), np.int32), offsets=np.empty(nblk, np.int64),
                   data=np.empty(nel, np.float64))
        lib.or_tresult_get(res, _p(out["index"]), _p(out["offsets"]), _p(out["data"]))
        out["npairs"] = int(sz[3])
        out["nfiltered"] = int(sz[4])
        out["flops"] = float(lib.or_tresult_flops(res))
        return out
    finally:
        lib.or_tresult_free(res)


def contract_sample(T1, T2, c1, c2, f1, f2, result_order, R_in, alpha, beta, eps, req,
                    result_block_sizes):
    """Values of the requested result blocks (req: nreq x rank tuples in result order),
    same definition as :func:`contract`.  Returns (packed values, present flags)."""
    lib = _load()
    t1, t2 = _TenArgs(T1), _TenArgs(T2)
    ri = _TenArgs(R_in) if R_in is not None else None
    c1, c2, f1, f2 = _i32(c1), _i32(c2), _i32(f1), _i32(f2)
    ro = _i32(result_order) if result_order is not None else None
    req = np.ascontiguousarray(req, np.int32)
    lens = np.ones(len(req), np.int64)
    for d, sz in enumerate(result_block_sizes):
        lens *= np.asarray(sz, np.int64)[req[:, d]]
    out = np.empty(int(lens.sum()), np.float64)
    present = np.empty(len(req), np.int8)
    st = lib.or_contract_sample(t1.ref, t2.ref, len(c1), _p(c1), _p(c2), len(f1), _p(f1),
                                len(f2), _p(f2), _p(ro), ri.ref if ri else None, alpha, beta,
                                eps, len(req), _p(req), _p(out), _p(present))
    if st:
        raise OracleError(st, "contract_sample")
    return out, present.astype(bool)


def contract_adjoint(T1, T2, c1, c2, f1, f2, result_order, R_in, alpha, beta, eps, dR):
    """(dT1, dT2, dR_in) of the filtered contraction, each in its tensor's packing."""
    lib = _load()
    t1, t2 = _TenArgs(T1), _TenArgs(T2)
    ri = _TenArgs(R_in) if R_in is not None else None
    c1, c2, f1, f2 = _i32(c1), _i32(c2), _i32(f1), _i32(f2)
    ro = _i32(result_order) if result_order is not None else None
    dR = np.ascontiguousarray(dR, np.float64)
    d1 = np.empty(len(t1.d), np.float64)
    d2 = np.empty(len(t2.d), np.float64)
    dri = np.empty(len(ri.d), np.float64) if ri else None
    st = lib.or_contract_adjoint(t1.ref, t2.ref, len(c1), _p(c1), _p(c2), len(f1), _p(f1),
                                 len(f2), _p(f2), _p(ro), ri.ref if ri else None, alpha, beta,
                                 eps, _p(dR), _p(d1), _p(d2), _p(dri))
    if st:
        raise OracleError(st, "contract_adjoint")
    return d1, d2, dri


class _Blocks:
    """A block-sparse matrix as plain arrays (the attribute names of the generators')."""

    def __init__(self, row_sizes, col_sizes, rows, cols, data):
        self.row_sizes = np.ascontiguousarray(row_sizes, np.int32)
        self.col_sizes = np.ascontiguousarray(col_sizes, np.int32)
        self.rows = np.ascontiguousarray(rows, np.int32)
        self.cols = np.ascontiguousarray(cols, np.int32)
        self.data = np.ascontiguousarray(data, np.float64)
        self.nblocks = len(self.rows)


def filter_blocks(m, eps):
    """Post-filter, a reading (the paper names the sign iteration, Sec. 2, but defines
    no filter on a product's result): the blocks of m, in canonical order, whose
    Frobenius norm (the same norm as the product filter) is >= eps; data unchanged."""
    norms = block_norms(m)
    lens = (np.asarray(m.row_sizes, np.int64)[np.asarray(m.rows)] *
            np.asarray(m.col_sizes, np.int64)[np.asarray(m.cols)])
    starts = np.concatenate([[0], np.cumsum(lens)])
    keep = norms >= eps
    data = [np.asarray(m.data)[starts[b]:starts[b + 1]] for b in range(len(lens)) if keep[b]]
    return _Blocks(m.row_sizes, m.col_sizes, np.asarray(m.rows)[keep], np.asarray(m.cols)[keep],
                   np.concatenate(data) if data else np.zeros(0))


def sign_iteration(X, iters, eps=0.0, eps_post=0.0):
    """The matrix-sign Newton-Schulz iteration X <- (3 X - X^3) / 2 as a chain of filtered
    block-sparse products: T = filter(X X), X <- filter(-1/2 T X + 3/2 X), each product
    with the block-norm filter eps and each result with the post-filter eps_post.
    Returns the list of iterates (X_1 .. X_iters)."""
    out = []
    for _ in range(iters):
        t = multiply(X, X, None, 1.0, 0.0, eps)
        T = filter_blocks(_Blocks(X.row_sizes, X.col_sizes, t["rows"], t["cols"], t["data"]),
                          eps_post)
        x = multiply(T, X, X, -0.5, 1.5, eps)
        X = filter_blocks(_Blocks(X.row_sizes, X.col_sizes, x["rows"], x["cols"], x["data"]),
                          eps_post)
        out.append(X)
    return out
