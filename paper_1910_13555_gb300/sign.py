"""Chained filtered block-sparse products: the matrix-sign Newton-Schulz iteration.

Paper Sec. 2 names the sign-matrix iteration among DBCSR's operations (linear-scaling
DFT takes the density matrix from the matrix sign function, computed by iterations made of
block-sparse products).  The paper defines no filter; here sparsity is kept by the
library's two readings: the block-norm filter of each product (eps of the multiply) and a
post-filter that drops the result blocks of norm below eps_post.  One step here is

    T = filter(X X, eps_post)
    X <- filter(-1/2 T X + 3/2 X, eps_post)        (= (3 X - X^3) / 2)

with every product planned and executed by the library (symbolic phase, stacks and the
numeric kernels on the GPU) and the post-filter run by bst_matrix_filter on the GPU; this
module only sequences the calls.
"""
from __future__ import annotations

from . import bst


def sign_step(X: bst.Matrix, eps=0.0, eps_post=0.0, precision=bst.BST_FP64, device=0,
              stream=None):
    """One Newton-Schulz step; returns (X_next, stats) with the flops of the two products."""
    p1 = bst.multiply(X, X, None, 1.0, 0.0, eps, precision=precision, device=device,
                      stream=stream)
    T = bst.filter_blocks(p1.result, eps_post, device, stream)
    p2 = bst.multiply(T, X, X, -0.5, 1.5, eps, precision=precision, device=device, stream=stream)
    Xn = bst.filter_blocks(p2.result, eps_post, device, stream)
    flops = p1.stats()["flops"] + p2.stats()["flops"]
    return Xn, {"flops": flops, "blocks_T": T.info[2], "blocks_X": Xn.info[2]}


def sign_iteration(X: bst.Matrix, iters, eps=0.0, eps_post=0.0, precision=bst.BST_FP64,
                   device=0, stream=None):
    """`iters` Newton-Schulz steps from X; returns the iterates and per-step statistics."""
    xs, stats = [], []
    for _ in range(iters):
        X, st = sign_step(X, eps, eps_post, precision, device, stream)
        xs.append(X)
        stats.append(st)
    return xs, stats
