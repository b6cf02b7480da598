"""CPU FP64 oracle of the in-solve algebraic coarsening step.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never imports it.

The arithmetic lives in ``agipc_oracle.c`` (plain single-threaded C, FP64),
compiled with gcc into ``oracle/_build/liboracle.so`` by :func:`build`.
Each wrapper below marshals numpy arrays into that library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "agipc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

NOT_CONVERGED = -5


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.oracle_labels.argtypes = [i32, i64, P, P, P]
        lib.oracle_labels.restype = i32
        lib.oracle_coarse_gradient.argtypes = [i32, i32, P, P, P]
        lib.oracle_coarse_gradient.restype = ctypes.c_int
        lib.oracle_full_terms.argtypes = [i32, P, P, i64]
        lib.oracle_full_terms.restype = i64
        lib.oracle_galerkin.argtypes = [i32, i32, P, P, P, P, i64, P, P, P, P, P, i64]
        lib.oracle_galerkin.restype = i64
        lib.oracle_block_jacobi.argtypes = [i32, P, P, P, P]
        lib.oracle_block_jacobi.restype = ctypes.c_int
        lib.oracle_spmv.argtypes = [i32, P, P, P, P, P]
        lib.oracle_spmv.restype = None
        lib.oracle_pcg.argtypes = [i32, P, P, P, P, P, P, P, f64, i32, P, P]
        lib.oracle_pcg.restype = ctypes.c_int
        lib.oracle_prolongate.argtypes = [i32, i32, P, P, P]
        lib.oracle_prolongate.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleError(RuntimeError):
    pass


def labels(n: int, edges, tags):
    """Canonical super-node labels and n_c (connected components of the
    collapsible-edge graph, ranked by each component's smallest fine index)."""
    edges = _c(edges, np.int32).reshape(-1, 2)
    tags = _c(tags, np.uint8)
    out = np.empty(n, np.int32)
    nc = _load().oracle_labels(n, edges.shape[0], _p(edges), _p(tags), _p(out))
    if nc < 0:
        raise OracleError("oracle_labels: invalid input")
    return out, int(nc)


def coarse_gradient(labels_, n_c: int, g):
    labels_ = _c(labels_, np.int32)
    g = _c(g, np.float64).reshape(-1, 3)
    out = np.empty((n_c, 3))
    if _load().oracle_coarse_gradient(labels_.size, n_c, _p(labels_), _p(g), _p(out)) != 0:
        raise OracleError("oracle_coarse_gradient: invalid label")
    return out


def galerkin(labels_, n_c: int, row_ptr, col, val, pair_idx, pair_blk):
    """H_c = U H U^T in full storage with sorted columns: (row_ptr, col, val[nnz,3,3])."""
    lib = _load()
    labels_ = _c(labels_, np.int32)
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64).reshape(-1, 9)
    pair_idx = _c(pair_idx, np.int32).reshape(-1, 4)
    pair_blk = _c(pair_blk, np.float64).reshape(-1, 90)
    n = labels_.size
    cap = lib.oracle_full_terms(n, _p(row_ptr), _p(col), pair_idx.shape[0])
    crp = np.empty(n_c + 1, np.int32)
    cci = np.empty(max(cap, 1), np.int32)
    cval = np.empty((max(cap, 1), 9))
    nnz = lib.oracle_galerkin(n, n_c, _p(labels_), _p(row_ptr), _p(col), _p(val), pair_idx.shape[0],
                              _p(pair_idx), _p(pair_blk), _p(crp), _p(cci), _p(cval), cap)
    if nnz < 0:
        raise OracleError("oracle_galerkin: status %d" % nnz)
    return crp, cci[:nnz].copy(), cval[:nnz].reshape(-1, 3, 3).copy()


def block_jacobi(row_ptr, col, val):
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    n = row_ptr.size - 1
    out = np.empty((n, 3, 3))
    if _load().oracle_block_jacobi(n, _p(row_ptr), _p(col), _p(val), _p(out)) != 0:
        raise OracleError("oracle_block_jacobi: singular or missing diagonal block")
    return out


def spmv(row_ptr, col, val, x):
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64).reshape(-1, 3)
    n = row_ptr.size - 1
    y = np.empty((n, 3))
    _load().oracle_spmv(n, _p(row_ptr), _p(col), _p(val), _p(x), _p(y))
    return y


def pcg(row_ptr, col, val, dinv, b, tol: float, max_iter: int, x0=None):
    """Block-Jacobi PCG from x0 (default 0): returns (x, iters, relres, converged)."""
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    dinv = _c(dinv, np.float64)
    b = _c(b, np.float64).reshape(-1, 3)
    n = row_ptr.size - 1
    x = np.empty((n, 3))
    x0 = None if x0 is None else _c(x0, np.float64).reshape(-1, 3)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = _load().oracle_pcg(n, _p(row_ptr), _p(col), _p(val), _p(dinv), _p(b), _p(x), _p(x0), tol, max_iter,
                            ctypes.byref(it), ctypes.byref(rr))
    if st not in (0, NOT_CONVERGED):
        raise OracleError("oracle_pcg: status %d" % st)
    return x, int(it.value), float(rr.value), st == 0


def prolongate(labels_, y):
    labels_ = _c(labels_, np.int32)
    y = _c(y, np.float64).reshape(-1, 3)
    dx = np.empty((labels_.size, 3))
    if _load().oracle_prolongate(labels_.size, y.shape[0], _p(labels_), _p(y), _p(dx)) != 0:
        raise OracleError("oracle_prolongate: invalid label")
    return dx


def coarsened_step(scene, tol: float, max_iter: int = 100000):
    """One coarsened Newton-step solve on a scene, in the paper's order:
    labels -> (g_c, H_c) -> d_c = -H_c^{-1} g_c -> d_f = U^T d_c."""
    lab, nc = labels(scene.n, scene.edges, scene.tags)
    gc = coarse_gradient(lab, nc, scene.g)
    crp, cci, cval = galerkin(lab, nc, scene.row_ptr, scene.col, scene.val, scene.pair_idx, scene.pair_blk)
    dinv = block_jacobi(crp, cci, cval)
    y, it, rr, conv = pcg(crp, cci, cval, dinv, -gc, tol, max_iter)
    dx = prolongate(lab, y)
    return dict(labels=lab, n_c=nc, g_c=gc, row_ptr=crp, col=cci, val=cval, dinv=dinv, y=y, iters=it,
                relres=rr, converged=conv, dx=dx)


def fine_system(scene):
    """The fine system in full storage (identity labels): the no-coarsening arm."""
    lab = np.arange(scene.n, dtype=np.int32)
    return galerkin(lab, scene.n, scene.row_ptr, scene.col, scene.val, scene.pair_idx, scene.pair_blk)


def fine_system_csr_blocks(scene):
    """The full fine system (contacts merged) as a scipy CSR matrix (3n x 3n)."""
    import scipy.sparse as sp
    rp, ci, val = fine_system(scene)
    return sp.bsr_matrix((val, ci, rp), shape=(3 * scene.n, 3 * scene.n)).tocsr()
