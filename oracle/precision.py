"""CPU oracle of the precision form's input split (the FP32 / FP64 rule of
the precision form: Hessian blocks in FP32, barrier terms at small gap
distances kept in FP64).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.

Reading taken (the paper computes everything in FP64): a barrier stencil
whose gap d is below ``gap_limit`` (0.05 dhat in the workloads) keeps its ten
3x3 blocks in FP64, because its stiffness grows like (dhat / d)^2 and the
FP32 rounding of it would dominate the coarse system's error; every other
stencil and every fine block is rounded to FP32 (round to nearest even).  The
two stencil lists keep the input order.  The decision d < gap_limit is taken
in FP64 on both sides, so the split is exact.
"""
from __future__ import annotations

import numpy as np


def split(val, pair_idx, pair_blk, pair_gap, gap_limit: float) -> dict:
    """val [nnzb][9] FP64, pair_idx [P][4], pair_blk [P][90] FP64, pair_gap [P]
    FP64 -> dict(val32, pair_idx32, pair_blk32, pair_idx64, pair_blk64)."""
    val = np.asarray(val, dtype=np.float64).reshape(-1, 9)
    pair_idx = np.asarray(pair_idx, dtype=np.int32).reshape(-1, 4)
    pair_blk = np.asarray(pair_blk, dtype=np.float64).reshape(-1, 90)
    gap = np.asarray(pair_gap, dtype=np.float64).reshape(-1)
    small = gap < np.float64(gap_limit)
    return dict(val32=val.astype(np.float32),
                pair_idx32=np.ascontiguousarray(pair_idx[~small]),
                pair_blk32=np.ascontiguousarray(pair_blk[~small].astype(np.float32)),
                pair_idx64=np.ascontiguousarray(pair_idx[small]),
                pair_blk64=np.ascontiguousarray(pair_blk[small]))


def scene_split(sc, fp64_gap: float = 0.05) -> dict:
    """split() on a generated scene: gaps from its metadata, limit
    fp64_gap * dhat."""
    gap = np.asarray(sc.meta["pair_d"], dtype=np.float64) if sc.n_pairs else np.zeros(0)
    return split(sc.val, sc.pair_idx, sc.pair_blk, gap, fp64_gap * sc.meta["dhat"])
