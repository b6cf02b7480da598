"""Pins of the precision form's input split (oracle/precision.py): the rule
gap < limit keeps a stencil in FP64, everything else is rounded to FP32 to
nearest, and both lists keep the input order."""
import numpy as np

from oracle import precision


def test_split_by_gap_keeps_order_and_boundary():
    P = 5
    idx = np.arange(4 * P, dtype=np.int32).reshape(P, 4)
    blk = np.arange(90 * P, dtype=np.float64).reshape(P, 90) + 0.5
    dhat = 1e-3
    gap = np.array([0.1, 0.04, 0.05, 0.01, 0.9]) * dhat
    out = precision.split(np.zeros((1, 9)), idx, blk, gap, 0.05 * dhat)
    # 0.05 dhat itself is not below the limit: it is rounded to FP32
    assert np.array_equal(out["pair_idx64"], idx[[1, 3]])
    assert np.array_equal(out["pair_blk64"], blk[[1, 3]])
    assert np.array_equal(out["pair_idx32"], idx[[0, 2, 4]])
    assert out["pair_blk32"].dtype == np.float32
    assert np.array_equal(out["pair_blk32"].astype(np.float64), blk[[0, 2, 4]])  # small integers + 0.5: exact


def test_fp32_rounding_is_round_to_nearest():
    # 1/3 and 2/3 round to the nearest FP32 values; 1 + 2^-24 is a tie that
    # rounds to even (1.0), 1 + 3 * 2^-24 rounds up to 1 + 2^-22
    v = np.array([[1.0 / 3.0, 2.0 / 3.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -0.1, 0.0, 1e-45, 3.4e38, 1e300]])
    with np.errstate(over="ignore"):
        out = precision.split(v, np.zeros((0, 4)), np.zeros((0, 90)), np.zeros(0), 1.0)
    got = out["val32"].astype(np.float64)[0]
    assert got[0] == 0.3333333432674408 and got[1] == 0.6666666865348816
    assert got[2] == 1.0 and got[3] == 1.0 + 2.0 ** -22
    assert abs(got[4] + 0.1) <= 2.0 ** -27
    assert got[5] == 0.0 and got[6] == 1.401298464324817e-45 and np.isinf(got[8])
    assert out["pair_idx32"].shape == (0, 4) and out["pair_idx64"].shape == (0, 4)
