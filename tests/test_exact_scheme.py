"""Invariants of the integer-slice block products (CPU only).

The tensor-core kernel in csrc/tc_ozaki.cu is exact only while its
constants respect bounds that follow from the scheme: S signed 7-bit digits
per operand (balanced base-128 digits of |N|, N = rint(2^(7S) a), signed
afterwards), digit-pair products summed per level in fp32 over chunks of K,
and levels folded into int64 accumulators.  This test reads the constants
from the source and checks:
  * the digit decomposition reconstructs N exactly, with |d_t| <= 64
    (t >= 1), |d_0| <= 128, and digits(-a) = -digits(a);
  * the worst level sum of a chunk is below 2^24 (fp32 holds every integer
    up to 2^24), for both digit counts;
  * the int64 accumulators cannot overflow up to the largest K accepted.
"""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1208_4869_gb300", "csrc", "tc_ozaki.cu")


def constants():
    text = open(SRC).read()
    cfg = {}
    for s, body in re.findall(r"template <> struct Cfg<(\d+)> \{\s*static constexpr int ([^;]+);", text):
        vals = dict(kv.strip().split(" = ") for kv in body.split(","))
        cfg[int(s)] = {k: int(v) for k, v in vals.items()}
    bk = int(re.search(r"constexpr int BM = \d+, BK = (\d+);", text).group(1))
    kmax = int(re.search(r"constexpr int64_t kMaxK = (\d+);", text).group(1))
    return cfg, bk, kmax


def digits(N, S):
    """The kernel's decomposition of one integer (balanced digits of |N|)."""
    sg = -1 if N < 0 else 1
    m = abs(N)
    d = [0] * S
    for t in range(S - 1, 0, -1):
        r = ((m + 64) & 127) - 64
        d[t] = sg * r
        m = (m - r) >> 7
    d[0] = sg * m
    return d


def test_constants_are_found():
    cfg, bk, kmax = constants()
    assert set(cfg) == {4, 8} and bk == 32 and kmax > 0
    for s in (4, 8):
        assert {"BN", "STAGES", "CHUNK_KB"} <= set(cfg[s])


def test_digit_decomposition():
    rng = np.random.default_rng(0)
    for S in (4, 8):
        top = 2 ** (7 * S)
        samples = [0, 1, -1, 64, -64, 127, top, -top, top - 1, -(top - 1)]
        samples += [int(rng.integers(-top, top, dtype=np.int64)) for _ in range(2000)]
        for N in samples:
            d = digits(N, S)
            assert sum(dt * 128 ** (S - 1 - t) for t, dt in enumerate(d)) == N
            assert abs(d[0]) <= 128 and all(abs(x) <= 64 for x in d[1:]), (N, d)
            assert digits(-N, S) == [-x for x in d]


def worst_level_sum(S, K):
    """Largest |level sum| over a chunk of K terms: every pair product at its
    bound with one sign (|d_0| <= 128, |d_t| <= 64)."""
    bound = [128] + [64] * (S - 1)
    worst = 0
    for lvl in range(S):
        per_term = sum(bound[t] * bound[lvl - t] for t in range(lvl + 1))
        worst = max(worst, per_term * K)
    return worst


def test_level_sums_are_exact_in_fp32():
    cfg, bk, _ = constants()
    for S, c in cfg.items():
        K = c["CHUNK_KB"] * bk
        w = worst_level_sum(S, K)
        assert w < 2 ** 24, (S, K, math.log2(w))


def test_int64_accumulators_do_not_overflow():
    cfg, bk, kmax = constants()
    for S in cfg:
        # A = sum_{l<4} L_l 2^(7(3-l)), B = sum_{l>=4} L_l 2^(7(7-l)), each L_l summed over all K
        bound = [128] + [64] * (S - 1)
        per_term = [sum(bound[t] * bound[l - t] for t in range(l + 1)) for l in range(S)]
        acc_a = sum(per_term[l] * kmax * 2 ** (7 * (3 - l)) for l in range(min(S, 4)))
        acc_b = sum(per_term[l] * kmax * 2 ** (7 * (7 - l)) for l in range(4, S))
        assert acc_a < 2 ** 53 and acc_b < 2 ** 53, (S, math.log2(acc_a), acc_b and math.log2(acc_b))
