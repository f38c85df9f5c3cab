"""The error-free digit splitting behind the tensor-core products, restated in exact
integer arithmetic on the CPU (no CUDA): the scaling, the balanced base-256 digits, the
exact per-diagonal sums, the 64-bit recombination and its bounds.

This pins the design (the bounds the CUDA kernels are tested against on the GPU):
  * every digit is an integer in [-128, 127] (exact in bfloat16) and the leading one in
    [-64, 64];
  * a diagonal sum over K <= 64 terms (products) or 128 rows (Gram) stays below 2^24, so an
    FP32 accumulator holds it exactly;
  * the 64-bit sums stay below 2^63;
  * |split - exact| <= 6 u max|x_r| max|c_j| + u |exact| for the product, and the Gram
    error relative to sum |a||b| stays below the FP64 bound on the same data.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

U53 = 2.0 ** -53
ZERO_EXP = -1100


def bexp(x):
    """Biased exponent of a normal double; for a subnormal its leading-bit equivalent."""
    b = struct.unpack("<Q", struct.pack("<d", float(x)))[0]
    E = (b >> 52) & 0x7FF
    if E:
        return E
    M = b & ((1 << 52) - 1)
    return ZERO_EXP if M == 0 else (M.bit_length() - 1) - 51


def fixed(x, emax):
    """Y = round(x 2^(62 - e)), e = emax - 1022, as a Python integer."""
    b = struct.unpack("<Q", struct.pack("<d", float(x)))[0]
    E = (b >> 52) & 0x7FF
    M = b & ((1 << 52) - 1)
    if E:
        M |= 1 << 52
    s = (E if E else 1) - emax + 9
    if M == 0:
        Y = 0
    elif s >= 0:
        Y = M << s
    elif s > -63:
        Y = (M + (1 << (-s - 1))) >> (-s)
    else:
        Y = 0
    return -Y if b >> 63 else Y


def digits(Y):
    z = (Y + 0x8080808080808080) % (1 << 64)
    return [((z >> (8 * (7 - p))) & 0xFF) - 128 for p in range(8)]


def shift(D, sh):
    return D << sh if sh >= 0 else (D + (1 << (-sh - 1))) >> (-sh)


def split_product(X, C):
    """X [n][K] C [K][N] by the per-row / per-column split (the step-(d) kernel)."""
    n, K = X.shape
    N = C.shape[1]
    er = [max([ZERO_EXP] + [bexp(v) for v in X[r]]) for r in range(n)]
    fc = [max([ZERO_EXP] + [bexp(v) for v in C[:, j]]) for j in range(N)]
    A = [[digits(fixed(X[r, k], er[r])) for k in range(K)] for r in range(n)]
    B = [[digits(fixed(C[k, j], fc[j])) for j in range(N)] for k in range(K)]
    out = np.zeros((n, N))
    stats = {"maxD": 0, "maxT": 0, "lead": 0}
    for r in range(n):
        stats["lead"] = max(stats["lead"], max(abs(A[r][k][0]) for k in range(K)))
        for j in range(N):
            T = 0
            for d in range(2, 10):
                D = sum(A[r][k][p - 1] * B[k][j][d - p - 1] for p in range(1, d) if p <= 8 and d - p <= 8
                        for k in range(K))
                stats["maxD"] = max(stats["maxD"], abs(D))
                T += shift(D, 60 - 8 * d)
            stats["maxT"] = max(stats["maxT"], abs(T))
            out[r, j] = math.ldexp(float(T), er[r] + fc[j] - 2100) if T else 0.0
    return out, stats


def split_gram(A, B, drain=128):
    """A^T B by the per-column split over rows, drained every `drain` rows (step (b))."""
    n, ma = A.shape
    mb = B.shape[1]
    ea = [max([ZERO_EXP] + [bexp(v) for v in A[:, i]]) for i in range(ma)]
    fb = [max([ZERO_EXP] + [bexp(v) for v in B[:, j]]) for j in range(mb)]
    Ad = [[digits(fixed(A[r, i], ea[i])) for i in range(ma)] for r in range(n)]
    Bd = [[digits(fixed(B[r, j], fb[j])) for j in range(mb)] for r in range(n)]
    G = np.zeros((ma, mb))
    stats = {"maxD": 0, "maxT": 0}
    for i in range(ma):
        for j in range(mb):
            acc = 0
            for c0 in range(0, n, drain):
                for d in range(2, 10):
                    D = sum(Ad[r][i][p - 1] * Bd[r][j][d - p - 1] for p in range(1, d) if p <= 8 and d - p <= 8
                            for r in range(c0, min(c0 + drain, n)))
                    stats["maxD"] = max(stats["maxD"], abs(D))
                    acc += shift(D, 52 - 8 * d)
            stats["maxT"] = max(stats["maxT"], abs(acc))
            G[i, j] = math.ldexp(float(acc), ea[i] + fb[j] - 2044 - 48) if acc else 0.0
    return G, stats


def exact_product(X, C):
    return [[sum(Fraction(float(X[r, k])) * Fraction(float(C[k, j])) for k in range(X.shape[1]))
             for j in range(C.shape[1])] for r in range(X.shape[0])]


def test_digits_are_exact_and_balanced():
    rng = np.random.default_rng(0)
    vals = list(rng.standard_normal(200) * np.exp2(rng.integers(-40, 40, 200))) + [0.0, -0.0, 1e-310, -3e-320]
    emax = max(bexp(v) for v in vals)
    for v in vals:
        Y = fixed(v, emax)
        a = digits(Y)
        assert abs(Y) < 2 ** 62
        assert all(-128 <= t <= 127 for t in a) and abs(a[0]) <= 64
        assert sum(t * 256 ** (7 - p) for p, t in enumerate(a)) == Y         # the digits are Y
        # the scaled value is x up to half a unit of 2^(e - 62)
        e = emax - 1022
        assert abs(Fraction(float(v)) - Fraction(Y) * Fraction(2) ** (e - 62)) <= Fraction(2) ** (e - 63)


@pytest.mark.parametrize("K", [8, 56, 64])
def test_split_product_bound(K):
    rng = np.random.default_rng(K)
    n, N = 6, 5
    X = rng.standard_normal((n, K)) * np.exp2(rng.integers(-40, 41, size=(n, 1)))
    X[1] *= np.exp2(rng.integers(-60, 1, size=K))                 # entries spread inside a row
    X[2, : K // 2] = 1e-310                                         # subnormal entries
    X[3] = 0.0                                                      # zero row
    C = rng.standard_normal((K, N)) * np.exp2(rng.integers(-20, 21, size=(1, N)))
    Y, st = split_product(X, C)
    assert st["maxD"] < 2 ** 23 and st["maxT"] < 2 ** 62 and st["lead"] <= 64
    ex = exact_product(X, C)
    scale = np.abs(X).max(axis=1)[:, None] * np.abs(C).max(axis=0)[None, :]
    for r in range(n):
        for j in range(N):
            err = abs(Fraction(float(Y[r, j])) - ex[r][j])
            bound = Fraction(6 * U53) * Fraction(float(scale[r, j])) + Fraction(U53) * abs(ex[r][j]) \
                + Fraction(2.0 ** -1074)
            assert err <= bound, (r, j, float(err), float(bound))


def test_split_gram_bound_and_headroom():
    rng = np.random.default_rng(7)
    n, m = 300, 4
    A = rng.standard_normal((n, m)) * np.exp2(rng.integers(-20, 20, size=(1, m)))
    B = rng.standard_normal((n, m)) * np.exp2(rng.integers(-20, 20, size=(1, m)))
    B[:, 0] = A[:, 0] * 1e-3
    G, st = split_gram(A, B)
    assert st["maxD"] < 2 ** 24 and st["maxT"] < 2 ** 63
    ex = [[sum(Fraction(float(A[r, i])) * Fraction(float(B[r, j])) for r in range(n)) for j in range(m)]
          for i in range(m)]
    sumabs = np.abs(A).T @ np.abs(B)
    fp = A.T @ B
    worst_split = max(float(abs(Fraction(float(G[i, j])) - ex[i][j])) / sumabs[i, j] for i in range(m) for j in range(m))
    worst_fp64 = max(float(abs(Fraction(float(fp[i, j])) - ex[i][j])) / sumabs[i, j] for i in range(m) for j in range(m))
    assert worst_split <= 8 * U53, worst_split / U53
    assert worst_split <= max(2 * worst_fp64, 2 * U53)


def test_worst_case_diagonal_sums_fit_fp32():
    """Largest possible |D_d| with the digit ranges: K = 64 (products) and 128 rows (Gram)
    stay below 2^24, so the FP32 accumulation is exact."""
    lead, other = 64, 128
    for K in (64, 128):
        worst = 0
        for d in range(2, 10):
            pairs = [(p, d - p) for p in range(1, d) if p <= 8 and d - p <= 8]
            worst = max(worst, K * sum((lead if p == 1 else other) * (lead if q == 1 else other) for p, q in pairs))
        assert worst < 2 ** 24, (K, worst)
