"""The dense products on the tensor cores (split digits, `split_gemm = 1`), step (d) W C_W
and the step-(b) Gram blocks, against the oracle through the C ABI (needs a GPU).

With C_H = 0, pase_prolongate returns U = W C_W.  Bound checked on every entry (the
error analysis of the split product: dropped digit diagonals, floor shifts, digit
rounding, final rounding):
    |U - W C_W| <= 8 u max_k |w_rk| max_k |c_kj| + u |W C_W| + K 2^-1074,   u = 2^-53,
where W C_W is exact: rational arithmetic on sampled entries, and elsewhere the FP64
oracle product with its own error bound K u sum_k |w_rk||c_kj| added.  Inputs stress the
scaling: rows at 2^-40..2^40, entries spread over 2^60 inside a row, zero rows,
subnormal entries, a ragged last tile (N = 31^3 is not a multiple of 128), every padded
width K, N in {16, 32, 48, 64}, widths 72-128 (two K and N blocks) and 136 (the FP64
kernel).
"""
from fractions import Fraction

import numpy as np
import pytest

import pase_inputs as pin
from oracle import pase as opase

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def p3d():
    return pin.build_problem(3, 32, 8, kappa_seed=5, mg_min=4)


def _handle(pb, split, **kw):
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    opt.split_gemm = split
    for k, v in kw.items():
        setattr(opt, k, v)
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
    except Exception:
        P.pase_destroy(h)
        raise
    return h


def _operands(N, m, seed):
    rng = np.random.default_rng(seed)
    W = pin.start_vectors(seed, N, m)
    W *= np.exp2(rng.integers(-40, 41, size=(N, 1)))           # row scales
    wide = rng.choice(N, size=N // 16, replace=False)           # entries spread inside a row
    W[wide] *= np.exp2(rng.integers(-60, 1, size=(len(wide), m)))
    W[rng.choice(N, size=8, replace=False)] = 0.0               # zero rows
    sub = rng.choice(N, size=4, replace=False)
    W[sub[:2], : m // 2] = 1e-310                               # subnormal entries
    W[sub[2:]] = 1e-310 * pin.start_vectors(seed + 2, 2, m)     # whole rows subnormal
    W[N - 1] *= 3.0                                             # last (ragged-tile) row
    C = pin.start_vectors(seed + 1, m, m) * np.exp2(rng.integers(-20, 21, size=(1, m)))
    return W, C


def _prolong(h, pb, m, W, C):
    U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
    CH = torch.zeros(pb.N_H, m, dtype=torch.float64, device="cuda")
    P.pase_prolongate(h, m, torch.from_numpy(W).cuda(), CH, torch.from_numpy(C).cuda(), U)
    return U.cpu().numpy()


def _check_bound(pb, W, C, U, sample_rows):
    """The split bound; widths above 64 add two K blocks in FP64 (twice the bound plus one
    rounding); above 128 the FP64 kernel runs, with the usual K u sum_k |w_rk||c_kj|."""
    K = W.shape[1]
    scale = np.abs(W).max(axis=1)[:, None] * np.abs(C).max(axis=0)[None, :]
    if K > 128:
        scale = (K / 8.0) * (np.abs(W) @ np.abs(C))
    elif K > 64:
        scale = 2.0 * scale + np.abs(W) @ np.abs(C) / 8.0
    ref = opase.prolongate(pb.P, W, np.zeros((pb.N_H, K)), C)
    refbound = K * U53 * (np.abs(W) @ np.abs(C))                # the oracle's own rounding
    err = np.abs(U - ref)
    tiny = K * 2.0 ** -1074                                        # subnormal results
    assert np.all(err <= 8 * U53 * scale + U53 * np.abs(ref) + refbound + tiny), (err / np.maximum(scale, 1e-300)).max()
    for r in sample_rows:                                      # exact products, no oracle rounding
        for j in range(C.shape[1]):
            ex = sum(Fraction(float(W[r, k])) * Fraction(float(C[k, j])) for k in range(K))
            e = abs(Fraction(float(U[r, j])) - ex)
            assert e <= Fraction(8 * U53) * Fraction(float(scale[r, j])) + Fraction(U53) * abs(ex) + Fraction(tiny), (r, j)


@pytest.mark.parametrize("m", [8, 16, 24, 40, 56, 64, 72, 112, 128, 136])
def test_split_product_error_bound(p3d, m):
    pb = p3d
    h = _handle(pb, 1)
    try:
        W, C = _operands(pb.N, m, 40 + m)
        U = _prolong(h, pb, m, W, C)
    finally:
        P.pase_destroy(h)
    rng = np.random.default_rng(m)
    rows = list(rng.choice(pb.N, size=6, replace=False)) + [pb.N - 1, 0] + list(np.flatnonzero(np.abs(W).max(axis=1) < 1e-300))
    _check_bound(pb, W, C, U, rows)


def test_split_and_fp64_kernels_agree(p3d):
    """The two kernels behind split_gemm = 1 and 0 give the same product to the bound."""
    pb, m = p3d, 56
    W, C = _operands(pb.N, m, 7)
    out = {}
    for split in (1, 0):
        h = _handle(pb, split)
        try:
            out[split] = _prolong(h, pb, m, W, C)
        finally:
            P.pase_destroy(h)
    scale = np.abs(W).max(axis=1)[:, None] * np.abs(C).max(axis=0)[None, :]
    K = m
    tol = (8 + 2 * K) * U53 * scale + 2 * U53 * np.abs(out[0]) + 2 * K * 2.0 ** -1074
    assert np.all(np.abs(out[1] - out[0]) <= tol)
    # on O(1) random blocks the split product is at least as close to exact as FP64
    Wr, Cr = pin.start_vectors(3, pb.N, m), pin.start_vectors(4, m, m)
    res = {}
    for split in (1, 0):
        h = _handle(pb, split)
        try:
            res[split] = _prolong(h, pb, m, Wr, Cr)
        finally:
            P.pase_destroy(h)
    rows = range(0, pb.N, 997)
    exact = np.array([[float(sum(Fraction(float(Wr[r, k])) * Fraction(float(Cr[k, j])) for k in range(K)))
                       for j in range(m)] for r in rows])
    e_split = np.abs(res[1][list(rows)] - exact).max()
    e_fp64 = np.abs(res[0][list(rows)] - exact).max()
    assert e_split <= 2 * e_fp64 + 1e-300, (e_split, e_fp64)


def test_split_nonfinite_rows_and_columns(p3d):
    """Inf/NaN in a row of W or a column of C_W come out as in an FP64 product."""
    pb, m = p3d, 24
    W, C = _operands(pb.N, m, 11)
    W[5, 3] = np.nan
    W[200, 0] = np.inf
    C[2, 7] = -np.inf
    h = _handle(pb, 1)
    try:
        U = _prolong(h, pb, m, W, C)
    finally:
        P.pase_destroy(h)
    with np.errstate(invalid="ignore", over="ignore"):
        ref = W @ C
    assert np.array_equal(np.isnan(U), np.isnan(ref))
    assert np.array_equal(np.isposinf(U), np.isposinf(ref))
    assert np.array_equal(np.isneginf(U), np.isneginf(ref))
    fin = np.isfinite(ref)
    scale = np.abs(np.where(np.isfinite(W), W, 0)).max(axis=1)[:, None] * \
        np.abs(np.where(np.isfinite(C), C, 0)).max(axis=0)[None, :]
    err = np.abs(U[fin] - ref[fin])
    assert np.all(err <= ((8 + 2 * m) * U53 * scale + 2 * U53 * np.abs(ref) + 2 * m * 2.0 ** -1074)[fin])


def test_split_kernel_timing_entry(p3d):
    """pase_time_kernel runs the split kernel for m <= 128 and refuses wider blocks."""
    pb = p3d
    h = _handle(pb, 1)
    try:
        P.pase_reserve(h, 56)
        assert P.pase_time_kernel(h, "prolong_split", 56, 2) > 0.0
    finally:
        P.pase_destroy(h)
    h = _handle(pb, 1)
    try:
        P.pase_reserve(h, 136)
        with pytest.raises(P.PaseError):
            P.pase_time_kernel(h, "prolong_split", 136, 2)
    finally:
        P.pase_destroy(h)


def _project(h, pb, m, W):
    aH = torch.empty(pb.N_H, m, dtype=torch.float64, device="cuda")
    bH = torch.empty_like(aH)
    GA = torch.empty(m, m, dtype=torch.float64, device="cuda")
    GM = torch.empty_like(GA)
    P.pase_project(h, m, torch.from_numpy(np.ascontiguousarray(W)).cuda(), aH, bH, GA, GM)
    return GA.cpu().numpy(), GM.cpu().numpy()


def _gram_operand(N, m, seed):
    rng = np.random.default_rng(seed)
    W = pin.start_vectors(seed, N, m)
    W *= np.exp2(rng.integers(-30, 31, size=(1, m)))             # column scales
    spread = rng.choice(N, size=N // 8, replace=False)           # entries spread inside columns
    W[spread] *= np.exp2(rng.integers(-20, 1, size=(len(spread), m)))
    return W


@pytest.mark.parametrize("m", [24, 56, 112])
def test_split_gram_no_worse_than_fp64(p3d, m):
    """Step (b) Gram blocks W^T(A_h W), W^T(M_h W) with split_gemm = 1 and 0 against an
    extended-precision evaluation of the same definition (upper triangle mirrored): the
    largest error relative to sum_r |w_ri||y_rj| is at most twice the FP64 kernel's (both
    include the rounding of A_h W by the FP64 sparse product) and below 64 u.""" 
    pb = p3d
    W = _gram_operand(pb.N, m, 60 + m)
    res = {}
    for split in (1, 0):
        h = _handle(pb, split)
        try:
            res[split] = _project(h, pb, m, W)
        finally:
            P.pase_destroy(h)
    Wl = W.astype(np.longdouble)
    for idx, Mat in ((0, pb.A), (1, pb.M)):
        Y = Mat.astype(np.longdouble) @ Wl
        ref = Wl.T @ Y
        ref = np.triu(ref) + np.triu(ref, 1).T                 # upper triangle mirrored
        scale = (np.abs(Wl).T @ np.abs(Y)).astype(np.float64)
        scale = np.maximum(np.triu(scale), np.triu(scale, 1).T)
        ref = ref.astype(np.float64)
        r_s = (np.abs(res[1][idx] - ref) / scale).max() / U53   # worst error in units of u sum|w||y|
        r_f = (np.abs(res[0][idx] - ref) / scale).max() / U53
        assert r_s <= max(2.0 * r_f, 2.0) and r_s <= 64.0, (idx, r_s, r_f)


def test_split_gram_nonfinite(p3d):
    """A NaN in W gives the same NaN entries of the Gram blocks as the FP64 kernel.  The
    fine-level products run in FP64 here (spmm_df64 = 0): their double-float form reports a
    non-finite block entry as PASE_ERR_NAN instead of propagating it."""
    pb, m = p3d, 16
    W = pin.start_vectors(70, pb.N, m)
    W[1234, 5] = np.nan
    res = {}
    for split in (1, 0):
        h = _handle(pb, split, spmm_df64=0)
        try:
            res[split] = _project(h, pb, m, W)
        finally:
            P.pase_destroy(h)
    for idx in (0, 1):
        assert np.array_equal(np.isnan(res[1][idx]), np.isnan(res[0][idx]))
        assert np.isnan(res[1][idx]).any()
        fin = np.isfinite(res[0][idx])
        np.testing.assert_allclose(res[1][idx][fin], res[0][idx][fin], rtol=1e-12, atol=1e-12 * np.abs(res[0][idx][fin]).max())


def _gram_refs(pb, W):
    """Extended-precision Gram blocks of the definition (upper triangle mirrored), the
    componentwise scales sum_r |w_ri||y_rj| and the normwise scales ||w_i||_2 ||y_j||_2."""
    Wl = W.astype(np.longdouble)
    out = []
    for Mat in (pb.A, pb.M):
        Y = Mat.astype(np.longdouble) @ Wl
        ref = Wl.T @ Y
        ref = (np.triu(ref) + np.triu(ref, 1).T).astype(np.float64)
        comp = (np.abs(Wl).T @ np.abs(Y)).astype(np.float64)
        comp = np.maximum(np.triu(comp), np.triu(comp, 1).T)
        nw = np.linalg.norm(W, axis=0)
        ny = np.linalg.norm(Y.astype(np.float64), axis=0)
        norm = np.outer(nw, ny)
        norm = np.maximum(np.triu(norm), np.triu(norm, 1).T)
        out.append((ref, comp, norm))
    return out


def test_split_gram_wide_row_range(p3d):
    """Rows scaled by 2^k, k uniform in [-30, 30] and shared by the row's columns (the shape
    of localised vectors): the split Gram's largest error relative to sum_r |w_ri||y_rj|
    stays within twice the FP64 kernel's and below 64 u."""
    pb, m = p3d, 24
    rng = np.random.default_rng(80)
    W = pin.start_vectors(80, pb.N, m) * np.exp2(rng.integers(-30, 31, size=(pb.N, 1)))
    res = {}
    for split in (1, 0):
        h = _handle(pb, split)
        try:
            res[split] = _project(h, pb, m, W)
        finally:
            P.pase_destroy(h)
    for idx, (ref, comp, _) in enumerate(_gram_refs(pb, W)):
        r_s = (np.abs(res[1][idx] - ref) / comp).max() / U53
        r_f = (np.abs(res[0][idx] - ref) / comp).max() / U53
        print(f"\nwide row range, block {idx}: split {r_s:.2f} u, FP64 {r_f:.2f} u (of sum |w||y|)")
        assert r_s <= max(2.0 * r_f, 2.0) and r_s <= 64.0, (idx, r_s, r_f)


def test_split_gram_disjoint_localised_columns(p3d):
    """Columns localised in disjoint row ranges (1 on their own range, 2^-40 noise elsewhere):
    the off-diagonal Gram entries are sums of products of a large and a tiny value, where the
    split form, which scales each column by its largest entry, is not accurate relative to
    sum_r |w_ri||y_rj|.  It stays accurate normwise, relative to ||w_i||_2 ||y_j||_2 (the
    measure that bounds the Rayleigh-Ritz perturbation): below 8 u there."""
    pb, m = p3d, 16
    N = pb.N
    W = 2.0 ** -40 * pin.start_vectors(81, N, m)
    span = N // m
    for j in range(m):
        W[j * span:(j + 1) * span, j] = 1.0 + 0.5 * pin.start_vectors(82 + j, span, 1)[:, 0]
    h = _handle(pb, 1)
    try:
        G = _project(h, pb, m, W)
    finally:
        P.pase_destroy(h)
    for idx, (ref, comp, norm) in enumerate(_gram_refs(pb, W)):
        rn = (np.abs(G[idx] - ref) / norm).max() / U53
        rc = (np.abs(G[idx] - ref) / comp).max() / U53
        print(f"\ndisjoint localised columns, block {idx}: {rn:.2f} u normwise, {rc:.3g} u of sum |w||y|")
        assert rn <= 8.0, (idx, rn)
