"""Pins of the FP64 oracle and of the shared input generators (CPU only).

Each test ties a piece of the oracle to something other than itself: a published
test vector, textbook stencils, the closed-form Q1 spectrum, brute-force dense
eigensolves, an independent loop-based assembly, or an invariant the paper states.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import pase_inputs as pin
from oracle import dense, mg, pase, spectrum

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- inputs


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.strip() and l[0] != "#"]
    got = [int(x) for x in pin.splitmix64(0, 3)]
    assert got == vals


def test_start_vectors_layout_and_range():
    U = pin.start_vectors(7, 5, 3)
    z = pin.splitmix64(7, 15)
    # entry (i, j) is output i*3 + j
    assert U[1, 2] == 2.0 * (int(z[5]) >> 11) * 2.0 ** -53 - 1.0
    assert U.min() >= -1.0 and U.max() < 1.0


def test_normals_moments():
    g = pin.standard_normals(1, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    # Box-Muller pairs: the second of a pair uses the sin branch of the same radius
    z = pin.splitmix64(1, 2)
    u1 = ((int(z[0]) >> 11) + 1) * 2.0 ** -53
    u2 = (int(z[1]) >> 11) * 2.0 ** -53
    assert np.isclose(g[1], np.sqrt(-2 * np.log(u1)) * np.sin(2 * np.pi * u2), rtol=0, atol=1e-15)


def _parse_frac(tok, h):
    return float(Fraction(tok))


@pytest.mark.parametrize("d", [2, 3])
def test_q1_stencils_textbook(d):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "q1_stencils.txt")) if l.strip() and l[0] != "#"]
    n = 8
    h = 1.0 / n
    A, M = pin.q1_matrices(d, n)
    n1 = n - 1
    centre = sum(3 * n1 ** k for k in range(d))  # node (4,4[,4]) -> all 3^d neighbours interior
    for r in rows:
        if int(r[0]) != d:
            continue
        scale = {"1": 1.0, "h": h, "h^2/36": h * h / 36, "h^3/216": h ** 3 / 216}[r[2]]
        want = np.array([float(Fraction(t)) for t in r[3:]]) * scale
        X = A if r[1] == "A" else M
        row = X.getrow(centre).toarray().ravel()
        offs = np.array(np.meshgrid(*([[-1, 0, 1]] * d), indexing="ij")).reshape(d, -1).T
        offs = offs[np.lexsort(offs.T)]
        got = np.array([row[centre + sum(o[k] * n1 ** k for k in range(d))] for o in offs])
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-15 * abs(want).max())


def _loop_assembly(d, n, kappa):
    """Independent brute-force assembly: loop over elements and local node pairs on the
    full node grid (boundary included), then drop boundary rows/columns."""
    h = 1.0 / n
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
    Ke = {2: np.kron(k1, m1) + np.kron(m1, k1),
          3: np.kron(k1, np.kron(m1, m1)) + np.kron(m1, np.kron(k1, m1)) + np.kron(m1, np.kron(m1, k1))}[d]
    Me = {2: np.kron(m1, m1), 3: np.kron(m1, np.kron(m1, m1))}[d]
    nn = n + 1
    Af = np.zeros((nn ** d, nn ** d))
    Mf = np.zeros_like(Af)
    for e in range(n ** d):
        ec = [(e // n ** k) % n for k in range(d)]
        # local node ordering of np.kron(first, second...): first factor slowest -> z slowest
        loc = []
        for lz in (range(2) if d == 3 else [0]):
            for ly in range(2):
                for lx in range(2):
                    c = [ec[0] + lx, ec[1] + ly] + ([ec[2] + lz] if d == 3 else [])
                    loc.append(sum(c[k] * nn ** k for k in range(d)))
        for a in range(2 ** d):
            for b in range(2 ** d):
                Af[loc[a], loc[b]] += kappa[e] * Ke[a, b]
                Mf[loc[a], loc[b]] += Me[a, b]
    assert np.isclose(Mf.sum(), 1.0)  # the mass of the unit domain
    interior = [i for i in range(nn ** d) if all(0 < (i // nn ** k) % nn < n for k in range(d))]
    return Af[np.ix_(interior, interior)], Mf[np.ix_(interior, interior)]


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_q1_assembly_matches_loop_assembly_variable_kappa(d, n):
    kappa = pin.lognormal_kappa(d, n, seed=3)
    A, M = pin.q1_matrices(d, n, kappa)
    Ab, Mb = _loop_assembly(d, n, kappa)
    np.testing.assert_allclose(A.toarray(), Ab, rtol=0, atol=1e-13 * abs(Ab).max())
    np.testing.assert_allclose(M.toarray(), Mb, rtol=0, atol=1e-15)


def test_q1_kronecker_form():
    n = 12
    h = 1.0 / n
    K1 = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n - 1, n - 1)) / h
    M1 = sp.diags([1.0, 4.0, 1.0], [-1, 0, 1], shape=(n - 1, n - 1)) * (h / 6)
    A, M = pin.q1_matrices(2, n)
    assert abs(A - (sp.kron(K1, M1) + sp.kron(M1, K1))).max() < 1e-13
    assert abs(M - sp.kron(M1, M1)).max() < 1e-16


@pytest.mark.parametrize("d,n", [(2, 4), (2, 9), (2, 16), (3, 4), (3, 8)])
def test_closed_form_spectrum_vs_brute_force(d, n):
    A, M = pin.q1_matrices(d, n)
    lam_dense = sl.eigh(A.toarray(), M.toarray(), eigvals_only=True)
    lam_cf = spectrum.q1_laplace_eigenvalues(d, n)
    np.testing.assert_allclose(lam_dense, lam_cf, rtol=1e-12)


def test_closed_form_first_values():
    # as h -> 0 the discrete values approach the continuous pi^2 (k1^2 + ... ) from above
    lam = spectrum.q1_laplace_eigenvalues(3, 128, 4)
    cont = np.pi ** 2 * np.array([3, 6, 6, 6])
    assert np.all(lam > cont) and np.all((lam - cont) / cont < 2e-4)


def test_dense_smallest_pairs_m_orthonormal():
    A, M = pin.q1_matrices(2, 8, pin.lognormal_kappa(2, 8, 5))
    lam, U = dense.smallest_pairs(A, M, 6)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(A @ U, (M @ U) * lam, atol=1e-10)


def test_shift_invert_matches_dense():
    A, M = pin.q1_matrices(2, 24, pin.lognormal_kappa(2, 24, 9))
    lam_d, _ = dense.smallest_pairs(A, M, 8)
    lam_s, U = dense.smallest_pairs_shift_invert(A, M, 8)
    np.testing.assert_allclose(lam_s, lam_d, rtol=1e-11)


# --------------------------------------------------------------------- interpolation


def test_interpolation_reproduces_bilinear_functions():
    d, nf, nc = 2, 16, 4
    P = pin.q1_interpolation(d, nf, nc)
    # f(x, y) = x y (1-x)(1-y) is not bilinear; use a Q1 function on the coarse mesh:
    # nodal values of the coarse hat sum are reproduced exactly by the fine interpolant.
    Xc = np.arange(1, nc) / nc
    c = np.add.outer(np.zeros(nc - 1), np.zeros(nc - 1))
    rng = np.random.default_rng(0)
    c = rng.standard_normal((nc - 1) ** 2)
    fine = P @ c
    # evaluate the coarse Q1 interpolant at fine nodes by brute force
    xf = np.arange(1, nf) / nf
    H = 1.0 / nc
    hat = lambda x, X: np.maximum(0, 1 - np.abs(x - X) / H)
    want = np.zeros((nf - 1) ** 2)
    for J in range(nc - 1):
        for I in range(nc - 1):
            want += c[I + J * (nc - 1)] * np.outer(hat(xf, Xc[J]), hat(xf, Xc[I])).ravel()
    np.testing.assert_allclose(fine, want, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_chain_product_equals_direct_and_galerkin_equals_rediscretisation(d):
    nf = 16 if d == 3 else 32
    P1 = pin.q1_interpolation(d, nf, nf // 2)
    P2 = pin.q1_interpolation(d, nf // 2, nf // 4)
    Pd = pin.q1_interpolation(d, nf, nf // 4)
    assert abs(P1 @ P2 - Pd).max() < 1e-15
    A, M = pin.q1_matrices(d, nf)
    Ac, Mc = pin.q1_matrices(d, nf // 4)
    assert abs(pin.galerkin(Pd, A) - Ac).max() < 1e-12 * abs(Ac).max()
    assert abs(pin.galerkin(Pd, M) - Mc).max() < 1e-12 * abs(Mc).max()


def test_problem_levels():
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    assert pb.mesh_sizes == [64, 32, 16, 8, 4]
    assert pb.coarse_level == 3
    assert pb.P.shape == (63 * 63, 49)
    assert pin.guard_columns(10) == 16 and pin.guard_columns(50) == 56 and pin.guard_columns(100) == 112


# -------------------------------------------------------------------------- solvers


def test_vcycle_converges_and_is_symmetric():
    pb = pin.build_problem(2, 32, 4)
    H = mg.Hierarchy(pb.A, pb.chain)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((pb.N, 3))
    x = H.solve(b, 12)
    xs = spl.spsolve(pb.A.tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    # one V-cycle from zero is a symmetric operator (equal pre/post damped Jacobi)
    y, z = rng.standard_normal(pb.N), rng.standard_normal(pb.N)
    Vy = H.vcycle(0, y[:, None])[:, 0]
    Vz = H.vcycle(0, z[:, None])[:, 0]
    assert abs(z @ Vy - y @ Vz) < 1e-12 * abs(z @ Vy)
    # and a contraction: energy-norm reduction per cycle well below 1
    e0 = xs[:, 0]
    e1 = xs[:, 0] - H.vcycle(0, b[:, :1])[:, 0]
    en = lambda v: np.sqrt(v @ (pb.A @ v))
    assert en(e1) / en(e0) < 0.2


def test_cg_matches_direct():
    A, _ = pin.q1_matrices(2, 16)
    rng = np.random.default_rng(2)
    F = rng.standard_normal((A.shape[0], 2))
    X = mg.cg(A, F, np.zeros_like(F), 200)
    np.testing.assert_allclose(X, spl.spsolve(A.tocsc(), F), rtol=1e-9, atol=1e-12)


def test_pcg_exact_preconditioner_one_step():
    """With B = A^-1 the first search direction is the error itself: one step is exact."""
    A, _ = pin.q1_matrices(2, 12, pin.lognormal_kappa(2, 12, 4, 1.0))
    F = np.random.default_rng(3).standard_normal((A.shape[0], 3))
    lu = spl.splu(A.tocsc())
    X = mg.pcg(A, F, np.zeros_like(F), 1, lu.solve)
    np.testing.assert_allclose(X, lu.solve(F), rtol=1e-10, atol=1e-13)


def test_pcg_finite_termination_brute_force():
    """Tiny dense SPD system, random SPD preconditioner: n steps reach the solution, and
    the energy norm of the error never grows (the CG minimisation property)."""
    rng = np.random.default_rng(5)
    n = 7
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    H = rng.standard_normal((n, n))
    B = H @ H.T + 0.5 * np.eye(n)
    F = rng.standard_normal((n, 2))
    x = np.linalg.solve(A, F)
    errs = []
    for k in range(n + 1):
        X = mg.pcg(A, F, np.zeros_like(F), k, lambda R: B @ R)
        E = X - x
        errs.append(np.sqrt(np.einsum("ij,ij->j", E, A @ E)))
    assert np.all(np.diff(np.array(errs), axis=0) <= 1e-12 * errs[0])
    np.testing.assert_allclose(mg.pcg(A, F, np.zeros_like(F), n, lambda R: B @ R), x, rtol=1e-9)


def test_mgcg_beats_cg_on_rough_coefficients():
    """V-cycle-preconditioned CG against plain CG and against plain V-cycles at equal step
    counts on a lognormal (sigma 2) coefficient: the preconditioned error is orders of
    magnitude smaller than either."""
    pb = pin.build_problem(2, 32, 4, kappa_seed=9, sigma=2.0)
    F = np.random.default_rng(1).standard_normal((pb.N, 2))
    x = spl.spsolve(pb.A.tocsc(), F)
    H = mg.Hierarchy(pb.A, pb.chain)
    e_cg = np.linalg.norm(mg.cg(pb.A, F, np.zeros_like(F), 20) - x)
    e_v = np.linalg.norm(H.solve(F, 20) - x)
    e_mg = np.linalg.norm(mg.pcg(pb.A, F, np.zeros_like(F), 20, lambda R: H.solve(R, 1)) - x)
    assert e_mg < 1e-3 * e_cg
    assert e_mg < 1e-2 * e_v
    assert e_mg < 1e-4 * np.linalg.norm(x)


# ----------------------------------------------------------------- augmented subspace


def _tiny(d=2, n=16, nc=4, kappa_seed=None):
    return pin.build_problem(d, n, nc, kappa_seed=kappa_seed)


@pytest.mark.parametrize("kappa_seed", [None, 11])
def test_as_solve_matches_brute_force(kappa_seed):
    pb = _tiny(kappa_seed=kappa_seed)
    nev, m = 4, pin.guard_columns(4)
    S = pase.Solver(pb.A, pb.M, pb.chain)
    lam, U, info = S.solve(nev, m, 1e-10, U0=pin.start_vectors(0, pb.N, m), s=2, max_iter=50)
    assert info["converged"]
    lam_d, U_d = dense.smallest_pairs(pb.A, pb.M, m)
    np.testing.assert_allclose(lam[:nev], lam_d[:nev], rtol=1e-10)
    np.testing.assert_allclose(U.T @ pb.M @ U, np.eye(m), atol=1e-10)
    assert np.all(pase.relative_residuals(pb.A, pb.M, U[:, :nev], lam[:nev]) <= 1e-10)
    # subspace match of the first nev vectors (eigenvalues of this pencil are simple
    # or exactly degenerate; compare projectors)
    Q = U_d[:, :nev]
    Uc = U[:, :nev]
    proj = Uc - Q @ (Q.T @ (pb.M @ Uc))
    assert np.sqrt(np.max(np.einsum("ij,ij->j", proj, pb.M @ proj))) < 1e-7


def test_as_solve_closed_form_2d_128():
    pb = pin.build_problem(2, 128, 16)
    m = pin.guard_columns(10)
    S = pase.Solver(pb.A, pb.M, pb.chain)
    lam, U, info = S.solve(10, m, 1e-8, U0=pin.start_vectors(0, pb.N, m), s=2, max_iter=40)
    assert info["converged"]
    ex = spectrum.q1_laplace_eigenvalues(2, 128, 10)
    np.testing.assert_allclose(lam[:10], ex, rtol=1e-10)


def test_cg_solver_form_converges():
    pb = _tiny()
    m = 8
    S = pase.Solver(pb.A, pb.M, pb.chain)
    lam, U, info = S.solve(4, m, 1e-9, U0=pin.start_vectors(1, pb.N, m), s=10, max_iter=60, solver="cg")
    assert info["converged"]
    np.testing.assert_allclose(lam[:4], spectrum.q1_laplace_eigenvalues(2, 16, 4), rtol=1e-10)


def test_mgcg_solver_form_matches_brute_force_rough():
    pb = pin.build_problem(2, 16, 4, kappa_seed=13, sigma=2.0)
    m = 8
    S = pase.Solver(pb.A, pb.M, pb.chain)
    lam, U, info = S.solve(4, m, 1e-10, U0=pin.start_vectors(2, pb.N, m), s=3, max_iter=80, solver="mgcg")
    assert info["converged"]
    np.testing.assert_allclose(lam[:4], dense.smallest_pairs(pb.A, pb.M, 4)[0], rtol=1e-10)


def test_coarse_start_is_galerkin_coarse_spectrum():
    pb = _tiny()
    lam, U0 = pase.coarse_start(pb.A_H, pb.M_H, pb.P, 4)
    np.testing.assert_allclose(lam, spectrum.q1_laplace_eigenvalues(2, 4, 4), rtol=1e-12)
    # interpolated coarse eigenvectors keep their Rayleigh quotients on the fine pencil
    np.testing.assert_allclose(pase.rayleigh_quotients(pb.A, pb.M, U0), lam, rtol=1e-12)


def test_warm_start_fixed_point():
    """If W holds exact eigenvectors, the augmented problem returns them (u_H = 0,
    gamma = I is the solution, §3 discussion of the initial guess)."""
    pb = _tiny()
    m = 6
    lam_d, U_d = dense.smallest_pairs(pb.A, pb.M, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, U_d)
    lam, C_H, C_W = pase.augmented_eig(pb.A_H, pb.M_H, aH, bH, GA, GM, m)
    np.testing.assert_allclose(lam, lam_d, rtol=1e-12)
    U = pase.prolongate(pb.P, U_d, C_H, C_W)
    # U spans the same space as U_d (degenerate pairs may come back rotated)
    G = U_d.T @ (pb.M @ U)
    np.testing.assert_allclose(G.T @ G, np.eye(m), atol=1e-9)
    np.testing.assert_allclose(U_d @ G, U, atol=1e-9)


def test_precond_a_congruence_preserves_spectrum():
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    Ahat, Bhat = pase.augmented_pencil(pb.A_H, pb.M_H, aH, bH, GA, GM)
    ref = sl.eigh(Ahat, Bhat, eigvals_only=True)
    ahat, alpha_t, b_t, beta_t = pase.precond_a(pb.A_H, pb.M_H, aH, bH, GA, GM)
    NH = pb.N_H
    At = np.block([[pb.A_H.toarray(), np.zeros((NH, m))], [np.zeros((m, NH)), alpha_t]])
    Bt = np.block([[pb.M_H.toarray(), b_t], [b_t.T, beta_t]])
    got = sl.eigh(0.5 * (At + At.T), 0.5 * (Bt + Bt.T), eigvals_only=True)
    np.testing.assert_allclose(got, ref, rtol=1e-10)
    # back transform gives eigenvectors of the original pencil
    lt, Yt = sl.eigh(0.5 * (At + At.T), 0.5 * (Bt + Bt.T), subset_by_index=[0, m - 1])
    uH, g = pase.precond_a_back(ahat, Yt[:NH], Yt[NH:])
    Y = np.vstack([uH, g])
    np.testing.assert_allclose(Ahat @ Y, Bhat @ Y * lt, atol=1e-8 * abs(lt).max())


def _congruence_T(NH, m, Z):
    return np.block([[np.eye(NH), Z], [np.zeros((m, NH)), np.eye(m)]])


def test_precond_b_congruence():
    """PRECOND-B's blocks equal T^-T A_Hh T^-1 and T^-T B_Hh T^-1 for T = [[I, B_H^-1 b_h],
    [0, I]] formed densely (which pins every term of the formulas), B_Hh becomes block
    diagonal, the spectrum is unchanged and eigenvectors map back."""
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    Ahat, Bhat = pase.augmented_pencil(pb.A_H, pb.M_H, aH, bH, GA, GM)
    NH = pb.N_H
    bhat, a_t, alpha_t, beta_t = pase.precond_b(pb.A_H, pb.M_H, aH, bH, GA, GM)
    Ti = np.linalg.inv(_congruence_T(NH, m, bhat))
    At_dense = Ti.T @ Ahat @ Ti
    Bt_dense = Ti.T @ Bhat @ Ti
    At = np.block([[pb.A_H.toarray(), a_t], [a_t.T, alpha_t]])
    Bt = np.block([[pb.M_H.toarray(), np.zeros((NH, m))], [np.zeros((m, NH)), beta_t]])
    scale = np.abs(Ahat).max()
    np.testing.assert_allclose(At_dense, At, atol=1e-11 * scale)
    np.testing.assert_allclose(Bt_dense, Bt, atol=1e-11 * np.abs(Bhat).max())
    ref = sl.eigh(Ahat, Bhat, eigvals_only=True)
    got = sl.eigh(0.5 * (At + At.T), 0.5 * (Bt + Bt.T), eigvals_only=True)
    np.testing.assert_allclose(got, ref, rtol=1e-10)
    lt, Yt = sl.eigh(0.5 * (At + At.T), 0.5 * (Bt + Bt.T), subset_by_index=[0, m - 1])
    uH, g = pase.precond_a_back(bhat, Yt[:NH], Yt[NH:])
    Y = np.vstack([uH, g])
    np.testing.assert_allclose(Ahat @ Y, Bhat @ Y * lt, atol=1e-8 * abs(lt).max())


def test_precond_a_blocks_equal_dense_congruence():
    """PRECOND-A's blocks equal T^-T A_Hh T^-1, T^-T B_Hh T^-1 for T = [[I, A_H^-1 a_h],[0, I]]."""
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    Ahat, Bhat = pase.augmented_pencil(pb.A_H, pb.M_H, aH, bH, GA, GM)
    NH = pb.N_H
    ahat, alpha_t, b_t, beta_t = pase.precond_a(pb.A_H, pb.M_H, aH, bH, GA, GM)
    Ti = np.linalg.inv(_congruence_T(NH, m, ahat))
    At = np.block([[pb.A_H.toarray(), np.zeros((NH, m))], [np.zeros((m, NH)), alpha_t]])
    Bt = np.block([[pb.M_H.toarray(), b_t], [b_t.T, beta_t]])
    np.testing.assert_allclose(Ti.T @ Ahat @ Ti, At, atol=1e-11 * np.abs(Ahat).max())
    np.testing.assert_allclose(Ti.T @ Bhat @ Ti, Bt, atol=1e-11 * np.abs(Bhat).max())


def test_precond_ba_factorisation():
    """PRECOND-B-A: the factors reproduce the B-transformed A_Hh, and the factorisation is
    the one PRECOND-A applies (its Schur complement has the PRECOND-A form on the
    transformed blocks)."""
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    NH = pb.N_H
    bhat, a_t, alpha_t, beta_t, ahat2, S = pase.precond_ba(pb.A_H, pb.M_H, aH, bH, GA, GM)
    At = np.block([[pb.A_H.toarray(), a_t], [a_t.T, alpha_t]])
    L = np.block([[np.eye(NH), np.zeros((NH, m))], [ahat2.T, np.eye(m)]])
    D = np.block([[pb.A_H.toarray(), np.zeros((NH, m))], [np.zeros((m, NH)), S]])
    np.testing.assert_allclose(L @ D @ L.T, At, atol=1e-11 * np.abs(At).max())
    ahat_a, alpha_a, _, _ = pase.precond_a(pb.A_H, pb.M_H, a_t, np.zeros_like(bH), alpha_t, beta_t)
    np.testing.assert_allclose(ahat_a, ahat2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(alpha_a, S, atol=1e-11 * np.abs(S).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)  # a Schur complement of an SPD matrix


def test_convergence_rate_independent_of_h():
    """Theorem 2.1: for a fixed coarse space the contraction per iteration does not
    deteriorate as h decreases.  Band test on the first pair, 2D, H = 1/8."""
    rates = []
    for n in (32, 64, 128):
        pb = pin.build_problem(2, n, 8)
        m = 8
        S = pase.Solver(pb.A, pb.M, pb.chain)
        _, _, info = S.solve(4, m, 1e-13, U0=pin.start_vectors(0, pb.N, m), s=2, max_iter=12)
        h = np.array([r[0] for r in info["history"]])
        k = min(len(h) - 1, 5)
        rates.append((h[k] / h[1]) ** (1.0 / (k - 1)))
    assert max(rates) < 0.5
    assert max(rates) / min(rates) < 4.0


# ------------------------------------------------------------ planted-mistake checks


def _mutant_augmented_pencil(A_H, M_H, aH, bH, GA, GM):
    Ahat = np.block([[A_H.toarray(), aH], [aH.T, GA]])
    Bhat = np.block([[M_H.toarray(), 0 * bH], [0 * bH.T, GM]])  # dropped coupling term
    return Ahat, Bhat


def test_planted_mistakes_are_caught(monkeypatch):
    pb = _tiny()
    m = 6
    lam_d, U_d = dense.smallest_pairs(pb.A, pb.M, m)
    W = U_d + 0.01 * pin.start_vectors(3, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    good, _, _ = pase.augmented_eig(pb.A_H, pb.M_H, aH, bH, GA, GM, m)
    # Ritz values of a subspace containing V_H and near-eigenvectors: upper bounds, close
    assert np.all(good >= lam_d - 1e-9) and np.all((good - lam_d) / lam_d < 1e-3)
    monkeypatch.setattr(pase, "augmented_pencil", _mutant_augmented_pencil)
    bad, _, _ = pase.augmented_eig(pb.A_H, pb.M_H, aH, bH, GA, GM, m)
    assert not (np.all(bad >= lam_d - 1e-9) and np.all((bad - lam_d) / lam_d < 1e-3))
    monkeypatch.undo()
    # a transposed restriction (P instead of P^T on the wrong side) breaks the shapes
    with pytest.raises(ValueError):
        pb.P @ (pb.A @ W)


# ------------------------------------------------------------ the acceptance residual


def test_relative_residuals_hand_computed():
    """relative_residuals on a 2x2 diagonal pencil, values worked out by hand.

    A = diag(2, 3), M = diag(1, 4), u = (1, 1):  A u = (2, 3), M u = (1, 4), ||M u|| = sqrt(17).
      lambda = 1:  A u - M u   = (1, -1)  ->  sqrt(2) / sqrt(17)
      lambda = 2:  A u - 2 M u = (0, -5)  ->  5 / (2 sqrt(17))
      lambda = -1: A u + M u   = (3, 7)   ->  sqrt(58) / sqrt(17)   (|lambda| in the scale)
    Dividing by ||u|| = sqrt(2) instead of ||M u||, by lambda^2 instead of |lambda|, or
    dropping M from the residual changes every one of these numbers."""
    import scipy.sparse as sp
    A = sp.csr_matrix(np.diag([2.0, 3.0]))
    M = sp.csr_matrix(np.diag([1.0, 4.0]))
    U = np.ones((2, 3))
    lam = np.array([1.0, 2.0, -1.0])
    want = np.array([np.sqrt(2.0 / 17.0), 5.0 / (2.0 * np.sqrt(17.0)), np.sqrt(58.0 / 17.0)])
    np.testing.assert_allclose(pase.relative_residuals(A, M, U, lam), want, rtol=1e-15)
    # an exact eigenpair of the pencil has zero residual; scaling u leaves the value unchanged
    e = np.array([[0.0], [1.0]])
    assert pase.relative_residuals(A, M, 7.0 * e, np.array([0.75]))[0] == 0.0
    V = np.array([[1.0, 3.0], [2.0, -1.0]])
    np.testing.assert_allclose(pase.relative_residuals(A, M, 5.0 * V, np.array([1.5, 2.5])),
                               pase.relative_residuals(A, M, V, np.array([1.5, 2.5])), rtol=1e-15)


def test_relative_residuals_planted_mistakes_fail_the_pin():
    """The hand-computed pin rejects the plausible slips in the residual's definition."""
    import scipy.sparse as sp
    A = sp.csr_matrix(np.diag([2.0, 3.0]))
    M = sp.csr_matrix(np.diag([1.0, 4.0]))
    U = np.ones((2, 3))
    lam = np.array([1.0, 2.0, -1.0])
    want = pase.relative_residuals(A, M, U, lam)
    R = A @ U - (M @ U) * lam
    slips = [
        np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(U, axis=0)),           # ||u||
        np.linalg.norm(R, axis=0) / (lam ** 2 * np.linalg.norm(M @ U, axis=0)),          # lambda^2
        np.linalg.norm(A @ U - U * lam, axis=0) / (np.abs(lam) * np.linalg.norm(M @ U, axis=0)),  # no M
        np.linalg.norm(R, axis=0) / np.abs(lam),                                          # paper's raw form
    ]
    for s in slips:
        assert np.max(np.abs(s - want) / want) > 0.1


def test_post_solve_form_matches_brute_force():
    """Alg. 3's two-solve form (step-7 solve after each Rayleigh-Ritz) reaches the brute-force
    pairs and, doing two linear solves per iteration, needs no more iterations than the
    one-solve form."""
    pb = _tiny()
    nev, m = 4, 8
    lam_d, _ = dense.smallest_pairs(pb.A, pb.M, nev)
    solver = pase.Solver(pb.A, pb.M, pb.chain, pb.coarse_level)
    U0 = pin.start_vectors(0, pb.N, m)
    lam1, U1, info1 = solver.solve(nev, m, 1e-10, U0=U0)
    lam2, U2, info2 = solver.solve(nev, m, 1e-10, U0=U0, post_solve=True)
    assert info1["converged"] and info2["converged"]
    np.testing.assert_allclose(lam2[:nev], lam_d, rtol=1e-10)
    assert info2["iterations"] <= info1["iterations"]
    # the returned block is the Rayleigh-Ritz one: M-orthonormal
    np.testing.assert_allclose(U2.T @ (pb.M @ U2), np.eye(m), atol=1e-10)


# ------------------------------------------------------------ variable tensor + potential operator


def _const_tensor(d, T):
    return lambda X: np.broadcast_to(np.asarray(T, dtype=float), X.shape[:-1] + (d, d))


def test_coefficient_assembly_reduces_to_laplace_and_shift():
    """T = I, phi = 0 gives the Q1 Laplace stiffness; phi = c adds c times the mass."""
    for d, n in ((2, 7), (3, 5)):
        A0, M0 = pin.q1_matrices(d, n)
        A, M = pin.q1_matrices_coefficients(d, n, _const_tensor(d, np.eye(d)), lambda X: np.zeros(X.shape[:-1]))
        assert abs(A - A0).max() < 1e-13 * abs(A0).max() and abs(M - M0).max() == 0.0
        A, _ = pin.q1_matrices_coefficients(d, n, _const_tensor(d, np.eye(d)), lambda X: np.full(X.shape[:-1], 2.5))
        assert abs(A - (A0 + 2.5 * M0)).max() < 1e-13 * abs(A0).max()


def test_coefficient_assembly_anisotropic_closed_form():
    """T = diag(a) constant: the pencil is sum_k a_k K_k against the tensor mass, whose
    eigenvalues are sum_k a_k mu_{i_k} with mu the 1D P1 values (6/h^2)(1-cos)/(2+cos)."""
    d, n = 3, 6
    a = np.array([1.0, 2.5, 0.5])
    A, M = pin.q1_matrices_coefficients(d, n, _const_tensor(d, np.diag(a)), lambda X: np.zeros(X.shape[:-1]))
    h = 1.0 / n
    k = np.arange(1, n)
    mu = (6.0 / h ** 2) * (1.0 - np.cos(k * np.pi * h)) / (2.0 + np.cos(k * np.pi * h))
    ref = np.sort((a[0] * mu[:, None, None] + a[1] * mu[None, :, None] + a[2] * mu[None, None, :]).ravel())
    got = sl.eigh(A.toarray(), M.toarray(), eigvals_only=True)
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def _loop_coefficient_assembly(d, n, tensor, potential, q=3):
    """Element-by-element assembly with explicit loops (written independently of the
    vectorised one): Gauss-Legendre points, P1 hats and their gradients evaluated per point."""
    h = 1.0 / n
    n1 = n - 1
    N = n1 ** d
    A = np.zeros((N, N))
    xg, wg = np.polynomial.legendre.leggauss(q)
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg
    import itertools
    for ec in itertools.product(range(n), repeat=d):          # ec = (ex, ey[, ez])
        for qi in itertools.product(range(q), repeat=d):
            xi = np.array([xg[j] for j in qi])
            w = np.prod([wg[j] for j in qi]) * h ** d
            X = (np.array(ec) + xi) * h
            T = tensor(X[None, None, :])[0, 0]
            ph = potential(X[None, None, :])[0, 0]
            locs, vals, grads = [], [], []
            for a in itertools.product((0, 1), repeat=d):
                node = [ec[k] + a[k] for k in range(d)]
                if not all(1 <= v <= n1 for v in node):
                    continue
                gi = sum((node[k] - 1) * n1 ** k for k in range(d))
                l = [xi[k] if a[k] else 1.0 - xi[k] for k in range(d)]
                dl = [(1.0 if a[k] else -1.0) / h for k in range(d)]
                g = np.array([dl[k] * np.prod([l[j] for j in range(d) if j != k]) for k in range(d)])
                locs.append(gi)
                vals.append(np.prod(l))
                grads.append(g)
            for i, gi in enumerate(locs):
                for j, gj in enumerate(locs):
                    A[gi, gj] += w * (grads[i] @ T @ grads[j] + ph * vals[i] * vals[j])
    return A


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_coefficient_assembly_matches_loop_assembly(d, n):
    """The section-6.3 coefficients (full tensor, potential) against the loop assembly."""
    T, phi = pin.tensor_potential_coefficients(d)
    A, _ = pin.q1_matrices_coefficients(d, n, T, phi)
    ref = _loop_coefficient_assembly(d, n, T, phi)
    np.testing.assert_allclose(A.toarray(), ref, atol=1e-13 * np.abs(ref).max())


def test_tensor_potential_spectrum_sandwich():
    """T(x) = I + y y^T (y = x - 1/2) has eigenvalues in [1, 1 + d/4] and phi = exp(prod y)
    lies in [e^-1/8, e^1/8] on the cube, and the quadrature weights are positive, so by
    Courant-Fischer every eigenvalue lies between lambda_i(Laplace) + e^-1/8 and
    (1 + d/4) lambda_i(Laplace) + e^1/8."""
    d, n = 3, 8
    pb = pin.build_problem(d, n, 4, operator="tensor")
    lam = sl.eigh(pb.A.toarray(), pb.M.toarray(), eigvals_only=True)
    lap = spectrum.q1_laplace_eigenvalues(d, n, len(lam))
    assert np.all(lam >= lap + np.exp(-0.125) - 1e-9)
    assert np.all(lam <= (1 + d / 4.0) * lap + np.exp(0.125) + 1e-9)
    assert abs(pb.A - pb.A.T).max() < 1e-14 * abs(pb.A).max()


# ------------------------------------------------------------ batch scheme (§5)


def test_component_norms_equal_explicit_projection():
    """||Pi_h v_i||_b^2 from the X beta X^T formula equals the b-norm of the b-orthogonal
    projection of the explicitly formed fine vector v_i onto span(W)."""
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    rng = np.random.default_rng(3)
    uH = rng.standard_normal((pb.N_H, 7))
    gam = rng.standard_normal((m, 7))
    V = pb.P @ uH + W @ gam
    MW = pb.M @ W
    Pv = W @ np.linalg.solve(W.T @ MW, MW.T @ V)          # b-orthogonal projection onto span(W)
    ref = np.einsum("ij,ij->j", Pv, pb.M @ Pv)
    np.testing.assert_allclose(pase.component_norms(uH, gam, bH, GM), ref, rtol=1e-10)
    # a vector of span(W) is its own projection; one b-orthogonal to span(W) has none
    np.testing.assert_allclose(pase.component_norms(np.zeros((pb.N_H, m)), np.eye(m), bH, GM), np.diag(GM),
                               rtol=1e-12)


def test_nearest_pairs_are_the_closest_to_the_shift():
    pb = _tiny(kappa_seed=4)
    m = 5
    W = pin.start_vectors(2, pb.N, m)
    aH, bH, GA, GM = pase.projection(pb.A, pb.M, pb.P, W)
    Ahat, Bhat = pase.augmented_pencil(pb.A_H, pb.M_H, aH, bH, GA, GM)
    full = sl.eigh(Ahat, Bhat, eigvals_only=True)
    theta = 0.5 * (full[6] + full[7])
    lam, CH, CW = pase.nearest_pairs(pb.A_H, pb.M_H, aH, bH, GA, GM, theta, 4)
    # four eigenvalues of the pencil, ascending, none farther from theta than any left out
    dist = np.abs(full - theta)
    inside = np.array([np.min(np.abs(full - l)) for l in lam])
    assert np.all(inside <= 1e-9 * np.abs(full).max()) and np.all(np.diff(lam) > 0)
    kept = np.argsort(dist)[:4]
    assert np.max(np.abs(lam - theta)) <= np.min(np.delete(dist, kept)) + 1e-9
    Y = np.vstack([CH, CW])
    np.testing.assert_allclose(Ahat @ Y, Bhat @ Y * lam, atol=1e-9 * np.abs(lam).max())


def test_batch_bounds_keep_clusters_together():
    lam = np.array([1.0, 2.0, 3.0, 3.0, 3.0, 5.0, 6.0, 7.0, 7.0000001, 9.0])
    assert pase.batch_bounds(lam, 9, 3) == [(0, 5), (5, 9)]
    assert pase.batch_bounds(lam, 8, 2) == [(0, 2), (2, 5), (5, 7), (7, 8)]  # nev ends the last batch


def test_batch_scheme_matches_the_smallest_pairs():
    """Alg. 7 with three batches on the section-6.3 operator (2D, 64^2 mesh, coarse 32^2)
    returns the first 24 pairs of the pencil, M-orthonormal across batches."""
    pb = pin.build_problem(2, 64, 32, mg_min=4, operator="tensor")
    solver = pase.Solver(pb.A, pb.M, pb.chain, pb.coarse_level)
    nev = 24
    lam, U, info = pase.batch_scheme(solver, nev, 8, 1e-9, guard=4, max_iter=40)
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)
    assert np.all(pase.relative_residuals(pb.A, pb.M, U, lam) <= 1e-9)
    np.testing.assert_allclose(U.T @ (pb.M @ U), np.eye(nev), atol=1e-9)
    assert len(info["iterations"]) == 3
