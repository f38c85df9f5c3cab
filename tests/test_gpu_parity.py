"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

Tolerances (FP64 path): kernels that only reorder a sum (sparse products, Gram blocks,
restriction, prolongation, V-cycle) agree to 1e-12 relative in the norm of each column;
eigenvalues to 1e-10 relative (the accuracy target of the method); eigenvectors by
subspace (degenerate Laplace pairs may come back rotated); relative residuals of the
returned pairs <= the requested tolerance, recomputed on the CPU by the oracle.
"""
import numpy as np
import pytest

import pase_inputs as pin
from oracle import dense, mg, pase as opase, spectrum

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _colrel(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))


class Ctx:
    def __init__(self, pb, precision=P.PASE_PREC_FP64, **kw):
        self.pb = pb
        opt = P.pase_default_options()
        opt.precision = precision
        opt.coarse_level = pb.coarse_level
        for k, v in kw.items():
            setattr(opt, k, v)
        self.h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
        try:
            P.pase_setup(self.h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        except Exception:
            P.pase_destroy(self.h)
            raise

    def close(self):
        P.pase_destroy(self.h)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def p2d():
    return pin.build_problem(2, 64, 8, mg_min=4)


@pytest.fixture(scope="module")
def p3d():
    return pin.build_problem(3, 32, 8, kappa_seed=5, mg_min=4)


@pytest.mark.parametrize("which,m", [("p2d", 8), ("p2d", 24), ("p3d", 16), ("p3d", 40)])
def test_spmm_am_parity(which, m, request):
    pb = request.getfixturevalue(which)
    c = Ctx(pb)
    try:
        X = pin.start_vectors(3, pb.N, m)
        AX = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        MX = torch.empty_like(AX)
        P.pase_spmm_am(c.h, m, dev(X), AX, MX)
        assert _colrel(host(AX), pb.A @ X) < 1e-13
        assert _colrel(host(MX), pb.M @ X) < 1e-13
    finally:
        c.close()


def test_spmm_am_fresh_handles_repeat(p2d):
    """The fused A_h/M_h product from 100 fresh handles in a row (set-up, autotuner and
    first launch each time), every result checked: a wrong M_h X once seen on the first
    call of a process must not come back on any first call of a handle."""
    pb, m = p2d, 8
    X = pin.start_vectors(3, pb.N, m)
    Xd = dev(X)
    AXr, MXr = pb.A @ X, pb.M @ X
    bad = []
    for k in range(100):
        c = Ctx(pb)
        try:
            AX = torch.full((pb.N, m), np.nan, dtype=torch.float64, device="cuda")
            MX = torch.full_like(AX, np.nan)
            P.pase_spmm_am(c.h, m, Xd, AX, MX)
            ea, em = _colrel(host(AX), AXr), _colrel(host(MX), MXr)
            if not (ea < 1e-13 and em < 1e-13):
                bad.append((k, ea, em))
        finally:
            c.close()
    assert not bad, bad


_FIRST_CALL = r"""
import numpy as np, torch, pase_inputs as pin
from paper_2502_04589_gb300 import pase as P
pb = pin.build_problem(2, 64, 8, mg_min=4)
opt = P.pase_default_options(); opt.coarse_level = pb.coarse_level
h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
m = 8
X = pin.start_vectors(3, pb.N, m)
AX = torch.empty(pb.N, m, dtype=torch.float64, device="cuda"); MX = torch.empty_like(AX)
P.pase_spmm_am(h, m, torch.from_numpy(X).cuda(), AX, MX)
rel = lambda a, b: np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))
ea, em = rel(AX.cpu().numpy(), pb.A @ X), rel(MX.cpu().numpy(), pb.M @ X)
P.pase_destroy(h)
print("ERR", ea, em)
assert ea < 1e-13 and em < 1e-13
"""


def test_spmm_am_first_call_of_fresh_processes():
    """The same product as the first GPU work of three fresh processes."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    for _ in range(3):
        r = subprocess.run([sys.executable, "-c", _FIRST_CALL], cwd=root, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("which,m", [("p2d", 8), ("p3d", 40)])
def test_spmm_df64_matches_fp64_and_definition(which, m, request):
    """The double-float fused product (default) against the FP64 kernel (spmm_df64 = 0) and
    the definition, entry by entry: within 2048 u of sum_k |a_ik||x_kj| (the split loses 5
    of 53 bits per operand, the sums gather a few 2^-48 per term); inputs spread over 2^+-60."""
    pb = request.getfixturevalue(which)
    rng = np.random.default_rng(5)
    X = pin.start_vectors(21, pb.N, m) * np.exp2(rng.integers(-60, 61, size=(pb.N, 1)))
    out = {}
    for df in (1, 0):
        c = Ctx(pb, spmm_df64=df)
        try:
            AX = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
            MX = torch.empty_like(AX)
            P.pase_spmm_am(c.h, m, dev(X), AX, MX)
            out[df] = (host(AX), host(MX))
        finally:
            c.close()
    u = 2.0 ** -53
    for q, Mat in ((0, pb.A), (1, pb.M)):
        scale = abs(Mat) @ np.abs(X)
        ref = Mat @ X
        assert np.all(np.abs(out[1][q] - ref) <= 2048 * u * scale)
        assert np.all(np.abs(out[1][q] - out[0][q]) <= 2048 * u * scale)


def test_spmm_df64_reports_out_of_range_entries(p2d):
    """An entry above 2^100 cannot be split into FP32 pairs: the call reports PASE_ERR_NAN,
    and the next call on ordinary data works (the flag is cleared)."""
    pb, m = p2d, 8
    c = Ctx(pb)
    try:
        X = pin.start_vectors(22, pb.N, m)
        X[17, 3] = 1e40
        AX = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        MX = torch.empty_like(AX)
        with pytest.raises(P.PaseError) as e:
            P.pase_spmm_am(c.h, m, dev(X), AX, MX)
        assert e.value.code == -5
        X[17, 3] = 0.5
        P.pase_spmm_am(c.h, m, dev(X), AX, MX)
        assert _colrel(host(AX), pb.A @ X) < 1e-13
    finally:
        c.close()


def test_residual_parity(p3d):
    pb = p3d
    m = 16
    c = Ctx(pb)
    try:
        U = pin.start_vectors(4, pb.N, m)
        lam = np.linspace(10.0, 200.0, m)
        R = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        rr = torch.empty(m, dtype=torch.float64, device="cuda")
        P.pase_residual(c.h, m, dev(U), dev(lam), R, rr)
        Rref = (pb.M @ U) * lam - pb.A @ U
        assert _colrel(host(R), Rref) < 1e-13
        np.testing.assert_allclose(host(rr), opase.relative_residuals(pb.A, pb.M, U, lam), rtol=1e-12)
    finally:
        c.close()


@pytest.mark.parametrize("which", ["p2d", "p3d"])
def test_linear_solve_parity(which, request):
    pb = request.getfixturevalue(which)
    m = 16
    c = Ctx(pb)
    try:
        U = pin.start_vectors(5, pb.N, m)
        lam = np.linspace(20.0, 300.0, m)
        W = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        P.pase_linear_solve(c.h, m, dev(U), dev(lam), None, W)
        hier = mg.Hierarchy(pb.A, pb.chain)
        Wref = opase.linear_solve(pb.A, pb.M, U, lam, 2, hier)
        assert _colrel(host(W) - U, Wref - U) < 1e-11
    finally:
        c.close()


@pytest.mark.parametrize("solver,name", [(P.PASE_SOLVER_CG, "cg"), (P.PASE_SOLVER_MGCG, "mgcg")])
@pytest.mark.parametrize("which", ["p2d", "p3d"])
def test_linear_solve_cg_forms_parity(which, solver, name, request):
    """CG and V-cycle-preconditioned CG step (a), FP64: the same recurrences as the
    oracle, so only summation order differs."""
    pb = request.getfixturevalue(which)
    m = 16
    c = Ctx(pb, linear_solver=solver, inner_steps=3)
    try:
        U = pin.start_vectors(5, pb.N, m)
        lam = np.linspace(20.0, 300.0, m)
        W = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        P.pase_linear_solve(c.h, m, dev(U), dev(lam), None, W)
        hier = mg.Hierarchy(pb.A, pb.chain)
        Wref = opase.linear_solve(pb.A, pb.M, U, lam, 3, hier, name)
        assert _colrel(host(W) - U, Wref - U) < 1e-11
    finally:
        c.close()


def test_linear_solve_mgcg_mixed_parity(p3d):
    """MIXED precision: the V-cycle preconditioner runs in FP32 (unit roundoff 6e-8), the
    CG recurrences in FP64; the correction agrees with the FP64 oracle to about 1e-6."""
    pb = p3d
    m = 16
    c = Ctx(pb, P.PASE_PREC_MIXED, linear_solver=P.PASE_SOLVER_MGCG, inner_steps=3)
    try:
        U = pin.start_vectors(5, pb.N, m)
        lam = np.linspace(20.0, 300.0, m)
        W = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        P.pase_linear_solve(c.h, m, dev(U), dev(lam), None, W)
        Wref = opase.linear_solve(pb.A, pb.M, U, lam, 3, mg.Hierarchy(pb.A, pb.chain), "mgcg")
        assert _colrel(host(W) - U, Wref - U) < 1e-5
    finally:
        c.close()


@pytest.mark.parametrize("which", ["p2d", "p3d"])
def test_project_parity(which, request):
    pb = request.getfixturevalue(which)
    m = 24
    c = Ctx(pb)
    try:
        W = pin.start_vectors(6, pb.N, m)
        aH = torch.empty(pb.N_H, m, dtype=torch.float64, device="cuda")
        bH, GA, GM = torch.empty_like(aH), torch.empty(m, m, dtype=torch.float64, device="cuda"), None
        GM = torch.empty_like(GA)
        P.pase_project(c.h, m, dev(W), aH, bH, GA, GM)
        ra, rb, rga, rgm = opase.projection(pb.A, pb.M, pb.P, W)
        assert _colrel(host(aH), ra) < 1e-12
        assert _colrel(host(bH), rb) < 1e-12
        assert _rel(host(GA), rga) < 1e-12
        assert _rel(host(GM), rgm) < 1e-12
        assert np.array_equal(host(GA), host(GA).T)  # exactly symmetric
    finally:
        c.close()


@pytest.mark.parametrize("which,m", [("p2d", 8), ("p2d", 16), ("p3d", 24), ("p3d", 96)])
def test_augmented_eig_parity(which, m, request):
    """m = 96 gives Rayleigh-Ritz blocks of 3m = 288 whose triangles no longer fit in
    shared memory, so the global-memory variants of the small eigensolver run."""
    _augmented_eig_check(request.getfixturevalue(which), m)


@pytest.mark.parametrize("tri,chol", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1), (2, 0)])
@pytest.mark.parametrize("which,m", [("p2d", 16), ("p3d", 24), ("p3d", 96)])
def test_augmented_eig_small_eigensolver_forms(which, m, tri, chol, request):
    """Every form of the Rayleigh-Ritz eigensolver, fixed for all its sizes (m, 2m, 3m):
    tridiagonalisation on one CTA, a cluster of 8 or of 16 SMs; Cholesky on one CTA or a
    cluster of 8 SMs.  Late passes soft-lock converged columns, so the Gram matrices carry
    dropped directions through every form."""
    _augmented_eig_check(request.getfixturevalue(which), m, sygv_tridiag=tri, sygv_cholesky=chol)


@pytest.mark.parametrize("transform", [P.PASE_AUG_PRECOND_A, P.PASE_AUG_PRECOND_B, P.PASE_AUG_PRECOND_BA])
@pytest.mark.parametrize("which,m", [("p2d", 16), ("p3d", 24)])
def test_augmented_eig_transform_parity(which, m, transform, request):
    """Step (c) through the PRECOND-A / -B / -B-A congruences of §4 returns the pairs of the
    untransformed pencil (dense oracle), mapped back to the original basis."""
    _augmented_eig_check(request.getfixturevalue(which), m, aug_transform=transform)


@pytest.fixture(scope="module")
def p3d_small():
    return pin.build_problem(3, 16, 4, kappa_seed=7, mg_min=4)


def test_augmented_eig_dense_small_space(p3d_small):
    """N_H + m = 27 + 16 <= 3m: the augmented pencil is assembled densely and solved in one
    generalized eigensolve (the block eigensolver's basis would exceed the space)."""
    _augmented_eig_check(p3d_small, 16)


@pytest.mark.parametrize("graph_solve", [0, 1])
def test_solve_small_coarse_space_dense_steps(p3d_small, graph_solve):
    """Coarse start and every step (c) dense (N_H = 27 <= 3m): pairs against shift-invert,
    M-orthonormal block."""
    pb, nev, m = p3d_small, 5, 16
    c = Ctx(pb, graph_solve=graph_solve)
    try:
        U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        rc, st = P.pase_solve(c.h, nev, 1e-9, m, None, lam, U)
        assert rc == P.PASE_OK
        ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
        _check_pairs(pb, host(lam), host(U), nev, ref, 1e-9)
    finally:
        c.close()


def _augmented_eig_check(pb, m, **kw):
    c = Ctx(pb, aug_adaptive=0, aug_max_iter=200, **kw)
    try:
        if pb.N <= 5000:
            lam_d, U_d = dense.smallest_pairs(pb.A, pb.M, m)
        else:
            lam_d, U_d = dense.smallest_pairs_shift_invert(pb.A, pb.M, m)
        W = U_d + 1e-3 * pin.start_vectors(7, pb.N, m)  # near-converged block, as in late iterations
        ra, rb, rga, rgm = opase.projection(pb.A, pb.M, pb.P, W)
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        CH = torch.empty(pb.N_H, m, dtype=torch.float64, device="cuda")
        CW = torch.empty(m, m, dtype=torch.float64, device="cuda")
        it = P.pase_augmented_eig(c.h, m, dev(ra), dev(rb), dev(rga), dev(rgm), lam, CH, CW)
        lref, CHref, CWref = opase.augmented_eig(pb.A_H, pb.M_H, ra, rb, rga, rgm, m)
        np.testing.assert_allclose(host(lam), lref, rtol=1e-10)
        U = opase.prolongate(pb.P, W, host(CH), host(CW))
        Uref = opase.prolongate(pb.P, W, CHref, CWref)
        # M-orthonormal, and the same invariant subspaces (compare M-projectors)
        np.testing.assert_allclose(U.T @ (pb.M @ U), np.eye(m), atol=1e-10)
        G = Uref.T @ (pb.M @ U)
        np.testing.assert_allclose(G.T @ G, np.eye(m), atol=1e-8)
        assert it >= 0
    finally:
        c.close()


def test_prolongate_parity(p3d):
    pb = p3d
    m = 16
    c = Ctx(pb)
    try:
        W = pin.start_vectors(8, pb.N, m)
        CH = pin.start_vectors(9, pb.N_H, m)
        CW = pin.start_vectors(10, m, m)
        U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        P.pase_prolongate(c.h, m, dev(W), dev(CH), dev(CW), U)
        assert _colrel(host(U), opase.prolongate(pb.P, W, CH, CW)) < 1e-13
    finally:
        c.close()


def test_one_iteration_parity(p2d):
    """One whole iteration from identical inputs: Ritz values and vectors vs the oracle
    (inner solve to a fixed 1e-12, no adaptive loosening)."""
    pb = p2d
    m = 8
    c = Ctx(pb, aug_adaptive=0, aug_max_iter=200)
    try:
        S = opase.Solver(pb.A, pb.M, pb.chain, coarse_level=pb.coarse_level)
        U0 = pin.start_vectors(0, pb.N, m)
        lam1, U1, _ = S.iteration(U0, None, 2, solve=False)  # first iteration: W = U0
        lam2, U2, inter = S.iteration(U1, lam1, 2, solve=True)
        Ug = dev(U0)
        lg = torch.zeros(m, dtype=torch.float64, device="cuda")
        P.pase_iterate(c.h, m, m, Ug, lg, False)
        np.testing.assert_allclose(host(lg), lam1, rtol=1e-9)
        # continue from the oracle's block so both see the same input
        Ug = dev(U1)
        lg = dev(lam1)
        P.pase_iterate(c.h, m, m, Ug, lg, True)
        np.testing.assert_allclose(host(lg), lam2, rtol=1e-10)
        G = U2.T @ (pb.M @ host(Ug))
        np.testing.assert_allclose(np.abs(G.T @ G), np.eye(m), atol=1e-7)
    finally:
        c.close()


def test_iterate_host_pointers_match_device(p2d):
    pb = p2d
    m = 8
    c = Ctx(pb)
    try:
        U0 = pin.start_vectors(11, pb.N, m)
        Uh = U0.copy()
        lh = np.zeros(m)
        P.pase_iterate(c.h, m, m, Uh, lh, False)
        Ud = dev(U0)
        ld = torch.zeros(m, dtype=torch.float64, device="cuda")
        P.pase_iterate(c.h, m, m, Ud, ld, False)
        np.testing.assert_array_equal(lh, host(ld))
        np.testing.assert_array_equal(Uh, host(Ud))
    finally:
        c.close()


def _solve(pb, nev, tol=1e-9, precision=P.PASE_PREC_FP64, m=None, seed=0, **kw):
    m = m or pin.guard_columns(nev)
    c = Ctx(pb, precision, **kw)
    try:
        U0 = dev(pin.start_vectors(seed, pb.N, m))
        U = torch.empty_like(U0)
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        rc, st = P.pase_solve(c.h, nev, tol, m, U0, lam, U)
        return rc, st, host(lam), host(U)
    finally:
        c.close()


def _check_pairs(pb, lam, U, nev, ref, tol):
    np.testing.assert_allclose(lam[:nev], ref[:nev], rtol=1e-10)
    res = opase.relative_residuals(pb.A, pb.M, U[:, :nev], lam[:nev])
    assert np.all(res <= tol), res
    np.testing.assert_allclose(U.T @ (pb.M @ U), np.eye(U.shape[1]), atol=1e-10)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_solve_laplace_2d_128(precision):
    """Config 1: 2D Q1 128x128, coarse 16x16, nev 10, two V-cycles per iteration."""
    pb = pin.build_problem(2, 128, 16, mg_min=4)
    rc, st, lam, U = _solve(pb, 10, 1e-8, precision)
    assert rc == P.PASE_OK, st
    _check_pairs(pb, lam, U, 10, spectrum.q1_laplace_eigenvalues(2, 128, 10), 1e-8)


def test_solve_variable_kappa_2d():
    pb = pin.build_problem(2, 64, 8, kappa_seed=21, mg_min=4)
    nev = 6
    rc, st, lam, U = _solve(pb, nev, 1e-9)
    assert rc == P.PASE_OK, st
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check_pairs(pb, lam, U, nev, ref, 1e-9)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_solve_rough_kappa_mgcg(precision):
    """Lognormal coefficient with sigma 1.9 (contrast ~1e6), where plain V-cycles stall:
    V-cycle-preconditioned CG in step (a) converges."""
    pb = pin.build_problem(2, 64, 8, kappa_seed=1634308976, sigma=1.9, mg_min=4)
    nev = 12
    rc, st, lam, U = _solve(pb, nev, 1e-8, precision, linear_solver=P.PASE_SOLVER_MGCG, inner_steps=3,
                            max_iter=100)
    assert rc == P.PASE_OK, st
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check_pairs(pb, lam, U, nev, ref, 1e-8)


def test_solve_plain_cg():
    pb = pin.build_problem(2, 32, 4, mg_min=4)
    rc, st, lam, U = _solve(pb, 4, 1e-9, m=8, linear_solver=P.PASE_SOLVER_CG, inner_steps=10, max_iter=60)
    assert rc == P.PASE_OK, st
    _check_pairs(pb, lam, U, 4, spectrum.q1_laplace_eigenvalues(2, 32, 4), 1e-9)


def test_solve_laplace_3d_32_cluster():
    """3D with a degenerate cluster cut by the block: nev = 10 sits inside the 10..12
    cluster? (k = (1,1,2) perms are 2..4, (1,2,2) 5..7, (1,1,3) 8..10, (2,2,2) 11)."""
    pb = pin.build_problem(3, 32, 8, mg_min=4)
    nev = 10
    rc, st, lam, U = _solve(pb, nev, 1e-8)
    assert rc == P.PASE_OK, st
    _check_pairs(pb, lam, U, nev, spectrum.q1_laplace_eigenvalues(3, 32, nev), 1e-8)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
@pytest.mark.parametrize("tri,chol", [(1, 1), (2, 1)])
def test_solve_cluster_small_eigensolver(precision, tri, chol):
    """Whole solves (3D Laplace 32^3, nev 12) with the cluster Cholesky and an 8- or 16-SM
    tridiagonalisation forced for every Rayleigh-Ritz size, against the closed form."""
    pb = pin.build_problem(3, 32, 8, mg_min=4)
    nev = 12
    rc, st, lam, U = _solve(pb, nev, 1e-8, precision, sygv_tridiag=tri, sygv_cholesky=chol)
    assert rc == P.PASE_OK, st
    _check_pairs(pb, lam, U, nev, spectrum.q1_laplace_eigenvalues(3, 32, nev), 1e-8)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_solve_post_solve_form(precision):
    """Alg. 3's two-solve form (step-7 solve after every Rayleigh-Ritz that has not
    converged): the closed-form pairs, no more outer iterations than the one-solve form, and
    (FP64) the oracle's iteration count of the same form within one."""
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    nev = 8
    m = pin.guard_columns(nev)
    ref = spectrum.q1_laplace_eigenvalues(2, 64, nev)
    rc1, st1, _, _ = _solve(pb, nev, 1e-9, precision, m=m)
    rc2, st2, lam, U = _solve(pb, nev, 1e-9, precision, m=m, post_solve=1)
    assert rc1 == P.PASE_OK and rc2 == P.PASE_OK, (st1, st2)
    _check_pairs(pb, lam, U, nev, ref, 1e-9)
    assert st2["iterations"] <= st1["iterations"], (st1["iterations"], st2["iterations"])
    if precision == P.PASE_PREC_FP64:  # step (c) to 1e-12 every time, as the oracle's dense solve
        rc3, st3, _, _ = _solve(pb, nev, 1e-9, precision, m=m, post_solve=1, aug_adaptive=0)
        solver = opase.Solver(pb.A, pb.M, pb.chain, pb.coarse_level)
        _, _, info = solver.solve(nev, m, 1e-9, U0=pin.start_vectors(0, pb.N, m), post_solve=True)
        assert rc3 == P.PASE_OK and abs(info["iterations"] - st3["iterations"]) <= 1, (info["iterations"], st3)


@pytest.mark.parametrize("transform", [P.PASE_AUG_PLAIN, P.PASE_AUG_PRECOND_A, P.PASE_AUG_PRECOND_B,
                                       P.PASE_AUG_PRECOND_BA])
def test_solve_with_aug_transform(transform):
    """Whole solves with each step-(c) variant reach the same pairs (variable kappa, 3D)."""
    pb = pin.build_problem(3, 32, 8, kappa_seed=5, mg_min=4)
    nev = 10
    rc, st, lam, U = _solve(pb, nev, 1e-9, aug_transform=transform)
    assert rc == P.PASE_OK, st
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check_pairs(pb, lam, U, nev, ref, 1e-9)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_solve_tensor_potential_3d(precision):
    """The operator of the numerical section's batch-scheme test, -div(T grad u) + phi u with
    T = I + (x - 1/2)(x - 1/2)^T and phi = exp(prod (x_k - 1/2)), on a 32^3 Q1 mesh: the 20
    smallest pairs against shift-invert Lanczos on the same matrices."""
    pb = pin.build_problem(3, 32, 8, mg_min=4, operator="tensor")
    nev = 20
    rc, st, lam, U = _solve(pb, nev, 1e-9, precision)
    assert rc == P.PASE_OK, st
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check_pairs(pb, lam, U, nev, ref, 1e-9)


def test_batch_scheme_first_pairs():
    """The batch scheme of §5 on the section-6.3 operator (2D, 64^2 mesh, coarse 32^2), FP64:
    the first 24 pairs in three batches of 8 (block 16) equal shift-invert Lanczos's, meet
    the residual tolerance, and are M-orthonormal across batches; the oracle's batch scheme
    gives the same eigenvalues.  (With the FP32 linear solve the rounding noise that the
    corrections put into the earlier batches' directions grows from iteration to iteration,
    which V_H does not remove, and a later batch stalls; the scheme is run in FP64.)"""
    pb = pin.build_problem(2, 64, 32, mg_min=4, operator="tensor")
    nev, k, m = 24, 8, 16
    precision = P.PASE_PREC_FP64
    c = Ctx(pb, precision)
    try:
        lam = np.empty(nev)
        U = np.empty((pb.N, nev))
        rc, st = P.pase_solve_batches(c.h, nev, k, m, 1e-9, lam, U)
    finally:
        c.close()
    print("\nbatch scheme:", st)
    assert rc == P.PASE_OK, st
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)
    assert np.all(opase.relative_residuals(pb.A, pb.M, U, lam) <= 1e-9)
    np.testing.assert_allclose(U.T @ (pb.M @ U), np.eye(nev), atol=1e-9)
    solver = opase.Solver(pb.A, pb.M, pb.chain, pb.coarse_level)
    lo, _, _ = opase.batch_scheme(solver, nev, k, 1e-9, guard=m - k)
    np.testing.assert_allclose(lam, lo, rtol=1e-10)


def test_setup_forms_coarse_pencil_when_not_given():
    """A_H = M_H = NULL: the library's Galerkin products through the chain give the same
    solve as the caller's."""
    pb = pin.build_problem(2, 64, 8, kappa_seed=21, mg_min=4)
    nev, m = 6, 16
    out = []
    for given in (True, False):
        opt = P.pase_default_options()
        opt.coarse_level = pb.coarse_level
        h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
        try:
            if given:
                P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
            else:
                P.pase_setup(h, pb.A, pb.M, pb.chain)
            U0 = dev(pin.start_vectors(0, pb.N, m))
            U = torch.empty_like(U0)
            lam = torch.empty(m, dtype=torch.float64, device="cuda")
            rc, st = P.pase_solve(h, nev, 1e-9, m, U0, lam, U)
            assert rc == P.PASE_OK
            out.append((st["iterations"], host(lam)[:nev]))  # guard columns are not converged
        finally:
            P.pase_destroy(h)
    assert out[0][0] == out[1][0]
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-12)


def test_coarse_start():
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    nev, m = 5, 16
    c = Ctx(pb)
    try:
        U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        rc, st = P.pase_solve(c.h, nev, 1e-9, m, None, lam, U)
        assert rc == P.PASE_OK
        _check_pairs(pb, host(lam), host(U), nev, spectrum.q1_laplace_eigenvalues(2, 64, nev), 1e-9)
    finally:
        c.close()


def test_minimum_block_and_nev1():
    pb = pin.build_problem(2, 32, 4, mg_min=4)
    rc, st, lam, U = _solve(pb, 1, 1e-9, m=8)
    assert rc == P.PASE_OK
    np.testing.assert_allclose(lam[0], spectrum.q1_laplace_eigenvalues(2, 32, 1)[0], rtol=1e-10)


def test_not_converged_status():
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    rc, st, lam, U = _solve(pb, 4, 1e-14, m=8, max_iter=2)
    assert rc == P.PASE_ERR_NOT_CONVERGED and st["iterations"] == 2


def test_errors_are_reported_not_raised_on_device(p2d):
    pb = p2d
    # pattern mismatch
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    try:
        M2 = pb.M.copy().tolil()
        M2[0, 5] = 1e-3
        M2[5, 0] = 1e-3
        with pytest.raises(P.PaseError) as e:
            P.pase_setup(h, pb.A, M2.tocsr(), pb.chain, pb.A_H, pb.M_H)
        assert e.value.code == -3
        # solve before setup
        with pytest.raises(P.PaseError) as e:
            P.pase_reserve(h, 8)
        assert e.value.code == -10
    finally:
        P.pase_destroy(h)
    c = Ctx(pb)
    try:
        with pytest.raises(P.PaseError) as e:
            P.pase_reserve(c.h, 12)
        assert e.value.code == -1
    finally:
        c.close()


@pytest.fixture(scope="module")
def p3d_128():
    """The benchmark workload: 3D Q1 Laplace 128^3, coarse 16^3, multigrid down to 4^3."""
    return pin.build_problem(3, 128, 16, mg_min=4)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_full_size_laplace_3d_128_nev50(p3d_128, precision):
    """Full-size parity at the benchmark configuration (same options as bench.py):
    eigenvalues vs the closed form, residuals and M-orthonormality recomputed on the CPU."""
    pb = p3d_128
    nev, m = 50, pin.guard_columns(50)
    rc, st, lam, U = _solve(pb, nev, 1e-8, precision, m=m, seed=0)
    assert rc == P.PASE_OK, st
    ref = spectrum.q1_laplace_eigenvalues(3, 128, nev)
    np.testing.assert_allclose(lam[:nev], ref, rtol=1e-10)
    res = opase.relative_residuals(pb.A, pb.M, U[:, :nev], lam[:nev])
    assert np.all(res <= 1e-8), res.max()
    MU = pb.M @ U
    np.testing.assert_allclose(U.T @ MU, np.eye(m), atol=1e-10)


def test_full_size_split_prolongation_sampled(p3d_128):
    """Step (d) on the tensor cores at the benchmark size (N_h = 2,048,383, m = 56, the
    launch bench.py times): sampled rows of U = W C_W against exact rational products."""
    from fractions import Fraction
    pb = p3d_128
    m = pin.guard_columns(50)
    c = Ctx(pb)
    try:
        W = pin.start_vectors(21, pb.N, m)
        CW = pin.start_vectors(22, m, m)
        U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        CH = torch.zeros(pb.N_H, m, dtype=torch.float64, device="cuda")
        P.pase_prolongate(c.h, m, dev(W), CH, dev(CW), U)
        Uh = host(U)
    finally:
        c.close()
    u = 2.0 ** -53
    rows = list(range(0, pb.N, 40961)) + [pb.N - 1]
    for r in rows:
        smax = np.abs(W[r]).max() * np.abs(CW).max(axis=0)
        for j in range(m):
            ex = sum(Fraction(float(W[r, k])) * Fraction(float(CW[k, j])) for k in range(m))
            assert abs(Fraction(float(Uh[r, j])) - ex) <= Fraction(8 * u) * Fraction(float(smax[j])) + Fraction(u) * abs(ex)
    assert _colrel(Uh, W @ CW) < 1e-14


def _jacobi_bound(A, b, x, omega, gamma):
    """Elementwise bound on the change of one damped-Jacobi sweep x + omega D^-1 (b - A x)
    when it runs in FP32: inputs, coefficients and 1/a_ii rounded (one unit each), the sum
    of the row's products accumulated in FP32 (one unit per term), gamma = (terms + 8) u."""
    d = np.abs(1.0 / A.diagonal())[:, None]
    absA = abs(A)
    return gamma * (np.abs(x) + omega * d * (np.abs(b) + absA @ np.abs(x))), d, absA


@pytest.mark.parametrize("d,n,kseed", [(3, 32, 5), (3, 20, 6), (2, 64, 7), (2, 38, 8)])
@pytest.mark.parametrize("m", [8, 56])
@pytest.mark.parametrize("stencil,cols", [(1, 4), (1, 2), (0, 0)])
def test_fp32_smoothing_parity(d, n, kseed, m, stencil, cols):
    """Two FP32 damped-Jacobi sweeps on the fine level (the mixed form's smoother) against
    the oracle's FP64 sweeps, entry by entry, within the FP32 rounding bound of the two
    sweeps (the first sweep's error carried through the second by |I| + omega |D^-1||A|).
    stencil=1 runs the structured-grid kernel (grids of 31^3, 19^3, 63^2, 37^2 nodes: ragged
    against its 16 x 4 / 64-node tiles) with 4 or 2 columns per thread, stencil=0 the CSR
    kernel (the autotuner, which may pick either per level, is off)."""
    pb = pin.build_problem(d, n, n // 2, kappa_seed=kseed)
    c = Ctx(pb, precision=P.PASE_PREC_MIXED, stencil=stencil, autotune=0, stencil_columns=cols)
    try:
        assert P.pase_smoother_form(c.h) == (d if stencil else 0)
        B = pin.start_vectors(30 + m, pb.N, m)
        X0 = pin.start_vectors(31 + m, pb.N, m)
        X = X0.copy()
        P.pase_smooth(c.h, m, 2, B, X)
        assert P.pase_smoother_form(c.h) == (d if stencil else 0)
    finally:
        c.close()
    hier = mg.Hierarchy(pb.A, pb.chain)
    om = hier.omega
    x1 = hier.smooth(0, B, X0, 1)
    x2 = hier.smooth(0, B, x1, 1)
    gamma = (3 ** d + 8) * 2.0 ** -24
    e1, dd, absA = _jacobi_bound(pb.A, B, X0, om, gamma)
    e2, _, _ = _jacobi_bound(pb.A, B, x1, om, gamma)
    e2 = e2 + e1 + om * dd * (absA @ e1)
    err = np.abs(X - x2)
    assert np.all(err <= 2.0 * e2), (np.max(err / e2), np.argmax(err / e2))
    assert np.max(err) > 0.0  # FP32 arithmetic did run


def test_fp32_smoothing_non_stencil_matrix_uses_csr():
    """A fine matrix with one coupling outside the grid neighbourhood is not taken for a
    stencil: the CSR kernel runs, with the same bound."""
    import scipy.sparse as sp
    pb = pin.build_problem(2, 32, 16, kappa_seed=3)
    N = pb.N
    E = sp.csr_matrix(([-0.1, -0.1, 0.1, 0.1], ([0, N - 1, 0, N - 1], [N - 1, 0, 0, N - 1])), shape=(N, N))
    A = pin.canonical_csr(pb.A + E)  # still symmetric and diagonally dominant
    rows, cols = A.nonzero()
    M = sp.csr_matrix((np.asarray(pb.M[rows, cols]).ravel(), A.indices.copy(), A.indptr.copy()), shape=A.shape)
    opt = P.pase_default_options()
    opt.precision = P.PASE_PREC_MIXED
    opt.coarse_level = 1
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    m = 16
    try:
        P.pase_setup(h, A, M, pb.chain)
        assert P.pase_smoother_form(h) == 0
        B = pin.start_vectors(40, N, m)
        X0 = pin.start_vectors(41, N, m)
        X = X0.copy()
        P.pase_smooth(h, m, 1, B, X)
    finally:
        P.pase_destroy(h)
    hier = mg.Hierarchy(A, pb.chain)
    x1 = hier.smooth(0, B, X0, 1)
    e1, _, _ = _jacobi_bound(A, B, X0, hier.omega, 20 * 2.0 ** -24)
    assert np.all(np.abs(X - x1) <= 2.0 * e1)
