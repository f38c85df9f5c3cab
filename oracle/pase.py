"""The augmented subspace iteration, step by step (Alg. 1, Alg. 2, Alg. 3 of the paper).

One iteration ("Correction", Alg. 1; steps 3-6 of Alg. 3), with U = [u_1..u_m] the
current block and Lambda its Ritz values:

 (a) linear solve   A_h w_i = lambda_i M_h u_i from the initial guess u_i     (Alg. 3 step 3)
 (b) projection     aH = P^T A_h W, bH = P^T M_h W, GA = W^T A_h W, GM = W^T M_h W
                    (the blocks a_h, b_h, alpha, beta of Alg. 3 step 4)
 (c) augmented eig  [[A_H, aH],[aH^T, GA]] c = lambda [[M_H, bH],[bH^T, GM]] c,
                    the m smallest pairs, B-normalised                        (Alg. 3 step 5);
                    the PRECOND-A / -B / -B-A congruences of §4 transform this pencil
 (d) prolongation   U <- P C_H + W C_W                                        (Alg. 3 step 6)

Readings taken where the paper is silent or garbled:
* Alg. 3 step 6 prints the product as gamma u-hat; the shapes (N x k times k x k)
  force u-hat gamma, i.e. W C_W.
* One linear-solve phase per Rayleigh-Ritz (Alg. 1) by default; Solver.solve(...,
  post_solve=True) runs the two-solve form of Alg. 3 (steps 3 and 7).
* Vectors are M-normalised (U^T M U = I) rather than a(u,u) = 1; the two differ by the
  factor sqrt(lambda) per column.
* Convergence is ||A u - lambda M u||_2 / (lambda ||M u||_2) <= tol for the first nev
  columns (the paper's §6 criterion divides by |lambda| only).
* With a random start the first iteration skips step (a) and uses W = U0, which gives
  coarse-quality Ritz pairs at once.
"""
import numpy as np
import scipy.linalg as sl

from .mg import Hierarchy, cg, pcg


def relative_residuals(A, M, U, lam):
    """||A u_i - lam_i M u_i||_2 / (|lam_i| ||M u_i||_2) for every column: the stopping test
    of the numerical section (§6 divides by |lambda| only; the factor ||M u||_2 is added here
    so that the test does not depend on how u is scaled)."""
    AU = A @ U
    MU = M @ U
    R = AU - MU * lam
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MU, axis=0))


def rayleigh_quotients(A, M, U):
    return np.einsum("ij,ij->j", U, A @ U) / np.einsum("ij,ij->j", U, M @ U)


def linear_solve(A, M, U, lam, s, hier=None, solver="vcycle"):
    """Step (a): W with A W = M U Lambda approximately, initial guess U.

    V-cycle form: correction E from s V-cycles on A E = M U Lambda - A U, E0 = 0, then
    W = U + E (the same iterate as s V-cycles from the initial guess U).
    CG form: s CG steps per column from the initial guess U.
    MGCG form: s CG steps per column preconditioned by one V-cycle, from U.
    """
    F = (M @ U) * lam
    if solver == "vcycle":
        R = F - A @ U
        E = hier.solve(R, s)
        return U + E
    if solver == "mgcg":
        return pcg(A, F, U, s, lambda R: hier.solve(R, 1))
    if solver != "cg":
        raise ValueError(solver)
    return cg(A, F, U, s)


def projection(A, M, P, W):
    """Step (b): aH = P^T A W, bH = P^T M W, GA = W^T A W, GM = W^T M W."""
    AW = A @ W
    MW = M @ W
    return P.T @ AW, P.T @ MW, W.T @ AW, W.T @ MW


def augmented_pencil(A_H, M_H, aH, bH, GA, GM):
    """The composite matrices A_Hh, B_Hh of Alg. 3 step 4, dense."""
    Ahat = np.block([[A_H.toarray(), aH], [aH.T, GA]])
    Bhat = np.block([[M_H.toarray(), bH], [bH.T, GM]])
    return 0.5 * (Ahat + Ahat.T), 0.5 * (Bhat + Bhat.T)


def augmented_eig(A_H, M_H, aH, bH, GA, GM, m):
    """Step (c): the m smallest pairs of the augmented pencil (dense LAPACK).

    Returns (lam[m], C_H[N_H][m], C_W[m][m]) with [C_H; C_W] B_Hh-orthonormal.
    """
    Ahat, Bhat = augmented_pencil(A_H, M_H, aH, bH, GA, GM)
    lam, Y = sl.eigh(Ahat, Bhat, subset_by_index=[0, m - 1])
    NH = A_H.shape[0]
    return lam, Y[:NH], Y[NH:]


def precond_a(A_H, M_H, aH, bH, GA, GM):
    """PRECOND-A (§4, Alg. 5 step 1): the congruence with [[I, A_H^-1 aH],[0, I]].

    Returns (ahat, alpha_t, b_t, beta_t) where ahat = A_H^-1 aH,
    alpha_t = GA - ahat^T aH, b_t = bH - M_H ahat,
    beta_t = GM - bH^T ahat - ahat^T bH + ahat^T M_H ahat.
    The transformed pencil is [[A_H, 0],[0, alpha_t]], [[M_H, b_t],[b_t^T, beta_t]].
    """
    ahat = sl.cho_solve(sl.cho_factor(A_H.toarray()), aH)
    alpha_t = GA - ahat.T @ aH
    b_t = bH - M_H @ ahat
    beta_t = GM - bH.T @ ahat - ahat.T @ bH + ahat.T @ (M_H @ ahat)
    return ahat, alpha_t, b_t, beta_t


def precond_a_back(ahat, uH_t, gamma_t):
    """Alg. 5 step 3: u_H = u~_H - ahat gamma~, gamma = gamma~."""
    return uH_t - ahat @ gamma_t, gamma_t


def precond_b(A_H, M_H, aH, bH, GA, GM):
    """PRECOND-B (§4): the same kind of congruence built from B_Hh's factorisation,
    [[I, B_H^-1 b_h],[0, I]], which makes B_Hh block diagonal.

    Returns (bhat, a_t, alpha_t, beta_t) with bhat = M_H^-1 bH, a_t = aH - A_H bhat,
    alpha_t = GA - bhat^T aH - aH^T bhat + bhat^T A_H bhat, beta_t = GM - bH^T bhat.
    The transformed pencil is [[A_H, a_t],[a_t^T, alpha_t]], [[M_H, 0],[0, beta_t]];
    its eigenvectors map back as in precond_a_back (with bhat in place of ahat)."""
    bhat = sl.cho_solve(sl.cho_factor(M_H.toarray()), bH)
    a_t = aH - A_H @ bhat
    alpha_t = GA - bhat.T @ aH - aH.T @ bhat + bhat.T @ (A_H @ bhat)
    beta_t = GM - bH.T @ bhat
    return bhat, a_t, alpha_t, beta_t


def precond_ba(A_H, M_H, aH, bH, GA, GM):
    """PRECOND-B-A (§4): PRECOND-B, and for the linear solves inside the augmented
    eigensolver the block factorisation of the transformed A_Hh, as PRECOND-A factors A_Hh:
        [[A_H, a_t],[a_t^T, alpha_t]] = L diag(A_H, S) L^T,  L = [[I, 0],[ahat2^T, I]],
    ahat2 = A_H^-1 a_t, S = alpha_t - a_t^T ahat2.
    Returns (bhat, a_t, alpha_t, beta_t, ahat2, S)."""
    bhat, a_t, alpha_t, beta_t = precond_b(A_H, M_H, aH, bH, GA, GM)
    ahat2 = sl.cho_solve(sl.cho_factor(A_H.toarray()), a_t)
    return bhat, a_t, alpha_t, beta_t, ahat2, alpha_t - a_t.T @ ahat2


def prolongate(P, W, C_H, C_W):
    """Step (d): U = P C_H + W C_W."""
    return P @ C_H + W @ C_W


def coarse_start(A_H, M_H, P, m):
    """Alg. 3 steps 1-2: coarse eigenpairs, interpolated to the fine space."""
    lam, UH = sl.eigh(A_H.toarray(), M_H.toarray(), subset_by_index=[0, m - 1])
    return lam, P @ UH


class Solver:
    """The whole method (Alg. 2 / Alg. 3) on one pencil, dense step (c)."""

    def __init__(self, A, M, chain, coarse_level=None, omega=2.0 / 3.0, nu1=2, nu2=2):
        self.A, self.M = A.tocsr(), M.tocsr()
        self.chain = chain
        self.coarse_level = len(chain) if coarse_level is None else coarse_level
        P = None
        for k in range(self.coarse_level):
            P = chain[k] if P is None else P @ chain[k]
        self.P = P.tocsr()
        self.hier = Hierarchy(self.A, chain, omega, nu1, nu2)
        self.A_H = (self.P.T @ self.A @ self.P).tocsr()
        self.M_H = (self.P.T @ self.M @ self.P).tocsr()

    def iteration(self, U, lam, s, solve=True, solver="vcycle"):
        """One augmented subspace iteration; returns (lam, U, intermediates)."""
        m = U.shape[1]
        W = linear_solve(self.A, self.M, U, lam, s, self.hier, solver) if solve else U
        aH, bH, GA, GM = projection(self.A, self.M, self.P, W)
        lam_new, C_H, C_W = augmented_eig(self.A_H, self.M_H, aH, bH, GA, GM, m)
        U_new = prolongate(self.P, W, C_H, C_W)
        return lam_new, U_new, dict(W=W, aH=aH, bH=bH, GA=GA, GM=GM, C_H=C_H, C_W=C_W)

    def solve(self, nev, m, tol, U0=None, s=2, max_iter=100, solver="vcycle", post_solve=False):
        """Iterate from U0 (random start, first step (a) skipped) or from the coarse
        start until the first nev relative residuals are <= tol.

        post_solve: the two-solve form of Alg. 3 - an iteration that has not converged is
        followed by the step-7 solve A_h u = lambda M_h u-hat from the Rayleigh-Ritz block
        u-hat, whose result is the next iteration's step-3 initial guess."""
        if U0 is None:
            lam, U = coarse_start(self.A_H, self.M_H, self.P, m)
            first_solve = True
        else:
            U, lam = U0, None
            first_solve = False
        history = []
        it = 0
        for it in range(1, max_iter + 1):
            if post_solve and it > 1:
                U = linear_solve(self.A, self.M, U, lam, s, self.hier, solver)
            lam, U, _ = self.iteration(U, lam, s, solve=first_solve or it > 1, solver=solver)
            res = relative_residuals(self.A, self.M, U, lam)
            history.append(res.copy())
            if np.all(res[:nev] <= tol):
                break
        return lam, U, dict(iterations=it, history=history, converged=bool(np.all(history[-1][:nev] <= tol)))


# ------------------------------------------------------------ batch scheme (§5, Alg. 6 and Alg. 7)


def component_norms(uH, gamma, bH, GM):
    """Selection rule of the batch scheme: for candidates v_i = I_H^h u_{i,H} + W gamma_i,
    ||Pi_h v_i||_b^2 with Pi_h the b-orthogonal projection onto span(W).  With
    Pi_h v_i = W x_i, the projection equations give X GM = uH^T bH + gamma^T GM (X has rows
    x_i^T), and ||Pi_h v_i||_b^2 = X(i,:) GM X(i,:)^T."""
    R = uH.T @ bH + gamma.T @ GM
    X = np.linalg.solve(GM.T, R.T).T
    return np.einsum("ij,jk,ik->i", X, GM, X)


def nearest_pairs(A_H, M_H, aH, bH, GA, GM, theta, n):
    """The n eigenpairs of the augmented pencil closest to the shift theta (Alg. 7 step (d)),
    by a dense solve of the whole pencil, returned in ascending order of eigenvalue:
    (lam[n], C_H[N_H][n], C_W[m][n]), B_Hh-orthonormal."""
    Ahat, Bhat = augmented_pencil(A_H, M_H, aH, bH, GA, GM)
    lam, Y = sl.eigh(Ahat, Bhat)
    idx = np.sort(np.argsort(np.abs(lam - theta), kind="stable")[:n])
    NH = A_H.shape[0]
    return lam[idx], Y[:NH, idx], Y[NH:, idx]


def batch_bounds(lam_H, nev, k, gap=1e-3):
    """Batch boundaries (Alg. 7 step 2): batches of k pairs, a boundary moved up past any
    coarse eigenvalue within a relative gap of its predecessor, so that no cluster of the
    coarse spectrum is split between two batches (the paper does not say how it batches)."""
    bounds, m0 = [], 0
    while m0 < nev:
        e = min(nev, m0 + k)
        while e < nev and lam_H[e] - lam_H[e - 1] <= gap * lam_H[e]:
            e += 1
        bounds.append((m0, e))
        m0 = e
    return bounds


def batch_scheme(solver, nev, k, tol, guard=4, n_window=None, s=2, max_iter=100, linear="vcycle"):
    """Alg. 7: the first nev eigenpairs in batches of k, one batch after the other.

    Coarse eigenpairs (lam_H, U_H) first (step 1); batches from batch_bounds (step 2).
    Batch i owns pairs m_i .. m_i + k_i - 1 and iterates them with `guard` further columns (the next coarse pairs; read here as the
    guard columns of the one-batch method, without which the last owned pair converges at
    the rate of its gap to the first pair above the batch):
    (a) U = I_H^h U_H[:, block], Lambda = lam_H[block], block = the k_i + guard columns;
    (b) theta = (lam_H[m_i] + lam_H[m_i + k_i - 1]) / 2 (the midpoint; the printed minus sign
        is read as a plus);
    then until the owned pairs' relative residuals are <= tol:
    (c) s linear-solve steps on A_h w = lambda M_h u from u;
    (d) the n_window (default twice the block) eigenpairs of the augmented pencil closest to
        theta;
    (e) the block's worth of them with the largest component ||Pi_h v||_b^2 in span(W), in
        ascending order, prolongated;
    (f) if not converged, s linear-solve steps on A_h u = lambda M_h u-hat from u-hat.
    Returns (lam[nev], U[N][nev], info), the owned pairs of each batch in ascending order."""
    A, M, P = solver.A, solver.M, solver.P
    NH = solver.A_H.shape[0]
    top = min(NH, nev + k + guard)
    lam_H, U_H = sl.eigh(solver.A_H.toarray(), solver.M_H.toarray(), subset_by_index=[0, top - 1])
    out_lam, out_U, iters = [], [], []
    for m0, e in batch_bounds(lam_H, nev, k):
        kb = e - m0
        mb = min(kb + guard, top - m0)
        nw = min(n_window or 2 * mb, NH + mb)
        U = P @ U_H[:, m0:m0 + mb]
        lam = lam_H[m0:m0 + mb].copy()
        theta = 0.5 * (lam_H[m0] + lam_H[m0 + kb - 1])
        it = 0
        for it in range(1, max_iter + 1):
            W = linear_solve(A, M, U, lam, s, solver.hier, linear)
            aH, bH, GA, GM = projection(A, M, P, W)
            lw, CH, CW = nearest_pairs(solver.A_H, solver.M_H, aH, bH, GA, GM, theta, nw)
            comp = component_norms(CH, CW, bH, GM)
            sel = np.sort(np.argsort(-comp, kind="stable")[:mb])
            lam = lw[sel]
            U = prolongate(P, W, CH[:, sel], CW[:, sel])
            if np.all(relative_residuals(A, M, U[:, :kb], lam[:kb]) <= tol):
                break
            U = linear_solve(A, M, U, lam, s, solver.hier, linear)
        out_lam.append(lam[:kb])
        out_U.append(U[:, :kb])
        iters.append(it)
    return np.concatenate(out_lam), np.hstack(out_U), dict(iterations=iters)

