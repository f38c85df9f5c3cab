"""Linear solves of the correction step (Alg. 1 first step; Alg. 3 step 3).

The paper solves A_h w_i = lambda_i B_h u_i for every column with a few multigrid or
block-CG steps (§6 uses block CG with at most 40 steps; the linear solver is left to
the implementation).  Two plain references are given here:

* `Hierarchy.vcycle`: a geometric V-cycle on Galerkin levels A_{l+1} = P_l^T A_l P_l
  (exact for nested spaces, §2.2), damped Jacobi smoothing x <- x + omega D^-1 (b - A x)
  with nu1 pre- and nu2 post-sweeps, residual restriction by P^T, prolongation by P,
  and a dense Cholesky solve on the coarsest level.
* `cg`: conjugate gradients run independently on every column (the reading of
  "block CG" used here: one CG per right-hand side, column-wise inner products).
* `pcg`: the same with a symmetric positive definite preconditioner applied to the
  residual (here one V-cycle from zero, which is symmetric because pre- and
  post-smoothing use the same number of damped Jacobi sweeps): textbook preconditioned
  CG, z = B r, alpha = (r, z) / (p, A p), beta = (r_new, z_new) / (r, z).
"""
import numpy as np
import scipy.linalg as sl


class Hierarchy:
    """fine_smoother (optional): a callable r -> correction that replaces each damped
    Jacobi sweep on level 0 (x <- x + S(b - A x)); coarser levels keep Jacobi."""

    def __init__(self, A0, chain, omega=2.0 / 3.0, nu1=2, nu2=2, fine_smoother=None):
        self.A = [A0.tocsr()]
        for P in chain:
            self.A.append((P.T @ (self.A[-1] @ P)).tocsr())
        self.P = [P.tocsr() for P in chain]
        self.PT = [P.T.tocsr() for P in chain]
        self.Dinv = [1.0 / A.diagonal() for A in self.A]
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        self.fine_smoother = fine_smoother
        self.coarse_chol = sl.cho_factor(self.A[-1].toarray(), lower=True)

    @property
    def levels(self):
        return len(self.A)

    def smooth(self, l, b, x, sweeps):
        for _ in range(sweeps):
            if l == 0 and self.fine_smoother is not None:
                x = x + self.fine_smoother(b - self.A[l] @ x)
            else:
                x = x + self.omega * self.Dinv[l][:, None] * (b - self.A[l] @ x)
        return x

    def vcycle(self, l, b, x=None):
        """One V-cycle on level l for A_l x = b (b may hold several columns)."""
        if l == self.levels - 1:
            return sl.cho_solve(self.coarse_chol, b)
        if x is None:
            x = np.zeros_like(b)
        x = self.smooth(l, b, x, self.nu1)
        r = b - self.A[l] @ x
        e = self.vcycle(l + 1, self.PT[l] @ r)
        x = x + self.P[l] @ e
        return self.smooth(l, b, x, self.nu2)

    def solve(self, b, cycles, x=None):
        for _ in range(cycles):
            x = self.vcycle(0, b, x)
        return x


def cg(A, F, X0, steps):
    """`steps` CG iterations on A x_j = f_j for every column j, from X0."""
    X = X0.copy()
    R = F - A @ X
    Pd = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    for _ in range(steps):
        AP = A @ Pd
        pAp = np.einsum("ij,ij->j", Pd, AP)
        alpha = np.where(pAp > 0, rr / np.where(pAp > 0, pAp, 1.0), 0.0)
        X += Pd * alpha
        R -= AP * alpha
        rr_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(rr > 0, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        Pd = R + Pd * beta
        rr = rr_new
    return X


def pcg(A, F, X0, steps, precond):
    """`steps` preconditioned CG iterations on A x_j = f_j for every column j, from X0;
    precond(R) returns the preconditioned residual block Z = B R."""
    X = X0.copy()
    R = F - A @ X
    Z = precond(R)
    Pd = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    for _ in range(steps):
        AP = A @ Pd
        pAp = np.einsum("ij,ij->j", Pd, AP)
        alpha = np.where(pAp > 0, rz / np.where(pAp > 0, pAp, 1.0), 0.0)
        X += Pd * alpha
        R -= AP * alpha
        Z = precond(R)
        rz_new = np.einsum("ij,ij->j", R, Z)
        beta = np.where(rz > 0, rz_new / np.where(rz > 0, rz, 1.0), 0.0)
        Pd = Z + Pd * beta
        rz = rz_new
    return X
