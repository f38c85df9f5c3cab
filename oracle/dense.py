"""Brute-force reference: the plain definition of the discrete eigenproblem.

§2.1 defines the wanted pairs as the smallest eigenvalues of A_h u = lambda B_h u
(B_h = M_h here) with B_h-normalised eigenvectors; §3 Alg. 3 states the same in
matrix form (A_h u_h = B_h u_h Lambda).  For small meshes we solve it densely.
"""
import numpy as np
import scipy.linalg as sl
import scipy.sparse.linalg as spl


def smallest_pairs(A, M, k: int):
    """k smallest eigenpairs of the symmetric-definite pencil (A, M), dense LAPACK.

    Returns (lam[k] ascending, U[N][k]) with U^T M U = I.
    """
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    Md = M.toarray() if hasattr(M, "toarray") else np.asarray(M)
    lam, U = sl.eigh(Ad, Md, subset_by_index=[0, k - 1])
    return lam, U


def smallest_pairs_shift_invert(A, M, k: int, sigma: float = 0.0):
    """k smallest eigenpairs by shift-invert Lanczos (ARPACK) with a sparse LU; an
    algorithm independent of the augmented subspace method, for mid-size meshes."""
    lam, U = spl.eigsh(A.tocsc(), k=k, M=M.tocsc(), sigma=sigma, which="LM", tol=1e-14)
    order = np.argsort(lam)
    lam, U = lam[order], U[:, order]
    # M-normalise
    nrm = np.sqrt(np.einsum("ij,ij->j", U, M @ U))
    return lam, U / nrm
