"""Seeded synthetic inputs for the augmented subspace eigensolver.

This module builds the problem data that both sides consume: the bilinear (2D) /
trilinear (3D) Q1 finite element stiffness and mass matrices of the model problem
-div(kappa grad u) = lambda u on the unit square/cube with homogeneous Dirichlet
conditions (paper §2.1, the model problem and its weak form), the nodal
interpolation operators between nested uniform meshes (the nested-space assumption
V_H subset V_h of §2.2 and the interpolation chain of §3), the Galerkin coarse
matrices built from them, and the seeded random numbers (start vectors, log-normal
coefficient fields).

It contains none of the augmented subspace method's own arithmetic: no linear
solve, no projection, no eigensolve.  The test oracle and the CUDA path both read
their inputs from here, so the two receive identical matrices and start vectors.

Conventions
-----------
* Mesh: uniform n^d elements on (0,1)^d, h = 1/n.  Unknowns are the interior nodes
  (Dirichlet nodes are eliminated), N = (n-1)^d, ordered lexicographically with x
  fastest: idx = (ix-1) + (n-1)(iy-1) + (n-1)^2 (iz-1), 1 <= i* <= n-1.
* Elements are indexed by their lower corner e = ex + n ey + n^2 ez, 0 <= e* < n.
* Sparse matrices are scipy CSR with int64 indptr, int32 indices, float64 data,
  columns sorted within each row.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15

# --------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
# OOPSLA 2014): state advances by the golden gamma; each output is the state passed
# through the variant-13 finaliser.
# --------------------------------------------------------------------------------------


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed` (uint64 array)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0,1): the top 53 bits of each SplitMix64 output times 2^-53."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def start_vectors(seed: int, n_rows: int, n_cols: int) -> np.ndarray:
    """Start block U0 [n_rows][n_cols], entries uniform in [-1,1).

    Entry (i, j) is output i*n_cols + j of SplitMix64(seed), so the block is laid out
    row-major (node-major, the columns of one node contiguous).
    """
    u = uniform01(seed, n_rows * n_cols)
    return (2.0 * u - 1.0).reshape(n_rows, n_cols)


def start_vector_rows(seed: int, n_cols: int, row0: int, row1: int) -> np.ndarray:
    """Rows row0..row1-1 of the start block of start_vectors(seed, ., n_cols), generated
    alone (entry (i, j) is still output i*n_cols + j), for blocks too large to build at once."""
    u = uniform01(seed, (row1 - row0) * n_cols, start=row0 * n_cols)
    return (2.0 * u - 1.0).reshape(row1 - row0, n_cols)


def standard_normals(seed: int, count: int) -> np.ndarray:
    """Box-Muller normals from SplitMix64(seed).

    Pair p uses outputs 2p and 2p+1: u1 = (top53(z_2p) + 1) 2^-53 in (0,1],
    u2 = top53(z_2p+1) 2^-53; normal 2p = sqrt(-2 ln u1) cos(2 pi u2), normal 2p+1 the
    same with sin.  Normal k is the k-th of that sequence.
    """
    npairs = (count + 1) // 2
    z = splitmix64(seed, 2 * npairs)
    top = (z >> np.uint64(11)).astype(np.float64)
    u1 = (top[0::2] + 1.0) * (1.0 / 9007199254740992.0)
    u2 = top[1::2] * (1.0 / 9007199254740992.0)
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npairs)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:count]


def smoother_init(d: int, omega: float = 2.0 / 3.0, seed: int = 0, noise: float = 0.02) -> np.ndarray:
    """Initial parameters of the learned smoother network (2 -> 16 -> 16 -> 16 -> 1
    channels, 3^d taps, layout [W1, b1, ..., W4, b4], W in [c_out][c_in][tap] order):
    weights that reproduce damped Jacobi plus seeded normal noise of standard deviation
    `noise` on every parameter (normal k of standard_normals(seed, .) on parameter k).

    Jacobi part: channel 0 of layer 1 passes +s and channel 1 passes -s through the
    centre tap, layers 2 and 3 copy those two channels, layer 4 outputs
    omega * (ch0 - ch1), so with ReLU the output is omega * s."""
    T = 3 ** d
    c = (T - 1) // 2
    shapes = [(2, 16), (16, 16), (16, 16), (16, 1)]
    parts = []
    for li, (ci, co) in enumerate(shapes):
        W = np.zeros((co, ci, T))
        b = np.zeros(co)
        if li == 0:
            W[0, 0, c], W[1, 0, c] = 1.0, -1.0
        elif li < 3:
            W[0, 0, c], W[1, 1, c] = 1.0, 1.0
        else:
            W[0, 0, c], W[0, 1, c] = omega, -omega
        parts += [W.reshape(-1), b]
    p = np.concatenate(parts)
    if noise:
        p = p + noise * standard_normals(seed, p.size)
    return p.astype(np.float32)


def lognormal_kappa(d: int, n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Per-element coefficient kappa_e = exp(sigma * g_e), g_e ~ N(0,1) i.i.d.

    Element e (lexicographic, x fastest) takes normal number e of the seed's stream.
    """
    return np.exp(sigma * standard_normals(seed, n ** d))


# --------------------------------------------------------------------------------------
# Q1 element matrices (tensor products of the 1D P1 element matrices on [0, h])
# --------------------------------------------------------------------------------------


def _element_1d(h: float):
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    return k1, m1


def q1_matrices(d: int, n: int, kappa: np.ndarray | None = None):
    """Stiffness A and mass M of Q1 elements on the uniform n^d mesh, interior nodes.

    The stiffness of element e is kappa_e * sum_k (x)_j (K1 if j == k else M1), the
    mass is (x)_j M1 (no coefficient).  Each row is built directly from the (up to
    3^d) neighbour offsets: the entry for nodes i and i+o sums, over the elements
    that contain both nodes, the product of 1D element entries at the local indices.
    """
    assert d in (2, 3) and n >= 2
    h = 1.0 / n
    k1, m1 = _element_1d(h)
    n1 = n - 1
    N = n1 ** d
    if kappa is None:
        kappa = np.ones(n ** d)
    kappa = np.asarray(kappa, dtype=np.float64)
    assert kappa.shape == (n ** d,)
    idx = np.arange(N, dtype=np.int64)
    coords = [(idx // (n1 ** k)) % n1 + 1 for k in range(d)]  # x fastest
    offsets = np.array(np.meshgrid(*([[-1, 0, 1]] * d), indexing="ij")).reshape(d, -1).T
    # order offsets by increasing column index: sort key (o_{d-1}, ..., o_0)
    offsets = offsets[np.lexsort(offsets.T)]
    nb = offsets.shape[0]
    cols = np.empty((N, nb), dtype=np.int64)
    valid = np.ones((N, nb), dtype=bool)
    aval = np.zeros((N, nb))
    mval = np.zeros((N, nb))
    for t, o in enumerate(offsets):
        col = np.zeros(N, dtype=np.int64)
        ok = np.ones(N, dtype=bool)
        for k in range(d):
            j = coords[k] + o[k]
            ok &= (j >= 1) & (j <= n1)
            col += (j - 1) * (n1 ** k)
        cols[:, t] = np.where(ok, col, 0)
        valid[:, t] = ok
        # element lower-corner choices per dimension
        choices = []
        for k in range(d):
            if o[k] == 0:
                choices.append((-1, 0))
            elif o[k] == 1:
                choices.append((0,))
            else:
                choices.append((-1,))
        for combo in np.array(np.meshgrid(*choices, indexing="ij")).reshape(d, -1).T:
            e = np.zeros(N, dtype=np.int64)
            mass = np.ones(N)
            stiff = np.zeros(N)
            li = []
            lj = []
            for k in range(d):
                ek = coords[k] + combo[k]  # element coordinate in 0..n-1
                e += ek * (n ** k)
                li.append(int(-combo[k]))          # local index of node i in this element
                lj.append(int(o[k] - combo[k]))    # local index of node i+o
            for k in range(d):
                mass = mass * m1[li[k], lj[k]]
            for kk in range(d):
                term = 1.0
                for k in range(d):
                    term *= (k1 if k == kk else m1)[li[k], lj[k]]
                stiff = stiff + term
            aval[:, t] += kappa[e] * stiff
            mval[:, t] += mass
    counts = valid.sum(axis=1)
    indptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    indices = cols[valid].astype(np.int32)
    A = sp.csr_matrix((aval[valid], indices, indptr), shape=(N, N))
    M = sp.csr_matrix((mval[valid], indices.copy(), indptr.copy()), shape=(N, N))
    return A, M


def _gauss_legendre_01(q: int):
    """q-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def q1_matrices_coefficients(d: int, n: int, tensor, potential, quad: int = 3):
    """Stiffness of a(u, v) = int (T(x) grad u) . grad v + phi(x) u v and mass int u v with Q1
    elements on the uniform n^d mesh, interior nodes (the same ordering as q1_matrices).

    tensor(X) -> [..., d, d] and potential(X) -> [...] take points X [..., d]; both are
    integrated with the quad^d-point Gauss-Legendre rule on every element (exact for the
    mass and for polynomial coefficients of degree <= 2 quad - 3).  The element matrix is
    sum_q w_q h^d (sum_kl T_kl(x_q) dphi_a/dx_k dphi_b/dx_l + phi(x_q) phi_a phi_b) with
    phi_a the tensor-product P1 hats; entries are gathered per grid tap as in q1_matrices.
    """
    assert d in (2, 3) and n >= 2
    h = 1.0 / n
    n1 = n - 1
    N = n1 ** d
    xg, wg = _gauss_legendre_01(quad)
    # reference quadrature points (x fastest) and per-point basis values / gradients
    qpts = np.array(np.meshgrid(*([xg] * d), indexing="ij")).reshape(d, -1).T[:, ::-1]  # [Q][d], col 0 = x
    qw = np.prod(np.array(np.meshgrid(*([wg] * d), indexing="ij")).reshape(d, -1).T, axis=1)
    corners = np.array([[(a >> k) & 1 for k in range(d)] for a in range(2 ** d)])  # [2^d][d]
    Q, nb = len(qw), 2 ** d
    val = np.ones((Q, nb))
    grad = np.ones((Q, nb, d))
    for k in range(d):
        lk = np.where(corners[None, :, k] == 1, qpts[:, k:k + 1], 1.0 - qpts[:, k:k + 1])  # [Q][nb]
        dk = np.where(corners[None, :, k] == 1, 1.0, -1.0) / h
        val *= lk
        for j in range(d):
            grad[:, :, j] *= dk if j == k else lk
    # reference blocks: [Q][d*d + 1][nb][nb]
    G = np.zeros((Q, d * d + 1, nb, nb))
    for k in range(d):
        for l in range(d):
            G[:, k * d + l] = np.einsum("qa,qb->qab", grad[:, :, k], grad[:, :, l])
    G[:, d * d] = np.einsum("qa,qb->qab", val, val)
    G *= (qw * h ** d)[:, None, None, None]
    ne = n ** d
    taps = 3 ** d
    dia = np.zeros((taps, N))
    chunk = 1 << 16
    for e0 in range(0, ne, chunk):
        e = np.arange(e0, min(ne, e0 + chunk), dtype=np.int64)
        ec = np.stack([(e // n ** k) % n for k in range(d)], axis=1)  # [E][d] lower corners
        X = (ec[:, None, :] + qpts[None, :, :]) * h                      # [E][Q][d]
        T = tensor(X)
        C = np.concatenate([T.reshape(T.shape[:2] + (d * d,)), potential(X)[:, :, None]], axis=2)
        K = (C.reshape(len(e), -1) @ G.reshape(-1, nb * nb)).reshape(len(e), nb, nb)
        node = ec[:, None, :] + corners[None, :, :]                      # [E][nb][d] in 0..n
        inner = np.all((node >= 1) & (node <= n1), axis=2)
        gidx = np.zeros(node.shape[:2], dtype=np.int64)
        for k in range(d):
            gidx += (node[:, :, k] - 1) * n1 ** k
        for a in range(nb):
            for b in range(nb):
                ok = inner[:, a] & inner[:, b]
                o = corners[b] - corners[a]
                t = int(sum((o[k] + 1) * 3 ** k for k in range(d)))
                dia[t, gidx[ok, a]] += K[ok, a, b]
    idx = np.arange(N, dtype=np.int64)
    coords = [(idx // (n1 ** k)) % n1 + 1 for k in range(d)]
    valid = np.zeros((N, taps), dtype=bool)
    cols = np.zeros((N, taps), dtype=np.int64)
    for t in range(taps):
        o = [(t // 3 ** k) % 3 - 1 for k in range(d)]
        ok = np.ones(N, dtype=bool)
        col = np.zeros(N, dtype=np.int64)
        for k in range(d):
            j = coords[k] + o[k]
            ok &= (j >= 1) & (j <= n1)
            col += (j - 1) * n1 ** k
        valid[:, t] = ok
        cols[:, t] = col
    indptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(valid.sum(axis=1), out=indptr[1:])
    A = sp.csr_matrix((dia.T[valid], cols[valid].astype(np.int32), indptr), shape=(N, N))
    _, M = q1_matrices(d, n)
    return A, M


def tensor_potential_coefficients(d: int):
    """The coefficients of the batch-scheme test problem of the numerical section:
    T(x) = I + (x - 1/2)(x - 1/2)^T and phi(x) = exp(prod_k (x_k - 1/2)) on (0, 1)^d."""
    def tensor(X):
        y = X - 0.5
        return np.eye(d) + y[..., :, None] * y[..., None, :]

    def potential(X):
        return np.exp(np.prod(X - 0.5, axis=-1))

    return tensor, potential


def q1_interp_1d(n_fine: int, n_coarse: int) -> sp.csr_matrix:
    """1D nodal interpolation of coarse P1 hats at fine interior nodes.

    Row i-1 (fine node x = i/n_fine), column I-1 (coarse node X = I/n_coarse):
    max(0, 1 - |x - X| / H).
    """
    assert n_fine % n_coarse == 0
    r = n_fine // n_coarse
    i = np.arange(1, n_fine)[:, None]
    I = np.arange(1, n_coarse)[None, :]
    w = np.maximum(0.0, 1.0 - np.abs(i - r * I) / r)
    return sp.csr_matrix(w)


def q1_interpolation(d: int, n_fine: int, n_coarse: int) -> sp.csr_matrix:
    """Q1 nodal interpolation V_H -> V_h on interior nodes (tensor product, x fastest)."""
    p1 = q1_interp_1d(n_fine, n_coarse)
    P = p1
    for _ in range(d - 1):
        P = sp.kron(p1, P, format="csr")
    return canonical_csr(P)


def canonical_csr(X) -> sp.csr_matrix:
    """CSR with sorted columns, explicit zeros removed, int64 indptr / int32 indices."""
    X = sp.csr_matrix(X, dtype=np.float64)
    X.eliminate_zeros()
    X.sort_indices()
    return sp.csr_matrix((X.data.astype(np.float64), X.indices.astype(np.int32),
                          X.indptr.astype(np.int64)), shape=X.shape)


def galerkin(P: sp.csr_matrix, A: sp.csr_matrix) -> sp.csr_matrix:
    """P^T A P in CSR (the coarse operator of nested spaces)."""
    return canonical_csr((P.T @ (A @ P)).tocsr())


class Problem:
    """A fine pencil (A_h, M_h), the interpolation chain to the coarse space and the
    coarse pencil (A_H, M_H) = Galerkin products through the chain.

    chain[k] maps level k+1 to level k (level 0 is the fine mesh); the coarse space of
    the method is level `coarse_level`; levels below it (if any) only serve multigrid.
    """

    def __init__(self, d, n, n_coarse, kappa=None, mg_min=None):
        self.kappa = kappa
        self._init_from(d, n, n_coarse, q1_matrices(d, n, kappa), mg_min)

    def _init_from(self, d, n, n_coarse, AM, mg_min):
        self.d, self.n, self.n_coarse = d, n, n_coarse
        if not hasattr(self, "kappa"):
            self.kappa = None
        self.A, self.M = AM
        sizes = [n]
        while sizes[-1] > n_coarse:
            sizes.append(sizes[-1] // 2)
        assert sizes[-1] == n_coarse, "coarse mesh must be fine / 2^k"
        self.coarse_level = len(sizes) - 1
        if mg_min is not None:
            while sizes[-1] // 2 >= mg_min:
                sizes.append(sizes[-1] // 2)
        self.mesh_sizes = sizes
        self.chain = [q1_interpolation(d, sizes[k], sizes[k + 1]) for k in range(len(sizes) - 1)]

    # The coarse pencil and the direct interpolation are built on first use, so that large
    # fine meshes can be handed to a library that forms them itself.
    @functools.cached_property
    def _coarse(self):
        A, M = self.A, self.M
        for k in range(self.coarse_level):
            A, M = galerkin(self.chain[k], A), galerkin(self.chain[k], M)
        return A, M

    @property
    def A_H(self):
        return self._coarse[0]

    @property
    def M_H(self):
        return self._coarse[1]

    @functools.cached_property
    def P(self):
        """Direct V_H -> V_h interpolation (product of the chain down to the coarse level)."""
        P = self.chain[0] if self.chain else sp.identity(self.A.shape[0], format="csr")
        for k in range(1, self.coarse_level):
            P = P @ self.chain[k]
        return canonical_csr(P)

    @property
    def N(self):
        return self.A.shape[0]

    @property
    def N_H(self):
        return self.A_H.shape[0]


def guard_columns(nev: int) -> int:
    """Block width nev_w: nev plus max(4, ceil(nev/10)) guard columns, rounded up to 8."""
    w = nev + max(4, -(-nev // 10))
    return -(-w // 8) * 8


# Named workloads: sizes of the five configurations.
WORKLOADS = {
    "laplace2d_128": dict(d=2, n=128, n_coarse=16, nev=10, seed=0, kappa_seed=None),
    "laplace3d_128": dict(d=3, n=128, n_coarse=16, nev=50, seed=0, kappa_seed=None),
    "kappa3d_256": dict(d=3, n=256, n_coarse=32, nev=100, seed=0, kappa_seed=1),
    "tensor3d_128": dict(d=3, n=128, n_coarse=16, nev=50, seed=0, kappa_seed=None, operator="tensor"),
}


def batch_workload(seed: int, count: int, sizes=(64, 128, 256, 512), nev_range=(8, 32),
                   sigma_range=(0.5, 2.0)):
    """Independent 2D problems of uneven size for the batched launch: for problem i, draws
    4i..4i+3 of uniform01(seed) pick the fine mesh from `sizes`, the lognormal spread sigma
    from `sigma_range`, nev uniformly from the integer range and the kappa field's seed.
    Returns dicts (d, n, n_coarse = n/8, sigma, nev, kappa_seed)."""
    u = uniform01(seed, 4 * count)
    out = []
    for i in range(count):
        n = sizes[min(len(sizes) - 1, int(u[4 * i] * len(sizes)))]
        sigma = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[4 * i + 1]
        lo, hi = nev_range
        nev = lo + min(hi - lo, int(u[4 * i + 2] * (hi - lo + 1)))
        kseed = int(u[4 * i + 3] * 2**31)
        out.append(dict(d=2, n=n, n_coarse=n // 8, sigma=float(sigma), nev=nev, kappa_seed=kseed))
    return out


def build_problem(d, n, n_coarse, kappa_seed=None, sigma=1.0, mg_min=None, operator="kappa"):
    """operator "kappa": -div(kappa grad u) = lambda u with kappa per element (1 without a
    seed); "tensor": -div(T grad u) + phi u = lambda u with the coefficients of
    tensor_potential_coefficients."""
    if operator == "tensor":
        pb = Problem.__new__(Problem)
        pb._init_from(d, n, n_coarse, q1_matrices_coefficients(d, n, *tensor_potential_coefficients(d)), mg_min)
        return pb
    kappa = None if kappa_seed is None else lognormal_kappa(d, n, kappa_seed, sigma)
    return Problem(d, n, n_coarse, kappa, mg_min=mg_min)
