"""Learned fine-level smoother through the C ABI (needs a GPU): the inference pass
(tensor-core hidden layers) and the training pass (loss, gradients, Adam) against the
FP64 oracle, the V-cycle with the network against the oracle's V-cycle, and what
training gains over damped Jacobi.

Tolerances: training runs the network in FP32 (bf16 parameters, FP32 accumulation) and
the oracle in FP64 with the same bf16 parameters, so losses agree to about 1e-6 relative
and gradients (sums of many FP32 products) to 1e-4 relative in norm per layer and 1e-3 of
the layer's largest entry elementwise.  Inference stores hidden activations in bf16 as the
oracle's inference form does; where every sum is exact in FP32 the two agree bit for bit
(dyadic inputs), elsewhere an activation that FP32 and FP64 round to neighbouring bf16
values moves outputs by a few 1e-3 of the column's largest value.
"""
import numpy as np
import pytest

import pase_inputs as pin
from oracle import dense, mg, pase as opase, smoother as sm

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def _colrel(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))


def _problem(d, n, seed, sigma=1.0):
    nc = n // 4 if d == 2 else n // 2
    pb = pin.build_problem(d, n, nc, kappa_seed=seed, sigma=sigma, mg_min=4)
    return pb, np.log(pb.kappa)


def _handle(pb, d, lk, params=None, **kw):
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    for k, v in kw.items():
        setattr(opt, k, v)
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
    P.pase_set_grid(h, d, pb.n, lk)
    if params is not None:
        P.pase_smoother_state(h, d, (params,))
    return h


def _colmax_err(a, b):
    """Per column: max_i |a - b| / max_i |b| (elementwise, every node included)."""
    return np.max(np.abs(a - b), axis=0) / np.maximum(np.max(np.abs(b), axis=0), 1e-300)


def _problem_ragged(d, n, seed, sigma=1.0):
    """Grids whose interior size is not a multiple of the 8 x 16 inference tile (n - 1 = 37
    in 2D, 19 in 3D), one coarsening step."""
    pb = pin.build_problem(d, n, n // 2, kappa_seed=seed, sigma=sigma)
    return pb, np.log(pb.kappa)


@pytest.mark.parametrize("d,n", [(2, 32), (3, 16), (2, 38), (3, 20)])
def test_apply_matches_oracle(d, n):
    """Inference pass vs the oracle's inference form, elementwise at every node (tile edges
    and halo corners included; 37^2 and 19^3 leave ragged tiles).  The two round the same
    activations to bf16 from FP32 and FP64 sums, so an activation near a rounding boundary can
    go to neighbouring bf16 values; emulating the kernel's FP32 sums on the CPU, that moved
    an output by at most 2.7e-3 of its column's largest value, hence 1e-2."""
    pb, lk = _problem(d, n, 4) if n in (32, 16) else _problem_ragged(d, n, 4)
    params = pin.smoother_init(d, seed=3, noise=0.3)
    h = _handle(pb, d, lk, params)
    try:
        m = 16
        R = pin.start_vectors(8, pb.N, m)
        D = np.empty_like(R)
        P.pase_smoother_apply(h, m, R, D)
        dinv = 1.0 / pb.A.diagonal()
        feat = sm.node_features(d, n, lk)
        ref = sm.apply(params, R, dinv, feat, d, n - 1, act_bf16=True)
        assert np.max(_colmax_err(D, ref)) < 1e-2
        # and close to the FP32-activation network (the one training differentiates)
        ref32 = sm.apply(params, R, dinv, feat, d, n - 1, act_bf16=False)
        assert np.max(_colmax_err(D, ref32)) < 3e-2
    finally:
        P.pase_destroy(h)


def _dyadic_case(d, n, seed=7):
    """Inputs on which every sum of the inference pass is exact in FP32 and in FP64, so the
    kernel must reproduce the oracle's inference form bit for bit: weights in {0, +-1/4},
    biases in {0, 1/4}, the Jacobi-scaled residual +-1 in every column (a diagonal of 4 in 2D,
    1/4 in 3D, so rho = 1 exactly), node features integers (log kappa in {0, +-2^d})."""
    n1 = n - 1
    pb = pin.build_problem(d, n, n // 2)
    A = pb.A.tolil()
    A.setdiag(4.0 if d == 2 else 0.25)  # still strictly diagonally dominant, so SPD
    A = pin.canonical_csr(A)
    P_ = sm.n_params(d)
    u = pin.uniform01(seed, n ** d + 2 * P_ + n1 ** d)
    o = n ** d
    logk = (np.array([-1.0, 0.0, 1.0]) * 2 ** d)[np.minimum(2, (u[:o] * 3).astype(int))]
    sign = np.where(u[o:o + P_] < 0.5, -1.0, 1.0)
    dens = u[o + P_:o + 2 * P_]
    o += 2 * P_
    params = np.zeros(P_)
    off, T = 0, 3 ** d
    for li, (ci, co, _) in enumerate(sm.layer_shapes(d)):
        nw = co * ci * T
        params[off:off + nw] = np.where(dens[off:off + nw] < (0.3 if li == 0 else 0.1), 0.25 * sign[off:off + nw], 0.0)
        off += nw
        params[off:off + co] = np.where(dens[off:off + co] < 0.5, 0.25, 0.0)
        off += co
    q = np.where(u[o:o + n1 ** d] < 0.5, -1.0, 1.0)
    Q = np.stack([np.roll(q, 7 * j) * (1.0 if j % 2 == 0 else -1.0) for j in range(16)], axis=1)
    return pb, A, logk, params.astype(np.float32), Q


@pytest.mark.parametrize("d,n", [(2, 38), (3, 20)])
def test_apply_bit_exact_on_dyadic_inputs(d, n):
    pb, A, logk, params, Q = _dyadic_case(d, n)
    dinv = 1.0 / A.diagonal()
    R = Q / dinv[:, None]
    feat = sm.node_features(d, n, logk)
    ref = sm.apply(params, R, dinv, feat, d, n - 1, act_bf16=True)
    # precondition, on the CPU: every partial sum is a multiple of 2^-8 below 2^15 in
    # magnitude (exact in FP32), and the scale rho is exactly 1
    s, rho = sm.normalise(R, dinv)
    assert np.all(rho == 1.0)
    _, (p, cache) = sm.forward(params, s, feat, d, n - 1, True, act_bf16=True)
    for li, (x, z) in enumerate(cache):
        W, b, _ = sm.unpack(p, d)[li]
        assert np.max(sm.conv(np.abs(x), np.abs(W), np.abs(b), d, n - 1)) < 2.0 ** 15
        assert np.all(z * 256.0 == np.round(z * 256.0))
    opt = P.pase_default_options()
    opt.coarse_level = 1
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    try:
        P.pase_setup(h, A, pb.M, pb.chain)
        P.pase_set_grid(h, d, n, logk)
        P.pase_smoother_state(h, d, (params,))
        D = np.empty_like(R)
        P.pase_smoother_apply(h, 16, R, D)
    finally:
        P.pase_destroy(h)
    bad = np.argwhere(D != ref)
    assert bad.size == 0, (bad[:8], D[tuple(bad[0])], ref[tuple(bad[0])])


@pytest.mark.parametrize("d,n", [(2, 32), (3, 16)])
def test_loss_gradient_and_adam_match_oracle(d, n):
    pb, lk = _problem(d, n, 5)
    params = pin.smoother_init(d, seed=4, noise=0.2)
    h = _handle(pb, d, lk, params)
    try:
        E = pin.start_vectors(9, pb.N, 8)
        R = pb.A @ E
        feat = sm.node_features(d, n, lk)
        dinv = 1.0 / pb.A.diagonal()
        loss, grad = P.pase_smoother_step(h, E, R, want_grad=True, P=P.pase_smoother_nparams(d))
        _, Lj, gref = sm.loss_and_grad(params.astype(np.float64), E, R, pb.A, dinv, feat, d, n - 1)
        np.testing.assert_allclose(loss, Lj, rtol=1e-5)
        off = 0  # per layer: weights, then bias; in norm and entry by entry
        T = 3 ** d
        for ci, co, _ in sm.layer_shapes(d):
            for size in (co * ci * T, co):
                g, gr = grad[off:off + size], gref[off:off + size]
                assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr) + 1e-12, (off, size)
                assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr)) + 1e-12, (off, size)
                off += size
        # one Adam step from zero moments applies the oracle's update to the library's
        # gradient; the library's hyper-parameters are float32 (0.999 is 0.99900001287)
        lr = 1e-3
        P.pase_smoother_step(h, E, R, update=True, lr=lr)
        p1, m1, v1, t1 = P.pase_smoother_state(h, d)
        f32 = lambda x: float(np.float32(x))
        pref, mref, vref = sm.adam(params.astype(np.float64), grad.astype(np.float32).astype(np.float64),
                                   np.zeros(params.size), np.zeros(params.size), 1, f32(lr), f32(0.9), f32(0.999),
                                   f32(1e-8))
        assert t1 == 1
        np.testing.assert_allclose(m1, mref, rtol=1e-6, atol=1e-30)
        np.testing.assert_allclose(v1, vref, rtol=1e-5, atol=1e-30)
        np.testing.assert_allclose(p1, pref, rtol=1e-6, atol=1e-6 * lr)
    finally:
        P.pase_destroy(h)


def test_learned_vcycle_matches_oracle():
    d, n = 2, 32
    pb, lk = _problem(d, n, 6)
    params = pin.smoother_init(d, seed=5, noise=0.05)
    h = _handle(pb, d, lk, params, smoother=P.PASE_SMOOTHER_LEARNED)
    try:
        m = 16
        U = pin.start_vectors(5, pb.N, m)
        lam = np.linspace(20.0, 300.0, m)
        W = np.empty_like(U)
        P.pase_linear_solve(h, m, U, lam, None, W)
        dinv = 1.0 / pb.A.diagonal()
        hier = mg.Hierarchy(pb.A, pb.chain,
                            fine_smoother=sm.fine_smoother(params, dinv, sm.node_features(d, n, lk), d, n - 1))
        Wref = opase.linear_solve(pb.A, pb.M, U, lam, 2, hier)
        assert _colrel(W - U, Wref - U) < 1e-3
        assert np.max(_colmax_err(W - U, Wref - U)) < 5e-3
    finally:
        P.pase_destroy(h)


def _vcycle_energy_factor(h, pb, m=16, seed=11):
    """||e||_A / ||e0||_A after the handle's step (a) (two V-cycles) on A e = A e0 from 0."""
    e0 = pin.start_vectors(seed, pb.N, m)
    U = np.zeros_like(e0)
    R = pb.A @ e0
    W = np.empty_like(e0)
    P.pase_linear_solve(h, m, U, np.ones(m), R, W)
    E = e0 - W
    return np.sqrt(np.einsum("ij,ij->j", E, pb.A @ E) / np.einsum("ij,ij->j", e0, pb.A @ e0))


def test_training_gains_over_jacobi():
    """Trained on one lognormal field and evaluated on a held-out one: the energy loss on
    the last training samples is below damped Jacobi's on the same samples, the library's
    own validation accepts
    the network, the two-V-cycle error factor on the held-out field is smaller than with
    Jacobi, and the eigen-solve with the learned smoother meets the same gates."""
    d, n = 2, 64
    pb, lk = _problem(d, n, 21, sigma=1.0)
    params = pin.smoother_init(d, seed=1, noise=0.02)
    h = _handle(pb, d, lk, params, smoother=P.PASE_SMOOTHER_LEARNED)
    try:
        out = P.pase_train_smoother(h, steps=600, lr=1e-3, seed=3)
        trained = P.pase_smoother_state(h, d)
    finally:
        P.pase_destroy(h)
    print("\ntraining:", out)
    # the samples come from the network's own V-cycle, so the loss of later steps is taken
    # on harder states than the first; the comparison that holds is with Jacobi on the
    # same samples
    assert out["loss_last"] < out["loss_jacobi"], out
    assert out["accepted"], out
    pbt, lkt = _problem(d, n, 77, sigma=1.0)
    hj = _handle(pbt, d, lkt, None)
    hl = _handle(pbt, d, lkt, trained[0], smoother=P.PASE_SMOOTHER_LEARNED)
    try:
        fj = _vcycle_energy_factor(hj, pbt)
        fl = _vcycle_energy_factor(hl, pbt)
        print(f"held-out field, two V-cycles, energy error factor: learned {np.mean(fl):.4f}, "
              f"Jacobi {np.mean(fj):.4f}")
        assert np.mean(fl) < np.mean(fj), (fl, fj)
        nev, m = 6, 16
        U0 = pin.start_vectors(0, pbt.N, m)
        U, lam = np.empty_like(U0), np.empty(m)
        rc, st = P.pase_solve(hl, nev, 1e-9, m, U0, lam, U)
        assert rc == P.PASE_OK
        ref, _ = dense.smallest_pairs_shift_invert(pbt.A, pbt.M, nev)
        np.testing.assert_allclose(lam[:nev], ref, rtol=1e-10)
        assert np.all(opase.relative_residuals(pbt.A, pbt.M, U[:, :nev], lam[:nev]) <= 1e-9)
    finally:
        P.pase_destroy(hj)
        P.pase_destroy(hl)


def test_smoother_argument_errors():
    pb, lk = _problem(2, 16, 2)
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        with pytest.raises(P.PaseError):
            P.pase_set_grid(h, 2, 17, lk)  # wrong size
        with pytest.raises(P.PaseError):
            P.pase_smoother_apply(h, 8, np.zeros((pb.N, 8)), np.zeros((pb.N, 8)))  # no grid yet
        P.pase_set_grid(h, 2, 16, lk)
        with pytest.raises(P.PaseError):
            P.pase_set_grid(h, 2, 16, lk)  # twice
        with pytest.raises(P.PaseError):
            P.pase_train_smoother(h, steps=5)  # no parameters yet
        assert P.pase_smoother_nparams(2) == sm.n_params(2) and P.pase_smoother_nparams(3) == sm.n_params(3)
        assert P.pase_smoother_nparams(4) == 0
    finally:
        P.pase_destroy(h)
