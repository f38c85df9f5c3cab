"""Pins of the learned-smoother oracle (no GPU): convolution against scipy.ndimage,
gradients against finite differences, positive homogeneity, the Jacobi-equivalent
weights, Adam's first step in closed form, the loss at delta = 0 and delta = e, and the
learned V-cycle reducing to the Jacobi V-cycle, and the bf16 inference form within its
derived rounding-error bound of the FP32-activation network."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import pase_inputs as pin
from oracle import mg, smoother as sm


@pytest.mark.parametrize("d,n1", [(2, 7), (3, 5)])
def test_conv_matches_scipy_correlate(d, n1):
    rng = np.random.default_rng(d)
    B, ci, co = 2, 3, 4
    N = n1 ** d
    X = rng.standard_normal((B, ci, N))
    W = rng.standard_normal((co, ci, 3 ** d))
    b = rng.standard_normal(co)
    Y = sm.conv(X, W, b, d, n1)
    for bb in range(B):
        for o in range(co):
            ref = np.full((n1,) * d, b[o])
            for c in range(ci):
                # tap t = sum_k (o_k+1) 3^k, x fastest -> C-order kernel [o_{d-1}+1]...[o_0+1]
                K = W[o, c].reshape((3,) * d)
                ref += ndi.correlate(X[bb, c].reshape((n1,) * d), K, mode="constant", cval=0.0)
            np.testing.assert_allclose(Y[bb, o].reshape((n1,) * d), ref, rtol=1e-12, atol=1e-12)


def test_bf16_round_known_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 2.0 / 3.0, -3.0e38], dtype=np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even -> 1
    # 1 + 3*2^-9 lies above the midpoint -> 1 + 2^-7; 2/3 -> 0.66796875 (171/256)
    exp = np.array([1.0, 1.0, 1.0 + 2 ** -7, 0.66796875, -(226 / 128) * 2.0 ** 127])  # 3e38 = 1.7632 * 2^127
    np.testing.assert_allclose(sm.bf16_round(x), exp, rtol=1e-7)


def _tiny(d):
    """A small variable-coefficient stiffness matrix and its node features."""
    n = 8 if d == 2 else 5
    kappa = pin.lognormal_kappa(d, n, 3, 1.0)
    A, _ = pin.q1_matrices(d, n, kappa)
    return A, n, sm.node_features(d, n, np.log(kappa))


@pytest.mark.parametrize("d", [2, 3])
def test_gradient_matches_finite_differences(d):
    A, n, feat = _tiny(d)
    n1 = n - 1
    N = A.shape[0]
    dinv = 1.0 / A.diagonal()
    rng = np.random.default_rng(7)
    params = pin.smoother_init(d, seed=2, noise=0.3).astype(np.float64)
    e = rng.standard_normal((N, 3))
    r = A @ e
    L, _, g = sm.loss_and_grad(params, e, r, A, dinv, feat, d, n1, round_bf16=False)
    idx = rng.choice(params.size, 25, replace=False)
    for k in idx:
        h = 1e-6 * max(1.0, abs(params[k]))
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        Lp = sm.loss_and_grad(pp, e, r, A, dinv, feat, d, n1, round_bf16=False)[0]
        Lm = sm.loss_and_grad(pm, e, r, A, dinv, feat, d, n1, round_bf16=False)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_positive_homogeneity_and_jacobi_weights():
    A, n, feat = _tiny(2)
    n1 = n - 1
    dinv = 1.0 / A.diagonal()
    r = np.random.default_rng(1).standard_normal((A.shape[0], 4))
    p = pin.smoother_init(2, seed=5, noise=0.2)
    np.testing.assert_allclose(sm.apply(p, 3.5 * r, dinv, feat, 2, n1), 3.5 * sm.apply(p, r, dinv, feat, 2, n1),
                               rtol=1e-12)
    pj = pin.smoother_init(2, omega=2.0 / 3.0, noise=0.0)
    om = sm.bf16_round(np.float32(2.0 / 3.0))
    np.testing.assert_allclose(sm.apply(pj, r, dinv, feat, 2, n1), om * dinv[:, None] * r, rtol=1e-12,
                               atol=1e-14)
    assert np.all(sm.apply(pj, 0.0 * r, dinv, feat, 2, n1) == 0.0)


def test_loss_at_zero_and_exact_correction():
    A, n, feat = _tiny(2)
    N = A.shape[0]
    e = np.random.default_rng(4).standard_normal((N, 2))
    r = A @ e
    dinv = 1.0 / A.diagonal()
    # zero network (all parameters 0): delta = 0, loss 1 for every column
    L0, Lj, _ = sm.loss_and_grad(np.zeros(sm.n_params(2)), e, r, A, dinv, feat, 2, n - 1)
    np.testing.assert_allclose(Lj, 1.0, rtol=1e-14)
    # the energy-norm identity for a Jacobi correction: L = 1 - 2w (q^T r)/(e^T r) + w^2 q^T A q/(e^T r)
    pj = pin.smoother_init(2, noise=0.0)
    w = sm.bf16_round(np.float32(2.0 / 3.0))
    q = dinv[:, None] * r
    exp = (np.einsum("ij,ij->j", e, r) - 2 * w * np.einsum("ij,ij->j", q, r)
           + w * w * np.einsum("ij,ij->j", q, A @ q)) / np.einsum("ij,ij->j", e, r)
    np.testing.assert_allclose(sm.loss_and_grad(pj, e, r, A, dinv, feat, 2, n - 1)[1], exp, rtol=1e-12)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = sm.adam(p, g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    np.testing.assert_allclose(p1, p - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_node_features_average_the_adjacent_elements():
    n = 4
    lk = np.arange(n * n, dtype=float)  # element (ex, ey) -> ex + 4 ey
    f = sm.node_features(2, n, lk)
    # interior node (cx, cy) = (1, 2) touches elements ex in {1, 2}, ey in {2, 3}
    i = 1 + 3 * 2
    assert f[i] == np.mean([1 + 8, 2 + 8, 1 + 12, 2 + 12])


def test_learned_vcycle_with_jacobi_weights_is_the_jacobi_vcycle():
    pb = pin.build_problem(2, 16, 4, kappa_seed=2)
    n1 = 15
    dinv = 1.0 / pb.A.diagonal()
    feat = sm.node_features(2, 16, np.log(pb.kappa))
    om = float(sm.bf16_round(np.float32(2.0 / 3.0)))
    pj = pin.smoother_init(2, omega=2.0 / 3.0, noise=0.0)
    H_l = mg.Hierarchy(pb.A, pb.chain, omega=om,
                       fine_smoother=sm.fine_smoother(pj, dinv, feat, 2, n1, act_bf16=False))
    H_j = mg.Hierarchy(pb.A, pb.chain, omega=om)
    b = np.random.default_rng(0).standard_normal((pb.N, 3))
    np.testing.assert_allclose(H_l.solve(b, 2), H_j.solve(b, 2), rtol=1e-11, atol=1e-13)


def test_bf16_activations_exact_when_representable():
    """Inference form: rounding the hidden activations to bfloat16 changes nothing when
    every activation is a bfloat16 number already (Jacobi weights on a residual whose
    Jacobi-scaled values are +-1, so that their RMS is 1 and the activations are 0 or 1),
    and stays within bfloat16 precision otherwise."""
    A, n, feat = _tiny(2)
    n1 = n - 1
    dinv = 1.0 / A.diagonal()
    q = np.ones((A.shape[0], 1))
    q[1::2, 0] = -1.0
    r = q / dinv[:, None]   # D^-1 r = q
    pj = pin.smoother_init(2, noise=0.0)
    a = sm.apply(pj, r, dinv, feat, 2, n1, act_bf16=True)
    b = sm.apply(pj, r, dinv, feat, 2, n1, act_bf16=False)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_inference_form_within_rounding_bound(d, seed):
    """The inference form (bf16 input and hidden activations) differs from the FP32-activation
    network by less than the probabilistic bound derived from the bf16 unit roundoff (c = 5)
    and by less than twice the first-order worst case; the probabilistic bound is a small
    fraction of the output scale, so it means something."""
    A, n, feat = _tiny(d)
    n1 = n - 1
    dinv = 1.0 / A.diagonal()
    p = pin.smoother_init(d, seed=3 + seed, noise=0.3)
    r = np.random.default_rng(2 + seed).standard_normal((A.shape[0], 3))
    a = sm.apply(p, r, dinv, feat, d, n1, act_bf16=True)
    b = sm.apply(p, r, dinv, feat, d, n1, act_bf16=False)
    worst = sm.inference_error_bound(p, r, dinv, feat, d, n1, kind="worst")
    prob = sm.inference_error_bound(p, r, dinv, feat, d, n1, kind="prob")
    slack = 1e-12 * np.max(np.abs(b), axis=0)
    assert np.any(np.abs(a - b) > 0.0)  # the roundings do act
    assert np.all(np.abs(a - b) <= 2.0 * worst + slack)  # 2: second-order terms, flips
    assert np.all(np.abs(a - b) <= prob + slack)
    assert np.all(prob <= worst * 5.0 + slack)
    assert np.max(prob) < 0.1 * np.max(np.abs(b))


def test_inference_bound_rejects_coarser_rounding(monkeypatch):
    """Planted mistake: activations rounded to 4 significand bits instead of 8 leave the
    probabilistic bf16 bound."""
    A, n, feat = _tiny(2)
    n1 = n - 1
    dinv = 1.0 / A.diagonal()
    p = pin.smoother_init(2, seed=3, noise=0.3)
    r = np.random.default_rng(2).standard_normal((A.shape[0], 3))
    b = sm.apply(p, r, dinv, feat, 2, n1, act_bf16=False)
    bound = sm.inference_error_bound(p, r, dinv, feat, 2, n1, kind="prob")
    pr = sm.bf16_round(p)  # the parameters as the forward pass uses them
    exact = sm.bf16_round

    def coarse(x):
        y = exact(x)
        e = np.floor(np.log2(np.maximum(np.abs(y), 1e-300)))
        q = 2.0 ** (e - 3)
        return np.where(y == 0, 0.0, np.round(y / q) * q)

    monkeypatch.setattr(sm, "bf16_round", coarse)
    a = sm.apply(pr, r, dinv, feat, 2, n1, round_bf16=False, act_bf16=True)
    monkeypatch.undo()
    assert np.any(np.abs(a - b) > bound)
