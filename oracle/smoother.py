"""Learned fine-level smoother: a small convolutional network in place of damped Jacobi
inside the V-cycle of the step-(a) linear solve (test infrastructure only).

The paper has no learned smoother; this module states the definition the CUDA path is
checked against, in plain float64 NumPy:

Grid.  The fine level is the (n-1)^d interior-node grid of the uniform n^d Q1 mesh,
node i = sum_k c_k (n-1)^k (x fastest).  The node feature f_i is the mean of log kappa
over the 2^d elements that contain node i.

Network (per column of a block, independently).  Input channels: s_i = (D^-1 r)_i / rho
and f_i, rho = sqrt(mean_i (D^-1 r)_i^2) (the column's root-mean-square Jacobi-scaled
residual; rho = 0 gives a zero correction).  Four 3^d convolutions with zero padding,
2 -> 16 -> 16 -> 16 -> 1 channels, ReLU after the first three.  Convolution:
    y[b, co, i] = bias[co] + sum_ci sum_t W[co, ci, t] x[b, ci, i + o_t],
tap t = sum_k (o_k + 1) 3^k for offsets o in {-1, 0, 1}^d (x fastest).
Correction: delta = rho * y, so S(alpha r) = alpha S(r) for alpha > 0.

Parameters: one flat vector [W1, b1, W2, b2, W3, b3, W4, b4], W_l in [co][ci][t] order.
The forward pass uses the parameters rounded to bfloat16 (round to nearest even); the
master copy that Adam updates stays in float32 (straight-through: the gradient with
respect to the rounded parameters is applied to the master copy).

Training loss (per column j; r = A e is the residual of the error e that the solver's
iterate still carries):  L_j = (e - delta)^T A (e - delta) / (e^T r), the squared energy
norm of the error left after one smoothing step relative to the error before it; the
batch loss is the mean over columns.  Adam as in Kingma & Ba (2015).

Use in the V-cycle: on level 0 each of the nu1 pre- and nu2 post-smoothing sweeps
x <- x + omega D^-1 (b - A x) becomes x <- x + S(b - A x); coarser levels keep Jacobi.
Inference (the V-cycle, `apply(..., act_bf16=True)`) rounds the network input and stores
the hidden activations in bfloat16 between layers: tensor-core MMAs of kind f16 take both
operands in 16-bit form, so the activations that feed them are bfloat16 numbers.  Training
differentiates the same network with FP32 inputs and activations; `inference_error_bound`
bounds, elementwise, how far the inference form can move from it.

Parity: pinned in tests/test_oracle_smoother.py (convolution against scipy.ndimage,
finite-difference gradients, positive homogeneity, the Jacobi-equivalent weights,
Adam's first step in closed form, the loss at delta = 0 and delta = e, the inference
form within its rounding-error bound of the FP32-activation network).
"""
import numpy as np

CHANNELS = 16


def layer_shapes(d):
    """(c_in, c_out, relu) of the four layers."""
    return [(2, CHANNELS, True), (CHANNELS, CHANNELS, True), (CHANNELS, CHANNELS, True), (CHANNELS, 1, False)]


def taps(d):
    return 3 ** d


def n_params(d):
    return sum(co * ci * taps(d) + co for ci, co, _ in layer_shapes(d))


def unpack(params, d):
    """[(W [co][ci][t], b [co], relu)] views of the flat parameter vector."""
    out, o = [], 0
    T = taps(d)
    for ci, co, relu in layer_shapes(d):
        W = params[o:o + co * ci * T].reshape(co, ci, T)
        o += co * ci * T
        b = params[o:o + co]
        o += co
        out.append((W, b, relu))
    assert o == len(params)
    return out


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def offsets(d):
    """Offset vectors o_t, t = sum_k (o_k + 1) 3^k."""
    T = taps(d)
    return [tuple((t // 3 ** k) % 3 - 1 for k in range(d)) for t in range(T)]


def _shift(X, o, d, n1):
    """X[..., i + o] on the grid with zero outside; X [..., N] with N = n1^d (x fastest)."""
    lead = X.shape[:-1]
    G = X.reshape(lead + (n1,) * d)  # axes: ..., c_{d-1}, ..., c_0
    out = np.zeros_like(G)
    src, dst = [], []
    for k in reversed(range(d)):  # grid axis order: highest coordinate first
        ok = o[k]
        if ok == 0:
            src.append(slice(None))
            dst.append(slice(None))
        elif ok > 0:
            src.append(slice(ok, None))
            dst.append(slice(None, -ok))
        else:
            src.append(slice(None, ok))
            dst.append(slice(-ok, None))
    out[(Ellipsis,) + tuple(dst)] = G[(Ellipsis,) + tuple(src)]
    return out.reshape(X.shape)


def conv(X, W, b, d, n1):
    """X [B][ci][N] -> [B][co][N], zero padding."""
    B, ci, N = X.shape
    co = W.shape[0]
    Y = np.broadcast_to(b[None, :, None], (B, co, N)).astype(np.float64).copy()
    for t, o in enumerate(offsets(d)):
        Xs = _shift(X, o, d, n1)
        Y += np.einsum("oc,bcn->bon", W[:, :, t], Xs)
    return Y


def node_features(d, n, log_kappa):
    """Mean of log kappa over the 2^d elements around each interior node."""
    n1 = n - 1
    L = np.asarray(log_kappa, dtype=np.float64).reshape((n,) * d)
    acc = np.zeros((n1,) * d)
    for corner in range(2 ** d):
        sl = []
        for k in reversed(range(d)):
            lo = (corner >> k) & 1
            sl.append(slice(lo, lo + n1))
        acc += L[tuple(sl)]
    return (acc / 2 ** d).reshape(-1)


def forward(params, s, feat, d, n1, round_bf16=True, act_bf16=False):
    """s [B][N] (normalised Jacobi-scaled residual), feat [N] -> y [B][N] and a cache.
    act_bf16: the network input (s, f) and the hidden activations (outputs of the three
    ReLU layers) are rounded to bfloat16, as the library's inference path stores them."""
    p = bf16_round(params) if round_bf16 else np.asarray(params, dtype=np.float64)
    B = s.shape[0]
    x = np.stack([s, np.broadcast_to(feat, s.shape)], axis=1)
    if act_bf16:
        x = bf16_round(x.astype(np.float32))
    cache = []
    for W, bb, relu in unpack(p, d):
        z = conv(x, W, bb, d, n1)
        cache.append((x, z))
        x = np.maximum(z, 0.0) if relu else z
        if relu and act_bf16:
            x = bf16_round(x.astype(np.float32))
    return x[:, 0, :], (p, cache)


def backward(cache, gy, d, n1):
    """Gradient of sum(gy * y) with respect to the (rounded) parameters, flat."""
    p, layers = cache
    grads = []
    g = gy[:, None, :]
    for li in reversed(range(len(layers))):
        W, bb, relu = unpack(p, d)[li]
        x, z = layers[li]
        if relu:
            g = g * (z > 0.0)
        gW = np.zeros_like(W)
        for t, o in enumerate(offsets(d)):
            gW[:, :, t] = np.einsum("bon,bcn->oc", g, _shift(x, o, d, n1))
        gb = g.sum(axis=(0, 2))
        grads.append((gW, gb))
        if li > 0:  # gradient with respect to this layer's input (transposed convolution)
            gx = np.zeros_like(x)
            for t, o in enumerate(offsets(d)):
                gx += _shift(np.einsum("oc,bon->bcn", W[:, :, t], g), tuple(-v for v in o), d, n1)
            g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return np.concatenate(flat)


def normalise(r, dinv):
    """r [N][B] -> s [B][N] and rho [B]."""
    q = (dinv[:, None] * r).T
    rho = np.sqrt(np.mean(q * q, axis=1))
    s = np.where(rho[:, None] > 0, q / np.where(rho > 0, rho, 1.0)[:, None], 0.0)
    return s, rho


def apply(params, r, dinv, feat, d, n1, round_bf16=True, act_bf16=False):
    """The correction delta = S(r) for a residual block r [N][B]; returns [N][B].
    act_bf16=True is the inference form (hidden activations stored in bfloat16)."""
    s, rho = normalise(r, dinv)
    y, _ = forward(params, s, feat, d, n1, round_bf16, act_bf16)
    return (y * rho[:, None]).T


# Relative change of one rounding of the inference form: float64 -> float32 -> bfloat16,
# each to nearest (8 significand bits: 2^-8; the float32 step adds at most 2^-24 and its
# product with the first term, covered by 2^-23).
BF16_UNIT_ROUNDOFF = 2.0 ** -8 + 2.0 ** -23


def inference_error_bound(params, r, dinv, feat, d, n1, kind="worst", c=5.0, round_bf16=True):
    """Elementwise bound on |apply(act_bf16=True) - apply(act_bf16=False)|, [N][B].

    The inference form rounds the inputs x_l of the four layers (the network input and the
    three ReLU outputs) to bfloat16, a fresh rounding error e_l with |e_l| <= u |x_l| (u =
    BF16_UNIT_ROUNDOFF) at each.  To first order in u the output moves by sum_l J_l e_l, J_l
    the Jacobian of the output with respect to x_l in the FP32-activation network (with that
    network's ReLU masks), times the column scale rho.

    kind="worst": the first-order worst case  u sum_l sum_k |J_l[i,k]| |x_l[k]|.
    kind="prob":  c sqrt(sum_l sum_k (u J_l[i,k] x_l[k])^2), the probabilistic bound of
      rounding-error analysis (Higham and Mary, SIAM J. Sci. Comput. 41, 2019): with the
      roundings modelled as independent, mean-zero and bounded by u |x|, Hoeffding's
      inequality puts the first-order output error above it with probability at most
      2 exp(-c^2 / 2) (7.5e-6 for c = 5).
    Terms of second order in u, and ReLU outputs whose sign the roundings flip, are not in
    either (a flip moves a value by no more than its own first-order perturbation)."""
    if kind not in ("worst", "prob"):
        raise ValueError(kind)
    u = BF16_UNIT_ROUNDOFF
    s, rho = normalise(r, dinv)
    _, (p, cache) = forward(params, s, feat, d, n1, round_bf16)
    layers = unpack(p, d)
    B, N = s.shape
    eye = np.arange(N)
    out = np.zeros((B, N))
    for b in range(B):
        g = np.zeros((N, 1, N))  # g[i] = derivative of output node i
        g[eye, 0, eye] = 1.0
        for li in reversed(range(len(layers))):
            W, _, relu = layers[li]
            x, z = cache[li]  # the layer's input and pre-activation
            if relu:
                g = g * (z[b] > 0.0)[None]
            gx = np.zeros((N, W.shape[1], N))
            for t, o in enumerate(offsets(d)):
                gx += _shift(np.einsum("oc,ion->icn", W[:, :, t], g), tuple(-v for v in o), d, n1)
            if kind == "worst":
                out[b] += u * np.einsum("icn,cn->i", np.abs(gx), np.abs(x[b]))
            else:
                out[b] += u * u * np.einsum("icn,cn->i", gx * gx, x[b] * x[b])
            g = gx
    if kind == "prob":
        out = c * np.sqrt(out)
    return (out * rho[:, None]).T


def loss_and_grad(params, e, r, A, dinv, feat, d, n1, round_bf16=True):
    """Batch loss mean_j (e_j - delta_j)^T A (e_j - delta_j) / (e_j^T r_j) and its gradient.
    e, r: [N][B] with r = A e."""
    s, rho = normalise(r, dinv)
    y, cache = forward(params, s, feat, d, n1, round_bf16)
    delta = (y * rho[:, None]).T
    E = e - delta
    AE = A @ E
    den = np.einsum("ij,ij->j", e, r)
    B = e.shape[1]
    L = np.einsum("ij,ij->j", E, AE) / den
    gy = (-2.0 * AE * rho[None, :] / (B * den[None, :])).T
    return float(L.mean()), L, backward(cache, gy, d, n1)


def adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def fine_smoother(params, dinv, feat, d, n1, round_bf16=True, act_bf16=True):
    """Callable x-correction S(r) for `mg.Hierarchy(..., fine_smoother=...)` (inference
    form by default)."""
    return lambda r: apply(params, r, dinv, feat, d, n1, round_bf16, act_bf16)
