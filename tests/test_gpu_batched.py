"""Many problems at once (pase_solve_batched), the CUDA-graph replay of the linear solve
and the block-size autotuner, through the C ABI (needs a GPU).

Each problem of a batch must come out exactly as it would alone: eigenvalues against the
closed form or a shift-invert reference to 1e-10 relative, residuals recomputed by the
oracle below the requested tolerance, M-orthonormal blocks.  Graph replay runs the same
kernels in the same order as eager launches, so it must agree with them to rounding.
"""
import numpy as np
import pytest

import pase_inputs as pin
from oracle import dense, pase as opase, spectrum

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def _handle(pb, stream, **kw):
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    for k, v in kw.items():
        setattr(opt, k, v)
    h = P.pase_create(opt, stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
    except Exception:
        P.pase_destroy(h)
        raise
    return h


def _check(pb, lam, U, nev, ref, tol):
    np.testing.assert_allclose(lam[:nev], ref[:nev], rtol=1e-10)
    res = opase.relative_residuals(pb.A, pb.M, U[:, :nev], lam[:nev])
    assert np.all(res <= tol), res
    np.testing.assert_allclose(U.T @ (pb.M @ U), np.eye(U.shape[1]), atol=1e-10)


def _solve_one(pb, nev, tol, m, stream, **kw):
    h = _handle(pb, stream, **kw)
    try:
        with torch.cuda.stream(stream):
            U0 = torch.from_numpy(pin.start_vectors(0, pb.N, m)).to("cuda")
            U = torch.empty_like(U0)
            lam = torch.empty(m, dtype=torch.float64, device="cuda")
        stream.synchronize()
        rc, st = P.pase_solve(h, nev, tol, m, U0, lam, U)
        return rc, st, lam.cpu().numpy(), U.cpu().numpy()
    finally:
        P.pase_destroy(h)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_graph_replay_matches_eager(precision):
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    s = torch.cuda.Stream()
    out = {}
    for g in (0, 1):
        out[g] = _solve_one(pb, 6, 1e-9, 16, s, use_graphs=g, autotune=0, precision=precision)
    (rc0, st0, l0, U0), (rc1, st1, l1, U1) = out[0], out[1]
    assert rc0 == rc1 == P.PASE_OK
    assert st0["iterations"] == st1["iterations"]
    assert st0["kernel_launches"] == st1["kernel_launches"]
    np.testing.assert_allclose(l1, l0, rtol=1e-13)
    assert np.max(np.abs(np.abs(U1) - np.abs(U0))) < 1e-9
    _check(pb, l1, U1, 6, spectrum.q1_laplace_eigenvalues(2, 64, 6), 1e-9)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_autotuned_block_sizes_keep_results(precision):
    """The autotuner's choices (block sizes; in the mixed form also CSR vs the structured
    kernel and the latter's schedule per level) leave the solution within the gates."""
    pb = pin.build_problem(3, 32, 8, mg_min=4)
    s = torch.cuda.Stream()
    ref = spectrum.q1_laplace_eigenvalues(3, 32, 8)
    for tune in (0, 1):
        rc, st, lam, U = _solve_one(pb, 8, 1e-9, 16, s, autotune=tune, precision=precision)
        assert rc == P.PASE_OK
        _check(pb, lam, U, 8, ref, 1e-9)


def test_batched_matches_single_solves():
    probs = [
        (pin.build_problem(2, 64, 8, mg_min=4), 4, 1e-9, "closed"),
        (pin.build_problem(2, 64, 8, kappa_seed=21, mg_min=4), 6, 1e-9, "si"),
        (pin.build_problem(3, 32, 8, mg_min=4), 10, 1e-8, "closed"),
        (pin.build_problem(2, 128, 16, mg_min=4), 8, 1e-9, "closed"),
        (pin.build_problem(3, 16, 4, kappa_seed=7, mg_min=4), 5, 1e-9, "si"),
    ]
    streams = [torch.cuda.Stream() for _ in probs]
    handles, U0s, Us, lams, ms = [], [], [], [], []
    try:
        for (pb, nev, tol, _), s in zip(probs, streams):
            m = pin.guard_columns(nev)
            handles.append(_handle(pb, s))
            ms.append(m)
            U0s.append(torch.from_numpy(pin.start_vectors(0, pb.N, m)).to("cuda"))
            Us.append(torch.empty(pb.N, m, dtype=torch.float64, device="cuda"))
            lams.append(torch.empty(m, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        rc, sts = P.pase_solve_batched(handles, [p[1] for p in probs], [p[2] for p in probs], ms, U0s,
                                       lams, Us)
        assert rc == P.PASE_OK, sts
    finally:
        for h in handles:
            P.pase_destroy(h)
    for i, (pb, nev, tol, kind) in enumerate(probs):
        lam, U = lams[i].cpu().numpy(), Us[i].cpu().numpy()
        if kind == "closed":
            ref = spectrum.q1_laplace_eigenvalues(pb.d, pb.n, nev)
        else:
            ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
        _check(pb, lam, U, nev, ref, tol)
        assert sts[i]["converged"] >= nev
        # the same problem alone gives the same iteration count and eigenvalues
        rc1, st1, l1, _ = _solve_one(pb, nev, tol, ms[i], torch.cuda.Stream())
        assert rc1 == P.PASE_OK and st1["iterations"] == sts[i]["iterations"]
        np.testing.assert_allclose(lam[:nev], l1[:nev], rtol=1e-12)


def test_batched_host_buffers_and_partial_failure():
    """Host-memory start blocks and outputs; one problem capped at one iteration reports
    NOT_CONVERGED for the batch while the others still converge."""
    pbs = [pin.build_problem(2, 32, 4, mg_min=4), pin.build_problem(2, 64, 8, mg_min=4)]
    streams = [torch.cuda.Stream() for _ in pbs]
    handles = [_handle(pbs[0], streams[0]), _handle(pbs[1], streams[1], max_iter=1)]
    try:
        m = 8
        U0s = [pin.start_vectors(1, pb.N, m) for pb in pbs]
        Us = [np.empty((pb.N, m)) for pb in pbs]
        lams = [np.empty(m) for _ in pbs]
        rc, sts = P.pase_solve_batched(handles, [3, 3], [1e-9, 1e-12], [m, m], U0s, lams, Us)
        assert rc == P.PASE_ERR_NOT_CONVERGED
        assert sts[1]["iterations"] == 1
        _check(pbs[0], lams[0], Us[0], 3, spectrum.q1_laplace_eigenvalues(2, 32, 3), 1e-9)
    finally:
        for h in handles:
            P.pase_destroy(h)


def test_batched_argument_errors():
    assert P.load_library().pase_solve_batched(None, 0, None, None, None, None, None, None, None) == P.PASE_OK
    with pytest.raises(P.PaseError):
        P.pase_solve_batched([None], [2], [1e-9], [8], [None], [np.empty(8)], [np.empty((16, 8))])
