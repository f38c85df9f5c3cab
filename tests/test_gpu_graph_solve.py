"""Device-decided solves (option graph_solve) and the single-graph batch, through the C ABI
(needs a GPU).

A recorded solve runs the same kernels in the same order as the host-driven solve; only
who evaluates the stopping tests differs (a one-thread kernel instead of the host, on the
same numbers).  So, with the block-size autotuner off (its timing-based choices change
summation orders between handles), it must take the same number of outer and inner
iterations and return the same pairs to rounding.  The pairs are also checked against the
closed form or a shift-invert reference (1e-10 relative), their residuals recomputed by the
oracle, and the block's M-orthonormality.
"""
import numpy as np
import pytest

import pase_inputs as pin
from oracle import dense, pase as opase, spectrum

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def _handle(pb, stream=None, **kw):
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    for k, v in kw.items():
        setattr(opt, k, v)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    h = P.pase_create(opt, s)
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


def _run(pb, nev, tol, m, start_seed=0, repeats=1, **kw):
    kw.setdefault("autotune", 0)
    h = _handle(pb, **kw)
    try:
        U0 = None if start_seed is None else torch.from_numpy(pin.start_vectors(start_seed, pb.N, m)).cuda()
        U = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(repeats):
            rc, st = P.pase_solve(h, nev, tol, m, U0, lam, U)
            outs.append((rc, st, lam.cpu().numpy(), U.cpu().numpy()))
        return outs
    finally:
        P.pase_destroy(h)


@pytest.mark.parametrize("precision", [P.PASE_PREC_FP64, P.PASE_PREC_MIXED])
def test_graph_solve_matches_host_driven(precision):
    """2D Q1 128^2, coarse 16^2, nev 10: the whole solve as one graph launch."""
    pb = pin.build_problem(2, 128, 16, mg_min=4)
    nev, m = 10, 16
    (rc0, st0, l0, U0), = _run(pb, nev, 1e-8, m, precision=precision)
    (rc1, st1, l1, U1), = _run(pb, nev, 1e-8, m, precision=precision, graph_solve=1)
    assert rc0 == rc1 == P.PASE_OK
    assert st1["graph_launches"] == 1
    assert (st1["iterations"], st1["aug_iterations"], st1["converged"]) == \
        (st0["iterations"], st0["aug_iterations"], st0["converged"])
    assert st1["kernel_launches"] > 50 * st1["iterations"]
    np.testing.assert_allclose(l1, l0, rtol=1e-13)
    assert np.max(np.abs(np.abs(U1) - np.abs(U0))) < 1e-9
    _check(pb, l1, U1, nev, spectrum.q1_laplace_eigenvalues(2, 128, nev), 1e-8)


def test_graph_solve_replay_is_reproducible():
    """The second call replays the recorded graph: bit-identical output."""
    pb = pin.build_problem(2, 64, 8, kappa_seed=21, mg_min=4)
    nev, m = 6, 16
    outs = _run(pb, nev, 1e-9, m, repeats=3, graph_solve=1)
    for rc, st, lam, U in outs:
        assert rc == P.PASE_OK and st["graph_launches"] == 1
    for rc, st, lam, U in outs[1:]:
        np.testing.assert_array_equal(lam, outs[0][2])
        np.testing.assert_array_equal(U, outs[0][3])
        assert st["iterations"] == outs[0][1]["iterations"]
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check(pb, outs[0][2], outs[0][3], nev, ref, 1e-9)


@pytest.mark.parametrize("kw", [dict(), dict(post_solve=1), dict(aug_transform=P.PASE_AUG_PRECOND_BA),
                                dict(linear_solver=P.PASE_SOLVER_MGCG, inner_steps=2,
                                     precision=P.PASE_PREC_MIXED)])
def test_graph_solve_coarse_start_and_variants(kw):
    """Coarse start (no U0), the two-solve form, a transformed step (c) and mixed MGCG,
    each recorded whole: same iterations and pairs as the host-driven solve."""
    pb = pin.build_problem(3, 32, 8, kappa_seed=5, mg_min=4)
    nev, m = 8, 16
    (rc0, st0, l0, U0), = _run(pb, nev, 1e-9, m, start_seed=None, **kw)
    (rc1, st1, l1, U1), = _run(pb, nev, 1e-9, m, start_seed=None, graph_solve=1, **kw)
    assert rc0 == rc1 == P.PASE_OK
    assert (st1["iterations"], st1["aug_iterations"]) == (st0["iterations"], st0["aug_iterations"])
    np.testing.assert_allclose(l1, l0, rtol=1e-12)
    ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
    _check(pb, l1, U1, nev, ref, 1e-9)


def test_graph_solve_not_converged_status():
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    (rc, st, lam, U), = _run(pb, 4, 1e-14, 8, graph_solve=1, max_iter=2)
    assert rc == P.PASE_ERR_NOT_CONVERGED
    assert st["iterations"] == 2


def test_pass_limit_ends_device_loop_with_timeout():
    """A recorded loop capped at two passes (graph_pass_limit) while the solve needs about
    ten: the device ends the loop and the call reports PASE_ERR_TIMEOUT; the context stays
    usable and the next solve succeeds."""
    pb = pin.build_problem(2, 64, 8, mg_min=4)
    nev, m = 6, 16
    with pytest.raises(P.PaseError) as e:
        _run(pb, nev, 1e-10, m, graph_solve=1, graph_pass_limit=2)
    assert e.value.code == P.PASE_ERR_TIMEOUT
    (rc, st, lam, U), = _run(pb, nev, 1e-9, m, graph_solve=1)
    assert rc == P.PASE_OK
    _check(pb, lam, U, nev, spectrum.q1_laplace_eigenvalues(2, 64, nev), 1e-9)


def _batch(probs, **kw):
    streams = [torch.cuda.Stream() for _ in probs]
    handles, U0s, Us, lams, ms = [], [], [], [], []
    try:
        for (pb, nev, tol, _), s in zip(probs, streams):
            m = pin.guard_columns(nev)
            handles.append(_handle(pb, s, **kw))
            ms.append(m)
            U0s.append(torch.from_numpy(pin.start_vectors(0, pb.N, m)).to("cuda"))
            Us.append(torch.empty(pb.N, m, dtype=torch.float64, device="cuda"))
            lams.append(torch.empty(m, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        runs = []
        for _ in range(2):  # the second call replays the batch graph
            rc, sts = P.pase_solve_batched(handles, [p[1] for p in probs], [p[2] for p in probs], ms, U0s,
                                           lams, Us)
            runs.append((rc, sts, [l.cpu().numpy() for l in lams], [u.cpu().numpy() for u in Us]))
        return runs, ms
    finally:
        for h in handles:
            P.pase_destroy(h)


def test_batched_one_graph_matches_single_solves():
    probs = [
        (pin.build_problem(2, 64, 8, mg_min=4), 4, 1e-9, "closed"),
        (pin.build_problem(2, 64, 8, kappa_seed=21, mg_min=4), 6, 1e-9, "si"),
        (pin.build_problem(3, 32, 8, mg_min=4), 10, 1e-8, "closed"),
        (pin.build_problem(2, 128, 16, mg_min=4), 8, 1e-9, "closed"),
        (pin.build_problem(3, 16, 4, kappa_seed=7, mg_min=4), 5, 1e-9, "si"),
    ]
    runs, ms = _batch(probs, graph_solve=1, autotune=0)
    for rc, sts, lams, Us in runs:
        assert rc == P.PASE_OK, sts
        assert sum(s["graph_launches"] for s in sts) == 1
    for i, (pb, nev, tol, kind) in enumerate(probs):
        lam, U = runs[0][2][i], runs[0][3][i]
        np.testing.assert_array_equal(runs[1][2][i], lam)
        if kind == "closed":
            ref = spectrum.q1_laplace_eigenvalues(pb.d, pb.n, nev)
        else:
            ref, _ = dense.smallest_pairs_shift_invert(pb.A, pb.M, nev)
        _check(pb, lam, U, nev, ref, tol)
        # the same problem alone (host-driven) takes the same iterations
        (rc1, st1, l1, _), = _run(pb, nev, tol, ms[i])
        assert rc1 == P.PASE_OK and st1["iterations"] == runs[0][1][i]["iterations"]
        np.testing.assert_allclose(lam[:nev], l1[:nev], rtol=1e-12)


def test_batched_one_graph_host_buffers_and_partial_failure():
    pbs = [pin.build_problem(2, 32, 4, mg_min=4), pin.build_problem(2, 64, 8, mg_min=4)]
    streams = [torch.cuda.Stream() for _ in pbs]
    handles = [_handle(pbs[0], streams[0], graph_solve=1), _handle(pbs[1], streams[1], graph_solve=1, max_iter=1)]
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
