"""The allocation-free residual entry point against the ordinary one (needs a GPU).

pase_residual_noalloc serves callers that cannot call cudaMalloc (a memory arena that
owns the whole device, a host runtime whose callbacks forbid allocation, allocation-free
serving paths).  It must give the same residual block and relative residuals as
pase_residual, within the tolerance of the residual parity test, on consecutive calls
that share its fixed scratch array.  This file is collected last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import pase_inputs as pin

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def _colrel(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))


@pytest.mark.parametrize("m", [16, 64])
def test_residual_noalloc_matches_residual(m):
    pb = pin.build_problem(3, 24, 6, kappa_seed=7, mg_min=3)
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    stream = torch.cuda.current_stream()
    h = P.pase_create(opt, stream.cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        rowptr = torch.from_numpy(pb.A.indptr.astype(np.int64)).cuda()
        colind = torch.from_numpy(pb.A.indices.astype(np.int32)).cuda()
        aval = torch.from_numpy(pb.A.data.copy()).cuda()
        mval = torch.from_numpy(pb.M.data.copy()).cuda()
        for call, seed in enumerate((11, 12)):  # two calls in a row share the scratch
            U = torch.from_numpy(pin.start_vectors(seed, pb.N, m)).cuda()
            lam = torch.linspace(20.0, 400.0 + 10 * call, m, dtype=torch.float64, device="cuda")
            R_ref = torch.empty(pb.N, m, dtype=torch.float64, device="cuda")
            rr_ref = torch.empty(m, dtype=torch.float64, device="cuda")
            P.pase_residual(h, m, U, lam, R_ref, rr_ref)
            R = torch.full((pb.N, m), np.nan, dtype=torch.float64, device="cuda")
            rr = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
            P.pase_residual_noalloc(pb.N, m, rowptr, colind, aval, mval, U, lam, R, rr, stream)
            torch.cuda.synchronize()
            assert _colrel(R.cpu().numpy(), R_ref.cpu().numpy()) < 1e-13
            np.testing.assert_allclose(rr.cpu().numpy(), rr_ref.cpu().numpy(), rtol=1e-12)
    finally:
        P.pase_destroy(h)


def test_residual_noalloc_rejects_oversize_block():
    n, m = 8, 72
    z64 = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    z32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    U = torch.zeros(n, m, dtype=torch.float64, device="cuda")
    lam = torch.ones(m, dtype=torch.float64, device="cuda")
    rr = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PaseError) as e:
        P.pase_residual_noalloc(n, m, z64, z32, v, v, U, lam, None, rr)
    assert e.value.code == -1
