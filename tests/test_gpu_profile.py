"""Live kernel timing (pase_profile_kernel / pase_profile_read) through the C ABI (needs a GPU)."""
import numpy as np
import pytest

import pase_inputs as pin

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2502_04589_gb300.pase")

pytestmark = pytest.mark.gpu


def test_profile_counts_fine_level_jacobi_launches():
    """Two V-cycles with 2+2 sweeps from zero: the first cycle's first sweep is the scaled
    right-hand side, so the fine level sees 1 + 2 + 2 + 2 = 7 Jacobi launches per step."""
    pb = pin.build_problem(3, 32, 8, mg_min=4)
    m = 16
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    s = torch.cuda.Stream()
    h = P.pase_create(opt, s)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        with torch.cuda.stream(s):
            U = torch.from_numpy(pin.start_vectors(0, pb.N, m)).cuda()
            lam = torch.zeros(m, dtype=torch.float64, device="cuda")
        s.synchronize()
        P.pase_iterate(h, 8, m, U, lam, False)
        P.pase_profile_kernel(h, "jacobi_fp64")
        for _ in range(3):
            P.pase_iterate(h, 8, m, U, lam, True)
        n, ms = P.pase_profile_read(h)
        assert n == 3 * 7 and ms > 0.0
        n2, ms2 = P.pase_profile_read(h)  # a read starts a new count
        assert n2 == 0 and ms2 == 0.0
        P.pase_profile_kernel(h, None)
        P.pase_iterate(h, 8, m, U, lam, True)
        assert P.pase_profile_read(h) == (0, 0.0)
        with pytest.raises(P.PaseError):
            P.pase_profile_kernel(h, "gram_fp64")
        assert np.all(np.isfinite(lam.cpu().numpy()))
    finally:
        P.pase_destroy(h)
