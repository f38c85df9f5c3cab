"""The seeded generator of the batched workload: deterministic, inside its ranges, and
drawn from the stated sizes (no GPU)."""
import pase_inputs as pin


def test_batch_workload_is_seeded_and_in_range():
    a = pin.batch_workload(0, 64)
    assert a == pin.batch_workload(0, 64)
    assert a != pin.batch_workload(1, 64)
    assert pin.batch_workload(0, 8) == a[:8]  # problem i depends on draws 4i..4i+3 only
    for p in a:
        assert p["d"] == 2 and p["n"] in (64, 128, 256, 512) and p["n_coarse"] * 8 == p["n"]
        assert 0.5 <= p["sigma"] < 2.0 and 8 <= p["nev"] <= 32 and 0 <= p["kappa_seed"] < 2**31
    assert {p["n"] for p in a} == {64, 128, 256, 512}
    assert len({p["nev"] for p in a}) > 10


def test_start_vector_rows_are_slices_of_the_block():
    full = pin.start_vectors(3, 50, 24)
    parts = [pin.start_vector_rows(3, 24, a, b) for a, b in ((0, 7), (7, 31), (31, 50))]
    import numpy as np
    np.testing.assert_array_equal(np.vstack(parts), full)
