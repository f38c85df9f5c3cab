"""The C ABI library loads and exports every function include/pase.h declares (CPU only;
no compute calls), and the binding fails loudly without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pase.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(pase_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2502_04589_gb300 import build
    build.build()
    from paper_2502_04589_gb300 import pase as P
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2502_04589_gb300 import pase as P
    assert sorted(P.EXPORTED) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_2502_04589_gb300 import pase as P
    assert P.pase_status_string(0) == "ok"
    assert "pattern" in P.pase_status_string(-3)
    o = P.pase_default_options()
    assert (o.inner_steps, o.nu1, o.nu2, o.coarse_level) == (2, 2, 2, -1)
    assert abs(o.omega - 2.0 / 3.0) < 1e-15


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    from paper_2502_04589_gb300 import pase as P
    with pytest.raises(P.PaseError) as e:
        P.pase_create(P.pase_default_options())
    assert e.value.code == -8


def test_missing_library_fails_loudly(tmp_path):
    from paper_2502_04589_gb300 import pase as P
    saved = P._lib
    try:
        P._lib = None
        with pytest.raises(RuntimeError):
            P.load_library(str(tmp_path / "nope.so"))
    finally:
        P._lib = saved
