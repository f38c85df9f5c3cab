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


@pytest.mark.parametrize("field,value", [("sygv_tridiag", 3), ("sygv_tridiag", -2), ("sygv_cholesky", 2),
                                         ("stencil_columns", 3), ("aug_factor", 0.0), ("omega", 2.0)])
def test_create_rejects_invalid_options_before_any_device_call(lib, field, value):
    """Options are validated before the device is touched, so a bad field is reported as an
    invalid argument on any machine (a valid set on a machine without a GPU is a CUDA
    error, as above)."""
    from paper_2502_04589_gb300 import pase as P
    o = P.pase_default_options()
    setattr(o, field, value)
    with pytest.raises(P.PaseError) as e:
        P.pase_create(o)
    assert e.value.code == -1  # PASE_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path):
    from paper_2502_04589_gb300 import pase as P
    saved = P._lib
    try:
        P._lib = None
        with pytest.raises(RuntimeError):
            P.load_library(str(tmp_path / "nope.so"))
    finally:
        P._lib = saved


_CTYPES = {"int": "c_int", "double": "c_double", "float": "c_float", "unsigned": "c_uint",
           "int64_t": "c_int64"}


def _header_struct(name):
    """(field, C type, array length) of `typedef struct {...} name;` in include/pase.h."""
    src = open(os.path.join(ROOT, "include", "pase.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(const\s+)?([A-Za-z_0-9]+\s*\**)\s*(.*)", decl)
        ctype = m.group(2).replace(" ", "")
        for var in m.group(3).split(","):
            var = var.strip()
            if var.startswith("*"):
                ctype, var = ctype + "*", var[1:].strip()
            am = re.match(r"([A-Za-z_0-9]+)\s*(?:\[(\d+)\])?", var)
            out.append((am.group(1), ctype, int(am.group(2)) if am.group(2) else 0))
    return out


@pytest.mark.parametrize("cname,pyname", [("pase_options", "PaseOptions"), ("pase_stats", "PaseStats"),
                                          ("pase_train_options", "PaseTrainOptions"), ("pase_csr", "PaseCSR")])
def test_binding_structs_match_header(cname, pyname):
    """Field names, order and types of the ctypes mirrors equal the header's structs."""
    import ctypes
    from paper_2502_04589_gb300 import pase as P
    fields = getattr(P, pyname)._fields_
    decl = _header_struct(cname)
    assert [f[0] for f in fields] == [d[0] for d in decl]
    for (fname, ftype), (_, ctype, n) in zip(fields, decl):
        if ctype.endswith("*"):
            assert ftype is ctypes.c_void_p, fname
        elif n:
            assert ftype._length_ == n and ftype._type_ is getattr(ctypes, _CTYPES[ctype]), fname
        else:
            assert ftype is getattr(ctypes, _CTYPES[ctype]), fname


def test_default_options_of_the_later_fields(lib):
    from paper_2502_04589_gb300 import pase as P
    o = P.pase_default_options()
    assert (o.use_graphs, o.autotune, o.smoother, o.split_gemm, o.aug_adaptive) == (1, 1, P.PASE_SMOOTHER_JACOBI, 1, 1)
    assert (o.stencil, o.post_solve, o.aug_transform, o.spmm_df64, o.graph_solve) == (1, 0, P.PASE_AUG_PLAIN, 1, 0)
    assert (o.graph_pass_limit, o.stencil_columns, o.aug_factor, o.sygv_tridiag, o.sygv_cholesky) == (0, 0, 1e-4, -1, -1)
