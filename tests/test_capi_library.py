"""CPU-side checks of the C ABI library: it builds, loads, exports every entry
point declared in include/te.h, and reports the missing GPU as an error status."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, cuda_available


@pytest.fixture(scope="module")
def libte():
    from paper_2205_15346_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def header_functions():
    src = open(os.path.join(ROOT, "include", "te.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(te_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for required in ["te_create", "te_destroy", "te_build_csr", "te_build_model", "te_evolve",
                     "te_submit", "te_poll", "te_cancel", "te_request_free", "te_spmv",
                     "te_matrix_free", "te_last_error"]:
        assert required in names


def test_library_exports_every_header_function(libte):
    missing = [n for n in header_functions() if not hasattr(libte, n)]
    assert not missing, missing


def test_binding_covers_every_header_function():
    from paper_2205_15346_gb300 import te
    assert set(header_functions()) <= set(te.exported_symbols())


def test_host_only_entry_points(libte):
    from paper_2205_15346_gb300 import te
    assert "sm_103a" in te.te_version()
    assert te.te_status_string(te.TE_ERR_STEP_UNDERFLOW) == "TE_ERR_STEP_UNDERFLOW"
    o = te.te_default_options()
    assert (o.gauss_n, o.n_substeps, o.t_step0, o.shrink, o.quad_rel_tol, o.quad_max_levels) == \
        (20, 10, 0.1, 0.97, 1e-3, 15)


def test_bose_basis_index_matches_oracle_host(libte):
    """te_model_basis_index is host code: check it against the oracle's enumeration."""
    import workloads as W
    from oracle import models
    from paper_2205_15346_gb300 import te
    for K, N in [(3, 2), (5, 4), (8, 5)]:
        p = W.bose_params(K, N, seed=1)
        b = models.BoseBasis(K, N)
        for i in range(0, len(b), max(1, len(b) // 37)):
            assert te.te_model_basis_index(p, b.states[i]) == i
    p = W.bose_params(4, 3, seed=1)
    with pytest.raises(te.TEError):
        te.te_model_basis_index(p, (1, 1, 0, 0))     # wrong particle number


@pytest.mark.skipif(cuda_available(), reason="checks the no-device path")
def test_create_without_device_reports_error(libte):
    from paper_2205_15346_gb300 import te
    with pytest.raises(te.TEError):
        te.te_create(0, stream=0)


def test_binding_constants_match_the_header():
    """Every numeric #define of include/te.h has the same value in the binding."""
    from paper_2205_15346_gb300 import te
    src = open(os.path.join(ROOT, "include", "te.h")).read()
    defines = re.findall(r"^#define\s+(TE_[A-Z0-9_]+)\s+(-?(?:0x[0-9a-fA-F]+|\d+))u?\b", src, flags=re.M)
    assert len(defines) > 30
    for name, value in defines:
        assert hasattr(te, name), name
        assert getattr(te, name) == int(value, 0), name


def test_binding_structs_match_the_header():
    """The ctypes structures of the binding have the fields, order and types of
    the header's structs (a mismatch would corrupt every call silently)."""
    import ctypes as C

    from paper_2205_15346_gb300 import te
    src = open(os.path.join(ROOT, "include", "te.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint32_t": C.c_uint32,
             "double": C.c_double}
    structs = re.findall(r"typedef struct (te_[a-z_]+) \{(.*?)\} \1;", src, flags=re.S)
    assert {n for n, _ in structs} >= {"te_options", "te_stats", "te_matrix_info",
                                        "te_model_desc", "te_operator_desc"}
    for name, body in structs:
        fields = []
        for decl in (x.strip() for x in body.split(";") if x.strip()):
            fp = re.match(r"^.*\(\s*\*\s*([a-zA-Z0-9_]+)\s*\)\s*\((.*)\)$", decl, flags=re.S)
            if fp:                                   # function pointer: (name, argument count)
                fields.append(("fn", fp.group(2).count(",") + 1, fp.group(1)))
                continue
            f = re.match(r"^(?:const\s+)?([a-z0-9_]+)\s*(\*?)\s*([a-zA-Z0-9_]+)$", decl)
            assert f, (name, decl)
            fields.append(f.groups())
        py = getattr(te, name)._fields_
        assert [f[2] for f in fields] == [p[0] for p in py], name
        for (typ, star, fname), (_, pytype) in zip(fields, py):
            if typ == "fn":
                assert len(pytype._argtypes_) == star, (name, fname)
            elif typ == "void" and star:
                assert pytype is C.c_void_p, (name, fname)
            else:
                want = C.POINTER(ctype[typ]) if star else ctype[typ]
                assert pytype == want, (name, fname)


def test_binding_signatures_match_the_header():
    """Each entry point's ctypes signature has the header's arity, return type
    and scalar argument types (pointers may be typed or void)."""
    import ctypes as C

    from paper_2205_15346_gb300 import te
    src = open(os.path.join(ROOT, "include", "te.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    scalar = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint32_t": C.c_uint32,
              "double": C.c_double, "te_status": C.c_int32}
    protos = re.findall(r"^\s*(?:const\s+)?([a-z_0-9]+)\s*(\*?)\s*(te_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
                        src, flags=re.M)
    assert len(protos) >= 30
    for ret, rstar, name, args in protos:
        restype, argtypes = te._SIGS[name]
        if rstar:
            assert restype in (C.c_char_p, C.c_void_p), name
        elif ret == "void":
            assert restype is None, name
        else:
            assert restype == scalar[ret], name
        args = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert len(args) == len(argtypes), name
        for a, t in zip(args, argtypes):
            if "*" in a:
                assert t is C.c_void_p or hasattr(t, "contents") or t is C.c_char_p, (name, a)
            else:
                typ = a.replace("const ", "").split()[0]
                assert t == scalar[typ], (name, a)
