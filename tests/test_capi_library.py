"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/sbec.h declares (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sbec.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sbec_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_01194_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sbec_create", "sbec_destroy", "sbec_energy", "sbec_grad", "sbec_hessvec",
              "sbec_retract", "sbec_sync", "sbec_scalars", "sbec_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (sbec_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_resolves(lib):
    from paper_1907_01194_gb300 import sbec
    assert set(sbec.library_symbols()) == set(sbec.EXPORTED)
    assert sbec._lib.sbec_status_string(sbec.ERR_DOMAIN).decode().startswith("point outside")



def test_solve_defaults_and_option_layout(lib):
    # sbec_solve_defaults is host-only: the paper's solver settings plus the CG
    # chunking defaults; the binding's struct matches the header's field order
    import ctypes
    from paper_1907_01194_gb300 import sbec
    o = sbec.SolveOpts()
    sbec._lib.sbec_solve_defaults(ctypes.byref(o))
    assert (o.method, o.retraction, o.tol, o.maxit) == (sbec.ARNT, 1, 1e-6, 10000)
    assert (o.rgbb_tol, o.rgbb_maxit, o.project_initial) == (1e-2, 2000, 1)
    assert (o.cg_chunk, o.cuda_graphs, o.refine_cg_fp32) == (4, 1, 1)
    hdr = open(os.path.join(ROOT, "include", "sbec.h")).read()
    body = hdr[hdr.index("typedef struct sbec_solve_opts"):hdr.index("} sbec_solve_opts;")]
    fields = re.findall(r"^\s*(?:int|double)\s+(\w+);", body, re.M)
    assert fields == [f for f, _ in sbec.SolveOpts._fields_]


def test_tune_struct_layout(lib):
    from paper_1907_01194_gb300 import sbec
    hdr = open(os.path.join(ROOT, "include", "sbec.h")).read()
    body = hdr[hdr.index("typedef struct sbec_tune"):hdr.index("} sbec_tune;")]
    fields = re.findall(r"^\s*(?:int|double)\s+(\w+)", body, re.M)
    assert fields == [f for f, _ in sbec.Tune._fields_]
