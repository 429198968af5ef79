"""Host-side checks of the C ABI library (no GPU needed).

The shared library must load and export every entry point that
include/msdd.h declares; the product package must not import the oracle;
argument validation that happens before any device work is exercised.
"""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msdd.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msdd_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2106_06404_gb300 import msdd
    return msdd.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "msdd_setup" in names and "msdd_solve" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2106_06404_gb300 import msdd
    assert sorted(msdd.EXPORTED) == _declared()


def test_struct_sizes_match_c_layout(lib):
    """ctypes mirrors of the ABI structs have the C sizes (compiled probe)."""
    from paper_2106_06404_gb300 import msdd
    src = r'''
#include <stdio.h>
#include "msdd.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu\n", sizeof(msdd_mesh), sizeof(msdd_coeff), sizeof(msdd_decomp),
 sizeof(msdd_spectral), sizeof(msdd_options), sizeof(msdd_stats));return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    py = [ctypes.sizeof(t) for t in (msdd.Mesh, msdd.Coeff, msdd.Decomp, msdd.Spectral, msdd.Options, msdd.Stats)]
    assert sizes == py


def test_num_unknowns_and_validation(lib):
    from paper_2106_06404_gb300 import msdd
    assert msdd.num_unknowns((64, 64), 0b1) == 64 * 65
    assert msdd.num_unknowns((512, 512), 0b1) == 262656
    assert msdd.num_unknowns((4, 4, 4), 0b1) == 4 * 5 * 5
    assert lib.msdd_num_unknowns(ctypes.byref(msdd.make_mesh((8, 8), 0))) == -1     # no Dirichlet face
    opt = msdd.default_options()
    assert opt.eig_maxit == 200 and opt.sigma == 1e-2 and opt.precision == 0
    # NULL arguments are rejected before any device work
    h = ctypes.c_void_p()
    st = lib.msdd_setup(None, None, None, None, None, ctypes.byref(h))
    assert st == -1 and b"invalid mesh" in lib.msdd_last_error()


def test_hybrid_and_gmres_reject_null_arguments(lib):
    """The hybrid preconditioner and GMRES entry points validate their
    arguments before any device work."""
    buf = (ctypes.c_double * 4)()
    it = ctypes.c_int(-7)
    rel = ctypes.c_double(0.0)
    st = lib.msdd_apply_hybrid_preconditioner(None, buf, buf)
    assert st == -1 and b"NULL" in lib.msdd_last_error()
    st = lib.msdd_solve_gmres(None, buf, ctypes.c_double(1e-8), 200, 1000, buf, ctypes.byref(it), ctypes.byref(rel))
    assert st == -1 and b"NULL" in lib.msdd_last_error()
    assert it.value == -7                                 # outputs untouched on error


def test_product_package_does_not_import_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_2106_06404_gb300; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle imported'") % ROOT
    subprocess.check_call([sys.executable, "-c", code])


def test_no_source_mentions_oracle_in_library():
    csrc = os.path.join(ROOT, "paper_2106_06404_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read().lower()
        assert "oracle" not in txt, f


def _setup_args(msdd):
    mesh = msdd.make_mesh((16, 16), 0b1)
    coeff = msdd.Coeff()
    coeff.kind = 0
    coeff.data = ctypes.c_void_p(0x1000)     # never dereferenced: every case fails validation first
    dec = msdd.Decomp()
    for d, v in enumerate((4, 4, 1)):
        dec.parts[d] = v
        dec.group[d] = 2
    dec.overlap, dec.levels = 1, 3
    spec = msdd.Spectral()
    spec.nev_max, spec.eta, spec.blf = 6, 0.3, 1
    return mesh, coeff, dec, spec, msdd.default_options()


SETUP_CASES = [
    # (field, value, expected status, message fragment)
    ("mesh.dim", 4, -1, b"invalid mesh"),
    ("mesh.dirichlet_faces", 0, -1, b"invalid mesh"),
    ("coeff.kind", 2, -1, b"invalid coefficient"),
    ("dec.levels", 1, -1, b"levels must be"),
    ("dec.levels", 4, -7, b"2 or 3 levels"),
    ("dec.overlap", 0, -1, b"overlap"),
    ("dec.parts", 17, -1, b"parts"),
    ("dec.group", 0, -1, b"group"),
    ("spec.nev_max", 25, -1, b"nev_max"),
    ("spec.eta", 0.0, -1, b"eta"),
    ("spec.blf", 4, -1, b"blf"),
    ("opt.precision", 2, -1, b"precision"),
    ("opt.block_p", 6, -1, b"block_p must exceed nev_max"),
    ("opt.block_p", 33, -1, b"block_p out of range"),
    ("opt.sigma", 0.0, -1, b"eigensolver options"),
    ("opt.reg_tol", 1.0, -1, b"eigensolver options"),
    ("opt.warm_cols", 0, -1, b"warm_cols"),
]


@pytest.mark.parametrize("field,value,status,msg", SETUP_CASES)
def test_setup_rejects_invalid_arguments_before_device_work(lib, field, value, status, msg):
    from paper_2106_06404_gb300 import msdd
    mesh, coeff, dec, spec, opt = _setup_args(msdd)
    obj, name = field.split(".")
    target = {"mesh": mesh, "coeff": coeff, "dec": dec, "spec": spec, "opt": opt}[obj]
    if name in ("parts", "group"):
        getattr(target, name)[0] = value
    else:
        setattr(target, name, value)
    if field == "opt.warm_cols":
        opt.warm_start = ctypes.c_void_p(0x2000)
    h = ctypes.c_void_p(0x1234)
    st = lib.msdd_setup(ctypes.byref(mesh), ctypes.byref(coeff), ctypes.byref(dec), ctypes.byref(spec),
                        ctypes.byref(opt), ctypes.byref(h))
    assert st == status, (field, st, lib.msdd_last_error())
    assert msg in lib.msdd_last_error()
    assert not h.value                                    # *out cleared on failure


@pytest.mark.parametrize("n,parts,overlap,faces", [
    ((16, 16), (4, 4), 1, 0b1),
    ((52, 44), (6, 5), 2, 0b1),
    ((37, 23), (5, 3), 3, 0b0101),          # Dirichlet on x = 0 and y = 0
    ((20, 9), (3, 2), 2, 0b1010),           # Dirichlet on x = 1 and y = 1
    ((12, 10, 8), (3, 2, 2), 1, 0b1),
    ((11, 9, 7), (2, 3, 2), 2, 0b100001),   # Dirichlet on x = 0 and z = 1
])
def test_fine_boxes_match_oracle_decomposition(lib, n, parts, overlap, faces):
    """The library's fine box partition with overlap (the same host code the
    set-up uses) gives each subdomain the Neumann box of the oracle's
    decomposition (Section 2.2 box partition, first N mod P blocks one element
    larger), in the same order, with row offsets the running sums."""
    from oracle import fem
    from oracle.decomposition import Decomposition
    from paper_2106_06404_gb300 import msdd
    lay = msdd.fine_layout(n, parts, overlap, faces)
    mesh = fem.Mesh(n, faces)
    dec = Decomposition(mesh, parts, overlap, 2, (1,) * len(n))
    assert lay.shape == (len(dec.fine), 4)
    off = 0
    for i, s in enumerate(dec.fine):
        want = [hi - lo + 1 for lo, hi in s.neumann_box] + [1] * (3 - len(n))
        assert list(lay[i, :3]) == want, (i, list(lay[i]), want)
        assert lay[i, 3] == off
        off += int(np.prod(want))


def test_status_names_match_header_enum():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef enum msdd_status \{(.*?)\} msdd_status;", txt, flags=re.S).group(1)
    enum = {int(v): k for k, v in re.findall(r"(MSDD_[A-Z_]+)\s*=\s*(-?\d+)", body)}
    from paper_2106_06404_gb300 import msdd
    assert enum == msdd.STATUS_NAMES
    assert enum[-8] == "MSDD_ERR_TIMEOUT"


def _batch_call(lib, msdd, meshes, coeffs, decs, spec, opt, nworkers=2, tol=1e-8, maxit=100, bptr=0x3000):
    k = len(meshes)
    M, C, D = (msdd.Mesh * k)(*meshes), (msdd.Coeff * k)(*coeffs), (msdd.Decomp * k)(*decs)
    bp = (ctypes.c_void_p * k)(*([bptr] * k))
    xp = (ctypes.c_void_p * k)(*([0x4000] * k))
    st = (ctypes.c_int * k)()
    return lib.msdd_batch_run(k, M, C, D, ctypes.byref(spec), ctypes.byref(opt), bp, tol, maxit, xp, nworkers, None,
                              None, st, None, None)


def test_batch_run_rejects_invalid_problems_before_device_work(lib):
    """msdd_batch_run checks every problem (naming it) and the shared element
    shape before it touches the device: these calls need no GPU."""
    from paper_2106_06404_gb300 import msdd
    mesh, coeff, dec, spec, opt = _setup_args(msdd)
    # a problem whose decomposition is invalid: named by its index
    bad = msdd.Decomp()
    ctypes.memmove(ctypes.byref(bad), ctypes.byref(dec), ctypes.sizeof(dec))
    bad.overlap = 0
    assert _batch_call(lib, msdd, [mesh, mesh], [coeff, coeff], [dec, bad], spec, opt) == -1
    assert b"problem 1" in lib.msdd_last_error() and b"overlap" in lib.msdd_last_error()
    # elements of another shape (32 x 16 elements on the unit square) cannot share the reference matrices
    other = msdd.make_mesh((32, 16), 0b1)
    assert _batch_call(lib, msdd, [mesh, other], [coeff, coeff], [dec, dec], spec, opt) == -7
    assert b"problem 1" in lib.msdd_last_error() and b"one shape" in lib.msdd_last_error()
    # NULL right-hand side, no worker, a non-positive tolerance
    assert _batch_call(lib, msdd, [mesh], [coeff], [dec], spec, opt, bptr=0) == -1
    assert _batch_call(lib, msdd, [mesh], [coeff], [dec], spec, opt, nworkers=0) == -1
    assert _batch_call(lib, msdd, [mesh], [coeff], [dec], spec, opt, tol=0.0) == -1
