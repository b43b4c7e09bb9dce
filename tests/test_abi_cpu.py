"""C-ABI checks that need no GPU: the library loads, exports every function
include/lbm.h declares, and its host-only parts (DVM utilities, argument
validation of lbm_create_in) behave as documented.  No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

from lbm_inputs import DVM_TABLES, TEXTBOOK_TABLES
from oracle import dvm as odvm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1510_08886_gb300 import _lib
    return _lib


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(L):
    lib = L.lib()
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each one
    assert declared <= set(L.SIGNATURES), declared - set(L.SIGNATURES)


def test_strerror(L):
    assert L.lib().lbm_strerror(L.LBM_EDEGREE).decode().startswith("quadrature")
    assert L.lib().lbm_strerror(12345).decode() == "unknown error"


@pytest.mark.parametrize("name", sorted(DVM_TABLES) + sorted(TEXTBOOK_TABLES))
def test_expand_matches_oracle(L, name):
    import paper_1510_08886_gb300 as lbm
    t = {**DVM_TABLES, **TEXTBOOK_TABLES}[name]
    e, w, c = lbm.dvm_from_groups(t)
    e2, w2, _ = odvm.expand(t)
    a = sorted(zip(map(tuple, e.tolist()), w.tolist()))
    b = sorted(zip(map(tuple, e2.tolist()), w2.tolist()))
    assert a == b


@pytest.mark.parametrize("name", ["D3V107xz", "D3V96xz", "D3V112xz", "D3V77xz", "D3V66xz",
                                  "D3V59xz", "D3V64xz"])
def test_marginal_matches_oracle(L, name):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm(name)
    e2, w2, _ = odvm.dvm2d(name, DVM_TABLES)
    a = dict(zip(map(tuple, e.tolist()), w.tolist()))
    b = dict(zip(map(tuple, e2.tolist()), w2.tolist()))
    assert a.keys() == b.keys()
    assert max(abs(a[k] - b[k]) for k in a) < 1e-16


@pytest.mark.parametrize("name", ["D2V16", "D2V33", "D2V32", "D3V107xz", "D3V96xz"])
def test_quadrature_order_matches_oracle(L, name):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm(name)
    assert lbm.quadrature_order(e, w, c) == odvm.quadrature_order(e.astype(np.int64), w, c)


def _create_in(L, e, w, c, order=3, Nx=4, Ny=16, Kn=0.1, g=1e-3, prec=0, ws=1 << 20,
               nbytes=None):
    import paper_1510_08886_gb300 as lbm
    d = lbm._DVM(e, w, c)
    h = ctypes.c_void_p()
    if nbytes is None:
        n = ctypes.c_size_t(0)
        rc = L.lib().lbm_workspace_bytes(d.ref(), Nx, Ny, prec, ctypes.byref(n))
        nbytes = n.value if rc == 0 else 1 << 30
    # a fake, never dereferenced device address: lbm_create_in only records it
    rc = L.lib().lbm_create_in(d.ref(), order, Nx, Ny, Kn, g, prec, None,
                               ctypes.c_void_p(ws), nbytes, ctypes.byref(h))
    if rc == 0:
        L.lib().lbm_destroy(h)
    return rc


def test_create_validation(L):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    assert _create_in(L, e, w, c, order=4) == 0
    assert _create_in(L, e, w, c, order=5) == L.LBM_EDEGREE     # beyond 4
    assert _create_in(L, e, w, c, order=1) == L.LBM_EDEGREE
    assert _create_in(L, e, w, c, Ny=3) == L.LBM_EINVAL        # Ny < max |e_y| = 4
    assert _create_in(L, e, w, c, Ny=4) == 0
    assert _create_in(L, e, w, c, Kn=0.0) == L.LBM_EINVAL
    assert _create_in(L, e, w, c, Kn=float("nan")) == L.LBM_EINVAL
    assert _create_in(L, e, w, c, Nx=0) == L.LBM_EINVAL
    assert _create_in(L, e, w, c, prec=7) == L.LBM_EINVAL
    assert _create_in(L, e, w, c, ws=1 << 20 | 8) == L.LBM_EINVAL   # misaligned
    assert _create_in(L, e, w, c, nbytes=1024) == L.LBM_ENOMEM
    w2 = w.copy()
    w2[0] *= 1.001                                                # sum w != 1
    assert _create_in(L, e, w2, c) == L.LBM_EINVAL
    e2 = e.copy()
    e2[1] = e2[2]                                                 # duplicate velocity
    assert _create_in(L, e2, w, c) == L.LBM_EINVAL
    # not closed under e -> -e: drop a pair member and renormalise
    keep = [i for i in range(len(w)) if not (e[i, 0] == 3 and e[i, 1] == 0)]
    assert _create_in(L, e[keep], w[keep] / w[keep].sum(), c) == L.LBM_EINVAL


def test_degree_check_uses_measured_order(L):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V16")                  # Q = 7
    assert _create_in(L, e, w, c, order=4) == 0  # (Q+1)/2 admissible
    t = dict(D=2, c=np.sqrt(3.0), groups=[((0, 0), 1, 4 / 9), ((1, 0), 4, 1 / 9),
                                          ((1, 1), 4, 1 / 36)])
    e9, w9, c9 = lbm.dvm_from_groups(t)          # D2Q9, Q = 5
    assert lbm.quadrature_order(e9, w9, c9) == 5
    assert _create_in(L, e9, w9, c9, order=3, Ny=8) == 0
    assert _create_in(L, e9, w9, c9, order=4, Ny=8) == L.LBM_EDEGREE
    # c away from the tabulated value breaks the quadrature
    assert _create_in(L, e9, w9, 1.5, order=2, Ny=8) == L.LBM_EDEGREE


def test_solver_requires_cuda(L):
    import torch
    import paper_1510_08886_gb300 as lbm
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    e, w, c = lbm.dvm("D2V16")
    with pytest.raises(RuntimeError, match="CUDA"):
        lbm.Solver(e, w, c, 3, 1, 16, 0.1, 1e-3)


def test_compiled_set_header_is_current():
    """csrc/dvm_sets.h is generated from the paper's tables; it must match a
    fresh generation, and each compiled set must be the velocity set the
    library's own expansion produces."""
    import paper_1510_08886_gb300 as lbm
    from paper_1510_08886_gb300 import gen_dvm_sets as gen
    assert open(gen.HEADER).read() == gen.render()
    for ident, tname, marg in gen.SETS:
        e, w, c = lbm.dvm(tname + ("xz" if marg else ""))
        rest, pos = gen.pairs_of({tuple(v) for v in e.tolist()})
        assert len(pos) * 2 + rest == len(e)


def test_average_and_fma_rate_validate_before_any_device_call(L):
    """lbm_average and lbm_fma_rate reject bad arguments with LBM_EINVAL
    before touching a device (so this runs without a GPU)."""
    lib = L.lib()
    out = ctypes.c_double(0.0)
    assert lib.lbm_average(None, 10, 1) == L.LBM_EINVAL
    assert lib.lbm_fma_rate(L.LBM_FP16, None, ctypes.byref(out)) == L.LBM_EINVAL
    assert lib.lbm_fma_rate(7, None, ctypes.byref(out)) == L.LBM_EINVAL
    assert lib.lbm_fma_rate(L.LBM_FP64, None, None) == L.LBM_EINVAL


def test_engine_schedule_rejects_a_null_engine(L):
    """The schedule setter and getter check the handle before anything else
    (no device call)."""
    lib = L.lib()
    tw, tc, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    f = ctypes.c_double(0.0)
    assert lib.lbm_engine_set_schedule(None, -1, 32, 256, 4, 1.0) == L.LBM_EINVAL
    assert lib.lbm_engine_get_schedule(None, 0, ctypes.byref(tw), ctypes.byref(tc), ctypes.byref(g),
                                       ctypes.byref(f)) == L.LBM_EINVAL
