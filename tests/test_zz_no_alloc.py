"""lbm_observables_noalloc: the observables for callers that may not allocate
device memory (their device memory belongs to another runtime's pool, or
cudaMalloc's implicit synchronisation is not allowed where they run).

Called through the C ABI on two consecutive calls, it must reproduce what
lbm_mass_flow and lbm_slip_velocity return for the same velocity field, at
the fp64 parity tolerance of the other tests.  This file is collected last so
that a failure here cannot hide another test's result."""
import ctypes

import numpy as np
import pytest

import oracle
from lbm_inputs import rho_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _field_and_reference(Nx, Ny, Kn, steps, seed):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    g = oracle.force_for_mach(Kn)
    s = lbm.Solver(e, w, c, 4, Nx, Ny, Kn, g).init(rho_field(Nx, Ny, seed=seed)).step(steps)
    ux = s.moments()[1]
    return ux, s.mass_flow(), s.slip_velocity(), s.mean_ux(), g


def test_observables_noalloc_matches_solver_twice():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1510_08886_gb300 import _lib
    L = _lib.lib()
    stream = torch.cuda.current_stream()
    for Nx, Ny, Kn, steps, seed in [(256, 64, 0.1, 200, 1), (33, 37, 0.5, 100, 2)]:
        ux, mdot, us, mean, g = _field_and_reference(Nx, Ny, Kn, steps, seed)
        d_ux = torch.tensor(ux, dtype=torch.float64, device="cuda")
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.lbm_observables_noalloc(ctypes.c_void_p(d_ux.data_ptr()), Nx, Ny, Kn, g,
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] / mean - 1) < 1e-12
        assert abs(got[1] / mdot - 1) < 1e-12
        assert abs(got[2] / us - 1) < 1e-12


def test_observables_noalloc_rejects_oversized_fields():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1510_08886_gb300 import _lib
    L = _lib.lib()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(d.data_ptr())
    assert L.lbm_observables_noalloc(ptr, 4097, 4096, 0.1, 1e-3, ptr, None) == _lib.LBM_EINVAL
    assert L.lbm_observables_noalloc(ptr, 2, 3, 0.1, 1e-3, ptr, None) == _lib.LBM_EINVAL
