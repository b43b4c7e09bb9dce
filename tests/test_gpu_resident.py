"""Resident chunks of tiny fp64 and fp32 channels (one thread-block cluster, both
lattices in distributed shared memory, many steps per launch) against the
per-step launches of the same step: bitwise equal states, moments and
convergence decisions; and against the fp64 oracle."""
import numpy as np
import pytest

import oracle
from lbm_inputs import rho_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build_library()


def _solver(name, N, Nx, Ny, Kn, resident, stream=None, rho=None, precision="fp64"):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm(name)
    g = oracle.force_for_mach(Kn, 1e-2)
    s = lbm.Solver(e, w, c, N, Nx, Ny, Kn, g, stream=stream, precision=precision)
    return s.set_resident(resident).init(rho)


# config 1; Nx > 1 with a ragged last CTA; rows per CTA < max|e_y| (the wall
# sums and the pulls cross several CTAs); one row per CTA; Ny = max|e_y|;
# LP = 8 / 16 / 32 lanes per node
SHAPES = [("D2V16", 3, 1, 64), ("D2V16", 3, 5, 37), ("D2V33", 4, 3, 20), ("D2V33", 4, 1, 9),
          ("D2V16", 3, 2, 4), ("D3V107xz", 3, 1, 48), ("D2V32", 3, 2, 21), ("D2V16", 2, 1, 16)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,N,Nx,Ny", SHAPES)
def test_resident_steps_bitwise_equal_launched(name, N, Nx, Ny, precision):
    rho = rho_field(Nx, Ny, seed=5, amplitude=1e-3)
    a = _solver(name, N, Nx, Ny, 0.2, True, rho=rho, precision=precision)
    b = _solver(name, N, Nx, Ny, 0.2, False, rho=rho, precision=precision)
    assert a.resident_ctas() > 0 and b.resident_ctas() == 0
    for n in (1, 2, 123):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations())
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,N,Nx,Ny", SHAPES[:4])
def test_resident_run_to_steady_bitwise(name, N, Nx, Ny, precision):
    a = _solver(name, N, Nx, Ny, 0.1, True, precision=precision)
    b = _solver(name, N, Nx, Ny, 0.1, False, precision=precision)
    ra = a.run_to_steady(1e-9, 20000, check_every=50)
    rb = b.run_to_steady(1e-9, 20000, check_every=50)
    assert ra == rb
    assert np.array_equal(a.populations(), b.populations())
    assert a.mass_flow() == b.mass_flow() and a.slip_velocity() == b.slip_velocity()
    a.step(3)                       # odd lattice parity, then a tail chunk of 1 step
    b.step(3)
    ra = a.run_to_steady(1e-16, a.steps + 101, check_every=50)
    rb = b.run_to_steady(1e-16, b.steps + 101, check_every=50)
    assert ra == rb and ra[1] == a.steps
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("check_every", [2, 3])
def test_resident_smallest_chunks(check_every):
    """Chunks of 2 and 3 steps: the step that writes u_x for the convergence
    test is the chunk's first (or second) step; tests and steps agree with the
    per-step launches bit for bit, on the default stream and in graphs."""
    for stream in (None, torch.cuda.Stream()):
        a = _solver("D2V16", 3, 1, 64, 0.1, True, stream=stream)
        b = _solver("D2V16", 3, 1, 64, 0.1, False, stream=stream)
        ra = a.run_to_steady(1e-16, 41, check_every=check_every)
        rb = b.run_to_steady(1e-16, 41, check_every=check_every)
        assert ra == rb and ra[1] == 41
        assert np.array_equal(a.populations(), b.populations())
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)


def test_resident_graph_chunks_and_long_launch_split():
    """Graph-captured resident chunks on a side stream, and an lbm_step longer
    than one resident launch (4096 steps), equal the per-step launches."""
    a = _solver("D2V16", 3, 1, 64, 0.1, True, stream=torch.cuda.Stream())
    b = _solver("D2V16", 3, 1, 64, 0.1, False)
    assert a.run_to_steady(1e-10, 50000) == b.run_to_steady(1e-10, 50000)
    assert np.array_equal(a.populations(), b.populations())
    a.step(4096 + 5)
    b.step(4096 + 5)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.moments()[1], b.moments()[1])


def test_config1_resident_matches_oracle():
    """Config 1 (D2V16, N = 3, 1 x 64, Kn = 0.1, Ma 1e-3, tol 1e-10) on the
    resident path: same step count as the oracle, mass flow to 1e-12."""
    import paper_1510_08886_gb300 as lbm
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    e, w, c = lbm.dvm("D2V16")
    s = lbm.Solver(e, w, c, 3, 1, 64, Kn, g).init()
    assert s.resident_ctas() > 0
    ref = oracle.channel("D2V16", 3, 1, 64, Kn, g).init()
    conv, steps, _ = s.run_to_steady(1e-10, 50000)
    conv_o, steps_o, _ = ref.run_to_steady(1e-10, 50000)
    assert conv and conv_o and steps == steps_o
    assert abs(s.mass_flow() / ref.mass_flow() - 1) < 1e-12
    ux_o = ref.moments()[1]
    assert np.max(np.abs(s.moments()[1] - ux_o)) < 1e-12 * np.max(np.abs(ux_o))


def test_resident_checkpoint_into_launched_solver():
    """State taken from a resident run and restored into a per-step solver
    continues bit for bit."""
    a = _solver("D2V33", 4, 3, 20, 0.3, True)
    b = _solver("D2V33", 4, 3, 20, 0.3, False)
    a.step(77)
    b.set_state(a.get_state())
    a.step(41)
    b.step(41)
    assert np.array_equal(a.populations(), b.populations())


def test_config1_fp32_resident_matches_oracle():
    """Config 1 in fp32 on the resident path: mass flow and slip velocity at
    steady state within the fp32 tolerance (1e-4) of the fp64 oracle."""
    import paper_1510_08886_gb300 as lbm
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    e, w, c = lbm.dvm("D2V16")
    s = lbm.Solver(e, w, c, 3, 1, 64, Kn, g, precision="fp32").init()
    assert s.resident_ctas() > 0
    ref = oracle.channel("D2V16", 3, 1, 64, Kn, g).init()
    assert s.run_to_steady(1e-10, 50000)[0] and ref.run_to_steady(1e-10, 50000)[0]
    assert abs(s.mass_flow() / ref.mass_flow() - 1) < 1e-4
    assert abs(s.slip_velocity() / ref.slip_velocity() - 1) < 1e-4


def test_resident_solvers_of_different_sizes_coexist():
    """Two resident solvers of different sizes on the same kernel: planning
    the second leaves the first stepping bit for bit like its per-step twin."""
    big = _solver("D2V16", 3, 1, 512, 0.2, True)         # 32 rows per CTA
    small = _solver("D2V16", 3, 1, 20, 0.2, True)
    assert big.resident_ctas() > 0 and small.resident_ctas() > 0
    big_ref = _solver("D2V16", 3, 1, 512, 0.2, False)
    for s in (big, small, big_ref):
        s.step(30)
    assert big.status() == 0
    assert np.array_equal(big.populations(), big_ref.populations())


def test_resident_eligibility():
    """Only fp64 and fp32 channels small enough for one cluster run resident."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V16")
    assert lbm.Solver(e, w, c, 3, 64, 512, 0.1, 1e-3).resident_ctas() == 0
    assert lbm.Solver(e, w, c, 3, 1, 64, 0.1, 1e-3, precision="fp32").resident_ctas() > 0
    assert lbm.Solver(e, w, c, 3, 1, 64, 0.1, 1e-3, precision="fp16").resident_ctas() == 0
    s = lbm.Solver(e, w, c, 3, 1, 64, 0.1, 1e-3)
    assert 1 <= s.resident_ctas() <= 16
    assert s.set_resident(False).resident_ctas() == 0
    assert s.set_resident(True).resident_ctas() > 0
