"""GPU parity: the CUDA path through the C ABI against the fp64 oracle, on
the same seeded inputs, element by element.

Tolerances (from the arithmetic):
* fp64: both sides evaluate the same step in double with different rounding
  orders; populations are O(w), so differences are O(1e-16) per step and
  stay bounded (the scheme is contractive).  Velocities u ~ 1e-3..1e-2:
  relative L_inf 1e-12 of max|u| on u, 1e-13 on the populations.
* fp32: deviations fbar - w stored and computed in float (relative 6e-8 on
  O(Ma) quantities): relative 1e-4 on mass flow and slip velocity at steady
  state, 2e-5 of max|u| on the velocity field after a few hundred steps.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import DVM_TABLES, rho_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (DVM, Hermite order): every register-resident shape plus generic-kernel sets
CASES = [("D2V16", 3), ("D2V33", 4), ("D2V32", 3), ("D3V107xz", 3), ("D3V96xz", 3),
         ("D3V112xz", 3), ("D3V77xz", 3), ("D3V66xz", 3), ("D3V59xz", 3), ("D2V33", 3),
         ("D2V16", 4), ("D2V16", 2), ("D2Q9", 2), ("D2Q9", 3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build_library()


def _tables():
    from lbm_inputs import TEXTBOOK_TABLES
    return {**DVM_TABLES, **TEXTBOOK_TABLES}


def _pair(name, N, Nx, Ny, Kn, g, rho, precision="fp64"):
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm(name, _tables())
    s = lbm.Solver(e, w, c, N, Nx, Ny, Kn, g, precision=precision).init(rho)
    ref = oracle.channel(name, N, Nx, Ny, Kn, g, tables=_tables()).init(rho)
    return s, ref, e


def _match_planes(e_gpu, ref):
    """Index of each GPU velocity in the oracle's velocity list."""
    lut = {(int(x), int(y)): i for i, (x, y) in enumerate(zip(ref.ex, ref.ey))}
    return np.array([lut[(int(x), int(y))] for x, y in e_gpu])


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name,N", CASES)
@pytest.mark.parametrize("Nx,Ny", [(37, 29), (1, 64), (5, 13)])
def test_fp64_parity_after_steps(name, N, Nx, Ny):
    """Moments and every post-collision population after 60 steps, seeded
    density perturbation, body force on; sizes span several 256-thread
    blocks with a ragged tail, Nx = 1 and Nx < max |e_x| (multiple wraps)."""
    e, _, _ = __import__("paper_1510_08886_gb300").dvm(name, _tables())
    Ny = max(Ny, int(np.max(np.abs(e[:, 1]))))
    Kn = 0.2
    g = oracle.force_for_mach(Kn, 1e-2)
    rho = rho_field(Nx, Ny, seed=11, amplitude=1e-3)
    s, ref, e = _pair(name, N, Nx, Ny, Kn, g, rho)
    s.step(60)
    # the GPU keeps the post-collision state fbar*(t) = collide(fbar(t)); the
    # oracle keeps fbar(t): compare moments at t = 60 and fbar* element-wise
    ref.step(60)
    rho_g, ux_g, uy_g = s.moments()
    rho_o, ux_o, uy_o = ref.moments()
    assert np.max(np.abs(rho_g - rho_o)) < 1e-13
    assert _rel(ux_g, ux_o) < 1e-12
    assert np.max(np.abs(uy_g - uy_o)) < 1e-12 * np.max(np.abs(ux_o))
    fs_o = ref.collide(ref.f)
    fs_g = s.populations()
    idx = _match_planes(e, ref)
    assert np.max(np.abs(fs_g - fs_o[idx])) < 1e-13


@pytest.mark.parametrize("name,N", [("D2V33", 4), ("D2V16", 3), ("D2V32", 3), ("D3V107xz", 3)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parity_interior_fast_path(name, N, precision):
    """Nx = 1024: 128-node blocks in interior rows take the fixed-offset pull
    path, the blocks at x = 0 and x = Nx - 128 the wrapping path (their warps
    away from the ends at fixed offsets), the wall rows the wall path -- for
    the sets with four wall rows as 32-column strips; all must agree with the
    oracle."""
    Nx, Ny, Kn = 1024, 30, 0.2
    g = oracle.force_for_mach(Kn, 1e-2)
    rho = rho_field(Nx, Ny, seed=21)
    s, ref, e = _pair(name, N, Nx, Ny, Kn, g, rho, precision=precision)
    s.step(12)
    ref.step(12)
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert _rel(s.moments()[1], ref.moments()[1]) < tol
    if precision == "fp64":
        idx = _match_planes(e, ref)
        assert np.max(np.abs(s.populations() - ref.collide(ref.f)[idx])) < 1e-13


@pytest.mark.parametrize("name,N", [("D2V16", 3), ("D2V33", 4), ("D3V107xz", 3)])
def test_fp64_minimum_ny(name, N):
    """Ny = max |e_y|: every row is a wall row of both walls."""
    e, _, _ = __import__("paper_1510_08886_gb300").dvm(name)
    Ny = int(np.max(np.abs(e[:, 1])))
    Kn = 0.5
    g = oracle.force_for_mach(Kn, 1e-2)
    rho = rho_field(3, Ny, seed=3)
    s, ref, e = _pair(name, N, 3, Ny, Kn, g, rho)
    s.step(40)
    ref.step(40)
    assert np.max(np.abs(s.moments()[0] - ref.moments()[0])) < 1e-13
    assert _rel(s.moments()[1], ref.moments()[1]) < 1e-12


def test_fp64_no_force_rest_state():
    """g = 0, rho = 1: the rest state stays a fixed point on the GPU."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    s = lbm.Solver(e, w, c, 4, 8, 16, 0.1, 0.0).init().step(200)
    f = s.populations()
    assert np.max(np.abs(f - w[:, None, None])) < 1e-15
    assert np.isnan(s.mass_flow())


def test_config1_steady_state_fp64():
    """D2V16, N = 3, Nx = 1 x Ny = 64, Kn = 0.1, Ma ~ 1e-3, run until
    max|du| < 1e-10 (<= 50k steps): steady profile, mass flow (Eq. pf.1) and
    slip velocity (Eq. defSlip) against the oracle."""
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    s, ref, _ = _pair("D2V16", 3, 1, 64, Kn, g, None)
    conv, steps, du = s.run_to_steady(1e-10, 50000)
    conv_o, steps_o, du_o = ref.run_to_steady(1e-10, 50000)
    assert conv and conv_o
    assert steps == steps_o
    assert _rel(s.moments()[1], ref.moments()[1]) < 1e-12
    assert abs(s.mass_flow() / ref.mass_flow() - 1) < 1e-12
    assert abs(s.slip_velocity() / ref.slip_velocity() - 1) < 1e-12


@pytest.mark.parametrize("Kn", [0.01, 0.1, 1.0])
def test_fp32_steady_state_mass_flow_and_slip(Kn):
    """fp32 deviation storage: steady mass flow and slip velocity within
    1e-4 relative of the fp64 oracle."""
    g = oracle.force_for_mach(Kn)
    s, ref, _ = _pair("D2V16", 3, 1, 64, Kn, g, None, precision="fp32")
    conv, _, _ = s.run_to_steady(1e-10, 200000)
    conv_o, _, _ = ref.run_to_steady(1e-10, 200000)
    assert conv_o
    assert abs(s.mass_flow() / ref.mass_flow() - 1) < 1e-4
    assert abs(s.slip_velocity() / ref.slip_velocity() - 1) < 1e-4


@pytest.mark.parametrize("name,N", [("D2V33", 4), ("D2V16", 3), ("D3V107xz", 3)])
def test_fp32_parity_after_steps(name, N):
    Kn = 0.1
    g = oracle.force_for_mach(Kn, 1e-2)
    rho = rho_field(33, 40, seed=2)
    s, ref, _ = _pair(name, N, 33, 40, Kn, g, rho, precision="fp32")
    s.step(300)
    ref.step(300)
    assert np.max(np.abs(s.moments()[0] - ref.moments()[0])) < 1e-6
    assert _rel(s.moments()[1], ref.moments()[1]) < 2e-5


def _window_oracle(name, N, Nx_full, Ny, Kn, g, rho, x0, width, steps, margin):
    """Oracle on columns [x0 - margin, x0 + width + margin) treated as a
    periodic channel: after `steps` steps the central `width` columns equal
    the full channel's (information travels max|e_x| columns per step)."""
    cols = [(x0 - margin + i) % Nx_full for i in range(width + 2 * margin)]
    ref = oracle.channel(name, N, len(cols), Ny, Kn, g).init(rho[:, cols]).step(steps)
    return ref.moments(), margin


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_full_size_config2_sampled(precision, tol):
    """Config 2 shape: D2V33, N = 4, 4096 x 512, Kn = 0.1, seeded rho =
    1 + 1e-3 N(0, 1), the benchmark's launch configuration.  After 3 steps
    the oracle recomputes three column windows (an edge at x = 0, the
    middle, the last column) exactly; mass is conserved over the run."""
    import paper_1510_08886_gb300 as lbm
    Nx, Ny, Kn, steps = 4096, 512, 0.1, 3
    g = oracle.force_for_mach(Kn)
    rho = rho_field(Nx, Ny, seed=20151029)
    e, w, c = lbm.dvm("D2V33")
    s = lbm.Solver(e, w, c, 4, Nx, Ny, Kn, g, precision=precision).init(rho).step(steps)
    rho_g, ux_g, _ = s.moments()
    umax = None
    for x0 in (0, 2048, 4090):
        (r_o, u_o, _), m = _window_oracle("D2V33", 4, Nx, Ny, Kn, g, rho, x0, 6, steps, 4 * steps + 2)
        cols = [(x0 + i) % Nx for i in range(6)]
        u_c = u_o[:, m:m + 6]
        umax = np.max(np.abs(u_c)) if umax is None else max(umax, np.max(np.abs(u_c)))
        assert np.max(np.abs(ux_g[:, cols] - u_c)) < tol * np.max(np.abs(u_c))
        assert np.max(np.abs(rho_g[:, cols] - r_o[:, m:m + 6])) < (1e-13 if precision == "fp64" else 1e-6)
    # total mass: sum fbar over the lattice equals the initial mass
    assert abs(rho_g.sum() / rho.sum() - 1) < (1e-13 if precision == "fp64" else 1e-7)


def test_init_from_device_tensor():
    import paper_1510_08886_gb300 as lbm
    rho = rho_field(16, 12, seed=9)
    e, w, c = lbm.dvm("D2V16")
    a = lbm.Solver(e, w, c, 3, 16, 12, 0.1, 1e-3).init(rho).step(10)
    b = lbm.Solver(e, w, c, 3, 16, 12, 0.1, 1e-3).init(torch.tensor(rho, device="cuda")).step(10)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_bitwise(precision):
    import paper_1510_08886_gb300 as lbm
    rho = rho_field(9, 20, seed=4)
    e, w, c = lbm.dvm("D2V33")
    a = lbm.Solver(e, w, c, 4, 9, 20, 0.3, 1e-3, precision=precision).init(rho).step(25)
    blob = a.get_state()
    a.step(30)
    b = lbm.Solver(e, w, c, 4, 9, 20, 0.3, 1e-3, precision=precision).set_state(blob)
    assert b.steps == 25
    assert np.array_equal(b.moments()[1], lbm.Solver(e, w, c, 4, 9, 20, 0.3, 1e-3,
                                                     precision=precision).init(rho).step(25).moments()[1])
    b.step(30)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.moments()[1], b.moments()[1])


def test_nonfinite_density_is_reported():
    """Host-injected fault: a NaN in the initial density sets the status word
    (no device trap); observables then return LBM_ENONFINITE."""
    import paper_1510_08886_gb300 as lbm
    rho = rho_field(8, 16, seed=1)
    rho[5, 3] = np.nan
    e, w, c = lbm.dvm("D2V16")
    s = lbm.Solver(e, w, c, 3, 8, 16, 0.1, 1e-3).init(rho).step(3)
    assert s.status() == lbm._lib.LBM_ENONFINITE
    with pytest.raises(lbm.LBMError):
        s.mass_flow()
    s.init(rho_field(8, 16, seed=1)).step(3)
    assert s.status() == 0


def test_not_converged_is_reported():
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V16")
    s = lbm.Solver(e, w, c, 3, 1, 32, 0.1, oracle.force_for_mach(0.1)).init()
    conv, steps, du = s.run_to_steady(1e-14, 300, check_every=100)
    assert not conv and steps == 300 and du > 1e-14


def test_stream_argument_is_used():
    """Work goes on the given stream: results equal the default-stream run."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V16")
    st = torch.cuda.Stream()
    a = lbm.Solver(e, w, c, 3, 4, 16, 0.1, 1e-3, stream=st).init().step(20)
    b = lbm.Solver(e, w, c, 3, 4, 16, 0.1, 1e-3).init().step(20)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_chunks_equal_launched_steps(precision):
    """On a non-default stream lbm_run_to_steady replays CUDA-graph chunks;
    the result is bit-identical to the step-by-step launches of the default
    stream (same kernels, same arguments), including odd chunk lengths."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V16")
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    a = lbm.Solver(e, w, c, 3, 1, 64, Kn, g, precision=precision).init()
    b = lbm.Solver(e, w, c, 3, 1, 64, Kn, g, precision=precision,
                   stream=torch.cuda.Stream()).init()
    ra = a.run_to_steady(1e-10, 50000)
    rb = b.run_to_steady(1e-10, 50000)
    assert ra == rb
    assert np.array_equal(a.populations(), b.populations())
    assert a.mass_flow() == b.mass_flow()
    a.step(3)
    b.step(3)                                  # odd number of steps: other lattice parity
    ra = a.run_to_steady(1e-14, a.steps + 351, check_every=50)
    rb = b.run_to_steady(1e-14, b.steps + 351, check_every=50)
    assert ra == rb
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("name", ["D3V96xz", "D2V16"])
def test_knudsen_layer_parity(name):
    """u_neq(y) (Eq. uNEQ) from the GPU state against the oracle's, fp64."""
    Kn = 0.05
    g = oracle.force_for_mach(Kn)
    s, ref, _ = _pair(name, 3, 2, 96, Kn, g, None)
    s.run_to_steady(1e-11, 200000)
    ref.run_to_steady(1e-11, 200000)
    un_g = s.knudsen_layer()
    un_o = ref.knudsen_layer()
    uc = ref.centre_velocity()
    assert np.max(np.abs(un_g - un_o)) < 1e-11 * uc


def test_knudsen_minimum_s3_not_s4_on_gpu():
    """Sect. VI.B/C on the GPU engine (fp32): the S3 marginal has its mass-flow
    minimum between Kn 0.7 and 1.4, the S4 marginal none up to Kn 3."""
    import paper_1510_08886_gb300 as lbm
    kns = [0.45, 0.7, 1.0, 1.4, 2.0, 3.0]
    eng = lbm.Engine("fp32", max_solves=16, arena_bytes=32 << 20)
    slots = {}
    for name in ("D3V107xz", "D3V96xz"):
        e, w, c = lbm.dvm(name)
        for Kn in kns:
            slots[(name, Kn)] = eng.add(e, w, c, 3, 1, 48, Kn, oracle.force_for_mach(Kn))
    res = eng.run(60)
    s3 = np.array([res[slots[("D3V107xz", k)], 1] for k in kns])
    s4 = np.array([res[slots[("D3V96xz", k)], 1] for k in kns])
    assert 1 <= int(np.argmin(s3)) <= 3 and s3[-1] > 1.05 * s3.min()
    assert np.all(np.diff(s4) < 0)


@pytest.mark.parametrize("name,Kn", [("D3V66xz", 0.4514), ("D3V112xz", 0.1), ("D3V112xz", 0.4514),
                                     ("D3V112xz", 1.0), ("D3V77xz", 0.1), ("D3V77xz", 0.4514),
                                     ("D3V77xz", 1.0)])
def test_marginal_models_steady_state_fp64(name, Kn):
    """(x, z) marginals of the S1 model with the smallest |sigma_zxx| (D3V66,
    Sect. VI.A: mass flow near the DSMC 1.76 at Kn = 0.4514), the scattering
    S4 model D3V112 and the augmented S3 model D3V77 (Sect. VI.B-C), run to
    max|du| < 1e-11 on the GPU in fp64: the oracle's stopping step, mass flow
    and slip velocity."""
    g = oracle.force_for_mach(Kn)
    s, ref, _ = _pair(name, 3, 1, 64, Kn, g, None)
    conv, steps, _ = s.run_to_steady(1e-11, 100000)
    conv_o, steps_o, _ = ref.run_to_steady(1e-11, 100000)
    assert conv and conv_o and steps == steps_o
    assert abs(s.mass_flow() / ref.mass_flow() - 1) < 1e-12
    assert abs(s.slip_velocity() / ref.slip_velocity() - 1) < 1e-11
    if name == "D3V66xz":
        assert abs(s.mass_flow() / 1.76 - 1) < 0.03


def test_marginal_s4_engine_kn_sweep_fp32():
    """The D3V112 (x, z) marginal (a compiled set) in the fp32 engine at
    three Kn, run to max|du| < 1e-9 (fp32 storage resolves du only to about
    1e-10): steady mass flow within 1e-4 of the fp64 oracle's steady state."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D3V112xz")
    eng = lbm.Engine("fp32", max_solves=4, arena_bytes=64 << 20)
    kns = (0.1, 0.4514, 1.0)
    slots = [eng.add(e, w, c, 3, 1, 64, Kn, oracle.force_for_mach(Kn)) for Kn in kns]
    live = dict(zip(slots, kns))
    mdot = {}
    for _ in range(1000):
        res = eng.run(1)
        for sl in [sl for sl in live if res[sl, 0] < 1e-9]:
            mdot[live.pop(sl)] = float(res[sl, 1])
            eng.remove(sl)
        if not live:
            break
    assert not live
    eng.close()
    for Kn in kns:
        ref = oracle.channel("D3V112xz", 3, 1, 64, Kn, oracle.force_for_mach(Kn)).init()
        assert ref.run_to_steady(1e-10, 100000)[0]
        assert abs(mdot[Kn] / ref.mass_flow() - 1) < 1e-4, Kn


def test_long_horizon_mass_and_rest_state_fp64():
    """50,000 forced fp64 steps with walls and a seeded density: total mass
    constant to 1e-13 relative; g = 0 at rest: fbar = w over 10,000 steps."""
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    rho = rho_field(16, 24, seed=7)
    s = lbm.Solver(e, w, c, 4, 16, 24, 0.1, oracle.force_for_mach(0.1), precision="fp64").init(rho)
    s.step(50000)
    assert abs(s.moments()[0].sum() / rho.sum() - 1) < 1e-13
    r = lbm.Solver(e, w, c, 4, 2, 16, 0.1, 0.0, precision="fp64").init().step(10000)
    f = r.populations()
    assert np.max(np.abs(f - np.asarray(w)[:, None, None])) < 1e-14
