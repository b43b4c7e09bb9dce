"""Multi-solve engine: batched channels of uneven sizes and different velocity
sets in one persistent launch per set, CUDA-graph chunks, admission by arena
footprint, continuous add/remove.

Key property: a solve's arithmetic does not depend on the other solves in
the engine -- results alone and in the mix are bit-identical, and identical
to the single-solve API (same per-node code, deterministic per-solve
reductions)."""
import numpy as np
import pytest

import oracle
from lbm_inputs import batch_workload, rho_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build_library()


MIX = [("D2V33", 4, 256, 40, 0.05), ("D3V107xz", 3, 64, 33, 0.3), ("D2V33", 4, 1, 77, 1.0),
       ("D2V16", 3, 1, 64, 0.1), ("D3V107xz", 3, 256, 20, 0.01), ("D2V32", 3, 5, 30, 0.2),
       ("D2V33", 4, 64, 129, 0.5), ("D3V96xz", 3, 17, 14, 0.7)]


def _add(eng, spec, seed):
    import paper_1510_08886_gb300 as lbm
    name, N, Nx, Ny, Kn = spec
    e, w, c = lbm.dvm(name)
    return eng.add(e, w, c, N, Nx, Ny, Kn, oracle.force_for_mach(Kn, 1e-2),
                   rho=rho_field(Nx, Ny, seed=seed))


def test_alone_vs_mix_bitwise_and_vs_single_solver():
    import paper_1510_08886_gb300 as lbm
    mix = lbm.Engine("fp32", max_solves=16, arena_bytes=256 << 20, chunk=50)
    slots = [_add(mix, s, seed=i + 1) for i, s in enumerate(MIX)]
    res_mix = mix.run(2).copy()
    for i, spec in enumerate(MIX):
        name, N, Nx, Ny, Kn = spec
        alone = lbm.Engine("fp32", max_solves=2, arena_bytes=64 << 20, chunk=50)
        s = _add(alone, spec, seed=i + 1)
        res_alone = alone.run(2)
        m_mix = mix.moments(slots[i], Nx, Ny)
        m_alone = alone.moments(s, Nx, Ny)
        for a, b in zip(m_mix, m_alone):
            assert np.array_equal(a, b)
        assert np.array_equal(res_mix[slots[i]], res_alone[s])
        # the single-solve API runs the same arithmetic
        e, w, c = lbm.dvm(name)
        single = lbm.Solver(e, w, c, N, Nx, Ny, Kn, oracle.force_for_mach(Kn, 1e-2),
                            precision="fp32").init(rho_field(Nx, Ny, seed=i + 1)).step(100)
        r, ux, uy = single.moments()
        assert np.max(np.abs(ux - m_mix[1])) <= 1e-6 * np.max(np.abs(ux))
        assert np.max(np.abs(r - m_mix[0])) <= 1e-6
        alone.close()
        assert mix.info(slots[i], status=True) == (100, 0)


def test_engine_vs_oracle_steady_state():
    """Config-1 channel run to steady state inside a busy engine."""
    import paper_1510_08886_gb300 as lbm
    eng = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20)
    others = [_add(eng, s, seed=5) for s in MIX[:3]]
    e, w, c = lbm.dvm("D2V16")
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    slot = eng.add(e, w, c, 3, 1, 64, Kn, g)
    for _ in range(100):
        res = eng.run(1)
        if res[slot, 0] < 1e-10:
            break
    assert res[slot, 0] < 1e-10
    ref = oracle.channel("D2V16", 3, 1, 64, Kn, g).init()
    ref.run_to_steady(1e-10, 50000)
    assert abs(res[slot, 1] / ref.mass_flow() - 1) < 1e-4
    assert abs(res[slot, 2] / ref.slip_velocity() - 1) < 1e-4
    assert abs(res[slot, 3] / ref.mean_ux() - 1) < 1e-4
    assert len(others) == 3


def test_admission_by_footprint_and_reuse():
    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    per = lbm.Engine.solve_bytes(e, w, c, 256, 256, "fp32")
    eng = lbm.Engine("fp32", max_solves=64, arena_bytes=3 * per + (8 << 20))
    free0 = eng.free_bytes()
    slots = []
    while True:
        s = eng.add(e, w, c, 4, 256, 256, 0.1, 1e-3)
        if s is None:
            break
        slots.append(s)
    assert len(slots) >= 3
    eng.run(1)
    eng.remove(slots[1])
    s = eng.add(e, w, c, 4, 256, 256, 0.1, 1e-3)
    assert s is not None
    assert eng.add(e, w, c, 4, 256, 256, 0.1, 1e-3) is None
    for x in slots[:1] + slots[2:] + [s]:
        eng.remove(x)
    assert eng.free_bytes() == free0


def test_remove_then_add_does_not_disturb_others():
    import paper_1510_08886_gb300 as lbm
    a = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=20)
    b = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=20)
    keep_a = _add(a, MIX[0], seed=3)
    keep_b = _add(b, MIX[0], seed=3)
    tmp = _add(a, MIX[1], seed=4)
    a.run(1)
    b.run(1)
    a.remove(tmp)
    _add(a, MIX[5], seed=9)
    a.run(2)
    b.run(2)
    Nx, Ny = MIX[0][2], MIX[0][3]
    assert np.array_equal(a.moments(keep_a, Nx, Ny)[1], b.moments(keep_b, Nx, Ny)[1])


def test_autotune_keeps_results_exact():
    """Autotuning changes launch shapes only: after it, a solve still equals
    a reference engine advanced by the same number of steps."""
    import paper_1510_08886_gb300 as lbm
    a = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=10)
    b = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=10)
    sa = [_add(a, s, seed=7) for s in MIX[:4]]
    sb = [_add(b, s, seed=7) for s in MIX[:4]]
    ms = a.autotune()
    assert ms > 0
    steps = a.info(sa[0])[0]
    # two tiled groups (D2V33 N=4 at 256 x 40, D3V107xz N=3 at 64 x 33; the
    # one-column channels are resident): the current schedule, 10 more shapes
    # for both groups, per group 10 more shapes and 4 more grabs, then the
    # other grid fraction; 3 chunks of 10 steps each
    assert steps == (12 + 14 * 2) * 3 * 10
    for slot in sa:
        sched = a.schedule(slot)
        assert sched["tile_width"] in (0, 32, 64, 128) and sched["tile_cells"] in (128, 256, 512)
        assert sched["grab"] in (1, 2, 4, 8, 16) and sched["grid_fraction"] in (0.5, 1.0)
    a.run(1)
    b.run(steps // 10 + 1)
    for x, y, spec in zip(sa, sb, MIX[:4]):
        assert np.array_equal(a.moments(x, spec[2], spec[3])[1], b.moments(y, spec[2], spec[3])[1])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_16bit_engine_close_to_fp32(precision):
    import paper_1510_08886_gb300 as lbm
    e32 = lbm.Engine("fp32", max_solves=4, arena_bytes=64 << 20)
    e16 = lbm.Engine(precision, max_solves=4, arena_bytes=64 << 20)
    s32 = _add(e32, MIX[0], seed=2)
    s16 = _add(e16, MIX[0], seed=2)
    e32.run(2)
    e16.run(2)
    Nx, Ny = MIX[0][2], MIX[0][3]
    u32 = e32.moments(s32, Nx, Ny)[1]
    u16 = e16.moments(s16, Nx, Ny)[1]
    tol = 2e-3 if precision == "fp16" else 2e-2
    assert np.max(np.abs(u16 - u32)) < tol * np.max(np.abs(u32))


def test_config4_workload_runs():
    """The 256-channel config-4 list (seeded) fits, runs, and every solve
    stays finite with a positive mass flow."""
    import paper_1510_08886_gb300 as lbm
    work = batch_workload(256)
    need = sum(lbm.Engine.solve_bytes(*lbm.dvm(it["dvm"]), it["Nx"], it["Ny"], "fp32")
               for it in work)
    eng = lbm.Engine("fp32", max_solves=256, arena_bytes=need + (64 << 20), chunk=20)
    slots = []
    for it in work:
        e, w, c = lbm.dvm(it["dvm"])
        s = eng.add(e, w, c, it["order"], it["Nx"], it["Ny"], it["Kn"],
                    oracle.force_for_mach(it["Kn"]))
        assert s is not None
        slots.append(s)
    res = eng.run(2)
    for s in slots:
        assert eng.info(s, status=True)[1] == 0
        assert res[s, 1] > 0 and np.isfinite(res[s, 1])


# Channels for the resident-chunk path: x wrap by constant offset (Nx = 1),
# by one compare (Nx >= max|e_x|) and by a modulo (1 < Nx < max|e_x|); the
# narrowest channel (Ny = max|e_y|); the largest bundle entry (4096 nodes
# would not fit 227 KB for D2V16 fp32, 2048 does); one over the node limit
# (tiled in both engines); more small channels than one bundle holds.
RESIDENT_MIX = ([("D2V16", 3, 1, 2048, 0.02), ("D2V16", 3, 1, 4, 0.5), ("D2V33", 4, 3, 21, 0.1),
                 ("D2V32", 3, 5, 12, 0.3), ("D3V96xz", 3, 17, 14, 0.7), ("D2V33", 4, 64, 31, 0.05),
                 ("D3V107xz", 3, 2, 19, 0.2), ("D2V16", 2, 1, 5000, 0.1), ("D2V33", 2, 1, 9, 1.0)]
                + [("D2V16", 3, 1, 16 + (i % 7), 0.01 * (1 + i)) for i in range(70)])


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp64"])
def test_resident_chunks_bitwise_equal_tiled(precision):
    """A whole chunk in shared memory (two-step in-place streaming, ghost
    rows at the walls) gives bitwise the per-step tiled kernel's states,
    observables and status, also after slots are removed and added."""
    import paper_1510_08886_gb300 as lbm
    engines = [lbm.Engine(precision, max_solves=96, arena_bytes=256 << 20, chunk=20,
                          resident=r) for r in (True, False)]
    slots = [[_add(eng, s, seed=11 + i) for i, s in enumerate(RESIDENT_MIX)] for eng in engines]
    # resident when V Nx (Ny + 2 max|e_y|) elements fit the block's shared
    # memory (the opt-in limit less 4 KiB, 256-byte granules) and the padded
    # node count is at most 4096 (include/lbm.h, lbm_engine_set_resident)
    cap = (torch.cuda.get_device_properties(0).shared_memory_per_block_optin - 4096) & ~255
    es = {"fp32": 4, "fp16": 2, "bf16": 2, "fp64": 8}[precision]
    n_res = 0
    for name, N, Nx, Ny, Kn in RESIDENT_MIX:
        e, w, c = lbm.dvm(name)
        G = int(np.max(np.abs(np.asarray(e)[:, 1])))
        n_res += len(w) * Nx * (Ny + 2 * G) * es <= cap and ((Nx * Ny + 31) & ~31) <= 4096
    assert 0 < n_res < len(RESIDENT_MIX)
    assert engines[0].paths() == (len(RESIDENT_MIX) - n_res, n_res)
    assert engines[1].paths() == (len(RESIDENT_MIX), 0)
    res = [eng.run(2).copy() for eng in engines]

    def compare(live):
        for i in live:
            Nx, Ny = RESIDENT_MIX[i][2], RESIDENT_MIX[i][3]
            ma = engines[0].moments(slots[0][i], Nx, Ny)
            mb = engines[1].moments(slots[1][i], Nx, Ny)
            for a, b in zip(ma, mb):
                assert np.array_equal(a, b), (i, RESIDENT_MIX[i])
            assert np.array_equal(res[0][slots[0][i]], res[1][slots[1][i]]), i
            assert engines[0].info(slots[0][i], status=True) == engines[1].info(slots[1][i],
                                                                                status=True)

    live = list(range(len(RESIDENT_MIX)))
    compare(live)
    for eng, sl in zip(engines, slots):
        for i in (0, 3, 20, 40):
            eng.remove(sl[i])
    live = [i for i in live if i not in (0, 3, 20, 40)]
    extra = ("D2V33", 4, 7, 40, 0.08)
    xs = [_add(eng, extra, seed=99) for eng in engines]
    res = [eng.run(1).copy() for eng in engines]
    compare(live)
    for a, b in zip(engines[0].moments(xs[0], 7, 40), engines[1].moments(xs[1], 7, 40)):
        assert np.array_equal(a, b)
    for eng in engines:
        eng.close()


def test_resident_switch_validates():
    import paper_1510_08886_gb300 as lbm
    eng = lbm.Engine("fp32", max_solves=2, arena_bytes=16 << 20)
    from paper_1510_08886_gb300 import _lib
    assert _lib.lib().lbm_engine_set_resident(eng._h, 2) == _lib.LBM_EINVAL
    eng.set_resident(False)
    eng.set_resident(True)
    eng.close()


def test_engine_checkpoint_restores_bitwise():
    """A slot's checkpoint restored into another engine's slot continues
    bit-identically (fp32); a checkpoint of a different solve is refused."""
    import paper_1510_08886_gb300 as lbm
    from paper_1510_08886_gb300 import _lib
    spec = ("D2V33", 4, 16, 24, 0.2)
    a = lbm.Engine("fp32", max_solves=4, arena_bytes=64 << 20, chunk=10)
    sa = _add(a, spec, seed=21)
    a.run(3)
    ck = a.get_state(sa)
    a.run(2)
    b = lbm.Engine("fp32", max_solves=4, arena_bytes=64 << 20, chunk=10, resident=False)
    _add(b, MIX[1], seed=1)                   # another solve first: a different slot
    sb = _add(b, spec, seed=99)                # different initial state, same solve
    b.set_state(sb, ck)
    assert b.info(sb)[0] == 30
    b.run(2)
    for x, y in zip(a.moments(sa, 16, 24), b.moments(sb, 16, 24)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.get_state(sa)[64:], b.get_state(sb)[64:])
    other = _add(b, ("D2V33", 4, 16, 25, 0.2), seed=3)
    with pytest.raises(RuntimeError):
        b.set_state(other, ck)
    bad = ck.copy()
    bad[:8] = 0
    assert _lib.lib().lbm_engine_set_state(b._h, sb, bad.ctypes.data_as(_lib.ctypes.c_void_p),
                                           bad.nbytes) == _lib.LBM_EINVAL
    a.close()
    b.close()


def test_launch_wait_equals_run():
    """Asynchronous chunks give the results of the synchronous ones, chunk
    by chunk; run, autotune and a third launch are refused while launches
    are outstanding; a solve removed between launch and wait still gets the
    queued chunk."""
    import paper_1510_08886_gb300 as lbm
    from paper_1510_08886_gb300 import _lib
    a = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=10)
    b = lbm.Engine("fp32", max_solves=8, arena_bytes=128 << 20, chunk=10)
    sa = [_add(a, s, seed=41 + i) for i, s in enumerate(MIX[:5])]
    sb = [_add(b, s, seed=41 + i) for i, s in enumerate(MIX[:5])]
    ra = [a.run(1).copy() for _ in range(3)]
    b.launch(1)
    b.launch(1)
    assert _lib.lib().lbm_engine_launch(b._h, 1) == _lib.LBM_EINVAL
    assert _lib.lib().lbm_engine_run(b._h, 1, None) == _lib.LBM_EINVAL
    assert _lib.lib().lbm_engine_autotune(b._h, None) == _lib.LBM_EINVAL
    rb = [b.wait().copy()]
    b.launch(1)
    rb += [b.wait().copy(), b.wait().copy()]
    assert _lib.lib().lbm_engine_wait(b._h, None) == _lib.LBM_EINVAL
    for x, y in zip(ra, rb):
        for s1, s2 in zip(sa, sb):
            assert np.array_equal(x[s1], y[s2])
    # removal between launch and wait: the removed solve's result is that chunk's
    a.run(1)
    b.launch(1)
    b.remove(sb[0])
    rb4 = b.wait().copy()
    ra4 = a.results.copy()
    assert np.array_equal(ra4[sa[0]], rb4[sb[0]])
    a.close()
    b.close()


def test_fp64_engine_equals_single_solver():
    """fp64 storage and arithmetic in the engine: every solve of the mix
    (tiled and resident, all compiled velocity sets) matches the fp64
    single-solve API within fp64 rounding, and alone equals in the mix bit
    for bit."""
    import paper_1510_08886_gb300 as lbm
    mix = lbm.Engine("fp64", max_solves=16, arena_bytes=512 << 20, chunk=50)
    slots = [_add(mix, s, seed=i + 1) for i, s in enumerate(MIX)]
    assert sum(mix.paths()) == len(MIX) and mix.paths()[1] > 0
    res_mix = mix.run(2).copy()
    for i, spec in enumerate(MIX):
        name, N, Nx, Ny, Kn = spec
        alone = lbm.Engine("fp64", max_solves=2, arena_bytes=128 << 20, chunk=50)
        s = _add(alone, spec, seed=i + 1)
        res_alone = alone.run(2)
        m_mix = mix.moments(slots[i], Nx, Ny)
        for a, b in zip(m_mix, alone.moments(s, Nx, Ny)):
            assert np.array_equal(a, b)
        assert np.array_equal(res_mix[slots[i]], res_alone[s])
        alone.close()
        e, w, c = lbm.dvm(name)
        single = lbm.Solver(e, w, c, N, Nx, Ny, Kn, oracle.force_for_mach(Kn, 1e-2),
                            precision="fp64").init(rho_field(Nx, Ny, seed=i + 1)).step(100)
        r, ux, uy = single.moments()
        assert np.max(np.abs(ux - m_mix[1])) <= 1e-12 * np.max(np.abs(ux)), spec
        assert np.max(np.abs(r - m_mix[0])) <= 1e-13, spec
        assert abs(res_mix[slots[i], 1] / single.mass_flow() - 1) < 1e-12, spec
    mix.close()


def test_fp64_engine_stops_with_the_oracle():
    """Config-1 channel to max|du| < 1e-10 in a busy fp64 engine: the same
    stopping chunk as the oracle's run_to_steady and its mass flow to 1e-12."""
    import paper_1510_08886_gb300 as lbm
    eng = lbm.Engine("fp64", max_solves=8, arena_bytes=256 << 20)
    for s in MIX[:3]:
        _add(eng, s, seed=5)
    e, w, c = lbm.dvm("D2V16")
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    slot = eng.add(e, w, c, 3, 1, 64, Kn, g)
    for _ in range(500):
        res = eng.run(1)
        if res[slot, 0] < 1e-10:
            break
    assert res[slot, 0] < 1e-10
    ref = oracle.channel("D2V16", 3, 1, 64, Kn, g).init()
    conv, steps, _ = ref.run_to_steady(1e-10, 50000)
    assert conv and eng.info(slot)[0] == steps
    assert abs(res[slot, 1] / ref.mass_flow() - 1) < 1e-12
    assert abs(res[slot, 2] / ref.slip_velocity() - 1) < 1e-11
    eng.close()


SCHEDULE_MIX = [("D2V33", 4, 256, 40, 0.05), ("D3V107xz", 3, 64, 33, 0.3), ("D2V33", 4, 128, 9, 0.2),
                ("D2V16", 3, 1, 64, 0.1), ("D3V107xz", 3, 256, 20, 0.01), ("D2V32", 3, 5, 30, 0.2),
                ("D2V33", 4, 64, 129, 0.5), ("D3V96xz", 3, 96, 14, 0.7), ("D2V33", 4, 32, 300, 1.0)]
SCHEDULES = [(0, 128, 4, 1.0), (0, 512, 1, 0.5), (32, 128, 2, 1.0), (32, 512, 8, 1.0),
             (64, 256, 1, 1.0), (64, 512, 4, 0.5), (128, 256, 16, 1.0), (128, 512, 3, 1.0)]


@pytest.mark.parametrize("precision", ["fp32", "fp16", "fp64"])
def test_schedules_bitwise_equal(precision):
    """Tile shape, cells per tile, grab and grid only decide which block
    updates a node: every schedule gives bitwise the same states, observables
    and status.  The mix has channels that take 2-D tiles (Nx a multiple of
    the width, Ny clipped by the tile's rows or not), channels that fall back
    to linear tiles (Nx = 1, 5; Ny below the tile's rows), tall and short."""
    import paper_1510_08886_gb300 as lbm
    engines, slots = [], []
    for tw, tc, grab, frac in SCHEDULES:
        eng = lbm.Engine(precision, max_solves=16, arena_bytes=128 << 20, chunk=20, resident=False)
        sl = [_add(eng, s, seed=31 + i) for i, s in enumerate(SCHEDULE_MIX)]
        eng.set_schedule(tw, tc, grab, frac)
        # per group: the first D2V33 solve's group also takes a second schedule
        other = SCHEDULES[(SCHEDULES.index((tw, tc, grab, frac)) + 3) % len(SCHEDULES)]
        eng.set_schedule(*other[:3], frac, slot=sl[0])
        for i in range(len(sl)):
            want = other[:3] if SCHEDULE_MIX[i][:2] == ("D2V33", 4) else (tw, tc, grab)
            assert eng.schedule(sl[i]) == {"tile_width": want[0], "tile_cells": want[1],
                                           "grab": want[2], "grid_fraction": frac}
        slots.append(sl)
        engines.append(eng)
    res = [eng.run(2).copy() for eng in engines]
    for j in range(1, len(engines)):
        for i, (name, N, Nx, Ny, Kn) in enumerate(SCHEDULE_MIX):
            ma = engines[0].moments(slots[0][i], Nx, Ny)
            mb = engines[j].moments(slots[j][i], Nx, Ny)
            for a, b in zip(ma, mb):
                assert np.array_equal(a, b), (SCHEDULES[j], SCHEDULE_MIX[i])
            assert np.array_equal(res[0][slots[0][i]], res[j][slots[j][i]])
            assert engines[0].info(slots[0][i], status=True) == engines[j].info(slots[j][i],
                                                                                status=True)
            assert np.array_equal(engines[0].get_state(slots[0][i]), engines[j].get_state(slots[j][i]))
    for eng in engines:
        eng.close()


def test_schedule_validates():
    import paper_1510_08886_gb300 as lbm
    eng = lbm.Engine("fp32", max_solves=2, arena_bytes=16 << 20)
    for bad in [(16, 128, 4, 1.0), (32, 64, 4, 1.0), (32, 1024, 4, 1.0), (0, 128, 0, 1.0),
                (0, 128, 65, 1.0), (0, 128, 4, 0.0), (0, 128, 4, 1.5)]:
        with pytest.raises(lbm.LBMError):
            eng.set_schedule(*bad)
    # a slot must be in use
    with pytest.raises(lbm.LBMError):
        eng.set_schedule(0, 128, 4, 1.0, slot=0)
    with pytest.raises(lbm.LBMError):
        eng.schedule(1)
    s = _add(eng, ("D2V16", 3, 1, 64, 0.1), seed=1)
    eng.set_schedule(32, 256, 2, 0.5, slot=s)
    assert eng.schedule(s) == {"tile_width": 32, "tile_cells": 256, "grab": 2, "grid_fraction": 0.5}
    eng.close()
