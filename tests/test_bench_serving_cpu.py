"""Host-side accounting of the serving section of bench.py on hand-made
request records (no GPU): the count of reference solves that met the stopping
test at the first check, and the rates over the solves that ran past it."""
import math

import bench
from paper_1510_08886_gb300.serving import Request


def _req(rid, tol, steps, t_arrival=0.0, t_done=1.0, mdot=1.0, status=0):
    r = Request(rid, t_arrival, "D2V16", 3, 1, 64, 0.1, tol)
    r.steps, r.t_done, r.mdot, r.status = steps, t_done, mdot, status
    return r


def test_first_check_stops_counts_by_tolerance():
    ref = {0: _req(0, 1e-6, 100), 1: _req(1, 1e-6, 2500), 2: _req(2, 1e-8, 100),
           3: _req(3, 1e-8, 34000), 4: _req(4, 1e-8, 41000), 5: _req(5, 1e-6, 100, status=1)}
    out = bench._first_check_stops(ref)
    assert out["check_steps"] == 100
    assert out["stopped"] == 2 and out["of"] == 5            # the failed solve is left out
    assert out["by_tol"] == {"tol_1e-06": {"stopped": 1, "of": 2},
                             "tol_1e-08": {"stopped": 1, "of": 3}}


def test_beyond_first_check_rates_and_gate():
    ref = {i: _req(i, 1e-6, s) for i, s in enumerate([100, 200, 300, 400])}
    done = {i: _req(i, 1e-6, s, t_arrival=0.0, t_done=float(i + 1))
            for i, s in enumerate([100, 200, 300, 400])}
    # without the gate: requests 1, 2, 3 ran past the first check
    out = bench._beyond_first_check(done, ref, wall=2.0)
    assert out["requests"] == 3 and out["solves_per_s"] == 1.5
    assert out["p50_s"] == 3.0
    # with the gate: request 2 fails it, request 5 has no reference
    errs = {0: 0.0, 1: 5e-5, 2: 2e-4, 3: 1e-4}
    done[5] = _req(5, 1e-6, 500)
    out = bench._beyond_first_check(done, ref, wall=2.0, errs=errs)
    assert out["requests"] == 2 and out["solves_per_s"] == 1.0
    assert math.isclose(out["p99_s"], 2.0 + 0.99 * 2.0)


def test_beyond_first_check_empty():
    out = bench._beyond_first_check({}, {}, wall=1.0)
    assert out["requests"] == 0 and out["solves_per_s"] == 0.0 and math.isnan(out["p50_s"])


def test_first_check_du_is_the_bulk_acceleration():
    """Why tol = 1e-6 requests can stop at the first check: the walls reach at
    most max|e_y| rows per step, so after 100 steps the centre of a channel of
    more than 2 x 300 rows is still uniform bulk, accelerating by exactly g dt
    per step (dt = 1/(Ny c)), and max|du| there is g dt.  On the oracle,
    D2V16, N = 3."""
    import numpy as np
    import oracle
    from lbm_inputs.tables import DVM_TABLES
    c = DVM_TABLES["D2V16"]["c"]
    for Ny, Kn in ((768, 0.02), (1024, 0.3)):
        g = oracle.force_for_mach(Kn)
        ch = oracle.channel("D2V16", 3, 1, Ny, Kn, g)
        ch.init()
        ch.step(99)
        u0 = ch.moments()[1].copy()
        ch.step(1)
        du = np.abs(ch.moments()[1] - u0)
        mid = du.reshape(Ny)[Ny // 2]
        assert abs(mid / (g / (Ny * c)) - 1) < 1e-9
        assert abs(du.max() / (g / (Ny * c)) - 1) < 1e-9
