"""The two readings of the diffuse wall in fbar variables (Sect. V, Eq. nm.14
with Eq. nm.7), in the oracle:

* plain (the reading used everywhere): the unknown fbar_a = Psi rho_w w_a;
* transformed: the wall condition holds for f, and fbar_a = f_a + (dt/2 tau)
  (f_a - f0_a(rho, u)) with the node's own moments (fixed point per node).

At rest both leave the equilibrium unchanged.  In the force-driven channel
their steady mass flows (Eq. pf.1) differ at first order in dt / tau and
approach the same limit as Ny grows; the plain reading conserves mass to
rounding and is already close to that limit at coarse resolution."""
import numpy as np
import pytest

import oracle


def test_transformed_wall_keeps_rest_state():
    ch = oracle.channel("D2V16", 3, 3, 12, 0.2, 0.0, wall="transformed").init()
    ch.step(300)
    assert np.max(np.abs(ch.f - ch.w[:, None, None])) < 1e-14


def _steady(Ny, wall, Kn=0.1):
    g = oracle.force_for_mach(Kn)
    ch = oracle.channel("D2V16", 3, 1, Ny, Kn, g, wall=wall).init()
    conv, _, _ = ch.run_to_steady(1e-13, 100000)
    assert conv
    return ch.mass_flow(), float(ch.f.sum())


@pytest.fixture(scope="module")
def flows():
    return {(Ny, wall): _steady(Ny, wall) for Ny in (16, 32, 64)
            for wall in ("plain", "transformed")}


def test_readings_differ_at_first_order(flows):
    d = [abs(flows[(Ny, "transformed")][0] / flows[(Ny, "plain")][0] - 1) for Ny in (16, 32, 64)]
    # halving dt halves the difference (first order in dt / tau)
    assert 1.7 < d[0] / d[1] < 2.3 and 1.7 < d[1] / d[2] < 2.3
    assert d[2] < 0.06


def test_plain_reading_conserves_mass_and_resolves_early(flows):
    for Ny in (16, 32, 64):
        assert abs(flows[(Ny, "plain")][1] / Ny - 1) < 1e-12
    step_plain = abs(flows[(64, "plain")][0] / flows[(32, "plain")][0] - 1)
    step_transformed = abs(flows[(64, "transformed")][0] / flows[(32, "transformed")][0] - 1)
    assert step_plain < 0.1 * step_transformed
