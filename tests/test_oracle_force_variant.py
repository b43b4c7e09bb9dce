"""Reading c5 of the force term for N = 4 and its variant, in the oracle.

The paper prints the force term (Eq. nm.4) up to the third Hermite order.  The
variant adds the fourth-order term of the Hermite expansion of the force,
(1/3!) g_i a^(3)_jkl H^(4)_ijkl(xi) w, with a^(3) = rho u u u.  Pins, from the
orthogonality of the Hermite polynomials under a quadrature of degree >= 8
(D2V33, Q = 9):
* the added term has no mass, momentum, second or third moment: those
  moments of the force are the same with and without it;
* its fourth moment along any direction n is 4! / 3! rho (g.n)(u.n)^3 =
  4 rho (g.n)(u.n)^3.
In the force-driven channel at Ma ~ 1e-3 the two readings give the same mass
flow to far below the fp32 tolerance."""
import numpy as np
import pytest

import oracle


def _forces(rho, u, g, Pi):
    out = {}
    for force in ("nm4", "nm4+a3"):
        ch = oracle.channel("D2V33", 4, 3, 8, 0.1, 0.0, force=force)
        ch.p.gx, ch.p.gy = g
        out[force] = ch.force(rho, *u, Pi)
    xi = ch.c * np.stack([ch.ex, ch.ey], 1).astype(float)
    return out, xi


RHO, U, G = 0.97, np.array([0.05, -0.02]), np.array([0.013, 0.004])
PI = np.array([[1.08, 0.03], [0.03, 0.93]])


def test_added_term_has_no_low_moments():
    F, xi = _forces(RHO, U, G, PI)
    d = F["nm4+a3"] - F["nm4"]
    assert np.max(np.abs(d)) > 1e-9                     # the term is there
    assert abs(d.sum()) < 1e-17
    assert np.max(np.abs(d @ xi)) < 1e-17
    assert np.max(np.abs(np.einsum("a,ai,aj->ij", d, xi, xi))) < 1e-16
    assert np.max(np.abs(np.einsum("a,ai,aj,ak->ijk", d, xi, xi, xi))) < 1e-16


@pytest.mark.parametrize("angle", [0.0, 0.4, 1.3, 2.2])
def test_added_term_fourth_moment(angle):
    F, xi = _forces(RHO, U, G, PI)
    d = F["nm4+a3"] - F["nm4"]
    n = np.array([np.cos(angle), np.sin(angle)])
    got = d @ (xi @ n) ** 4
    want = 4.0 * RHO * (G @ n) * (U @ n) ** 3
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))


def test_channel_mass_flow_insensitive_to_variant():
    Kn = 0.1
    g = oracle.force_for_mach(Kn)
    m = {}
    for force in ("nm4", "nm4+a3"):
        ch = oracle.channel("D2V33", 4, 1, 32, Kn, g, force=force).init()
        assert ch.run_to_steady(1e-13, 100000)[0]
        m[force] = ch.mass_flow()
    assert abs(m["nm4+a3"] / m["nm4"] - 1) < 1e-12
