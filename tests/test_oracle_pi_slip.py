"""Pins of two oracle parts that the other CPU tests leave free:

* the momentum flux Pi of f that enters the force term of Eq. nm.4 (step (3)
  of the oracle's collision: Pi of f = (2 tau Pibar + dt Pi_eq) / (2 tau + dt),
  Eq. nm.7 inverted).  The second moment of F does not depend on Pi, but its
  third moment does: for a quadrature of degree >= 6 the Hermite expansion of
  Eq. nm.4 gives  sum_a F_a xi_i xi_j xi_k = g_i Pi_jk + g_j Pi_ik + g_k Pi_ij,
  and the equilibrium's third moment is rho (u u u + sym(u delta)) (Eq. ce.13).
  So the post-collision third moment of Eq. nm.8 is fixed in closed form by
  the pre-collision moments alone;
* the slip velocity u_s = u(wall) / u(centre) of Eq. defSlip with the
  quadratic wall extrapolation and the centre interpolation, both exact for a
  profile a + b (1 - 4 z^2): u_s = a / (a + b), u(centre) = a + b.

Each pin is shown to fail under the plausible mistakes it guards against,
planted in a CPU copy of the oracle (never in the library).
"""
import inspect
import os
import shutil
import subprocess
import textwrap

import numpy as np
import pytest

import oracle
from lbm_inputs import DVM_TABLES
from oracle import dvm

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.join(os.path.dirname(HERE), "oracle")

SETS = [("D2V16", 3), ("D2V33", 4), ("D2V32", 3), ("D3V107xz", 3), ("D2V16", 4),
        ("D2V33", 3), ("D2V16", 2)]

# ---------------------------------------------------------------------------
# Pi of f: the third moment of the collision


def _chan(name, N, g=(0.3, -0.2), Kn=0.05, Nx=2, Ny=8):
    e, w, c = dvm.dvm2d(name, DVM_TABLES)
    return oracle.Channel(e, w, c, N, Nx, Ny, Kn, g[0], gy=g[1])


def _third_moment_prediction(ch, f, Pi_kind="f"):
    """Post-collision third moments per node from the pre-collision state:
    (1 - omega) M3(fbar) + omega [M3(f0) + tau M3(F)], with
    M3(f0) = rho (u u u + sym(u delta)) for N >= 3 (rho sym(u delta) for N = 2),
    M3(F) = sym3(g Pi) for N >= 3 (rho sym3(g delta) for N = 2) and
    Pi = (2 tau Pibar + dt Pi_eq) / (2 tau + dt),
    Pi_eq = rho (delta + u u + tau (g u + u g)).
    Pi_kind "bar" / "no_eq" give the predictions of the two mistaken forms
    (Pi = Pibar; Pi = 2 tau Pibar / (2 tau + dt))."""
    xi = ch.c * np.stack([ch.ex, ch.ey], 1).astype(float)
    g = np.array([ch.p.gx, ch.p.gy])
    tau, dt, om = ch.tau, ch.dt, ch.omega
    d = np.eye(2)
    out = np.empty((ch.Ny, ch.Nx, 2, 2, 2))
    for y in range(ch.Ny):
        for x in range(ch.Nx):
            fa = f[:, y, x]
            rho = fa.sum()
            u = (fa @ xi + 0.5 * dt * rho * g) / rho          # Eq. nm.10
            Pbar = np.einsum("a,ai,aj->ij", fa, xi, xi)
            M3 = np.einsum("a,ai,aj,ak->ijk", fa, xi, xi, xi)
            Peq = rho * (d + np.outer(u, u) + tau * (np.outer(g, u) + np.outer(u, g)))
            if Pi_kind == "f":
                Pi = (2 * tau * Pbar + dt * Peq) / (2 * tau + dt)
            elif Pi_kind == "bar":
                Pi = Pbar
            else:
                Pi = 2 * tau * Pbar / (2 * tau + dt)
            if ch.N < 3:
                Pi = rho * d                   # no third-order force term
            M0 = np.einsum("i,jk->ijk", rho * u, d)
            sym_ud = M0 + M0.transpose(1, 0, 2) + M0.transpose(1, 2, 0)
            f0_3 = sym_ud + (rho * np.einsum("i,j,k->ijk", u, u, u) if ch.N >= 3 else 0.0)
            G = np.einsum("i,jk->ijk", g, Pi)
            F_3 = G + G.transpose(1, 0, 2) + G.transpose(1, 2, 0)
            out[y, x] = (1 - om) * M3 + om * (f0_3 + tau * F_3)
    return out


def _third_moment(ch, f):
    xi = ch.c * np.stack([ch.ex, ch.ey], 1).astype(float)
    return np.einsum("ayx,ai,aj,ak->yxijk", f, xi, xi, xi)


def _random_far_state(ch, seed):
    """Populations far from equilibrium, so Pibar - Pi_eq is O(1)."""
    rng = np.random.default_rng(seed)
    return ch.w[:, None, None] * (1 + 0.3 * rng.standard_normal((ch.V, ch.Ny, ch.Nx)))


@pytest.mark.parametrize("name,N", SETS)
def test_collision_third_moment_closed_form(name, N):
    ch = _chan(name, N)
    assert dvm.quadrature_order(np.stack([ch.ex, ch.ey], 1), ch.w, ch.c) >= 6
    f = _random_far_state(ch, 11)
    got = _third_moment(ch, ch.collide(f))
    ref = _third_moment_prediction(ch, f)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < 1e-13 * scale
    if N >= 3:
        # the closed form separates the readings: Pibar or a dropped dt Pi_eq
        # move the third moment by far more than the tolerance
        for kind in ("bar", "no_eq"):
            alt = _third_moment_prediction(ch, f, kind)
            assert np.max(np.abs(alt - ref)) > 1e-6 * scale


def _mutant_oracle(tmp_path, old, new):
    """Build a copy of the C oracle with one planted change; returns its path."""
    src = open(os.path.join(ORACLE_DIR, "lbm_oracle.c")).read()
    assert src.count(old) == 1, old
    d = tmp_path / "mut"
    d.mkdir()
    (d / "lbm_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE_DIR, "lbm_oracle.h"), d / "lbm_oracle.h")
    lib = str(d / "libmut.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", lib, str(d / "lbm_oracle.c"), "-lm"])
    return lib


PI_LINE = "double fa = (2.0 * tau * fin[a] + dt * feq) / (2.0 * tau + dt);"
PI_SLIPS = {
    "Pibar in place of Pi of f": "double fa = fin[a]; (void)feq;",
    "dt Pi_eq term dropped": "double fa = (2.0 * tau * fin[a]) / (2.0 * tau + dt); (void)feq;",
    "tau and dt swapped": "double fa = (2.0 * dt * fin[a] + tau * feq) / (2.0 * dt + tau);",
}


@pytest.mark.parametrize("slip", sorted(PI_SLIPS))
def test_third_moment_pin_catches_planted_pi_slips(slip, tmp_path, monkeypatch):
    lib = _mutant_oracle(tmp_path, PI_LINE, PI_SLIPS[slip])
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: lib)
    for name, N in [("D2V16", 3), ("D2V33", 4)]:
        ch = _chan(name, N)
        f = _random_far_state(ch, 11)
        got = _third_moment(ch, ch.collide(f))
        ref = _third_moment_prediction(ch, f)
        # the planted slip breaks the pin
        assert np.max(np.abs(got - ref)) > 1e-6 * np.max(np.abs(ref))
        # and leaves the mass and momentum checks of the other pins intact
        fs = ch.collide(f)
        assert np.allclose(fs.sum(0), f.sum(0), rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# slip velocity and centre velocity (Eq. defSlip)


def _quadratic_state(ch, a, b, seed=3):
    """fbar_a = w_a (1 + xi_a . v) with v_x = a + b (1 - 4 z^2) + p(x),
    v_y = 0, p a column pattern of zero mean.  With g = 0 this gives rho = 1
    and u_x = v_x exactly (sum w xi = 0, sum w xi xi = delta)."""
    rng = np.random.default_rng(seed)
    z = (np.arange(ch.Ny) + 0.5) / ch.Ny - 0.5
    p = rng.standard_normal(ch.Nx) * 0.2 * b
    p -= p.mean()
    vx = a + b * (1 - 4 * z ** 2)[:, None] + p[None, :]
    xi_x = ch.c * ch.ex.astype(float)
    return ch.w[:, None, None] * (1 + xi_x[:, None, None] * vx[None, :, :])


SLIP_SHAPES = [(1, 9), (1, 10), (3, 16), (4, 17), (2, 64), (5, 33)]


@pytest.mark.parametrize("Nx,Ny", SLIP_SHAPES)
@pytest.mark.parametrize("name", ["D2V16", "D2V33"])
def test_slip_velocity_exact_on_quadratic_profile(name, Nx, Ny):
    e, w, c = dvm.dvm2d(name, DVM_TABLES)
    ch = oracle.Channel(e, w, c, 3, Nx, Ny, 0.1, 0.0)
    a, b = 3e-4, 1e-3
    ch.f[:] = _quadratic_state(ch, a, b)
    # u_x = sum fbar xi_x cancels O(1) terms down to O(1e-3): ~1e-13 relative
    assert abs(ch.centre_velocity() - (a + b)) < 1e-11 * (a + b)
    assert abs(ch.slip_velocity() - a / (a + b)) < 1e-10 * a / (a + b)
    # midpoint rule of Eq. pf.1: mean of (2 z_j)^2 over the nodes is (1 - 1/Ny^2)/3
    assert abs(ch.mean_ux() - (a + b * (1 - (1 - 1 / Ny ** 2) / 3))) < 1e-14


def _mutant_channel(old, new):
    """A Channel whose slip_velocity / centre_velocity carry one planted change."""
    cls_src = textwrap.dedent(inspect.getsource(oracle.Channel))
    assert cls_src.count(old) >= 1, old
    ns = dict(vars(oracle))
    exec(compile(cls_src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["Channel"]


SLIP_SLIPS = {
    "linear wall extrapolation": ("(15.0 * u[0] - 10.0 * u[1] + 3.0 * u[2]) / 8.0",
                                  "(3.0 * u[0] - u[1]) / 2.0"),
    "wall value at the first node": ("(15.0 * u[0] - 10.0 * u[1] + 3.0 * u[2]) / 8.0", "u[0]"),
    "two-point centre for even Ny": ("(9.0 * (u[m - 1] + u[m]) - (u[m - 2] + u[m + 1])) / 16.0",
                                     "(u[m - 1] + u[m]) / 2.0"),
    "first column only": ("uw = 0.5 * (np.mean(bot) + np.mean(top))",
                          "uw = 0.5 * (bot[0] + top[0])"),
}


@pytest.mark.parametrize("slip", sorted(SLIP_SLIPS))
def test_slip_pin_catches_planted_slips(slip):
    Mut = _mutant_channel(*SLIP_SLIPS[slip])
    e, w, c = dvm.dvm2d("D2V16", DVM_TABLES)
    a, b = 3e-4, 1e-3
    caught = False
    for Nx, Ny in SLIP_SHAPES:
        ch = Mut(e, w, c, 3, Nx, Ny, 0.1, 0.0)
        ch.f[:] = _quadratic_state(ch, a, b)
        caught |= abs(ch.slip_velocity() - a / (a + b)) > 1e-6
        caught |= abs(ch.centre_velocity() - (a + b)) > 1e-6 * (a + b)
    assert caught
