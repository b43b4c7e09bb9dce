"""Oracle: plain, slow, fp64 CPU restatement of the paper's LB-BGK channel
solver (Sect. V and VI).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The library
(``paper_1510_08886_gb300``) never imports it and shares no code with it.

* ``oracle.dvm``: DVM expansion and quadrature / wall-moment properties.
* ``Channel``: a channel solve (ctypes over lbm_oracle.c) with the
  observables of Sect. VI: mass flow (Eq. pf.1) and slip velocity
  (Eq. defSlip).

Units (Sect. II and V): lengths in l0 = channel width, velocities in
c0 = sqrt(R theta0), times in l0/c0.  Ny nodes across the channel give
dx = 1/Ny, dt = dx/c, tau = sqrt(2/pi) Kn (Eq. nm.13).
"""
import ctypes
import math

import numpy as np

from . import build as _build
from . import dvm  # noqa: F401  (re-export)

_lib = None


def _load(path=None):
    global _lib
    if _lib is None or path is not None:
        lib = ctypes.CDLL(path or _build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_Params)
        lib.oracle_run.argtypes = [P, dp, dp, ctypes.c_long]
        lib.oracle_collide.argtypes = [P, dp, dp]
        lib.oracle_stream.argtypes = [P, dp, dp]
        lib.oracle_moments.argtypes = [P, dp, dp, dp, dp]
        lib.oracle_moments.restype = None
        lib.oracle_equilibrium.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, dp]
        lib.oracle_equilibrium.restype = None
        lib.oracle_force.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp, dp]
        lib.oracle_force.restype = None
        lib.oracle_threads.argtypes = [ctypes.c_int]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def use_openmp(threads):
    """Switch this process to the OpenMP build of the oracle (the CPU
    baseline's timing on all host cores; the per-node arithmetic is the
    serial build's) with `threads` threads.  Returns the thread count in use,
    or None when no OpenMP build is available (the serial build stays)."""
    path = _build.build_omp()
    if path is None:
        return None
    return _load(path).oracle_threads(int(threads))


class _Params(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int), ("Nx", ctypes.c_int), ("Ny", ctypes.c_int),
                ("N", ctypes.c_int),
                ("ex", ctypes.POINTER(ctypes.c_int)),
                ("ey", ctypes.POINTER(ctypes.c_int)),
                ("w", ctypes.POINTER(ctypes.c_double)),
                ("c", ctypes.c_double), ("tau", ctypes.c_double),
                ("dt", ctypes.c_double), ("gx", ctypes.c_double),
                ("gy", ctypes.c_double), ("wall_mode", ctypes.c_int),
                ("force_a3", ctypes.c_int)]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tau_of_kn(Kn):
    """Eq. nm.13: Kn = sqrt(pi/2) tau (tau in units of l0/c0)."""
    return math.sqrt(2.0 / math.pi) * Kn


def force_for_mach(Kn, mach=1e-3):
    """Body acceleration whose no-slip Navier-Stokes centre-line speed
    u_c = g l0^2 / (8 nu) (Sect. VI, below Eq. pf.1) equals ``mach``;
    nu = tau (Eq. nm.11)."""
    return 8.0 * tau_of_kn(Kn) * mach


class Channel:
    """One force-driven channel solve on the CPU, fp64.

    e: (V, 2) integer velocities (x, y), y the wall normal; w: (V,) weights;
    c: lattice speed; N: Hermite order; g: body acceleration along x.
    """

    def __init__(self, e, w, c, N, Nx, Ny, Kn, g, gy=0.0, wall="plain", force="nm4"):
        e = np.asarray(e)
        self.V = len(e)
        self.Nx, self.Ny, self.N = int(Nx), int(Ny), int(N)
        self.c, self.Kn, self.g = float(c), float(Kn), float(g)
        self.ex = np.ascontiguousarray(e[:, 0], dtype=np.int32)
        self.ey = np.ascontiguousarray(e[:, 1], dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.tau = tau_of_kn(Kn)
        self.dt = (1.0 / Ny) / c
        self.p = _Params(self.V, self.Nx, self.Ny, self.N,
                         self.ex.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         self.ey.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         _dp(self.w), self.c, self.tau, self.dt, self.g, float(gy),
                         {"plain": 0, "transformed": 1}[wall],
                         {"nm4": 0, "nm4+a3": 1}[force])
        self.f = np.zeros((self.V, self.Ny, self.Nx))
        self.work = np.zeros_like(self.f)
        self.steps = 0

    @property
    def omega(self):
        """Relaxation factor dt/(tau + dt/2) of Eq. nm.8."""
        return self.dt / (self.tau + 0.5 * self.dt)

    def init(self, rho=None):
        """fbar_a = rho w_a (fluid at rest, no force in the initial state)."""
        r = np.ones((self.Ny, self.Nx)) if rho is None else np.asarray(rho, dtype=np.float64)
        self.f[:] = self.w[:, None, None] * r[None, :, :]
        self.steps = 0
        return self

    def step(self, n=1):
        if _load().oracle_run(ctypes.byref(self.p), _dp(self.f), _dp(self.work), int(n)):
            raise MemoryError("oracle_run failed")
        self.steps += int(n)
        return self

    def collide(self, f):
        out = np.empty_like(f)
        _load().oracle_collide(ctypes.byref(self.p), _dp(np.ascontiguousarray(f)), _dp(out))
        return out

    def stream(self, fstar):
        out = np.empty_like(fstar)
        _load().oracle_stream(ctypes.byref(self.p), _dp(np.ascontiguousarray(fstar)), _dp(out))
        return out

    def moments(self, f=None):
        """(rho, u_x, u_y), each (Ny, Nx), of the state (Eq. nm.10)."""
        f = self.f if f is None else np.ascontiguousarray(f)
        rho = np.empty((self.Ny, self.Nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        _load().oracle_moments(ctypes.byref(self.p), _dp(f), _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def mean_ux(self):
        """<u_x>: midpoint rule over the half-way nodes of Eq. pf.1's
        integral, i.e. the mean over all nodes."""
        return float(np.mean(self.moments()[1]))

    def mass_flow(self):
        """Normalised mass flow, Eq. pf.1: mdot = <u>/(4 u_c Kn) with
        u_c = g l0^2/(8 nu), nu = tau, l0 = 1  =>  mdot = 2 tau <u>/(g Kn)."""
        return 2.0 * self.tau * self.mean_ux() / (self.g * self.Kn)

    def slip_velocity(self):
        """u_s = u(l0/2)/u(0), Eq. defSlip.  The wall value is the quadratic
        extrapolation of the three nodes nearest to each wall (nodes at
        0.5, 1.5, 2.5 spacings: weights 15/8, -10/8, 3/8), averaged over both
        walls and all columns; the centre value is the centre node (odd Ny)
        or the four-point midpoint interpolation (even Ny)."""
        u = self.moments()[1]
        Ny = self.Ny
        bot = (15.0 * u[0] - 10.0 * u[1] + 3.0 * u[2]) / 8.0
        top = (15.0 * u[Ny - 1] - 10.0 * u[Ny - 2] + 3.0 * u[Ny - 3]) / 8.0
        uw = 0.5 * (np.mean(bot) + np.mean(top))
        if Ny % 2:
            uc = np.mean(u[(Ny - 1) // 2])
        else:
            m = Ny // 2
            uc = np.mean((9.0 * (u[m - 1] + u[m]) - (u[m - 2] + u[m + 1])) / 16.0)
        return float(uw / uc)

    def centre_velocity(self, u=None):
        """u(0): x-averaged u_x at the channel centre (centre node for odd Ny,
        four-point midpoint interpolation for even Ny), as for u_s."""
        u = self.moments()[1] if u is None else u
        Ny = self.Ny
        if Ny % 2:
            return float(np.mean(u[(Ny - 1) // 2]))
        m = Ny // 2
        return float(np.mean((9.0 * (u[m - 1] + u[m]) - (u[m - 2] + u[m + 1])) / 16.0))

    def knudsen_layer(self):
        """Non-equilibrium velocity profile u^(neq)(z) = u(z) - u^(NS)(z)
        (Eq. uNEQ), u^(NS) the parabola through u(0) with the same mass flow
        (Eq. uNS): u^(NS)(z) = u(0) (1 - 3 (1 - <u>/u(0)) (z/(l0/2))^2),
        <u> the mean over the nodes (the integral of Eq. uNS by the midpoint
        rule), z_j = (j + 1/2)/Ny - 1/2.  Returns an array of Ny values
        (u averaged over x)."""
        u = self.moments()[1]
        uc = self.centre_velocity(u)
        prof = np.mean(u, axis=1)
        z = (np.arange(self.Ny) + 0.5) / self.Ny - 0.5
        uns = uc * (1.0 - 3.0 * (1.0 - np.mean(u) / uc) * (z / 0.5) ** 2)
        return prof - uns

    def run_to_steady(self, tol, max_steps, check_every=100):
        """Step until max |u_x(t) - u_x(t - dt)| < tol, tested every
        ``check_every`` steps.  Returns (converged, steps, last_du)."""
        du = math.inf
        while self.steps < max_steps:
            n = min(check_every, max_steps - self.steps)
            if n > 1:
                self.step(n - 1)
            prev = self.moments()[1]
            self.step(1)
            du = float(np.max(np.abs(self.moments()[1] - prev)))
            if du < tol:
                return True, self.steps, du
        return False, self.steps, du

    # single-node helpers used by the pins
    def equilibrium(self, rho, ux, uy):
        out = np.empty(self.V)
        _load().oracle_equilibrium(ctypes.byref(self.p), rho, ux, uy, _dp(out))
        return out

    def force(self, rho, ux, uy, Pi):
        out = np.empty(self.V)
        Pi = np.ascontiguousarray(np.asarray(Pi, dtype=np.float64).reshape(4))
        _load().oracle_force(ctypes.byref(self.p), rho, ux, uy, _dp(Pi), _dp(out))
        return out


def channel(name, N, Nx, Ny, Kn, g, tables=None, wall="plain", force="nm4"):
    """Channel for a named DVM (a 2D table, or '<3D name>xz' for the (x, z)
    marginal of a 3D table).  wall: "plain" (the unknown fbar is Psi rho_w w_a)
    or "transformed" (the condition holds for f, fbar through Eq. nm.7).
    force: "nm4" (Eq. nm.4 as printed) or, for N = 4, "nm4+a3" (plus the
    fourth-order Hermite force term with a^(3) = rho u u u)."""
    if tables is None:
        from lbm_inputs import DVM_TABLES as tables
    e, w, c = dvm.dvm2d(name, tables)
    return Channel(e, w, c, N, Nx, Ny, Kn, g, wall=wall, force=force)
