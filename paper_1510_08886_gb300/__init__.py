"""GB300-native high-order lattice Boltzmann solver for force-driven plane
channels with diffuse Maxwell walls (Feuchter & Schleifenbaum, Sect. V, VI).

Thin Python binding over the C ABI of include/lbm.h: every step of the
solve runs in the library's CUDA kernels; PyTorch only provides device
memory (the solver workspace) and the CUDA stream.

    import paper_1510_08886_gb300 as lbm
    e, w, c = lbm.dvm("D2V33")
    s = lbm.Solver(e, w, c, order=4, Nx=4096, Ny=512, Kn=0.1,
                   force=lbm.force_for_mach(0.1), precision="fp32")
    s.init(); s.step(1000); print(s.mass_flow(), s.slip_velocity())
"""
import ctypes
import math

import numpy as np

from . import _lib
from ._lib import LBMError, check, lbm_dvm

__all__ = ["dvm", "dvm_from_groups", "Solver", "LBMError", "force_for_mach", "tau_of_kn",
           "quadrature_order", "dvm_weights", "dvm_find_c", "dvm_nontrivial_moments",
           "dvm_augment", "Engine"]

PRECISIONS = {"fp64": _lib.LBM_FP64, "fp32": _lib.LBM_FP32, "fp16": _lib.LBM_FP16,
              "bf16": _lib.LBM_BF16}


def tau_of_kn(Kn):
    """tau = sqrt(2/pi) Kn (Eq. nm.13), in units of l0/c0."""
    return math.sqrt(2.0 / math.pi) * Kn


def force_for_mach(Kn, mach=1e-3):
    """g such that the no-slip Navier-Stokes centre-line speed g/(8 nu),
    nu = tau (Eq. nm.11, Sect. VI), equals ``mach`` (in units of c0)."""
    return 8.0 * tau_of_kn(Kn) * mach


def _ip(a):
    return a.ctypes.data_as(_lib.c_int_p)


def _dp(a):
    return a.ctypes.data_as(_lib.c_double_p)


def dvm_from_groups(table):
    """Expand a printed group table (dict with D, c, groups) with the
    library's lbm_dvm_expand.  Returns (e int32 (V, D), w float64 (V,), c)."""
    D = int(table["D"])
    reps = np.ascontiguousarray([list(g[0]) for g in table["groups"]], dtype=np.int32)
    vg = np.ascontiguousarray([g[1] for g in table["groups"]], dtype=np.int32)
    wg = np.ascontiguousarray([g[2] for g in table["groups"]], dtype=np.float64)
    cap = int(vg.sum())
    e = np.zeros((cap, D), dtype=np.int32)
    w = np.zeros(cap)
    V = ctypes.c_int(0)
    check(_lib.lib().lbm_dvm_expand(D, len(wg), _ip(reps), _ip(vg), _dp(wg), cap, _ip(e),
                                    _dp(w), ctypes.byref(V)), "lbm_dvm_expand")
    return e[:V.value], w[:V.value], float(table["c"])


def dvm(name, tables=None):
    """Velocity set of a named DVM for the 2D channel: a 2D table of the
    paper as printed, or '<3D name>xz' for the (x, z) marginal of a 3D table
    (lbm_dvm_marginal_xz)."""
    if tables is None:
        from lbm_inputs import DVM_TABLES as tables
    if name.endswith("xz"):
        e3, w3, c = dvm_from_groups(tables[name[:-2]])
        e3 = np.ascontiguousarray(e3, dtype=np.int32)
        cap = len(w3)
        e = np.zeros((cap, 2), dtype=np.int32)
        w = np.zeros(cap)
        V = ctypes.c_int(0)
        check(_lib.lib().lbm_dvm_marginal_xz(len(w3), _ip(e3), _dp(np.ascontiguousarray(w3)),
                                             cap, _ip(e), _dp(w), ctypes.byref(V)),
              "lbm_dvm_marginal_xz")
        return e[:V.value], w[:V.value], c
    e, w, c = dvm_from_groups(tables[name])
    if e.shape[1] != 2:
        raise ValueError(f"{name} is three-dimensional; use '{name}xz'")
    return e, w, c


class _DVM:
    """Keeps the arrays of an lbm_dvm alive."""

    def __init__(self, e, w, c):
        self.e = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 2))
        self.w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        self.s = lbm_dvm(2, len(self.w), _ip(self.e), _dp(self.w), float(c))

    def ref(self):
        return ctypes.byref(self.s)


def quadrature_order(e, w, c):
    d = _DVM(e, w, c)
    Q = ctypes.c_int(-1)
    check(_lib.lib().lbm_dvm_quadrature_order(d.ref(), ctypes.byref(Q)))
    return Q.value


def _stencil(e):
    e = np.ascontiguousarray(np.asarray(e), dtype=np.int32)
    if e.ndim != 2 or e.shape[1] not in (2, 3):
        raise ValueError("velocities must be an (V, 2) or (V, 3) integer array")
    return e, e.shape[1], e.shape[0]


def dvm_weights(e, c, Q):
    """Weights of a stencil from its velocities (Sect. III, Eq. defQua,
    defK): returns (w, nullity); w is None unless dim ker K = 1."""
    e, D, V = _stencil(e)
    w = np.empty(V)
    n = ctypes.c_int(-1)
    check(_lib.lib().lbm_dvm_solve_weights(D, V, _ip(e), float(c), int(Q), _dp(w), ctypes.byref(n)),
          "lbm_dvm_solve_weights")
    return (w if n.value == 1 else None), n.value


def dvm_find_c(e, Q, c_lo, c_hi):
    """Lattice speed c* in [c_lo, c_hi] of a minimal DVM of order Q with
    positive weights (Eq. dimker), or None."""
    e, D, V = _stencil(e)
    c = ctypes.c_double(0.0)
    rc = _lib.lib().lbm_dvm_find_c(D, V, _ip(e), int(Q), float(c_lo), float(c_hi), ctypes.byref(c))
    if rc == _lib.LBM_ENOTCONV:
        return None
    check(rc, "lbm_dvm_find_c")
    return c.value


def dvm_nontrivial_moments(D, Q):
    """Exponents (m_x, m_y, m_z) of the non-trivial wall moments (Eq. nontriv)."""
    L = ctypes.c_int(0)
    check(_lib.lib().lbm_dvm_nontrivial_moments(int(D), int(Q), 0, None, ctypes.byref(L)))
    out = np.zeros(3 * max(L.value, 1), dtype=np.int32)
    check(_lib.lib().lbm_dvm_nontrivial_moments(int(D), int(Q), L.value, _ip(out), ctypes.byref(L)),
          "lbm_dvm_nontrivial_moments")
    return [tuple(int(x) for x in out[3 * k:3 * k + 3]) for k in range(L.value)]


def dvm_augment(e, c, Q, constraints):
    """Wall-augmented weights (Sect. IV, Eq. 9.13, wallEq, defA) imposing the
    selected non-trivial wall moments (indices into dvm_nontrivial_moments)
    and sum w = 1.  Returns (w, residual)."""
    e, D, V = _stencil(e)
    k = np.ascontiguousarray(constraints, dtype=np.int32)
    w = np.empty(V)
    r = ctypes.c_double(0.0)
    check(_lib.lib().lbm_dvm_augment(D, V, _ip(e), float(c), int(Q), len(k),
                                     _ip(k) if len(k) else None, _dp(w), ctypes.byref(r)),
          "lbm_dvm_augment")
    return w, r.value


def fma_rate(precision="fp64", stream=None):
    """Sustained FMA rate of the current device in flop/s (lbm_fma_rate):
    the measured peak of an arithmetic-bound step."""
    torch = _torch_cuda()
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double(0)
    prec = {"fp64": _lib.LBM_FP64, "fp32": _lib.LBM_FP32}[precision]
    check(_lib.lib().lbm_fma_rate(prec, ctypes.c_void_p(st.cuda_stream), ctypes.byref(out)),
          "lbm_fma_rate")
    return out.value


def _torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1510_08886_gb300.Solver needs a CUDA device "
                           "(there is no CPU fallback)")
    return torch


class Solver:
    """One channel solve on the GPU (see include/lbm.h for the semantics).

    e (V, 2) integer velocities (x, y), y = wall normal; w (V,) weights;
    c lattice speed; order = Hermite order N; Nx periodic nodes, Ny nodes
    between the walls; Kn Knudsen number; force = g_x; precision 'fp64',
    'fp32', 'fp16' or 'bf16'.  Device memory comes from a torch uint8 tensor (the workspace);
    work is issued on ``stream`` (a torch.cuda.Stream) or torch's current
    stream.
    """

    def __init__(self, e, w, c, order, Nx, Ny, Kn, force, precision="fp64", stream=None,
                 device=None):
        torch = _torch_cuda()
        self._torch = torch
        self.dvm = _DVM(e, w, c)
        self.V = len(self.dvm.w)
        self.order, self.Nx, self.Ny = int(order), int(Nx), int(Ny)
        self.Kn, self.force, self.c = float(Kn), float(force), float(c)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        prec = PRECISIONS[precision]
        nbytes = ctypes.c_size_t(0)
        L = _lib.lib()
        check(L.lbm_workspace_bytes(self.dvm.ref(), self.Nx, self.Ny, prec, ctypes.byref(nbytes)),
              "lbm_workspace_bytes")
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = ctypes.c_void_p()
        check(L.lbm_create_in(self.dvm.ref(), self.order, self.Nx, self.Ny, self.Kn, self.force,
                              prec, ctypes.c_void_p(self.stream.cuda_stream),
                              ctypes.c_void_p(aligned), nbytes.value, ctypes.byref(h)),
              "lbm_create_in")
        self._h = h
        self.tau = tau_of_kn(self.Kn)
        self.dt = 1.0 / (self.Ny * self.c)

    # lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def workspace_bytes(self):
        return self.workspace.numel()

    # stepping ---------------------------------------------------------------
    def init(self, rho=None):
        """fbar = rho w (fluid at rest).  rho: None (uniform 1), a host array
        (Ny, Nx), or a CUDA float64 tensor of that shape."""
        L = _lib.lib()
        if rho is None:
            check(L.lbm_init(self._h, None), "lbm_init")
        elif hasattr(rho, "is_cuda") and rho.is_cuda:
            r = rho.to(self._torch.float64).contiguous()
            if r.numel() != self.Nx * self.Ny:
                raise ValueError("rho has the wrong size")
            self._rho_dev = r           # keep alive until the init kernel ran
            check(L.lbm_init_device(self._h, ctypes.c_void_p(r.data_ptr())), "lbm_init_device")
        else:
            r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.Ny, self.Nx))
            check(L.lbm_init(self._h, _dp(r)), "lbm_init")
        return self

    def step(self, n=1):
        check(_lib.lib().lbm_step(self._h, int(n)), "lbm_step")
        return self

    def average(self, n, every=1):
        """Advance n steps and leave in the moment fields the mean of the
        moments of every `every`-th step (lbm_average): the observables then
        report time averages, the steady state of 16-bit storage."""
        check(_lib.lib().lbm_average(self._h, int(n), int(every)), "lbm_average")
        return self

    def set_resident(self, enable):
        """Resident cluster chunks for a tiny fp64 / fp32 channel on (default) or off."""
        check(_lib.lib().lbm_set_resident(self._h, 1 if enable else 0), "lbm_set_resident")
        return self

    def resident_ctas(self):
        """CTAs of the cluster running this solve's resident chunks (0: per-step launches)."""
        n = ctypes.c_int(0)
        check(_lib.lib().lbm_resident_ctas(self._h, ctypes.byref(n)), "lbm_resident_ctas")
        return n.value

    def run_to_steady(self, tol, max_steps, check_every=100):
        """Returns (converged, steps_done, last_du)."""
        steps = ctypes.c_long(0)
        du = ctypes.c_double(0)
        rc = _lib.lib().lbm_run_to_steady(self._h, float(tol), int(max_steps), int(check_every),
                                          ctypes.byref(steps), ctypes.byref(du))
        if rc not in (_lib.LBM_OK, _lib.LBM_ENOTCONV):
            raise LBMError(rc, "lbm_run_to_steady")
        return rc == _lib.LBM_OK, steps.value, du.value

    # observables ------------------------------------------------------------
    def moments(self):
        rho = np.empty((self.Ny, self.Nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        check(_lib.lib().lbm_moments(self._h, _dp(rho), _dp(ux), _dp(uy)), "lbm_moments")
        return rho, ux, uy

    def mass_flow(self):
        m = ctypes.c_double(0)
        check(_lib.lib().lbm_mass_flow(self._h, ctypes.byref(m), None), "lbm_mass_flow")
        return m.value

    def mean_ux(self):
        u = ctypes.c_double(0)
        check(_lib.lib().lbm_mass_flow(self._h, None, ctypes.byref(u)), "lbm_mass_flow")
        return u.value

    def slip_velocity(self):
        u = ctypes.c_double(0)
        check(_lib.lib().lbm_slip_velocity(self._h, ctypes.byref(u)), "lbm_slip_velocity")
        return u.value

    def knudsen_layer(self):
        """u_neq(y) = u(y) - u_NS(y) (Eq. uNEQ), Ny values."""
        out = np.empty(self.Ny)
        check(_lib.lib().lbm_knudsen_layer(self._h, _dp(out)), "lbm_knudsen_layer")
        return out

    def status(self):
        return _lib.lib().lbm_status(self._h)

    @property
    def steps(self):
        n = ctypes.c_long(0)
        check(_lib.lib().lbm_steps_done(self._h, ctypes.byref(n)))
        return n.value

    def populations(self):
        """Post-collision fbar* of the last step, (V, Ny, Nx), caller order."""
        f = np.empty((self.V, self.Ny, self.Nx))
        check(_lib.lib().lbm_populations(self._h, _dp(f)), "lbm_populations")
        return f

    def get_state(self):
        n = ctypes.c_size_t(0)
        check(_lib.lib().lbm_state_bytes(self._h, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        check(_lib.lib().lbm_get_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value),
              "lbm_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(_lib.lib().lbm_set_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes),
              "lbm_set_state")
        return self


class Engine:
    """Many channel solves advanced together (include/lbm.h, engine section).

    Solves are admitted with ``add`` (returns a slot, or None when the arena
    or the slot table is full), advanced with ``run`` in chunks of
    ``chunk`` steps (one CUDA-graph replay per chunk) and released with
    ``remove``.  The arena is a torch uint8 tensor on the current device.
    ``resident`` runs solves that fit in shared memory a whole chunk per
    launch (bitwise the same results as the per-step launches).
    """

    def __init__(self, precision="fp32", max_solves=256, arena_bytes=1 << 30, stream=None,
                 chunk=100, resident=True):
        torch = _torch_cuda()
        self._torch = torch
        self.precision = precision
        self.max_solves = int(max_solves)
        self.arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.arena.data_ptr() + 255) & ~255
        self.stream = stream
        h = ctypes.c_void_p()
        check(_lib.lib().lbm_engine_create(
            PRECISIONS[precision], self.max_solves, ctypes.c_void_p(aligned), int(arena_bytes),
            ctypes.c_void_p(stream.cuda_stream) if stream is not None else None, ctypes.byref(h)),
            "lbm_engine_create")
        self._h = h
        self._dvm_cache = {}
        self.results = np.zeros((self.max_solves, 4))
        self.set_chunk(chunk)
        self.set_resident(resident)

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().lbm_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def solve_bytes(e, w, c, Nx, Ny, precision="fp32"):
        d = _DVM(e, w, c)
        n = ctypes.c_size_t(0)
        check(_lib.lib().lbm_engine_solve_bytes(d.ref(), int(Nx), int(Ny), PRECISIONS[precision],
                                                ctypes.byref(n)), "lbm_engine_solve_bytes")
        return n.value

    def set_chunk(self, steps):
        check(_lib.lib().lbm_engine_set_chunk(self._h, int(steps)), "lbm_engine_set_chunk")
        self.chunk = int(steps)

    def set_resident(self, enable):
        check(_lib.lib().lbm_engine_set_resident(self._h, int(bool(enable))),
              "lbm_engine_set_resident")
        self.resident = bool(enable)

    def paths(self):
        """Solves per path at the next chunk: (tiled, resident)."""
        t, r = ctypes.c_int(0), ctypes.c_int(0)
        check(_lib.lib().lbm_engine_paths(self._h, ctypes.byref(t), ctypes.byref(r)),
              "lbm_engine_paths")
        return t.value, r.value

    def _dvm(self, e, w, c):
        """The lbm_dvm of a velocity set, built once per distinct set (the
        library copies it at each add)."""
        e = np.asarray(e, dtype=np.int32)
        w = np.asarray(w, dtype=np.float64)
        key = (e.tobytes(), w.tobytes(), float(c))
        d = self._dvm_cache.get(key)
        if d is None:
            d = self._dvm_cache[key] = _DVM(e, w, c)
        return d

    def add(self, e, w, c, order, Nx, Ny, Kn, force, rho=None):
        d = self._dvm(e, w, c)
        slot = ctypes.c_int(-1)
        r = None
        if rho is not None:
            r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(int(Ny), int(Nx)))
        rc = _lib.lib().lbm_engine_add(self._h, d.ref(), int(order), int(Nx), int(Ny), float(Kn),
                                       float(force), _dp(r) if r is not None else None,
                                       ctypes.byref(slot))
        if rc == _lib.LBM_ENOMEM:
            return None
        check(rc, "lbm_engine_add")
        return slot.value

    def remove(self, slot):
        check(_lib.lib().lbm_engine_remove(self._h, int(slot)), "lbm_engine_remove")

    def run(self, chunks=1):
        """Advance every resident solve by chunks x chunk steps; returns the
        (max_solves, 4) array {max|du|, mdot, u_s, <u_x>} per slot."""
        check(_lib.lib().lbm_engine_run(self._h, int(chunks), _dp(self.results)), "lbm_engine_run")
        return self.results

    def launch(self, chunks=1):
        """Queue chunks x chunk steps and return at once (at most two
        launches outstanding); collect their results with ``wait``."""
        check(_lib.lib().lbm_engine_launch(self._h, int(chunks)), "lbm_engine_launch")

    def wait(self):
        """Results of the oldest outstanding launch (the array ``run`` returns)."""
        check(_lib.lib().lbm_engine_wait(self._h, _dp(self.results)), "lbm_engine_wait")
        return self.results

    def autotune(self):
        """Pick the tiled kernel's schedule (tile shape, cells per tile, grid,
        grab) by timing; returns the best time per step in ms."""
        ms = ctypes.c_double(0)
        check(_lib.lib().lbm_engine_autotune(self._h, ctypes.byref(ms)), "lbm_engine_autotune")
        return ms.value

    def set_schedule(self, tile_width=0, tile_cells=128, grab=4, grid_fraction=1.0, slot=-1):
        """Set the tiled kernel's schedule of the velocity-set group of
        ``slot`` (-1: every group): tile_width 0 (linear tiles) or 32, 64, 128
        columns; tile_cells 128, 256 or 512 nodes; grab tiles per atomic grab;
        grid_fraction of the occupancy limit (common to all groups)."""
        check(_lib.lib().lbm_engine_set_schedule(self._h, int(slot), int(tile_width), int(tile_cells),
                                                 int(grab), float(grid_fraction)),
              "lbm_engine_set_schedule")

    def schedule(self, slot):
        """The schedule of the velocity-set group of ``slot`` as a dict (the
        autotuner's choice after autotune)."""
        tw, tc, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        f = ctypes.c_double(0)
        check(_lib.lib().lbm_engine_get_schedule(self._h, int(slot), ctypes.byref(tw), ctypes.byref(tc),
                                                 ctypes.byref(g), ctypes.byref(f)),
              "lbm_engine_get_schedule")
        return {"tile_width": tw.value, "tile_cells": tc.value, "grab": g.value,
                "grid_fraction": f.value}

    def info(self, slot, status=False):
        """(steps done, status); the status (a device read) only when asked."""
        steps = ctypes.c_long(0)
        st = ctypes.c_int(0)
        check(_lib.lib().lbm_engine_info(self._h, int(slot), ctypes.byref(steps),
                                         ctypes.byref(st) if status else None),
              "lbm_engine_info")
        return steps.value, st.value

    def moments(self, slot, Nx, Ny):
        rho = np.empty((Ny, Nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        check(_lib.lib().lbm_engine_moments(self._h, int(slot), _dp(rho), _dp(ux), _dp(uy)),
              "lbm_engine_moments")
        return rho, ux, uy

    def get_state(self, slot):
        """Checkpoint of a slot (header, populations, moment fields) as a uint8 array."""
        n = ctypes.c_size_t(0)
        check(_lib.lib().lbm_engine_state_bytes(self._h, int(slot), ctypes.byref(n)),
              "lbm_engine_state_bytes")
        buf = np.empty(n.value, dtype=np.uint8)
        check(_lib.lib().lbm_engine_get_state(self._h, int(slot), buf.ctypes.data_as(ctypes.c_void_p),
                                              buf.nbytes), "lbm_engine_get_state")
        return buf

    def set_state(self, slot, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(_lib.lib().lbm_engine_set_state(self._h, int(slot), buf.ctypes.data_as(ctypes.c_void_p),
                                              buf.nbytes), "lbm_engine_set_state")
        return self

    def free_bytes(self):
        n = ctypes.c_size_t(0)
        check(_lib.lib().lbm_engine_free_bytes(self._h, ctypes.byref(n)))
        return n.value
