"""Oracle: discrete velocity models (DVMs) and their quadrature properties.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use it.

Plain numpy restatements, in fp64, of:

* group expansion by the reflections of the lattice (Eq. wdach),
* the quadrature order of a DVM via the Gaussian moments (Eq. genQua, orth),
* the stencil energy E (Eq. Ssymbol and the definition of E above it),
* the equilibrium wall moments W, their quadrature W^DVM over strictly
  n.xi > 0 (Eq. Wscalar, wallQuad), the wall errors sigma (Eq. wallError),
  sigma_Sigma (Eq. sigmaSigma) and the wall accuracy index Lambda_index
  (Eq. defbin) over the non-trivial moments of Eq. nontriv,
* the (x, z) marginal of a 3D DVM for a channel that is uniform along y.
"""
import itertools
import math

import numpy as np


def expand(table):
    """Expand printed group rows into (e, w, c).

    e: int array (V, D) of integer velocities xi/c; w: float64 (V,); c: float.
    The orbit of a representative under the lattice reflections is every
    permutation of its components combined with every sign flip (Eq. wdach);
    in 2D that is the symmetry group of the square.
    """
    D = table["D"]
    es, ws = [], []
    for rep, vg, wg in table["groups"]:
        orbit = set()
        for perm in itertools.permutations(rep):
            for signs in itertools.product((1, -1), repeat=D):
                orbit.add(tuple(s * p for s, p in zip(signs, perm)))
        orbit = sorted(orbit)
        if len(orbit) != vg:
            raise ValueError(f"group {rep}: orbit has {len(orbit)} velocities, table says {vg}")
        es.extend(orbit)
        ws.extend([wg] * len(orbit))
    e = np.array(es, dtype=np.int64)
    w = np.array(ws, dtype=np.float64)
    if len(e) != table["V"]:
        raise ValueError("velocity count differs from the stencil symbol")
    return e, w, float(table["c"])


def marginal_xz(e3, w3):
    """(x, z) marginal of a 3D DVM: sum the weights of velocities with equal
    (e_x, e_z).  For a flow uniform along y every moment that contains no
    xi_y is unchanged, so the 2D set keeps the quadrature order and the
    (x, z) wall moments of the 3D set."""
    acc = {}
    for (ex, ey, ez), wa in zip(e3.tolist(), w3.tolist()):
        acc[(ex, ez)] = acc.get((ex, ez), 0.0) + wa
    keys = sorted(acc)
    return np.array(keys, dtype=np.int64), np.array([acc[k] for k in keys])


def gaussian_moment_1d(m):
    """int xi^m exp(-xi^2/2) dxi / sqrt(2 pi) = (m-1)!! for even m, else 0."""
    if m % 2:
        return 0.0
    r = 1.0
    for k in range(m - 1, 0, -2):
        r *= k
    return r


def moment_error(e, w, c, degree):
    """Largest relative deviation of sum_a w_a xi_a^m from the Gaussian
    moment, over all monomials of exactly the given total degree."""
    xi = c * e.astype(np.float64)
    D = e.shape[1]
    worst = 0.0
    for ms in itertools.product(range(degree + 1), repeat=D):
        if sum(ms) != degree:
            continue
        num = np.sum(w * np.prod(xi ** np.array(ms), axis=1))
        ref = np.prod([gaussian_moment_1d(m) for m in ms])
        worst = max(worst, abs(num - ref) / max(1.0, abs(ref)))
    return worst


def quadrature_order(e, w, c, max_degree=16, rtol=1e-9):
    """Highest Q with every moment of degree <= Q exact (Eq. orth, genQua)."""
    q = -1
    for deg in range(max_degree + 1):
        if moment_error(e, w, c, deg) > rtol:
            break
        q = deg
    return q


def energy(e):
    """Stencil energy E = (1/2) sum_a |e_a|^2 (velocities in units of c)."""
    return float(np.sum(e.astype(np.int64) ** 2)) / 2.0


def nontrivial_moments(D, Q):
    """Exponents (m_x, m_y, m_z) of the non-trivial wall moments (Eq. nontriv)
    in the paper's order: increasing n, then decreasing m_z, then decreasing
    m_x.  In 2D m_y = 0 (Appendix B)."""
    out = []
    for n in range(Q + 1):
        for mz in sorted([m for m in range(n + 1) if m == 0 or m % 2 == 1],
                         reverse=True):
            for mx in range(n - mz, -1, -1):
                my = n - mz - mx
                if mx % 2 or my % 2 or my > mx:
                    continue
                if D == 2 and my != 0:
                    continue
                out.append((mx, my, mz))
    return out


def wall_moment_exact(D, mx, my, mz):
    """Equilibrium wall moment W over the half space xi_z > 0 with the
    Gaussian weight omega (Eq. defW), by the Gamma-function closed form of
    Eq. Wscalar; for D = 2 the y factor is dropped."""
    if mx % 2 or my % 2:
        return 0.0
    g = math.gamma
    if D == 3:
        return (math.sqrt(2.0) ** (mx + my + mz) / (8.0 * math.sqrt(math.pi) ** 3)
                * 4.0 * g((mx + 1) / 2) * g((my + 1) / 2) * g((mz + 1) / 2))
    if my:
        return 0.0
    return (math.sqrt(2.0) ** (mx + mz) / (4.0 * math.pi)
            * 2.0 * g((mx + 1) / 2) * g((mz + 1) / 2))


def wall_moment_dvm(e, w, c, mx, my, mz):
    """W^DVM: the quadrature over velocities with n.xi > 0 strictly
    (Eq. wallQuad), n = e_z the inward wall normal (last component)."""
    xi = c * e.astype(np.float64)
    D = e.shape[1]
    x = xi[:, 0]
    z = xi[:, -1]
    y = xi[:, 1] if D == 3 else np.zeros_like(x)
    sel = z > 0
    return float(np.sum(w[sel] * x[sel] ** mx * y[sel] ** my * z[sel] ** mz))


def wall_errors(e, w, c, Q):
    """sigma_k = (W^DVM - W)/W for the non-trivial moments of Eq. nontriv.

    Sign convention: the one of the printed tables (Tab. bulk, Wzxx, W0);
    Eq. wallError prints the opposite sign.  Returns a list of
    ((m_x, m_y, m_z), sigma)."""
    D = e.shape[1]
    out = []
    for m in nontrivial_moments(D, Q):
        W = wall_moment_exact(D, *m)
        out.append((m, (wall_moment_dvm(e, w, c, *m) - W) / W))
    return out


def sigma_sigma(errors):
    """Aggregate wall error (Eq. sigmaSigma): |sigma| weighted by e^-n over
    the non-trivial moments, normalised by the sum of the weights."""
    num = sum(abs(s) * math.exp(-sum(m)) for m, s in errors)
    den = sum(math.exp(-sum(m)) for m, _ in errors)
    return num / den


def lambda_index(errors, tol=1e-10):
    """Wall accuracy index (Eq. defbin): bit k-1 set when constraint k holds,
    a constraint counted as met when |sigma_k| < tol."""
    return sum(1 << k for k, (_, s) in enumerate(errors) if abs(s) < tol)


def dvm2d(name, tables):
    """2D velocity set for a channel run: a 2D table as printed, or the
    (x, z) marginal of a 3D table when the name ends in 'xz'."""
    if name.endswith("xz"):
        e3, w3, c = expand(tables[name[:-2]])
        e, w = marginal_xz(e3, w3)
        return e, w, c
    e, w, c = expand(tables[name])
    if e.shape[1] != 2:
        raise ValueError(f"{name} is not two-dimensional")
    return e, w, c
