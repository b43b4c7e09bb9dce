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
* the (x, z) marginal of a 3D DVM for a channel that is uniform along y,
* the weight solver of Sect. III: the matrix K(S) of Eq. defK built with the
  scalar-product recurrence of the Hermite tensors printed below it, its null
  space (Eq. defQua, dimker), the lattice speed c* at which a stencil becomes
  a minimal DVM, and the wall augmentation of Sect. IV (Eq. 9.13, wallEq,
  defA).
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


# ---- weight solver (Sect. III) and wall augmentation (Sect. IV) -------------

def hermite_product_polys(Q):
    """P_m(a, b, s) = H^(m)(xi) . H^(m)(eta) (all indices contracted) as
    polynomials in a = xi.xi, b = eta.eta, s = xi.eta, for m = 0..Q, from the
    recurrence below Eq. defK:
        P_{m+1} = (xi.eta - xi.d_eta - eta.d_xi + d_xi.d_eta) P_m.
    With f = f(a, b, s): d_xi_i f = 2 xi_i f_a + eta_i f_s and
    d_eta_i f = 2 eta_i f_b + xi_i f_s, hence
        xi.d_eta f  = 2 s f_b + a f_s,      eta.d_xi f = 2 s f_a + b f_s,
        d_xi.d_eta f = 4 s f_ab + 2 b f_bs + 2 a f_as + s f_ss + D f_s.
    The dimension D enters, so polynomials are returned as functions of D:
    a list of dicts {(i, j, k, l): coeff} meaning coeff a^i b^j s^k D^l."""
    def add(out, key, v):
        if v:
            out[key] = out.get(key, 0) + v

    P = [{(0, 0, 0, 0): 1}]
    for _ in range(Q):
        cur, nxt = P[-1], {}
        for (i, j, k, l), v in cur.items():
            add(nxt, (i, j, k + 1, l), v)                      # s P
            if j:
                add(nxt, (i, j - 1, k + 1, l), -2 * j * v)     # -2 s P_b
            if k:
                add(nxt, (i + 1, j, k - 1, l), -k * v)         # -a P_s
            if i:
                add(nxt, (i - 1, j, k + 1, l), -2 * i * v)     # -2 s P_a
            if k:
                add(nxt, (i, j + 1, k - 1, l), -k * v)         # -b P_s
            if i and j:
                add(nxt, (i - 1, j - 1, k + 1, l), 4 * i * j * v)      # 4 s P_ab
            if j and k:
                add(nxt, (i, j, k - 1, l), 2 * j * k * v)              # 2 b P_bs
            if i and k:
                add(nxt, (i, j, k - 1, l), 2 * i * k * v)              # 2 a P_as
            if k >= 2:
                add(nxt, (i, j, k - 1, l), k * (k - 1) * v)            # s P_ss
            if k:
                add(nxt, (i, j, k - 1, l + 1), k * v)                  # D P_s
        P.append({key: v for key, v in nxt.items() if v})
    return P


def kmatrix_orders(e, c, Q):
    """The Q blocks K^(m)_{ab} = H^(m)(xi_a) . H^(m)(xi_b), m = 1..Q, whose
    sum is K(S) of Eq. defK; xi = c e."""
    xi = c * np.asarray(e, dtype=np.float64)
    D = xi.shape[1]
    a = np.sum(xi * xi, axis=1)
    A, B = np.meshgrid(a, a, indexing="ij")
    S = xi @ xi.T
    out = []
    for poly in hermite_product_polys(Q)[1:]:
        K = np.zeros_like(S)
        for (i, j, k, l), v in poly.items():
            K += v * A ** i * B ** j * S ** k * float(D) ** l
        out.append(K)
    return out


def kmatrix(e, c, Q):
    """K(S) of Eq. defK."""
    return sum(kmatrix_orders(e, c, Q))


def symmetry_groups(e):
    """Group index of each velocity (Eq. wdach): velocities related by the
    lattice reflections (component permutations and sign flips) share the
    multiset of absolute components.  Groups are numbered in order of first
    appearance; raises if an orbit is incomplete."""
    keys, gid = {}, []
    for row in np.asarray(e).tolist():
        key = tuple(sorted(abs(x) for x in row))
        gid.append(keys.setdefault(key, len(keys)))
    gid = np.array(gid)
    for key, g in keys.items():
        orbit = set()
        for perm in itertools.permutations(key):
            for signs in itertools.product((1, -1), repeat=len(key)):
                orbit.add(tuple(sg * p for sg, p in zip(signs, perm)))
        if int(np.sum(gid == g)) != len(orbit):
            raise ValueError(f"incomplete symmetry group {key}")
    return gid


def reduced_kmatrix(e, c, Q):
    """K reduced to one unknown per symmetry group (weights equal within a
    group, Eq. wdach): Kg = G^T (sum_m K^(m) / max|K^(m)|) G with G the
    velocity-group incidence matrix.  Scaling each order by a positive
    factor leaves the null space unchanged, because w.K.w is the sum over m
    of the squared Hermite moments (the argument below Eq. defK), so w is in
    the null space exactly when every order's moment vanishes."""
    gid = symmetry_groups(e)
    Gm = np.zeros((len(gid), gid.max() + 1))
    Gm[np.arange(len(gid)), gid] = 1.0
    K = np.zeros((len(gid), len(gid)))
    for Km in kmatrix_orders(e, c, Q):
        scale = np.max(np.abs(Km))
        if scale > 0:
            K += Km / scale
    return Gm.T @ K @ Gm, gid


def null_space(e, c, Q, rtol=1e-12):
    """Null space of the reduced K: (basis of group weight vectors as
    columns, eigenvalues ascending, group index of each velocity).  The
    matrix is first equilibrated, Kh = d^-1/2 Kg d^-1/2 with d = diag(Kg)
    (a change of unknowns W = d^-1/2 Wh, so the null spaces correspond); the
    nullity (Eq. dimker) is the number of eigenvalues of Kh below rtol times
    the largest."""
    Kg, gid = reduced_kmatrix(e, c, Q)
    dh = 1.0 / np.sqrt(np.diag(Kg))
    lam, vec = np.linalg.eigh(dh[:, None] * Kg * dh[None, :])
    n = int(np.sum(lam < rtol * lam[-1]))
    return dh[:, None] * vec[:, :n], lam, gid


def solve_weights(e, c, Q):
    """Weights of a stencil (Eq. defQua): the normalised (sum w = 1) null
    vector of K when dim ker K = 1.  Returns (w, nullity)."""
    basis, _, gid = null_space(e, c, Q)
    n = basis.shape[1]
    if n != 1:
        return None, n
    wg = basis[:, 0]
    w = wg[gid]
    return w / np.sum(w), 1


def hermite_1d(n, x):
    """Probabilists' Hermite polynomial He_n(x): He_0 = 1, He_1 = x,
    He_{k+1} = x He_k - k He_{k-1}."""
    h0, h1 = np.ones_like(x), x
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, x * h1 - k * h0
    return h1


def multi_indices(D, m):
    """Exponent tuples (n_1..n_D), sum m: the distinct components of a
    symmetric rank-m tensor in D dimensions."""
    return [t for t in itertools.product(range(m + 1), repeat=D) if sum(t) == m]


def moment_matrix(e, c, Q):
    """The orthogonality conditions of Eq. orth with n = 0, written per
    symmetry group: row (m, n_1..n_D), column g holds
    sum_{a in g} H^(m)_{n}(xi_a), where the Hermite tensor component with
    n_d indices equal to d is prod_d He_{n_d}(xi_d) (the Gaussian weight
    factorises over the components).  Each order m is scaled by the norm of
    the same sums taken over absolute values, so that rows that vanish by
    symmetry stay at rounding level.  Returns (M, group index)."""
    gid = symmetry_groups(e)
    G = gid.max() + 1
    xi = c * np.asarray(e, dtype=np.float64)
    D = xi.shape[1]
    He = [[hermite_1d(n, xi[:, d]) for n in range(Q + 1)] for d in range(D)]
    blocks = []
    for m in range(1, Q + 1):
        rows, arows = [], []
        for t in multi_indices(D, m):
            v = np.prod([He[d][t[d]] for d in range(D)], axis=0)
            rows.append(np.bincount(gid, weights=v, minlength=G))
            arows.append(np.bincount(gid, weights=np.abs(v), minlength=G))
        A, Aa = np.array(rows), np.array(arows)
        scale = np.linalg.norm(Aa)
        if scale > 0:
            blocks.append(A / scale)
    return np.vstack(blocks), gid


def orth_gap(e, c, Q):
    """Smallest over largest singular value of the moment matrix with
    unit-norm columns: zero where the stencil admits weights of order Q
    (c = c*), linear in |c - c*| near it."""
    M, _ = moment_matrix(e, c, Q)
    M = M / np.linalg.norm(M, axis=0)
    s = np.linalg.svd(M, compute_uv=False)
    return s[-1] / s[0]


def find_c(e, Q, c_lo, c_hi, n_scan=400):
    """Lattice speed c* in [c_lo, c_hi] at which the stencil is a minimal DVM
    of order Q (dim ker K = 1) with positive weights: scan orth_gap for local
    minima, refine each by golden-section search (the gap has a kink at c*),
    and return the smallest c* whose weights are all positive, or None."""
    cs = np.linspace(c_lo, c_hi, n_scan)
    f = np.array([orth_gap(e, c, Q) for c in cs])
    phi = (math.sqrt(5.0) - 1.0) / 2.0
    for i in range(1, n_scan - 1):
        if not (f[i] <= f[i - 1] and f[i] <= f[i + 1]):
            continue
        lo, hi = cs[i - 1], cs[i + 1]
        x1, x2 = hi - phi * (hi - lo), lo + phi * (hi - lo)
        f1, f2 = orth_gap(e, x1, Q), orth_gap(e, x2, Q)
        while hi - lo > 4e-16 * hi:
            if f1 <= f2:
                hi, x2, f2 = x2, x1, f1
                x1 = hi - phi * (hi - lo)
                f1 = orth_gap(e, x1, Q)
            else:
                lo, x1, f1 = x1, x2, f2
                x2 = lo + phi * (hi - lo)
                f2 = orth_gap(e, x2, Q)
        c = 0.5 * (lo + hi)
        if orth_gap(e, c, Q) > 1e-9:
            continue
        w, n = solve_weights(e, c, Q)
        if n == 1 and np.all(w > 0):
            return float(c)
    return None


def augment(e, c, Q, constraints):
    """Wall-augmented weights (Sect. IV): w = x_j w^(j) over an orthogonal
    basis of the null space of K (Eq. 9.13), x from the equations of
    Eq. wallEq, A_kj = sum_{n.xi_a > 0} T^a_k w^(j)_a (Eq. defA) with
    b_k = W_k (Eq. Wscalar), for the selected non-trivial wall moments
    (indices into nontrivial_moments(D, Q)), together with sum w = 1;
    least squares when overdetermined.  Returns (w, residual norm)."""
    basis, _, gid = null_space(e, c, Q)
    if basis.shape[1] == 0:
        raise ValueError("K(S) is regular at this c")
    xi = c * np.asarray(e, dtype=np.float64)
    D = xi.shape[1]
    moms = nontrivial_moments(D, Q)
    Wb = basis[gid, :]                        # velocity weights of each basis vector
    up = xi[:, -1] > 0
    rows, rhs = [], []
    for k in constraints:
        mx, my, mz = moms[k]
        T = xi[:, 0] ** mx * (xi[:, 1] ** my if D == 3 else 1.0) * xi[:, -1] ** mz
        rows.append(T[up] @ Wb[up])
        rhs.append(wall_moment_exact(D, mx, my, mz))
    rows.append(np.sum(Wb, axis=0))
    rhs.append(1.0)
    A, b = np.array(rows), np.array(rhs)
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    return Wb @ x, float(np.linalg.norm(A @ x - b))
