"""Pins of the oracle's weight solver (Sect. III, Eq. defQua, defK, dimker)
and wall augmentation (Sect. IV, Eq. 9.13, wallEq, defA).

K(S) comes from the paper's scalar-product recurrence of Hermite tensors; it
is checked against Hermite tensors built index by index (a different
derivation) and against closed forms of the first products.  The solver
must then recover, from the velocities alone, the weights and the lattice
speed c* that the paper prints for each stencil.
"""
import itertools
import math

import numpy as np
import pytest

from lbm_inputs import DVM_TABLES, TEXTBOOK_TABLES
from oracle import dvm

ALL = {**DVM_TABLES, **TEXTBOOK_TABLES}
AUGMENTED = ("D3V77", "D3V107")         # Tab. dvmD3Q7Set3, dvmD3Q7Set3b: augmented, set S3


def tensors_by_index(xi, Q):
    """H^(m)_{i1..im}(xi) for every index tuple, from
    H^(m+1)_{I j} = xi_j H^(m)_I - sum_k delta_{j i_k} H^(m-1)_{I without i_k}
    (the derivatives of the Gaussian, Eq. defH)."""
    D = len(xi)
    H = [{(): 1.0}]
    for m in range(Q):
        nxt = {}
        for idx in itertools.product(range(D), repeat=m + 1):
            head, j = idx[:-1], idx[-1]
            v = xi[j] * H[m][head]
            for k in range(m):
                if head[k] == j:
                    v -= H[m - 1][head[:k] + head[k + 1:]]
            nxt[idx] = v
        H.append(nxt)
    return H


def kmatrix_by_index(e, c, Q):
    xi = c * np.asarray(e, dtype=np.float64)
    Hs = [tensors_by_index(x, Q) for x in xi]
    K = np.zeros((len(xi), len(xi)))
    for m in range(1, Q + 1):
        keys = list(Hs[0][m])
        A = np.array([[h[m][k] for k in keys] for h in Hs])
        K += A @ A.T
    return K


def test_scalar_product_closed_forms():
    """P_1 = s, P_2 = s^2 - a - b + D, P_3 = s^3 - 3 (a + b) s + (3 D + 6) s
    (contractions of xi_i, xi_i xi_j - delta_ij, and the rank-3 tensor)."""
    P = dvm.hermite_product_polys(3)
    assert P[1] == {(0, 0, 1, 0): 1}
    assert P[2] == {(0, 0, 2, 0): 1, (1, 0, 0, 0): -1, (0, 1, 0, 0): -1, (0, 0, 0, 1): 1}
    assert P[3] == {(0, 0, 3, 0): 1, (1, 0, 1, 0): -3, (0, 1, 1, 0): -3, (0, 0, 1, 0): 6,
                    (0, 0, 1, 1): 3}


@pytest.mark.parametrize("name,Q", [("D2Q9", 5), ("D3Q19", 5), ("D2V16", 7), ("D3V15", 5)])
def test_kmatrix_recurrence_matches_tensors(name, Q):
    e, _, c = dvm.expand(ALL[name])
    Kr = dvm.kmatrix(e, c, Q)
    Ki = kmatrix_by_index(e, c, Q)
    assert np.max(np.abs(Kr - Ki)) <= 1e-12 * np.max(np.abs(Ki))


def test_kmatrix_random_stencil_and_psd():
    rng = np.random.default_rng(5)
    e = rng.integers(-3, 4, size=(7, 2))
    K = dvm.kmatrix(e, 0.9, 6)
    assert np.allclose(K, K.T, rtol=0, atol=1e-9 * np.max(np.abs(K)))
    assert np.max(np.abs(K - kmatrix_by_index(e, 0.9, 6))) <= 1e-12 * np.max(np.abs(K))
    # w.K.w is the sum over orders of the squared Hermite moments (Sect. III)
    w = rng.random(7)
    xi = 0.9 * e
    Hs = [tensors_by_index(x, 6) for x in xi]
    sq = sum(sum(sum(w[a] * Hs[a][m][k] for a in range(7)) ** 2 for k in Hs[0][m])
             for m in range(1, 7))
    assert math.isclose(w @ K @ w, sq, rel_tol=1e-11)


def test_moment_matrix_components_factorise():
    """prod_d He_{n_d}(xi_d) is the Hermite tensor component with n_d indices
    equal to d."""
    e, _, c = dvm.expand(ALL["D3Q19"])
    M, gid = dvm.moment_matrix(e, c, 5)
    xi = c * e
    Hs = [tensors_by_index(x, 5) for x in xi]
    row = 0
    for m in range(1, 6):
        ts = dvm.multi_indices(3, m)
        comp = []
        for t in ts:
            idx = tuple(d for d in range(3) for _ in range(t[d]))
            comp.append([sum(Hs[a][m][idx] for a in range(len(e)) if gid[a] == g)
                         for g in range(gid.max() + 1)])
        comp = np.array(comp)
        absn = np.linalg.norm([[sum(abs(Hs[a][m][tuple(d for d in range(3) for _ in range(t[d]))])
                                    for a in range(len(e)) if gid[a] == g)
                                for g in range(gid.max() + 1)] for t in ts])
        if absn == 0:
            continue
        assert np.allclose(M[row:row + len(ts)], comp / absn, rtol=0, atol=1e-13)
        row += len(ts)
    assert row == M.shape[0]


def test_symmetry_groups():
    """(3, 0, 0) and (2, 2, 1) share |xi|^2 but not a group (Sect. III)."""
    e = np.array([p for v in ((3, 0, 0), (2, 2, 1)) for p in
                  {tuple(s * x for s, x in zip(sg, perm))
                   for perm in itertools.permutations(v)
                   for sg in itertools.product((1, -1), repeat=3)}])
    gid = dvm.symmetry_groups(e)
    assert gid.max() == 1 and np.sum(gid == 0) == 6 and np.sum(gid == 1) == 24
    with pytest.raises(ValueError):
        dvm.symmetry_groups(e[1:])


@pytest.mark.parametrize("name", [n for n in ALL if n not in AUGMENTED])
def test_null_space_gives_printed_weights(name):
    """Minimal and scattering stencils: dim ker K = 1 at the printed c, and
    the normalised null vector is the printed weight vector."""
    t = ALL[name]
    e, w, c = dvm.expand(t)
    ws, n = dvm.solve_weights(e, c, t["Q"])
    assert n == 1
    assert np.max(np.abs(ws / w - 1)) < 1e-8


@pytest.mark.parametrize("name", ["D2V16", "D2V33", "D2V32", "D3V15", "D3V79", "D2Q9", "D3Q19"])
def test_find_c_recovers_printed_speed(name):
    """From the velocities alone: the lattice speed at which K(S) becomes
    singular with positive weights (Eq. dimker) is the printed c."""
    t = ALL[name]
    e, _, c = dvm.expand(t)
    cs = dvm.find_c(e, t["Q"], 0.8 * c, 1.2 * c)
    assert cs is not None and abs(cs / c - 1) < 1e-12


@pytest.mark.parametrize("name", ["D2V16", "D3V38a", "D2Q9"])
def test_regular_away_from_c_star(name):
    """For c != c*, K(S) is regular: no weights of order Q exist."""
    t = ALL[name]
    e, _, c = dvm.expand(t)
    _, n = dvm.solve_weights(e, 1.05 * c, t["Q"])
    assert n == 0
    assert dvm.orth_gap(e, 1.05 * c, t["Q"]) > 1e-6


@pytest.mark.parametrize("name", AUGMENTED)
def test_augmented_sets_from_wall_condition(name):
    """The augmented S3 stencils have a two-dimensional null space; imposing
    the wall moment W_zxx (m = (2, 0, 1), Eq. wallCond) with sum w = 1 gives
    the printed weights, and W_zxx is then exact."""
    t = ALL[name]
    e, w, c = dvm.expand(t)
    basis, _, _ = dvm.null_space(e, c, t["Q"])
    assert basis.shape[1] == 2
    moms = dvm.nontrivial_moments(3, t["Q"])
    k = moms.index((2, 0, 1))
    wa, res = dvm.augment(e, c, t["Q"], [k])
    assert res < 1e-12
    assert np.max(np.abs(wa / w - 1)) < 1e-9
    assert abs(dict(dvm.wall_errors(e, wa, c, 7))[(2, 0, 1)]) < 1e-12
