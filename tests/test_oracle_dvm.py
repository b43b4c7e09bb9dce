"""Pins of the oracle's DVM code against what the paper prints.

Each printed table (App. A, App. B) must expand to V velocities with
sum w = 1, integrate Gaussian moments exactly up to its stated order Q and
no further (Eq. orth), have the stated energy E (Eq. Ssymbol), and reproduce
the printed wall-moment errors (Tab. bulk, Wzxx, W0) and wall accuracy
indices (Eq. lambdaS3, lambdaS4, App. B).
"""
import math
import os

import numpy as np
import pytest

from lbm_inputs import DVM_TABLES, TEXTBOOK_TABLES
from oracle import dvm

ALL = {**DVM_TABLES, **TEXTBOOK_TABLES}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name", sorted(ALL))
def test_table_sum_degree_energy(name):
    t = ALL[name]
    e, w, c = dvm.expand(t)
    assert len(e) == t["V"]
    assert abs(w.sum() - 1.0) < 1e-12
    assert (w > 0).all()
    assert dvm.quadrature_order(e, w, c) == t["Q"]
    # exactly Q: the first moment past Q must fail clearly, not marginally
    assert dvm.moment_error(e, w, c, t["Q"] + 1) > 1e-6
    assert dvm.energy(e) == t["E"]


def test_gaussian_moments_closed_form():
    # (m-1)!!: 1, 1, 3, 15, 105 for m = 0, 2, 4, 6, 8 (textbook normal moments)
    assert [dvm.gaussian_moment_1d(m) for m in (0, 1, 2, 3, 4, 6, 8)] == \
        [1.0, 0.0, 1.0, 0.0, 3.0, 15.0, 105.0]


def test_wall_moment_closed_form_matches_numerical_integral():
    """Eq. Wscalar against a direct numerical half-space integral."""
    from scipy import integrate
    for D, (mx, my, mz) in [(3, (0, 0, 0)), (3, (2, 0, 1)), (3, (2, 2, 3)),
                             (2, (4, 0, 1)), (2, (0, 0, 7)), (2, (6, 0, 0))]:
        f1 = lambda x, m: x ** m * math.exp(-x * x / 2) / math.sqrt(2 * math.pi)
        ix = integrate.quad(f1, -np.inf, np.inf, args=(mx,))[0]
        iz = integrate.quad(f1, 0, np.inf, args=(mz,))[0]
        iy = integrate.quad(f1, -np.inf, np.inf, args=(my,))[0] if D == 3 else 1.0
        assert math.isclose(dvm.wall_moment_exact(D, mx, my, mz), ix * iy * iz,
                            rel_tol=1e-10)


def test_nontrivial_moment_lists():
    """L = 19 (3D, Q = 7) in the order of Eq. defT; L = 14 in 2D (Eq. defT2D)."""
    l3 = dvm.nontrivial_moments(3, 7)
    assert len(l3) == 19
    assert l3[:7] == [(0, 0, 0), (0, 0, 1), (2, 0, 0), (0, 0, 3), (2, 0, 1),
                      (4, 0, 0), (2, 2, 0)]
    assert l3[-6:] == [(0, 0, 7), (2, 0, 5), (4, 0, 3), (2, 2, 3), (6, 0, 1),
                       (4, 2, 1)]
    l2 = dvm.nontrivial_moments(2, 7)
    assert len(l2) == 14
    assert l2 == [(0, 0, 0), (0, 0, 1), (2, 0, 0), (0, 0, 3), (2, 0, 1), (4, 0, 0),
                  (0, 0, 5), (2, 0, 3), (4, 0, 1), (6, 0, 0), (0, 0, 7), (2, 0, 5),
                  (4, 0, 3), (6, 0, 1)]


def _golden_rows(fname):
    rows = []
    with open(os.path.join(GOLDEN, fname)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


COLS = {"sigma": (0, 0, 0), "sigma_z": (0, 0, 1), "sigma_xx": (2, 0, 0),
        "sigma_zxx": (2, 0, 1), "sigma_zzzxx": (2, 0, 3), "sigma_xxzzzzz": (2, 0, 5)}


@pytest.mark.parametrize("row", _golden_rows("wall_errors.txt"), ids=lambda r: r[0])
def test_printed_wall_errors(row):
    name = row[0]
    t = ALL[name]
    e, w, c = dvm.expand(t)
    errs = dvm.wall_errors(e, w, c, t["Q"])   # sigma_Sigma sums n <= Q
    by_m = dict(errs)
    for col, val in zip(["sigma", "sigma_z", "sigma_xx", "sigma_zxx", "sigma_zzzxx",
                         "sigma_xxzzzzz"], row[2:8]):
        if val == "-":
            continue
        got = by_m[COLS[col]]
        if val.startswith("~"):
            assert abs(abs(got) - abs(float(val[1:]))) <= 5e-5, (col, got, val)
        else:
            assert abs(got - float(val)) <= 5e-5 + 1e-12, (col, got, val)
    assert abs(dvm.sigma_sigma(errs) - float(row[8])) <= 5e-5


def test_intro_example_wall_errors():
    """Intro (Sect. I): W_zxx error about 28 % for D3Q19 and 2 % for D3V15."""
    for name, expect in (("D3Q19", 0.28), ("D3V15", 0.02)):
        e, w, c = dvm.expand(ALL[name])
        s = dict(dvm.wall_errors(e, w, c, 5))[(2, 0, 1)]
        assert round(abs(s), 2) == expect


@pytest.mark.parametrize("row", _golden_rows("lambda_index.txt"), ids=lambda r: r[0])
def test_printed_lambda_index(row):
    name, expect = row[0], int(row[1])
    t = ALL[name]
    e, w, c = dvm.expand(t)
    assert dvm.lambda_index(dvm.wall_errors(e, w, c, min(t["Q"], 7))) == expect


def test_scattering_sets_have_exact_even_wall_moments():
    """Eq. S4prop: no wall-parallel velocity => every even wall moment exact."""
    for name in ("D2V32", "D3V96", "D3V112"):
        e, w, c = dvm.expand(ALL[name])
        assert (e[:, -1] != 0).all()
        for m, s in dvm.wall_errors(e, w, c, 7):
            if m[2] == 0:
                assert abs(s) < 1e-12


@pytest.mark.parametrize("name,V", [("D3V107", 53), ("D3V96", 40), ("D3V112", 48),
                                    ("D3V77", 37), ("D3V66", 41)])
def test_xz_marginal_keeps_degree_and_wall_errors(name, V):
    """The (x, z) marginal of a 3D set keeps every moment without xi_y, so it
    keeps the quadrature order and the (x, z) wall errors of the 3D set."""
    e3, w3, c = dvm.expand(DVM_TABLES[name])
    e, w = dvm.marginal_xz(e3, w3)
    assert len(e) == V
    assert dvm.quadrature_order(e, w, c) == 7
    s3 = dict(dvm.wall_errors(e3, w3, c, 7))
    for m, s in dvm.wall_errors(e, w, c, 7):
        assert abs(s - s3[m]) < 1e-12


def test_symmetric_pairs():
    """Every 2D set used by the channel is closed under e -> -e with equal
    weights (needed by the wall flux balance: denominators of both walls)."""
    for name in ("D2V16", "D2V33", "D2V32", "D3V107xz", "D3V96xz", "D3V112xz"):
        e, w, c = dvm.dvm2d(name, DVM_TABLES)
        lut = {tuple(v): wa for v, wa in zip(e.tolist(), w.tolist())}
        for v, wa in lut.items():
            assert lut[(-v[0], -v[1])] == wa
