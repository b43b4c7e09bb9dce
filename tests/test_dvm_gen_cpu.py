"""The library's DVM generator (host code behind the C ABI) against the
oracle and the paper's printed tables: weights from the velocities alone
(Sect. III), the lattice speed c* of minimal DVMs (Eq. dimker), the wall
augmentation of Sect. IV, and the argument checks.  No GPU is involved."""
import numpy as np
import pytest

from lbm_inputs import DVM_TABLES, TEXTBOOK_TABLES
from oracle import dvm as odvm

ALL = {**DVM_TABLES, **TEXTBOOK_TABLES}
AUGMENTED = ("D3V77", "D3V107")


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_1510_08886_gb300 as m
    return m


@pytest.mark.parametrize("name", list(ALL))
def test_weights_and_nullity_match_oracle_and_tables(lbm, name):
    t = ALL[name]
    e, w, c = odvm.expand(t)
    wl, n = lbm.dvm_weights(e, c, t["Q"])
    _, no, _ = odvm.null_space(e, c, t["Q"])
    wo, n_oracle = odvm.solve_weights(e, c, t["Q"])
    assert n == n_oracle == (2 if name in AUGMENTED else 1)
    if n == 1:
        assert np.max(np.abs(wl / w - 1)) < 1e-10           # printed weights
        assert np.max(np.abs(wl / wo - 1)) < 1e-8            # oracle (K null space)
        assert abs(np.sum(wl) - 1) < 1e-14
    else:
        assert wl is None


@pytest.mark.parametrize("name", [n for n in ALL if n not in AUGMENTED])
def test_find_c_matches_printed_speed_and_oracle(lbm, name):
    t = ALL[name]
    e, _, c = odvm.expand(t)
    cl = lbm.dvm_find_c(e, t["Q"], 0.8 * c, 1.2 * c)
    assert cl is not None and abs(cl / c - 1) < 1e-12
    if name in ("D2V16", "D2V33", "D3V15", "D2Q9"):
        co = odvm.find_c(e, t["Q"], 0.8 * c, 1.2 * c)
        assert abs(cl / co - 1) < 1e-12


def test_find_c_none_without_root(lbm):
    e, _, c = odvm.expand(ALL["D2V16"])
    assert lbm.dvm_find_c(e, 7, 1.05 * c, 1.2 * c) is None


@pytest.mark.parametrize("name", AUGMENTED)
def test_augmentation_matches_oracle_and_tables(lbm, name):
    t = ALL[name]
    e, w, c = odvm.expand(t)
    moms = lbm.dvm_nontrivial_moments(3, t["Q"])
    assert moms == [tuple(m) for m in odvm.nontrivial_moments(3, t["Q"])]
    k = [moms.index((2, 0, 1))]
    wl, res = lbm.dvm_augment(e, c, t["Q"], k)
    wo, _ = odvm.augment(e, c, t["Q"], k)
    assert res < 1e-12
    assert np.max(np.abs(wl / w - 1)) < 1e-10
    assert np.max(np.abs(wl / wo - 1)) < 1e-9


def test_augmentation_overdetermined_least_squares(lbm):
    """All 19 wall moments of Q = 7 on a two-dimensional null space: the
    least-squares residual equals the oracle's."""
    t = ALL["D3V107"]
    e, _, c = odvm.expand(t)
    k = list(range(len(odvm.nontrivial_moments(3, 7))))
    _, rl = lbm.dvm_augment(e, c, 7, k)
    _, ro = odvm.augment(e, c, 7, k)
    assert rl > 1e-3 and abs(rl / ro - 1) < 1e-8


@pytest.mark.parametrize("D,Q", [(2, 7), (2, 9), (3, 7), (3, 9)])
def test_nontrivial_moment_lists(lbm, D, Q):
    assert lbm.dvm_nontrivial_moments(D, Q) == [tuple(m) for m in odvm.nontrivial_moments(D, Q)]


def test_regular_away_from_c_star_and_arguments(lbm):
    from paper_1510_08886_gb300 import _lib
    e, _, c = odvm.expand(ALL["D2V16"])
    w, n = lbm.dvm_weights(e, 1.05 * c, 7)
    assert n == 0 and w is None
    with pytest.raises(_lib.LBMError):
        lbm.dvm_augment(e, 1.05 * c, 7, [0])                  # K regular: LBM_EDEGREE
    with pytest.raises(_lib.LBMError):
        lbm.dvm_weights(e[1:], c, 7)                          # incomplete orbit
    with pytest.raises(_lib.LBMError):
        lbm.dvm_weights(e, -1.0, 7)
    with pytest.raises(_lib.LBMError):
        lbm.dvm_weights(e, c, 17)
    with pytest.raises(_lib.LBMError):
        lbm.dvm_augment(e, c, 7, [99])
    with pytest.raises(ValueError):
        lbm.dvm_weights(np.zeros((4, 4), dtype=int), c, 7)
