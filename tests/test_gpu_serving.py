"""Serving on the GPU: requests run to their tolerance with continuous
batching give the same result as the same request served alone (the
spec requirement), and agree with the fp64 oracle."""
import copy

import numpy as np
import pytest

import oracle
from paper_1510_08886_gb300.serving import ContinuousBatcher, Request

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build_library()


def _requests():
    rng = np.random.default_rng(99)
    out = []
    for i in range(10):
        out.append(Request(i, 0.0, "D2V16", 3, 1, int(rng.integers(16, 200)),
                           float(np.exp(rng.uniform(np.log(0.05), np.log(1.0)))),
                           float(rng.choice([1e-6, 1e-8]))))
    return out


def test_served_results_equal_alone_and_match_oracle():
    import paper_1510_08886_gb300 as lbm
    sets = {"D2V16": lbm.dvm("D2V16")}
    eng = lbm.Engine("fp32", max_solves=16, arena_bytes=64 << 20)
    mixed = ContinuousBatcher(eng, sets)
    reqs = _requests()
    st = mixed.serve(copy.deepcopy(reqs), realtime=False)
    assert st.completed == len(reqs)
    by_id = {r.rid: r for r in mixed.done}
    for r in reqs:
        solo_eng = lbm.Engine("fp32", max_solves=1, arena_bytes=16 << 20)
        solo = ContinuousBatcher(solo_eng, sets)
        solo.serve([copy.deepcopy(r)], realtime=False)
        a, b = by_id[r.rid], solo.done[0]
        assert a.converged and b.converged
        assert (a.steps, a.mdot, a.us) == (b.steps, b.mdot, b.us)
        solo_eng.close()
    for r in reqs[:3]:
        ref = oracle.channel("D2V16", 3, 1, r.Ny, r.Kn, r.force).init()
        ref.run_to_steady(r.tol, 200000, 100)
        got = by_id[r.rid]
        assert abs(got.mdot / ref.mass_flow() - 1) < 1e-4
