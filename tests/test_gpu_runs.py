"""A run description executed on the GPU: config 1 through the command line,
recorded as JSON lines, against the oracle."""
import json

import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build_library()


def test_config1_run_recorded(tmp_path):
    from paper_1510_08886_gb300 import runs
    cfg = {"dvm": "D2V16", "order": 3, "Nx": 1, "Ny": 64, "Kn": 0.1, "precision": "fp64"}
    (tmp_path / "c.json").write_text(json.dumps([cfg, dict(cfg, precision="fp32")]))
    log = tmp_path / "runs.jsonl"
    assert runs.main([str(tmp_path / "c.json"), "--log", str(log)]) == 0
    recs = [json.loads(l) for l in log.read_text().splitlines()]
    assert len(recs) == 2 and all(r["converged"] and r["status"] == 0 for r in recs)
    ref = oracle.channel("D2V16", 3, 1, 64, 0.1, oracle.force_for_mach(0.1)).init()
    ref.run_to_steady(1e-10, 50000)
    assert abs(recs[0]["mass_flow"] / ref.mass_flow() - 1) < 1e-12
    assert abs(recs[1]["mass_flow"] / ref.mass_flow() - 1) < 1e-4
