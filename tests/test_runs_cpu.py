"""Run descriptions without a GPU: JSON round trip, validation, the seeded
initial density, and the JSON-lines log."""
import json

import numpy as np
import pytest

from paper_1510_08886_gb300 import runs


def test_config_json_round_trip():
    cfg = runs.SolveConfig(dvm="D2V16", order=3, Nx=5, Ny=40, Kn=0.3, precision="fp32",
                           seed=7, amplitude=2e-3)
    back = runs.SolveConfig.from_json(cfg.to_json())
    assert back == cfg


@pytest.mark.parametrize("bad", [{"precision": "fp8"}, {"order": 5}, {"Ny": 0}, {"Kn": 0.0},
                                 {"Kn": float("inf")}, {"check_every": 1}, {"tol": 0.0},
                                 {"mach": float("nan")}])
def test_config_rejects_invalid(bad):
    with pytest.raises(ValueError):
        runs.SolveConfig.from_dict(bad)


def test_config_rejects_unknown_keys():
    with pytest.raises(ValueError, match="unknown"):
        runs.SolveConfig.from_dict({"Nz": 3})


def test_initial_density_is_seeded():
    cfg = runs.SolveConfig(Nx=4, Ny=6, seed=11, amplitude=1e-3)
    a, b = runs._initial_density(cfg), runs._initial_density(cfg)
    assert a.shape == (6, 4) and np.array_equal(a, b)
    assert np.max(np.abs(a - 1)) < 1e-2
    assert runs._initial_density(runs.SolveConfig(seed=-1)) is None


def test_jsonl_appends_one_line_per_record(tmp_path):
    rec = runs.RunRecord(config={"Ny": 8}, converged=True, steps=100, last_du=1e-11,
                         mass_flow=1.5, slip_velocity=0.2, status=0, seconds=0.01, glups=0.1,
                         host_cores=4)
    path = tmp_path / "runs.jsonl"
    runs.append_jsonl(path, rec)
    runs.append_jsonl(path, rec)
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[1])["steps"] == 100
