"""Run descriptions and run records for channel solves.

A ``SolveConfig`` is a complete, JSON-serialisable description of one channel
solve (velocity set, Hermite order, grid, Knudsen number, forcing, storage
precision, convergence test, initial density perturbation).  ``run`` executes
it on the GPU through ``Solver`` and returns a ``RunRecord``; ``append_jsonl``
writes the record as one line of a JSON-lines log.  The module holds no
arithmetic of the method: it only marshals arguments to the library.

Command line:  python -m paper_1510_08886_gb300.runs CONFIG.json [--log runs.jsonl]
where CONFIG.json holds one config object or a list of them.
"""
import dataclasses
import json
import math
import os
import sys
import time

PRECISIONS = ("fp64", "fp32", "fp16", "bf16")


@dataclasses.dataclass
class SolveConfig:
    dvm: str = "D2V33"            # a velocity set known to ``dvm()`` (table name or '<3D>xz')
    order: int = 4                # Hermite order N of the equilibrium (Eq. nm.3)
    Nx: int = 1                   # periodic nodes along the channel
    Ny: int = 64                  # nodes between the walls
    Kn: float = 0.1               # Knudsen number; tau = sqrt(2/pi) Kn (Eq. nm.13)
    mach: float = 1e-3            # body force g = 8 tau mach (no-slip centre speed mach c0)
    precision: str = "fp64"       # storage / arithmetic: fp64, fp32, fp16, bf16
    tol: float = 1e-10            # convergence: max |u_x(t) - u_x(t - dt)| < tol
    max_steps: int = 50000
    check_every: int = 100
    seed: int = -1                # >= 0: rho = 1 + amplitude N(0, 1) from numpy's PCG64(seed)
    amplitude: float = 1e-3

    def validate(self):
        """Raise ValueError for a config the library would reject or that is
        malformed; the velocity set's own checks happen in the library."""
        if self.precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {PRECISIONS}")
        if self.order not in (2, 3, 4):
            raise ValueError("order must be 2, 3 or 4")
        if self.Nx < 1 or self.Ny < 1:
            raise ValueError("Nx and Ny must be >= 1")
        if not (self.Kn > 0 and math.isfinite(self.Kn)):
            raise ValueError("Kn must be a positive finite number")
        if not math.isfinite(self.mach):
            raise ValueError("mach must be finite")
        if not (self.tol > 0) or self.max_steps < 0 or self.check_every < 2:
            raise ValueError("need tol > 0, max_steps >= 0, check_every >= 2")
        if self.seed >= 0 and not (self.amplitude >= 0 and math.isfinite(self.amplitude)):
            raise ValueError("amplitude must be finite and >= 0")
        return self

    def to_json(self):
        return json.dumps(dataclasses.asdict(self), sort_keys=True)

    @classmethod
    def from_dict(cls, d):
        known = {f.name for f in dataclasses.fields(cls)}
        unknown = set(d) - known
        if unknown:
            raise ValueError(f"unknown config keys: {sorted(unknown)}")
        return cls(**d).validate()

    @classmethod
    def from_json(cls, text):
        return cls.from_dict(json.loads(text))


@dataclasses.dataclass
class RunRecord:
    config: dict
    converged: bool
    steps: int
    last_du: float
    mass_flow: float              # Eq. pf.1
    slip_velocity: float          # Eq. defSlip
    status: int                   # library status word (0: all densities finite and positive)
    seconds: float                # host wall time of the solve (init excluded)
    glups: float                  # node updates per second / 1e9
    host_cores: int

    def to_json(self):
        return json.dumps(dataclasses.asdict(self), sort_keys=True)


def _initial_density(cfg):
    if cfg.seed < 0:
        return None
    import numpy as np
    rng = np.random.default_rng(cfg.seed)
    return 1.0 + cfg.amplitude * rng.standard_normal((cfg.Ny, cfg.Nx))


def run(cfg):
    """Run one config to its convergence test on the GPU; returns a RunRecord."""
    import paper_1510_08886_gb300 as lbm
    cfg.validate()
    e, w, c = lbm.dvm(cfg.dvm)
    s = lbm.Solver(e, w, c, cfg.order, cfg.Nx, cfg.Ny, cfg.Kn,
                   lbm.force_for_mach(cfg.Kn, cfg.mach), precision=cfg.precision)
    try:
        s.init(_initial_density(cfg))
        t0 = time.perf_counter()
        conv, steps, du = s.run_to_steady(cfg.tol, cfg.max_steps, cfg.check_every)
        dt = time.perf_counter() - t0
        return RunRecord(config=dataclasses.asdict(cfg), converged=bool(conv), steps=int(steps),
                         last_du=float(du), mass_flow=float(s.mass_flow()),
                         slip_velocity=float(s.slip_velocity()), status=int(s.status()),
                         seconds=dt, glups=cfg.Nx * cfg.Ny * steps / dt / 1e9 if dt > 0 else 0.0,
                         host_cores=os.cpu_count() or 1)
    finally:
        s.close()


def append_jsonl(path, record):
    with open(path, "a") as fh:
        fh.write(record.to_json() + "\n")


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("config", help="JSON file: one config object or a list")
    ap.add_argument("--log", default=None, help="append one JSON line per run here")
    a = ap.parse_args(argv)
    with open(a.config) as fh:
        data = json.load(fh)
    configs = [SolveConfig.from_dict(d) for d in (data if isinstance(data, list) else [data])]
    for cfg in configs:
        rec = run(cfg)
        print(rec.to_json(), flush=True)
        if a.log:
            append_jsonl(a.log, rec)
    return 0


if __name__ == "__main__":
    sys.exit(main())
