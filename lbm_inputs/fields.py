"""Seeded synthetic inputs for channel solves.

The paper's runs are force-driven plane Poiseuille channels (Sect. VI):
uniform density, fluid at rest, a small constant body force.  Its lattice
resolution and DSMC comparison data are not available, so every workload
here is synthetic: the shapes follow the channel runs and the random
numbers come from numpy's PCG64 generator with fixed seeds.
"""
import numpy as np


def rho_field(Nx, Ny, seed=20151029, amplitude=1e-3):
    """Initial density rho(x, y) = 1 + amplitude * N(0, 1) per node.

    Returned as a C-contiguous float64 array of shape (Ny, Nx) (row-major,
    x fastest).  ``amplitude=0`` gives the uniform rest density of the
    paper's Poiseuille runs.
    """
    if amplitude == 0.0:
        return np.ones((Ny, Nx), dtype=np.float64)
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.standard_normal((Ny, Nx))


def kn_sweep(points=8, lo=0.01, hi=1.0):
    """Knudsen numbers log-spaced over [lo, hi] (8 points by default)."""
    k = np.arange(points)
    return lo * (hi / lo) ** (k / (points - 1))


def batch_workload(n=256, seed=20151030, dvms=("D2V33", "D3V107xz"),
                   orders=(4, 3), ny_range=(16, 512), nx_choices=(1, 64, 256),
                   kn_range=(0.01, 1.0)):
    """Seeded list of independent channel solves of uneven sizes.

    Each item is a dict with keys dvm, order, Nx, Ny, Kn.  The DVM is drawn
    50/50 from ``dvms`` with the Hermite order from ``orders``; Ny is uniform
    on the closed integer range, Nx is drawn from ``nx_choices`` and Kn is
    log-uniform on ``kn_range``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        j = int(rng.integers(0, len(dvms)))
        out.append(dict(dvm=dvms[j], order=int(orders[j]),
                        Nx=int(rng.choice(nx_choices)),
                        Ny=int(rng.integers(ny_range[0], ny_range[1] + 1)),
                        Kn=float(np.exp(rng.uniform(np.log(kn_range[0]),
                                                    np.log(kn_range[1]))))))
    return out


def serving_workload(duration_s=60.0, rate_hz=200.0, seed=20151031,
                     dvm="D2V16", order=3, ny_range=(16, 2048),
                     kn_range=(0.01, 1.0), tolerances=(1e-6, 1e-8)):
    """Seeded Poisson stream of channel-solve requests.

    Returns a list of dicts (t_arrival [s], dvm, order, Nx=1, Ny, Kn, tol),
    arrivals with exponential gaps of mean 1/rate_hz up to ``duration_s``.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        out.append(dict(t_arrival=t, dvm=dvm, order=order, Nx=1,
                        Ny=int(rng.integers(ny_range[0], ny_range[1] + 1)),
                        Kn=float(np.exp(rng.uniform(np.log(kn_range[0]),
                                                    np.log(kn_range[1])))),
                        tol=float(rng.choice(tolerances))))
    return out
