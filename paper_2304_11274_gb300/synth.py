"""Seeded synthetic inputs for the TPFA assembly (no method arithmetic here).

This module is shared by the CUDA path's tests and benchmark and by the oracle
checks, so it holds only input construction: grid shapes, rock fields,
pressure fields and cotangent vectors.  It computes no density, flux,
transmissibility or residual.

The paper publishes no geomodel (Section 7 gives only the 750 x 994 x 246 grid
shape), so every workload here is synthetic:

* permeability: log10 k ~ N(-13, 0.5) m^2, i.i.d. per cell, isotropic; or the
  layered high-contrast medium, log10 k ~ U[-18, -12] per z-layer;
* porosity phi0 ~ U[0.1, 0.3];
* cells of 10 x 10 x 2 m; depth of cell (i, j, k) = (k + 1/2) dz (z grows
  downward, layer k = 0 on top);
* pressure: 1e7 Pa at the top cell centre plus a hydrostatic gradient at the
  reference density, rho_ref g (depth - dz/2), plus U[-1e5, 1e5] per cell; the
  previous-time-step pressure p^n is the same field without the perturbation;
* the layered precision-study field: 5e6 + 2.5e7 k/(nz-1) + U[-1e5, 1e5],
  clipped to [5e6, 3e7], with p^n the noise-free field.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 20230422

# Physical constants of the workloads (SI units).
PHYSICS = dict(
    rho_ref=1000.0,   # kg/m^3
    p_ref=1.0e7,      # Pa
    c_f=4.5e-10,      # 1/Pa
    mu=1.0e-3,        # Pa s
    g=9.81,           # m/s^2
    dt=86400.0,       # s
    c_r=0.0,          # 1/Pa, constant porosity unless a test sets it
    dx=10.0, dy=10.0, dz=2.0,  # m
    connectivity=10,
)


def physics(**over) -> dict:
    d = dict(PHYSICS)
    d.update(over)
    return d


@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    phys: dict
    perm: np.ndarray   # (N,) float64, m^2
    poro: np.ndarray   # (N,) float64
    depth: np.ndarray  # (N,) float64, m, positive down
    p: np.ndarray      # (N,) float64, Pa
    pn: np.ndarray     # (N,) float64, Pa (previous time step)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def depth_field(nx, ny, nz, dz):
    k = np.arange(nz, dtype=np.float64)
    z = (k + 0.5) * dz
    return np.broadcast_to(z[:, None, None], (nz, ny, nx)).reshape(-1).copy()


def make_problem(nx, ny, nz, seed, *, connectivity=10, layered=False, layered_pressure=False,
                 perturb=1.0e5, **phys_over) -> Problem:
    """A seeded problem with the paper-shaped distributions described above.
    Cell (i, j, k) is element i + nx (j + ny k) of every field."""
    rng = np.random.default_rng(seed)
    phys = physics(connectivity=connectivity, **phys_over)
    N = nx * ny * nz
    if layered:
        lk = rng.uniform(-18.0, -12.0, size=nz)
        log10k = np.broadcast_to(lk[:, None, None], (nz, ny, nx)).reshape(-1)
    else:
        log10k = rng.normal(-13.0, 0.5, size=N)
    perm = np.power(10.0, log10k)
    poro = rng.uniform(0.1, 0.3, size=N)
    depth = depth_field(nx, ny, nz, phys["dz"])
    if layered_pressure:
        kk = np.repeat(np.arange(nz, dtype=np.float64), nx * ny)
        base = 5.0e6 + 2.5e7 * kk / max(nz - 1, 1)
        noise = rng.uniform(-perturb, perturb, size=N)
        p = np.clip(base + noise, 5.0e6, 3.0e7)
        pn = base.copy()
    else:
        base = 1.0e7 + phys["rho_ref"] * phys["g"] * (depth - 0.5 * phys["dz"])
        p = base + rng.uniform(-perturb, perturb, size=N)
        pn = base.copy()
    return Problem(nx, ny, nz, phys, perm, poro, depth, p, pn)


def pressure_sequence(prob: Problem, count: int, seed: int, perturb=1.0e5):
    """`count` further pressure vectors around p^n (distinct perturbations),
    for the repeated-application protocol of Section 3 (a new pressure vector
    at every call)."""
    rng = np.random.default_rng(seed)
    return [prob.pn + rng.uniform(-perturb, perturb, size=prob.n) for _ in range(count)]


def cotangent(n, seed):
    """v ~ N(0, 1), the random cotangent of the adjoint workload."""
    return np.random.default_rng(seed).standard_normal(n)


def ensemble_shapes(count=64, seed=BASE_SEED + 3, nxy=(64, 256), nz=(32, 128)):
    """Grid shapes of the uneven ensemble: nx, ny ~ U{64..256}, nz ~ U{32..128}."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(nxy[0], nxy[1] + 1)), int(rng.integers(nxy[0], nxy[1] + 1)),
             int(rng.integers(nz[0], nz[1] + 1))) for _ in range(count)]


def round_to_f32(prob: Problem) -> Problem:
    """The same problem with every field that the mixed path stores in FP32
    (pressure, depth) rounded to FP32 and widened back, so that an FP64
    evaluation sees exactly the values the mixed path sees."""
    r = lambda a: a.astype(np.float32).astype(np.float64)
    return dataclasses.replace(prob, p=r(prob.p), pn=r(prob.pn), depth=r(prob.depth))


# The five workloads: (nx, ny, nz, connectivity, precision, extra).
CONFIGS = {
    0: dict(shape=(32, 32, 32), connectivity=6, precision="fp64", layered=False),
    1: dict(shape=(512, 512, 256), connectivity=10, precision="mixed", layered=False),
    2: dict(shape=(256, 256, 256), connectivity=10, precision="both", layered=True),
    3: dict(shape=None, connectivity=10, precision="mixed", layered=False),
    4: dict(shape=(128, 128, 128), connectivity=10, precision="mixed", layered=False),
}


def config_problem(idx: int, shape=None) -> Problem:
    c = CONFIGS[idx]
    nx, ny, nz = shape if shape is not None else c["shape"]
    return make_problem(nx, ny, nz, BASE_SEED + idx, connectivity=c["connectivity"],
                        layered=c["layered"], layered_pressure=c["layered"])
