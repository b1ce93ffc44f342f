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


# ---------------------------------------------------------------- general meshes


@dataclasses.dataclass
class Mesh:
    """A mesh given as a connection list (cell indices ci[c], cj[c] and the
    transmissibility T[c] of connection c) with per-cell fields."""
    n: int
    phys: dict
    ci: np.ndarray     # (nc,) int64
    cj: np.ndarray     # (nc,) int64
    T: np.ndarray      # (nc,) float64, m^3
    V: np.ndarray      # (n,) float64, m^3
    poro: np.ndarray
    depth: np.ndarray
    p: np.ndarray
    pn: np.ndarray

    @property
    def nc(self) -> int:
        return int(self.ci.size)


def structured_pairs(nx, ny, nz, connectivity):
    """Cell pairs of a structured grid's links, each listed once from its
    owner: +x, +y, +z, and with 10 links (+x,+y) and (-x,+y).  Returns linear
    indices (a, b) and the link kind 0..4 in that order.  Topology only."""
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="xy")
    i, j, k = (np.moveaxis(x, 2, 0).reshape(-1) for x in (i, j, k))
    lin = i + nx * (j + ny * k)
    out_a, out_b, out_k = [], [], []
    steps = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if connectivity == 10:
        steps += [(1, 1, 0), (-1, 1, 0)]
    for kind, (di, dj, dk) in enumerate(steps):
        ok = (i + di >= 0) & (i + di < nx) & (j + dj < ny) & (k + dk < nz)
        out_a.append(lin[ok])
        out_b.append((i + di + nx * (j + dj + ny * (k + dk)))[ok])
        out_k.append(np.full(int(ok.sum()), kind))
    return np.concatenate(out_a), np.concatenate(out_b), np.concatenate(out_k)


def make_mesh(nx, ny, nz, seed, *, connectivity=6, fault=True, inactive=0.05, perturb=1.0e5, **phys_over) -> Mesh:
    """A corner-point-like mesh with a fault, the kind of topology the paper
    defers to future work: the cells of a structured nx x ny x nz grid, the
    block x >= nx/2 thrown down by half a layer (so the faces across the
    fault become two non-neighbour connections per cell, to the cells at the
    same and at the next shallower layer), a fraction of inactive (pinched-
    out) cells removed with their connections, and per-cell volumes varying
    by +-20 %.  Transmissibilities are drawn directly, log10 T ~ N(-12.7, 0.5)
    m^3 (the magnitude of a 1e-13 m^2 face of 10 x 10 x 2 m cells); the rest
    follows make_problem's distributions.  Active cells keep the structured
    (x fastest) order."""
    rng = np.random.default_rng(seed)
    phys = physics(connectivity=connectivity, **phys_over)
    dz = phys["dz"]
    N = nx * ny * nz
    i = np.tile(np.arange(nx), ny * nz)
    k = np.repeat(np.arange(nz), nx * ny)
    xf = nx // 2 if (fault and nx >= 2) else nx
    depth_all = (k + 0.5) * dz + np.where(i >= xf, 0.5 * dz, 0.0)
    a, b, kind = structured_pairs(nx, ny, nz, connectivity)
    if xf < nx:
        ia, ib = a % nx, b % nx
        crosses = (np.minimum(ia, ib) < xf) & (np.maximum(ia, ib) >= xf)
        a, b = a[~crosses], b[~crosses]
        left = np.flatnonzero(i == xf - 1)
        a = np.concatenate([a, left, left[k[left] >= 1]])
        b = np.concatenate([b, left + 1, left[k[left] >= 1] + 1 - nx * ny])
    active = rng.random(N) >= inactive
    if not active.any():
        active[0] = True
    keep = active[a] & active[b]
    a, b = a[keep], b[keep]
    idx = np.cumsum(active) - 1
    ci, cj = idx[a].astype(np.int64), idx[b].astype(np.int64)
    n = int(active.sum())
    T = np.power(10.0, rng.normal(-12.7, 0.5, size=ci.size))
    V = phys["dx"] * phys["dy"] * dz * rng.uniform(0.8, 1.2, size=n)
    poro = rng.uniform(0.1, 0.3, size=n)
    depth = depth_all[active]
    base = 1.0e7 + phys["rho_ref"] * phys["g"] * (depth - 0.5 * dz)
    p = base + rng.uniform(-perturb, perturb, size=n)
    return Mesh(n, phys, ci, cj, T, V, poro, depth, p, base.copy())


def round_mesh_to_f32(m: Mesh) -> Mesh:
    """The mesh with the fields the mixed path stores in FP32 (pressure,
    depth, transmissibility) rounded to FP32 and widened back."""
    r = lambda x: x.astype(np.float32).astype(np.float64)
    return dataclasses.replace(m, p=r(m.p), pn=r(m.pn), depth=r(m.depth), T=r(m.T))


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
