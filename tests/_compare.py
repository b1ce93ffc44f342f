"""Comparison helpers for the GPU-vs-oracle parity tests: the error
measures and the oracle reference with admissible upwind alternatives live
in oracle/compare.py (shared with the benchmark's precision statement);
this module adds the problems built to contain exact ties."""
from __future__ import annotations

import numpy as np

from oracle.compare import *  # noqa: F401,F403
from oracle.compare import EPS32, EPS64, ambiguous_links, entry_stats, jacobian_row_error, reference, \
    residual_error, subgrid_row  # noqa: F401
from paper_2304_11274_gb300 import synth


def tie_sweep_problem(precision, conn=10):
    """Exact ties dPhi == 0 on links the tiled kernel reuses from the previous
    y-row: row j = 0 at p = p_ref = 0 (rho = rho_ref exactly) and depth 1 m,
    row j = 1 at depth 3 m with g = 0.5 (so g dz = -1 exactly and dPhi =
    rho_avg - p_1), its pressures sweeping 4096 consecutive representable
    values around the root of p_1 = rho_avg(p_1).  Over the sweep rho_avg
    stays one representable value (c_f = 1e-6 moves it by far less than an
    ulp), so exactly one p_1 of the sweep equals it: there the y-link and
    both diagonal links into that cell are exact ties, in either precision."""
    dt = np.float32 if precision == "mixed" else np.float64
    nx, ny, nz = 4096, 2, 1
    phys = synth.physics(connectivity=conn, p_ref=0.0, c_f=1e-6, g=0.5, c_r=0.0)
    r = dt(1000.0)
    for _ in range(60):  # fixed point p = (rho_ref + rho(p)) / 2 in the path's precision
        r = dt(0.5) * (dt(1000.0) + dt(1000.0) * dt(np.exp(dt(1e-6) * r)))
    sweep = [r]
    lo = hi = r
    for _ in range(nx // 2):
        lo = np.nextafter(lo, dt(-np.inf))
        hi = np.nextafter(hi, dt(np.inf))
        sweep = [lo] + sweep + [hi]
    p1 = np.array(sweep[:nx], dtype=np.float64)
    p = np.concatenate([np.zeros(nx), p1])
    depth = np.concatenate([np.full(nx, 1.0), np.full(nx, 3.0)])
    rng = np.random.default_rng(9)
    perm = np.full(nx * ny * nz, 1e-13)
    poro = rng.uniform(0.1, 0.3, nx * ny * nz)
    return synth.Problem(nx, ny, nz, phys, perm, poro, depth, p, p.copy())


def tie_pairs_problem(precision, conn=10, shape=(130, 37, 5), seed=31, frac=0.15):
    """Exact ties dPhi == 0 on in-plane links of every direction: a random
    problem in which a fraction of the cells take the pressure of one of
    their in-plane neighbours (x, y or diagonal, chosen at random).  Both
    cells of such a pair lie in one plane (same depth), so the link's dPhi
    is exactly zero in either precision.  The pairs fall inside a lane's two
    cells, across lanes and across segments alike."""
    prob = synth.make_problem(*shape, seed=seed, connectivity=conn)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    nx, ny, nz = shape
    rng = np.random.default_rng(seed + 1)
    p = prob.p.reshape(nz, ny, nx).copy()
    dirs = [(1, 0), (-1, 0), (0, 1), (0, -1)] + ([(1, 1), (-1, -1), (1, -1), (-1, 1)] if conn == 10 else [])
    for _ in range(int(frac * nx * ny * nz)):
        k, j, i = rng.integers(nz), rng.integers(ny), rng.integers(nx)
        di, dj = dirs[rng.integers(len(dirs))]
        if 0 <= i + di < nx and 0 <= j + dj < ny:
            p[k, j + dj, i + di] = p[k, j, i]
    prob.p = p.reshape(-1)
    return prob
