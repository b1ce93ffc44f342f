"""Comparison helpers for the GPU-vs-oracle parity tests.

Error measures (the paper gives none; these are the normwise readings):
  residual : ||R_gpu - R_ref||_inf / ||R_ref||_inf
  Jacobian : max over rows of ||J_gpu,i - J_ref,i||_inf / ||J_ref,i||_inf

Upwinding turns the sign of dPhi into a choice of density, so a link whose
dPhi lies within the rounding error of the path's arithmetic can legitimately
be upwinded either way: the flux is continuous there, its derivatives are
not.  Such links are found from the oracle's dPhi and a bound on the GPU's
rounding, the oracle is re-run with those links' upwind choice reversed, and
a GPU value is accepted if it matches either admissible evaluation.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2304_11274_gb300 import synth

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53


def ambiguous_links(prob, ref, eps, factor=32.0):
    """Boolean mask over CSR entries whose dPhi is within `factor * eps` of the
    magnitudes that form it."""
    rp, ci, dphi = ref["row_ptr"], ref["col_idx"], ref["dphi"]
    rows = np.repeat(np.arange(prob.n), np.diff(rp))
    off = ci != rows
    scale = (np.abs(prob.p[rows] - prob.p[ci]) +
             1.1 * prob.phys["rho_ref"] * abs(prob.phys["g"]) * np.abs(prob.depth[rows] - prob.depth[ci]))
    return off & (np.abs(dphi) <= factor * eps * scale)


def reference(prob, eps):
    """Oracle R, J for `prob` plus the alternative evaluation for ambiguous
    links (J_alt is None when there are none)."""
    pat = oracle.pattern(prob.nx, prob.ny, prob.nz, prob.phys["connectivity"])
    ref = oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                          prob.p, prob.pn, pat=pat, want_links=True)
    amb = ambiguous_links(prob, ref, eps)
    ref["ambiguous"] = amb
    ref["J_alt"] = None
    ref["R_alt"] = None
    if amb.any():
        alt = oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                              prob.p, prob.pn, pat=pat, flip=amb.astype(np.uint8))
        ref["J_alt"] = alt["J"]
        ref["R_alt"] = alt["R"]
    return ref


def residual_error(R_gpu, ref):
    R_ref = ref["R"]
    diff = np.abs(R_gpu - R_ref)
    if ref.get("R_alt") is not None:
        diff = np.minimum(diff, np.abs(R_gpu - ref["R_alt"]))
    return float(diff.max() / np.abs(R_ref).max())


def jacobian_row_error(J_gpu, ref):
    rp = ref["row_ptr"]
    J = ref["J"]
    diff = np.abs(J_gpu - J)
    if ref.get("J_alt") is not None:
        diff = np.minimum(diff, np.abs(J_gpu - ref["J_alt"]))
    starts = rp[:-1]
    num = np.maximum.reduceat(diff, starts)
    den = np.maximum.reduceat(np.abs(J), starts)
    return float((num / den).max())


def entry_stats(J_gpu, ref, floor_rel=1e-30):
    """Max and RMS entrywise relative error |J_gpu - J_ref| / max(|J_ref|, floor)."""
    rp = ref["row_ptr"]
    J = ref["J"]
    diff = np.abs(J_gpu - J)
    if ref.get("J_alt") is not None:
        diff = np.minimum(diff, np.abs(J_gpu - ref["J_alt"]))
    scale = np.repeat(np.maximum.reduceat(np.abs(J), rp[:-1]), np.diff(rp))
    rel = diff / np.maximum(np.abs(J), floor_rel * scale)
    return float(rel.max()), float(np.sqrt(np.mean(rel ** 2)))


def subgrid_row(prob, i, j, k):
    """Oracle row of cell (i, j, k) of `prob` computed on the clipped
    3 x 3 x 3 box around it: the row depends only on the cell and its
    neighbours, all inside the box.  Returns (R_K, {column: J_KL},
    {column: dPhi_KL})."""
    i0, i1 = max(i - 1, 0), min(i + 2, prob.nx)
    j0, j1 = max(j - 1, 0), min(j + 2, prob.ny)
    k0, k1 = max(k - 1, 0), min(k + 2, prob.nz)
    sx, sy, sz = i1 - i0, j1 - j0, k1 - k0

    def box(a):
        return a.reshape(prob.nz, prob.ny, prob.nx)[k0:k1, j0:j1, i0:i1].reshape(-1)

    out = oracle.assemble(sx, sy, sz, prob.phys, box(prob.perm), box(prob.poro), box(prob.depth),
                          box(prob.p), box(prob.pn), want_links=True)
    li = (i - i0) + sx * ((j - j0) + sy * (k - k0))
    rp, ci = out["row_ptr"], out["col_idx"]
    cols, Jrow, dphi = {}, {}, {}
    for e in range(rp[li], rp[li + 1]):
        c = ci[e]
        ci_, cj, ck = c % sx, (c // sx) % sy, c // (sx * sy)
        g = (i0 + ci_) + prob.nx * ((j0 + cj) + prob.ny * (k0 + ck))
        Jrow[g] = out["J"][e]
        dphi[g] = out["dphi"][e]
    return out["R"][li], Jrow, dphi


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
