"""Comparison of GPU results with the oracle (test infrastructure).

Used by the parity tests and by the benchmark's precision statement; never
by the library.

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


