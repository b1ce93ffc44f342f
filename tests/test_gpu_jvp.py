"""Matrix-free J w against the oracle's assembled Jacobian times w.

Error measure: J w sums products J_KL w_L, so its rounding is bounded by the
entries' errors times |w|.  With every Jacobian entry within tol of its row's
largest entry (the Jacobian bar), |(J w)_gpu - (J w)_ref|_K is at most
tol * (|J| |w|)_K; the test gates ||diff||_inf / ||(|J| |w|)||_inf <= tol
(1e-12 FP64, 1e-6 mixed).  R from the same pass must equal the assembly's R
bit for bit.
"""
import numpy as np
import pytest
import torch

import _compare as C
import oracle
from paper_2304_11274_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}
EPS = {"fp64": C.EPS64, "mixed": C.EPS32}
SHAPES = [(1, 1, 1), (1, 6, 1), (2, 3, 4), (7, 5, 3), (33, 17, 9), (70, 41, 11)]


def _grid(prob, precision):
    from paper_2304_11274_gb300.api import Grid
    return Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth)


def _problem(shape, conn, precision, c_r=0.0, seed=29):
    prob = synth.make_problem(*shape, seed=seed, connectivity=conn, c_r=c_r)
    return synth.round_to_f32(prob) if precision == "mixed" else prob


def _jvp_error(Jw, prob, w, eps):
    """Error of Jw against the oracle's J w, taking the better of the two
    admissible upwind evaluations of ambiguous links row by row."""
    ref = C.reference(prob, eps)
    rp, ci = ref["row_ptr"], ref["col_idx"]
    starts = rp[:-1]
    cands = [np.add.reduceat(ref["J"] * w[ci], starts)]
    if ref["J_alt"] is not None:
        cands.append(np.add.reduceat(ref["J_alt"] * w[ci], starts))
    Jw_ref, _ = oracle.jvp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                           prob.p, prob.pn, w)
    assert np.allclose(cands[0], Jw_ref, rtol=0, atol=1e-13 * np.abs(Jw_ref).max())
    scale = np.add.reduceat(np.abs(ref["J"]) * np.abs(w[ci]), starts).max()
    diff = np.min([np.abs(Jw - c) for c in cands], axis=0)
    return float(diff.max() / scale)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_jvp_matches_oracle(shape, conn, precision, c_r):
    prob = _problem(shape, conn, precision, c_r)
    w = synth.cotangent(prob.n, seed=5)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        Jw, R = g.jvp(w, want_residual=True)
        R_asm = g.assemble_residual()
        g.sync_status()
        Jw, R, R_asm = Jw.cpu().numpy(), R.cpu().numpy(), R_asm.cpu().numpy()
    assert np.array_equal(R, R_asm)
    assert _jvp_error(Jw, prob, w, EPS[precision]) <= TOL[precision]


# shapes with full interior segments (nx > 64), ragged x/y/z tails and
# degenerate axes, so both the interior and the boundary rows of the march run
VARIANT_SHAPES = [(1, 1, 1), (5, 1, 7), (33, 2, 1), (70, 41, 11), (72, 41, 11), (97, 70, 9)]


@pytest.mark.parametrize("shape", VARIANT_SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_jvp_kernel_variants_bit_identical(shape, conn, c_r):
    """The mixed path's y-march and naive gather: identical bits for J w and R,
    under every tiling the autotuner may pick."""
    prob = _problem(shape, conn, "mixed", c_r)
    w = synth.cotangent(prob.n, seed=13)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        Jn, Rn = g.jvp(w, want_residual=True, kernel="naive")
        Jn, Rn = Jn.cpu().numpy(), Rn.cpu().numpy()
        for JY, W in [(16, 4), (32, 8), (64, 4)]:
            g.set_tiling(JY, W)
            Jt, Rt = g.jvp(w, want_residual=True, kernel="tiled")
            g.sync_status()
            assert np.array_equal(Jt.cpu().numpy(), Jn), (JY, W)
            assert np.array_equal(Rt.cpu().numpy(), Rn), (JY, W)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_jvp_consistent_with_vjp(precision):
    """v^T (J w) = (J^T v)^T w between the two matrix-free kernels."""
    prob = _problem((40, 37, 6), 10, precision, c_r=1e-9)
    rng = np.random.default_rng(3)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        for _ in range(3):
            v = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
            w = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
            Jw, _ = g.jvp(w)
            g_p, _ = g.vjp(v, want_lnk=False)
            a, b = float(v @ Jw), float(g_p @ w)
            scale = float(torch.abs(v) @ torch.abs(Jw))
            assert abs(a - b) <= 10 * TOL[precision] * scale
        g.sync_status()


def test_jvp_matches_assembled_matrix_product():
    """The mixed path's J w against its own assembled CSR (FP32 off-diagonals,
    FP64 diagonal) applied to w in FP64: the off-diagonals are the same FP32
    link derivatives; the assembled diagonal is their compensated FP32 sum
    (error a few eps32 of the row scale) where J w sums them in FP64."""
    prob = _problem((70, 41, 11), 10, "mixed")
    w = synth.cotangent(prob.n, seed=9)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        _, vals, diag = g.assemble_jacobian()
        rp, ci = g.pattern()
        Jw, _ = g.jvp(w)
        g.sync_status()
        rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
        vals = vals.double().cpu().numpy()
        diag = diag.cpu().numpy()
        Jw = Jw.cpu().numpy()
    rows = np.repeat(np.arange(prob.n), np.diff(rp))
    vals[ci == rows] = diag
    prod = np.add.reduceat(vals * w[ci], rp[:-1])
    scale = np.add.reduceat(np.abs(vals) * np.abs(w[ci]), rp[:-1]).max()
    assert np.abs(Jw - prod).max() <= 4 * C.EPS32 * scale


def test_jvp_adjoint_size_against_oracle():
    """128^3, 10 links, mixed path: the adjoint workload's grid."""
    prob = synth.round_to_f32(synth.config_problem(4))
    w = synth.cotangent(prob.n, seed=synth.BASE_SEED + 40)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        Jw, _ = g.jvp(w)
        g.sync_status()
        Jw = Jw.cpu().numpy()
    assert _jvp_error(Jw, prob, w, EPS["mixed"]) <= TOL["mixed"]


def test_jvp_errors():
    from paper_2304_11274_gb300._capi import TPFAError
    prob = _problem((5, 4, 3), 10, "mixed")
    with _grid(prob, "mixed") as g:
        with pytest.raises(TPFAError) as e:
            g.jvp(np.zeros(prob.n))
        assert e.value.code == -6  # TPFA_ERR_NO_STATE
        g.set_state(prob.p, prob.pn)
        with pytest.raises(ValueError):
            g.jvp(np.zeros(prob.n + 1))
        assert g.lib.tpfa_jvp(g.handle, None, None, None, None) == -1  # TPFA_ERR_INVALID_ARG


@pytest.mark.slow
def test_jvp_full_size_sampled():
    """512 x 512 x 256, 10 links, mixed, autotuned tiling (the benchmark's
    J w launch): sampled rows against the oracle row of each cell's clipped
    3 x 3 x 3 box dotted with w, plus the eight corners."""
    from paper_2304_11274_gb300.api import Grid
    prob = synth.round_to_f32(synth.config_problem(1))
    w = synth.cotangent(prob.n, synth.BASE_SEED + 40)
    rng = np.random.default_rng(5)
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    cells = [(i, j, k) for i in (0, nx - 1) for j in (0, ny - 1) for k in (0, nz - 1)]
    cells += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(3000)]
    with Grid(nx, ny, nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth) as g:
        g.set_state(prob.p, prob.pn)
        g.autotune(None)
        Jw, _ = g.jvp(w)
        g.sync_status()
        lin = np.array([i + nx * (j + ny * k) for (i, j, k) in cells])
        got = Jw[torch.as_tensor(lin, device="cuda")].cpu().numpy()
        del Jw
    worst, skipped = 0.0, 0
    for n, (i, j, k) in enumerate(cells):
        c = lin[n]
        _, Jrow, dphi = C.subgrid_row(prob, i, j, k)
        amb = any(abs(dphi[L]) <= 32 * C.EPS32 * (abs(prob.p[c] - prob.p[L]) +
                                                 1.1e3 * 9.81 * abs(prob.depth[c] - prob.depth[L]))
                  for L in Jrow if L != c)
        if amb:
            skipped += 1
            continue
        ref = sum(Jrow[L] * w[L] for L in Jrow)
        scale = sum(abs(Jrow[L] * w[L]) for L in Jrow)
        worst = max(worst, abs(got[n] - ref) / scale)
    assert worst <= TOL["mixed"], worst
    assert skipped <= len(cells) // 100


@pytest.mark.parametrize("conn", [6, 10])
def test_jvp_reused_link_ties_are_fixed_up(conn):
    """Exact ties on the links the J w march reuses from the previous y-row:
    the march recomputes those rows and matches the naive kernel bit for bit."""
    prob = C.tie_sweep_problem("mixed", conn)
    w = synth.cotangent(prob.n, seed=21)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        Jn, Rn = g.jvp(w, want_residual=True, kernel="naive")
        Jt, Rt = g.jvp(w, want_residual=True, kernel="tiled")
        g.sync_status()
        assert torch.equal(Jn, Jt) and torch.equal(Rn, Rt)
