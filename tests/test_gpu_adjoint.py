"""Adjoint (VJP) kernel against the oracle's gradient and finite differences."""
import numpy as np
import pytest
import torch

import _compare as C
import oracle
from paper_2304_11274_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}


def _grid(prob, precision):
    from paper_2304_11274_gb300.api import Grid
    return Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth)


def _normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _gp_reference(prob, v, eps):
    """J^T v from the oracle's Jacobian, and from its alternative evaluation
    where upwind choices are ambiguous (either is admissible)."""
    ref = C.reference(prob, eps)
    rp, ci = ref["row_ptr"], ref["col_idx"]
    rows = np.repeat(np.arange(prob.n), np.diff(rp))
    out = [np.bincount(ci, weights=ref["J"] * v[rows], minlength=prob.n)]
    if ref["J_alt"] is not None:
        out.append(np.bincount(ci, weights=ref["J_alt"] * v[rows], minlength=prob.n))
    return out


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (7, 5, 3), (33, 17, 9), (40, 37, 6)])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_vjp_matches_oracle(shape, conn, precision, c_r):
    prob = synth.make_problem(*shape, seed=17, connectivity=conn, c_r=c_r)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
        prob.perm = prob.perm.astype(np.float32).astype(np.float64)  # the adjoint's k is stored in FP32
    v = synth.cotangent(prob.n, seed=3)
    g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                    prob.p, prob.pn, v)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        g_p, g_lnk = g.vjp(v)
        g.sync_status()
        g_p, g_lnk = g_p.cpu().numpy(), g_lnk.cpu().numpy()
    eps = C.EPS32 if precision == "mixed" else C.EPS64
    cands = _gp_reference(prob, v, eps)
    assert np.allclose(cands[0], g_p_ref, rtol=1e-12, atol=1e-12 * np.abs(g_p_ref).max())
    e_p = min(_normwise(g_p, c) for c in cands)
    assert e_p <= TOL[precision], e_p
    if prob.n > 1:
        assert _normwise(g_lnk, g_lnk_ref) <= TOL[precision]


# odd and even nx (the two-cell march needs nx even: on odd nx "tiled2"
# runs the one-cell march), one-row and one-plane grids, x-segments cut by
# the grid edge, a single 64-cell segment and several
VARIANT_SHAPES = [(1, 1, 1), (5, 1, 7), (33, 2, 1), (70, 41, 11), (72, 41, 11), (97, 70, 9), (2, 3, 2),
                  (64, 5, 3), (66, 9, 5), (130, 41, 11), (256, 1, 6), (6, 70, 1)]


@pytest.mark.parametrize("shape", VARIANT_SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_vjp_kernel_variants_bit_identical(shape, conn, c_r):
    """The mixed path's adjoint: the one-cell and two-cell marches and the
    naive gather give identical bits under every tiling the autotuner may
    pick."""
    prob = synth.round_to_f32(synth.make_problem(*shape, seed=23, connectivity=conn, c_r=c_r))
    v = synth.cotangent(prob.n, seed=8)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        gp_n, gk_n = (x.cpu().numpy() for x in g.vjp(v, kernel="naive"))
        for JY, W in [(16, 4), (32, 8), (64, 4), (7, 4)]:
            g.set_tiling(JY, W)
            for kernel in ["tiled", "tiled2", "auto"]:
                gp_t, gk_t = g.vjp(v, kernel=kernel)
                g.sync_status()
                assert np.array_equal(gp_t.cpu().numpy().view(np.uint64), gp_n.view(np.uint64)), (JY, W, kernel)
                assert np.array_equal(gk_t.cpu().numpy().view(np.uint64), gk_n.view(np.uint64)), (JY, W, kernel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel", ["naive", "tiled"])
def test_vjp_every_link_a_tie(precision, kernel):
    """Uniform pressure without gravity: dPhi = 0 on every link, so each row
    takes the other cell's density and dF_Li/dp_i != -dF_iL/dp_i everywhere;
    the gradient still matches the oracle (which evaluates each row from its
    own side)."""
    prob = synth.make_problem(37, 9, 6, seed=25, connectivity=10, g=0.0, c_f=1e-8, perturb=0.0)
    prob.p = np.full(prob.n, 1.2e7)
    v = synth.cotangent(prob.n, seed=9)
    g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                    prob.p, prob.pn, v)
    if precision == "mixed":
        prob.perm = prob.perm.astype(np.float32).astype(np.float64)
        g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                        prob.p, prob.pn, v)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        g_p, g_lnk = (x.cpu().numpy() for x in g.vjp(v, kernel=kernel))
        g.sync_status()
    assert _normwise(g_p, g_p_ref) <= TOL[precision]
    assert np.abs(g_lnk).max() <= TOL[precision] * np.abs(g_p_ref).max()  # F = 0: no permeability gradient
    assert np.abs(g_lnk_ref).max() == 0.0


def test_vjp_smooth_cotangent_keeps_relative_accuracy():
    """v = 1 + 1e-6 u: the permeability gradient depends only on the small
    differences v_K - v_L, which the mixed path forms from FP32 pairs
    (hi_K - hi_L) + (lo_K - lo_L), accurate relative to the difference
    itself, so its relative error stays at the FP32 level."""
    prob = synth.round_to_f32(synth.make_problem(40, 37, 6, seed=27, connectivity=10))
    prob.perm = prob.perm.astype(np.float32).astype(np.float64)
    v = 1.0 + 1e-6 * synth.cotangent(prob.n, seed=10)
    g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                    prob.p, prob.pn, v)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        g_p, g_lnk = (x.cpu().numpy() for x in g.vjp(v))
    assert _normwise(g_lnk, g_lnk_ref) <= 1e-6
    assert _normwise(g_p, g_p_ref) <= 1e-6


def test_vjp_adjoint_size_against_oracle():
    """128^3 with 10 links on the mixed path: the adjoint workload's grid."""
    prob = synth.round_to_f32(synth.config_problem(4))
    prob.perm = prob.perm.astype(np.float32).astype(np.float64)
    v = synth.cotangent(prob.n, seed=synth.BASE_SEED + 4)
    g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                    prob.p, prob.pn, v)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        g_p, g_lnk = g.vjp(v)
        g.sync_status()
        g_p, g_lnk = g_p.cpu().numpy(), g_lnk.cpu().numpy()
    assert _normwise(g_p, g_p_ref) <= 1e-6
    assert _normwise(g_lnk, g_lnk_ref) <= 1e-6


def test_autograd_fp64_against_central_differences():
    """TPFAResidual on a 16^3 grid (FP64 path): directional derivatives of
    v^T R in p and ln k against central differences, h = 1e-6 relative."""
    from paper_2304_11274_gb300.api import Grid, residual
    prob = synth.make_problem(16, 16, 16, seed=synth.BASE_SEED + 4, connectivity=10)
    rng = np.random.default_rng(7)
    v = torch.as_tensor(synth.cotangent(prob.n, seed=11), device="cuda")
    with Grid(prob.nx, prob.ny, prob.nz, prob.phys, "fp64", prob.perm, prob.poro, prob.depth) as g:
        pn = torch.as_tensor(prob.pn, device="cuda")
        p0 = torch.as_tensor(prob.p, device="cuda")
        g.set_state(p0, pn)
        p = p0.clone().requires_grad_(True)
        lk = torch.log(torch.as_tensor(prob.perm, device="cuda")).requires_grad_(True)
        R = residual(g, p, lk)
        (R * v).sum().backward()
        gp, gk = p.grad.clone(), lk.grad.clone()

        def f(pp, ll):
            with torch.no_grad():
                return float((residual(g, pp.contiguous(), ll.contiguous()) * v).sum())

        for _ in range(3):
            d = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
            h = 1e-6 * torch.abs(p0)
            fd = (f(p0 + h * d, lk.detach()) - f(p0 - h * d, lk.detach())) / 2.0
            assert fd == pytest.approx(float((gp * h * d).sum()), rel=1e-5)
            hk = 1e-6
            fdk = (f(p0, lk.detach() + hk * d) - f(p0, lk.detach() - hk * d)) / (2 * hk)
            assert fdk == pytest.approx(float((gk * d).sum()), rel=1e-5)


def test_autograd_mixed_matches_oracle_gradient():
    from paper_2304_11274_gb300.api import Grid, residual
    prob = synth.round_to_f32(synth.make_problem(16, 16, 16, seed=synth.BASE_SEED + 4, connectivity=10))
    prob.perm = prob.perm.astype(np.float32).astype(np.float64)
    v = synth.cotangent(prob.n, seed=11)
    g_p_ref, g_lnk_ref = oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                    prob.p, prob.pn, v)
    with Grid(prob.nx, prob.ny, prob.nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth) as g:
        pn = torch.as_tensor(prob.pn, device="cuda", dtype=torch.float32)
        p = torch.as_tensor(prob.p, device="cuda", dtype=torch.float32)
        g.set_state(p, pn)
        p = p.clone().requires_grad_(True)
        lk = torch.log(torch.as_tensor(prob.perm, device="cuda")).requires_grad_(True)
        R = residual(g, p, lk)
        (R * torch.as_tensor(v, device="cuda")).sum().backward()
        assert _normwise(lk.grad.cpu().numpy(), g_lnk_ref) <= 1e-6
        # p.grad is returned in p's dtype (FP32)
        assert _normwise(p.grad.double().cpu().numpy(), g_p_ref) <= 1e-6


@pytest.mark.parametrize("conn", [6, 10])
def test_vjp_reused_link_ties(conn):
    """Exact ties on the links the adjoint march reuses from the previous
    y-row (where dF_Li/dp_i != -dF_iL/dp_i): march and naive gather agree bit
    for bit."""
    prob = C.tie_sweep_problem("mixed", conn)
    v = synth.cotangent(prob.n, seed=22)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        a = g.vjp(v, kernel="naive")
        for kernel in ["tiled", "tiled2"]:
            b = g.vjp(v, kernel=kernel)
            g.sync_status()
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), kernel


@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("shape", [(130, 37, 5), (64, 64, 3)])
def test_vjp_two_cell_ties_in_every_direction(conn, shape):
    """Exact ties on x, y and diagonal links, inside a lane's pair of cells,
    across lanes and across segments: the two-cell adjoint march recomputes
    those rows and matches the naive gather bit for bit."""
    prob = C.tie_pairs_problem("mixed", conn, shape=shape)
    v = synth.cotangent(prob.n, seed=24)
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        a = g.vjp(v, kernel="naive")
        for tiling in [(32, 4), (5, 8)]:
            g.set_tiling(*tiling)
            b = g.vjp(v, kernel="tiled2")
            g.sync_status()
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), tiling
