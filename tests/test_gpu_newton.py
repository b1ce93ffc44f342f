"""Newton step and its Krylov solve (BiCGStab + Jacobi) against the oracle.

Bars (no tolerance is printed in the paper; these follow from the solver's
stopping rule and the Jacobian bars):
  * backward error against the oracle's Jacobian J_ref:
      ||J_ref x - b||_2 <= 2 rtol ||b||_2 + tolJ || |J_ref| |x| ||_2
    with tolJ the Jacobian bar of the path (1e-12 FP64, 1e-6 mixed): the
    solver stops at ||b - J x|| <= rtol ||b|| for its own J, which is J_ref
    up to tolJ entrywise relative to each row;
  * FP64 path, forward error against the oracle's direct solve: within
    cond(J_ref) (rtol + tolJ), times 10 for rounding.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2304_11274_gb300 import synth

pytestmark = pytest.mark.gpu

TOLJ = {"fp64": 1e-12, "mixed": 1e-6}


def _grid(prob, precision):
    from paper_2304_11274_gb300.api import Grid
    return Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth)


def _problem(shape, precision, seed=41, **over):
    over.setdefault("c_r", 1e-8)
    over.setdefault("dt", 3600.0)
    prob = synth.make_problem(*shape, seed=seed, connectivity=over.pop("connectivity", 10), **over)
    return synth.round_to_f32(prob) if precision == "mixed" else prob


def _ref(prob):
    out = oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p, prob.pn)
    return oracle.jacobian_csr(out, prob.n), out["R"]


def _backward_ok(J, x, b, rtol, tolj):
    res = np.linalg.norm(J @ x - b)
    bound = 2 * rtol * np.linalg.norm(b) + tolj * np.linalg.norm(abs(J) @ np.abs(x))
    return res <= bound, res, bound


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 4, 3), (12, 10, 6), (33, 9, 4), (7, 3, 19)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("precond", ["zline", "jacobi"])
def test_linear_solve_matches_oracle(shape, precision, conn, precond):
    prob = _problem(shape, precision, connectivity=conn)
    J, _ = _ref(prob)
    b = synth.cotangent(prob.n, seed=7)
    rtol = 1e-10
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        x, st = g.linear_solve(b, rtol=rtol, max_iters=2000, precond=precond)
        x = x.cpu().numpy()
    assert st["converged"] == 1 and st["rel_residual"] <= rtol
    ok, res, bound = _backward_ok(J, x, b, rtol, TOLJ[precision])
    assert ok, (res, bound)
    if precision == "fp64":
        from scipy.sparse.linalg import spsolve
        x_ref = np.atleast_1d(spsolve(J.tocsc(), b))
        kappa = np.linalg.cond(J.toarray()) if prob.n <= 4000 else 1e8
        err = np.abs(x - x_ref).max() / np.abs(x_ref).max()
        assert err <= 10 * kappa * (rtol + TOLJ["fp64"]), (err, kappa)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zline_preconditioner_needs_fewer_iterations(precision):
    """Thin cells (dz = dx / 5) couple vertically 25 times more strongly than
    horizontally: the z-line preconditioner, exact on those couplings, needs
    far fewer BiCGStab iterations than the diagonal one."""
    prob = _problem((24, 20, 32), precision, dt=86400.0, c_r=0.0)
    b = synth.cotangent(prob.n, seed=12)
    its = {}
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        for pc in ("jacobi", "zline"):
            _, st = g.linear_solve(b, rtol=1e-8, max_iters=5000, precond=pc)
            its[pc] = st["iterations"]
    assert its["zline"] * 2 <= its["jacobi"], its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_step_matches_oracle(precision):
    prob = _problem((12, 10, 6), precision)
    J, R_ref = _ref(prob)
    rtol = 1e-10
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        p0 = g._p.clone()
        p = g._p.clone()
        st, R, d = g.newton_step(p, rtol=rtol, want_residual=True, want_delta=True)
        R, d, p1 = R.cpu().numpy(), d.cpu().numpy(), p.cpu()
    assert st["converged"] == 1
    # R(p) before the update is the assembly's residual
    assert np.abs(R - R_ref).max() <= (1e-12 if precision == "fp64" else 1e-6) * np.abs(R_ref).max()
    ok, res, bound = _backward_ok(J, d, -R_ref, rtol, TOLJ[precision])
    assert ok, (res, bound)
    # the update is p + delta rounded once to the field type
    expect = (p0.cpu().double() + torch.as_tensor(d)).to(p1.dtype)
    assert torch.equal(p1, expect)
    if precision == "fp64":
        _, d_ref, _ = oracle.newton_step(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                         prob.p, prob.pn)
        kappa = np.linalg.cond(J.toarray())
        assert np.abs(d - d_ref).max() <= 10 * kappa * (rtol + 1e-12) * np.abs(d_ref).max()


def test_newton_solves_linear_problem_in_one_step():
    """c_f = 0: R is affine in p, one step reaches R = 0 (up to the solve's
    tolerance times the conditioning)."""
    prob = _problem((12, 10, 6), "fp64", c_f=0.0)
    with _grid(prob, "fp64") as g:
        g.set_state(prob.p, prob.pn)
        R0 = g.assemble_residual().cpu().numpy()
        p = g._p.clone()
        g.newton_step(p, rtol=1e-12, max_iters=3000)
        g.set_pressure(p)
        R1 = g.assemble_residual().cpu().numpy()
    assert np.linalg.norm(R1) <= 1e-9 * np.linalg.norm(R0)


def test_newton_iterations_converge_quadratically():
    """Strongly compressible fluid, FP64 path: three GPU Newton steps follow
    the oracle's iterates and the residual falls superlinearly."""
    prob = _problem((12, 10, 6), "fp64", c_f=1e-7)
    args = (prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth)
    with _grid(prob, "fp64") as g:
        g.set_state(prob.p, prob.pn)
        p = g._p.clone()
        norms = []
        p_ref = prob.p.copy()
        for _ in range(3):
            st, R, _ = g.newton_step(p, rtol=1e-12, max_iters=3000, want_residual=True)
            norms.append(np.abs(R.cpu().numpy()).max())
            p_ref, _, _ = oracle.newton_step(*args, p_ref, prob.pn)
            assert np.abs(p.cpu().numpy() - p_ref).max() <= 1e-9 * np.abs(p_ref).max()
    assert norms[1] < 0.5 * norms[0]
    assert norms[2] / norms[1] < 0.2 * norms[1] / norms[0] or norms[2] < 1e-10 * norms[0]


def test_nonconvergence_is_reported_and_leaves_p():
    from paper_2304_11274_gb300._capi import TPFAError
    prob = _problem((12, 10, 6), "mixed")
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        p = g._p.clone()
        before = p.clone()
        with pytest.raises(TPFAError) as e:
            g.newton_step(p, rtol=1e-14, max_iters=2, check_every=1)
        assert e.value.code == -9  # TPFA_ERR_NO_CONVERGENCE
        assert g.last_stats["iterations"] == 2 and g.last_stats["converged"] == 0
        assert torch.equal(p, before)


def test_zero_right_hand_side():
    prob = _problem((5, 4, 3), "fp64")
    with _grid(prob, "fp64") as g:
        g.set_state(prob.p, prob.pn)
        x, st = g.linear_solve(np.zeros(prob.n))
        assert st["iterations"] == 0 and st["converged"] == 1
        assert torch.count_nonzero(x).item() == 0


def test_linear_solve_adjoint_grid_properties():
    """128^3, 10 links, mixed path: the solve converges and its solution
    satisfies J x = b when J is applied by the independent matrix-free
    product (tpfa_jvp), whose FP32 products are exact to a few float ulps of
    |J| |x| (|J| from the assembled CSR)."""
    prob = synth.round_to_f32(synth.config_problem(4))
    b = synth.cotangent(prob.n, seed=synth.BASE_SEED + 50)
    rtol = 1e-8
    with _grid(prob, "mixed") as g:
        g.set_state(prob.p, prob.pn)
        x, st = g.linear_solve(b, rtol=rtol, max_iters=5000)
        Jx, _ = g.jvp(x)
        _, vals, diag = g.assemble_jacobian()
        rp, ci = g.pattern()
        rows = torch.repeat_interleave(torch.arange(prob.n, device="cuda"), rp[1:] - rp[:-1])
        a = vals.double().abs()
        a[ci.long() == rows] = diag.abs()
        absJx = torch.zeros(prob.n, dtype=torch.float64, device="cuda").index_add_(0, rows, a * x.abs()[ci.long()])
        bt = torch.as_tensor(b, device="cuda")
        res = float(torch.linalg.norm(Jx - bt))
        bound = 2 * rtol * float(torch.linalg.norm(bt)) + 4 * 2.0 ** -24 * float(torch.linalg.norm(absJx))
    assert st["converged"] == 1
    assert res <= bound, (res, bound)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_iterations_give_the_same_bits_on_every_stream(precision):
    """The solve replays its batches of iterations as a CUDA graph on a
    library stream ordered with the caller's: the solution is the same, bit
    for bit, on the default stream, on a user stream, with a new solution
    buffer (a new graph), with another batch size (a new graph) and again
    after those."""
    prob = _problem((24, 20, 12), precision, seed=47)
    b = synth.cotangent(prob.n, seed=48)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        x0, st0 = g.linear_solve(b, rtol=1e-10, max_iters=2000)
        x0 = x0.cpu()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            x1, st1 = g.linear_solve(b, rtol=1e-10, max_iters=2000, stream=s)
        s.synchronize()
        assert torch.equal(x1.cpu(), x0) and st1["iterations"] == st0["iterations"]
        x2, _ = g.linear_solve(b, rtol=1e-10, max_iters=2000, out=torch.empty_like(x1))
        assert torch.equal(x2.cpu(), x0)
        x3, st3 = g.linear_solve(b, rtol=1e-10, max_iters=2000, check_every=3)
        assert torch.equal(x3.cpu(), x0) and st3["iterations"] == st0["iterations"]
        x4, _ = g.linear_solve(b, rtol=1e-10, max_iters=2000)
        assert torch.equal(x4.cpu(), x0)
