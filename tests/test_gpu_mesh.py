"""General meshes (connection lists) on the GPU against the oracle.

Bars as for the structured grid: pattern bit-exact; FP64 <= 1e-12 (normwise
residual, row-normwise Jacobian); mixed <= 1e-6 on FP32-rounded inputs, where
the mixed path also stores the transmissibilities in FP32 (the oracle gets
them rounded the same way).
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


def _mesh(m, precision):
    from paper_2304_11274_gb300.api import Mesh
    return Mesh(m.n, m.ci, m.cj, m.T, m.V, m.poro, m.depth, m.phys, precision)


def _reference(m, eps):
    """Oracle R, J and the alternative evaluation of links whose dPhi lies
    within rounding of zero (either upwind choice is admissible there)."""
    pat = oracle.mesh_pattern(m.n, m.ci, m.cj)
    args = (m.n, m.phys, m.ci, m.cj, m.T, m.V, m.poro, m.depth, m.p, m.pn)
    ref = oracle.mesh_assemble(*args, pat=pat, want_links=True)
    rp, ci = ref["row_ptr"], ref["col_idx"]
    rows = np.repeat(np.arange(m.n), np.diff(rp))
    scale = np.abs(m.p[rows] - m.p[ci]) + 1.1e3 * 9.81 * np.abs(m.depth[rows] - m.depth[ci])
    amb = (ci != rows) & (np.abs(ref["dphi"]) <= 32 * eps * scale)
    ref["J_alt"] = ref["R_alt"] = None
    if amb.any():
        alt = oracle.mesh_assemble(*args, pat=pat, flip=amb.astype(np.uint8))
        ref["J_alt"], ref["R_alt"] = alt["J"], alt["R"]
    return ref


def _run(m, precision):
    with _mesh(m, precision) as g:
        g.set_state(m.p, m.pn)
        R, vals, diag = g.assemble()
        R_only = g.assemble_residual()
        g.sync_status()
        rp, ci = g.pattern()
        out = dict(R=R.cpu().numpy(), R_only=R_only.cpu().numpy(), vals=vals.double().cpu().numpy(),
                   diag=None if diag is None else diag.cpu().numpy(), rp=rp.cpu().numpy(), ci=ci.cpu().numpy())
    return out


def _prepare(shape, precision, conn, c_r=0.0, seed=61, **kw):
    m = synth.make_mesh(*shape, seed=seed, connectivity=conn, c_r=c_r, **kw)
    return synth.round_mesh_to_f32(m) if precision == "mixed" else m


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (5, 4, 3), (16, 9, 7), (40, 33, 6)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_mesh_parity_vs_oracle(shape, precision, conn, c_r):
    m = _prepare(shape, precision, conn, c_r)
    got = _run(m, precision)
    ref = _reference(m, EPS[precision])
    assert np.array_equal(got["rp"], ref["row_ptr"])
    assert np.array_equal(got["ci"], ref["col_idx"])
    assert np.array_equal(got["R"], got["R_only"])
    J = got["vals"].copy()
    if got["diag"] is not None:
        rows = np.repeat(np.arange(m.n), np.diff(got["rp"]))
        J[got["ci"] == rows] = got["diag"]
    assert C.residual_error(got["R"], ref) <= TOL[precision]
    assert C.jacobian_row_error(J, ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_structured_grid_as_mesh_matches_grid_kernel(precision):
    """A structured grid passed as its connection list (transmissibilities
    read back from the grid) reproduces the structured kernel: same pattern,
    off-diagonal values bit-identical, R and the diagonal to rounding of the
    cell volume factor."""
    from paper_2304_11274_gb300.api import Grid, Mesh
    pr = synth.make_problem(37, 21, 9, seed=62, connectivity=10)
    if precision == "mixed":
        pr = synth.round_to_f32(pr)
    with Grid(pr.nx, pr.ny, pr.nz, pr.phys, precision, pr.perm, pr.poro, pr.depth) as g:
        g.set_state(pr.p, pr.pn)
        Rg, vg, dg = g.assemble_jacobian(kernel="naive")
        rpg, cig = g.pattern()
        Ts = [g.transmissibility(w).double().cpu().numpy() for w in range(5)]
        Rg, vg = Rg.cpu().numpy(), vg.double().cpu().numpy()
        dg = None if dg is None else dg.cpu().numpy()
        rpg, cig = rpg.cpu().numpy(), cig.cpu().numpy()
    a, b, kind = synth.structured_pairs(pr.nx, pr.ny, pr.nz, 10)
    T = np.array([Ts[k][x] for x, k in zip(a, kind)])
    V = np.full(pr.n, pr.phys["dx"] * pr.phys["dy"] * pr.phys["dz"])
    with Mesh(pr.n, a, b, T, V, pr.poro, pr.depth, pr.phys, precision) as m:
        m.set_state(pr.p, pr.pn)
        Rm, vm, dm = m.assemble()
        rpm, cim = m.pattern()
        Rm, vm = Rm.cpu().numpy(), vm.double().cpu().numpy()
        dm = None if dm is None else dm.cpu().numpy()
        rpm, cim = rpm.cpu().numpy(), cim.cpu().numpy()
    assert np.array_equal(rpg, rpm) and np.array_equal(cig, cim)
    rows = np.repeat(np.arange(pr.n), np.diff(rpg))
    off = cig != rows
    assert np.array_equal(vg[off], vm[off])
    tol = 1e-14 if precision == "fp64" else 1e-6
    assert np.abs(Rg - Rm).max() <= tol * np.abs(Rg).max()
    dgv = dg if dg is not None else vg[~off]
    dmv = dm if dm is not None else vm[~off]
    assert np.abs(dgv - dmv).max() <= tol * np.abs(dgv).max()


def test_mesh_bad_lists_are_rejected():
    from paper_2304_11274_gb300._capi import TPFAError
    from paper_2304_11274_gb300.api import Mesh
    phys = synth.physics()
    V = np.full(3, 200.0)
    base = dict(V=V, poro=np.full(3, 0.2), depth=np.ones(3), phys=phys)
    for ci, cj in (([0, 1], [1, 1]), ([0, 1], [1, 0]), ([0], [3])):
        with pytest.raises(TPFAError) as e:
            Mesh(3, ci, cj, np.full(len(ci), 1e-13), **base)
        assert e.value.code == -1  # TPFA_ERR_INVALID_ARG
    with pytest.raises(TPFAError):
        Mesh(3, [0], [1], [-1.0], **base)


def test_mesh_without_connections():
    """Isolated cells: R = A, J = dA/dp (accumulation only)."""
    from paper_2304_11274_gb300.api import Mesh
    m = _prepare((4, 1, 1), "fp64", 6, c_r=1e-9, inactive=0.0)
    with Mesh(m.n, [], [], [], m.V, m.poro, m.depth, m.phys, "fp64") as g:
        g.set_state(m.p, m.pn)
        R, vals, _ = g.assemble()
        R, vals = R.cpu().numpy(), vals.cpu().numpy()
    ref = oracle.mesh_assemble(m.n, m.phys, np.zeros(0), np.zeros(0), np.zeros(0), m.V, m.poro, m.depth, m.p, m.pn)
    assert vals.size == m.n
    assert np.abs(R - ref["R"]).max() <= 1e-12 * np.abs(ref["R"]).max()
    assert np.abs(vals - ref["J"]).max() <= 1e-12 * np.abs(ref["J"]).max()


def test_mesh_benchmark_size_against_oracle():
    """The faulted-mesh workload of the benchmark (256 x 256 x 128 before
    pinch-outs, 6 faces + fault connections, mixed): every row."""
    m = synth.round_mesh_to_f32(synth.make_mesh(256, 256, 128, seed=synth.BASE_SEED + 5))
    got = _run(m, "mixed")
    ref = _reference(m, EPS["mixed"])
    assert np.array_equal(got["ci"], ref["col_idx"])
    J = got["vals"].copy()
    rows = np.repeat(np.arange(m.n), np.diff(got["rp"]))
    J[got["ci"] == rows] = got["diag"]
    assert C.residual_error(got["R"], ref) <= 1e-6
    assert C.jacobian_row_error(J, ref) <= 1e-6
