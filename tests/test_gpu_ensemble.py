"""Batched ensemble assembly (one persistent, graph-captured launch) and the autotuner."""
import os

import numpy as np
import pytest
import torch

import _compare as C
from paper_2304_11274_gb300 import synth

pytestmark = pytest.mark.gpu

UNEVEN = [(40, 37, 6), (65, 3, 9), (33, 17, 9), (7, 5, 3), (1, 1, 1), (100, 70, 12), (2, 130, 4), (96, 64, 8)]


def _models(shapes, conn=10, c_r=0.0, seed0=100):
    from paper_2304_11274_gb300.api import Grid
    probs, grids = [], []
    for m, shp in enumerate(shapes):
        prob = synth.round_to_f32(synth.make_problem(*shp, seed=seed0 + m, connectivity=conn, c_r=c_r))
        g = Grid(prob.nx, prob.ny, prob.nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth)
        g.set_state(prob.p, prob.pn)
        probs.append(prob)
        grids.append(g)
    return probs, grids


def _single(g):
    R, vals, diag = g.assemble_jacobian()
    torch.cuda.synchronize()
    return R.clone(), vals.clone(), diag.clone()


def _same(a, b):
    return all(torch.equal(x.view(torch.int64) if x.dtype == torch.float64 else x.view(torch.int32),
                           y.view(torch.int64) if y.dtype == torch.float64 else y.view(torch.int32))
               for x, y in zip(a, b))


@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_batch_bit_identical_to_single_grid_launches(conn, c_r):
    from paper_2304_11274_gb300.api import Ensemble
    probs, grids = _models(UNEVEN, conn=conn, c_r=c_r)
    singles = [_single(g) for g in grids]
    with Ensemble(grids) as ens:
        outs = ens.allocate_outputs()
        ens.assemble()
        torch.cuda.synchronize()
        for m in range(len(grids)):
            assert _same(outs[m], singles[m]), m
            grids[m].sync_status()
        info = ens.tiling()
        assert info["tiles"] > 0 and info["blocks"] > 0
    for g in grids:
        g.close()


def test_batch_matches_oracle():
    from paper_2304_11274_gb300.api import Ensemble
    probs, grids = _models(UNEVEN[:4])
    with Ensemble(grids) as ens:
        outs = ens.allocate_outputs()
        ens.assemble()
        torch.cuda.synchronize()
        for m, prob in enumerate(probs):
            ref = C.reference(prob, C.EPS32)
            R, vals, diag = (t.cpu().numpy() for t in outs[m])
            J = vals.astype(np.float64)
            rows = np.repeat(np.arange(prob.n), np.diff(ref["row_ptr"]))
            J[ref["col_idx"] == rows] = diag
            assert C.residual_error(R, ref) <= 1e-6
            assert C.jacobian_row_error(J, ref) <= 1e-6
    for g in grids:
        g.close()


def test_batch_follows_state_changes_and_repeats():
    from paper_2304_11274_gb300.api import Ensemble
    probs, grids = _models(UNEVEN[:5])
    with Ensemble(grids) as ens:
        outs = ens.allocate_outputs()
        for rep in range(3):
            newp = []
            for m, (prob, g) in enumerate(zip(probs, grids)):
                p = synth.pressure_sequence(prob, 1, seed=rep * 10 + m)[0].astype(np.float32)
                t = torch.as_tensor(p, device="cuda")
                g.set_pressure(t)
                newp.append(t)
            ens.assemble()
            torch.cuda.synchronize()
            for m, g in enumerate(grids):
                assert _same(outs[m], _single(g)), (rep, m)
    for g in grids:
        g.close()


def test_ensemble_autotune_and_cache(tmp_path):
    from paper_2304_11274_gb300.api import Ensemble
    probs, grids = _models(UNEVEN[:6])
    cache = str(tmp_path / "tune.txt")
    with Ensemble(grids) as ens:
        outs = ens.allocate_outputs()
        info = ens.autotune(cache)
        assert info["rows_per_march"] in (8, 16, 24, 32, 40, 48, 64) and info["warps_per_block"] in (4, 8)
        assert os.path.exists(cache)
        text = open(cache).read()
        assert "ensemble/" in text
        ens.assemble()
        torch.cuda.synchronize()
        for m, g in enumerate(grids):
            assert _same(outs[m], _single(g))
    with Ensemble(grids) as ens2:  # the cached choice is reused without timing
        ens2.allocate_outputs()
        assert ens2.autotune(cache)["rows_per_march"] == info["rows_per_march"]
    for g in grids:
        g.close()


def test_grid_autotune_keeps_results(tmp_path):
    probs, grids = _models([(70, 41, 11)])
    g = grids[0]
    before = _single(g)
    jy, w = g.autotune(str(tmp_path / "t.txt"))
    assert jy in (8, 16, 24, 32, 40, 48, 64) and w in (4, 8)
    assert _same(before, _single(g))
    for jy, w in [(7, 4), (1, 8), (64, 4)]:
        g.set_tiling(jy, w)
        assert _same(before, _single(g))
    from paper_2304_11274_gb300.api import TPFAError
    with pytest.raises(TPFAError):
        g.set_tiling(65, 4)  # a march longer than 64 rows is rejected
    g.close()


def test_ensemble_argument_checks():
    from paper_2304_11274_gb300.api import Ensemble, Grid, TPFAError
    prob = synth.make_problem(8, 8, 4, seed=1, connectivity=10)
    g64 = Grid(prob.nx, prob.ny, prob.nz, prob.phys, "fp64", prob.perm, prob.poro, prob.depth)
    with pytest.raises(TPFAError):
        Ensemble([g64])
    probs, grids = _models([(8, 8, 4), (9, 7, 3)], conn=10)
    _, grids6 = _models([(8, 8, 4)], conn=6)
    with pytest.raises(TPFAError):
        Ensemble([grids[0], grids6[0]])
    with Ensemble(grids) as ens:
        with pytest.raises(TPFAError) as ei:
            ens.assemble()  # outputs not bound
        assert ei.value.name == "TPFA_ERR_INVALID_ARG"
    for g in grids + grids6 + [g64]:
        g.close()


@pytest.mark.slow
def test_uneven_64_model_ensemble_bit_identical():
    """The 64-model ensemble (nx, ny ~ U{64..256}, nz ~ U{32..128}, own seed
    per model): batched launch against 64 single-grid launches."""
    from paper_2304_11274_gb300.api import Ensemble
    shapes = synth.ensemble_shapes()
    probs, grids = _models(shapes, seed0=synth.BASE_SEED + 1000)
    with Ensemble(grids) as ens:
        outs = ens.allocate_outputs()
        ens.assemble()
        torch.cuda.synchronize()
        for m, g in enumerate(grids):
            assert _same(outs[m], _single(g)), m
            g.sync_status()
        # sampled rows of four models against the oracle (each row on its
        # clipped 3 x 3 x 3 box); the residual bar is normwise over the
        # sample, the Jacobian bar row-wise
        rng = np.random.default_rng(31)
        for m in (0, 17, 40, 63):
            prob, g = probs[m], grids[m]
            R, vals, diag = (x.cpu().numpy() for x in outs[m])
            rp, ci = (x.cpu().numpy() for x in g.pattern())
            worst_R, scale_R = 0.0, 0.0
            for _ in range(100):
                i, j, k = (int(rng.integers(n)) for n in (prob.nx, prob.ny, prob.nz))
                c = i + prob.nx * (j + prob.ny * k)
                R_ref, Jrow, dphi = C.subgrid_row(prob, i, j, k)
                worst_R = max(worst_R, abs(R[c] - R_ref))
                scale_R = max(scale_R, abs(R_ref))
                cols = ci[rp[c]:rp[c + 1]]
                assert sorted(Jrow) == list(cols)
                if any(abs(dphi[L]) <= 32 * C.EPS32 * (abs(prob.p[c] - prob.p[L]) + 1.1e4 * abs(prob.depth[c] - prob.depth[L]))
                       for L in Jrow if L != c):
                    continue
                row = vals[rp[c]:rp[c + 1]].astype(np.float64)
                row[list(cols).index(c)] = diag[c]
                ref = np.array([Jrow[L] for L in cols])
                assert np.abs(row - ref).max() <= 1e-6 * np.abs(ref).max(), (m, i, j, k)
            assert worst_R <= 1e-6 * scale_R, (m, worst_R, scale_R)
    for g in grids:
        g.close()
