"""GPU assembly (C ABI through the Python binding) against the FP64 oracle.

Bars: pattern bit-exact; FP64 path <= 1e-12 (normwise residual, row-normwise
Jacobian); mixed path <= 1e-6 on the same FP32-rounded inputs; kernel
variants bit-identical to each other.
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

# Shapes spanning several 32-wide x-segments, several 32-row y-runs and
# several 4-plane z-blocks, with ragged tails and degenerate axes.
SHAPES = [(1, 1, 1), (1, 1, 5), (1, 6, 1), (5, 1, 1), (2, 3, 4), (7, 5, 3), (33, 17, 9), (40, 37, 6), (65, 3, 2)]


def _grid(prob, precision):
    from paper_2304_11274_gb300.api import Grid
    return Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth)


def run_gpu(prob, precision, kernel="auto", tiling=None):
    with _grid(prob, precision) as g:
        if tiling is not None:
            g.set_tiling(*tiling)
        g.set_state(prob.p, prob.pn)
        R, vals, diag = g.assemble_jacobian(kernel=kernel)
        g.sync_status()
        rp, ci = g.pattern()
        torch.cuda.synchronize()
        out = dict(R=R.cpu().numpy(), vals=vals.cpu().numpy(), rp=rp.cpu().numpy(), ci=ci.cpu().numpy(),
                   diag=None if diag is None else diag.cpu().numpy())
    return out


def problem(shape, conn, precision, c_r=0.0, seed=7, **kw):
    prob = synth.make_problem(*shape, seed=seed, connectivity=conn, c_r=c_r, **kw)
    return synth.round_to_f32(prob) if precision == "mixed" else prob


def gpu_jacobian_f64(out, ref):
    """GPU Jacobian values as FP64, with the FP64 diagonal on the mixed path."""
    J = out["vals"].astype(np.float64)
    if out["diag"] is not None:
        rp, ci = ref["row_ptr"], ref["col_idx"]
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        d = ci == rows
        J[d] = out["diag"]
    return J


@pytest.mark.parametrize("shape", SHAPES + [(32, 32, 32)])
@pytest.mark.parametrize("conn", [6, 10])
def test_pattern_bit_exact(shape, conn):
    prob = problem(shape, conn, "fp64")
    out = run_gpu(prob, "fp64")
    rp, ci = oracle.pattern(*shape, conn)
    assert np.array_equal(out["rp"], rp)
    assert np.array_equal(out["ci"].astype(np.int64), ci)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_parity_vs_oracle(shape, conn, precision, c_r):
    prob = problem(shape, conn, precision, c_r=c_r)
    ref = C.reference(prob, EPS[precision])
    out = run_gpu(prob, precision)
    eR = C.residual_error(out["R"], ref)
    eJ = C.jacobian_row_error(gpu_jacobian_f64(out, ref), ref)
    assert eR <= TOL[precision], eR
    assert eJ <= TOL[precision], eJ
    if precision == "mixed":
        # the float diagonal slot is the FP32 rounding of the compensated sum
        rows = np.repeat(np.arange(prob.n), np.diff(ref["row_ptr"]))
        d = ref["col_idx"] == rows
        assert np.allclose(out["vals"][d].astype(np.float64), out["diag"], rtol=2 * C.EPS32, atol=0)


@pytest.mark.parametrize("shape", [(70, 41, 11), (72, 41, 11), (71, 41, 11)])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_kernel_variants_bit_identical(shape, conn, precision, c_r):
    """Every variant gives the naive kernel's bits (TILED2 runs TILED where it
    does not apply: odd nx, the FP64 path)."""
    prob = problem(shape, conn, precision, c_r=c_r, seed=3)
    a = run_gpu(prob, precision, "naive")
    for kernel in ["tiled", "tiled2", "auto"]:
        b = run_gpu(prob, precision, kernel)
        assert np.array_equal(a["R"].view(np.uint64), b["R"].view(np.uint64)), kernel
        assert np.array_equal(a["vals"], b["vals"]), kernel
        if precision == "mixed":
            assert np.array_equal(a["diag"].view(np.uint64), b["diag"].view(np.uint64)), kernel


# nx even (the two-cell march's condition): one pair, one exact segment, a
# segment plus a 2-cell tail, a segment plus a 30-cell tail, several
# segments with ragged y-runs, single rows and more planes than a block holds.
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resolved_kernel_follows_the_documented_rule(precision):
    """AUTO runs TILED2 for mixed grids at least 256 wide with nx even, or
    128 or 192 wide, else TILED; TILED2 on odd nx or the FP64 path runs
    TILED."""
    from paper_2304_11274_gb300.api import Grid
    for shape, auto, two in [((256, 3, 2), "tiled2", "tiled2"), ((254, 3, 2), "tiled", "tiled2"),
                             ((257, 3, 2), "tiled", "tiled"), ((33, 4, 4), "tiled", "tiled"),
                             ((128, 3, 2), "tiled2", "tiled2"), ((192, 3, 2), "tiled2", "tiled2"),
                             ((160, 3, 2), "tiled", "tiled2"), ((64, 3, 2), "tiled", "tiled2")]:
        prob = problem(shape, 6, precision, seed=2)
        with Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth) as g:
            g.set_state(prob.p, prob.pn)
            want = (auto, two) if precision == "mixed" else ("tiled", "tiled")
            assert (g.kernel_in_use("auto"), g.kernel_in_use("tiled2")) == want, shape
            assert g.kernel_in_use("naive") == "naive" and g.kernel_in_use("tiled") == "tiled"


X2_SHAPES = [(2, 3, 2), (64, 5, 3), (66, 9, 5), (94, 7, 4), (128, 66, 9), (130, 41, 11), (256, 1, 6), (6, 70, 1)]


@pytest.mark.parametrize("shape", X2_SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_two_cell_march_bit_identical(shape, conn, c_r):
    """The march with two cells per lane (links as paired halves, x-links and
    the links into the previous row reused by negation, ties recomputed
    after the march) gives the naive kernel's bits under every tiling."""
    prob = problem(shape, conn, "mixed", c_r=c_r, seed=5)
    a = run_gpu(prob, "mixed", "naive")
    for tiling in [(32, 4), (1, 8), (7, 4), (64, 8), (16, 4)]:
        _same_bits(a, run_gpu(prob, "mixed", "tiled2", tiling=tiling), "mixed")


@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("shape", [(130, 37, 5), (64, 64, 3)])
def test_two_cell_march_ties_in_every_direction(conn, shape):
    """Exact ties dPhi == 0 on x, y and diagonal links, inside a lane's pair,
    across lanes and across segments: the reused links at a tie are
    recomputed, so the rows equal the naive kernel's bit for bit."""
    prob = C.tie_pairs_problem("mixed", conn, shape=shape)
    a = run_gpu(prob, "mixed", "naive")
    for tiling in [(32, 4), (5, 8)]:
        _same_bits(a, run_gpu(prob, "mixed", "tiled2", tiling=tiling), "mixed")
        _same_bits(a, run_gpu(prob, "mixed", "tiled", tiling=tiling), "mixed")


def _same_bits(a, b, precision):
    assert np.array_equal(a["R"].view(np.uint64), b["R"].view(np.uint64))
    assert np.array_equal(a["vals"].view(np.uint32 if precision == "mixed" else np.uint64),
                          b["vals"].view(np.uint32 if precision == "mixed" else np.uint64))
    if precision == "mixed":
        assert np.array_equal(a["diag"].view(np.uint64), b["diag"].view(np.uint64))


# nx a multiple of 4 (the TMA march's condition): one partial segment, a
# segment plus a ragged 4-cell tail, several segments with ragged y-runs, a
# single row, and more planes than a block holds.
TMA_SHAPES = [(4, 3, 2), (36, 5, 3), (72, 41, 11), (128, 66, 9), (64, 1, 5)]


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_tma_march_bit_identical(shape, conn, c_r):
    """The march with its row inputs delivered as TMA boxes (elements outside
    the grid zero-filled by the copy engine; x-segments past the grid's
    extent only keep the ring's protocol) gives the naive kernel's bits
    under every tiling, and so does the library's automatic choice."""
    prob = problem(shape, conn, "mixed", c_r=c_r, seed=5)
    a = run_gpu(prob, "mixed", "naive")
    for tiling in [(32, 4), (1, 8), (7, 4), (64, 8)]:
        _same_bits(a, run_gpu(prob, "mixed", "tiled_tma", tiling=tiling), "mixed")
    _same_bits(a, run_gpu(prob, "mixed", "auto"), "mixed")


def test_tma_march_follows_the_bound_pressure():
    """The tensor map of p is re-encoded when the bound pointer changes
    (set_pressure, set_state): each call assembles the pressure bound at
    that moment."""
    base = problem((72, 40, 9), 10, "mixed", seed=8)
    ps = [base.p] + synth.pressure_sequence(base, 2, seed=4)
    with _grid(base, "mixed") as g:
        g.set_state(ps[0], base.pn)
        for p in ps + [ps[0]]:
            g.set_pressure(p)
            R_t, v_t, d_t = (x.clone() for x in g.assemble_jacobian(kernel="tiled_tma"))
            R_n, v_n, d_n = g.assemble_jacobian(kernel="naive")
            torch.cuda.synchronize()
            assert torch.equal(R_t, R_n) and torch.equal(v_t, v_n) and torch.equal(d_t, d_n)
        g.sync_status()


def test_tma_march_conditions():
    """The TMA march refuses what it cannot load (nx not a multiple of 4, an
    FP64 grid, a pressure pointer off a 16-byte boundary); the automatic
    choice (the per-lane march) still assembles such a state, with the naive
    kernel's bits."""
    from paper_2304_11274_gb300.api import TPFAError
    for shape, precision in [((70, 9, 5), "mixed"), ((72, 9, 5), "fp64")]:
        prob = problem(shape, 10, precision)
        with _grid(prob, precision) as g:
            g.set_state(prob.p, prob.pn)
            with pytest.raises(TPFAError) as ei:
                g.assemble_jacobian(kernel="tiled_tma")
            assert ei.value.name == "TPFA_ERR_INVALID_ARG"
    prob = problem((72, 9, 5), 10, "mixed")
    buf = torch.zeros(prob.n + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.as_tensor(prob.p, dtype=torch.float32, device="cuda")
    p_off = buf[1:]  # 4 bytes past a 16-byte boundary
    with _grid(prob, "mixed") as g:
        g.set_state(p_off, prob.pn)
        with pytest.raises(TPFAError) as ei:
            g.assemble_jacobian(kernel="tiled_tma")
        assert ei.value.name == "TPFA_ERR_INVALID_ARG"
        R_a, v_a, d_a = (x.clone() for x in g.assemble_jacobian(kernel="auto"))
        R_n, v_n, d_n = g.assemble_jacobian(kernel="naive")
        torch.cuda.synchronize()
        assert torch.equal(R_a, R_n) and torch.equal(v_a, v_n) and torch.equal(d_a, d_n)
        g.sync_status()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_only_equals_fused(precision):
    prob = problem((37, 29, 7), 10, precision)
    with _grid(prob, precision) as g:
        g.set_state(prob.p, prob.pn)
        R1 = g.assemble_residual()
        R2, _, _ = g.assemble_jacobian()
        torch.cuda.synchronize()
        assert torch.equal(R1, R2)


def test_config0_full_parity():
    """32^3, 6 face links, plain FP64 (the small seeded workload)."""
    prob = synth.config_problem(0)
    ref = C.reference(prob, C.EPS64)
    out = run_gpu(prob, "fp64")
    assert C.residual_error(out["R"], ref) <= 1e-12
    assert C.jacobian_row_error(gpu_jacobian_f64(out, ref), ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_layered_high_contrast(precision):
    """The precision study's medium (log10 k per layer ~ U[-18, -12], 5e6 to
    3e7 Pa) on a grid the oracle finishes in seconds."""
    prob = synth.make_problem(24, 20, 16, seed=synth.BASE_SEED + 2, connectivity=10, layered=True,
                              layered_pressure=True)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    ref = C.reference(prob, EPS[precision])
    out = run_gpu(prob, precision)
    assert C.residual_error(out["R"], ref) <= TOL[precision]
    assert C.jacobian_row_error(gpu_jacobian_f64(out, ref), ref) <= TOL[precision]


@pytest.mark.parametrize("conn", [6, 10])
def test_transmissibility_matches_oracle(conn):
    prob = problem((9, 8, 5), conn, "fp64")
    from paper_2304_11274_gb300.api import Grid
    with Grid(prob.nx, prob.ny, prob.nz, prob.phys, "fp64", prob.perm, prob.poro, prob.depth) as g:
        Ts = [g.transmissibility(w).cpu().numpy() for w in range(5 if conn == 10 else 3)]
    offs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 1, 0)]
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    for w, T in enumerate(Ts):
        di, dj, dk = offs[w]
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    c = i + nx * (j + ny * k)
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        d = ii + nx * (jj + ny * kk)
                        expect = oracle.link_trans(prob.phys, prob.perm[c], prob.perm[d], di, dj, dk)
                        assert T[c] == pytest.approx(expect, rel=1e-15)
                    else:
                        assert T[c] == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,kernel", [((8, 8, 4), "auto"), ((128, 6, 4), "tiled2"), ((130, 6, 4), "tiled2")])
@pytest.mark.parametrize("bad", [37, -1, np.inf])
def test_nonfinite_pressure_is_reported(precision, shape, kernel, bad):
    """A NaN or infinite pressure, inside the grid or at its last cell,
    with the one-cell and the two-cell marches."""
    from paper_2304_11274_gb300.api import TPFAError
    prob = problem(shape, 10, precision)
    p = prob.p.copy()
    if bad == np.inf:
        p[prob.n // 2] = np.inf
    else:
        p[bad] = np.nan
    with _grid(prob, precision) as g:
        g.set_state(p, prob.pn)
        g.assemble_jacobian(kernel=kernel)
        with pytest.raises(TPFAError) as ei:
            g.sync_status()
        assert ei.value.name == "TPFA_ERR_NONFINITE"
        # the flag is cleared once reported
        g.set_state(prob.p, prob.pn)
        g.assemble_jacobian()
        g.sync_status()


def test_assemble_before_state_is_an_error():
    from paper_2304_11274_gb300.api import TPFAError
    prob = problem((4, 4, 4), 6, "fp64")
    with _grid(prob, "fp64") as g:
        with pytest.raises(TPFAError) as ei:
            g.assemble_jacobian()
        assert ei.value.name == "TPFA_ERR_NO_STATE"


@pytest.mark.parametrize("shape", [(35, 21, 6), (33, 17, 40), (20, 9, 137)])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("tiling", [(32, 4), (16, 8)])
def test_host_buffer_entry_point_matches_device_call(shape, precision, tiling):
    """The host-buffer entry point pipelines uploads, assembly and downloads
    over z-slabs (one slab for nz <= 8, several above): every output equals
    the device call's bit for bit, whatever the block height."""
    prob = problem(shape, 10, precision)
    dt = torch.float32 if precision == "mixed" else torch.float64
    with _grid(prob, precision) as g:
        g.set_tiling(*tiling)
        g.set_state(prob.p, prob.pn)
        R, vals, diag = g.assemble_jacobian()
        torch.cuda.synchronize()
        ph = torch.as_tensor(prob.p).to(dt).pin_memory()
        Rh = torch.full((prob.n,), np.nan, dtype=torch.float64).pin_memory()
        vh = torch.full((g.nnz,), np.nan, dtype=dt).pin_memory()
        dh = torch.full((prob.n,), np.nan, dtype=torch.float64).pin_memory() if precision == "mixed" else None
        g.assemble_jacobian_host(ph, Rh, vh, dh)
        assert torch.equal(Rh, R.cpu())
        assert torch.equal(vh, vals.cpu())
        if dh is not None:
            assert torch.equal(dh, diag.cpu())
        g.sync_status()


def test_alloc_failure_reports_oom(monkeypatch):
    from paper_2304_11274_gb300.api import TPFAError
    prob = problem((6, 5, 4), 10, "mixed")
    before = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("TPFA_FAULT_INJECT", "alloc")
    with pytest.raises(TPFAError) as ei:
        _grid(prob, "mixed")
    assert ei.value.name == "TPFA_ERR_OOM"
    monkeypatch.delenv("TPFA_FAULT_INJECT")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= before - (4 << 20)


# ------------------------------------------------------------------ full sizes, sampled rows


def _sampled_rows(prob, precision, nsample, seed):
    """GPU rows at full size against the oracle on each row's clipped
    3 x 3 x 3 box, for random cells plus the eight corners."""
    from paper_2304_11274_gb300.api import Grid
    rng = np.random.default_rng(seed)
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    cells = [(i, j, k) for i in (0, nx - 1) for j in (0, ny - 1) for k in (0, nz - 1)]
    cells += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(nsample)]
    with Grid(nx, ny, nz, prob.phys, precision, prob.perm, prob.poro, prob.depth) as g:
        g.set_state(prob.p, prob.pn)
        R, vals, diag = g.assemble_jacobian()
        g.sync_status()
        rp, ci = g.pattern()
        lin = torch.as_tensor([i + nx * (j + ny * k) for (i, j, k) in cells], device="cuda")
        starts = rp[lin]
        ends = rp[lin + 1]
        width = int((ends - starts).max())
        idx = (starts[:, None] + torch.arange(width, device="cuda")[None, :]).clamp(max=g.nnz - 1)
        Rs = R[lin].cpu().numpy()
        Vs = vals[idx].double().cpu().numpy()
        Cs = ci[idx].cpu().numpy()
        Ds = diag[lin].cpu().numpy() if diag is not None else None
        lens = (ends - starts).cpu().numpy()
        del R, vals, diag, rp, ci
    worst_R, worst_J, scale_R, skipped = 0.0, 0.0, 0.0, 0
    eps = EPS[precision]
    for n, (i, j, k) in enumerate(cells):
        R_ref, Jrow, dphi = C.subgrid_row(prob, i, j, k)
        c = i + nx * (j + ny * k)
        cols = Cs[n, :lens[n]]
        assert sorted(Jrow.keys()) == list(cols), "pattern row mismatch"
        scale_R = max(scale_R, abs(R_ref))
        worst_R = max(worst_R, abs(Rs[n] - R_ref))
        amb = any(abs(dphi[L]) <= 32 * eps * (abs(prob.p[c] - prob.p[L]) + 1.1e3 * 9.81 * abs(prob.depth[c] - prob.depth[L]))
                  for L in Jrow if L != c)
        if amb:
            skipped += 1
            continue
        row = Vs[n, :lens[n]].copy()
        if Ds is not None:
            row[list(cols).index(c)] = Ds[n]
        ref = np.array([Jrow[L] for L in cols])
        worst_J = max(worst_J, float(np.abs(row - ref).max() / np.abs(ref).max()))
    return worst_R / scale_R, worst_J, skipped, len(cells)


@pytest.mark.slow
def test_full_size_paper_shaped_grid_sampled():
    """512 x 512 x 256, 10 links, mixed path: the benchmark's workload."""
    prob = synth.round_to_f32(synth.config_problem(1))
    eR, eJ, skipped, n = _sampled_rows(prob, "mixed", 3000, seed=1)
    assert eR <= 1e-6 and eJ <= 1e-6, (eR, eJ)
    assert skipped <= n // 100


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_layered_grid_sampled(precision):
    """256^3 high-contrast layered medium, both paths."""
    prob = synth.config_problem(2)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    eR, eJ, skipped, n = _sampled_rows(prob, precision, 2000, seed=2)
    assert eR <= TOL[precision] and eJ <= TOL[precision], (eR, eJ)
    assert skipped <= n // 100


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_precision_study_layered_full_grid(precision):
    """The precision study on every row of the 256^3 layered medium (log10 k
    per layer ~ U[-18, -12], 5e6 to 3e7 Pa): normwise residual and row-wise
    Jacobian errors within the bars, and the max / RMS entrywise relative
    error printed for the record."""
    prob = synth.config_problem(2)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    out = run_gpu(prob, precision)
    ref = C.reference(prob, EPS[precision])
    J = gpu_jacobian_f64(out, ref)
    eR = C.residual_error(out["R"], ref)
    eJ = C.jacobian_row_error(J, ref)
    emax, erms = C.entry_stats(J, ref)
    print(f"\nprecision study 256^3 layered {precision}: residual {eR:.3e}, jacobian row {eJ:.3e}, "
          f"entrywise max {emax:.3e} rms {erms:.3e}, ambiguous links {int(ref['ambiguous'].sum())}")
    assert eR <= TOL[precision] and eJ <= TOL[precision], (eR, eJ)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("conn", [6, 10])
def test_reused_link_ties_are_fixed_up(precision, conn):
    """The tiled kernel reuses the links into the previous y-row by negation
    and recomputes the rows where one was an exact tie: its output must equal
    the naive kernel's bit for bit on a grid built to contain such ties."""
    prob = C.tie_sweep_problem(precision, conn)
    if precision == "fp64":
        ref = oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p,
                              prob.pn, want_links=True)
        rows = np.repeat(np.arange(prob.n), np.diff(ref["row_ptr"]))
        vertical = (rows >= prob.nx) & (ref["col_idx"] < prob.nx)  # row-1 cells' links into row 0
        assert np.any(ref["dphi"][vertical] == 0.0)
    a = run_gpu(prob, precision, "naive")
    for kernel in ["tiled", "tiled_tma", "tiled2"] if precision == "mixed" else ["tiled"]:
        _same_bits(a, run_gpu(prob, precision, kernel), precision)
