"""z-slabs of one grid (the decomposition over GPUs): every slab's owned rows
equal the whole grid's rows bit for bit once its halo planes hold the
neighbouring slabs' pressure (moved here by the library's peer-copy
exchange; all slabs on one device)."""
import numpy as np
import pytest
import torch

from paper_2304_11274_gb300 import synth

pytestmark = pytest.mark.gpu


def _planes(a, nxy, e0, e1):
    return a[e0 * nxy:e1 * nxy]


# nx < 256 (the one-cell march) and nx >= 256 even (the two-cell march);
# a slab of a single plane; more slabs than a block's planes
CASES = [((70, 41, 11), 10, "mixed", 2), ((70, 41, 11), 6, "fp64", 3), ((260, 37, 13), 10, "mixed", 3),
         ((260, 37, 13), 10, "fp64", 2), ((33, 17, 5), 10, "mixed", 5), ((64, 9, 20), 6, "mixed", 4)]


@pytest.mark.parametrize("shape,conn,precision,parts", CASES)
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_slabs_reproduce_the_whole_grid(shape, conn, precision, parts, c_r):
    from paper_2304_11274_gb300.api import Grid, Slab, slab_bounds
    nx, ny, nz = shape
    nxy = nx * ny
    prob = synth.make_problem(nx, ny, nz, seed=41, connectivity=conn, c_r=c_r)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    dtype = torch.float32 if precision == "mixed" else torch.float64
    with Grid(nx, ny, nz, prob.phys, precision, prob.perm, prob.poro, prob.depth) as g:
        g.set_state(prob.p, prob.pn)
        R, vals, diag = g.assemble_jacobian()
        g.sync_status()
        ref = (R.cpu(), vals.cpu(), None if diag is None else diag.cpu())
        starts = g.pattern()[0][::nxy].cpu()  # first CSR entry of each plane (and nnz)
    slabs, pres = [], []
    for r in range(parts):
        k0, k1, e0, e1 = slab_bounds(nz, parts, r)
        s = Slab(nx, ny, nz, k0, k1, prob.phys, precision, _planes(prob.perm, nxy, e0, e1),
                 _planes(prob.poro, nxy, e0, e1), _planes(prob.depth, nxy, e0, e1))
        p = torch.as_tensor(_planes(prob.p, nxy, e0, e1), device="cuda", dtype=dtype).clone()
        if k0 > e0:
            p[:nxy] = float("nan")  # halo planes start unknown: the exchange must fill them
        if e1 > k1:
            p[-nxy:] = float("nan")
        pn = torch.as_tensor(_planes(prob.pn, nxy, e0, e1), device="cuda", dtype=dtype)
        slabs.append(s)
        pres.append((p, pn))
    for lo, hi, (pl, _), (ph, _) in zip(slabs, slabs[1:], pres, pres[1:]):
        lo.exchange_with(hi, pl, ph)
    for s, (p, pn) in zip(slabs, pres):
        s.set_state(p, pn)
        R, vals, diag = s.assemble_jacobian()
        s.sync_status()
        Ro, vo, do = s.owned(R, vals, diag)
        k0, k1 = s.k0, s.k1
        assert torch.equal(Ro.cpu(), ref[0][k0 * nxy:k1 * nxy])
        assert torch.equal(vo.cpu(), ref[1][int(starts[k0]):int(starts[k1])])
        if do is not None:
            assert torch.equal(do.cpu(), ref[2][k0 * nxy:k1 * nxy])
        s.close()


def test_slab_rejects_calls_it_does_not_support():
    from paper_2304_11274_gb300.api import Slab
    from paper_2304_11274_gb300._capi import TPFAError
    prob = synth.make_problem(8, 6, 6, seed=3, connectivity=10)
    with Slab(8, 6, 6, 2, 4, prob.phys, "fp64", prob.perm[8 * 6:8 * 6 * 5], prob.poro[8 * 6:8 * 6 * 5],
              prob.depth[8 * 6:8 * 6 * 5]) as s:
        n = s.n
        s.set_state(prob.p[:n], prob.pn[:n])
        with pytest.raises(TPFAError):
            s.vjp(np.ones(n))
        with pytest.raises(TPFAError):
            s.jvp(np.ones(n))
