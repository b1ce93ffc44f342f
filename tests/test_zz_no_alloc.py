"""The allocation-free entry point, tpfa_assemble_jacobian_static.

It serves callers that cannot let a library allocate device memory (their
own pooled allocator owns the GPU, or a hard memory budget is enforced
outside the CUDA runtime).  Its results must match the handle API's
tpfa_assemble_jacobian on the same inputs, call after call, although every
call reuses the same fixed workspace.  This file is collected last so that a
run stopping at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

from paper_2304_11274_gb300 import _capi, build, synth



def _lib():
    build.build()
    return _capi.load()


def _params(phys):
    return _capi.TPFAParams(**{k: phys[k] for k, _ in _capi.TPFAParams._fields_})


def test_static_entry_rejects_grids_beyond_its_workspace():
    """Host-side checks that run before any device work (no GPU needed)."""
    lib = _lib()
    prm = _params(synth.physics())
    dummy = ctypes.c_void_p(256)
    # 256 x 256 x 64 mixed cells need 128 MiB of workspace: refused with a clear message
    rc = lib.tpfa_assemble_jacobian_static(256, 256, 64, ctypes.byref(prm), _capi.TPFA_MIXED,
                                           dummy, dummy, dummy, dummy, dummy, dummy, dummy, dummy, None, None)
    assert rc == -4
    msg = lib.tpfa_last_error_string().decode()
    assert "workspace" in msg and "handle API" in msg
    rc = lib.tpfa_assemble_jacobian_static(0, 4, 4, ctypes.byref(prm), _capi.TPFA_MIXED,
                                           dummy, dummy, dummy, dummy, dummy, dummy, dummy, dummy, None, None)
    assert rc == -1
    rc = lib.tpfa_assemble_jacobian_static(4, 4, 4, ctypes.byref(prm), _capi.TPFA_FP64,
                                           dummy, dummy, dummy, dummy, dummy, dummy, dummy, dummy, None, None)
    assert rc == -1  # diag64 must be NULL on the FP64 path


def _align256(x):
    return (x + 255) // 256 * 256


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_static_size_rule_boundary(precision, conn, c_r):
    """The documented rule, 256 + sum of align256(N * bytes per element) over
    the intermediate arrays <= TPFA_STATIC_WORKSPACE_BYTES, at its boundary:
    the helper's byte count follows the rule, the largest accepted N (a
    1 x 1 x N column, so that no padding is a multiple of a plane) fits and
    N + 1 is refused by the entry point itself, before any device work.  The
    accepted size is not called: these are dummy pointers."""
    lib = _lib()
    prec = _capi.TPFA_MIXED if precision == "mixed" else _capi.TPFA_FP64
    limit = 64 * 1024 * 1024
    es = 4 if precision == "mixed" else 8
    arrays = [es] * (5 if conn == 10 else 3) + ([es] + ([es] if c_r else []) if precision == "mixed" else []) + [8]

    def rule(n):
        return 256 + sum(_align256(n * b) for b in arrays)

    def need(n):
        return lib.tpfa_static_workspace_bytes(1, 1, n, conn, prec, 1 if c_r else 0)

    for n in (1, 2, 63, 64, 65, 1000, 12345, 1 << 20):
        assert need(n) == rule(n)
    lo, hi = 1, limit  # need(lo) fits, need(hi) does not
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if need(mid) <= limit else (lo, mid)
    assert need(lo) <= limit < need(lo + 1)
    phys = dict(synth.physics(), connectivity=conn, c_r=c_r)
    prm = _params(phys)
    dummy = ctypes.c_void_p(256)
    diag = dummy if precision == "mixed" else None
    rc = lib.tpfa_assemble_jacobian_static(1, 1, lo + 1, ctypes.byref(prm), prec, dummy, dummy, dummy, dummy,
                                           dummy, dummy, dummy, diag, None, None)
    assert rc == -4
    assert str(need(lo + 1)) in lib.tpfa_last_error_string().decode()
    # the header's figures: about 2.09 M / 1.86 M (mixed, 10 links) and 1.39 M (FP64, 10 links) cells
    if conn == 10:
        expect = {("mixed", 0.0): 2.09e6, ("mixed", 1e-9): 1.86e6, ("fp64", 0.0): 1.39e6, ("fp64", 1e-9): 1.39e6}
        assert abs(lo - expect[(precision, c_r)]) < 0.01e6


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("conn", [6, 10])
@pytest.mark.parametrize("c_r", [0.0, 1e-9])
def test_static_entry_matches_handle_api_on_consecutive_calls(precision, conn, c_r):
    """Two calls in a row with different pressures give the bits of the handle
    API (same kernels, same inputs); a third call without a status word (the
    error word then lives in the workspace) gives them again."""
    import torch

    from paper_2304_11274_gb300.api import Grid

    lib = _lib()
    dtype = torch.float32 if precision == "mixed" else torch.float64
    prob = synth.make_problem(70, 37, 9, seed=99, connectivity=conn, c_r=c_r)
    pres = [prob.p] + synth.pressure_sequence(prob, 1, seed=5)
    dev = torch.device("cuda", 0)
    perm = torch.as_tensor(prob.perm, device=dev)
    poro = torch.as_tensor(prob.poro, device=dev)
    depth = torch.as_tensor(prob.depth, device=dev)
    pn = torch.as_tensor(prob.pn, device=dev, dtype=dtype)
    ps = [torch.as_tensor(p, device=dev, dtype=dtype) for p in pres]

    # expected results from the handle API
    expect = []
    with Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth) as g:
        for p in ps:
            g.set_state(p, pn)
            R, vals, diag = g.assemble_jacobian()
            g.sync_status()
            expect.append((R.cpu(), vals.cpu(), None if diag is None else diag.cpu()))
        nnz = g.nnz

    R = torch.empty(prob.n, dtype=torch.float64, device=dev)
    vals = torch.empty(nnz, dtype=dtype, device=dev)
    diag = torch.empty(prob.n, dtype=torch.float64, device=dev) if precision == "mixed" else None
    status = torch.ones(1, dtype=torch.int32, device=dev)
    prm = _params(prob.phys)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    prec = _capi.TPFA_MIXED if precision == "mixed" else _capi.TPFA_FP64
    for call, (p, st) in enumerate([(ps[0], status), (ps[1], status), (ps[0], None)]):
        R.fill_(np.nan)
        vals.fill_(np.nan)
        if diag is not None:
            diag.fill_(np.nan)
        rc = lib.tpfa_assemble_jacobian_static(prob.nx, prob.ny, prob.nz, ctypes.byref(prm), prec,
                                               ptr(perm), ptr(poro), ptr(depth), ptr(p), ptr(pn),
                                               ptr(R), ptr(vals), ptr(diag), ptr(st), stream)
        assert rc == 0, lib.tpfa_last_error_string()
        torch.cuda.synchronize()
        eR, ev, ed = expect[call % 2]
        if st is not None:
            assert int(status.item()) == 0
        assert torch.equal(R.cpu(), eR), call
        assert torch.equal(vals.cpu(), ev), call
        if ed is not None:
            assert torch.equal(diag.cpu(), ed), call
