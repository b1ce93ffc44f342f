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

TOL = {"fp64": 1e-12, "mixed": 1e-6}


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


def _normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_handle_api_on_consecutive_calls(precision):
    import torch

    from paper_2304_11274_gb300.api import Grid

    lib = _lib()
    dtype = torch.float32 if precision == "mixed" else torch.float64
    prob = synth.make_problem(70, 37, 9, seed=99, connectivity=10, c_r=1e-9)
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
            torch.cuda.synchronize()
            expect.append((R.cpu().numpy(), vals.double().cpu().numpy(),
                           None if diag is None else diag.cpu().numpy()))
        nnz = g.nnz
        row_starts = g.pattern()[0][:-1].cpu().numpy()

    R = torch.empty(prob.n, dtype=torch.float64, device=dev)
    vals = torch.empty(nnz, dtype=dtype, device=dev)
    diag = torch.empty(prob.n, dtype=torch.float64, device=dev) if precision == "mixed" else None
    status = torch.ones(1, dtype=torch.int32, device=dev)
    prm = _params(prob.phys)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    prec = _capi.TPFA_MIXED if precision == "mixed" else _capi.TPFA_FP64
    for call, p in enumerate(ps):  # two calls in a row, different pressures
        R.fill_(np.nan)
        vals.fill_(np.nan)
        if diag is not None:
            diag.fill_(np.nan)
        rc = lib.tpfa_assemble_jacobian_static(prob.nx, prob.ny, prob.nz, ctypes.byref(prm), prec,
                                               ptr(perm), ptr(poro), ptr(depth), ptr(p), ptr(pn),
                                               ptr(R), ptr(vals), ptr(diag), ptr(status), stream)
        assert rc == 0, lib.tpfa_last_error_string()
        torch.cuda.synchronize()
        eR, ev, ed = expect[call]
        assert int(status.item()) == 0
        assert _normwise(R.cpu().numpy(), eR) <= TOL[precision]
        got = vals.double().cpu().numpy()
        row_err = (np.maximum.reduceat(np.abs(got - ev), row_starts) /
                   np.maximum.reduceat(np.abs(ev), row_starts))
        assert float(row_err.max()) <= TOL[precision]
        if ed is not None:
            assert _normwise(diag.cpu().numpy(), ed) <= TOL[precision]
