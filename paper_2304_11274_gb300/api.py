"""PyTorch-facing wrapper of the TPFA C ABI (include/tpfa.h).

PyTorch supplies device memory and streams; every step of the assembly runs
in the library's CUDA kernels.  Tensors handed to ``set_state`` are borrowed
by the library, so this wrapper keeps references to them.

Physics follows arXiv 2304.11274, Section 3 (Eq. vk, Eq. flux-calc, Eq.
density, Algorithm 1); see include/tpfa.h for the conventions.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _capi
from ._capi import TPFA_FP64, TPFA_MIXED, TPFAError, check

PRECISIONS = {"fp64": TPFA_FP64, "mixed": TPFA_MIXED}


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _unused_mesh_params() -> dict:
    """Placeholders for the parameters a mesh does not use (cell sizes and
    connectivity), so that a mesh's physics dict may omit them."""
    return {"dx": 1.0, "dy": 1.0, "dz": 1.0, "connectivity": 6}


def params_struct(phys: dict) -> _capi.TPFAParams:
    return _capi.TPFAParams(**{k: phys[k] for k, _ in _capi.TPFAParams._fields_})


def _dev_f64(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)


class Grid:
    """A structured grid with its rock properties resident on the GPU.

    nx, ny, nz  : grid size (cell (i, j, k) is element i + nx (j + ny k))
    phys        : dict of rho_ref, p_ref, c_f, mu, g, dt, c_r, dx, dy, dz, connectivity
    precision   : "fp64" or "mixed"
    perm, poro, depth : N values each (array-like or tensors), SI units
    """

    def __init__(self, nx, ny, nz, phys, precision, perm, poro, depth, device="cuda"):
        self.lib = _capi.load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self.phys = dict(phys)
        self.precision = precision
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float32 if precision == "mixed" else torch.float64
        prm = params_struct(self.phys)
        with torch.cuda.device(self.device):
            k = _dev_f64(perm, self.device)
            ph = _dev_f64(poro, self.device)
            z = _dev_f64(depth, self.device)
            h = ctypes.c_void_p()
            self._create(h, prm, k, ph, z)
        self.handle = h
        nnz = ctypes.c_longlong()
        check(self.lib.tpfa_grid_info(h, None, None, None, None, ctypes.byref(nnz), None))
        self.nnz = int(nnz.value)
        self._p = None
        self._pn = None

    def _create(self, h, prm, k, ph, z):
        check(self.lib.tpfa_create_grid(ctypes.byref(h), self.nx, self.ny, self.nz, ctypes.byref(prm),
                                        PRECISIONS[self.precision], _ptr(k), _ptr(ph), _ptr(z), _stream()))

    # -- lifetime
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.tpfa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state
    def _field(self, x):
        if isinstance(x, torch.Tensor) and x.device == self.device and x.dtype == self.dtype and x.is_contiguous():
            t = x
        else:
            t = torch.as_tensor(np.asarray(x) if not isinstance(x, torch.Tensor) else x).to(
                device=self.device, dtype=self.dtype).contiguous()
        if t.numel() != self.n:
            raise ValueError(f"expected {self.n} values, got {t.numel()}")
        return t

    def set_state(self, p, pn, stream=None):
        """Bind p^{n+1} and p^n (computes m^n on the device)."""
        p, pn = self._field(p), self._field(pn)
        check(self.lib.tpfa_set_state(self.handle, _ptr(p), _ptr(pn), _stream(stream)))
        self._p, self._pn = p, pn

    def set_pressure(self, p):
        p = self._field(p)
        check(self.lib.tpfa_set_pressure(self.handle, _ptr(p)))
        self._p = p

    # -- outputs
    def empty_outputs(self):
        R = torch.empty(self.n, dtype=torch.float64, device=self.device)
        vals = torch.empty(self.nnz, dtype=self.dtype, device=self.device)
        diag = torch.empty(self.n, dtype=torch.float64, device=self.device) if self.precision == "mixed" else None
        return R, vals, diag

    def assemble_residual(self, R=None, stream=None):
        if R is None:
            R = torch.empty(self.n, dtype=torch.float64, device=self.device)
        check(self.lib.tpfa_assemble_residual(self.handle, _ptr(R), _stream(stream)))
        return R

    def assemble_jacobian(self, R=None, vals=None, diag=None, kernel="auto", stream=None, want_residual=True):
        """Fused residual + Jacobian.  Returns (R, vals, diag64); diag64 is
        None on the FP64 path (the diagonal is in vals)."""
        if vals is None:
            R0, vals, diag0 = self.empty_outputs()
            R = R0 if (R is None and want_residual) else R
            diag = diag0 if diag is None else diag
        check(self.lib.tpfa_assemble_jacobian_kernel(self.handle, _capi.KERNELS[kernel], _ptr(R), _ptr(vals),
                                                     _ptr(diag), _stream(stream)))
        return R, vals, diag

    def assemble_jacobian_host(self, p_host: torch.Tensor, R_host=None, vals_host=None, diag_host=None, stream=None):
        """End-to-end call with host buffers (pinned CPU tensors recommended)."""
        if p_host.device.type != "cpu" or p_host.dtype != self.dtype or p_host.numel() != self.n:
            raise ValueError("p_host must be a CPU tensor of the field dtype with N values")
        check(self.lib.tpfa_assemble_jacobian_host(self.handle, _ptr(p_host), _ptr(R_host), _ptr(vals_host),
                                                   _ptr(diag_host), _stream(stream)))
        return R_host, vals_host, diag_host

    def set_permeability(self, perm, stream=None):
        """Replace k (m^2); recomputes the transmissibilities on the device."""
        k = _dev_f64(perm, self.device)
        if k.numel() != self.n:
            raise ValueError(f"expected {self.n} values, got {k.numel()}")
        check(self.lib.tpfa_set_permeability(self.handle, _ptr(k), _stream(stream)))
        self._perm = k  # read asynchronously: keep it alive

    def set_log_permeability(self, log_k, stream=None):
        """Replace ln k (natural log of m^2); the library forms k = exp(ln k)
        and recomputes the transmissibilities on the device."""
        lk = _dev_f64(log_k, self.device)
        if lk.numel() != self.n:
            raise ValueError(f"expected {self.n} values, got {lk.numel()}")
        check(self.lib.tpfa_set_log_permeability(self.handle, _ptr(lk), _stream(stream)))
        self._perm = lk  # read asynchronously: keep it alive

    def vjp(self, v, want_lnk=True, kernel="auto", stream=None):
        """(g_p, g_lnk) = (v^T dR/dp, v^T dR/d ln k) at the bound state, FP64."""
        v = _dev_f64(v, self.device)
        g_p = torch.empty(self.n, dtype=torch.float64, device=self.device)
        g_lnk = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_lnk else None
        check(self.lib.tpfa_vjp_kernel(self.handle, _capi.KERNELS[kernel], _ptr(v), _ptr(g_p), _ptr(g_lnk),
                                       _stream(stream)))
        self._v = v
        return g_p, g_lnk

    def jvp(self, w, want_residual=False, out=None, kernel="auto", stream=None):
        """J w at the bound state without storing J (FP64); with
        ``want_residual`` also R of the same pass.  Returns (Jw, R or None)."""
        w = _dev_f64(w, self.device)
        if w.numel() != self.n:
            raise ValueError(f"expected {self.n} values, got {w.numel()}")
        Jw = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        R = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_residual else None
        check(self.lib.tpfa_jvp_kernel(self.handle, _capi.KERNELS[kernel], _ptr(w), _ptr(Jw), _ptr(R),
                                       _stream(stream)))
        self._w = w
        return Jw, R

    @staticmethod
    def _krylov(rtol, max_iters, check_every, precond="zline"):
        return _capi.TPFAKrylovOpts(int(max_iters), float(rtol), int(check_every), _capi.PRECONDITIONERS[precond])

    @staticmethod
    def _stats(st):
        return {k: getattr(st, k) for k, _ in _capi.TPFAKrylovStats._fields_}

    def linear_solve(self, b, rtol=1e-8, max_iters=1000, check_every=8, precond="zline", out=None, stream=None):
        """x with J x = b (J at the bound state; BiCGStab preconditioned by
        the z-line ("zline") or diagonal ("jacobi") part of J, FP64 vectors).
        Returns (x, stats); raises TPFAError (TPFA_ERR_NO_CONVERGENCE) if the
        tolerance is not met."""
        b = _dev_f64(b, self.device)
        if b.numel() != self.n:
            raise ValueError(f"expected {self.n} values, got {b.numel()}")
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        st = _capi.TPFAKrylovStats()
        opts = self._krylov(rtol, max_iters, check_every, precond)
        rc = self.lib.tpfa_linear_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(st),
                                        _stream(stream))
        self.last_stats = self._stats(st)
        check(rc)
        return x, self.last_stats

    def newton_step(self, p, rtol=1e-8, max_iters=1000, check_every=8, want_residual=False, want_delta=False,
                    precond="zline", stream=None):
        """One Newton step of Eq. vk in place on p (a device tensor of the
        field dtype, bound as the pressure).  Returns (stats, R(p) or None,
        delta or None)."""
        if not isinstance(p, torch.Tensor) or p.device != self.device or p.dtype != self.dtype \
                or not p.is_contiguous() or p.numel() != self.n:
            raise ValueError("p must be a contiguous device tensor of the field dtype with N values")
        R = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_residual else None
        d = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_delta else None
        st = _capi.TPFAKrylovStats()
        opts = self._krylov(rtol, max_iters, check_every, precond)
        self._p = p
        rc = self.lib.tpfa_newton_step(self.handle, _ptr(p), ctypes.byref(opts), ctypes.byref(st), _ptr(R),
                                       _ptr(d), _stream(stream))
        self.last_stats = self._stats(st)
        check(rc)
        return self.last_stats, R, d

    def pattern(self, stream=None):
        """(row_ptr int64[N+1], col_idx int32[nnz]) as device tensors."""
        rp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        check(self.lib.tpfa_copy_pattern(self.handle, _ptr(rp), _ptr(ci), _stream(stream)))
        return rp, ci

    def transmissibility(self, which: int, stream=None):
        out = torch.empty(self.n, dtype=self.dtype, device=self.device)
        check(self.lib.tpfa_get_transmissibility(self.handle, int(which), _ptr(out), _stream(stream)))
        return out

    def sync_status(self, stream=None):
        check(self.lib.tpfa_sync_status(self.handle, _stream(stream)))

    # -- tiling
    def kernel_in_use(self, kernel="auto"):
        """Name of the variant an assemble_jacobian(kernel=...) call runs on
        this grid in its current state (the library resolves it)."""
        out = ctypes.c_int()
        check(self.lib.tpfa_resolve_kernel(self.handle, _capi.KERNELS[kernel], ctypes.byref(out)))
        return {v: k for k, v in _capi.KERNELS.items()}[out.value]

    def tiling(self):
        jy, w = ctypes.c_int(), ctypes.c_int()
        check(self.lib.tpfa_get_tiling(self.handle, ctypes.byref(jy), ctypes.byref(w)))
        return jy.value, w.value

    def set_tiling(self, rows_per_march, warps_per_block):
        check(self.lib.tpfa_set_tiling(self.handle, int(rows_per_march), int(warps_per_block)))

    def autotune(self, cache_path=None, stream=None):
        """Pick the tiling by timing (or from the cache file); returns it."""
        path = cache_path.encode() if cache_path else None
        check(self.lib.tpfa_autotune(self.handle, path, _stream(stream)))
        return self.tiling()


def slab_bounds(nz, parts, part):
    """(k0, k1, e0, e1): the planes [k0, k1) of z-slab `part` of `parts` and
    the planes [e0, e1) its handle holds (the slab and its halo planes)."""
    lib = _capi.load()
    v = [ctypes.c_int() for _ in range(4)]
    check(lib.tpfa_slab_bounds(int(nz), int(parts), int(part), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


MATH_FNS = {"exp_fp64": 0, "expm1_fp64": 1, "expm1_f32": 2}


def math_eval(fn: str, x: torch.Tensor, stream=None) -> torch.Tensor:
    """The library's exponential `fn` ("exp_fp64", "expm1_fp64" or
    "expm1_f32") of every element of x, as FP64 on x's device
    (tpfa_math_eval)."""
    lib = _capi.load()
    x = x.to(dtype=torch.float64).contiguous()
    y = torch.empty_like(x)
    check(lib.tpfa_math_eval(MATH_FNS[fn], _ptr(x), _ptr(y), x.numel(), _stream(stream)))
    return y


class Slab(Grid):
    """Planes [k0, k1) of an nx x ny x nz grid with one halo plane on each
    side that exists (a z-slab of a decomposition over GPUs; Section 5's
    element-per-column mapping with the exchange of neighbour values).

    perm, poro, depth, and the pressures bound later, hold the planes [e0, e1)
    of slab_bounds: n = nx ny (e1 - e0) values.  Outputs have the sizes of
    that local grid; assemblies write only the owned rows (see owned()),
    which equal the whole grid's rows once the halo planes hold the
    neighbouring slabs' pressure (exchange_with, or
    distributed.slab_halo_exchange across processes)."""

    def __init__(self, nx, ny, nz, k0, k1, phys, precision, perm, poro, depth, device="cuda"):
        self.nz_global, self.k0, self.k1 = int(nz), int(k0), int(k1)
        e0, e1 = max(self.k0 - 1, 0), min(self.k1 + 1, self.nz_global)
        self.e0, self.e1 = e0, e1
        super().__init__(nx, ny, e1 - e0, phys, precision, perm, poro, depth, device)
        k0_, k1_, o0, o1 = (ctypes.c_int() for _ in range(4))
        r0, r1, n0, n1 = (ctypes.c_longlong() for _ in range(4))
        check(self.lib.tpfa_slab_info(self.handle, *[ctypes.byref(x) for x in (k0_, k1_, o0, o1, r0, r1, n0, n1)]))
        self.own = (o0.value, o1.value)
        self.rows = (r0.value, r1.value)
        self.entries = (n0.value, n1.value)

    def _create(self, h, prm, k, ph, z):
        check(self.lib.tpfa_create_slab(ctypes.byref(h), self.nx, self.ny, self.nz_global, self.k0, self.k1,
                                        ctypes.byref(prm), PRECISIONS[self.precision], _ptr(k), _ptr(ph), _ptr(z),
                                        _stream()))

    def owned(self, R=None, vals=None, diag=None):
        """Views of the owned rows of this slab's outputs."""
        r0, r1 = self.rows
        e0, e1 = self.entries
        return (None if R is None else R[r0:r1], None if vals is None else vals[e0:e1],
                None if diag is None else diag[r0:r1])

    def exchange_with(self, upper, p_self, p_upper, stream=None):
        """Copy the halo planes between this slab (the lower one) and the
        adjacent `upper` slab (peer copies; same or different devices)."""
        check(self.lib.tpfa_slab_exchange(self.handle, _ptr(p_self), upper.handle, _ptr(p_upper), _stream(stream)))


class Ensemble:
    """Grids of uneven sizes assembled by one persistent, graph-captured launch.

    The grids (mixed path, same connectivity) are borrowed; keep them alive.
    Each model's outputs are bit-identical to its own Grid.assemble_jacobian."""

    def __init__(self, grids):
        self.lib = _capi.load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.handle.value for g in self.grids])
        h = ctypes.c_void_p()
        check(self.lib.tpfa_create_ensemble(ctypes.byref(h), len(self.grids), arr))
        self.handle = h
        self._outs = [None] * len(self.grids)

    def set_outputs(self, m, R, vals, diag):
        check(self.lib.tpfa_ensemble_set_outputs(self.handle, int(m), _ptr(R), _ptr(vals), _ptr(diag)))
        self._outs[m] = (R, vals, diag)

    def allocate_outputs(self):
        """Allocate and bind (R, vals, diag64) for every model; returns them."""
        outs = []
        for m, g in enumerate(self.grids):
            R, vals, diag = g.empty_outputs()
            self.set_outputs(m, R, vals, diag)
            outs.append((R, vals, diag))
        return outs

    def assemble(self, stream=None):
        check(self.lib.tpfa_assemble_batch(self.handle, _stream(stream)))

    def tiling(self):
        jy, w, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        tiles = ctypes.c_longlong()
        check(self.lib.tpfa_ensemble_tiling(self.handle, ctypes.byref(jy), ctypes.byref(w), ctypes.byref(tiles),
                                            ctypes.byref(b)))
        return {"rows_per_march": jy.value, "warps_per_block": w.value, "tiles": tiles.value, "blocks": b.value}

    def autotune(self, cache_path=None, stream=None):
        path = cache_path.encode() if cache_path else None
        check(self.lib.tpfa_ensemble_autotune(self.handle, path, _stream(stream)))
        return self.tiling()

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.tpfa_destroy_ensemble(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mesh:
    """A general mesh given as a connection list (cells ci[c], cj[c] joined by
    transmissibility T[c]) with per-cell volume, porosity and depth; the
    residual and Jacobian of Eq. vk on it, on the GPU.

    n           : number of cells
    ci, cj, T   : connection list (int cell indices, m^3 transmissibilities)
    V, poro, depth : per-cell fields (m^3, -, m positive down)
    phys        : dict of rho_ref, p_ref, c_f, mu, g, dt, c_r (cell sizes and
                  connectivity are not used)
    precision   : "mixed" or "fp64"
    """

    def __init__(self, n, ci, cj, T, V, poro, depth, phys, precision="mixed", device="cuda"):
        self.lib = _capi.load()
        self.n = int(n)
        self.phys = dict(phys)
        self.precision = precision
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float32 if precision == "mixed" else torch.float64
        prm = params_struct({**_unused_mesh_params(), **self.phys})
        with torch.cuda.device(self.device):
            a = torch.as_tensor(np.ascontiguousarray(ci, dtype=np.int32), device=self.device)
            b = torch.as_tensor(np.ascontiguousarray(cj, dtype=np.int32), device=self.device)
            t = _dev_f64(T, self.device)
            v, ph, z = (_dev_f64(x, self.device) for x in (V, poro, depth))
            if not (a.numel() == b.numel() == t.numel()):
                raise ValueError("ci, cj and T must have the same length")
            h = ctypes.c_void_p()
            check(self.lib.tpfa_create_mesh(ctypes.byref(h), self.n, a.numel(), ctypes.byref(prm),
                                            PRECISIONS[precision], _ptr(a), _ptr(b), _ptr(t), _ptr(v), _ptr(ph),
                                            _ptr(z), _stream()))
        self.handle = h
        nnz, nc = ctypes.c_longlong(), ctypes.c_longlong()
        check(self.lib.tpfa_mesh_info(h, None, ctypes.byref(nc), ctypes.byref(nnz), None))
        self.nnz, self.nc = int(nnz.value), int(nc.value)
        self._p = self._pn = None

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.tpfa_destroy_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    _field = Grid._field

    def set_state(self, p, pn, stream=None):
        p, pn = self._field(p), self._field(pn)
        check(self.lib.tpfa_mesh_set_state(self.handle, _ptr(p), _ptr(pn), _stream(stream)))
        self._p, self._pn = p, pn

    def set_pressure(self, p):
        p = self._field(p)
        check(self.lib.tpfa_mesh_set_pressure(self.handle, _ptr(p)))
        self._p = p

    def empty_outputs(self):
        R = torch.empty(self.n, dtype=torch.float64, device=self.device)
        vals = torch.empty(self.nnz, dtype=self.dtype, device=self.device)
        diag = torch.empty(self.n, dtype=torch.float64, device=self.device) if self.precision == "mixed" else None
        return R, vals, diag

    def assemble(self, R=None, vals=None, diag=None, want_residual=True, stream=None):
        """Fused residual + Jacobian: (R, vals, diag64), CSR order of pattern()."""
        if vals is None:
            R0, vals, diag0 = self.empty_outputs()
            R = R if R is not None else (R0 if want_residual else None)
            diag = diag if diag is not None else diag0
        check(self.lib.tpfa_mesh_assemble(self.handle, _ptr(R), _ptr(vals), _ptr(diag), _stream(stream)))
        return R, vals, diag

    def assemble_residual(self, R=None, stream=None):
        if R is None:
            R = torch.empty(self.n, dtype=torch.float64, device=self.device)
        check(self.lib.tpfa_mesh_assemble(self.handle, _ptr(R), None, None, _stream(stream)))
        return R

    def pattern(self, stream=None):
        rp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        check(self.lib.tpfa_mesh_copy_pattern(self.handle, _ptr(rp), _ptr(ci), _stream(stream)))
        return rp, ci

    def sync_status(self, stream=None):
        check(self.lib.tpfa_mesh_sync_status(self.handle, _stream(stream)))


class TPFAResidual(torch.autograd.Function):
    """R(p, ln k) of Eq. vk on a Grid whose previous-step state is bound.

    forward(grid, p, log_k) -> R (FP64, N).  log_k is the natural log of the
    permeability; the grid's transmissibilities are recomputed when it
    changes.  backward runs the library's adjoint kernel (checkpoint-free:
    nothing is saved but p and log_k)."""

    @staticmethod
    def forward(ctx, grid, p, log_k):
        _apply_log_k(grid, log_k)
        grid.set_pressure(p.detach())
        R = grid.assemble_residual()
        ctx.grid = grid
        ctx.save_for_backward(p, log_k)
        return R

    @staticmethod
    def backward(ctx, gR):
        p, log_k = ctx.saved_tensors
        grid = ctx.grid
        _apply_log_k(grid, log_k)
        grid.set_pressure(p.detach())
        g_p, g_lnk = grid.vjp(gR.detach().to(torch.float64).contiguous(), want_lnk=ctx.needs_input_grad[2])
        gp = g_p.to(p.dtype) if ctx.needs_input_grad[1] else None
        gk = g_lnk.to(log_k.dtype) if ctx.needs_input_grad[2] else None
        return None, gp, gk


def _apply_log_k(grid, log_k):
    # Always re-applied: a tensor's address and version do not identify its
    # contents (the caching allocator reuses addresses).
    grid.set_log_permeability(log_k.detach())


def residual(grid, p, log_k):
    """Differentiable residual: TPFAResidual.apply(grid, p, log_k)."""
    return TPFAResidual.apply(grid, p, log_k)


__all__ = ["Grid", "Slab", "slab_bounds", "Ensemble", "TPFAError", "PRECISIONS", "TPFAResidual", "residual"]
