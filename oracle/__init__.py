"""FP64 CPU oracle for the TPFA residual and Jacobian (arXiv 2304.11274, Section 3).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline, reference and precision-statement legs of ``bench.py`` (all
outside its timed regions) are the only callers.  The product library never
imports, links or loads anything from this directory.

The arithmetic lives in ``tpfa_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only builds it with gcc and marshals NumPy
arrays through ctypes.  The functions follow the paper's notation:

* ``pattern``   -- adj(K) of Section 5.1 cases (a)-(c), as CSR (row_ptr, col_idx)
* ``assemble``  -- R of Eq. vk and J = dR/dp, cell loop then neighbour loop as
  in Algorithm 1
* ``vjp``       -- v^T dR/dp and v^T dR/d(ln k)
* ``jvp``       -- J w, the assembled Jacobian of Eq. vk times a vector (the
  plain definition: a CSR matrix-vector product over ``assemble``'s J)
* ``newton_step`` -- one Newton iteration on Eq. vk, J delta = -R solved
  directly (sparse LU), p + delta
* ``mesh_pattern``, ``mesh_assemble`` -- the same residual and Jacobian on a
  general mesh given as a list of connections (K, L, Upsilon_KL) with
  per-cell volumes
* ``link_trans`` -- the transmissibility of one link
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpfa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("rho_ref", ctypes.c_double),
        ("p_ref", ctypes.c_double),
        ("c_f", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("g", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("c_r", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("dz", ctypes.c_double),
        ("connectivity", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available); returns the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    d, ll, u8 = P(ctypes.c_double), P(ctypes.c_longlong), P(ctypes.c_ubyte)
    lib.orc_pattern.argtypes = [ctypes.c_int] * 4 + [ll, ll]
    lib.orc_pattern.restype = ctypes.c_longlong
    lib.orc_assemble.argtypes = [ctypes.c_int] * 3 + [P(OracleParams)] + [d] * 5 + [ll, ll, u8] + [d] * 5
    lib.orc_assemble.restype = ctypes.c_int
    lib.orc_vjp.argtypes = [ctypes.c_int] * 3 + [P(OracleParams)] + [d] * 6 + [d, d]
    lib.orc_vjp.restype = ctypes.c_int
    lib.orc_link_trans.argtypes = [P(OracleParams), ctypes.c_double, ctypes.c_double] + [ctypes.c_int] * 3
    lib.orc_link_trans.restype = ctypes.c_double
    lib.orc_mesh_pattern.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ll, ll, ll, ll, ll]
    lib.orc_mesh_pattern.restype = ctypes.c_longlong
    lib.orc_mesh_assemble.argtypes = [ctypes.c_longlong, P(OracleParams)] + [d] * 6 + [ll, ll, ll, u8] + [d] * 5
    lib.orc_mesh_assemble.restype = ctypes.c_int
    lib.orc_max_threads.argtypes = []
    lib.orc_max_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_set_threads.restype = None
    _lib = lib
    return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_params(phys: dict) -> OracleParams:
    """phys: dict with rho_ref, p_ref, c_f, mu, g, dt, c_r, dx, dy, dz, connectivity."""
    return OracleParams(**{k: phys[k] for k, _ in OracleParams._fields_})


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's row loops from now on (for timing it
    single-threaded and on all cores)."""
    _load().orc_set_threads(int(n))


def pattern(nx: int, ny: int, nz: int, conn: int):
    """CSR pattern of the Jacobian: (row_ptr int64[N+1], col_idx int64[nnz])."""
    lib = _load()
    N = nx * ny * nz
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    nnz = lib.orc_pattern(nx, ny, nz, conn, _ptr(row_ptr, ctypes.c_longlong), None)
    if nnz < 0:
        raise ValueError("bad grid or connectivity")
    col_idx = np.zeros(nnz, dtype=np.int64)
    lib.orc_pattern(nx, ny, nz, conn, _ptr(row_ptr, ctypes.c_longlong), _ptr(col_idx, ctypes.c_longlong))
    return row_ptr, col_idx


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def assemble(nx, ny, nz, phys, perm, poro, depth, p, pn, pat=None, flip=None, want_links=False):
    """R (N) and CSR values J (nnz) of Eq. vk; optionally per-link F, dPhi and
    the accumulation term.  Returns a dict."""
    lib = _load()
    q = make_params(phys)
    if pat is None:
        pat = pattern(nx, ny, nz, phys["connectivity"])
    row_ptr, col_idx = pat
    N = nx * ny * nz
    nnz = int(row_ptr[-1])
    perm, poro, depth, p, pn = (_f64(x).reshape(-1) for x in (perm, poro, depth, p, pn))
    for x in (perm, poro, depth, p, pn):
        assert x.size == N
    R = np.zeros(N)
    J = np.zeros(nnz)
    F = np.zeros(nnz) if want_links else None
    dphi = np.zeros(nnz) if want_links else None
    acc = np.zeros(N) if want_links else None
    fl = None
    if flip is not None:
        fl = np.ascontiguousarray(flip, dtype=np.uint8)
        assert fl.size == nnz
    rc = lib.orc_assemble(nx, ny, nz, ctypes.byref(q),
                          _ptr(perm, ctypes.c_double), _ptr(poro, ctypes.c_double),
                          _ptr(depth, ctypes.c_double), _ptr(p, ctypes.c_double), _ptr(pn, ctypes.c_double),
                          _ptr(row_ptr, ctypes.c_longlong), _ptr(col_idx, ctypes.c_longlong),
                          _ptr(fl, ctypes.c_ubyte),
                          _ptr(R, ctypes.c_double), _ptr(J, ctypes.c_double),
                          _ptr(F, ctypes.c_double), _ptr(dphi, ctypes.c_double), _ptr(acc, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle assemble failed")
    out = {"R": R, "J": J, "row_ptr": row_ptr, "col_idx": col_idx}
    if want_links:
        out.update(F=F, dphi=dphi, acc=acc)
    return out


def vjp(nx, ny, nz, phys, perm, poro, depth, p, pn, v):
    """(g_p, g_lnk): v^T dR/dp and v^T dR/d(ln k)."""
    lib = _load()
    q = make_params(phys)
    N = nx * ny * nz
    perm, poro, depth, p, pn, v = (_f64(x).reshape(-1) for x in (perm, poro, depth, p, pn, v))
    g_p = np.zeros(N)
    g_lnk = np.zeros(N)
    rc = lib.orc_vjp(nx, ny, nz, ctypes.byref(q),
                     _ptr(perm, ctypes.c_double), _ptr(poro, ctypes.c_double), _ptr(depth, ctypes.c_double),
                     _ptr(p, ctypes.c_double), _ptr(pn, ctypes.c_double), _ptr(v, ctypes.c_double),
                     _ptr(g_p, ctypes.c_double), _ptr(g_lnk, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle vjp failed")
    return g_p, g_lnk


def jvp(nx, ny, nz, phys, perm, poro, depth, p, pn, w, pat=None):
    """(J w, R): row K of J, in its CSR order, dotted with w (Eq. vk's
    Jacobian applied to a direction), and the residual of the same state."""
    out = assemble(nx, ny, nz, phys, perm, poro, depth, p, pn, pat=pat)
    w = _f64(w).reshape(-1)
    row_ptr, col_idx, J = out["row_ptr"], out["col_idx"], out["J"]
    # every row holds its diagonal, so no row is empty and reduceat sums
    # exactly the entries of each row
    Jw = np.add.reduceat(J * w[col_idx], row_ptr[:-1])
    return Jw, out["R"]


def jacobian_csr(out, n):
    """assemble()'s J as a scipy CSR matrix."""
    import scipy.sparse as sp
    return sp.csr_matrix((out["J"], out["col_idx"], out["row_ptr"]), shape=(n, n))


def newton_step(nx, ny, nz, phys, perm, poro, depth, p, pn):
    """(p + delta, delta, R): Newton's method on R(p) = 0 (Eq. vk, backward
    Euler), the linear system J delta = -R solved by sparse LU."""
    from scipy.sparse.linalg import spsolve
    p = _f64(p).reshape(-1)
    out = assemble(nx, ny, nz, phys, perm, poro, depth, p, pn)
    J = jacobian_csr(out, nx * ny * nz)
    delta = np.atleast_1d(spsolve(J.tocsc(), -out["R"]))
    return p + delta, delta, out["R"]


def mesh_pattern(n, ci, cj):
    """(row_ptr, col_idx, conn_of) of a connection list, columns ascending;
    conn_of[e] is the connection of entry e (-1 on the diagonal)."""
    lib = _load()
    ci = np.ascontiguousarray(ci, dtype=np.int64)
    cj = np.ascontiguousarray(cj, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    L = ctypes.c_longlong
    nnz = lib.orc_mesh_pattern(n, ci.size, _ptr(ci, L), _ptr(cj, L), _ptr(row_ptr, L), None, None)
    if nnz < 0:
        raise ValueError("bad connection list")
    col_idx = np.zeros(nnz, dtype=np.int64)
    conn_of = np.zeros(nnz, dtype=np.int64)
    nnz = lib.orc_mesh_pattern(n, ci.size, _ptr(ci, L), _ptr(cj, L), _ptr(row_ptr, L), _ptr(col_idx, L),
                               _ptr(conn_of, L))
    if nnz < 0:
        raise ValueError("bad connection list (duplicate pair)")
    return row_ptr, col_idx, conn_of


def mesh_assemble(n, phys, ci, cj, T, V, poro, depth, p, pn, pat=None, flip=None, want_links=False):
    """R and CSR J of Eq. vk on a connection list (see ``assemble``)."""
    lib = _load()
    q = make_params(phys)
    if pat is None:
        pat = mesh_pattern(n, ci, cj)
    row_ptr, col_idx, conn_of = pat
    nnz = int(row_ptr[-1])
    T = _f64(T).reshape(-1)
    V, poro, depth, p, pn = (_f64(x).reshape(-1) for x in (V, poro, depth, p, pn))
    for x in (V, poro, depth, p, pn):
        assert x.size == n
    R = np.zeros(n)
    J = np.zeros(nnz)
    F = np.zeros(nnz) if want_links else None
    dphi = np.zeros(nnz) if want_links else None
    acc = np.zeros(n) if want_links else None
    fl = None
    if flip is not None:
        fl = np.ascontiguousarray(flip, dtype=np.uint8)
        assert fl.size == nnz
    D, L = ctypes.c_double, ctypes.c_longlong
    rc = lib.orc_mesh_assemble(n, ctypes.byref(q), _ptr(T, D), _ptr(V, D), _ptr(poro, D), _ptr(depth, D),
                               _ptr(p, D), _ptr(pn, D), _ptr(row_ptr, L), _ptr(col_idx, L), _ptr(conn_of, L),
                               _ptr(fl, ctypes.c_ubyte), _ptr(R, D), _ptr(J, D), _ptr(F, D), _ptr(dphi, D),
                               _ptr(acc, D))
    if rc != 0:
        raise ValueError("oracle mesh assemble failed")
    out = {"R": R, "J": J, "row_ptr": row_ptr, "col_idx": col_idx, "conn_of": conn_of}
    if want_links:
        out.update(F=F, dphi=dphi, acc=acc)
    return out


def link_trans(phys, kK, kL, di, dj, dk):
    """Transmissibility of one link with offset (di, dj, dk)."""
    lib = _load()
    q = make_params(phys)
    return float(lib.orc_link_trans(ctypes.byref(q), float(kK), float(kL), int(di), int(dj), int(dk)))
