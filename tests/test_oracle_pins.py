"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute-force
enumeration of Section 5.1's neighbour definition, closed forms, conservation
and antisymmetry identities, hand-derived two-cell systems, a textbook graph
Laplacian, and central finite differences.  A dropped term, a flipped sign or
a transposed index in ``oracle/tpfa_oracle.c`` fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2304_11274_gb300 import synth

# ---------------------------------------------------------------- helpers


def lin(i, j, k, nx, ny):
    return i + nx * (j + ny * k)


def stencil_offsets(conn):
    """Section 5.1: (a) x-y cardinal, (b) x-y diagonal (10-point only), (c) z."""
    a = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
    b = [(1, 1, 0), (-1, -1, 0), (-1, 1, 0), (1, -1, 0)]
    c = [(0, 0, 1), (0, 0, -1)]
    return a + (b if conn == 10 else []) + c


def nnz_closed_form(nx, ny, nz, conn):
    """N + 2 * (number of links): x-links (nx-1) ny nz, y-links nx (ny-1) nz,
    z-links nx ny (nz-1), and per x-y plane 2 (nx-1)(ny-1) diagonal links."""
    links = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    if conn == 10:
        links += 2 * (nx - 1) * (ny - 1) * nz
    return nx * ny * nz + 2 * links


def dense(out, N):
    J = np.zeros((N, N))
    rp, ci = out["row_ptr"], out["col_idx"]
    for r in range(N):
        for e in range(rp[r], rp[r + 1]):
            J[r, ci[e]] = out["J"][e]
    return J


def rho_of(phys, p):
    return phys["rho_ref"] * np.exp(phys["c_f"] * (p - phys["p_ref"]))


# ---------------------------------------------------------------- pattern


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (3, 3, 3), (4, 2, 5), (5, 4, 1), (1, 6, 2), (6, 1, 3)])
@pytest.mark.parametrize("conn", [6, 10])
def test_pattern_matches_bruteforce_adjacency(shape, conn):
    """Every pair of cells whose coordinate difference is one of Section 5.1's
    offsets is linked, nothing else is; each row also holds its diagonal and
    lists columns in ascending order."""
    nx, ny, nz = shape
    N = nx * ny * nz
    offs = set(stencil_offsets(conn))
    coords = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    A = np.zeros((N, N), dtype=bool)
    for a, (i, j, k) in enumerate(coords):
        for b, (i2, j2, k2) in enumerate(coords):
            if a == b or (i2 - i, j2 - j, k2 - k) in offs:
                A[a, b] = True
    rp, ci = oracle.pattern(nx, ny, nz, conn)
    B = np.zeros((N, N), dtype=bool)
    for r in range(N):
        cols = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(cols) > 0), "columns must be strictly ascending"
        B[r, cols] = True
    assert np.array_equal(A, B)
    assert rp[-1] == nnz_closed_form(nx, ny, nz, conn)


def test_nnz_closed_form_known_sizes():
    """The 32^3 face-connected grid and an odd 10-point grid, counted by the oracle."""
    for (nx, ny, nz, conn) in [(32, 32, 32, 6), (17, 9, 5, 10), (33, 17, 9, 10)]:
        rp, _ = oracle.pattern(nx, ny, nz, conn)
        assert rp[-1] == nnz_closed_form(nx, ny, nz, conn)
    assert nnz_closed_form(32, 32, 32, 6) == 223232
    assert nnz_closed_form(512, 512, 256, 10) == 736101376


# ---------------------------------------------------------------- transmissibility


def test_transmissibility_homogeneous_closed_forms():
    """Uniform k: Upsilon = k * face area / centre distance for faces; for the
    diagonal of a 10 x 10 x 2 m cell, area/distance = 1 m."""
    phys = synth.physics()
    k = 3.7e-13
    dx, dy, dz = phys["dx"], phys["dy"], phys["dz"]
    assert oracle.link_trans(phys, k, k, 1, 0, 0) == pytest.approx(k * dy * dz / dx, rel=1e-15)
    assert oracle.link_trans(phys, k, k, 0, -1, 0) == pytest.approx(k * dx * dz / dy, rel=1e-15)
    assert oracle.link_trans(phys, k, k, 0, 0, 1) == pytest.approx(k * dx * dy / dz, rel=1e-15)
    assert oracle.link_trans(phys, k, k, 1, 1, 0) == pytest.approx(k * 1.0, rel=1e-14)
    assert oracle.link_trans(phys, k, k, -1, 1, 0) == pytest.approx(k * 1.0, rel=1e-14)


def test_transmissibility_series_law():
    """Two half-cells in series: 1/Upsilon = (d/2)/(k_K A) + (d/2)/(k_L A);
    symmetric in K and L, and zero when either cell is impermeable."""
    phys = synth.physics(dx=7.0, dy=3.0, dz=1.5)
    kK, kL = 2.0e-13, 5.0e-15
    A, d = phys["dy"] * phys["dz"], phys["dx"]
    expect = 1.0 / ((d / 2) / (kK * A) + (d / 2) / (kL * A))
    assert oracle.link_trans(phys, kK, kL, 1, 0, 0) == pytest.approx(expect, rel=1e-14)
    assert oracle.link_trans(phys, kK, kL, -1, 0, 0) == oracle.link_trans(phys, kL, kK, 1, 0, 0)
    assert oracle.link_trans(phys, kK, 0.0, 0, 0, 1) == 0.0


# ---------------------------------------------------------------- two-cell hand derivations


def _two_cell(phys, kK, kL, pK, pL, zK=None, zL=None, axis=0, flip=None):
    shape = [1, 1, 1]
    shape[axis] = 2
    nx, ny, nz = shape
    dzv = phys["dz"]
    depth = np.array([zK if zK is not None else 0.5 * dzv, zL if zL is not None else 0.5 * dzv])
    out = oracle.assemble(nx, ny, nz, phys, np.array([kK, kL]), np.array([0.2, 0.25]), depth,
                          np.array([pK, pL]), np.array([pK, pL]), flip=flip, want_links=True)
    return out


def test_two_cell_horizontal_hand_derivation():
    """Cells K=0, L=1 side by side (same depth), p_K > p_L: mass flows K -> L
    carrying the upstream density rho_K; R_K = +F, R_L = -F; the Jacobian is
    the hand derivative of T rho(p_up)/mu (p_K - p_L)."""
    phys = synth.physics(connectivity=6, c_f=1e-8, dt=1e300)  # no accumulation term
    k = 1e-13
    T = k * phys["dy"] * phys["dz"] / phys["dx"]
    pK, pL = 1.02e7, 0.99e7
    out = _two_cell(phys, k, k, pK, pL)
    rK, rL = rho_of(phys, np.array([pK, pL]))
    mu, cf = phys["mu"], phys["c_f"]
    F = T * rK / mu * (pK - pL)
    assert out["R"][0] == pytest.approx(F, rel=1e-13)
    assert out["R"][1] == pytest.approx(-F, rel=1e-13)
    # rows: [J00, J01], [J10, J11]
    J = out["J"]
    assert J[0] == pytest.approx(T * (cf * rK / mu * (pK - pL) + rK / mu), rel=1e-13)
    assert J[1] == pytest.approx(-T * rK / mu, rel=1e-13)
    # row L sees dPhi_LK < 0, so its upstream is K as well
    assert J[2] == pytest.approx(-T * (cf * rK / mu * (pK - pL) + rK / mu), rel=1e-13)
    assert J[3] == pytest.approx(T * rK / mu, rel=1e-13)
    # flipping the upwind of link (K, L) uses rho_L instead
    fl = np.array([0, 1, 0, 0], dtype=np.uint8)
    out2 = _two_cell(phys, k, k, pK, pL, flip=fl)
    assert out2["R"][0] == pytest.approx(T * rL / mu * (pK - pL), rel=1e-13)
    assert out2["J"][1] == pytest.approx(T * (cf * rL / mu * (pK - pL) - rL / mu), rel=1e-13)


def test_two_cell_vertical_gravity_hand_derivation():
    """K on top of L (depth grows downward).  dPhi_KL = (p_K - p_L) -
    rho_avg g (z_K - z_L); with p_L = p_K + 1.5 rho g dz the deeper cell is
    over-pressured beyond hydrostatic, so mass flows up: F_KL < 0 and the
    upstream density is rho_L."""
    phys = synth.physics(connectivity=6, dt=1e300)  # no accumulation term
    k = 2e-14
    dz, g, mu, cf = phys["dz"], phys["g"], phys["mu"], phys["c_f"]
    T = k * phys["dx"] * phys["dy"] / dz
    pK = 1.0e7
    pL = pK + 1.5 * 1000.0 * g * dz
    zK, zL = 0.5 * dz, 1.5 * dz
    out = _two_cell(phys, k, k, pK, pL, zK, zL, axis=2)
    rK, rL = rho_of(phys, np.array([pK, pL]))
    ravg = 0.5 * (rK + rL)
    dphi = (pK - pL) - ravg * g * (zK - zL)
    assert dphi < 0
    F = T * rL / mu * dphi
    assert out["R"][0] == pytest.approx(F, rel=1e-12)
    assert out["R"][1] == pytest.approx(-F, rel=1e-12)
    dd_dpL = -1.0 - 0.5 * cf * rL * g * (zK - zL)
    dd_dpK = 1.0 - 0.5 * cf * rK * g * (zK - zL)
    assert out["J"][1] == pytest.approx(T * (cf * rL / mu * dphi + rL / mu * dd_dpL), rel=1e-12)
    assert out["J"][0] == pytest.approx(T * rL / mu * dd_dpK, rel=1e-12)


def test_single_cell_accumulation_only():
    """A 1 x 1 x 1 grid has no links: R = V (phi rho - phi^n rho^n) / dt with
    phi = phi0 (1 + c_r (p - p_ref)); R = 0 when p = p^n."""
    phys = synth.physics(c_r=3e-9, c_f=2e-9)
    V = phys["dx"] * phys["dy"] * phys["dz"]
    p, pn, phi0 = 1.3e7, 1.1e7, 0.21
    out = oracle.assemble(1, 1, 1, phys, [1e-13], [phi0], [1.0], [p], [pn])
    def m(x):
        return phi0 * (1 + phys["c_r"] * (x - phys["p_ref"])) * rho_of(phys, x)
    assert out["R"][0] == pytest.approx(V * (m(p) - m(pn)) / phys["dt"], rel=1e-12)
    h = 1.0
    fd = V * (m(p + h) - m(p - h)) / (2 * h) / phys["dt"]
    assert out["J"][0] == pytest.approx(fd, rel=1e-7)
    out0 = oracle.assemble(1, 1, 1, phys, [1e-13], [phi0], [1.0], [pn], [pn])
    assert out0["R"][0] == 0.0


# ---------------------------------------------------------------- invariants


@pytest.fixture(scope="module")
def random_problem():
    return synth.make_problem(7, 5, 4, seed=11, connectivity=10, c_r=1e-9)


def test_flux_antisymmetry_bitwise(random_problem):
    """F_KL = -F_LK exactly (negating every operand of round-to-nearest
    arithmetic negates the result) wherever dPhi != 0."""
    pr = random_problem
    out = oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn, want_links=True)
    rp, ci, F, dphi = out["row_ptr"], out["col_idx"], out["F"], out["dphi"]
    pos = {}
    for r in range(pr.n):
        for e in range(rp[r], rp[r + 1]):
            pos[(r, ci[e])] = e
    checked = 0
    for (r, c), e in pos.items():
        if r == c:
            continue
        e2 = pos[(c, r)]
        assert dphi[e] == -dphi[e2]
        if dphi[e] != 0:
            assert F[e] == -F[e2]
            checked += 1
    assert checked > 0


def test_global_conservation(random_problem):
    """sum_K (R_K - A_K) = sum of all fluxes = 0 up to summation rounding."""
    pr = random_problem
    out = oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn, want_links=True)
    flux_sum = out["R"] - out["acc"]
    scale = np.abs(out["F"]).max()
    assert abs(flux_sum.sum()) <= 2 * pr.n * 11 * np.finfo(float).eps * scale
    assert np.abs(out["acc"]).max() > 0


def test_uniform_pressure_no_gravity_zero_flux():
    pr = synth.make_problem(6, 5, 4, seed=3, connectivity=10, g=0.0)
    p = np.full(pr.n, 1.234e7)
    out = oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, p, p, want_links=True)
    assert np.all(out["F"] == 0.0)
    assert np.all(out["R"] == 0.0)


def test_discrete_hydrostatic_equilibrium_zero_flux():
    """A laterally uniform column solving p_{k+1} = p_k + rho_avg g dz (the
    discrete hydrostatic balance) carries no flux: vertical fluxes vanish to
    rounding, lateral ones exactly."""
    nx, ny, nz = 4, 3, 6
    pr = synth.make_problem(nx, ny, nz, seed=5, connectivity=10)
    phys = pr.phys
    g, dz = phys["g"], phys["dz"]
    col = [1.0e7]
    for _ in range(nz - 1):
        pk = col[-1]
        q = pk + 1000.0 * g * dz
        for _ in range(200):
            q_new = pk + 0.5 * (rho_of(phys, pk) + rho_of(phys, q)) * g * dz
            if q_new == q:
                break
            q = q_new
        col.append(q)
    p = np.repeat(np.array(col), nx * ny)
    out = oracle.assemble(nx, ny, nz, phys, pr.perm, pr.poro, pr.depth, p, p, want_links=True)
    rp, ci, F = out["row_ptr"], out["col_idx"], out["F"]
    kmax = pr.perm.max()
    scale = 2 * kmax * phys["dx"] * phys["dy"] / dz * 1000.0 / phys["mu"] * 1000.0 * g * dz
    for r in range(pr.n):
        for e in range(rp[r], rp[r + 1]):
            c = ci[e]
            if c == r:
                continue
            if abs(c - r) == nx * ny:
                assert abs(F[e]) <= 1e-9 * scale
            else:
                assert F[e] == 0.0


@pytest.mark.parametrize("conn", [6, 10])
def test_linear_pressure_closed_form(conn):
    """Homogeneous k, g = 0, p = a + b x: each link carries T rho_up b dx / mu
    with upstream on the high-pressure (low-x) side, so an interior cell's
    flux sum is (T_x + n_d T_d) b dx (rho_i - rho_{i+1}) / mu, n_d the number
    of diagonal links on each side; the x = 0 cell only loses mass."""
    nx, ny, nz = 6, 4, 3
    phys = synth.physics(connectivity=conn, g=0.0, c_f=5e-9)
    k = 1e-13
    N = nx * ny * nz
    a, b = 1.0e7, -2.0e3  # pressure falls along +x
    x = np.tile(np.arange(nx) * phys["dx"], ny * nz)
    p = a + b * x
    out = oracle.assemble(nx, ny, nz, phys, np.full(N, k), np.full(N, 0.2), np.zeros(N), p, p)
    rho = rho_of(phys, a + b * np.arange(nx) * phys["dx"])
    mu, dxv = phys["mu"], phys["dx"]
    Tx = k * phys["dy"] * phys["dz"] / dxv
    Td = k * 1.0 if conn == 10 else 0.0
    drop = -b * dxv  # p_i - p_{i+1} > 0
    for kk in range(nz):
        for j in range(ny):
            nd = (j > 0) + (j < ny - 1)
            for i in range(nx):
                r = lin(i, j, kk, nx, ny)
                expect = 0.0
                if i + 1 < nx:  # outflow to i+1, upstream i
                    expect += (Tx + nd * Td) * rho[i] / mu * drop
                if i > 0:  # inflow from i-1, upstream i-1
                    expect -= (Tx + nd * Td) * rho[i - 1] / mu * drop
                assert out["R"][r] == pytest.approx(expect, rel=1e-12, abs=1e-12 * Tx * rho[0] / mu * drop)


def test_incompressible_jacobian_is_graph_laplacian():
    """c_f = 0 and c_r = 0: the Jacobian is (rho_ref / mu) times the
    transmissibility-weighted graph Laplacian (row sums zero)."""
    pr = synth.make_problem(4, 3, 3, seed=9, connectivity=10, c_f=0.0)
    phys = pr.phys
    out = oracle.assemble(pr.nx, pr.ny, pr.nz, phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    J = dense(out, pr.n)
    L = np.zeros((pr.n, pr.n))
    coords = [(i, j, k) for k in range(pr.nz) for j in range(pr.ny) for i in range(pr.nx)]
    idx = {c: n for n, c in enumerate(coords)}
    for (i, j, k), a in idx.items():
        for (di, dj, dk) in stencil_offsets(10):
            c = (i + di, j + dj, k + dk)
            if c in idx:
                t = oracle.link_trans(phys, pr.perm[a], pr.perm[idx[c]], di, dj, dk)
                L[a, idx[c]] -= t
                L[a, a] += t
    expect = phys["rho_ref"] / phys["mu"] * L
    assert np.allclose(J, expect, rtol=1e-13, atol=1e-13 * np.abs(expect).max())
    assert np.abs(J.sum(axis=1)).max() <= 1e-12 * np.abs(J).max()


def test_flux_jacobian_column_sums_vanish(random_problem):
    """sum_K R_flux,K is identically zero in p, so every column of the flux
    Jacobian sums to zero (away from exact upwind ties)."""
    pr = random_problem
    phys = dict(pr.phys, c_r=0.0, dt=1e300)  # accumulation term -> 0
    out = oracle.assemble(pr.nx, pr.ny, pr.nz, phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    J = dense(out, pr.n)
    assert np.abs(J.sum(axis=0)).max() <= 1e-13 * np.abs(J).max()


# ---------------------------------------------------------------- finite differences


def _fd_problem():
    return synth.make_problem(5, 4, 3, seed=21, connectivity=10, c_r=2e-9, c_f=3e-9)


def test_jacobian_matches_central_differences():
    """J[:, j] against (R(p + h e_j) - R(p - h e_j)) / 2h, h = 1e-6 |p_j|;
    links whose dPhi is within 4h of zero (an upwind switch inside the
    stencil) are masked."""
    pr = _fd_problem()
    phys = pr.phys
    args = (pr.nx, pr.ny, pr.nz, phys, pr.perm, pr.poro, pr.depth)
    base = oracle.assemble(*args, pr.p, pr.pn, want_links=True)
    J = dense(base, pr.n)
    rp, ci, dphi = base["row_ptr"], base["col_idx"], base["dphi"]
    compared = 0
    for jcol in range(pr.n):
        h = 1e-6 * abs(pr.p[jcol])
        pp, pm = pr.p.copy(), pr.p.copy()
        pp[jcol] += h
        pm[jcol] -= h
        fd = (oracle.assemble(*args, pp, pr.pn)["R"] - oracle.assemble(*args, pm, pr.pn)["R"]) / (2 * h)
        for r in range(pr.n):
            row = slice(rp[r], rp[r + 1])
            if np.any((np.abs(dphi[row]) < 4 * h) & (ci[row] != r)):
                continue
            scale = np.abs(J[r]).max()
            assert abs(fd[r] - J[r, jcol]) <= 1e-6 * scale, (r, jcol)
            compared += 1
    assert compared > pr.n * pr.n // 2


def test_vjp_pressure_is_transpose_product():
    """g_p = J^T v: the dot-product identity v^T (J w) = (J^T v)^T w, with J
    from the assembly and g_p from the separate scatter-form adjoint."""
    pr = _fd_problem()
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    J = dense(oracle.assemble(*args), pr.n)
    rng = np.random.default_rng(4)
    v, w = rng.standard_normal(pr.n), rng.standard_normal(pr.n)
    g_p, _ = oracle.vjp(*args, v)
    assert np.allclose(g_p, J.T @ v, rtol=1e-13, atol=1e-13 * np.abs(J).max())
    assert float(v @ (J @ w)) == pytest.approx(float(g_p @ w), rel=1e-11)


def test_vjp_logperm_matches_central_differences():
    """d(v^T R)/d(ln k) along random directions, by central differences."""
    pr = _fd_problem()
    rng = np.random.default_rng(8)
    v = rng.standard_normal(pr.n)
    _, g_lnk = oracle.vjp(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn, v)
    lnk = np.log(pr.perm)
    for _ in range(4):
        d = rng.standard_normal(pr.n)
        h = 1e-6
        def f(x):
            return float(v @ oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, np.exp(x), pr.poro, pr.depth,
                                             pr.p, pr.pn)["R"])
        fd = (f(lnk + h * d) - f(lnk - h * d)) / (2 * h)
        assert fd == pytest.approx(float(g_lnk @ d), rel=1e-6)


def test_vjp_pressure_matches_central_differences():
    pr = _fd_problem()
    rng = np.random.default_rng(12)
    v = rng.standard_normal(pr.n)
    g_p, _ = oracle.vjp(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn, v)
    for _ in range(4):
        d = rng.standard_normal(pr.n)
        h = 10.0  # Pa = 1e-6 |p|: large against ulp(1e7), small against the 1e5 Pa field scale
        def f(x):
            return float(v @ oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth,
                                             x, pr.pn)["R"])
        fd = (f(pr.p + h * d) - f(pr.p - h * d)) / (2 * h)
        assert fd == pytest.approx(float(g_p @ d), rel=1e-6)


def test_jvp_matches_directional_central_differences():
    """J w against (R(p + h w) - R(p - h w)) / 2h along random directions:
    pins the CSR product of the oracle's J w to the residual itself."""
    pr = _fd_problem()
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth)
    rng = np.random.default_rng(16)
    for _ in range(4):
        w = rng.standard_normal(pr.n)
        Jw, R = oracle.jvp(*args, pr.p, pr.pn, w)
        assert np.array_equal(R, oracle.assemble(*args, pr.p, pr.pn)["R"])
        h = 10.0  # Pa, as in the VJP differences
        fd = (oracle.assemble(*args, pr.p + h * w, pr.pn)["R"] - oracle.assemble(*args, pr.p - h * w, pr.pn)["R"]) / (2 * h)
        assert np.abs(fd - Jw).max() <= 1e-6 * np.abs(Jw).max()


def test_jvp_dot_product_identity_with_adjoint():
    """v^T (J w) = (J^T v)^T w with J w from the assembled CSR and J^T v from
    the separate scatter-form adjoint."""
    pr = _fd_problem()
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    rng = np.random.default_rng(20)
    for _ in range(3):
        v, w = rng.standard_normal(pr.n), rng.standard_normal(pr.n)
        Jw, _ = oracle.jvp(*args, w)
        g_p, _ = oracle.vjp(*args, v)
        assert float(v @ Jw) == pytest.approx(float(g_p @ w), rel=1e-11)


def test_jvp_of_constant_direction_is_accumulation_only_when_incompressible():
    """c_f = c_r = 0: rho is constant, the flux Jacobian is a weighted graph
    Laplacian whose rows sum to zero, so J 1 = dA/dp = 0 as well (the
    accumulation term is constant in p): J 1 vanishes to rounding."""
    pr = synth.make_problem(4, 3, 3, seed=5, connectivity=10, c_f=0.0, c_r=0.0)
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    Jw, _ = oracle.jvp(*args, np.ones(pr.n))
    J = oracle.assemble(*args)["J"]
    assert np.abs(Jw).max() <= 1e-13 * np.abs(J).max()


def test_newton_step_solves_linear_problem_exactly():
    """c_f = 0 with c_r != 0: rho is constant and phi linear in p, so R is
    affine in p (the upwind choice does not change rho_up) and one Newton
    step lands on R = 0 up to rounding."""
    pr = synth.make_problem(6, 5, 4, seed=31, connectivity=10, c_f=0.0, c_r=1e-8)
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth)
    p1, delta, R0 = oracle.newton_step(*args, pr.p, pr.pn)
    R1 = oracle.assemble(*args, p1, pr.pn)["R"]
    assert np.abs(R0).max() > 0
    assert np.abs(R1).max() <= 1e-9 * np.abs(R0).max()
    assert np.abs(delta).max() > 1.0  # a real step, not a no-op


def test_newton_converges_superlinearly():
    """A strongly compressible fluid (c_f = 1e-7 /Pa, c_r = 1e-8 /Pa): the
    residual ratio shrinks from step to step (quadratic convergence), where a
    wrong Jacobian entry would leave it roughly constant."""
    pr = synth.make_problem(6, 5, 4, seed=33, connectivity=10, c_f=1e-7, c_r=1e-8)
    args = (pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth)
    p = pr.p.copy()
    norms = [np.abs(oracle.assemble(*args, p, pr.pn)["R"]).max()]
    for _ in range(3):
        p, _, _ = oracle.newton_step(*args, p, pr.pn)
        norms.append(np.abs(oracle.assemble(*args, p, pr.pn)["R"]).max())
    r = [norms[k + 1] / norms[k] for k in range(3)]
    assert r[0] < 0.5
    assert r[1] < 0.2 * r[0] or norms[2] <= 1e-12 * norms[0]


# ---------------------------------------------------------------- general meshes

_KIND_OFFSETS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 1, 0)]


def _structured_as_mesh(pr):
    """The structured problem pr as a connection list: its links, each
    transmissibility from the oracle's two-point formula, V = dx dy dz."""
    a, b, kind = synth.structured_pairs(pr.nx, pr.ny, pr.nz, pr.phys["connectivity"])
    T = np.array([oracle.link_trans(pr.phys, pr.perm[x], pr.perm[y], *_KIND_OFFSETS[t])
                  for x, y, t in zip(a, b, kind)])
    V = np.full(pr.n, pr.phys["dx"] * pr.phys["dy"] * pr.phys["dz"])
    return a, b, T, V


@pytest.mark.parametrize("conn", [6, 10])
def test_mesh_of_structured_grid_matches_structured_oracle(conn):
    """A structured grid given as a connection list: the mesh pattern is the
    structured pattern and R, J agree with the structured oracle (two
    separate codes: adjacency from the list vs. Section 5.1's offsets)."""
    pr = synth.make_problem(5, 4, 3, seed=51, connectivity=conn, c_r=1e-9)
    a, b, T, V = _structured_as_mesh(pr)
    ref = oracle.assemble(pr.nx, pr.ny, pr.nz, pr.phys, pr.perm, pr.poro, pr.depth, pr.p, pr.pn)
    out = oracle.mesh_assemble(pr.n, pr.phys, a, b, T, V, pr.poro, pr.depth, pr.p, pr.pn)
    assert np.array_equal(out["row_ptr"], ref["row_ptr"]) and np.array_equal(out["col_idx"], ref["col_idx"])
    assert np.abs(out["R"] - ref["R"]).max() <= 1e-13 * np.abs(ref["R"]).max()
    assert np.abs(out["J"] - ref["J"]).max() <= 1e-13 * np.abs(ref["J"]).max()


def test_mesh_pattern_matches_bruteforce():
    m = synth.make_mesh(7, 5, 4, seed=52, connectivity=10)
    rp, ci, co = oracle.mesh_pattern(m.n, m.ci, m.cj)
    A = np.eye(m.n, dtype=bool)
    A[m.ci, m.cj] = True
    A[m.cj, m.ci] = True
    for K in range(m.n):
        assert list(ci[rp[K]:rp[K + 1]]) == list(np.flatnonzero(A[K]))
        for e in range(rp[K], rp[K + 1]):
            c = co[e]
            assert (c == -1) == (ci[e] == K)
            if c >= 0:
                assert {int(m.ci[c]), int(m.cj[c])} == {K, int(ci[e])}


def test_mesh_rejects_bad_connection_lists():
    with pytest.raises(ValueError):
        oracle.mesh_pattern(3, [0, 1], [1, 1])  # a cell joined to itself
    with pytest.raises(ValueError):
        oracle.mesh_pattern(3, [0, 1], [1, 0])  # the same pair twice
    with pytest.raises(ValueError):
        oracle.mesh_pattern(3, [0], [3])  # out of range


def test_mesh_fluxes_antisymmetric_and_conservative():
    m = synth.make_mesh(8, 6, 5, seed=53, connectivity=10, c_r=1e-9)
    out = oracle.mesh_assemble(m.n, m.phys, m.ci, m.cj, m.T, m.V, m.poro, m.depth, m.p, m.pn, want_links=True)
    rp, ci, F, dphi = out["row_ptr"], out["col_idx"], out["F"], out["dphi"]
    pos = {}
    for K in range(m.n):
        for e in range(rp[K], rp[K + 1]):
            pos[(K, int(ci[e]))] = e
    for (K, L), e in pos.items():
        if K != L and dphi[e] != 0.0:
            assert F[e] == -F[pos[(L, K)]]
    flux = out["R"] - out["acc"]
    assert abs(flux.sum()) <= 1e-12 * np.abs(F).sum()


def test_mesh_jacobian_matches_central_differences():
    m = synth.make_mesh(5, 4, 3, seed=54, connectivity=6, c_r=2e-9, c_f=3e-9)
    base = oracle.mesh_assemble(m.n, m.phys, m.ci, m.cj, m.T, m.V, m.poro, m.depth, m.p, m.pn, want_links=True)
    J = dense(base, m.n)
    rp, ci, dphi = base["row_ptr"], base["col_idx"], base["dphi"]
    compared = 0
    for jcol in range(m.n):
        h = 1e-6 * abs(m.p[jcol])
        pp, pm = m.p.copy(), m.p.copy()
        pp[jcol] += h
        pm[jcol] -= h
        Rp = oracle.mesh_assemble(m.n, m.phys, m.ci, m.cj, m.T, m.V, m.poro, m.depth, pp, m.pn)["R"]
        Rm = oracle.mesh_assemble(m.n, m.phys, m.ci, m.cj, m.T, m.V, m.poro, m.depth, pm, m.pn)["R"]
        fd = (Rp - Rm) / (2 * h)
        for r in range(m.n):
            row = slice(rp[r], rp[r + 1])
            if np.any((np.abs(dphi[row]) < 4 * h) & (ci[row] != r)):
                continue
            assert abs(fd[r] - J[r, jcol]) <= 1e-6 * np.abs(J[r]).max(), (r, jcol)
            compared += 1
    assert compared > m.n * m.n // 2


def test_mesh_two_cells_hand_derivation():
    """Two cells, one connection, no gravity, c_r = 0: R_0 = A_0 + T rho_up/mu (p0 - p1)."""
    phys = synth.physics(g=0.0, c_r=0.0)
    p = np.array([1.02e7, 1.0e7])
    pn = np.array([1.0e7, 1.0e7])
    T, V, poro = 3e-13, np.array([150.0, 250.0]), np.array([0.2, 0.25])
    out = oracle.mesh_assemble(2, phys, [0], [1], [T], V, poro, np.array([1.0, 1.0]), p, pn)
    rho = phys["rho_ref"] * np.exp(phys["c_f"] * (p - phys["p_ref"]))
    rhon = phys["rho_ref"] * np.exp(phys["c_f"] * (pn - phys["p_ref"]))
    F = T * rho[0] / phys["mu"] * (p[0] - p[1])  # cell 0 is upstream
    A = V * poro * (rho - rhon) / phys["dt"]
    assert out["R"][0] == pytest.approx(A[0] + F, rel=1e-12)
    assert out["R"][1] == pytest.approx(A[1] - F, rel=1e-12)
    dF0 = T / phys["mu"] * (phys["c_f"] * rho[0] * (p[0] - p[1]) + rho[0])
    assert out["J"][0] == pytest.approx(dF0 + V[0] * poro[0] * phys["c_f"] * rho[0] / phys["dt"], rel=1e-12)
    assert out["J"][1] == pytest.approx(-T * rho[0] / phys["mu"], rel=1e-12)


def test_upwind_tie_takes_the_neighbour():
    """Section 3's upwind rule picks rho_K only when dPhi_KL > 0 and the
    neighbour's density otherwise, so at an exact tie each row uses the OTHER
    cell's density.  Two stacked cells with g dz = 1 (exact), p_K = p_ref = 0
    and p_L tuned ulp by ulp until the oracle reports dPhi == 0.0 exactly."""
    phys = synth.physics(connectivity=6, dt=1e300, p_ref=0.0, c_f=1e-6, g=0.5, dz=2.0)
    k = 1e-13
    T = k * phys["dx"] * phys["dy"] / phys["dz"]
    zK, zL = 1.0, 3.0
    pL = 1000.0
    for _ in range(60):  # fixed point of p_L = rho_avg(p_L) (g (z_L - z_K) = 1)
        pL = 0.5 * (1000.0 + 1000.0 * math.exp(1e-6 * pL))
    found = None
    for step in range(-64, 65):
        cand = pL + step * np.spacing(pL)
        out = _two_cell(phys, k, k, 0.0, cand, zK, zL, axis=2)
        if out["dphi"][1] == 0.0:
            found = (cand, out)
            break
    assert found is not None, "no exact tie within 64 ulps"
    pL, out = found
    rK, rL = 1000.0, 1000.0 * math.exp(1e-6 * pL)
    mu, cf = phys["mu"], phys["c_f"]
    gdz = phys["g"] * (zK - zL)  # -1
    # row K: dPhi_KL = 0 is not > 0, so lambda = rho_L / mu
    assert out["J"][1] == pytest.approx(T * rL / mu * (-1.0 - 0.5 * cf * rL * gdz), rel=1e-13)
    assert out["J"][0] == pytest.approx(T * rL / mu * (1.0 - 0.5 * cf * rK * gdz), rel=1e-13)
    # row L: dPhi_LK = -0 is not > 0 either, so lambda = rho_K / mu
    assert out["J"][2] == pytest.approx(T * rK / mu * (-1.0 + 0.5 * cf * rK * gdz), rel=1e-13)
    assert abs(rL - rK) > 1e-4 * rK  # the two choices are distinguishable
