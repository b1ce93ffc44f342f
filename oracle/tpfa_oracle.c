/*
 * tpfa_oracle.c -- plain, slow, FP64 CPU oracle for the TPFA residual and
 * Jacobian of single-phase compressible flow on a structured 3D grid
 * (arXiv 2304.11274, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library, and it is compiled on its own with
 * `gcc -O2 -ffp-contract=off` so that no multiply-add contraction changes
 * the order of operations written below.
 *
 * What it computes, in the paper's terms:
 *   - adj(K): the neighbours of Section 5.1's three cases -- (a) the four
 *     in-plane cardinal cells, (b) the four in-plane diagonal cells (only with
 *     10-point connectivity), (c) the cells above and below.  Cells outside
 *     the grid are not neighbours (closed, no-flow boundary).
 *   - rho(p) = rho_ref * exp(c_f (p - p_ref))                    (Eq. density)
 *   - phi(p) = phi0 * (1 + c_r (p - p_ref))   (the paper gives no porosity
 *     law; c_r = 0 makes phi = phi0)
 *   - dPhi_KL = (p_K - p_L) - rho_avg g (z_K - z_L), rho_avg the arithmetic
 *     mean of rho_K and rho_L, z the cell-centre depth (positive down).  This
 *     is Eq. flux-calc with K and L exchanged and z measured as depth, the
 *     form under which the upwind rule and the sign of Eq. vk agree: F_KL is
 *     the mass OUTFLOW from K to L.
 *   - upwind (Section 3): lambda = rho_K / mu if dPhi_KL > 0, else rho_L / mu.
 *   - F_KL = Upsilon_KL * lambda * dPhi_KL                      (Eq. flux-calc)
 *   - Upsilon_KL (the paper names it but gives no formula): two-point
 *     harmonic form, 2 k_K k_L / (k_K + k_L) times area / distance; for an
 *     in-plane diagonal the distance is sqrt(dx^2 + dy^2) and the area
 *     dz * dx * dy / sqrt(dx^2 + dy^2).
 *   - R_K = V (phi(p_K) rho(p_K) - phi(pn_K) rho(pn_K)) / dt + sum_L F_KL
 *                                                  (Eq. vk, Algorithm 1)
 *   - J_KL = dR_K / dp_L, written out analytically from the formulas above.
 *   - the vector-Jacobian product of R with respect to p and ln k.
 *
 * The loops follow Algorithm 1: an outer loop over cells K, an inner loop over
 * L in adj(K) in the order the paper lists the neighbours, densities
 * evaluated inside the inner loop, the flux added to r_K.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double rho_ref; /* reference density, kg/m^3 */
    double p_ref;   /* reference pressure, Pa */
    double c_f;     /* fluid compressibility, 1/Pa */
    double mu;      /* viscosity, Pa s */
    double g;       /* gravitational acceleration, m/s^2 */
    double dt;      /* time step, s */
    double c_r;     /* rock compressibility, 1/Pa (0 = constant porosity) */
    double dx, dy, dz; /* cell size, m */
    int connectivity;  /* 6 (faces) or 10 (faces + in-plane diagonals) */
} orc_params;

/* Neighbour offsets (di, dj, dk) in the order Section 5.1 lists them:
 * (a) cardinal x-y, (b) diagonal x-y, (c) vertical. */
static const int ORC_NB[10][3] = {
    {+1, 0, 0}, {-1, 0, 0}, {0, +1, 0}, {0, -1, 0},     /* (a) */
    {+1, +1, 0}, {-1, -1, 0}, {-1, +1, 0}, {+1, -1, 0}, /* (b) */
    {0, 0, +1}, {0, 0, -1},                              /* (c) */
};

static int orc_valid_params(int nx, int ny, int nz, const orc_params* q) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || q == NULL) return 0;
    if (q->connectivity != 6 && q->connectivity != 10) return 0;
    return 1;
}

/* Enumerate adj(K) in the paper's order.  Writes up to 10 linear indices and
 * the matching stencil slot numbers; returns how many. */
static int orc_adj(int nx, int ny, int nz, int conn, long long K, long long* L, int* slot) {
    long long nxy = (long long)nx * ny;
    int k = (int)(K / nxy);
    int j = (int)((K - (long long)k * nxy) / nx);
    int i = (int)(K - (long long)k * nxy - (long long)j * nx);
    int n = 0;
    for (int s = 0; s < 10; ++s) {
        if (conn == 6 && s >= 4 && s < 8) continue;
        int ii = i + ORC_NB[s][0], jj = j + ORC_NB[s][1], kk = k + ORC_NB[s][2];
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
        L[n] = (long long)kk * nxy + (long long)jj * nx + ii;
        slot[n] = s;
        ++n;
    }
    return n;
}

static double orc_density(const orc_params* q, double p) {
    return q->rho_ref * exp(q->c_f * (p - q->p_ref));
}

static double orc_porosity(const orc_params* q, double phi0, double p) {
    return phi0 * (1.0 + q->c_r * (p - q->p_ref));
}

/* Transmissibility between two cells a stencil offset apart. */
static double orc_trans(const orc_params* q, double kK, double kL, int di, int dj, int dk) {
    if (kK <= 0.0 || kL <= 0.0) return 0.0;
    double kh = 2.0 * kK * kL / (kK + kL);
    double area, dist;
    if (dk != 0) {
        area = q->dx * q->dy;
        dist = q->dz;
    } else if (di != 0 && dj != 0) {
        dist = sqrt(q->dx * q->dx + q->dy * q->dy);
        area = q->dz * q->dx * q->dy / dist;
    } else if (di != 0) {
        area = q->dy * q->dz;
        dist = q->dx;
    } else {
        area = q->dx * q->dz;
        dist = q->dy;
    }
    return kh * area / dist;
}

/* Pattern of the Jacobian: row K holds K itself and adj(K), columns
 * ascending.  row_ptr has N+1 entries; col_idx (may be NULL to count only)
 * has row_ptr[N] entries.  Returns nnz, or -1 on bad arguments. */
long long orc_pattern(int nx, int ny, int nz, int conn, long long* row_ptr, long long* col_idx) {
    orc_params q;
    memset(&q, 0, sizeof q);
    q.connectivity = conn;
    if (!orc_valid_params(nx, ny, nz, &q)) return -1;
    long long N = (long long)nx * ny * nz;
    long long nnz = 0;
    long long L[10];
    int slot[10];
    for (long long K = 0; K < N; ++K) {
        if (row_ptr) row_ptr[K] = nnz;
        int n = orc_adj(nx, ny, nz, conn, K, L, slot);
        long long cols[11];
        cols[0] = K;
        for (int a = 0; a < n; ++a) cols[a + 1] = L[a];
        /* insertion sort, at most 11 entries */
        for (int a = 1; a <= n; ++a) {
            long long v = cols[a];
            int b = a - 1;
            while (b >= 0 && cols[b] > v) { cols[b + 1] = cols[b]; --b; }
            cols[b + 1] = v;
        }
        if (col_idx)
            for (int a = 0; a <= n; ++a) col_idx[nnz + a] = cols[a];
        nnz += n + 1;
    }
    if (row_ptr) row_ptr[N] = nnz;
    return nnz;
}

/* CSR position of column c in row K, or -1. */
static long long orc_find(const long long* row_ptr, const long long* col_idx, long long K, long long c) {
    for (long long e = row_ptr[K]; e < row_ptr[K + 1]; ++e)
        if (col_idx[e] == c) return e;
    return -1;
}

/* One connection K -> L seen from row K: the flux and its two pressure
 * derivatives.  flip != 0 reverses the upwind choice (used by tests to build
 * the other admissible Jacobian where dPhi is within rounding of zero). */
typedef struct {
    double dphi, F, dF_dpK, dF_dpL, dF_dT;
    int up_is_K;
} orc_conn;

static orc_conn orc_connection(const orc_params* q, double T, double pK, double pL,
                               double zK, double zL, int flip) {
    orc_conn r;
    /* Algorithm 1: densities of K and L evaluated for this connection */
    double rhoK = orc_density(q, pK);
    double rhoL = orc_density(q, pL);
    double drhoK = q->c_f * rhoK; /* d rho / dp */
    double drhoL = q->c_f * rhoL;
    double rho_avg = 0.5 * (rhoK + rhoL);
    double gdz = q->g * (zK - zL);
    r.dphi = (pK - pL) - rho_avg * gdz;
    int up_K = r.dphi > 0.0;
    if (flip) up_K = !up_K;
    r.up_is_K = up_K;
    double rho_up = up_K ? rhoK : rhoL;
    double lam = rho_up / q->mu;
    r.F = T * lam * r.dphi;
    r.dF_dT = lam * r.dphi;
    double ddphi_dpK = 1.0 - 0.5 * drhoK * gdz;
    double ddphi_dpL = -1.0 - 0.5 * drhoL * gdz;
    double dlam_dpK = up_K ? drhoK / q->mu : 0.0;
    double dlam_dpL = up_K ? 0.0 : drhoL / q->mu;
    r.dF_dpK = T * (dlam_dpK * r.dphi + lam * ddphi_dpK);
    r.dF_dpL = T * (dlam_dpL * r.dphi + lam * ddphi_dpL);
    return r;
}

/* Accumulation term of Eq. vk and its derivative for one cell.  The mass
 * difference phi rho - phi^n rho^n is a difference of nearly equal numbers
 * (relative size c_f |p - p^n|, about 1e-5 here), so FP64 would lose about
 * eleven of its sixteen digits to cancellation; it is evaluated in long
 * double (80-bit or 128-bit) and rounded to double once. */
static void orc_accumulation_v(const orc_params* q, long double V, double phi0, double p, double pn,
                               double* A, double* dA) {
    long double rho = q->rho_ref * expl((long double)q->c_f * ((long double)p - q->p_ref));
    long double rhon = q->rho_ref * expl((long double)q->c_f * ((long double)pn - q->p_ref));
    long double phi = phi0 * (1.0L + (long double)q->c_r * ((long double)p - q->p_ref));
    long double phin = phi0 * (1.0L + (long double)q->c_r * ((long double)pn - q->p_ref));
    *A = (double)(V * (phi * rho - phin * rhon) / q->dt);
    *dA = (double)(V * (phi0 * q->c_r * rho + phi * q->c_f * rho) / q->dt);
}

/* The same for a cell of the structured grid, V = dx dy dz. */
static void orc_accumulation(const orc_params* q, double phi0, double p, double pn,
                             double* A, double* dA) {
    orc_accumulation_v(q, (long double)q->dx * q->dy * q->dz, phi0, p, pn, A, dA);
}

/*
 * Residual and Jacobian.
 *   perm, poro, depth, p, pn : N cell values (m^2, -, m, Pa, Pa)
 *   row_ptr, col_idx         : the pattern from orc_pattern
 *   flip                     : optional, nnz bytes; nonzero at a CSR position
 *                              (K, L) reverses the upwind choice of that link
 *   R                        : N outputs (may be NULL)
 *   J                        : nnz outputs in CSR order (may be NULL)
 *   F_out, dphi_out          : optional, nnz: the flux and potential
 *                              difference of link (K, L) at its CSR position
 *                              (0 on the diagonal)
 *   acc_out                  : optional, N: the accumulation term alone
 * Returns 0, or -1 on bad arguments.
 */
int orc_assemble(int nx, int ny, int nz, const orc_params* q,
                 const double* perm, const double* poro, const double* depth,
                 const double* p, const double* pn,
                 const long long* row_ptr, const long long* col_idx,
                 const unsigned char* flip,
                 double* R, double* J, double* F_out, double* dphi_out, double* acc_out) {
    if (!orc_valid_params(nx, ny, nz, q)) return -1;
    long long N = (long long)nx * ny * nz;
    long long nnz = row_ptr[N];
    if (J) memset(J, 0, sizeof(double) * (size_t)nnz);
    if (F_out) memset(F_out, 0, sizeof(double) * (size_t)nnz);
    if (dphi_out) memset(dphi_out, 0, sizeof(double) * (size_t)nnz);
    /* Rows are independent (each writes only its own row), so the cell loop
     * may run on several host threads without changing any result. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long long K = 0; K < N; ++K) {
        long long L[10];
        int slot[10];
        double rK = 0.0; /* (r_flux)_K := 0 */
        long long dpos = orc_find(row_ptr, col_idx, K, K);
        int n = orc_adj(nx, ny, nz, q->connectivity, K, L, slot);
        for (int a = 0; a < n; ++a) {
            int s = slot[a];
            double T = orc_trans(q, perm[K], perm[L[a]], ORC_NB[s][0], ORC_NB[s][1], ORC_NB[s][2]);
            long long pos = orc_find(row_ptr, col_idx, K, L[a]);
            int fl = flip ? flip[pos] != 0 : 0;
            orc_conn c = orc_connection(q, T, p[K], p[L[a]], depth[K], depth[L[a]], fl);
            rK += c.F;
            if (J) {
                J[dpos] += c.dF_dpK;
                J[pos] = c.dF_dpL;
            }
            if (F_out) F_out[pos] = c.F;
            if (dphi_out) dphi_out[pos] = c.dphi;
        }
        double A, dA;
        orc_accumulation(q, poro[K], p[K], pn[K], &A, &dA);
        if (R) R[K] = A + rK;
        if (J) J[dpos] += dA;
        if (acc_out) acc_out[K] = A;
    }
    return 0;
}

/*
 * Vector-Jacobian product of R: g_p = J^T v and g_lnk[i] = sum_K v_K dR_K/d(ln k_i),
 * written as a scatter over every (K, L) link in Algorithm 1's loop order.
 * Upsilon depends on k_K and k_L through the harmonic mean:
 * d Upsilon / d ln k_K = Upsilon * k_L / (k_K + k_L).
 */
int orc_vjp(int nx, int ny, int nz, const orc_params* q,
            const double* perm, const double* poro, const double* depth,
            const double* p, const double* pn, const double* v,
            double* g_p, double* g_lnk) {
    if (!orc_valid_params(nx, ny, nz, q)) return -1;
    long long N = (long long)nx * ny * nz;
    memset(g_p, 0, sizeof(double) * (size_t)N);
    memset(g_lnk, 0, sizeof(double) * (size_t)N);
    long long L[10];
    int slot[10];
    for (long long K = 0; K < N; ++K) {
        int n = orc_adj(nx, ny, nz, q->connectivity, K, L, slot);
        for (int a = 0; a < n; ++a) {
            int s = slot[a];
            long long l = L[a];
            double kK = perm[K], kL = perm[l];
            double T = orc_trans(q, kK, kL, ORC_NB[s][0], ORC_NB[s][1], ORC_NB[s][2]);
            orc_conn c = orc_connection(q, T, p[K], p[l], depth[K], depth[l], 0);
            g_p[K] += v[K] * c.dF_dpK;
            g_p[l] += v[K] * c.dF_dpL;
            if (kK > 0.0 && kL > 0.0) {
                g_lnk[K] += v[K] * c.dF_dT * T * kL / (kK + kL);
                g_lnk[l] += v[K] * c.dF_dT * T * kK / (kK + kL);
            }
        }
        double A, dA;
        orc_accumulation(q, poro[K], p[K], pn[K], &A, &dA);
        g_p[K] += v[K] * dA;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * General meshes: a list of connections (K, L, Upsilon_KL) -- the form the
 * paper names as its extension to arbitrary mesh topologies (Section 8).
 * Each connection joins two distinct cells; adj(K) is every cell sharing a
 * connection with K.  Upsilon is an input (a mesh generator computes it from
 * the cell geometry), the cell volume V_K varies per cell, and the flux,
 * upwinding, density and accumulation are those above.
 * ------------------------------------------------------------------------ */

/*
 * Pattern of a connection list: row K holds K and every cell connected to
 * it, columns ascending (insertion sort).  conn_of[e] is the connection of
 * entry e (-1 on the diagonal).  With col_idx == NULL only row_ptr is filled.
 * Returns nnz, or -1 for an index out of range, a connection of a cell with
 * itself, or the same pair listed twice.
 */
long long orc_mesh_pattern(long long n, long long nc, const long long* ci, const long long* cj,
                           long long* row_ptr, long long* col_idx, long long* conn_of) {
    if (n <= 0 || nc < 0) return -1;
    for (long long c = 0; c < nc; ++c)
        if (ci[c] < 0 || ci[c] >= n || cj[c] < 0 || cj[c] >= n || ci[c] == cj[c]) return -1;
    for (long long K = 0; K <= n; ++K) row_ptr[K] = 0;
    for (long long c = 0; c < nc; ++c) {
        row_ptr[ci[c] + 1] += 1;
        row_ptr[cj[c] + 1] += 1;
    }
    for (long long K = 0; K < n; ++K) row_ptr[K + 1] += row_ptr[K] + 1; /* + 1: the diagonal */
    long long nnz = row_ptr[n];
    if (!col_idx) return nnz;
    long long* fill = (long long*)malloc(sizeof(long long) * (size_t)n);
    if (!fill) return -1;
    for (long long K = 0; K < n; ++K) {
        fill[K] = row_ptr[K] + 1;
        col_idx[row_ptr[K]] = K;
        conn_of[row_ptr[K]] = -1;
    }
    for (long long c = 0; c < nc; ++c) {
        long long e = fill[ci[c]]++;
        col_idx[e] = cj[c];
        conn_of[e] = c;
        e = fill[cj[c]]++;
        col_idx[e] = ci[c];
        conn_of[e] = c;
    }
    free(fill);
    int dup = 0;
    for (long long K = 0; K < n; ++K) { /* insertion sort of each row by column */
        for (long long e = row_ptr[K] + 1; e < row_ptr[K + 1]; ++e) {
            long long cv = col_idx[e], cc = conn_of[e], f = e - 1;
            while (f >= row_ptr[K] && col_idx[f] > cv) {
                col_idx[f + 1] = col_idx[f];
                conn_of[f + 1] = conn_of[f];
                --f;
            }
            col_idx[f + 1] = cv;
            conn_of[f + 1] = cc;
        }
        for (long long e = row_ptr[K] + 1; e < row_ptr[K + 1]; ++e)
            if (col_idx[e] == col_idx[e - 1]) dup = 1;
    }
    return dup ? -1 : nnz;
}

/*
 * Residual and Jacobian of Eq. vk on a connection list, Algorithm 1's loops:
 * for each cell K, for each L in adj(K) (row K of the pattern), the flux of
 * connection (K, L) seen from K; then the accumulation term with V_K.
 *   T, V        : nc transmissibilities, n cell volumes
 *   poro, depth, p, pn, row_ptr, col_idx, conn_of : as orc_assemble / orc_mesh_pattern
 *   flip, R, J, F_out, dphi_out, acc_out          : as orc_assemble
 */
int orc_mesh_assemble(long long n, const orc_params* q, const double* T, const double* V,
                      const double* poro, const double* depth, const double* p, const double* pn,
                      const long long* row_ptr, const long long* col_idx, const long long* conn_of,
                      const unsigned char* flip, double* R, double* J, double* F_out, double* dphi_out,
                      double* acc_out) {
    if (n <= 0 || q == NULL || !(q->dt > 0.0) || !(q->mu > 0.0)) return -1;
    long long nnz = row_ptr[n];
    if (J) memset(J, 0, sizeof(double) * (size_t)nnz);
    if (F_out) memset(F_out, 0, sizeof(double) * (size_t)nnz);
    if (dphi_out) memset(dphi_out, 0, sizeof(double) * (size_t)nnz);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long long K = 0; K < n; ++K) {
        double rK = 0.0;
        long long dpos = orc_find(row_ptr, col_idx, K, K);
        for (long long e = row_ptr[K]; e < row_ptr[K + 1]; ++e) {
            long long L = col_idx[e];
            if (L == K) continue;
            int fl = flip ? flip[e] != 0 : 0;
            orc_conn c = orc_connection(q, T[conn_of[e]], p[K], p[L], depth[K], depth[L], fl);
            rK += c.F;
            if (J) {
                J[dpos] += c.dF_dpK;
                J[e] = c.dF_dpL;
            }
            if (F_out) F_out[e] = c.F;
            if (dphi_out) dphi_out[e] = c.dphi;
        }
        double A, dA;
        orc_accumulation_v(q, (long double)V[K], poro[K], p[K], pn[K], &A, &dA);
        if (R) R[K] = A + rK;
        if (J) J[dpos] += dA;
        if (acc_out) acc_out[K] = A;
    }
    return 0;
}

/* Transmissibility of one link, exported for the tests' closed-form checks. */
double orc_link_trans(const orc_params* q, double kK, double kL, int di, int dj, int dk) {
    return orc_trans(q, kK, kL, di, dj, dk);
}

/* Number of threads the row loop of orc_assemble may use (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of threads the row loops use from now on (n >= 1; ignored
 * without OpenMP).  For timing the oracle single-threaded and on all cores. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
