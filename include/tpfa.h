/*
 * tpfa.h -- C ABI of the GB300 (sm_103a) TPFA assembly library.
 *
 * The library assembles, on one GPU, the residual and the Jacobian of the
 * backward-Euler finite-volume discretisation of single-phase compressible
 * Darcy flow on a structured nx x ny x nz grid (arXiv 2304.11274, Section 3):
 *
 *   R_K = V (phi(p_K) rho(p_K) - phi(pn_K) rho(pn_K)) / dt + sum_{L in adj(K)} F_KL   (Eq. vk)
 *   F_KL = Upsilon_KL * lambda_up * dPhi_KL                                           (Eq. flux-calc)
 *   dPhi_KL = (p_K - p_L) - rho_avg g (z_K - z_L),  rho_avg = (rho_K + rho_L) / 2
 *   lambda_up = rho_K / mu if dPhi_KL > 0, else rho_L / mu                           (upwinding)
 *   rho(p) = rho_ref exp(c_f (p - p_ref))                                            (Eq. density)
 *   phi(p) = phi0 (1 + c_r (p - p_ref))
 *   J_KL = dR_K / dp_L
 *
 * Conventions shared by every entry point:
 *   - Cell (i, j, k) has linear index lin = i + nx (j + ny k): x fastest,
 *     z slowest, the layout of Section 6.  z is the cell-centre DEPTH
 *     (positive down), so F_KL is the mass outflow from K to L.  This is the
 *     paper's Eq. flux-calc with K and L exchanged and z measured downward:
 *     the form in which its upwind rule and the sign of Eq. vk agree.
 *   - adj(K) is Section 5.1's neighbour set: (a) the four in-plane cardinal
 *     cells, (b) the four in-plane diagonal cells when connectivity == 10,
 *     (c) the cells above and below; cells outside the grid are not
 *     neighbours (closed, no-flow boundary).
 *   - Upsilon (the paper names it without a formula) is the two-point
 *     harmonic form 2 k_K k_L / (k_K + k_L) * area / distance, with the
 *     in-plane diagonal's distance sqrt(dx^2 + dy^2) and area
 *     dz dx dy / sqrt(dx^2 + dy^2).
 *   - Every pointer named *_dev is DEVICE memory on the current CUDA device,
 *     owned by the caller unless stated otherwise.  `stream` is a
 *     cudaStream_t passed as void* (NULL = the legacy default stream); every
 *     call is asynchronous on it unless stated otherwise.
 *   - Every call returns TPFA_OK (0) or a negative TPFA_ERR_* code and, on
 *     error, sets a thread-local message read by tpfa_last_error_string().
 *     Errors raised on the device (non-finite results) are latched in the
 *     handle and returned by tpfa_sync_status().
 *   - There is no host fallback: without a usable GPU every call that
 *     computes returns TPFA_ERR_CUDA.
 */
#ifndef TPFA_H
#define TPFA_H

#ifdef __cplusplus
extern "C" {
#endif

#define TPFA_OK 0
#define TPFA_ERR_INVALID_ARG (-1) /* null handle/pointer, bad size, bad enum */
#define TPFA_ERR_OOM (-2)         /* device allocation failed; nothing leaked */
#define TPFA_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define TPFA_ERR_TOO_LARGE (-4)   /* N >= 2^31 cells, or a size beyond a stated limit */
#define TPFA_ERR_NONFINITE (-5)   /* a residual or Jacobian value came out NaN/Inf */
#define TPFA_ERR_NO_STATE (-6)    /* assemble called before tpfa_set_state */
#define TPFA_ERR_TIMEOUT (-7)     /* a bounded device-side wait ran out */
#define TPFA_ERR_DEVICE_CHECK (-8) /* a device-side bounds check failed (nothing was accessed) */
#define TPFA_ERR_NO_CONVERGENCE (-9) /* the Krylov solve stopped before its tolerance (breakdown or iteration limit) */

typedef struct tpfa_grid* tpfa_handle; /* opaque, library-owned */

typedef enum {
    TPFA_FP64 = 0,  /* every field, every operation and every output in FP64 */
    TPFA_MIXED = 1  /* FP32 fields and flux arithmetic, FP32 Kahan residual sum,
                       FP64 accumulation term and FP64 outputs R and diag64 */
} tpfa_precision;

/* Kernel variant used by the assemble calls.  All variants evaluate every
 * link and sum every row in the same order with the same roundings, so they
 * give bit-identical results. */
typedef enum {
    TPFA_KERNEL_AUTO = 0,  /* the library's choice: TILED2 for the fused residual
                              + Jacobian of TPFA_MIXED grids it accepts that
                              are at least 256 cells wide in x, or exactly
                              128 or 192 wide, else TILED */
    TPFA_KERNEL_NAIVE = 1, /* one thread per cell, every neighbour read from
                              global memory: the correctness baseline */
    TPFA_KERNEL_TILED = 2, /* a warp per 32-cell x-segment of a z-plane,
                              marching along y with rows j-1, j, j+1 held in
                              registers and x-neighbours exchanged by warp
                              shuffles; each lane prefetches its row inputs
                              with cp.async */
    TPFA_KERNEL_TILED_TMA = 3, /* TILED with 4 warps per block on 4
                              consecutive x-segments of one plane, each row's
                              inputs fetched for the whole block as a few
                              boxes by the tensor memory accelerator
                              (cp.async.bulk.tensor) into a shared ring;
                              assembly calls only, TPFA_MIXED, nx a multiple
                              of 4 and p, p^n 16-byte aligned, else
                              TPFA_ERR_INVALID_ARG */
    TPFA_KERNEL_TILED2 = 4 /* TILED with two adjacent cells per lane (64-cell
                              x-segments): each link is one half of a paired
                              FP32 instruction and every input moves as one
                              8-byte copy per lane for two cells; fused
                              residual + Jacobian of TPFA_MIXED with nx even
                              and 8-byte aligned fields (16-byte m^n), else
                              the call runs TILED */
} tpfa_kernel;

typedef struct {
    double rho_ref;   /* reference density rho_ref, kg/m^3 (Eq. density) */
    double p_ref;     /* reference pressure p_ref, Pa (Eq. density) */
    double c_f;       /* fluid compressibility c_f, 1/Pa (Eq. density) */
    double mu;        /* viscosity mu, Pa s (> 0) */
    double g;         /* gravitational acceleration g, m/s^2 */
    double dt;        /* time step dt, s (> 0) (Eq. vk) */
    double c_r;       /* rock compressibility c_r, 1/Pa; 0 = constant porosity */
    double dx, dy, dz;/* cell size, m (> 0); V = dx dy dz */
    int connectivity; /* 6 (faces) or 10 (faces + in-plane diagonals) */
} tpfa_params;

/*
 * Create a grid (Section 3 problem statement; Section 6 layout).
 *   out        : receives the handle.
 *   nx, ny, nz : grid size, each >= 1, N = nx ny nz < 2^31, and one z-plane's
 *                Jacobian entries addressable in 32 bits, 11 nx ny < 2^31
 *                (about 195 M cells per plane); else TPFA_ERR_TOO_LARGE.
 *   prm        : physical constants and connectivity (copied).
 *   prec       : TPFA_FP64 or TPFA_MIXED.
 *   perm_dev   : N doubles, permeability k (m^2, >= 0), read during the call only.
 *   poro_dev   : N doubles, reference porosity phi0, read during the call only.
 *   depth_dev  : N doubles, cell-centre depth z (m), read during the call only;
 *                the mixed path stores it rounded to FP32.
 * The library computes the owned transmissibilities (links to +x, +y, +z and,
 * with 10-point connectivity, to (+x,+y) and (-x,+y)) in FP64 and stores them
 * in the path's precision.  Synchronises `stream` before returning.
 */
int tpfa_create_grid(tpfa_handle* out, int nx, int ny, int nz, const tpfa_params* prm,
                     tpfa_precision prec, const double* perm_dev, const double* poro_dev,
                     const double* depth_dev, void* stream);

/*
 * Bind the Newton state (Eq. vk): p^{n+1} (the iterate) and p^n (the previous
 * time step).  p_dev and p_prev_dev hold N values of the handle's field type
 * (double for TPFA_FP64, float for TPFA_MIXED); the pointers are BORROWED and
 * must stay valid until the next set_state or destroy.  Computes
 * m^n = (V/dt) phi(p^n) rho(p^n) in FP64 into library-owned memory, so call it
 * again whenever p^n changes; when only p changes, tpfa_set_pressure is enough.
 */
int tpfa_set_state(tpfa_handle h, const void* p_dev, const void* p_prev_dev, void* stream);

/* Rebind only the iterate p (same type and lifetime rules as set_state). */
int tpfa_set_pressure(tpfa_handle h, const void* p_dev);

/*
 * Residual only (Algorithm 1 plus the accumulation term of Eq. vk).
 *   R_dev : N doubles, written.
 */
int tpfa_assemble_residual(tpfa_handle h, double* R_dev, void* stream);

/*
 * Residual and Jacobian in one fused pass.
 *   R_dev      : N doubles or NULL (then R is not written).
 *   vals_dev   : nnz values in the CSR order of tpfa_get_pattern (columns
 *                ascending within a row); double for TPFA_FP64, float for
 *                TPFA_MIXED (its diagonal slot holds (float) J_KK).
 *   diag64_dev : TPFA_MIXED: N doubles, the FP64 diagonal J_KK (may be NULL);
 *                TPFA_FP64: must be NULL.
 */
int tpfa_assemble_jacobian(tpfa_handle h, double* R_dev, void* vals_dev, double* diag64_dev,
                           void* stream);

/* As tpfa_assemble_jacobian with an explicit kernel variant. */
int tpfa_assemble_jacobian_kernel(tpfa_handle h, tpfa_kernel kern, double* R_dev, void* vals_dev,
                                  double* diag64_dev, void* stream);

/*
 * The variant a residual + Jacobian call with `kern` runs on this handle in
 * its current state (AUTO resolved; TILED2 on a grid or fields it does not
 * accept, and NAIVE on a slab handle, resolved to TILED), written to
 * *resolved as a tpfa_kernel value.  Launches nothing.  TPFA_ERR_NO_STATE
 * before tpfa_set_state (the bound pressure's alignment takes part);
 * TPFA_ERR_INVALID_ARG for TILED_TMA where the assembly call would refuse it.
 */
int tpfa_resolve_kernel(tpfa_handle h, tpfa_kernel kern, int* resolved);

/*
 * End-to-end form with HOST buffers (pinned memory recommended): copies the
 * N pressure values in p_host to a library-owned device buffer, binds it as
 * the iterate, assembles, and copies R (N doubles), the CSR values (nnz) and,
 * for TPFA_MIXED, diag64 (N doubles) back.  Any output pointer may be NULL.
 * Requires a prior tpfa_set_state for p^n.  Synchronises `stream`.
 */
int tpfa_assemble_jacobian_host(tpfa_handle h, const void* p_host, double* R_host,
                                void* vals_host, double* diag64_host, void* stream);

/*
 * Replace the permeability (for example while optimising log-permeability):
 * recomputes the owned transmissibilities and the stored k of the adjoint.
 * perm_dev: N doubles (m^2, >= 0), read asynchronously on `stream`.
 */
int tpfa_set_permeability(tpfa_handle h, const double* perm_dev, void* stream);

/*
 * As tpfa_set_permeability with the natural log of the permeability given:
 * log_perm_dev holds N doubles ln k (read asynchronously on `stream`); the
 * library forms k = exp(ln k) on the device.  This is the parameterisation
 * of the adjoint's g_lnk (tpfa_vjp), so an optimiser over ln k can bind its
 * iterate without any arithmetic of its own.
 */
int tpfa_set_log_permeability(tpfa_handle h, const double* log_perm_dev, void* stream);

/*
 * Adjoint of the residual (vector-Jacobian products) at the bound state:
 *   g_p[i]   = sum_K v_K dR_K/dp_i              (= J^T v)
 *   g_lnk[i] = sum_K v_K dR_K/d(ln k_i)         (natural log)
 * R as in Eq. vk with the flux of Eq. flux-calc; k enters only through the
 * harmonic transmissibilities, d Upsilon_KL/d ln k_K = Upsilon_KL k_L/(k_K + k_L).
 * Densities, upwind choices and mobilities are recomputed, nothing is stored
 * by the forward pass.  v_dev, g_p_dev: N doubles; g_lnk_dev: N doubles or
 * NULL.  TPFA_FP64: links, sums and outputs in FP64.  TPFA_MIXED: FP32 links;
 * each v is split once per call into an FP32 pair hi + lo (a library-owned
 * buffer of N pairs, allocated on the first call), each link's term is an
 * FP32 product with v_K - v_L formed in FP32 from the pairs (accurate
 * relative to the difference itself), the terms are compensated FP32 sums
 * combined in FP64, the outputs FP64.
 */
int tpfa_vjp(tpfa_handle h, const double* v_dev, double* g_p_dev, double* g_lnk_dev, void* stream);

/* As tpfa_vjp with an explicit kernel variant (TPFA_MIXED: the one-cell
 * march TILED, the two-cell march TILED2 (nx even; else TILED runs) and the
 * naive gather give identical bits; AUTO is TILED; TILED_TMA is refused;
 * TPFA_FP64 has one kernel and ignores the choice). */
int tpfa_vjp_kernel(tpfa_handle h, tpfa_kernel kern, const double* v_dev, double* g_p_dev, double* g_lnk_dev,
                    void* stream);

/*
 * Matrix-free Jacobian-vector product at the bound state (the operator a
 * Krylov solver of the backward-Euler system Eq. vk needs, without storing J):
 *   Jw[K] = sum_L dR_K/dp_L w_L
 *         = (dA_K/dp_K + sum_{L in adj(K)} dF_KL/dp_K) w_K + sum_L dF_KL/dp_L w_L
 * with the flux of Eq. flux-calc and the same upwind rule (tie -> L) as the
 * assembled Jacobian, so Jw equals the product of tpfa_assemble_jacobian's
 * matrix with w up to FP64 rounding.  w_dev, Jw_dev: N doubles (device,
 * caller-owned, w read and Jw written asynchronously on `stream`).
 * R_dev: N doubles or NULL; when given it receives R of Eq. vk with exactly
 * the bits tpfa_assemble_residual writes.  Links in the path's precision,
 * the w-weighted sums in FP64.  Device-side errors (non-finite output, an
 * out-of-range checked access) are reported by tpfa_sync_status.
 */
int tpfa_jvp(tpfa_handle h, const double* w_dev, double* Jw_dev, double* R_dev, void* stream);

/* As tpfa_jvp with an explicit kernel variant (TPFA_MIXED: the tiled march
 * and the naive gather give identical bits; TPFA_FP64 has one kernel and
 * ignores the choice). */
int tpfa_jvp_kernel(tpfa_handle h, tpfa_kernel kern, const double* w_dev, double* Jw_dev, double* R_dev,
                    void* stream);

/*
 * The static Jacobian pattern: row_ptr (N+1 int64) and col_idx (nnz int32),
 * columns ascending in each row.  Built on the first call (library-owned,
 * read-only, freed by destroy); synchronises `stream` on that first call.
 * Any out-pointer may be NULL.
 */
int tpfa_get_pattern(tpfa_handle h, const long long** row_ptr_dev, const int** col_idx_dev,
                     long long* nnz, void* stream);

/* Copy the pattern into caller-owned device buffers: row_ptr_out_dev (N+1
 * int64) and col_idx_out_dev (nnz int32); either may be NULL.  Builds the
 * library's copy first if needed (see tpfa_get_pattern).  Asynchronous on
 * `stream` after that first build. */
int tpfa_copy_pattern(tpfa_handle h, long long* row_ptr_out_dev, int* col_idx_out_dev, void* stream);

/* Number of Jacobian entries of an nx x ny x nz grid with the given
 * connectivity: N + 2 * (number of links), from the closed form of Section
 * 5.1's neighbour sets.  Host-only, needs no GPU.  Returns a negative
 * TPFA_ERR_* code for bad arguments. */
long long tpfa_nnz(int nx, int ny, int nz, int connectivity);

/* Grid facts: sizes, nnz (closed form, no pattern build), precision. */
int tpfa_grid_info(tpfa_handle h, int* nx, int* ny, int* nz, int* connectivity, long long* nnz,
                   int* precision);

/* Read the transmissibilities the library stores (for tests): `which` is
 * 0 (+x), 1 (+y), 2 (+z), 3 (+x,+y), 4 (-x,+y); out_dev holds N values of the
 * field type; links that leave the grid hold 0. */
int tpfa_get_transmissibility(tpfa_handle h, int which, void* out_dev, void* stream);

/*
 * Wait for `stream`, then report and clear device-side errors latched since
 * the last call: TPFA_ERR_TIMEOUT if a bounded device-side wait ran out (the
 * TMA march's row waits; that launch's outputs are incomplete), else
 * TPFA_ERR_DEVICE_CHECK if a checked device access was out of range (and
 * skipped), else TPFA_ERR_NONFINITE if any assembled value was NaN/Inf.
 */
int tpfa_sync_status(tpfa_handle h, void* stream);

/* ---------------------------------------------------------------- z-slabs of one grid */

/*
 * Decomposition of one grid over several GPUs into z-slabs.  Section 5 maps
 * the x-y plane of cells onto a grid of processing elements, keeps each
 * column's z-range in the element's memory and exchanges the neighbouring
 * values across element boundaries (Section 5.2); here each GPU holds a
 * contiguous range of z-planes and exchanges one plane of pressure with each
 * neighbouring slab before an assembly.  In-plane (cardinal and diagonal)
 * links never cross a slab boundary, so no corner cells are exchanged.
 *
 * tpfa_slab_bounds (host-only, needs no GPU): the planes [k0, k1) of slab
 * `part` of `parts` over nz planes (balanced: the first nz % parts slabs
 * hold one plane more; 1 <= parts <= nz) and the planes [e0, e1) its handle
 * holds: the slab and one halo plane on each side that exists.
 */
int tpfa_slab_bounds(int nz, int parts, int part, int* k0, int* k1, int* e0, int* e1);

/*
 * A slab handle: planes [k0, k1) of an nx x ny x nz grid.  perm_dev,
 * poro_dev and depth_dev hold the planes [e0, e1) of tpfa_slab_bounds (N =
 * nx ny (e1 - e0) doubles each; read during the call), so the handle's
 * owned transmissibilities include the vertical links into its halos.  The
 * handle behaves as a grid of e1 - e0 planes (tpfa_set_state /
 * tpfa_set_pressure bind N values, halo planes included, and every output
 * has the sizes of that grid: N residuals, its nnz values, N diagonals),
 * but tpfa_assemble_jacobian and tpfa_assemble_residual write only the rows
 * of the owned planes (tpfa_slab_info gives their ranges); those rows equal
 * the larger grid's rows bit for bit once the halo planes of the bound
 * pressure hold the neighbouring slabs' values (tpfa_slab_exchange, or any
 * copy such as an NCCL send/receive).  The kernel variant is the library's
 * choice (a naive request runs the tiled march).  tpfa_vjp, tpfa_jvp, the
 * Krylov / Newton calls, the host-buffer call and ensembles return
 * TPFA_ERR_INVALID_ARG on slabs.
 */
int tpfa_create_slab(tpfa_handle* out, int nx, int ny, int nz, int k0, int k1, const tpfa_params* prm,
                     tpfa_precision prec, const double* perm_dev, const double* poro_dev, const double* depth_dev,
                     void* stream);

/* A slab's owned planes: [k0, k1) of the larger grid and [own0, own1) of the
 * handle; its owned rows are cells [row0, row1) and CSR entries
 * [entry0, entry1) of the handle's outputs.  Any out-pointer may be NULL. */
int tpfa_slab_info(tpfa_handle h, int* k0, int* k1, int* own0, int* own1, long long* row0, long long* row1,
                   long long* entry0, long long* entry1);

/*
 * Halo exchange between adjacent slabs (upper's k0 == lower's k1) of one
 * grid, possibly on different devices: copies lower's last owned plane of
 * pressure into upper's bottom halo plane and upper's first owned plane into
 * lower's top halo plane (cudaMemcpyPeerAsync, asynchronous on `stream`).
 * p_lower_dev / p_upper_dev: the pressures bound (or to be bound) to each
 * slab, N values of the field type each.
 */
int tpfa_slab_exchange(tpfa_handle lower, void* p_lower_dev, tpfa_handle upper, void* p_upper_dev, void* stream);

/* ---------------------------------------------------------------- tiling */

/*
 * Tiling of the assembly kernel: a warp marches along y over
 * `rows_per_march` (1 to 64) rows of a 32-cell x-segment, and a block stacks
 * `warps_per_block` (4 or 8) consecutive z-planes.  Results do not depend on
 * the tiling (every row is summed in the same order); only speed does.  The
 * J w and adjoint marches use the same tiling, with the rows per march
 * halved (down to 8) while the launch has fewer than four blocks per
 * multiprocessor.
 */
int tpfa_set_tiling(tpfa_handle h, int rows_per_march, int warps_per_block);
int tpfa_get_tiling(tpfa_handle h, int* rows_per_march, int* warps_per_block);

/*
 * Choose the tiling by timing candidates (rows_per_march 8, 16, 24, 32, 40,
 * 48, 64 x warps_per_block 4, 8) on this grid at its bound state, or take it from
 * `cache_path` (a text file of "key rows warps" lines, key = device, path,
 * connectivity, porosity law and log2 of the cell count); a new choice is
 * written back.  cache_path may be NULL (no cache).  Allocates and frees
 * temporary outputs on `stream` and synchronises it.
 */
int tpfa_autotune(tpfa_handle h, const char* cache_path, void* stream);

/* ---------------------------------------------------------------- Newton step */

/*
 * One Newton iteration on the backward-Euler system Eq. vk (R(p^{n+1}) = 0):
 *   assemble R(p^k) and J = dR/dp at p^k (the fused kernel of
 *   tpfa_assemble_jacobian), solve J delta = -R with BiCGStab right-
 *   preconditioned by the tridiagonal part of J along z (each (i, j) column's
 *   vertical couplings, solved exactly; the vertical links of thin cells
 *   dominate) or by its diagonal, p^{k+1} = p^k + delta.
 * The paper names the implicit system and a Krylov solve of it as the use of
 * the flux operator but fixes neither the nonlinear nor the linear method;
 * these are the standard choices.  Vectors, dot products and the update are
 * FP64; the matrix is the path's assembled Jacobian (FP32 off-diagonals with
 * FP64 diagonal on TPFA_MIXED).  The matrix-vector product walks the
 * structured stencil (columns follow from the closed-form pattern), and the
 * solver's scalars live on the device: the host reads them every
 * `check_every` iterations.
 */
#define TPFA_PRECOND_ZLINE 0  /* tridiagonal part of J along z, solved exactly per (i, j) column */
#define TPFA_PRECOND_JACOBI 1 /* diagonal of J */

typedef struct {
    int max_iters;      /* BiCGStab iteration limit (<= 0: 1000) */
    double rtol;        /* stop when ||b - J x||_2 <= rtol ||b||_2 (<= 0: 1e-8) */
    int check_every;    /* iterations between host convergence checks (<= 0: 8) */
    int preconditioner; /* TPFA_PRECOND_ZLINE (default, 0) or TPFA_PRECOND_JACOBI */
} tpfa_krylov_opts;

typedef struct {
    int iterations;       /* BiCGStab iterations taken */
    int converged;        /* 1 if the tolerance was met */
    int breakdown;        /* 1 if a BiCGStab denominator vanished */
    double b_norm;        /* ||b||_2 (for a Newton step: ||R(p^k)||_2) */
    double rel_residual;  /* ||b - J x||_2 / ||b||_2 of the recursively updated residual */
} tpfa_krylov_stats;

/*
 * Solve J x = b, J the Jacobian at the bound state (assembled into
 * library-owned workspace by this call), x0 = 0.  b_dev, x_dev: N doubles
 * (device, caller-owned).  opts may be NULL (defaults); stats may be NULL.
 * Synchronous on `stream`: the iterations run after the work already queued
 * on `stream`, and the call returns once they are done.  They run on a
 * library-owned stream of the handle (it waits for `stream` before the solve
 * and `stream` waits for it after), each batch of check_every iterations as
 * one launch of a CUDA graph captured on the first solve into x_dev (and
 * again when x_dev or check_every change); a `stream` that is itself being
 * captured gets plain launches.  Returns TPFA_ERR_NO_CONVERGENCE when the
 * tolerance was not met (x_dev then holds the last iterate).  The first
 * call allocates the workspace: nnz values, 12 FP64 vectors of N (and, on
 * TPFA_MIXED, four FP32 vectors), and creates the stream and two events.
 */
int tpfa_linear_solve(tpfa_handle h, const double* b_dev, double* x_dev, const tpfa_krylov_opts* opts,
                      tpfa_krylov_stats* stats, void* stream);

/*
 * One Newton step in place: binds p_dev as the pressure (as
 * tpfa_set_pressure; N values of the field type), solves J delta = -R(p) as
 * tpfa_linear_solve does and writes p + delta back to p_dev (rounded to the
 * field type).  R_dev: N doubles or NULL, receives R(p) before the update.
 * delta_dev: N doubles or NULL, receives delta.  On
 * TPFA_ERR_NO_CONVERGENCE p_dev is left unchanged.  Synchronous on `stream`.
 */
int tpfa_newton_step(tpfa_handle h, void* p_dev, const tpfa_krylov_opts* opts, tpfa_krylov_stats* stats,
                     double* R_dev, double* delta_dev, void* stream);

/* ---------------------------------------------------------------- general meshes */

typedef struct tpfa_mesh_s* tpfa_mesh; /* opaque, library-owned */

/*
 * A general mesh given as a list of connections, the extension to arbitrary
 * mesh topologies (corner-point grids with faults and non-neighbour
 * connections, unstructured meshes) that Section 8 names as future work.
 * adj(K) is every cell sharing a connection with K; the flux of connection
 * (K, L) is Eq. flux-calc with Upsilon_KL given, the accumulation is Eq. vk's
 * with the cell's own volume V_K, and upwinding, density and porosity are as
 * on the structured grid (same arithmetic, same precision paths).
 *   n_cells, n_conn     : cells (< 2^31) and connections (>= 0)
 *   prm                 : rho_ref, p_ref, c_f, mu, g, dt, c_r are used;
 *                         dx, dy, dz and connectivity are ignored
 *   conn_i_dev, conn_j_dev : n_conn int32 cell indices each; i != j, both in
 *                         [0, n_cells), no pair listed twice (in either order)
 *   trans_dev           : n_conn Upsilon_KL (m^3, >= 0), FP64
 *   volume_dev, poro_dev, depth_dev : n_cells FP64 (m^3, -, m positive down)
 * All inputs are read during the call (copied, device, caller-owned).  The
 * pattern (row K: K and its neighbours, columns ascending, int64 row_ptr and
 * int32 col_idx) is built on the host and uploaded; the call synchronises
 * `stream`.  Bad lists return TPFA_ERR_INVALID_ARG with the first offending
 * connection in the message.
 */
int tpfa_create_mesh(tpfa_mesh* out, long long n_cells, long long n_conn, const tpfa_params* prm,
                     tpfa_precision prec, const int* conn_i_dev, const int* conn_j_dev, const double* trans_dev,
                     const double* volume_dev, const double* poro_dev, const double* depth_dev, void* stream);

/* As tpfa_set_state / tpfa_set_pressure: n_cells values of the field type;
 * m^n = (V_K/dt) phi(p^n) rho(p^n) is computed here. */
int tpfa_mesh_set_state(tpfa_mesh m, const void* p_dev, const void* p_prev_dev, void* stream);
int tpfa_mesh_set_pressure(tpfa_mesh m, const void* p_dev);

/* Residual and Jacobian (as tpfa_assemble_jacobian, in the CSR order of the
 * mesh's pattern); vals_dev NULL assembles the residual only. */
int tpfa_mesh_assemble(tpfa_mesh m, double* R_dev, void* vals_dev, double* diag64_dev, void* stream);

/* Copy the pattern into caller-owned device buffers (either may be NULL):
 * row_ptr (n_cells + 1 int64), col_idx (nnz int32). */
int tpfa_mesh_copy_pattern(tpfa_mesh m, long long* row_ptr_out_dev, int* col_idx_out_dev, void* stream);

/* Sizes: cells, connections, Jacobian entries (n_cells + 2 n_conn), precision. */
int tpfa_mesh_info(tpfa_mesh m, long long* n_cells, long long* n_conn, long long* nnz, int* precision);

/* As tpfa_sync_status. */
int tpfa_mesh_sync_status(tpfa_mesh m, void* stream);

/* Free the mesh; NULL-safe.  Synchronises the device. */
int tpfa_destroy_mesh(tpfa_mesh m);

/* ---------------------------------------------------------------- ensembles */

typedef struct tpfa_ensemble_s* tpfa_ensemble; /* opaque, library-owned */

/*
 * An ensemble of M grids of uneven sizes (for example geomodel realisations of
 * an uncertainty sweep) assembled by ONE persistent kernel launch, captured
 * with the reset of its tile counter in a CUDA graph.  All grids must use
 * TPFA_MIXED, the same connectivity, and either all c_r == 0 or all c_r != 0.
 * The grids are BORROWED (they must outlive the ensemble); each one's bound
 * state (tpfa_set_state / tpfa_set_pressure) is read at every batch call.
 * Each model's residual and Jacobian are bit-identical to its own
 * tpfa_assemble_jacobian call.
 */
int tpfa_create_ensemble(tpfa_ensemble* out, int M, const tpfa_handle* grids);

/* Outputs of model m, as in tpfa_assemble_jacobian (vals non-NULL; R and
 * diag64 may be NULL).  Device pointers, caller-owned. */
int tpfa_ensemble_set_outputs(tpfa_ensemble e, int m, double* R_dev, void* vals_dev, double* diag64_dev);

/* Assemble every model: uploads the model table when a bound state or an
 * output changed since the last call, then launches the graph on `stream`. */
int tpfa_assemble_batch(tpfa_ensemble e, void* stream);

/* The ensemble's tiling (see tpfa_set_tiling), its number of tiles and of
 * persistent blocks (the latter known after the first batch call). */
int tpfa_ensemble_tiling(tpfa_ensemble e, int* rows_per_march, int* warps_per_block, long long* tiles,
                         int* blocks);

/* Choose the ensemble's tiling by timing the batch call (or from the cache,
 * as tpfa_autotune).  Needs every model's state and outputs; synchronises. */
int tpfa_ensemble_autotune(tpfa_ensemble e, const char* cache_path, void* stream);

/* Free the ensemble (not its grids); NULL-safe.  Synchronises the device. */
int tpfa_destroy_ensemble(tpfa_ensemble e);

/* Size of the fixed device workspace of tpfa_assemble_jacobian_static. */
#define TPFA_STATIC_WORKSPACE_BYTES (64ULL * 1024ULL * 1024ULL)

/*
 * Residual and Jacobian with NO device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * call cudaMalloc (an application whose own pooled allocator has reserved
 * the GPU, a process with a hard device-memory budget, code running where
 * new allocations are not allowed).  It computes exactly what
 * tpfa_create_grid + tpfa_set_state + tpfa_assemble_jacobian compute, with
 * the same kernels, but keeps every intermediate array in one fixed
 * workspace: a file-scope device array of TPFA_STATIC_WORKSPACE_BYTES
 * (64 MiB) that every GPU which loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *   nx, ny, nz, prm, prec, perm_dev, poro_dev, depth_dev : as tpfa_create_grid
 *   p_dev, p_prev_dev : as tpfa_set_state (field type of `prec`)
 *   R_dev, vals_dev, diag64_dev : as tpfa_assemble_jacobian (CSR order of the
 *       pattern; tpfa_nnz gives the length of vals_dev)
 *   status_dev : optional device word; if non-NULL it is set (asynchronously)
 *       to 1 when an assembled value is NaN/Inf and to 0 otherwise
 *   stream     : cudaStream_t as void*; the call is asynchronous on it
 *
 * Limits: the workspace holds the error word (the first 256 bytes), then
 * each intermediate array starting on a 256-byte boundary: the owned
 * transmissibilities (3 with 6 links, 5 with 10; field type), on the mixed
 * path the FP32 depth (and the FP32 phi0 when c_r != 0), and m^n (FP64).
 * A grid is accepted exactly when
 *     256 + sum over those arrays of align256(N * bytes per element)
 *         <= TPFA_STATIC_WORKSPACE_BYTES,
 * align256(x) rounding x up to a multiple of 256; tpfa_static_workspace_bytes
 * evaluates the left-hand side.  That is about 32 bytes per cell with 10
 * links on the mixed path (36 with c_r != 0: about 2.09 M and 1.86 M cells)
 * and 48 bytes on the FP64 path (about 1.39 M cells).  Larger grids return
 * TPFA_ERR_TOO_LARGE, with a message giving the bytes needed, before any
 * device work; use the handle API for them.
 *
 * The workspace is shared by every call and keeps the last call's contents;
 * each call overwrites what it reads and clears its error word first.  Calls
 * whose GPU work overlaps (other streams or host threads without ordering)
 * race on it.  Each call outside stream capture looks up the workspace's
 * device address on the current device (cudaGetSymbolAddress) and keeps it;
 * a call made while `stream` is being captured uses the address kept from
 * an earlier call on that device, so make the first call on each device
 * before any stream capture (a first call under capture returns
 * TPFA_ERR_CUDA).
 */
int tpfa_assemble_jacobian_static(int nx, int ny, int nz, const tpfa_params* prm, tpfa_precision prec,
                                  const double* perm_dev, const double* poro_dev, const double* depth_dev,
                                  const void* p_dev, const void* p_prev_dev, double* R_dev, void* vals_dev,
                                  double* diag64_dev, unsigned int* status_dev, void* stream);

/* Bytes of the fixed workspace that tpfa_assemble_jacobian_static needs for
 * an nx x ny x nz grid (the left-hand side of its size rule above);
 * rock_compressible != 0 when c_r != 0.  Host-only, needs no GPU.  Returns
 * a negative TPFA_ERR_* code for bad arguments.  The paper has no
 * counterpart: this is a helper of the allocation-free entry point. */
long long tpfa_static_workspace_bytes(int nx, int ny, int nz, int connectivity, tpfa_precision prec,
                                      int rock_compressible);

/*
 * The library's own exponentials, evaluated element-wise so that they can be
 * checked against CUDA's exp / expm1 / expm1f over an argument sweep.  Eq.
 * density's exp(c_f (p - p_ref)) takes exp_fp64 on the FP64 path, and the
 * accumulation term of Eq. vk, written with expm1(c_f (p - p^n)), takes
 * expm1_fp64 on the FP64 path and expm1_f32 in the FP32 kernels.  Below
 * |x| < 2^-5 (FP64) and |x| < 2^-7 (FP32) they are Taylor series in Horner
 * form; larger arguments, NaN and infinities go to CUDA's exp / expm1 /
 * expm1f.
 *
 *   fn    : which routine (TPFA_MATH_EXPM1_FP32 rounds each x to FP32
 *           first; its FP32 result is widened exactly)
 *   x_dev : n doubles (device, caller-owned, read only)
 *   y_dev : n doubles (device, caller-owned), written
 *   n     : number of arguments; 0 launches nothing
 *   stream: cudaStream_t as void*; asynchronous on it, on the current
 *           device (x_dev and y_dev must live there)
 *
 * TPFA_ERR_INVALID_ARG for an unknown fn, n < 0, or a NULL pointer with
 * n > 0; TPFA_ERR_CUDA if the launch fails.  A test and diagnostics entry
 * point: no assembly call needs it.
 */
typedef enum {
    TPFA_MATH_EXP_FP64 = 0,
    TPFA_MATH_EXPM1_FP64 = 1,
    TPFA_MATH_EXPM1_FP32 = 2
} tpfa_math_fn;
int tpfa_math_eval(tpfa_math_fn fn, const double* x_dev, double* y_dev, long long n, void* stream);

/* Free everything the handle owns; NULL-safe.  Synchronises the device. */
int tpfa_destroy(tpfa_handle h);

/* Message of the last error on this host thread ("" if none). */
const char* tpfa_last_error_string(void);

/* Library version as major*10000 + minor*100 + patch. */
int tpfa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TPFA_H */
