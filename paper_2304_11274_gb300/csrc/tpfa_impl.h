// tpfa_impl.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/tpfa.h"
#include "tpfa_grid.h"
#include "tpfa_mesh.h"
#include "tpfa_tma.cuh"

namespace tpfa {

struct PhysF;
struct PhysD;

enum class AsmKernel { Naive, YMarch, YMarchTma, XMarch };

// JY: rows per warp march; W: warps (z-planes) per block, 4 or 8.  The tiled
// kernels may be restricted to the planes [k0, k1) (rows outside are not
// written; their cells are still read as neighbours); the default is the
// grid.  The naive kernel always covers the grid.
cudaError_t launch_assemble_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk,
                                  const AsmFields<float>& f, const AsmOut<float>& o, int JY, int W,
                                  cudaStream_t st, int k0 = 0, int k1 = -1);
cudaError_t launch_assemble_fp64(AsmKernel kern, const GridGeom& g, const PhysD& q, bool crk,
                                 const AsmFields<double>& f, const AsmOut<double>& o, int JY, int W,
                                 cudaStream_t st, int k0 = 0, int k1 = -1);
// The mixed march with TMA row loads (same rows, same bits).  The maps come
// from tma_encode_state (p, p^n: whenever the bound pointers change) and
// tma_encode_static (the library-owned fields); both return false when the
// grid (nx not a multiple of 4) or a pointer (not 16-byte aligned) rules TMA
// out, or the driver offers no tensor-map encoder.
cudaError_t launch_assemble_mixed_tma(const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                                      const AsmOut<float>& o, const TmaMaps& maps, int JY, int W, cudaStream_t st,
                                      int k0 = 0, int k1 = -1);
bool tma_grid_ok(const GridGeom& g);
// Whether the mixed path's fused residual + Jacobian runs the two-cell march
// on these fields (nx even, pair-aligned fields, 16-byte aligned m^n).
bool xmarch_ok(const GridGeom& g, const AsmFields<float>& f);

bool tma_encode_state(TmaMaps* m, const GridGeom& g, const float* p, const float* pn);
bool tma_encode_static(TmaMaps* m, const GridGeom& g, const AsmFields<float>& f, bool crk);

// Setup kernels (tpfa_setup.cu).
struct SetupPhys {
    double dx, dy, dz;
    double rho_ref, p_ref, c_f, c_r, V_dt;
};
// Owned transmissibilities from permeability, computed in FP64 and stored as
// `Real` (float or double).  Tpp/Tmp may be null with 6-point connectivity.
// With log_k the array holds ln k and k = exp(ln k) is formed per read.
cudaError_t launch_transmissibility_f32(const GridGeom& g, const SetupPhys& s, const double* perm,
                                        float* Tx, float* Ty, float* Tz, float* Tpp, float* Tmp,
                                        cudaStream_t st, bool log_k = false);
cudaError_t launch_transmissibility_f64(const GridGeom& g, const SetupPhys& s, const double* perm,
                                        double* Tx, double* Ty, double* Tz, double* Tpp, double* Tmp,
                                        cudaStream_t st, bool log_k = false);
cudaError_t launch_convert_f32(const double* in, float* out, long long n, cudaStream_t st);
cudaError_t launch_copy_f64(const double* in, double* out, long long n, cudaStream_t st);
// m^n = (V/dt) phi(p^n) rho(p^n) in FP64 from p^n of either field type.
cudaError_t launch_prev_mass_f32(const SetupPhys& s, const float* pn, const double* phi0, double* mn,
                                 long long n, cudaStream_t st);
cudaError_t launch_prev_mass_f64(const SetupPhys& s, const double* pn, const double* phi0, double* mn,
                                 long long n, cudaStream_t st);
// Adjoint (tpfa_vjp.cu).
struct LinkGeo;
// The mixed path's adjoint runs the y-march (JY rows per march, W warps per
// block) or its naive gather twin; lg: distance over area per link direction.
// vsplit: N float2 of workspace for the cotangent's FP32 pairs.
cudaError_t launch_vjp_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                             const float* kperm, const LinkGeo& lg, const double* v, float2* vsplit, double* g_p,
                             double* g_lnk, unsigned int* status, int JY, int W, cudaStream_t st);
cudaError_t launch_vjp_fp64(const GridGeom& g, const PhysD& q, bool crk, const AsmFields<double>& f,
                            const double* kperm, const double* v, double* g_p, double* g_lnk,
                            unsigned int* status, cudaStream_t st);
// Matrix-free J w (tpfa_jvp.cu); R may be null.  The mixed path runs the
// y-march (JY rows per march, W warps per block) or the naive gather.
cudaError_t launch_jvp_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                             const double* w, double* Jw, double* R, unsigned int* status, int JY, int W,
                             cudaStream_t st);
cudaError_t launch_jvp_fp64(const GridGeom& g, const PhysD& q, bool crk, const AsmFields<double>& f, const double* w,
                            double* Jw, double* R, unsigned int* status, cudaStream_t st);
// k in the path's precision (the adjoint's copy), from k or (log_k) ln k.
cudaError_t launch_store_perm_f32(const double* perm, float* out, long long n, cudaStream_t st, bool log_k = false);
cudaError_t launch_store_perm_f64(const double* perm, double* out, long long n, cudaStream_t st, bool log_k = false);

// Preconditioned BiCGStab (tpfa_krylov.cu).  The scalars live on the
// device; the host polls them.
struct KrylovScalars {
    double rho, alpha, omega, beta, rr, bb, tol2;
    int done, breakdown, iter, max_iters;
};
struct KrylovWork {
    double *x, *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;
    float *phh, *phl, *shh, *shl;  // p^ and s^ split into FP32 pairs (mixed path), else null
    double *lmul, *up;  // z-line factorisation: multipliers and super-diagonal
    double* part;       // 2 * krylov_partials() per-block partial sums
    KrylovScalars* S;
};
long long krylov_vec_blocks(long long n);
long long krylov_partials(const GridGeom& g, long long n);
// M^-1 data: the inverse diagonal (Jacobi) or the inverse pivots of the z-line
// factorisation (line).
cudaError_t krylov_dinv(const GridGeom& g, bool mixed, const void* vals, const double* diag64, double* dinv,
                        double* lmul, double* up, bool line, cudaStream_t st);
// x = 0, r = r^ = sign * b, scalars initialised (S->tol2, S->max_iters set by the caller)
cudaError_t krylov_start(const GridGeom& g, long long n, const double* b, double sign, const KrylovWork& w,
                         cudaStream_t st);
cudaError_t krylov_iteration(const GridGeom& g, long long n, bool mixed, const void* vals, const double* diag64,
                             const KrylovWork& w, bool line, cudaStream_t st);
cudaError_t krylov_add_delta(long long n, bool mixed, void* p, const double* d, cudaStream_t st);

// General meshes (tpfa_mesh.cu).
cudaError_t launch_mesh_vphi(long long n, double dt, bool mixed, const double* V, const double* poro,
                             double* vphi_d, void* vphi_r, cudaStream_t st);
cudaError_t launch_mesh_mixed(const MeshFields<float>& f, long long n, const PhysF& q, bool crk,
                              const AsmOut<float>& o, cudaStream_t st);
cudaError_t launch_mesh_fp64(const MeshFields<double>& f, long long n, const PhysD& q, bool crk,
                             const AsmOut<double>& o, cudaStream_t st);

// Sets the thread-local message of tpfa_last_error_string and returns code.
int report_error(int code, const char* msg);

// Raises `func`'s dynamic shared-memory limit to `bytes` in the current
// device's context.  The attribute belongs to the function in one context,
// so it is set once per (function, device) pair; the record of pairs done
// is guarded by a mutex, so host threads may launch concurrently.
cudaError_t ensure_smem_limit(const void* func, int bytes);

// CSR pattern (row_ptr int64 N+1, col_idx int32 nnz).
cudaError_t launch_pattern(const GridGeom& g, long long* row_ptr, int* col_idx, cudaStream_t st);

// y[i] = the library exponential `fn` (a tpfa_math_fn) of x[i], i < n.
cudaError_t launch_math_eval(int fn, const double* x, double* y, long long n, cudaStream_t st);

}  // namespace tpfa
