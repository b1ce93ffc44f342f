// tpfa_vjp.cu -- adjoint of the residual: vector-Jacobian products with
// respect to pressure and log-permeability (sm_103a).
//
// For a cotangent v (one value per cell) the kernel gathers, per cell i,
//   g_p[i]   = sum_K v_K dR_K/dp_i
//            = v_i (dA_i/dp_i + sum_L dF_iL/dp_i) + sum_L v_L dF_Li/dp_i
//   g_lnk[i] = sum_K v_K dR_K/d(ln k_i)
//            = sum_L (v_i - v_L) F_iL k_L / (k_i + k_L)
// (L over adj(i), Section 5.1; Eq. vk and Eq. flux-calc; the second line uses
// F_Li = -F_iL and d Upsilon_iL / d ln k_i = Upsilon_iL k_L / (k_i + k_L) of
// the harmonic two-point transmissibility).  dF_Li/dp_i is the derivative of
// row L's link seen from L; it equals -dF_iL/dp_i except at an exact tie
// dPhi = 0, where it is evaluated from L's side.  Nothing is stored between
// the forward assembly and this pass: densities, upwind choices and
// mobilities are recomputed (gather form, one thread per cell, no atomics).
//
// Arithmetic: links in the path's precision (FP32 on the mixed path), the
// v-weighted sums and both outputs in FP64.
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"

namespace tpfa {

namespace {

// Checked load: an index outside [0, N) or a NULL array latches
// STATUS_DEVICE_CHECK (reported as TPFA_ERR_DEVICE_CHECK by tpfa_sync_status)
// and reads nothing.  The adjoint kernel reads every field through it.
template <typename T>
__device__ __forceinline__ T ld_chk(const T* p, long long idx, long long N, unsigned int* status) {
    if (p == nullptr || idx < 0 || idx >= N) {
        atomicOr(status, STATUS_DEVICE_CHECK);
        return T(0);
    }
    return __ldg(p + idx);
}

template <typename Real>
__device__ __forceinline__ double to_f64(Real x) {
    if constexpr (sizeof(Real) == 4) return widen(x);
    else return x;
}

template <typename Real, bool CRK>
__global__ void __launch_bounds__(256) k_vjp(GridGeom g, typename PhysOf<Real>::type q, AsmFields<Real> f,
                                             const Real* __restrict__ kperm, const double* __restrict__ v,
                                             double* __restrict__ g_p, double* __restrict__ g_lnk,
                                             unsigned int* status) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int nx = g.nx, nxy = nx * g.ny;
    const int c = i + nx * j + nxy * k;
    const long long NN = (long long)nxy * g.nz;
    const unsigned mask = slot_mask(g, i, j, k);
    const int off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
    const CellVal<Real> me = make_cell(q, ld_chk(f.p, c, NN, status), ld_chk(f.z, c, NN, status));
    const double vi = ld_chk(v, c, NN, status);
    const Real ki = ld_chk(kperm, c, NN, status);
    double diag = 0.0, offs = 0.0, glnk = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        if (s == SLOT_SELF) continue;
        const bool valid = (mask & (1u << s)) != 0;
        // invalid slots keep an in-range index (the cell itself), so a load
        // scheduled ahead of the guard still reads inside the arrays
        const int d = valid ? c + off[s] : c;
        if (!valid) continue;
        const Real* Tp;
        int ti;
        switch (s) {
            case 0: Tp = f.Tz; ti = d; break;
            case 1: Tp = f.Tpp; ti = d; break;
            case 2: Tp = f.Ty; ti = d; break;
            case 3: Tp = f.Tmp; ti = d; break;
            case 4: Tp = f.Tx; ti = d; break;
            case 6: Tp = f.Tx; ti = c; break;
            case 7: Tp = f.Tmp; ti = c; break;
            case 8: Tp = f.Ty; ti = c; break;
            case 9: Tp = f.Tpp; ti = c; break;
            default: Tp = f.Tz; ti = c; break;
        }
        const Real T = ld_chk(Tp, ti, NN, status);
        const CellVal<Real> nb = make_cell(q, ld_chk(f.p, d, NN, status), ld_chk(f.z, d, NN, status));
        const LinkOut<Real> L = link(q, T, me, nb);
        // row L's derivative with respect to p_i
        const Real dLi = (L.F == Real(0) && T != Real(0)) ? link(q, T, nb, me).Db : -L.Da;
        const double vl = ld_chk(v, d, NN, status);
        const Real kl = ld_chk(kperm, d, NN, status);
        diag += to_f64(L.Da);
        offs = fma(vl, to_f64(dLi), offs);
        const Real ratio = (ki + kl) > Real(0) ? kl / (ki + kl) : Real(0);
        glnk = fma(vi - vl, to_f64(L.F) * to_f64(ratio), glnk);
    }
    Real pn = ld_chk(f.pn, c, NN, status);
    if constexpr (sizeof(Real) == 4) {
        const AccF acc = accumulation<CRK>(q, me.p, pn, ld_chk(f.mn, c, NN, status), me.rho, CRK ? ld_chk(f.phi0, c, NN, status) : 0.f);
        diag += widen(acc.dA);
    } else {
        const AccD acc = accumulation<CRK>(q, me.p, pn, ld_chk(f.mn, c, NN, status), me.rho, CRK ? ld_chk(f.phi0, c, NN, status) : 0.0);
        diag += acc.dA;
    }
    const double gp = fma(vi, diag, offs);
    if (c < 0 || c >= NN || g_p == nullptr) {
        atomicOr(status, STATUS_DEVICE_CHECK);
        return;
    }
    g_p[c] = gp;
    if (g_lnk) g_lnk[c] = glnk;
    if (nonfinite(gp) || nonfinite(glnk)) atomicOr(status, STATUS_NONFINITE);
}

// k stored in the path's precision for the adjoint.
template <typename Real>
__global__ void k_store_perm(const double* __restrict__ perm, Real* out, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = (Real)perm[c];
}

}  // namespace

template <typename Real>
static cudaError_t launch_vjp_t(const GridGeom& g, const typename PhysOf<Real>::type& q, bool crk,
                                const AsmFields<Real>& f, const Real* kperm, const double* v, double* g_p,
                                double* g_lnk, unsigned int* status, cudaStream_t st) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    if (crk) k_vjp<Real, true><<<grid, block, 0, st>>>(g, q, f, kperm, v, g_p, g_lnk, status);
    else k_vjp<Real, false><<<grid, block, 0, st>>>(g, q, f, kperm, v, g_p, g_lnk, status);
    return cudaGetLastError();
}

cudaError_t launch_vjp_mixed(const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                             const float* kperm, const double* v, double* g_p, double* g_lnk,
                             unsigned int* status, cudaStream_t st) {
    return launch_vjp_t<float>(g, q, crk, f, kperm, v, g_p, g_lnk, status, st);
}

cudaError_t launch_vjp_fp64(const GridGeom& g, const PhysD& q, bool crk, const AsmFields<double>& f,
                            const double* kperm, const double* v, double* g_p, double* g_lnk,
                            unsigned int* status, cudaStream_t st) {
    return launch_vjp_t<double>(g, q, crk, f, kperm, v, g_p, g_lnk, status, st);
}

cudaError_t launch_store_perm_f32(const double* perm, float* out, long long n, cudaStream_t st) {
    const long long b = (n + 255) / 256;
    k_store_perm<float><<<(unsigned)(b < (1LL << 30) ? (b > 0 ? b : 1) : (1LL << 30)), 256, 0, st>>>(perm, out, n);
    return cudaGetLastError();
}

cudaError_t launch_store_perm_f64(const double* perm, double* out, long long n, cudaStream_t st) {
    const long long b = (n + 255) / 256;
    k_store_perm<double><<<(unsigned)(b < (1LL << 30) ? (b > 0 ? b : 1) : (1LL << 30)), 256, 0, st>>>(perm, out, n);
    return cudaGetLastError();
}

}  // namespace tpfa
