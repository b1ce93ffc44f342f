// tpfa_setup.cu -- per-grid and per-time-step setup kernels (not on the
// per-Newton-iteration path): owned transmissibilities, the CSR pattern,
// field conversion and the previous-step mass m^n.
#include <cuda_runtime.h>

#include "tpfa_common.cuh"
#include "tpfa_impl.h"

namespace tpfa {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > (1LL << 30)) b = 1LL << 30;  // grid-stride loops cover the rest
    return (unsigned)(b > 0 ? b : 1);
}

// Two-point transmissibility (the paper names Upsilon_KL without a formula):
// half-transmissibilities k area / (d/2) in series, i.e.
// 2 k_K k_L / (k_K + k_L) * area / d; zero if either cell is impermeable.
__device__ __forceinline__ double two_point(double kK, double kL, double area_over_d) {
    if (!(kK > 0.0) || !(kL > 0.0)) return 0.0;
    return (2.0 * kK * kL / (kK + kL)) * area_over_d;
}

struct Geo {
    double ax, ay, az, ad;  // area / distance of x, y, z faces and of an in-plane diagonal
};

// Permeability of cell c: the stored value, or exp of the stored natural
// log (the adjoint's parameterisation, k = exp(ln k)).
template <bool LOG>
__device__ __forceinline__ double perm_at(const double* __restrict__ perm, long long c) {
    return LOG ? exp(perm[c]) : perm[c];
}

template <typename Real, bool LOG>
__global__ void k_trans(GridGeom g, Geo geo, const double* __restrict__ perm, Real* Tx, Real* Ty, Real* Tz,
                        Real* Tpp, Real* Tmp) {
    const long long nx = g.nx, nxy = nx * g.ny, N = nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(c / nxy);
        const int j = (int)((c - k * nxy) / nx);
        const int i = (int)(c - k * nxy - j * nx);
        // neighbour indices fall back to c itself where the link does not
        // exist, so every address formed is inside perm
        const double kc = perm_at<LOG>(perm, c);
        const bool xp = i + 1 < g.nx, yp = j + 1 < g.ny, zp = k + 1 < g.nz;
        Tx[c] = (Real)(xp ? two_point(kc, perm_at<LOG>(perm, xp ? c + 1 : c), geo.ax) : 0.0);
        Ty[c] = (Real)(yp ? two_point(kc, perm_at<LOG>(perm, yp ? c + nx : c), geo.ay) : 0.0);
        Tz[c] = (Real)(zp ? two_point(kc, perm_at<LOG>(perm, zp ? c + nxy : c), geo.az) : 0.0);
        if (g.diag) {
            const bool pp = yp && xp, mp = yp && i > 0;
            Tpp[c] = (Real)(pp ? two_point(kc, perm_at<LOG>(perm, pp ? c + nx + 1 : c), geo.ad) : 0.0);
            Tmp[c] = (Real)(mp ? two_point(kc, perm_at<LOG>(perm, mp ? c + nx - 1 : c), geo.ad) : 0.0);
        }
    }
}

// k in the path's precision for the adjoint, from k or from ln k.
template <typename Real, bool LOG>
__global__ void k_store_perm(const double* __restrict__ perm, Real* out, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = (Real)perm_at<LOG>(perm, c);
}

// The library's own exponentials, one argument per element: exp_fp64,
// expm1_fp64, and expm1_f32 of the argument rounded to FP32 (its result
// widened exactly).  Only tpfa_math_eval launches it.
__global__ void k_math_eval(int fn, const double* __restrict__ x, double* __restrict__ y, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double a = x[c];
        double r;
        if (fn == TPFA_MATH_EXP_FP64) r = exp_fp64(a);
        else if (fn == TPFA_MATH_EXPM1_FP64) r = expm1_fp64(a);
        else r = (double)expm1_f32(__double2float_rn(a));
        y[c] = r;
    }
}

Geo make_geo(const SetupPhys& s) {
    Geo q;
    q.ax = s.dy * s.dz / s.dx;
    q.ay = s.dx * s.dz / s.dy;
    q.az = s.dx * s.dy / s.dz;
    // diagonal: distance sqrt(dx^2 + dy^2), area dz dx dy / distance
    q.ad = s.dz * s.dx * s.dy / (s.dx * s.dx + s.dy * s.dy);
    return q;
}

__global__ void k_to_f32(const double* __restrict__ in, float* out, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = (float)in[c];
}

__global__ void k_copy_f64(const double* __restrict__ in, double* out, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = in[c];
}

// m^n = (V/dt) phi(p^n) rho(p^n), phi(p) = phi0 (1 + c_r (p - p_ref)),
// rho(p) = rho_ref exp(c_f (p - p_ref))  (Eq. density), in FP64.
template <typename Real>
__global__ void k_prev_mass(SetupPhys s, const Real* __restrict__ pn, const double* __restrict__ phi0, double* mn,
                            long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double p = (double)pn[c];
        const double dp = p - s.p_ref;
        const double phi = phi0[c] * (1.0 + s.c_r * dp);
        const double rho = s.rho_ref * exp(s.c_f * dp);
        mn[c] = s.V_dt * (phi * rho);
    }
}

// One thread per row: row_ptr[row] from the closed form, then the valid
// neighbours in ascending column order (the slot order of tpfa_row.cuh).
__global__ void k_pattern(GridGeom g, long long* row_ptr, int* col_idx) {
    const long long nx = g.nx, nxy = nx * g.ny, N = nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(c / nxy);
        const int j = (int)((c - k * nxy) / nx);
        const int i = (int)(c - k * nxy - j * nx);
        const long long rs = row_start(g, i, j, k);
        row_ptr[c] = rs;
        if (c == N - 1) row_ptr[N] = total_nnz(g);
        const bool xm = i > 0, xp = i + 1 < g.nx, ym = j > 0, yp = j + 1 < g.ny, zm = k > 0, zp = k + 1 < g.nz;
        const bool d = g.diag != 0;
        long long e = rs;
        if (zm) col_idx[e++] = (int)(c - nxy);
        if (d && xm && ym) col_idx[e++] = (int)(c - nx - 1);
        if (ym) col_idx[e++] = (int)(c - nx);
        if (d && xp && ym) col_idx[e++] = (int)(c - nx + 1);
        if (xm) col_idx[e++] = (int)(c - 1);
        col_idx[e++] = (int)c;
        if (xp) col_idx[e++] = (int)(c + 1);
        if (d && xm && yp) col_idx[e++] = (int)(c + nx - 1);
        if (yp) col_idx[e++] = (int)(c + nx);
        if (d && xp && yp) col_idx[e++] = (int)(c + nx + 1);
        if (zp) col_idx[e++] = (int)(c + nxy);
    }
}

}  // namespace

cudaError_t launch_transmissibility_f32(const GridGeom& g, const SetupPhys& s, const double* perm, float* Tx,
                                        float* Ty, float* Tz, float* Tpp, float* Tmp, cudaStream_t st, bool log_k) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    if (log_k) k_trans<float, true><<<blocks_for(N), kThreads, 0, st>>>(g, make_geo(s), perm, Tx, Ty, Tz, Tpp, Tmp);
    else k_trans<float, false><<<blocks_for(N), kThreads, 0, st>>>(g, make_geo(s), perm, Tx, Ty, Tz, Tpp, Tmp);
    return cudaGetLastError();
}

cudaError_t launch_transmissibility_f64(const GridGeom& g, const SetupPhys& s, const double* perm, double* Tx,
                                        double* Ty, double* Tz, double* Tpp, double* Tmp, cudaStream_t st,
                                        bool log_k) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    if (log_k) k_trans<double, true><<<blocks_for(N), kThreads, 0, st>>>(g, make_geo(s), perm, Tx, Ty, Tz, Tpp, Tmp);
    else k_trans<double, false><<<blocks_for(N), kThreads, 0, st>>>(g, make_geo(s), perm, Tx, Ty, Tz, Tpp, Tmp);
    return cudaGetLastError();
}

cudaError_t launch_store_perm_f32(const double* perm, float* out, long long n, cudaStream_t st, bool log_k) {
    if (log_k) k_store_perm<float, true><<<blocks_for(n), kThreads, 0, st>>>(perm, out, n);
    else k_store_perm<float, false><<<blocks_for(n), kThreads, 0, st>>>(perm, out, n);
    return cudaGetLastError();
}

cudaError_t launch_store_perm_f64(const double* perm, double* out, long long n, cudaStream_t st, bool log_k) {
    if (log_k) k_store_perm<double, true><<<blocks_for(n), kThreads, 0, st>>>(perm, out, n);
    else k_store_perm<double, false><<<blocks_for(n), kThreads, 0, st>>>(perm, out, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_f32(const double* in, float* out, long long n, cudaStream_t st) {
    k_to_f32<<<blocks_for(n), kThreads, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_copy_f64(const double* in, double* out, long long n, cudaStream_t st) {
    k_copy_f64<<<blocks_for(n), kThreads, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_prev_mass_f32(const SetupPhys& s, const float* pn, const double* phi0, double* mn, long long n,
                                 cudaStream_t st) {
    k_prev_mass<float><<<blocks_for(n), kThreads, 0, st>>>(s, pn, phi0, mn, n);
    return cudaGetLastError();
}

cudaError_t launch_prev_mass_f64(const SetupPhys& s, const double* pn, const double* phi0, double* mn, long long n,
                                 cudaStream_t st) {
    k_prev_mass<double><<<blocks_for(n), kThreads, 0, st>>>(s, pn, phi0, mn, n);
    return cudaGetLastError();
}

cudaError_t launch_pattern(const GridGeom& g, long long* row_ptr, int* col_idx, cudaStream_t st) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    k_pattern<<<blocks_for(N), kThreads, 0, st>>>(g, row_ptr, col_idx);
    return cudaGetLastError();
}

cudaError_t launch_math_eval(int fn, const double* x, double* y, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_math_eval<<<blocks_for(n), kThreads, 0, st>>>(fn, x, y, n);
    return cudaGetLastError();
}

}  // namespace tpfa
