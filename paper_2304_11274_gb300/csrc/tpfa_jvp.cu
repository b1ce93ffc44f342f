// tpfa_jvp.cu -- matrix-free Jacobian-vector product of the residual (sm_103a).
//
// For a direction w (one value per cell), per cell K (Algorithm 1's loops,
// the derivatives of Eq. vk with the flux of Eq. flux-calc):
//   (J w)_K = dA_K/dp_K w_K + sum_{L in adj(K)} ( dF_KL/dp_K w_K + dF_KL/dp_L w_L )
// without storing J: the operator a Krylov solver of Eq. vk needs.  The same
// pass can also produce R_K, summed exactly as the assembly kernels sum it,
// so R here is bit-identical to tpfa_assemble_residual's.  As in the
// assembly, the tiled kernel reuses the links into the previous y-row and
// recomputes, after its march, the rows where one of them was an exact tie.
//
// Mixed path: w is narrowed to FP32 (truncation, on the integer pipe); per
// link the term dF/dp_K w_K + dF/dp_L w_L is one FP32 fma of the link's FP32
// derivatives; the terms are Kahan-summed in FP32 in slot order, then
// dA/dp w_K, and the sum is combined in FP64.  The error is a few float ulps
// of sum_L |J_KL| |w_L|.  Two kernels give identical bits: the y-march (the
// production kernel, the assembly's march with w in its prefetch ring) and a
// one-thread-per-cell gather with checked loads.
//
// FP64 path: one thread per cell, links and sums in FP64 (bound by the FP64
// pipe, like the FP64 assembly).
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_ymarch.cuh"

namespace tpfa {

namespace {

template <typename T>
__device__ __forceinline__ T ldc(const T* p, long long idx, long long N, unsigned int* status) {
    if (p == nullptr || idx < 0 || idx >= N) {
        atomicOr(status, STATUS_DEVICE_CHECK);
        return T(0);
    }
    return __ldg(p + idx);
}

// Neighbour index and owned-transmissibility array of slot s of cell c.
template <typename Real>
__device__ __forceinline__ const Real* slot_T(const AsmFields<Real>& f, int s, int c, int d, int& ti) {
    switch (s) {
        case 0: ti = d; return f.Tz;
        case 1: ti = d; return f.Tpp;
        case 2: ti = d; return f.Ty;
        case 3: ti = d; return f.Tmp;
        case 4: ti = d; return f.Tx;
        case 6: ti = c; return f.Tx;
        case 7: ti = c; return f.Tmp;
        case 8: ti = c; return f.Ty;
        case 9: ti = c; return f.Tpp;
        default: ti = c; return f.Tz;
    }
}

// J w (and R) of cell (i, j, k) from global memory: the naive kernel's row,
// and the tiled kernel's for the rows whose reused links met an exact tie.
template <typename Real, bool CRK>
__device__ __forceinline__ void jvp_row(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                        const AsmFields<Real>& f, const double* __restrict__ w,
                                        double* __restrict__ Jw, double* __restrict__ R, unsigned int* status, int i,
                                        int j, int k) {
    const int nx = g.nx, nxy = nx * g.ny;
    const long long NN = (long long)nxy * g.nz;
    const int c = i + nx * j + nxy * k;
    const unsigned mask = slot_mask(g, i, j, k);
    const int off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
    const CellVal<Real> me = make_cell(q, ldc(f.p, c, NN, status), ldc(f.z, c, NN, status));
    double jw, r;
    if constexpr (sizeof(Real) == 4) {
        const float wc = narrow_rz(ldc(w, c, NN, status));
        Kahan32 rs, js;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s == SLOT_SELF || !(mask & (1u << s))) continue;
            const int d = c + off[s];
            int ti;
            const float* Tp = slot_T(f, s, c, d, ti);
            const CellVal<float> nb = make_cell(q, ldc(f.p, d, NN, status), ldc(f.z, d, NN, status));
            const LinkOut<float> L = link(q, ldc(Tp, ti, NN, status), me, nb);
            rs.add(L.F);
            js.add(__fmaf_rn(L.Da, wc, __fmul_rn(L.Db, narrow_rz(ldc(w, d, NN, status)))));
        }
        const AccF acc = accumulation<CRK>(q, me.p, ldc(f.pn, c, NN, status), ldc(f.mn, c, NN, status), me.rho,
                                           CRK ? ldc(f.phi0, c, NN, status) : 0.f);
        js.add(__fmul_rn(acc.dA, wc));
        jw = __dadd_rn(widen(js.s), -widen(js.c));
        r = __dadd_rn(__dadd_rn(acc.A, widen(rs.s)), -widen(rs.c));
    } else {
        const double wc = ldc(w, c, NN, status);
        double dsum = 0.0, osum = 0.0, rs = 0.0;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s == SLOT_SELF || !(mask & (1u << s))) continue;
            const int d = c + off[s];
            int ti;
            const double* Tp = slot_T(f, s, c, d, ti);
            const CellVal<double> nb = make_cell(q, ldc(f.p, d, NN, status), ldc(f.z, d, NN, status));
            const LinkOut<double> L = link(q, ldc(Tp, ti, NN, status), me, nb);
            rs = __dadd_rn(rs, L.F);
            dsum += L.Da;
            osum = fma(L.Db, ldc(w, d, NN, status), osum);
        }
        const AccD acc = accumulation<CRK>(q, me.p, ldc(f.pn, c, NN, status), ldc(f.mn, c, NN, status), me.rho,
                                           CRK ? ldc(f.phi0, c, NN, status) : 0.0);
        jw = fma(dsum + acc.dA, wc, osum);
        r = __dadd_rn(rs, acc.A);
    }
    Jw[c] = jw;
    if (R) R[c] = r;
    if (nonfinite(jw) || (R && nonfinite(r))) atomicOr(status, STATUS_NONFINITE);
}

template <typename Real, bool CRK>
__global__ void __launch_bounds__(256) k_jvp(GridGeom g, typename PhysOf<Real>::type q, AsmFields<Real> f,
                                             const double* __restrict__ w, double* __restrict__ Jw,
                                             double* __restrict__ R, unsigned int* status) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i < g.nx && j < g.ny) jvp_row<Real, CRK>(g, q, f, w, Jw, R, status, i, j, blockIdx.z);
}

// ---------------------------------------------------------------- y-march J w (mixed)

template <int W>
constexpr int jvp_smem_bytes() {
    using M = YMarch<float, true, false, false, W, true>;
    return W * (M::RING * M::NF * 32 * 4 + M::RING * 32 * 8 + M::RING * M::NW * 32 * 8);
}

template <bool DIAG, bool CRK, int W>
__global__ void __launch_bounds__(32 * W, 16 / W)
    k_jvp_ymarch(GridGeom g, PhysF q, AsmFields<float> f, AsmOut<float> o, const double* __restrict__ w,
                 double* __restrict__ Jw, int JY) {
    using M_t = YMarch<float, DIAG, CRK, false, W, true>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x, wi = threadIdx.y;
    const int k = blockIdx.z * W + wi;
    if (k >= g.nz) return;  // warp-uniform
    float* ring = reinterpret_cast<float*>(smem) + wi * M_t::RING * M_t::NF * 32;
    double* ringm = reinterpret_cast<double*>(reinterpret_cast<float*>(smem) + W * M_t::RING * M_t::NF * 32) +
                    wi * M_t::RING * 32;
    double* ringw = reinterpret_cast<double*>(reinterpret_cast<float*>(smem) + W * M_t::RING * M_t::NF * 32) +
                    W * M_t::RING * 32 + wi * M_t::RING * M_t::NW * 32;
    M_t M(g, q, f, o, lane, blockIdx.x * 32, k);
    M.ring = ring;
    M.ringm = ringm;
    M.ringw = ringw;
    M.wv = w;
    M.Jw = Jw;
    const int j0 = blockIdx.y * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;

    // prologue as in the assembly march: rows j0-1, j0, j0+1 into slots 0, 1, 2
    M.issue_row(j0 - 1, 0);
    M.issue_row(j0, 1);
    M.issue_row(j0 + 1, 2);
    M.wait_all_but_newest();
    YRow<float> P = M.row_cells(0);
    YRow<float> C = M.row_cells(1);
    YW wP = M.w_row(0);
    YW wC = M.w_row(1);
    float Ty_prev, Tpp_prev, Tmp_prev;
    {
        const YIn<float> Dp = M.read_in(0);
        Ty_prev = Dp.Ty;
        Tpp_prev = Dp.Tpp;
        Tmp_prev = Dp.Tmp;
    }
    YUp<float> U = M.up_links(P, C, Ty_prev, Tpp_prev, Tmp_prev);
    int s0 = 1, s1 = 2, s2 = 0;  // ring slots of rows j, j+1, j+2
    unsigned long long tie_rows = 0ull;  // rows recomputed after the march (as in the assembly)

    for (int j = j0; j < j1; ++j) {
        M.issue_row(j + 2, s2);
        M.wait_all_but_newest();
        if (__any_sync(0xffffffffu, U.tie)) tie_rows |= 1ull << (j - j0);
        const YRow<float> N = M.row_cells(s1);
        const YW wN = M.w_row(s1);
        const YIn<float> D = M.read_in(s0);
        const double* Wz = ringw + s0 * (M_t::NW * 32) + lane;
        const float wzm = narrow_rz(Wz[64]), wzp = narrow_rz(Wz[96]);
        const int st = s0;
        s0 = s1;
        s1 = s2;
        s2 = st;
        const bool injk = zint && j > 0 && j + 1 < M.ny;
        if (injk && M.xint) U = M.template row_jvp<2>(j, P, C, N, D, U, wP, wC, wN, wzm, wzp);
        else if (injk) U = M.template row_jvp<1>(j, P, C, N, D, U, wP, wC, wN, wzm, wzp);
        else U = M.template row_jvp<0>(j, P, C, N, D, U, wP, wC, wN, wzm, wzp);
        P = C;
        C = N;
        wP = wC;
        wC = wN;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tie_rows) {  // warp-uniform
        for (int b = 0; b < 64; ++b)
            if (((tie_rows >> b) & 1ull) && M.act) jvp_row<float, CRK>(g, q, f, w, Jw, o.R, o.status, M.i, j0 + b, k);
    }
}

template <bool DIAG, bool CRK, int W>
cudaError_t launch_jvp_ymarch_w(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const double* w,
                                double* Jw, double* R, unsigned int* status, int JY, cudaStream_t st) {
    constexpr int smem = jvp_smem_bytes<W>();
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(&k_jvp_ymarch<DIAG, CRK, W>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + JY - 1) / JY, (g.nz + W - 1) / W);
    AsmOut<float> o{R, nullptr, nullptr, status};
    k_jvp_ymarch<DIAG, CRK, W><<<grid, block, smem, st>>>(g, q, f, o, w, Jw, JY);
    return cudaGetLastError();
}

template <bool DIAG, bool CRK>
cudaError_t launch_jvp_ymarch_t(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const double* w,
                                double* Jw, double* R, unsigned int* status, int JY, int W, cudaStream_t st) {
    if (W == 8) return launch_jvp_ymarch_w<DIAG, CRK, 8>(g, q, f, w, Jw, R, status, JY, st);
    return launch_jvp_ymarch_w<DIAG, CRK, 4>(g, q, f, w, Jw, R, status, JY, st);
}

template <typename Real>
cudaError_t launch_jvp_naive(const GridGeom& g, const typename PhysOf<Real>::type& q, bool crk,
                             const AsmFields<Real>& f, const double* w, double* Jw, double* R, unsigned int* status,
                             cudaStream_t st) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    if (crk) k_jvp<Real, true><<<grid, block, 0, st>>>(g, q, f, w, Jw, R, status);
    else k_jvp<Real, false><<<grid, block, 0, st>>>(g, q, f, w, Jw, R, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_jvp_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                             const double* w, double* Jw, double* R, unsigned int* status, int JY, int W,
                             cudaStream_t st) {
    if (kern == AsmKernel::Naive) return launch_jvp_naive<float>(g, q, crk, f, w, Jw, R, status, st);
    if (g.diag) {
        return crk ? launch_jvp_ymarch_t<true, true>(g, q, f, w, Jw, R, status, JY, W, st)
                   : launch_jvp_ymarch_t<true, false>(g, q, f, w, Jw, R, status, JY, W, st);
    }
    return crk ? launch_jvp_ymarch_t<false, true>(g, q, f, w, Jw, R, status, JY, W, st)
               : launch_jvp_ymarch_t<false, false>(g, q, f, w, Jw, R, status, JY, W, st);
}

cudaError_t launch_jvp_fp64(const GridGeom& g, const PhysD& q, bool crk, const AsmFields<double>& f, const double* w,
                            double* Jw, double* R, unsigned int* status, cudaStream_t st) {
    return launch_jvp_naive<double>(g, q, crk, f, w, Jw, R, status, st);
}

}  // namespace tpfa
