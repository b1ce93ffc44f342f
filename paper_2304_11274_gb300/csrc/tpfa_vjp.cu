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
// mobilities are recomputed (gather form, no atomics).
//
// FP64 path: links, sums and outputs in FP64, one thread per cell.
//
// Mixed path: with dF_Li/dp_i = -dF_iL/dp_i except at an exact tie, and
// k_L / (k_i + k_L) = Upsilon_iL (d/A)_iL / (2 k_i) for the harmonic
// two-point transmissibility,
//   g_p[i]   = v_i dA_i/dp_i + sum_L dF_iL/dp_i (v_i - v_L) + sum_L v_L delta_iL
//   g_lnk[i] = sum_L F_iL Upsilon_iL (d/A)_iL / (2 k_i) (v_i - v_L)
// where delta_iL = dF_iL/dp_i + dF_Li/dp_i vanishes except at a tie.  Each v
// is split into an FP32 pair hi + lo, and v_i - v_L = (hi_i - hi_L) + (lo_i -
// lo_L) is formed in FP32, so each term is accurate relative to itself (a
// smooth v loses nothing); the pairs are formed once per call by a pre-pass
// (k_split_pairs), which keeps the FP64 unit out of the march.  The terms
// are FP32 products Kahan-summed in FP32 in slot order, then the cell's own
// term v_i dA_i/dp_i (one FP32 fused product of the pair), combined in
// FP64.  Two kernels give identical bits: the y-march of the
// assembly (its adjoint mode, the production kernel) and a
// one-thread-per-cell gather with checked loads.
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_xvjp.cuh"
#include "tpfa_ymarch.cuh"

namespace tpfa {

namespace {

// Checked load: an index outside [0, N) or a NULL array latches
// STATUS_DEVICE_CHECK (reported as TPFA_ERR_DEVICE_CHECK by tpfa_sync_status)
// and reads nothing.  The gather kernels read every field through it.
template <typename T>
__device__ __forceinline__ T ld_chk(const T* p, long long idx, long long N, unsigned int* status) {
    if (p == nullptr || idx < 0 || idx >= N) {
        atomicOr(status, STATUS_DEVICE_CHECK);
        return T{};
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

__device__ __forceinline__ float geo_of(const LinkGeo& lg, int s) {
    switch (s) {
        case 0:
        case 10: return lg.cz;
        case 2:
        case 8: return lg.cy;
        case 4:
        case 6: return lg.cx;
        default: return lg.cd;
    }
}

// The mixed path's adjoint of cell (i, j, k) from global memory: the naive
// kernel's row, and the tiled kernel's for the rows where a link had zero
// flux (every exact tie).
template <bool CRK>
__device__ __forceinline__ void vjp_row(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                        const float* __restrict__ kperm, const LinkGeo& lg,
                                        const float2* __restrict__ v, double* __restrict__ g_p,
                                        double* __restrict__ g_lnk, unsigned int* status, int i, int j, int k) {
    const int nx = g.nx, nxy = nx * g.ny;
    const int c = i + nx * j + nxy * k;
    const long long NN = (long long)nxy * g.nz;
    const unsigned mask = slot_mask(g, i, j, k);
    const int off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
    const CellVal<float> me = make_cell(q, ld_chk(f.p, c, NN, status), ld_chk(f.z, c, NN, status));
    const float2 vi = ld_chk(v, c, NN, status);
    const F2Split si{vi.x, vi.y};
    const float ki = ld_chk(kperm, c, NN, status);
    const float inv2k = ki > 0.f ? __fdiv_rn(0.5f, ki) : 0.f;
    Kahan32 kp, kk;
    double corr = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        if (s == SLOT_SELF || !(mask & (1u << s))) continue;
        const int d = c + off[s];
        const float* Tp;
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
        const float T = ld_chk(Tp, ti, NN, status);
        const CellVal<float> nb = make_cell(q, ld_chk(f.p, d, NN, status), ld_chk(f.z, d, NN, status));
        const LinkOut<float> L = link(q, T, me, nb);
        const float2 vl = ld_chk(v, d, NN, status);
        const F2Split sl{vl.x, vl.y};
        const float dv = diff_f2(si, sl);
        const float ratio = __fmul_rn(__fmul_rn(T, geo_of(lg, s)), inv2k);
        kp.add(__fmul_rn(L.Da, dv));
        kk.add(__fmul_rn(__fmul_rn(L.F, ratio), dv));
        const float dLK = link(q, T, nb, me).Db;
        const double vL = __dadd_rn(widen(sl.hi), widen(sl.lo));
        corr = __fma_rn(vL, widen(__fadd_rn(L.Da, dLK)), corr);
    }
    const AccF acc = accumulation<CRK>(q, me.p, ld_chk(f.pn, c, NN, status), ld_chk(f.mn, c, NN, status), me.rho,
                                       CRK ? ld_chk(f.phi0, c, NN, status) : 0.f);
    kp.add(__fmaf_rn(si.hi, acc.dA, __fmul_rn(si.lo, acc.dA)));
    const double gp = __dadd_rn(__dadd_rn(widen(kp.s), -widen(kp.c)), corr);
    const double gk = __dadd_rn(widen(kk.s), -widen(kk.c));
    g_p[c] = gp;
    if (g_lnk) g_lnk[c] = gk;
    if (nonfinite(gp) || nonfinite(gk)) atomicOr(status, STATUS_NONFINITE);
}

template <bool CRK>
__global__ void __launch_bounds__(256) k_vjp_mixed(GridGeom g, PhysF q, AsmFields<float> f,
                                                   const float* __restrict__ kperm, LinkGeo lg,
                                                   const float2* __restrict__ v, double* __restrict__ g_p,
                                                   double* __restrict__ g_lnk, unsigned int* status) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i < g.nx && j < g.ny) vjp_row<CRK>(g, q, f, kperm, lg, v, g_p, g_lnk, status, i, j, blockIdx.z);
}

// ---------------------------------------------------------------- y-march adjoint (mixed)

template <int W>
constexpr int vjp_smem_bytes() {
    using M = YMarch<float, true, false, false, W, false, true>;
    return W * (M::RING * M::NF * 32 * 4 + M::RING * 32 * 8 + M::RING * M::NW * 32 * 8);
}

template <bool DIAG, bool CRK, int W>
__global__ void __launch_bounds__(32 * W, 16 / W)
    k_vjp_ymarch(GridGeom g, PhysF q, AsmFields<float> f, AsmOut<float> o, const float* __restrict__ kperm,
                 LinkGeo lg, const float2* __restrict__ v, double* __restrict__ g_p, double* __restrict__ g_lnk,
                 int JY) {
    using M_t = YMarch<float, DIAG, CRK, false, W, false, true>;
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
    M.wv = reinterpret_cast<const double*>(v);  // 8-byte entries: the pairs (hi, lo)
    M.kperm = kperm;
    M.lg = lg;
    M.gP = g_p;
    M.gK = g_lnk;
    const int j0 = blockIdx.y * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;

    M.issue_row(j0 - 1, 0);
    M.issue_row(j0, 1);
    M.issue_row(j0 + 1, 2);
    M.wait_all_but_newest();
    YRow<float> P = M.row_cells(0);
    YRow<float> C = M.row_cells(1);
    YV vP = M.v_row(0);
    YV vC = M.v_row(1);
    float Ty_prev, Tpp_prev, Tmp_prev;
    {
        const YIn<float> Dp = M.read_in(0);
        Ty_prev = Dp.Ty;
        Tpp_prev = Dp.Tpp;
        Tmp_prev = Dp.Tmp;
    }
    YUp<float> U = M.up_links(P, C, Ty_prev, Tpp_prev, Tmp_prev);
    int s0 = 1, s1 = 2, s2 = 0;  // ring slots of rows j, j+1, j+2
    unsigned long long fix_rows = 0ull;  // rows with a zero flux, recomputed after the march

    for (int j = j0; j < j1; ++j) {
        M.issue_row(j + 2, s2);
        M.wait_all_but_newest();
        const YRow<float> N = M.row_cells(s1);
        const YV vN = M.v_row(s1);
        const YIn<float> D = M.read_in(s0);
        const F2Split vzm = M.v_at(s0, 2), vzp = M.v_at(s0, 3);
        const float kC = ring[s0 * (M_t::NF * 32) + M_t::F_K * 32 + lane];
        const int st = s0;
        s0 = s1;
        s1 = s2;
        s2 = st;
        const bool injk = zint && j > 0 && j + 1 < M.ny;
        bool fix;
        if (injk && M.xint)
            U = M.template row_vjp<2>(j, P, C, N, D, U, Ty_prev, Tpp_prev, Tmp_prev, vP, vC, vN, vzm, vzp, kC, fix);
        else if (injk)
            U = M.template row_vjp<1>(j, P, C, N, D, U, Ty_prev, Tpp_prev, Tmp_prev, vP, vC, vN, vzm, vzp, kC, fix);
        else
            U = M.template row_vjp<0>(j, P, C, N, D, U, Ty_prev, Tpp_prev, Tmp_prev, vP, vC, vN, vzm, vzp, kC, fix);
        if (fix) fix_rows |= 1ull << (j - j0);
        Ty_prev = D.Ty;
        Tpp_prev = D.Tpp;
        Tmp_prev = D.Tmp;
        P = C;
        C = N;
        vP = vC;
        vC = vN;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (fix_rows) {  // warp-uniform
        for (int b = 0; b < 64; ++b)
            if (((fix_rows >> b) & 1ull) && M.act)
                vjp_row<CRK>(g, q, f, kperm, lg, v, g_p, g_lnk, o.status, M.i, j0 + b, k);
    }
}

template <bool DIAG, bool CRK, int W>
cudaError_t launch_vjp_ymarch_w(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const float* kperm,
                                const LinkGeo& lg, const float2* v, double* g_p, double* g_lnk,
                                unsigned int* status, int JY, cudaStream_t st) {
    constexpr int smem = vjp_smem_bytes<W>();
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(&k_vjp_ymarch<DIAG, CRK, W>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + JY - 1) / JY, (g.nz + W - 1) / W);
    AsmOut<float> o{nullptr, nullptr, nullptr, status};
    k_vjp_ymarch<DIAG, CRK, W><<<grid, block, smem, st>>>(g, q, f, o, kperm, lg, v, g_p, g_lnk, JY);
    return cudaGetLastError();
}

template <bool DIAG, bool CRK>
cudaError_t launch_vjp_ymarch_t(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const float* kperm,
                                const LinkGeo& lg, const float2* v, double* g_p, double* g_lnk,
                                unsigned int* status, int JY, int W, cudaStream_t st) {
    if (W == 8) return launch_vjp_ymarch_w<DIAG, CRK, 8>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, st);
    return launch_vjp_ymarch_w<DIAG, CRK, 4>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, st);
}

// ---------------------------------------------------------------- two-cell adjoint march (mixed)

template <bool DIAG, bool CRK, int W>
__global__ void __launch_bounds__(32 * W, W == 4 ? 3 : 1)
    k_vjp_xmarch(GridGeom g, PhysF q, AsmFields<float> f, const float* __restrict__ kperm, LinkGeo lg,
                 const float2* __restrict__ v, double* __restrict__ g_p, double* __restrict__ g_lnk,
                 unsigned int* status, int JY) {
    using X = XVLayout<DIAG, CRK>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x, w = threadIdx.y;
    int bx, by, bz;
    segment_major(bx, by, bz);
    const int k = bz * W + w;
    if (k >= g.nz) return;  // warp-uniform
    XVState<DIAG, CRK, W> M(g, q, f, kperm, v, reinterpret_cast<float*>(smem) + w * X::RING * X::SLOT, lane, k, bx);
    const int j0 = by * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;
    const bool xint = M.i0 > 0 && M.i0 + 64 < g.nx;
    const bool out16 =
        ((reinterpret_cast<uintptr_t>(g_p) | reinterpret_cast<uintptr_t>(g_lnk)) & 15u) == 0;
    M.start(j0);
    unsigned long long fix_rows = 0ull;  // rows with a zero flux, recomputed after the march
    int sD = 1, sN = 2, sI = 0;          // slots of rows j, j+1 and j+2
    for (int j = j0; j < j1; ++j) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        const bool injk = zint && j > 0 && j + 1 < g.ny;
        bool fix;
        if (injk && xint) fix = M.template row<2>(j, sD, sN, sI, lg, g_p, g_lnk, out16, status);
        else if (injk) fix = M.template row<1>(j, sD, sN, sI, lg, g_p, g_lnk, out16, status);
        else fix = M.template row<0>(j, sD, sN, sI, lg, g_p, g_lnk, out16, status);
        if (fix) fix_rows |= 1ull << (j - j0);
        const int t = sD;
        sD = sN;
        sN = sI;
        sI = t;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (fix_rows) {  // warp-uniform
        for (int b = 0; b < 64; ++b)
            if (((fix_rows >> b) & 1ull) && M.act) {
                vjp_row<CRK>(g, q, f, kperm, lg, v, g_p, g_lnk, status, M.ia, j0 + b, k);
                vjp_row<CRK>(g, q, f, kperm, lg, v, g_p, g_lnk, status, M.ib, j0 + b, k);
            }
    }
}

template <bool DIAG, bool CRK, int W>
cudaError_t launch_vjp_xmarch_w(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const float* kperm,
                                const LinkGeo& lg, const float2* v, double* g_p, double* g_lnk,
                                unsigned int* status, int JY, cudaStream_t st) {
    constexpr int smem = xvjp_smem_bytes<DIAG, CRK, W>();
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(&k_vjp_xmarch<DIAG, CRK, W>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 63) / 64, (g.ny + JY - 1) / JY, (g.nz + W - 1) / W);
    k_vjp_xmarch<DIAG, CRK, W><<<grid, block, smem, st>>>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY);
    return cudaGetLastError();
}

template <bool DIAG, bool CRK>
cudaError_t launch_vjp_xmarch_t(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const float* kperm,
                                const LinkGeo& lg, const float2* v, double* g_p, double* g_lnk,
                                unsigned int* status, int JY, int W, cudaStream_t st) {
    if (W == 8) return launch_vjp_xmarch_w<DIAG, CRK, 8>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, st);
    return launch_vjp_xmarch_w<DIAG, CRK, 4>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, st);
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

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

// The cotangent as FP32 pairs: v = hi + lo with hi the truncation of v and lo
// the remainder truncated (F2Split), one pair per cell.
__global__ void k_split_pairs(const double* __restrict__ v, float2* __restrict__ out, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const F2Split t = split_f2(v[c]);
        out[c] = make_float2(t.hi, t.lo);
    }
}

cudaError_t launch_vjp_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                             const float* kperm, const LinkGeo& lg, const double* v_dbl, float2* vsplit, double* g_p,
                             double* g_lnk, unsigned int* status, int JY, int W, cudaStream_t st) {
    {
        const long long n = (long long)g.nx * g.ny * g.nz;
        const long long b = (n + 255) / 256;
        k_split_pairs<<<(unsigned)(b < (1LL << 30) ? (b > 0 ? b : 1) : (1LL << 30)), 256, 0, st>>>(v_dbl, vsplit, n);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const float2* v = vsplit;
    if (kern == AsmKernel::Naive) {
        dim3 block(32, 8, 1);
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
        if (crk) k_vjp_mixed<true><<<grid, block, 0, st>>>(g, q, f, kperm, lg, v, g_p, g_lnk, status);
        else k_vjp_mixed<false><<<grid, block, 0, st>>>(g, q, f, kperm, lg, v, g_p, g_lnk, status);
        return cudaGetLastError();
    }
    // two cells per lane: nx even, pair-aligned fields and k, 16-byte aligned m^n and pairs of v
    if (kern == AsmKernel::XMarch && xmarch_ok(g, f) && aligned(kperm, 8) && aligned(v, 16)) {
        if (g.diag)
            return crk ? launch_vjp_xmarch_t<true, true>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st)
                       : launch_vjp_xmarch_t<true, false>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st);
        return crk ? launch_vjp_xmarch_t<false, true>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st)
                   : launch_vjp_xmarch_t<false, false>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st);
    }
    if (g.diag) {
        return crk ? launch_vjp_ymarch_t<true, true>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st)
                   : launch_vjp_ymarch_t<true, false>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st);
    }
    return crk ? launch_vjp_ymarch_t<false, true>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st)
               : launch_vjp_ymarch_t<false, false>(g, q, f, kperm, lg, v, g_p, g_lnk, status, JY, W, st);
}

cudaError_t launch_vjp_fp64(const GridGeom& g, const PhysD& q, bool crk, const AsmFields<double>& f,
                            const double* kperm, const double* v, double* g_p, double* g_lnk,
                            unsigned int* status, cudaStream_t st) {
    return launch_vjp_t<double>(g, q, crk, f, kperm, v, g_p, g_lnk, status, st);
}

}  // namespace tpfa
