// tpfa_assemble.cu -- residual + Jacobian assembly kernels (sm_103a).
//
// Two kernels compute the same rows (see tpfa_row.cuh for the row layout and
// summation order), so their outputs are bit-identical:
//
//   k_assemble_naive  -- one thread per cell; the cell and its 10 neighbours
//                        read from global memory, densities recomputed per
//                        neighbour as in Algorithm 1.  The correctness
//                        baseline.
//   k_assemble_ymarch -- the production kernel (tpfa_ymarch.cuh): a warp per
//                        32-cell x-segment of a z-plane marching along y,
//                        with a register window of three rows, reuse of the
//                        links into the previous row and staged 16-byte CSR
//                        stores.
//   k_assemble_ymarch_tma -- the same march with its row inputs delivered by
//                        TMA tensor copies (mixed path, nx a multiple of 4).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"
#include "tpfa_ymarch.cuh"
#include "tpfa_xmarch.cuh"

namespace tpfa {

// ------------------------------------------------------------------ naive

template <typename Real, bool CRK, bool JAC>
__global__ void __launch_bounds__(256) k_assemble_naive(GridGeom g, typename PhysOf<Real>::type q,
                                                        AsmFields<Real> f, AsmOut<Real> o) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    naive_row<Real, CRK, JAC>(g, q, f, o, i < g.nx && j < g.ny, i, j, blockIdx.z);
}

// ------------------------------------------------------------------ launchers

template <typename Real, bool CRK, bool JAC>
static cudaError_t launch_naive_t(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                  const AsmFields<Real>& f, const AsmOut<Real>& o, cudaStream_t st) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    k_assemble_naive<Real, CRK, JAC><<<grid, block, 0, st>>>(g, q, f, o);
    return cudaGetLastError();
}

// Planes [k0, k1) of the grid; the whole grid by default.
template <typename Real, bool DIAG, bool CRK, bool JAC, int W>
static cudaError_t launch_ymarch_w(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                   const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int k0, int k1,
                                   cudaStream_t st) {
    constexpr int smem = ymarch_smem_bytes<Real, W>();
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(&k_assemble_ymarch<Real, DIAG, CRK, JAC, W>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + JY - 1) / JY, (k1 - k0 + W - 1) / W);
    k_assemble_ymarch<Real, DIAG, CRK, JAC, W><<<grid, block, smem, st>>>(g, q, f, o, JY, k0, k1);
    return cudaGetLastError();
}

template <typename Real, bool DIAG, bool CRK, bool JAC>
static cudaError_t launch_ymarch_t(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                   const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int W, int k0,
                                   int k1, cudaStream_t st) {
    if (W == 8) return launch_ymarch_w<Real, DIAG, CRK, JAC, 8>(g, q, f, o, JY, k0, k1, st);
    return launch_ymarch_w<Real, DIAG, CRK, JAC, 4>(g, q, f, o, JY, k0, k1, st);
}

// ------------------------------------------------------------------ two cells per lane

template <bool DIAG, bool CRK, int W, bool FAST>
static cudaError_t launch_xmarch_f(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                   const AsmOut<float>& o, int JY, int k0, int k1, cudaStream_t st) {
    constexpr int smem = xmarch_smem_bytes<DIAG, CRK, W>();
    const cudaError_t e =
        ensure_smem_limit(reinterpret_cast<const void*>(&k_assemble_xmarch<DIAG, CRK, W, FAST>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 63) / 64, (g.ny + JY - 1) / JY, (k1 - k0 + W - 1) / W);
    k_assemble_xmarch<DIAG, CRK, W, FAST><<<grid, block, smem, st>>>(g, q, f, o, JY, k0, k1);
    return cudaGetLastError();
}

// FAST: R and diag64 given, and R, diag64 and vals 16-byte aligned.
template <bool DIAG, bool CRK, int W>
static cudaError_t launch_xmarch_w(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                   const AsmOut<float>& o, int JY, int k0, int k1, cudaStream_t st) {
    const bool fast = o.R && o.diag64 &&
                      ((reinterpret_cast<uintptr_t>(o.R) | reinterpret_cast<uintptr_t>(o.diag64) |
                        reinterpret_cast<uintptr_t>(o.vals)) & 15u) == 0;
    if (fast) return launch_xmarch_f<DIAG, CRK, W, true>(g, q, f, o, JY, k0, k1, st);
    return launch_xmarch_f<DIAG, CRK, W, false>(g, q, f, o, JY, k0, k1, st);
}

template <bool DIAG, bool CRK>
static cudaError_t launch_xmarch_t(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                   const AsmOut<float>& o, int JY, int W, int k0, int k1, cudaStream_t st) {
    if (W == 8) return launch_xmarch_w<DIAG, CRK, 8>(g, q, f, o, JY, k0, k1, st);
    return launch_xmarch_w<DIAG, CRK, 4>(g, q, f, o, JY, k0, k1, st);
}

static bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// The two-cell march needs nx even and pair-aligned fields.
bool xmarch_ok(const GridGeom& g, const AsmFields<float>& f) {
    return g.nx % 2 == 0 && aligned_to(f.p, 8) && aligned_to(f.pn, 8) && aligned_to(f.z, 8) &&
           aligned_to(f.phi0, 8) && aligned_to(f.Tx, 8) && aligned_to(f.Ty, 8) && aligned_to(f.Tz, 8) &&
           aligned_to(f.Tpp, 8) && aligned_to(f.Tmp, 8) && aligned_to(f.mn, 16);
}

template <typename Real>
static cudaError_t dispatch(AsmKernel kern, const GridGeom& g, const typename PhysOf<Real>::type& q,
                            bool crk, const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int W, int k0,
                            int k1, cudaStream_t st) {
    const bool jac = o.vals != nullptr;
    if (k1 < 0 || k1 > g.nz) k1 = g.nz;
    if (k0 < 0 || k0 >= k1) k0 = 0;
    if (kern == AsmKernel::Naive) {
        if (crk) return jac ? launch_naive_t<Real, true, true>(g, q, f, o, st) : launch_naive_t<Real, true, false>(g, q, f, o, st);
        return jac ? launch_naive_t<Real, false, true>(g, q, f, o, st) : launch_naive_t<Real, false, false>(g, q, f, o, st);
    }
    if constexpr (sizeof(Real) == 4) {
        // two cells per lane: the mixed path's fused R + J on grids with nx even
        // and pair-aligned fields; otherwise (and for residual-only calls) the
        // one-cell march
        if (kern == AsmKernel::XMarch && jac && xmarch_ok(g, f)) {
            if (g.diag) return crk ? launch_xmarch_t<true, true>(g, q, f, o, JY, W, k0, k1, st)
                                   : launch_xmarch_t<true, false>(g, q, f, o, JY, W, k0, k1, st);
            return crk ? launch_xmarch_t<false, true>(g, q, f, o, JY, W, k0, k1, st)
                       : launch_xmarch_t<false, false>(g, q, f, o, JY, W, k0, k1, st);
        }
    }
    if (g.diag) {
        if (crk) return jac ? launch_ymarch_t<Real, true, true, true>(g, q, f, o, JY, W, k0, k1, st)
                            : launch_ymarch_t<Real, true, true, false>(g, q, f, o, JY, W, k0, k1, st);
        return jac ? launch_ymarch_t<Real, true, false, true>(g, q, f, o, JY, W, k0, k1, st)
                   : launch_ymarch_t<Real, true, false, false>(g, q, f, o, JY, W, k0, k1, st);
    }
    if (crk) return jac ? launch_ymarch_t<Real, false, true, true>(g, q, f, o, JY, W, k0, k1, st)
                        : launch_ymarch_t<Real, false, true, false>(g, q, f, o, JY, W, k0, k1, st);
    return jac ? launch_ymarch_t<Real, false, false, true>(g, q, f, o, JY, W, k0, k1, st)
               : launch_ymarch_t<Real, false, false, false>(g, q, f, o, JY, W, k0, k1, st);
}

// ------------------------------------------------------------------ TMA march

// The TMA march runs 4 warps per block (4 x-segments: its halo boxes of
// 136 cells stay within the copy engine's 256-element box limit), whatever
// the tiling's warps per block.
constexpr int kTmaWarps = 4;

template <bool DIAG, bool CRK, bool JAC>
static cudaError_t launch_tma_t(const GridGeom& g, const PhysF& q, const AsmFields<float>& f, const AsmOut<float>& o,
                                const TmaMaps& maps, int JY, int k0, int k1, cudaStream_t st) {
    constexpr int W = kTmaWarps;
    constexpr int smem = ymarch_tma_smem_bytes<W, YMarch<float, DIAG, CRK, JAC, W>::TRING>();
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(&k_assemble_ymarch_tma<DIAG, CRK, JAC, W>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 32 * W - 1) / (32 * W), (g.ny + JY - 1) / JY, k1 - k0);
    k_assemble_ymarch_tma<DIAG, CRK, JAC, W><<<grid, block, smem, st>>>(g, q, f, o, maps, JY, k0);
    return cudaGetLastError();
}

cudaError_t launch_assemble_mixed_tma(const GridGeom& g, const PhysF& q, bool crk, const AsmFields<float>& f,
                                      const AsmOut<float>& o, const TmaMaps& maps, int JY, int W, cudaStream_t st,
                                      int k0, int k1) {
    const bool jac = o.vals != nullptr;
    if (k1 < 0 || k1 > g.nz) k1 = g.nz;
    if (k0 < 0 || k0 >= k1) k0 = 0;
    if (g.diag) {
        if (crk) return jac ? launch_tma_t<true, true, true>(g, q, f, o, maps, JY, k0, k1, st)
                            : launch_tma_t<true, true, false>(g, q, f, o, maps, JY, k0, k1, st);
        return jac ? launch_tma_t<true, false, true>(g, q, f, o, maps, JY, k0, k1, st)
                   : launch_tma_t<true, false, false>(g, q, f, o, maps, JY, k0, k1, st);
    }
    if (crk) return jac ? launch_tma_t<false, true, true>(g, q, f, o, maps, JY, k0, k1, st)
                        : launch_tma_t<false, true, false>(g, q, f, o, maps, JY, k0, k1, st);
    return jac ? launch_tma_t<false, false, true>(g, q, f, o, maps, JY, k0, k1, st)
               : launch_tma_t<false, false, false>(g, q, f, o, maps, JY, k0, k1, st);
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiled encoder() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// One (nx, ny, nz) field with a box of (bx, 1, bz) elements; out-of-range
// elements of a box read as zero.
bool encode_field(CUtensorMap* m, const GridGeom& g, const void* base, bool fp64, unsigned bx, unsigned bz) {
    EncodeTiled fn = encoder();
    if (!fn || !base || !aligned16(base)) return false;
    const cuuint64_t es = fp64 ? 8 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * (cuuint64_t)g.ny * es};
    const cuuint32_t box[3] = {bx, 1u, bz};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tma_grid_ok(const GridGeom& g) { return g.nx % 4 == 0 && encoder() != nullptr; }

bool tma_encode_state(TmaMaps* m, const GridGeom& g, const float* p, const float* pn) {
    using TS = TmaSlot<kTmaWarps>;
    if (!tma_grid_ok(g)) return false;
    return encode_field(&m->p, g, p, false, TS::HX, 3) && encode_field(&m->pn, g, pn, false, TS::SX, 1);
}

bool tma_encode_static(TmaMaps* m, const GridGeom& g, const AsmFields<float>& f, bool crk) {
    using TS = TmaSlot<kTmaWarps>;
    if (!tma_grid_ok(g)) return false;
    bool ok = encode_field(&m->z, g, f.z, false, TS::HX, 3) && encode_field(&m->Tx, g, f.Tx, false, TS::HX, 1) &&
              encode_field(&m->Ty, g, f.Ty, false, TS::SX, 1) && encode_field(&m->Tz, g, f.Tz, false, TS::SX, 2) &&
              encode_field(&m->Tpp, g, f.Tpp, false, TS::HX, 1) && encode_field(&m->Tmp, g, f.Tmp, false, TS::HX, 1) &&
              encode_field(&m->mn, g, f.mn, true, TS::SX, 1);
    // phi0 is read only when c_r != 0; otherwise its map aliases z's
    ok = ok && encode_field(&m->phi, g, crk ? (const void*)f.phi0 : (const void*)f.z, false, TS::SX, 1);
    return ok;
}

cudaError_t launch_assemble_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk,
                                  const AsmFields<float>& f, const AsmOut<float>& o, int JY, int W,
                                  cudaStream_t st, int k0, int k1) {
    return dispatch<float>(kern, g, q, crk, f, o, JY, W, k0, k1, st);
}

cudaError_t launch_assemble_fp64(AsmKernel kern, const GridGeom& g, const PhysD& q, bool crk,
                                 const AsmFields<double>& f, const AsmOut<double>& o, int JY, int W,
                                 cudaStream_t st, int k0, int k1) {
    return dispatch<double>(kern, g, q, crk, f, o, JY, W, k0, k1, st);
}

}  // namespace tpfa
