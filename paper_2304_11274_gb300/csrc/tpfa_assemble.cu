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
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"
#include "tpfa_ymarch.cuh"

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

// Planes [k0, k1) of the grid (k0 a multiple of W); the whole grid by default.
template <typename Real, bool DIAG, bool CRK, bool JAC, int W>
static cudaError_t launch_ymarch_w(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                   const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int k0, int k1,
                                   cudaStream_t st) {
    constexpr int smem = ymarch_smem_bytes<Real, W>();
    static bool attr_set = false;  // per instantiation; the attribute is per function
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_assemble_ymarch<Real, DIAG, CRK, JAC, W>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + JY - 1) / JY, (k1 - k0 + W - 1) / W);
    k_assemble_ymarch<Real, DIAG, CRK, JAC, W><<<grid, block, smem, st>>>(g, q, f, o, JY, k0 / W);
    return cudaGetLastError();
}

template <typename Real, bool DIAG, bool CRK, bool JAC>
static cudaError_t launch_ymarch_t(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                   const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int W, int k0,
                                   int k1, cudaStream_t st) {
    if (W == 8) return launch_ymarch_w<Real, DIAG, CRK, JAC, 8>(g, q, f, o, JY, k0, k1, st);
    return launch_ymarch_w<Real, DIAG, CRK, JAC, 4>(g, q, f, o, JY, k0, k1, st);
}

template <typename Real>
static cudaError_t dispatch(AsmKernel kern, const GridGeom& g, const typename PhysOf<Real>::type& q,
                            bool crk, const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int W, int k0,
                            int k1, cudaStream_t st) {
    const bool jac = o.vals != nullptr;
    if (k1 < 0 || k1 > g.nz) k1 = g.nz;
    if (k0 < 0 || k0 % W != 0 || k0 >= k1) k0 = 0;  // only W-aligned plane ranges are split
    if (kern == AsmKernel::Naive) {
        if (crk) return jac ? launch_naive_t<Real, true, true>(g, q, f, o, st) : launch_naive_t<Real, true, false>(g, q, f, o, st);
        return jac ? launch_naive_t<Real, false, true>(g, q, f, o, st) : launch_naive_t<Real, false, false>(g, q, f, o, st);
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
