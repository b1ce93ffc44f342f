// tpfa_batch.cu -- persistent assembly of an ensemble of grids (sm_103a).
//
// An ensemble of geomodels of uneven sizes (for uncertainty sweeps) is
// assembled by one launch of a persistent kernel: one block per resident slot
// (SM count x blocks per SM), each block repeatedly claims the next tile from
// a global ticket, finds its model by binary search over the models' first
// tile numbers, copies that model's descriptor into shared memory and runs the
// same per-tile code as the single-grid kernel (ymarch_tile).  Rows therefore
// come out bit-identical to a single-grid launch of each model.  The host side
// (tpfa_api.cu) captures the ticket reset and this kernel in a CUDA graph.
#include <cuda_runtime.h>

#include "tpfa_batch.h"
#include "tpfa_impl.h"
#include "tpfa_ymarch.cuh"

namespace tpfa {

namespace {

template <bool DIAG, bool CRK, int W>
__global__ void __launch_bounds__(32 * W, 16 / W)
    k_assemble_batch(const BatchModel* __restrict__ models, int M, long long total, int JY,
                     unsigned long long* ticket) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchModel sm;
    __shared__ long long s_tile;
    __shared__ int s_bx, s_by, s_bz;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (;;) {
        if (tid == 0) {
            const long long t = (long long)atomicAdd(ticket, 1ULL);
            s_tile = t;
            if (t < total) {
                int lo = 0, hi = M - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (models[mid].first <= t) lo = mid;
                    else hi = mid - 1;
                }
                sm = models[lo];
                long long r = t - sm.first;
                s_bx = (int)(r % sm.tx);
                r /= sm.tx;
                s_by = (int)(r % sm.ty);
                s_bz = (int)(r / sm.ty);
            }
        }
        __syncthreads();
        if (s_tile >= total) break;
        ymarch_tile<float, DIAG, CRK, true, W, true>(sm.g, sm.q, sm.f, sm.o, JY, s_bx, s_by, s_bz, smem);
        __syncthreads();  // every warp is done with this tile's descriptor and buffers
    }
}

template <bool DIAG, bool CRK, int W>
cudaError_t config(const void** func, int* smem_bytes) {
    constexpr int smem = ymarch_smem_bytes<float, W>();
    const void* f = reinterpret_cast<const void*>(&k_assemble_batch<DIAG, CRK, W>);
    const cudaError_t e = ensure_smem_limit(f, smem);
    if (e != cudaSuccess) return e;
    *func = f;
    *smem_bytes = smem;
    return cudaSuccess;
}

}  // namespace

cudaError_t batch_kernel(bool diag, bool crk, int W, const void** func, int* smem_bytes) {
    if (W == 4) {
        if (diag) return crk ? config<true, true, 4>(func, smem_bytes) : config<true, false, 4>(func, smem_bytes);
        return crk ? config<false, true, 4>(func, smem_bytes) : config<false, false, 4>(func, smem_bytes);
    }
    if (W == 8) {
        if (diag) return crk ? config<true, true, 8>(func, smem_bytes) : config<true, false, 8>(func, smem_bytes);
        return crk ? config<false, true, 8>(func, smem_bytes) : config<false, false, 8>(func, smem_bytes);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_blocks_per_sm(bool diag, bool crk, int W, int* blocks) {
    const void* f = nullptr;
    int smem = 0;
    cudaError_t e = batch_kernel(diag, crk, W, &f, &smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, 32 * W, smem);
}

}  // namespace tpfa
