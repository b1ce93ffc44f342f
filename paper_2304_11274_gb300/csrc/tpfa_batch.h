// tpfa_batch.h -- ensemble (batched) assembly: the per-model table read by the
// persistent kernel, and its launch configuration.
#pragma once

#include <cuda_runtime.h>

#include "tpfa_common.cuh"

namespace tpfa {

// One model of an ensemble as the persistent kernel sees it: its grid, its
// physics, its fields and outputs, and its tiles (32-cell x-segments, runs of
// JY rows, blocks of W planes), numbered from `first`.
struct BatchModel {
    GridGeom g;
    PhysF q;
    AsmFields<float> f;
    AsmOut<float> o;
    int tx, ty, tz;
    int crk;  // c_r != 0
    long long first;
};

// Kernel and dynamic shared memory of the persistent ensemble kernel for a
// connectivity (diag), porosity law (crk) and block shape (W warps); sets the
// kernel's shared-memory limit on first use.
cudaError_t batch_kernel(bool diag, bool crk, int W, const void** func, int* smem_bytes);

// Blocks of W warps the kernel can keep resident on one SM.
cudaError_t batch_blocks_per_sm(bool diag, bool crk, int W, int* blocks);

}  // namespace tpfa
