// tpfa_tma.cuh -- tensor-memory-accelerator (TMA) row loads for the
// y-marching assembly (sm_103a).
//
// A block's warps own consecutive 32-cell x-segments of one z-plane and
// march along y together.  Per step the march needs one y-row of every input
// over the block's x-range, plus its x-halo cells and the vertical
// neighbours: a few boxes of 3-D fields (x fastest).  p and depth span 3
// planes (k - 1, k, k + 1) and 4 extra cells on each side (so the halo cells
// are inside and the box starts on a 16-byte boundary); Tz spans 2 planes
// (k - 1, k); the other fields one plane.  One thread requests every box of
// a row with cp.async.bulk.tensor into a block-wide ring slot and arms the
// slot's "full" mbarrier with the byte count; every warp waits on that phase
// before reading the slot and arrives on the slot's "empty" mbarrier when it
// is done with it, which the requesting thread waits for before refilling
// it.  Boxes that reach outside the grid are zero-filled by the copy engine,
// exactly the "missing value = 0" convention of the per-lane path.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace tpfa {

// Tensor maps of the mixed path's fields (FP32; m^n FP64), each a 3-D
// (nx, ny, nz) array.  Passed to the kernel as a __grid_constant__ parameter.
struct TmaMaps {
    CUtensorMap p, z, Tx, Ty, Tz, Tpp, Tmp, pn, phi, mn;
};

// One ring slot of a block whose SEG warps own SEG consecutive 32-cell
// x-segments (cells X0 .. X0 + 32 SEG - 1) of one z-plane: the boxes of one
// y-row, each starting on a 128-byte boundary.  Boxes that carry the x-halo
// span X0 - 4 .. X0 + 32 SEG + 3 (HX elements), the others X0 .. (SX).
template <int SEG>
struct TmaSlot {
    static constexpr int SX = 32 * SEG, HX = SX + 8;
    static constexpr int up128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int P = 0;                              // p: planes k-1, k, k+1 (HX each)
    static constexpr int Z = P + up128(3 * HX * 4);          // depth: 3 planes
    static constexpr int TX = Z + up128(3 * HX * 4);         // Tx: HX
    static constexpr int TY = TX + up128(HX * 4);            // Ty: SX
    static constexpr int TZ = TY + up128(SX * 4);            // Tz: planes k-1, k (SX each)
    static constexpr int TPP = TZ + up128(2 * SX * 4);       // T(+x,+y): HX
    static constexpr int TMP = TPP + up128(HX * 4);          // T(-x,+y): HX
    static constexpr int PN = TMP + up128(HX * 4);           // p^n: SX
    static constexpr int PHI = PN + up128(SX * 4);           // phi0: SX
    static constexpr int MN = PHI + up128(SX * 4);           // m^n: SX doubles
    static constexpr int BYTES = MN + up128(SX * 8);
    // bytes one row delivers (the full barrier's transaction count)
    static constexpr unsigned tx_bytes(bool diag, bool crk) {
        return (unsigned)(4 * (6 * HX + HX + SX + 2 * SX + (diag ? 2 * HX : 0) + SX + (crk ? SX : 0)) + 8 * SX);
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One probe of the phase with parity `par` (true once it completed); the
// thread may be suspended for at most about 20 us while it waits.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(par), "r"(20000u)
        : "memory");
    return ok != 0u;
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy ones (a slot's readers before its refill).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Probe limit of a barrier wait (about 5 s at the suspend hint); past it the
// kernel reports STATUS_TIMEOUT and stops instead of hanging.
constexpr int kTmaWaitLimit = 1 << 18;

// Bounded wait for the phase with parity `par` of the mbarrier at `bar`.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, unsigned par) {
    bool ok = mbar_try_wait(bar, par);
    for (int n = 1; !ok && n < kTmaWaitLimit; ++n) ok = mbar_try_wait(bar, par);
    return ok;
}

}  // namespace tpfa
