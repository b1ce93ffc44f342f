// tpfa_krylov.cu -- preconditioned BiCGStab on the assembled Jacobian (the
// linear solve of a Newton step on Eq. vk), sm_103a.
//
// BiCGStab (van der Vorst, 1992) with right preconditioning by M, the
// tridiagonal part of J along z (default) or its diagonal (Jacobi):
//   r = b, r^ = b, x = 0, rho = (r^, r)
//   repeat:  p = r + beta (p - omega v)            (p = r on the first pass)
//            p^ = M^-1 p,  v = J p^,  alpha = rho / (r^, v)
//            s = r - alpha v,  s^ = M^-1 s,  t = J s^,  omega = (t, s) / (t, t)
//            x += alpha p^ + omega s^,  r = s - omega t
//            rho' = (r^, r),  beta = (rho' / rho)(alpha / omega),  rho = rho'
//   until ||r||_2 <= rtol ||b||_2.
// Every scalar lives in a device-side KrylovScalars record: each dot product
// is reduced per block into a partial-sum array and summed in a fixed order
// by a one-block finalize kernel that also updates the scalars, so results
// are deterministic and the host only polls the record.  Once `done` is set
// every kernel returns at entry, so the host may enqueue several iterations
// between polls.
//
// The matrix-vector product walks the structured stencil: row (i, j, k)
// starts at the closed-form offset of the pattern and its columns follow the
// slot order, so neither row_ptr nor col_idx is read.  FP64 path: products
// and sums in FP64.  Mixed path: the FP32 off-diagonal values times the
// vector split into FP32 pairs (written by the update kernels), exact
// two-float products summed as a double-float, plus the FP64 diagonal times
// the FP64 vector.
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"

namespace tpfa {

namespace {

constexpr int kVecThreads = 256;
constexpr int kFinThreads = 1024;

__device__ __forceinline__ double as_f64(float x) { return widen(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }

// Sum of d0 (and d1) over the block, written by thread 0 to part[2 b], part[2 b + 1].
__device__ __forceinline__ void block_partials(double d0, double d1, double* part, long long b) {
    __shared__ double sh[2][32];
    const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
    }
    if ((t & 31) == 0) {
        sh[0][t >> 5] = d0;
        sh[1][t >> 5] = d1;
    }
    __syncthreads();
    if (t < 32) {
        const int nw = nt >> 5;
        d0 = t < nw ? sh[0][t] : 0.0;
        d1 = t < nw ? sh[1][t] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d0 += __shfl_down_sync(0xffffffffu, d0, o);
            d1 += __shfl_down_sync(0xffffffffu, d1, o);
        }
        if (t == 0) {
            part[2 * b] = d0;
            part[2 * b + 1] = d1;
        }
    }
}

// FP64 path: y = J x over the stencil in FP64; partials of (a, y) and (y, y).
__global__ void __launch_bounds__(256) k_spmv(GridGeom g, const double* __restrict__ vals, const double* __restrict__ x,
                                              double* __restrict__ y, const double* __restrict__ a, double* part,
                                              const KrylovScalars* S) {
    if (S->done) return;  // uniform over the grid
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    double d0 = 0.0, d1 = 0.0;
    if (i < g.nx && j < g.ny) {
        const int nx = g.nx, nxy = nx * g.ny;
        const int c = i + nx * j + nxy * k;
        const unsigned mask = slot_mask(g, i, j, k);
        const int off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
        const double* row = vals + row_start(g, i, j, k);
        double acc = 0.0;
        int pos = 0;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (!(mask & (1u << s))) continue;
            acc = fma(row[pos], x[c + off[s]], acc);
            ++pos;
        }
        y[c] = acc;
        d0 = a[c] * acc;
        d1 = acc * acc;
    }
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_partials(d0, d1, part, b);
}

// Mixed path: y = J x with x given as split pairs x = hi + lo (FP32) and the
// FP32 off-diagonals a: each a hi is formed exactly as p + e (e = fma(a, hi,
// -p)), a lo is added to e, and the terms are summed as a double-float
// (TwoSum on the leading parts, the trailing parts summed apart), about 48
// bits; the FP64 diagonal times the FP64 x is added in FP64.  Three FP64
// operations per row instead of eleven, the product as accurate as an FP64
// one for the Krylov iteration.
__global__ void __launch_bounds__(256) k_spmv_mixed(GridGeom g, const float* __restrict__ vals,
                                                    const double* __restrict__ diag64, const double* __restrict__ x,
                                                    const float* __restrict__ xhi, const float* __restrict__ xlo,
                                                    double* __restrict__ y, const double* __restrict__ a, double* part,
                                                    const KrylovScalars* S) {
    if (S->done) return;  // uniform over the grid
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    double d0 = 0.0, d1 = 0.0;
    if (i < g.nx && j < g.ny) {
        const int nx = g.nx, nxy = nx * g.ny;
        const int c = i + nx * j + nxy * k;
        const unsigned mask = slot_mask(g, i, j, k);
        const int off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
        const float* row = vals + row_start(g, i, j, k);
        float ah = 0.f, al = 0.f;
        int pos = 0;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (!(mask & (1u << s))) continue;
            if (s != SLOT_SELF) {
                const float av = row[pos], xh = xhi[c + off[s]], xl = xlo[c + off[s]];
                const float p = __fmul_rn(av, xh);
                const float t = __fmaf_rn(av, xl, __fmaf_rn(av, xh, -p));
                const float sum = __fadd_rn(ah, p);
                const float bb = __fsub_rn(sum, ah);
                const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
                ah = sum;
                al = __fadd_rn(al, __fadd_rn(err, t));
            }
            ++pos;
        }
        const double yc = __fma_rn(diag64[c], x[c], __dadd_rn(widen(ah), widen(al)));
        y[c] = yc;
        d0 = a[c] * yc;
        d1 = yc * yc;
    }
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_partials(d0, d1, part, b);
}

// M^-1 = 1 / diag(J) (1 where the diagonal is zero).
template <typename Real, bool MIXED>
__global__ void __launch_bounds__(256) k_dinv(GridGeom g, const Real* __restrict__ vals,
                                              const double* __restrict__ diag64, double* __restrict__ dinv) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int c = i + g.nx * (j + g.ny * k);
    double d;
    if (MIXED) {
        d = diag64[c];
    } else {
        const unsigned mask = slot_mask(g, i, j, k);
        d = as_f64(vals[row_start(g, i, j, k) + slot_pos(mask, SLOT_SELF)]);
    }
    dinv[c] = d != 0.0 ? 1.0 / d : 1.0;
}

// ---------------------------------------------------------------- z-line preconditioner
//
// M = the tridiagonal part of J along z (each cell's diagonal and its two
// vertical couplings), inverted exactly column by column with the Thomas
// algorithm: the vertical links of 10 x 10 x 2 m cells carry 25 times the
// transmissibility of the horizontal ones, so M captures most of J.  The
// factorisation (once per solve) stores three coalesced per-cell arrays:
// the elimination multiplier l_k = sub_k / b'_{k-1}, the super-diagonal
// u_k and the inverse pivot 1 / b'_k.  An application is one thread per
// (i, j) column, a forward sweep y_k = in_k - l_k y_{k-1} and a backward
// sweep z_k = (y_k - u_k z_{k+1}) / b'_k.  The columns are few (nx ny
// threads) and each sweep is a chain of dependent steps, so the bandwidth
// comes from loads in flight: every thread keeps its next kLineDepth steps'
// operands on the way into a shared-memory ring (8-byte cp.async per value,
// one commit group per step), one warp per block so that the 512 warps of a
// 128 x 128 grid spread evenly over the multiprocessors.

constexpr int kLineThreads = 64;  // the factorisation
constexpr int kApplyThreads = 32;  // the application: one warp per block
constexpr int kLineDepth = 16;     // steps in flight per column

template <typename Real, bool MIXED>
__global__ void __launch_bounds__(kLineThreads) k_line_factor(GridGeom g, const Real* __restrict__ vals,
                                                              const double* __restrict__ diag64,
                                                              double* __restrict__ inv_b, double* __restrict__ lmul,
                                                              double* __restrict__ up) {
    const long long nxy = (long long)g.nx * g.ny;
    const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (col >= nxy) return;
    const int i = (int)(col % g.nx), j = (int)(col / g.nx);
    double inv_prev = 0.0, sup_prev = 0.0;
    for (int k = 0; k < g.nz; ++k) {
        const long long c = col + nxy * k;
        const long long rs = row_start(g, i, j, k);
        const unsigned mask = slot_mask(g, i, j, k);
        const double diag = MIXED ? diag64[c] : as_f64(vals[rs + slot_pos(mask, SLOT_SELF)]);
        double b = diag, l = 0.0;
        if (k > 0) {
            l = as_f64(vals[rs]) * inv_prev;
            b = fma(-l, sup_prev, diag);
        }
        const double inv = b != 0.0 ? 1.0 / b : 1.0;
        const double sup = k + 1 < g.nz ? as_f64(vals[rs + __popc(mask) - 1]) : 0.0;
        inv_b[c] = inv;
        lmul[c] = l;
        up[c] = sup;
        sup_prev = sup;
        inv_prev = inv;
    }
}

__device__ __forceinline__ void cp8_async(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// out = M^-1 in; on the mixed path also out split into FP32 pairs.  Each
// lane copies and reads back only its own ring entries.  A step's slot is
// refilled only after the step's result has been computed from it (in-order
// issue puts the reads first).
__global__ void __launch_bounds__(kApplyThreads) k_line_apply(GridGeom g, const double* __restrict__ inv_b,
                                                              const double* __restrict__ lmul,
                                                              const double* __restrict__ up,
                                                              const double* __restrict__ in, double* __restrict__ out,
                                                              float* __restrict__ hi, float* __restrict__ lo,
                                                              const KrylovScalars* S) {
    __shared__ __align__(16) double ring[kLineDepth][3][kApplyThreads];
    if (S->done) return;
    const long long nxy = (long long)g.nx * g.ny;
    const long long col = blockIdx.x * (long long)kApplyThreads + threadIdx.x;
    if (col >= nxy) return;
    const int nz = g.nz, l = threadIdx.x;
    // forward: y_k = in_k - l_k y_{k-1}
    auto issue_f = [&](int k) {
        if (k < nz) {
            const long long c = col + nxy * k;
            cp8_async(&ring[k % kLineDepth][0][l], in + c);
            cp8_async(&ring[k % kLineDepth][1][l], lmul + c);
        }
        cp_commit();
    };
    for (int k = 0; k < kLineDepth; ++k) issue_f(k);
    double y = 0.0;
    for (int k = 0; k < nz; ++k) {
        cp_wait<kLineDepth - 1>();
        const int sl = k % kLineDepth;
        y = fma(-ring[sl][1][l], y, ring[sl][0][l]);
        out[col + nxy * k] = y;
        issue_f(k + kLineDepth);
    }
    cp_wait<0>();
    __threadfence_block();  // y stored above is read back below by this thread
    // back: z_k = (y_k - u_k z_{k+1}) / b'_k, steps k = nz-1 down to 0
    auto issue_b = [&](int q) {
        const int k = nz - 1 - q;
        if (k >= 0) {
            const long long c = col + nxy * k;
            cp8_async(&ring[q % kLineDepth][0][l], out + c);
            cp8_async(&ring[q % kLineDepth][1][l], up + c);
            cp8_async(&ring[q % kLineDepth][2][l], inv_b + c);
        }
        cp_commit();
    };
    for (int q = 0; q < kLineDepth; ++q) issue_b(q);
    double z = 0.0;
    for (int q = 0; q < nz; ++q) {
        cp_wait<kLineDepth - 1>();
        const int sl = q % kLineDepth;
        z = fma(-ring[sl][1][l], z, ring[sl][0][l]) * ring[sl][2][l];
        const long long c = col + nxy * (nz - 1 - q);
        out[c] = z;
        if (hi) {
            const F2Split sp = split_f2(z);
            hi[c] = sp.hi;
            lo[c] = sp.lo;
        }
        issue_b(q + kLineDepth);
    }
    cp_wait<0>();
}

// x = 0, r = r^ = sign * b; partials of (b, b).
__global__ void __launch_bounds__(kVecThreads) k_init(long long n, const double* __restrict__ b, double sign,
                                                      double* __restrict__ x, double* __restrict__ r,
                                                      double* __restrict__ rh, double* part) {
    double d0 = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double bc = sign * b[c];
        x[c] = 0.0;
        r[c] = bc;
        rh[c] = bc;
        d0 = fma(bc, bc, d0);
    }
    block_partials(d0, 0.0, part, blockIdx.x);
}

// p = r + beta (p - omega v) (p = r on the first pass), p^ = M^-1 p.
__global__ void __launch_bounds__(kVecThreads) k_update_p(long long n, const double* __restrict__ r,
                                                          const double* __restrict__ v, double* __restrict__ p,
                                                          double* __restrict__ ph, float* __restrict__ phh,
                                                          float* __restrict__ phl, const double* __restrict__ dinv,
                                                          const KrylovScalars* S) {
    if (S->done) return;
    const bool first = S->iter == 0;
    const double beta = S->beta, omega = S->omega;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double pc = first ? r[c] : fma(beta, fma(-omega, v[c], p[c]), r[c]);
        p[c] = pc;
        if (!dinv) continue;  // the line preconditioner writes p^
        const double phc = pc * dinv[c];
        ph[c] = phc;
        if (phh) {
            const F2Split sp = split_f2(phc);
            phh[c] = sp.hi;
            phl[c] = sp.lo;
        }
    }
}

// s = r - alpha v, s^ = M^-1 s.
__global__ void __launch_bounds__(kVecThreads) k_update_s(long long n, const double* __restrict__ r,
                                                          const double* __restrict__ v, double* __restrict__ s,
                                                          double* __restrict__ sh, float* __restrict__ shh,
                                                          float* __restrict__ shl, const double* __restrict__ dinv,
                                                          const KrylovScalars* S) {
    if (S->done) return;
    const double alpha = S->alpha;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double sc = fma(-alpha, v[c], r[c]);
        s[c] = sc;
        if (!dinv) continue;  // the line preconditioner writes s^
        const double shc = sc * dinv[c];
        sh[c] = shc;
        if (shh) {
            const F2Split sp = split_f2(shc);
            shh[c] = sp.hi;
            shl[c] = sp.lo;
        }
    }
}

// x += alpha p^ + omega s^, r = s - omega t; partials of (r^, r) and (r, r).
__global__ void __launch_bounds__(kVecThreads) k_update_xr(long long n, double* __restrict__ x,
                                                           const double* __restrict__ ph, const double* __restrict__ sh,
                                                           const double* __restrict__ s, const double* __restrict__ t,
                                                           double* __restrict__ r, const double* __restrict__ rh,
                                                           double* part, const KrylovScalars* S) {
    if (S->done) return;
    const double alpha = S->alpha, omega = S->omega;
    double d0 = 0.0, d1 = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        x[c] = fma(omega, sh[c], fma(alpha, ph[c], x[c]));
        const double rc = fma(-omega, t[c], s[c]);
        r[c] = rc;
        d0 = fma(rh[c], rc, d0);
        d1 = fma(rc, rc, d1);
    }
    block_partials(d0, d1, part, blockIdx.x);
}

__device__ __forceinline__ bool finite(double x) { return !nonfinite(x); }

// Sum the partials in a fixed order and advance the scalars.  stage 0:
// after k_init; 1: after v = J p^; 2: after t = J s^; 3: after k_update_xr.
__global__ void __launch_bounds__(kFinThreads) k_finalize(const double* part, long long nb, int stage,
                                                          KrylovScalars* S) {
    if (stage != 0 && S->done) return;
    __shared__ double sh[2][kFinThreads / 32];
    const int t = threadIdx.x;
    double d0 = 0.0, d1 = 0.0;
    for (long long b = t; b < nb; b += kFinThreads) {
        d0 += part[2 * b];
        d1 += part[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
    }
    if ((t & 31) == 0) {
        sh[0][t >> 5] = d0;
        sh[1][t >> 5] = d1;
    }
    __syncthreads();
    if (t != 0) return;
    d0 = 0.0;
    d1 = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) {
        d0 += sh[0][w];
        d1 += sh[1][w];
    }
    switch (stage) {
        case 0:  // rho = (r^, r) = (b, b)
            S->bb = d0;
            S->rho = d0;
            S->rr = d0;
            S->iter = 0;
            S->breakdown = 0;
            S->alpha = S->omega = 1.0;
            S->beta = 0.0;
            S->done = (d0 == 0.0) ? 1 : 0;  // b = 0: x = 0 is exact
            if (!finite(d0)) S->done = S->breakdown = 1;
            break;
        case 1:  // alpha = rho / (r^, v)
            if (d0 == 0.0 || !finite(d0)) {
                S->done = S->breakdown = 1;
            } else {
                S->alpha = S->rho / d0;
            }
            break;
        case 2:  // omega = (t, s) / (t, t); t = 0 means s = 0: the half step solved it
            S->omega = (d1 > 0.0 && finite(d1) && finite(d0)) ? d0 / d1 : 0.0;
            break;
        default: {  // rho' = (r^, r), rr = (r, r)
            S->iter += 1;
            S->rr = d1;
            if (!finite(d0) || !finite(d1)) {
                S->done = S->breakdown = 1;
            } else if (d1 <= S->tol2 * S->bb) {
                S->done = 1;
            } else if (S->omega == 0.0 || d0 == 0.0) {
                S->done = S->breakdown = 1;
            } else {
                S->beta = (d0 / S->rho) * (S->alpha / S->omega);
                S->rho = d0;
                if (S->iter >= S->max_iters) S->done = 1;
            }
        }
    }
}

// p = p + delta, rounded to the field type.
template <typename Real>
__global__ void __launch_bounds__(kVecThreads) k_add_delta(long long n, Real* p, const double* __restrict__ d) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        p[c] = (Real)((double)p[c] + d[c]);
}

dim3 stencil_grid(const GridGeom& g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }

}  // namespace

long long krylov_vec_blocks(long long n) {
    long long b = (n + kVecThreads - 1) / kVecThreads;
    const long long cap = 152LL * 8;  // eight 256-thread blocks per SM, grid-stride beyond
    return b < 1 ? 1 : (b > cap ? cap : b);
}

long long krylov_partials(const GridGeom& g, long long n) {
    const dim3 sg = stencil_grid(g);
    const long long ns = (long long)sg.x * sg.y * sg.z;
    const long long nv = krylov_vec_blocks(n);
    return ns > nv ? ns : nv;
}

cudaError_t krylov_dinv(const GridGeom& g, bool mixed, const void* vals, const double* diag64, double* dinv,
                        double* lmul, double* up, bool line, cudaStream_t st) {
    if (line) {
        const unsigned nb = (unsigned)(((long long)g.nx * g.ny + kLineThreads - 1) / kLineThreads);
        if (mixed)
            k_line_factor<float, true><<<nb, kLineThreads, 0, st>>>(g, (const float*)vals, diag64, dinv, lmul, up);
        else
            k_line_factor<double, false><<<nb, kLineThreads, 0, st>>>(g, (const double*)vals, diag64, dinv, lmul, up);
        return cudaGetLastError();
    }
    const dim3 blk(32, 8, 1);
    if (mixed) k_dinv<float, true><<<stencil_grid(g), blk, 0, st>>>(g, (const float*)vals, diag64, dinv);
    else k_dinv<double, false><<<stencil_grid(g), blk, 0, st>>>(g, (const double*)vals, diag64, dinv);
    return cudaGetLastError();
}

static cudaError_t line_apply(const GridGeom& g, const KrylovWork& w, const double* in, double* out, float* hi,
                              float* lo, cudaStream_t st) {
    const unsigned nb = (unsigned)(((long long)g.nx * g.ny + kApplyThreads - 1) / kApplyThreads);
    k_line_apply<<<nb, kApplyThreads, 0, st>>>(g, w.dinv, w.lmul, w.up, in, out, hi, lo, w.S);
    return cudaGetLastError();
}

cudaError_t krylov_start(const GridGeom& g, long long n, const double* b, double sign, const KrylovWork& w,
                         cudaStream_t st) {
    const long long nb = krylov_vec_blocks(n);
    k_init<<<(unsigned)nb, kVecThreads, 0, st>>>(n, b, sign, w.x, w.r, w.rh, w.part);
    k_finalize<<<1, kFinThreads, 0, st>>>(w.part, nb, 0, w.S);
    return cudaGetLastError();
}

cudaError_t krylov_iteration(const GridGeom& g, long long n, bool mixed, const void* vals, const double* diag64,
                             const KrylovWork& w, bool line, cudaStream_t st) {
    const long long nb = krylov_vec_blocks(n);
    const dim3 sg = stencil_grid(g), blk(32, 8, 1);
    const long long ns = (long long)sg.x * sg.y * sg.z;
    k_update_p<<<(unsigned)nb, kVecThreads, 0, st>>>(n, w.r, w.v, w.p, w.ph, mixed ? w.phh : nullptr,
                                                     mixed ? w.phl : nullptr, line ? nullptr : w.dinv, w.S);
    if (line) line_apply(g, w, w.p, w.ph, mixed ? w.phh : nullptr, mixed ? w.phl : nullptr, st);
    if (mixed)
        k_spmv_mixed<<<sg, blk, 0, st>>>(g, (const float*)vals, diag64, w.ph, w.phh, w.phl, w.v, w.rh, w.part, w.S);
    else
        k_spmv<<<sg, blk, 0, st>>>(g, (const double*)vals, w.ph, w.v, w.rh, w.part, w.S);
    k_finalize<<<1, kFinThreads, 0, st>>>(w.part, ns, 1, w.S);
    k_update_s<<<(unsigned)nb, kVecThreads, 0, st>>>(n, w.r, w.v, w.s, w.sh, mixed ? w.shh : nullptr,
                                                     mixed ? w.shl : nullptr, line ? nullptr : w.dinv, w.S);
    if (line) line_apply(g, w, w.s, w.sh, mixed ? w.shh : nullptr, mixed ? w.shl : nullptr, st);
    if (mixed)
        k_spmv_mixed<<<sg, blk, 0, st>>>(g, (const float*)vals, diag64, w.sh, w.shh, w.shl, w.t, w.s, w.part, w.S);
    else
        k_spmv<<<sg, blk, 0, st>>>(g, (const double*)vals, w.sh, w.t, w.s, w.part, w.S);
    k_finalize<<<1, kFinThreads, 0, st>>>(w.part, ns, 2, w.S);
    k_update_xr<<<(unsigned)nb, kVecThreads, 0, st>>>(n, w.x, w.ph, w.sh, w.s, w.t, w.r, w.rh, w.part, w.S);
    k_finalize<<<1, kFinThreads, 0, st>>>(w.part, nb, 3, w.S);
    return cudaGetLastError();
}

cudaError_t krylov_add_delta(long long n, bool mixed, void* p, const double* d, cudaStream_t st) {
    if (mixed) k_add_delta<float><<<(unsigned)krylov_vec_blocks(n), kVecThreads, 0, st>>>(n, (float*)p, d);
    else k_add_delta<double><<<(unsigned)krylov_vec_blocks(n), kVecThreads, 0, st>>>(n, (double*)p, d);
    return cudaGetLastError();
}

}  // namespace tpfa
