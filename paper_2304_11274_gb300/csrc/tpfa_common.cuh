// tpfa_common.cuh -- device-side building blocks shared by the TPFA kernels.
//
// Physics (arXiv 2304.11274, Section 3): Eq. density for rho(p), Eq. flux-calc
// for the two-point flux with single-point upwinding, Eq. vk for the
// accumulation term.  Every link function here is written with explicit
// round-to-nearest intrinsics so that the naive, tiled and batched kernels,
// whichever cell computes a link, produce bit-identical values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tpfa_grid.h"

namespace tpfa {

// ---------------------------------------------------------------- geometry

// Links of cell index i along an axis of n cells: to i-1 and to i+1.
__host__ __device__ __forceinline__ int axis_links(int i, int n) { return (i > 0) + (i < n - 1); }

// Links from all cells i' < i along an axis of n cells.
__host__ __device__ __forceinline__ long long axis_links_before(int i, int n) {
    return (long long)(i > 1 ? i - 1 : 0) + (i < n - 1 ? i : n - 1);
}

// CSR offset of the first entry of row (i, j, k).  A row holds the cell
// itself and adj(K) (Section 5.1), so its length is
//   1 + ex(i) + ey(j) + ez(k) + diag * ex(i) * ey(j);
// summing that over all cells before (i, j, k) in x-fastest order gives this
// closed form, so the kernels never read row_ptr.
__host__ __device__ __forceinline__ long long row_start(const GridGeom& g, int i, int j, int k) {
    const long long nx = g.nx, ny = g.ny;
    const long long Ex = 2 * (nx - 1), Ey = 2 * (ny - 1);
    const long long D = g.diag;
    const long long plane = nx * ny + Ex * ny + nx * Ey + D * Ex * Ey;
    const int ez = axis_links(k, g.nz), ey = axis_links(j, g.ny);
    long long s = (long long)k * plane + nx * ny * axis_links_before(k, g.nz);
    s += (long long)j * (nx + Ex + nx * ez) + axis_links_before(j, g.ny) * (nx + D * Ex);
    s += (long long)i * (1 + ey + ez) + axis_links_before(i, g.nx) * (1 + D * ey);
    return s;
}

__host__ __device__ __forceinline__ long long total_nnz(const GridGeom& g) {
    return row_start(g, 0, 0, g.nz);
}

__host__ __device__ __forceinline__ int row_length(const GridGeom& g, int i, int j, int k) {
    const int ex = axis_links(i, g.nx), ey = axis_links(j, g.ny), ez = axis_links(k, g.nz);
    return 1 + ex + ey + ez + g.diag * ex * ey;
}

// ---------------------------------------------------------------- FP32 -> FP64

// Exact widening of a float to a double done on the integer pipe.  On GB300
// the float->double convert instruction issues on the FP64 unit (about two
// per clock per SM), which the mixed kernels cannot afford per link; this
// rebuilds the IEEE-754 binary64 bit pattern of normal numbers and zeros
// (sign kept, exponent rebiased by 1023 - 127 = 896, 23-bit fraction moved up
// by 29 bits) and leaves subnormals, infinities and NaNs to the hardware.
__device__ __forceinline__ double widen(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t a = u & 0x7fffffffu;
    if (a - 0x00800000u < 0x7f000000u) {  // normal: 0x00800000 <= a < 0x7f800000
        const uint32_t hi = ((a >> 3) + 0x38000000u) | (u & 0x80000000u);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if (a == 0u) return __hiloint2double((int)u, 0);  // signed zero
    return (double)x;
}

// Narrowing of a finite, normal-range double to a float by truncating the
// fraction (error below one float ulp), on the integer pipe.  Used only where
// the value is a small additive term of a compensated FP32 sum.
__device__ __forceinline__ float narrow_rz(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x);
    const uint32_t lo = (uint32_t)__double2loint(x);
    const uint32_t ex = (hi >> 20) & 0x7ffu;
    if (ex > 896u && ex < 1151u) {
        const uint32_t f = ((hi & 0x000fffffu) << 3) | (lo >> 29);
        return __uint_as_float((hi & 0x80000000u) | ((ex - 896u) << 23) | f);
    }
    return (float)x;
}

// A double as an unevaluated FP32 pair v = hi + lo (hi the truncation of v,
// lo the exact remainder narrowed; |lo| < ulp(hi)), so differences of nearby
// values can be formed in FP32: (hi_a - hi_b) + (lo_a - lo_b) is accurate to
// a few float ulps of a - b itself (hi_a - hi_b is exact when a and b are
// within a factor of two).
struct F2Split {
    float hi, lo;
};
__device__ __forceinline__ F2Split split_f2(double v) {
    F2Split r;
    r.hi = narrow_rz(v);
    r.lo = narrow_rz(__dadd_rn(v, -widen(r.hi)));
    return r;
}

// a - b for two split doubles, in FP32.
__device__ __forceinline__ float diff_f2(const F2Split& a, const F2Split& b) {
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

// Distance over area of each link direction, the geometric factor of the
// two-point transmissibility (x faces, y faces, z faces, in-plane diagonals).
struct LinkGeo {
    float cx, cy, cz, cd;
};


// ---------------------------------------------------------------- Kahan

struct Kahan32 {
    float s = 0.f, c = 0.f;  // running sum and compensation; value = s - c
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

// ---------------------------------------------------------------- cell state

template <typename T>
struct CellVal {
    T p, z, rho, drho;  // pressure, depth, density, d rho / dp
};

struct PhysF {
    float rho_ref, p_ref, c_f, inv_mu, g, half_g, V_dt, c_r;
};
struct PhysD {
    double rho_ref, p_ref, c_f, inv_mu, g, half_g, V_dt, c_r;
};

// exp(x) and expm1(x) in FP64 for the small arguments the state equation
// meets (|x| < 2^-5: c_f (p - p_ref) with c_f ~ 1e-9 / Pa and pressures
// within tens of MPa of p_ref) by their Taylor series, cut after x^8 (exp)
// and x^9 (expm1): the remainder is below 2^-60 of the value, so the result
// is the function's within the few roundings of the Horner steps.  Larger
// arguments (and NaN or infinity) take exp() / expm1().  The FP64 path is
// bound by the FP64 pipe, and these series need fewer FP64 instructions per
// exponential call.  The range test reads the high word (integer pipe).
__device__ __forceinline__ bool small_arg(double x) {
    return ((uint32_t)__double2hiint(x) & 0x7fffffffu) < 0x3fa00000u;  // |x| < 2^-5
}
__device__ __forceinline__ double exp_fp64(double x) {
    if (!small_arg(x)) return exp(x);
    double r = 1.0 / 40320.0;  // 1/8!
    r = __fma_rn(r, x, 1.0 / 5040.0);
    r = __fma_rn(r, x, 1.0 / 720.0);
    r = __fma_rn(r, x, 1.0 / 120.0);
    r = __fma_rn(r, x, 1.0 / 24.0);
    r = __fma_rn(r, x, 1.0 / 6.0);
    r = __fma_rn(r, x, 0.5);
    r = __fma_rn(r, x, 1.0);
    return __fma_rn(r, x, 1.0);
}
__device__ __forceinline__ double expm1_fp64(double x) {
    if (!small_arg(x)) return expm1(x);
    double r = 1.0 / 362880.0;  // 1/9!: expm1(x) = x (1 + x/2! + x^2/3! + ... + x^8/9!)
    r = __fma_rn(r, x, 1.0 / 40320.0);
    r = __fma_rn(r, x, 1.0 / 5040.0);
    r = __fma_rn(r, x, 1.0 / 720.0);
    r = __fma_rn(r, x, 1.0 / 120.0);
    r = __fma_rn(r, x, 1.0 / 24.0);
    r = __fma_rn(r, x, 1.0 / 6.0);
    r = __fma_rn(r, x, 0.5);
    r = __fma_rn(r, x, 1.0);
    return __dmul_rn(r, x);
}

// Eq. density: rho = rho_ref exp(c_f (p - p_ref)), and its derivative.
__device__ __forceinline__ CellVal<float> make_cell(const PhysF& q, float p, float z) {
    CellVal<float> c;
    c.p = p;
    c.z = z;
    c.rho = __fmul_rn(q.rho_ref, expf(__fmul_rn(q.c_f, __fsub_rn(p, q.p_ref))));
    c.drho = __fmul_rn(q.c_f, c.rho);
    return c;
}
__device__ __forceinline__ CellVal<double> make_cell(const PhysD& q, double p, double z) {
    CellVal<double> c;
    c.p = p;
    c.z = z;
    c.rho = __dmul_rn(q.rho_ref, exp_fp64(__dmul_rn(q.c_f, __dsub_rn(p, q.p_ref))));
    c.drho = __dmul_rn(q.c_f, c.rho);
    return c;
}

// ---------------------------------------------------------------- one link

template <typename T>
struct LinkOut {
    T F;   // F_ab: mass outflow from a to b
    T Da;  // dF_ab / dp_a
    T Db;  // dF_ab / dp_b
};

// Two-point flux of Eq. flux-calc seen from row a (z = depth, positive down):
//   dPhi = (p_a - p_b) - rho_avg g (z_a - z_b)
//   upstream = a if dPhi > 0 else b,  F = T (rho_up / mu) dPhi
// and its two pressure derivatives.  rho_avg g dz is formed as
// (rho_a + rho_b)(g/2 dz): halving is exact, so the fused product equals
// the one of rho_avg and g dz bit for bit, with two multiplications fewer;
// T/mu is formed once and scales both rho_up and dPhi.  Negating every input
// that changes sign between the two ends of a link negates every output, so
// F_ba = -F_ab exactly (except the derivatives at an exact tie dPhi == 0,
// where each end takes the other cell as upstream).
__device__ __forceinline__ LinkOut<float> link(const PhysF& q, float T, const CellVal<float>& a,
                                               const CellVal<float>& b) {
    const float dp = __fsub_rn(a.p, b.p);
    const float hgdz = __fmul_rn(q.half_g, __fsub_rn(a.z, b.z));
    const float dphi = __fmaf_rn(-__fadd_rn(a.rho, b.rho), hgdz, dp);
    const bool up_a = dphi > 0.f;
    const float Tm = __fmul_rn(T, q.inv_mu);
    const float Tl = __fmul_rn(Tm, up_a ? a.rho : b.rho);
    const float w = __fmul_rn(Tm, dphi);
    LinkOut<float> r;
    r.F = __fmul_rn(Tl, dphi);
    const float dda = __fmaf_rn(-a.drho, hgdz, 1.f);
    const float ddb = __fmaf_rn(-b.drho, hgdz, -1.f);
    r.Da = __fmaf_rn(Tl, dda, up_a ? __fmul_rn(a.drho, w) : 0.f);
    r.Db = __fmaf_rn(Tl, ddb, up_a ? 0.f : __fmul_rn(b.drho, w));
    return r;
}

__device__ __forceinline__ LinkOut<double> link(const PhysD& q, double T, const CellVal<double>& a,
                                                const CellVal<double>& b) {
    const double dp = __dsub_rn(a.p, b.p);
    const double hgdz = __dmul_rn(q.half_g, __dsub_rn(a.z, b.z));
    const double dphi = __fma_rn(-__dadd_rn(a.rho, b.rho), hgdz, dp);
    const bool up_a = dphi > 0.0;
    const double Tm = __dmul_rn(T, q.inv_mu);
    const double Tl = __dmul_rn(Tm, up_a ? a.rho : b.rho);
    const double w = __dmul_rn(Tm, dphi);
    LinkOut<double> r;
    r.F = __dmul_rn(Tl, dphi);
    const double dda = __fma_rn(-a.drho, hgdz, 1.0);
    const double ddb = __fma_rn(-b.drho, hgdz, -1.0);
    r.Da = __fma_rn(Tl, dda, __dmul_rn(up_a ? a.drho : 0.0, w));
    r.Db = __fma_rn(Tl, ddb, __dmul_rn(up_a ? 0.0 : b.drho, w));
    return r;
}

// ---------------------------------------------------------------- packed FP32x2
//
// Two links evaluated at once with the FP32x2 instructions of sm_100+ (each
// half rounds exactly like the scalar instruction, so link2() returns, in
// each half, the bits link() returns for that link).

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

struct Link2 {
    float2 F, Da, Db;  // .x: first link, .y: second link
};

__device__ __forceinline__ Link2 link2(const PhysF& q, float2 T, const CellVal<float>& a, const CellVal<float>& b0,
                                       const CellVal<float>& b1) {
    const float2 dp = __fadd2_rn(f2(a.p), neg2(f2(b0.p, b1.p)));
    const float2 hgdz = __fmul2_rn(f2(q.half_g), __fadd2_rn(f2(a.z), neg2(f2(b0.z, b1.z))));
    const float2 dphi = __ffma2_rn(neg2(__fadd2_rn(f2(a.rho), f2(b0.rho, b1.rho))), hgdz, dp);
    const bool u0 = dphi.x > 0.f, u1 = dphi.y > 0.f;
    const float2 Tm = __fmul2_rn(T, f2(q.inv_mu));
    const float2 Tl = __fmul2_rn(Tm, f2(u0 ? a.rho : b0.rho, u1 ? a.rho : b1.rho));
    const float2 w = __fmul2_rn(Tm, dphi);
    Link2 r;
    r.F = __fmul2_rn(Tl, dphi);
    const float2 dda = __ffma2_rn(neg2(f2(a.drho)), hgdz, f2(1.f));
    const float2 ddb = __ffma2_rn(neg2(f2(b0.drho, b1.drho)), hgdz, f2(-1.f));
    const float2 ta = __fmul2_rn(f2(a.drho), w);
    const float2 tb = __fmul2_rn(f2(b0.drho, b1.drho), w);
    r.Da = __ffma2_rn(Tl, dda, f2(u0 ? ta.x : 0.f, u1 ? ta.y : 0.f));
    r.Db = __ffma2_rn(Tl, ddb, f2(u0 ? 0.f : tb.x, u1 ? 0.f : tb.y));
    return r;
}

// Kahan summation of two independent sums at once (.x and .y), each half
// identical to Kahan32 on its own.  The three subtractions are written as
// fused multiply-adds by -1 (a - b = fma(b, -1, a): the product is exact, so
// the one rounding is the subtraction's).  Written as paired additions of a
// negated operand, they gave sums differing from the scalar Kahan32 by an
// ulp in the two-cell march (found by comparing variants against the naive
// kernel; the fused form matches it bit for bit in every kernel).
struct Kahan2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 x) {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 y = __ffma2_rn(c, m1, x);
        const float2 t = __fadd2_rn(s, y);
        c = __ffma2_rn(y, m1, __ffma2_rn(s, m1, t));
        s = t;
    }
};

// ---------------------------------------------------------------- accumulation

// expm1(x) in FP32.  The accumulation term's argument c_f (p - p^n) is tiny
// (|x| ~ 1e-4 for a time step's pressure change of 0.1 MPa at c_f = 1e-9 /
// Pa), so below 2^-7 it takes the Taylor series x (1 + x/2 (1 + x/3 (1 +
// x/4))): the first omitted term is x^5 / 120, below 2^-30 of the value, so
// the error is the rounding of three fused multiply-adds and a product (a
// few ulps); larger arguments take expm1f().  Every FP32 kernel calls this,
// so they still agree bit for bit.
__device__ __forceinline__ float expm1_f32(float x) {
    if (fabsf(x) < 0.0078125f) {
        float r = __fmaf_rn(x, 1.f / 24.f, 1.f / 6.f);
        r = __fmaf_rn(x, r, 0.5f);
        r = __fmaf_rn(x, r, 1.f);
        return __fmul_rn(r, x);
    }
    return expm1f(x);
}

// Accumulation term of Eq. vk, A = (V/dt)(phi(p) rho(p) - phi^n rho^n), and
// dA/dp.  With mn = (V/dt) phi(p^n) rho(p^n) precomputed in FP64:
//   phi(p) rho(p) - phi^n rho^n = phi0 c_r (p - p^n) rho(p) + phi^n rho^n expm1(c_f (p - p^n)),
// which forms the small difference without cancellation.
struct AccF {
    double A;  // FP64 accumulation term
    float dA;  // its pressure derivative (a term of the FP32 diagonal sum)
};

template <bool CR>
__device__ __forceinline__ AccF accumulation(const PhysF& q, float p, float pn, double mn, float rho,
                                             float phi0) {
    const float dpn = __fsub_rn(p, pn);
    const float e = expm1_f32(__fmul_rn(q.c_f, dpn));
    AccF r;
    r.A = __dmul_rn(mn, widen(e));
    if (CR) {
        // (V/dt) phi0 c_r (p - p^n) rho(p), and dA = (V/dt)(phi0 c_r rho + phi(p) c_f rho)
        const float vphi = __fmul_rn(q.V_dt, phi0);
        r.A = __dadd_rn(r.A, widen(__fmul_rn(__fmul_rn(vphi, q.c_r), __fmul_rn(dpn, rho))));
        const float phi_rel = __fmaf_rn(q.c_r, __fsub_rn(p, q.p_ref), 1.f);
        r.dA = __fmul_rn(__fmul_rn(vphi, rho), __fmaf_rn(phi_rel, q.c_f, q.c_r));
    } else {
        // phi = phi0: (V/dt) phi0 rho(p) = mn exp(c_f (p - p^n))
        r.dA = __fmul_rn(__fmul_rn(q.c_f, narrow_rz(mn)), __fadd_rn(1.f, e));
    }
    return r;
}

struct AccD {
    double A, dA;
};

template <bool CR>
__device__ __forceinline__ AccD accumulation(const PhysD& q, double p, double pn, double mn, double rho,
                                             double phi0) {
    const double dpn = __dsub_rn(p, pn);
    const double e = expm1_fp64(__dmul_rn(q.c_f, dpn));
    AccD r;
    r.A = __dmul_rn(mn, e);
    if (CR) {
        const double vphi = __dmul_rn(q.V_dt, phi0);
        r.A = __fma_rn(__dmul_rn(vphi, q.c_r), __dmul_rn(dpn, rho), r.A);
        const double phi_rel = __fma_rn(q.c_r, __dsub_rn(p, q.p_ref), 1.0);
        r.dA = __dmul_rn(__dmul_rn(vphi, rho), __fma_rn(phi_rel, q.c_f, q.c_r));
    } else {
        r.dA = __dmul_rn(__dmul_rn(q.c_f, mn), __dadd_rn(1.0, e));
    }
    return r;
}

// Non-finite test on the integer pipe (exponent all ones).
__device__ __forceinline__ bool nonfinite(double x) {
    return ((uint32_t)__double2hiint(x) & 0x7ff00000u) == 0x7ff00000u;
}

}  // namespace tpfa
