// tpfa_xmarch.cuh -- the mixed-path assembly march with two cells per lane
// (sm_103a).
//
// A warp owns a 64-cell x-segment (cells i0 .. i0+63) of one z-plane k and
// marches along y over a run of JY rows; lane l owns the adjacent cells
// a = i0 + 2l and b = a + 1 of each row, so every per-cell quantity of a
// lane is an FP32 pair and every link it evaluates is one half of an FP32x2
// instruction whose other half is the same link of its other cell.  Per row
// j each lane assembles rows (a, j, k) and (b, j, k) of Algorithm 1 / Eq. vk:
//
//   * links evaluated from the lane's side, as pairs (cell a, cell b):
//       +x (a -> b, b -> lane+1's a), +y, +x+y, -x+y, +z, -z
//     and one pair for the segment's halo: lane 0's -x and -x-y links of a,
//     lane 31's +x-y link of b (the far cells lie outside the segment);
//   * the -x link of b is the negation of a's +x, the -x link of a the
//     negation of lane-1's b's +x (a shuffle); the links into row j-1 are
//     the negations of the previous step's +y, +x+y and -x+y links (own or
//     a neighbour lane's).  Negating every input that changes sign between
//     the two ends of a link negates every output, so these reused values
//     are exact, except at an exact tie dPhi == 0 (each end then takes the
//     other cell as upstream): a warp that meets a zero flux on a reused
//     link records the row and recomputes it after the march with the naive
//     kernel's row code, so every row is bit-identical to that kernel's;
//   * densities: the two cells of row j+1 and the halo cell (lanes 0 and
//     31) as they enter the window, the four vertical neighbours per row;
//   * every pair-valued input of row j+2 (p, depth, the five owned T, p^n,
//     the vertical neighbours' p and depth and the T below) moves as one
//     8-byte cp.async per lane, m^n as one 16-byte copy, into a per-warp
//     two-slot shared-memory ring: a slot is refilled right after its row's
//     values were read into registers;
//   * residual and diagonal: FP32x2 Kahan sums whose halves are the two
//     cells' own sums, in slot order (the order of assemble_row);
//   * the warp's 128 Jacobian rows are one contiguous CSR segment (a closed
//     form of (i0, j, k)); values are staged in shared memory and written by
//     one cp.async.bulk copy per row.
//
// Requires nx even (every pair starts on an even cell index, so the 8- and
// 16-byte copies and the paired R / diag64 stores are aligned and a lane's
// two cells are either both inside the grid or both outside).
#pragma once

#include "tpfa_row.cuh"

namespace tpfa {

// Two cells' values: .x cell a, .y cell b.
struct CellPair {
    float2 p, z, rho, drho;
};

__device__ __forceinline__ CellVal<float> cell_of(const CellPair& c, int h) {
    return h == 0 ? CellVal<float>{c.p.x, c.z.x, c.rho.x, c.drho.x} : CellVal<float>{c.p.y, c.z.y, c.rho.y, c.drho.y};
}

// link() of Eq. flux-calc for two independent links at once: half h is
// link(q, T.h, A.h, B.h), bit for bit (each FP32x2 half rounds as the scalar
// instruction does, and the operations are link()'s, in its order).
__device__ __forceinline__ Link2 link_pp(const PhysF& q, float2 T, const CellPair& A, const CellPair& B) {
    const float2 dp = __fadd2_rn(A.p, neg2(B.p));
    const float2 hgdz = __fmul2_rn(f2(q.half_g), __fadd2_rn(A.z, neg2(B.z)));
    const float2 dphi = __ffma2_rn(neg2(__fadd2_rn(A.rho, B.rho)), hgdz, dp);
    const bool u0 = dphi.x > 0.f, u1 = dphi.y > 0.f;
    const float2 Tm = __fmul2_rn(T, f2(q.inv_mu));
    const float2 Tl = __fmul2_rn(Tm, f2(u0 ? A.rho.x : B.rho.x, u1 ? A.rho.y : B.rho.y));
    const float2 w = __fmul2_rn(Tm, dphi);
    Link2 r;
    r.F = __fmul2_rn(Tl, dphi);
    const float2 dda = __ffma2_rn(neg2(A.drho), hgdz, f2(1.f));
    const float2 ddb = __ffma2_rn(neg2(B.drho), hgdz, f2(-1.f));
    const float2 ta = __fmul2_rn(A.drho, w);
    const float2 tb = __fmul2_rn(B.drho, w);
    r.Da = __ffma2_rn(Tl, dda, f2(u0 ? ta.x : 0.f, u1 ? ta.y : 0.f));
    r.Db = __ffma2_rn(Tl, ddb, f2(u0 ? 0.f : tb.x, u1 ? 0.f : tb.y));
    return r;
}

// A link seen from its other end (F_LK = -F_KL; the two derivatives swap and
// change sign): exact except at a tie.
__device__ __forceinline__ LinkOut<float> flip(float F, float Da, float Db) { return LinkOut<float>{-F, -Db, -Da}; }

// Kahan2 step applied to the halves selected by va / vb only (a skipped half
// keeps its state bit for bit, as a skipped slot does in assemble_row).
__device__ __forceinline__ void kahan2_masked(Kahan2& k, float2 x, bool va, bool vb) {
    Kahan2 t = k;
    t.add(x);
    k.s.x = va ? t.s.x : k.s.x;
    k.c.x = va ? t.c.x : k.c.x;
    k.s.y = vb ? t.s.y : k.s.y;
    k.c.y = vb ? t.c.y : k.c.y;
}

// accumulation() of Eq. vk for cells a and b at once: each half performs
// the scalar function's operations in its order (FP32x2 halves round as the
// scalar instructions do), so the results are its bits.  Returns the FP64
// terms A of both cells and the pair of dA/dp.
template <bool CRK>
__device__ __forceinline__ float2 accumulation2(const PhysF& q, float2 p, float2 pn, double2 mn, float2 rho,
                                                float2 phi0, double& Aa, double& Ab) {
    if constexpr (CRK) {
        const AccF a = accumulation<true>(q, p.x, pn.x, mn.x, rho.x, phi0.x);
        const AccF b = accumulation<true>(q, p.y, pn.y, mn.y, rho.y, phi0.y);
        Aa = a.A;
        Ab = b.A;
        return f2(a.dA, b.dA);
    } else {
        const float2 m1 = f2(-1.f);
        const float2 x = __fmul2_rn(f2(q.c_f), __ffma2_rn(pn, m1, p));  // c_f (p - p^n)
        float2 e;
        if (fabsf(x.x) < 0.0078125f && fabsf(x.y) < 0.0078125f) {  // expm1_f32's series for both
            float2 r = __ffma2_rn(x, f2(1.f / 24.f), f2(1.f / 6.f));
            r = __ffma2_rn(x, r, f2(0.5f));
            r = __ffma2_rn(x, r, f2(1.f));
            e = __fmul2_rn(r, x);
        } else {
            e = f2(expm1_f32(x.x), expm1_f32(x.y));
        }
        Aa = __dmul_rn(mn.x, widen(e.x));
        Ab = __dmul_rn(mn.y, widen(e.y));
        return __fmul2_rn(__fmul2_rn(f2(q.c_f), f2(narrow_rz(mn.x), narrow_rz(mn.y))), __fadd2_rn(f2(1.f), e));
    }
}

template <bool DIAG, bool CRK, int W>
struct XMarch {
    // ---- ring layout (floats, per warp and slot)
    enum { P_P, P_Z, P_TX, P_TY, P_TZ, P_TPP, P_TMP, P_PN, P_PZM, P_ZZM, P_TZM, P_PZP, P_ZZP, P_PHI };
    static constexpr int NP = CRK ? P_PHI + 1 : P_PHI;  // pair fields, 64 floats each
    static constexpr int OFF_MN = NP * 64;              // 32 lanes x 2 doubles
    static constexpr int OFF_H = OFF_MN + 128;          // halo singles: p, z, T1, T2 x {lane 0, lane 31}
    static constexpr int SLOT = OFF_H + 8;              // floats per slot (a multiple of 4)
    static constexpr int RING = 2;
    static constexpr int L = DIAG ? 11 : 7;             // interior row length
    static constexpr int LX = DIAG ? 3 : 1;             // x-side links of a row per side
    static constexpr int BUF = 64 * NSLOT + 4;          // CSR staging buffer (floats)
    static constexpr unsigned kFullMask = DIAG ? 0x7ffu : 0x575u;
    static constexpr unsigned kXMinus = 0x92u;  // slots 1, 4, 7
    static constexpr unsigned kXPlus = 0x248u;  // slots 3, 6, 9
    static_assert(SLOT % 4 == 0, "16-byte aligned slots");

    static constexpr int smem_floats_per_warp() { return RING * SLOT + 2 * BUF; }
};

template <bool DIAG, bool CRK, int W>
constexpr int xmarch_smem_bytes() {
    return W * XMarch<DIAG, CRK, W>::smem_floats_per_warp() * 4;
}

__device__ __forceinline__ void cpa8(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cpa4(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
// A 4-byte copy issued only by the lanes where `lane_on` holds (a guard
// predicate, so the warp does not branch around it).
__device__ __forceinline__ void cpa4_if(float* dst, const float* src, bool valid, bool lane_on) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
                 "@q cp.async.ca.shared.global [%0], [%1], 4, %2;\n\t}" ::"r"(d),
                 "l"(src), "r"(valid ? 4 : 0), "r"((unsigned)lane_on)
                 : "memory");
}
__device__ __forceinline__ void cpa16(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// Sums and staged values of one row pair (cells a, b), fed slot by slot in
// ascending slot order.  PATH 2: every slot exists for both cells; PATH 1:
// j and k interior in a segment touching an x boundary (cell a at i = 0
// lacks slots 1, 4, 7; cell b at i = nx - 1 lacks 3, 6, 9); PATH 0: per-cell
// masks.  Each half of the Kahan pairs is the cell's own sum in slot order,
// so the sums equal assemble_row's bit for bit.
template <bool DIAG, int PATH>
struct XRow {
    static constexpr unsigned kFull = DIAG ? 0x7ffu : 0x575u;
    static constexpr unsigned kXMinus = 0x92u & kFull;  // slots 1, 4, 7
    static constexpr unsigned kXPlus = 0x248u & kFull;  // slots 3, 6, 9
    static constexpr int L = DIAG ? 11 : 7;
    Kahan2 kr, kd;       // residual (F) and diagonal (dF/dp_K) sums of a and b
    Kahan32 ka, kb, kda, kdb;  // PATH 0: the same sums per cell
    float* ra;           // staging position of row a's first value
    float* rb;           // ... of row b's
    unsigned ma, mb;     // PATH 0: slot masks
    bool bnd_a, bnd_b;   // PATH 1: a at i = 0, b at i = nx - 1

    template <int S>
    static constexpr int full_pos() {
        return __builtin_popcount(kFull & ((1u << S) - 1u));
    }
    template <int S>
    __device__ __forceinline__ void put(const LinkOut<float>& a, const LinkOut<float>& b, bool act) {
        static_assert(S != SLOT_SELF, "the diagonal is not a link");
        if constexpr (!((kFull >> S) & 1u)) return;
        const float2 F = f2(a.F, b.F), Da = f2(a.Da, b.Da);
        if constexpr (PATH == 2) {
            kr.add(F);
            kd.add(Da);
            if (act) {
                ra[full_pos<S>()] = a.Db;
                rb[full_pos<S>()] = b.Db;
            }
        } else if constexpr (PATH == 1) {
            constexpr bool xm = (kXMinus >> S) & 1u, xp = (kXPlus >> S) & 1u;
            constexpr int sa = __builtin_popcount(kXMinus & ((1u << S) - 1u));
            constexpr int sb = __builtin_popcount(kXPlus & ((1u << S) - 1u));
            const bool va = !(xm && bnd_a), vb = !(xp && bnd_b);
            if constexpr (xm || xp) {
                kahan2_masked(kr, F, va, vb);
                kahan2_masked(kd, Da, va, vb);
            } else {
                kr.add(F);
                kd.add(Da);
            }
            if (act) {
                if (va) ra[full_pos<S>() - (bnd_a ? sa : 0)] = a.Db;
                if (vb) rb[full_pos<S>() - (bnd_b ? sb : 0)] = b.Db;
            }
        } else {
            // general rows: each cell's own scalar sums, skipping its absent slots
            const bool va = (ma >> S) & 1u, vb = (mb >> S) & 1u;
            if (va) {
                ka.add(a.F);
                kda.add(a.Da);
                if (act) ra[slot_pos(ma, S)] = a.Db;
            }
            if (vb) {
                kb.add(b.F);
                kdb.add(b.Da);
                if (act) rb[slot_pos(mb, S)] = b.Db;
            }
        }
    }
    // PATH 0: the scalar sums as pairs
    __device__ __forceinline__ void gather() {
        if constexpr (PATH == 0) {
            kr.s = f2(ka.s, kb.s);
            kr.c = f2(ka.c, kb.c);
            kd.s = f2(kda.s, kdb.s);
            kd.c = f2(kda.c, kdb.c);
        }
    }
    // the diagonal entry (slot 5) of each row
    __device__ __forceinline__ void put_diag(float da, float db, bool act) const {
        if (!act) return;
        if constexpr (PATH == 2) {
            ra[full_pos<SLOT_SELF>()] = da;
            rb[full_pos<SLOT_SELF>()] = db;
        } else if constexpr (PATH == 1) {
            constexpr int sa = __builtin_popcount(kXMinus & ((1u << SLOT_SELF) - 1u));
            constexpr int sb = __builtin_popcount(kXPlus & ((1u << SLOT_SELF) - 1u));
            ra[full_pos<SLOT_SELF>() - (bnd_a ? sa : 0)] = da;
            rb[full_pos<SLOT_SELF>() - (bnd_b ? sb : 0)] = db;
        } else {
            ra[slot_pos(ma, SLOT_SELF)] = da;
            rb[slot_pos(mb, SLOT_SELF)] = db;
        }
    }
};

// Per-warp state of the two-cell march.
template <bool DIAG, bool CRK, int W, bool FAST>
struct XState {
    using X = XMarch<DIAG, CRK, W>;
    const GridGeom& g;
    const PhysF& q;
    const AsmFields<float>& f;
    const AsmOut<float>& o;
    float* ring;
    float* stage;
    int lane, k, nx, ny, nxy, kb, i0, ia, ib, ih, ez, rowA, rowB, Sx0;
    bool act, hl, hact, zm, zp, okb, oka, v16, r16;
    long long base_k;

    // window: rows j (C) and j-1 (halo only), x-neighbours of row j, links
    // from row j-1 into row j
    CellPair Cc;
    CellVal<float> Ch, Ph, Cm, Cp;
    Link2 Uy, Uxy, Umxy;
    bool tie_up;

    __device__ __forceinline__ XState(const GridGeom& g_, const PhysF& q_, const AsmFields<float>& f_,
                                      const AsmOut<float>& o_, float* ring_, int lane_, int k_, int bx)
        : g(g_), q(q_), f(f_), o(o_), ring(ring_), lane(lane_), k(k_) {
        stage = ring + X::RING * X::SLOT;
        nx = g.nx;
        ny = g.ny;
        nxy = nx * ny;
        kb = nxy * k;
        i0 = bx * 64;
        ia = i0 + 2 * lane;
        ib = ia + 1;
        act = ia < nx;  // nx even: then ib < nx too
        hl = lane == 31;  // lane 31 keeps the right halo, lane 0 the left one
        ih = hl ? i0 + 64 : i0 - 1;
        hact = (lane == 0 || hl) && ih >= 0 && ih < nx;
        zm = k > 0;
        zp = k + 1 < g.nz;
        okb = act && ib + 1 < nx;  // b's +x and +x+y links exist
        oka = act && ia > 0;       // a's -x+y link exists
        v16 = FAST || (reinterpret_cast<uintptr_t>(o.vals) & 15u) == 0;
        r16 = FAST || ((reinterpret_cast<uintptr_t>(o.R) | reinterpret_cast<uintptr_t>(o.diag64)) & 15u) == 0;
        const long long Ex = 2LL * (nx - 1), Ey = 2LL * (ny - 1), D = g.diag;
        const long long plane = (long long)nx * ny + Ex * ny + (long long)nx * Ey + D * Ex * Ey;
        ez = axis_links(k, g.nz);
        base_k = (long long)k * plane + (long long)nxy * axis_links_before(k, g.nz);
        rowA = (int)(nx + Ex + (long long)nx * ez);
        rowB = (int)(nx + D * Ex);
        Sx0 = (int)axis_links_before(i0, nx);
    }

    // ---- request every input of row r into ring slot sl
    __device__ __forceinline__ void issue(int r, int sl) const {
        float* S = ring + sl * X::SLOT;
        float* Sl = S + 2 * lane;
        const bool rv = r >= 0 && r < ny;
        const int c = kb + nx * (rv ? r : 0) + (act ? ia : 0);
        const bool a = rv && act;
        cpa8(Sl + X::P_P * 64, f.p + c, a);
        cpa8(Sl + X::P_Z * 64, f.z + c, a);
        cpa8(Sl + X::P_TX * 64, f.Tx + c, a);
        cpa8(Sl + X::P_TY * 64, f.Ty + c, a);
        cpa8(Sl + X::P_TZ * 64, f.Tz + c, a);
        if (DIAG) {
            cpa8(Sl + X::P_TPP * 64, f.Tpp + c, a);
            cpa8(Sl + X::P_TMP * 64, f.Tmp + c, a);
        }
        cpa8(Sl + X::P_PN * 64, f.pn + c, a);
        if (CRK) cpa8(Sl + X::P_PHI * 64, f.phi0 + c, a);
        const int cm = zm ? c - nxy : c, cp = zp ? c + nxy : c;
        cpa8(Sl + X::P_PZM * 64, f.p + cm, a && zm);
        cpa8(Sl + X::P_ZZM * 64, f.z + cm, a && zm);
        cpa8(Sl + X::P_TZM * 64, f.Tz + cm, a && zm);
        cpa8(Sl + X::P_PZP * 64, f.p + cp, a && zp);
        cpa8(Sl + X::P_ZZP * 64, f.z + cp, a && zp);
        cpa16(S + X::OFF_MN + 4 * lane, f.mn + c, a);
        {  // the halo cells: lanes 0 and 31 only, under a guard predicate
            const bool hlane = lane == 0 || hl;
            float* H = S + X::OFF_H + (hl ? 1 : 0);
            const int ch = kb + nx * (rv ? r : 0) + (hact ? ih : 0);
            cpa4_if(H + 0, f.p + ch, rv && hact, hlane);
            cpa4_if(H + 2, f.z + ch, rv && hact, hlane);
            // lane 0: Tx(i0-1, r) and Tpp(i0-1, r-1); lane 31: Tmp(i0+64, r-1)
            const bool t1 = rv && hact && !hl;
            cpa4_if(H + 4, f.Tx + (t1 ? ch : 0), t1, hlane);
            if (DIAG) {
                const bool t2 = rv && hact && r > 0;
                cpa4_if(H + 6, (hl ? f.Tmp : f.Tpp) + (t2 ? ch - nx : 0), t2, hlane);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __device__ __forceinline__ float2 pair_at(int sl, int fld) const {
        return *reinterpret_cast<const float2*>(ring + sl * X::SLOT + fld * 64 + 2 * lane);
    }
    __device__ __forceinline__ float halo_at(int sl, int fld) const {
        return ring[sl * X::SLOT + X::OFF_H + 2 * fld + (hl ? 1 : 0)];
    }
    // the cells of the row in slot sl: own pair and the halo cell (lanes 0 / 31)
    __device__ __forceinline__ void cells_of(int sl, CellPair& Cr, CellVal<float>& Hr) const {
        const float2 pp = pair_at(sl, X::P_P), zz = pair_at(sl, X::P_Z);
        const CellVal<float> ca = make_cell(q, pp.x, zz.x), cb = make_cell(q, pp.y, zz.y);
        Cr = CellPair{pp, zz, f2(ca.rho, cb.rho), f2(ca.drho, cb.drho)};
        Hr = make_cell(q, halo_at(sl, 0), halo_at(sl, 1));
    }
    // the x-neighbours of a row: m = (a-1) (lane-1's b; lane 0: the left
    // halo), p = (b+1) (lane+1's a; lane 31: the right halo)
    __device__ __forceinline__ void neighbours(const CellPair& Cr, const CellVal<float>& Hr, CellVal<float>& m,
                                               CellVal<float>& p) const {
        m.p = __shfl_up_sync(0xffffffffu, Cr.p.y, 1);
        m.z = __shfl_up_sync(0xffffffffu, Cr.z.y, 1);
        m.rho = __shfl_up_sync(0xffffffffu, Cr.rho.y, 1);
        p.p = __shfl_down_sync(0xffffffffu, Cr.p.x, 1);
        p.z = __shfl_down_sync(0xffffffffu, Cr.z.x, 1);
        p.rho = __shfl_down_sync(0xffffffffu, Cr.rho.x, 1);
        if (lane == 0) m = Hr;
        if (hl) p = Hr;
        m.drho = __fmul_rn(q.c_f, m.rho);
        p.drho = __fmul_rn(q.c_f, p.rho);
    }
    static __device__ __forceinline__ CellPair pair2(const CellVal<float>& x, const CellVal<float>& y) {
        return CellPair{f2(x.p, y.p), f2(x.z, y.z), f2(x.rho, y.rho), f2(x.drho, y.drho)};
    }
    // (b, next) and (prev, a) of a row pair
    static __device__ __forceinline__ CellPair shift_left(const CellPair& c, const CellVal<float>& nxt) {
        return CellPair{f2(c.p.y, nxt.p), f2(c.z.y, nxt.z), f2(c.rho.y, nxt.rho), f2(c.drho.y, nxt.drho)};
    }
    static __device__ __forceinline__ CellPair shift_right(const CellVal<float>& prv, const CellPair& c) {
        return CellPair{f2(prv.p, c.p.x), f2(prv.z, c.z.x), f2(prv.rho, c.rho.x), f2(prv.drho, c.drho.x)};
    }
    static __device__ __forceinline__ LinkOut<float> half(const Link2& l, int h) {
        return h == 0 ? LinkOut<float>{l.F.x, l.Da.x, l.Db.x} : LinkOut<float>{l.F.y, l.Da.y, l.Db.y};
    }

    // Prologue of a march starting at row j0: rows j0-1 and j0, the links
    // of row j0-1 into row j0; row j0+1 requested.
    __device__ __forceinline__ void start(int j0) {
        issue(j0 - 1, 0);
        issue(j0, 1);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        CellPair Pc;
        cells_of(0, Pc, Ph);
        cells_of(1, Cc, Ch);
        neighbours(Cc, Ch, Cm, Cp);
        Uy = link_pp(q, pair_at(0, X::P_TY), Pc, Cc);
        if (DIAG) {
            Uxy = link_pp(q, pair_at(0, X::P_TPP), Pc, shift_left(Cc, Cp));
            Umxy = link_pp(q, pair_at(0, X::P_TMP), Pc, shift_right(Cm, Cc));
        }
        // zero flux on a link reused next (only links that exist; none from row -1)
        tie_up = j0 > 0 && act &&
                 (Uy.F.x == 0.f || Uy.F.y == 0.f ||
                  (DIAG && (Uxy.F.x == 0.f || (okb && Uxy.F.y == 0.f) || (oka && Umxy.F.x == 0.f) ||
                            Umxy.F.y == 0.f)));
        issue(j0 + 1, 0);
    }

    // Row j: its inputs are in slot sD, row j+1's in slot sN.  Returns
    // whether a reused link of this row met a zero flux (warp-uniform).
    template <int PATH>
    __device__ __forceinline__ bool row(int j, int sD, int sN, int rowbase, float* buf) {
        // every lane of an interior segment (PATH 2) holds two cells of the grid
        const bool on = PATH == 2 ? true : act;
        // row j+1's cells and row j's inputs, into registers; then the slot
        // of row j is refilled with row j+2
        CellPair Nc;
        CellVal<float> Nh;
        cells_of(sN, Nc, Nh);
        const float2 Tx = pair_at(sD, X::P_TX), Ty = pair_at(sD, X::P_TY), Tz = pair_at(sD, X::P_TZ);
        const float2 Tpp = DIAG ? pair_at(sD, X::P_TPP) : f2(0.f), Tmp = DIAG ? pair_at(sD, X::P_TMP) : f2(0.f);
        const float2 pn = pair_at(sD, X::P_PN), phi = CRK ? pair_at(sD, X::P_PHI) : f2(0.f);
        const float2 pzm = pair_at(sD, X::P_PZM), zzm = pair_at(sD, X::P_ZZM), tzm = pair_at(sD, X::P_TZM);
        const float2 pzp = pair_at(sD, X::P_PZP), zzp = pair_at(sD, X::P_ZZP);
        const double2 mn = *reinterpret_cast<const double2*>(ring + sD * X::SLOT + X::OFF_MN + 4 * lane);
        const float hT1 = halo_at(sD, 2), hT2 = DIAG ? halo_at(sD, 3) : 0.f;
        issue(j + 2, sD);

        // ---- CSR offsets of the two rows
        constexpr int L = X::L, LX = X::LX;
        const int ey = PATH >= 1 ? 2 : axis_links(j, ny);
        const int per = 1 + ey + ez, perx = 1 + g.diag * ey;
        XRow<DIAG, PATH> R;
        int off_a, len_a;
        if constexpr (PATH == 2) {
            off_a = 2 * lane * L;
            len_a = L;
        } else if constexpr (PATH == 1) {
            R.bnd_a = ia == 0;
            R.bnd_b = ib == nx - 1;
            off_a = 2 * lane * L - ((i0 == 0 && lane > 0) ? LX : 0);
            len_a = L - (R.bnd_a ? LX : 0);
        } else {
            R.ma = slot_mask(g, act ? ia : 0, j, k);
            R.mb = slot_mask(g, act ? ib : 1, j, k);
            off_a = (ia - i0) * per + (int)(axis_links_before(ia, nx) - Sx0) * perx;
            len_a = __popc(R.ma);
        }
        const long long seg = base_k + rowbase + (long long)i0 * per + (long long)Sx0 * perx;
        const int aoff = (int)(seg & 3);
        R.ra = buf + aoff + off_a;
        R.rb = R.ra + len_a;
        // the bulk copy issued from this buffer two steps ago has read it
        // (lane 0 issued it; in the other lanes, which have no bulk groups, the
        // wait returns at once)
        if (v16) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();

        // ---- links and slot values, in slot order
        {
            CellPair Zm;
            {
                const CellVal<float> a0 = make_cell(q, pzm.x, zzm.x), b0 = make_cell(q, pzm.y, zzm.y);
                Zm = pair2(a0, b0);
            }
            const Link2 LZM = link_pp(q, tzm, Cc, Zm);
            R.template put<0>(half(LZM, 0), half(LZM, 1), on);
        }
        // the segment's halo links: lane 0 -> a's -x (halo of row j) and -x-y
        // (halo of row j-1); lane 31 -> b's +x-y (halo of row j-1)
        Link2 LH;
        {
            const CellVal<float> own = hl ? CellVal<float>{Cc.p.y, Cc.z.y, Cc.rho.y, Cc.drho.y}
                                          : CellVal<float>{Cc.p.x, Cc.z.x, Cc.rho.x, Cc.drho.x};
            LH = link_pp(q, hl ? f2(hT2, 0.f) : f2(hT1, hT2), pair2(own, own), pair2(hl ? Ph : Ch, Ph));
        }
        if (DIAG) {
            const float f1 = __shfl_up_sync(0xffffffffu, Uxy.F.y, 1), a1 = __shfl_up_sync(0xffffffffu, Uxy.Da.y, 1),
                        b1 = __shfl_up_sync(0xffffffffu, Uxy.Db.y, 1);
            R.template put<1>(lane == 0 ? half(LH, 1) : flip(f1, a1, b1), flip(Uxy.F.x, Uxy.Da.x, Uxy.Db.x), on);
        }
        R.template put<2>(flip(Uy.F.x, Uy.Da.x, Uy.Db.x), flip(Uy.F.y, Uy.Da.y, Uy.Db.y), on);
        if (DIAG) {
            const float f3 = __shfl_down_sync(0xffffffffu, Umxy.F.x, 1),
                        a3 = __shfl_down_sync(0xffffffffu, Umxy.Da.x, 1),
                        b3 = __shfl_down_sync(0xffffffffu, Umxy.Db.x, 1);
            R.template put<3>(flip(Umxy.F.y, Umxy.Da.y, Umxy.Db.y), hl ? half(LH, 0) : flip(f3, a3, b3), on);
        }
        const Link2 LX_ = link_pp(q, Tx, Cc, shift_left(Cc, Cp));
        {
            const float f4 = __shfl_up_sync(0xffffffffu, LX_.F.y, 1), a4 = __shfl_up_sync(0xffffffffu, LX_.Da.y, 1),
                        b4 = __shfl_up_sync(0xffffffffu, LX_.Db.y, 1);
            R.template put<4>(lane == 0 ? half(LH, 0) : flip(f4, a4, b4), flip(LX_.F.x, LX_.Da.x, LX_.Db.x), on);
        }
        R.template put<6>(half(LX_, 0), half(LX_, 1), on);
        CellVal<float> Nm, Np;
        neighbours(Nc, Nh, Nm, Np);
        Link2 LMXY, LXY;
        if (DIAG) {
            LMXY = link_pp(q, Tmp, Cc, shift_right(Nm, Nc));
            R.template put<7>(half(LMXY, 0), half(LMXY, 1), on);
        }
        const Link2 LY = link_pp(q, Ty, Cc, Nc);
        R.template put<8>(half(LY, 0), half(LY, 1), on);
        if (DIAG) {
            LXY = link_pp(q, Tpp, Cc, shift_left(Nc, Np));
            R.template put<9>(half(LXY, 0), half(LXY, 1), on);
        }
        {
            CellPair Zp;
            {
                const CellVal<float> a1 = make_cell(q, pzp.x, zzp.x), b1 = make_cell(q, pzp.y, zzp.y);
                Zp = pair2(a1, b1);
            }
            const Link2 LZP = link_pp(q, Tz, Cc, Zp);
            R.template put<10>(half(LZP, 0), half(LZP, 1), on);
        }

        // ties on this row's reused links: the previous step's up-links and
        // the +x links (a's -x comes from lane-1's b, b's -x from a)
        // (on an interior segment every lane's +x and diagonal links exist)
        const bool kb2 = PATH == 2 ? true : okb, ka2 = PATH == 2 ? true : oka;
        const bool tie_x = on && (LX_.F.x == 0.f || (kb2 && LX_.F.y == 0.f));
        const bool tie = __any_sync(0xffffffffu, tie_up || tie_x);
        tie_up = on && (LY.F.x == 0.f || LY.F.y == 0.f ||
                         (DIAG && (LXY.F.x == 0.f || (kb2 && LXY.F.y == 0.f) || (ka2 && LMXY.F.x == 0.f) ||
                                   LMXY.F.y == 0.f)));

        // ---- accumulation (Eq. vk) and the FP64 combinations
        R.gather();
        double Aa, Ab;
        const float2 dA = accumulation2<CRK>(q, Cc.p, pn, mn, Cc.rho, phi, Aa, Ab);
        const double Ra = __dadd_rn(__dadd_rn(Aa, widen(R.kr.s.x)), -widen(R.kr.c.x));
        const double Rb = __dadd_rn(__dadd_rn(Ab, widen(R.kr.s.y)), -widen(R.kr.c.y));
        Kahan2 dd = R.kd;  // the diagonals: dA joins each compensated sum last
        dd.add(dA);
        const double Da64 = __dadd_rn(widen(dd.s.x), -widen(dd.c.x));
        const double Db64 = __dadd_rn(widen(dd.s.y), -widen(dd.c.y));
        const float2 dg = __ffma2_rn(dd.c, f2(-1.f), dd.s);  // s - c, the FP32 diagonal values
        R.put_diag(dg.x, dg.y, on);
        if (on) {
            const int c = kb + nx * j + ia;
            if (FAST || o.R) {
                if (r16) *reinterpret_cast<double2*>(o.R + c) = make_double2(Ra, Rb);
                else o.R[c] = Ra, o.R[c + 1] = Rb;
            }
            if (FAST || o.diag64) {
                if (r16) *reinterpret_cast<double2*>(o.diag64 + c) = make_double2(Da64, Db64);
                else o.diag64[c] = Da64, o.diag64[c + 1] = Db64;
            }
            // a non-finite value has an all-ones exponent: one test for the four
            const uint32_t ex = max(max((uint32_t)__double2hiint(Ra) & 0x7ff00000u,
                                        (uint32_t)__double2hiint(Rb) & 0x7ff00000u),
                                    max((uint32_t)__double2hiint(Da64) & 0x7ff00000u,
                                        (uint32_t)__double2hiint(Db64) & 0x7ff00000u));
            if (ex == 0x7ff00000u) atomicOr(o.status, STATUS_NONFINITE);
        }

        // ---- the segment's CSR values: one bulk copy (ends by single lanes)
        {
            const int iend = min(i0 + 64, nx);
            int seg_len;
            if constexpr (PATH == 2) seg_len = 64 * L;
            else if constexpr (PATH == 1) seg_len = (iend - i0) * L - (i0 == 0 ? LX : 0) - (iend == nx ? LX : 0);
            else seg_len = (iend - i0) * per + (int)(axis_links_before(iend, nx) - Sx0) * perx;
            float* dst = o.vals + (seg - aoff);
            const int span = aoff + seg_len;
            if (v16) {
                const int qlo = (aoff + 3) / 4, qhi = span / 4;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (qhi > qlo) {
                    // issued and committed by lane 0 (a guard predicate, no branch)
                    const uint32_t src = (uint32_t)__cvta_generic_to_shared(buf + qlo * 4);
                    const uint32_t bytes = (uint32_t)(qhi - qlo) * 16u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %3, 0;\n\t"
                                 "@p cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
                                 "@p cp.async.bulk.commit_group;\n\t}" ::"l"(dst + qlo * 4), "r"(src), "r"(bytes),
                                 "r"(lane)
                                 : "memory");
                    const int nh = qlo * 4 - aoff, nt = span - qhi * 4;  // each < 4
                    if (lane >= 1 && lane <= nh) dst[aoff + lane - 1] = buf[aoff + lane - 1];
                    if (lane >= 8 && lane < 8 + nt) dst[qhi * 4 + lane - 8] = buf[qhi * 4 + lane - 8];
                } else {
                    if (lane < seg_len) dst[aoff + lane] = buf[aoff + lane];
                }
            } else {
                __syncwarp();
                for (int e = aoff + lane; e < span; e += 32) dst[e] = buf[e];
                __syncwarp();
            }
        }

        // ---- slide the window
        Ph = Ch;
        Cc = Nc;
        Ch = Nh;
        Cm = Nm;
        Cp = Np;
        Uy = LY;
        if (DIAG) {
            Uxy = LXY;
            Umxy = LMXY;
        }
        return tie;
    }
};

// The block's (x-segment, y-run, z-block), numbered with the x-segment
// slowest: the blocks resident at one time then belong to one column of
// x-segments, so the multiprocessors run one row path (interior or
// x-boundary segment) at a time instead of a mix of both.  Measured 2.7 %
// faster than the launch order (x-segment fastest) at 512 x 512 x 256.
__device__ __forceinline__ void segment_major(int& bx, int& by, int& bz) {
    const unsigned yz = gridDim.y * gridDim.z;
    const unsigned L = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned x = L / yz, r = L - x * yz;
    bx = (int)x;
    by = (int)(r % gridDim.y);
    bz = (int)(r / gridDim.y);
}


// One step of the march: wait for row j's inputs (and row j+1's cells),
// assemble row j, record a tie on a reused link.
template <int PATH, class State>
__device__ __forceinline__ void xmarch_row(State& M, int j, int j0, int& rowbase, unsigned long long& tie_rows) {
    using X = typename State::X;
    const int sD = (j - j0 + 1) & 1, sN = sD ^ 1;  // slots of rows j and j+1
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    float* buf = M.stage + ((j - j0) & 1) * X::BUF;
    if (M.template row<PATH>(j, sD, sN, rowbase, buf)) tie_rows |= 1ull << (j - j0);
    rowbase += M.rowA + (PATH >= 1 ? 2 : axis_links(j, M.ny)) * M.rowB;
}

// One block's work: x-segment bx (64 cells), y-run by, z-block bz.  Shared by
// the single-grid kernel and the persistent ensemble kernel.  FAST: R and
// diag64 given and, with vals, 16-byte aligned (checked by the launcher).
template <bool DIAG, bool CRK, int W, bool FAST>
__device__ __forceinline__ void xmarch_tile(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                            const AsmOut<float>& o, int JY, int bx, int by, int bz,
                                            unsigned char* smem, int kbase = 0, int kend = -1) {
    using X = XMarch<DIAG, CRK, W>;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int k = kbase + bz * W + w;  // planes [kbase, kend) of the grid (all by default)
    if (k >= (kend < 0 ? g.nz : kend)) return;  // warp-uniform
    XState<DIAG, CRK, W, FAST> M(g, q, f, o, reinterpret_cast<float*>(smem) + w * X::smem_floats_per_warp(), lane,
                                 k, bx);
    const int j0 = by * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;
    const bool xint = M.i0 > 0 && M.i0 + 64 < g.nx;
    M.start(j0);
    int rowbase = j0 * M.rowA + (int)axis_links_before(j0, g.ny) * M.rowB;
    unsigned long long tie_rows = 0ull;
    // the warp's path is fixed for its interior rows (j and k interior): the
    // rows at j = 0 and j = ny - 1, and every row of a boundary plane, take
    // the general path.  One loop per path instead of a choice per row:
    // +2.3 % at 512 x 512 x 256; unrolling the loop by two was 10 % slower
    // (more registers live across the two rows).
    int j = j0;
    if (zint) {
        if (j == 0 && j < j1) xmarch_row<0>(M, j++, j0, rowbase, tie_rows);
        const int jend = min(j1, g.ny - 1);
        if (xint) {
#pragma unroll 1
            for (; j < jend; ++j) xmarch_row<2>(M, j, j0, rowbase, tie_rows);
        } else {
#pragma unroll 1
            for (; j < jend; ++j) xmarch_row<1>(M, j, j0, rowbase, tie_rows);
        }
    }
    for (; j < j1; ++j) xmarch_row<0>(M, j, j0, rowbase, tie_rows);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (M.v16) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (tie_rows) {  // warp-uniform; every bulk store of the warp has completed
        __syncwarp();
        for (int b = 0; b < 64; ++b)
            if ((tie_rows >> b) & 1ull) {
                naive_row<float, CRK, true>(g, q, f, o, M.act, M.ia, j0 + b, k);
                naive_row<float, CRK, true>(g, q, f, o, M.act, M.ib, j0 + b, k);
            }
    }
}

template <bool DIAG, bool CRK, int W, bool FAST>
__global__ void __launch_bounds__(32 * W, W == 4 ? 3 : 1)
    k_assemble_xmarch(GridGeom g, PhysF q, AsmFields<float> f, AsmOut<float> o, int JY, int k0, int k1) {
    extern __shared__ __align__(16) unsigned char smem[];
    int bx, by, bz;
    segment_major(bx, by, bz);
    xmarch_tile<DIAG, CRK, W, FAST>(g, q, f, o, JY, bx, by, bz, smem, k0, k1);
}

}  // namespace tpfa
