// tpfa_xvjp.cuh -- the mixed path's adjoint march with two cells per lane
// (sm_103a).
//
// The adjoint of the residual (the gradients g_p = J^T v and g_lnk of the
// comment at the top of tpfa_vjp.cu) computed the way the two-cell assembly
// march (tpfa_xmarch.cuh) computes the residual: a warp owns a 64-cell
// x-segment of one z-plane and marches along y; lane l owns the cells
// a = i0 + 2l and b = a + 1 of each row, so the links, the per-link terms
//   dF_iL/dp_i (v_i - v_L)                     (g_p)
//   F_iL Upsilon_iL (d/A)_iL / (2 k_i) (v_i - v_L)   (g_lnk)
// and their FP32 Kahan sums are FP32x2 instructions whose halves are the two
// cells.  The links come from link_pp, the x-links and the links into row
// j-1 are reused by negation as in the assembly; a row where any link has
// zero flux (every exact tie among them) is recomputed after the march by
// the one-thread-per-cell row of tpfa_vjp.cu, which adds the tie terms.
// Every half performs the one-cell row's operations in its order, so the
// results equal that row's bit for bit.
//
// Inputs of row j+2 are requested while row j is computed: the pair-valued
// fields as one 8-byte cp.async per lane, m^n and the split cotangent (hi,
// lo of both cells; own, z-1, z+1) as 16-byte copies, the halo cells' values
// (lanes 0 and 31) as 4- and 8-byte copies, into a per-warp three-slot
// ring (rows j, j+1 and j+2), so row j's inputs are read where they are used.
// Requires nx even and pair-aligned fields (the launcher checks).
#pragma once

#include "tpfa_xmarch.cuh"

namespace tpfa {

template <bool DIAG, bool CRK>
struct XVLayout {
    // pair fields, 64 floats each per slot
    enum { P_P, P_Z, P_TX, P_TY, P_TZ, P_TPP, P_TMP, P_PN, P_K, P_PZM, P_ZZM, P_TZM, P_PZP, P_ZZP, P_PHI };
    static constexpr int NP = CRK ? P_PHI + 1 : P_PHI;
    static constexpr int OFF_MN = NP * 64;      // 32 lanes x 2 doubles
    static constexpr int OFF_V = OFF_MN + 128;  // 32 lanes x (hi_a, lo_a, hi_b, lo_b)
    static constexpr int OFF_VZM = OFF_V + 128;
    static constexpr int OFF_VZP = OFF_VZM + 128;
    // halo cells of lanes 0 / 31: p, z, T1, T2 at 2 f + side, then (hi, lo) at 8 + 2 side
    static constexpr int OFF_H = OFF_VZP + 128;
    static constexpr int SLOT = OFF_H + 12;
    // rows j, j+1 and j+2 (in flight): row j's inputs stay in shared memory
    // while it is computed and are read where they are used
    static constexpr int RING = 3;
    static_assert(SLOT % 4 == 0 && OFF_MN % 4 == 0, "16-byte aligned slot fields");
};

template <bool DIAG, bool CRK, int W>
constexpr int xvjp_smem_bytes() {
    return W * XVLayout<DIAG, CRK>::RING * XVLayout<DIAG, CRK>::SLOT * 4;
}

// The cotangent of one row as FP32 pairs: hi, lo of cells (a, b), and of the
// cells left of a (m) and right of b (p).
struct VRow2 {
    float2 hi, lo;
    float mh, ml, ph, pl;
};

// x - y for FP32 pairs, each half rounded once (the fused form of a
// subtraction: the product by -1 is exact).
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2(-1.f), x); }

// The row's slots: per slot, (F, dF/dp_own) of cells (a, b), the link's T
// and the far cell's v (hi, lo) for each cell.
struct XVSlot {
    float2 F, Da, T, vh, vl;
};

template <bool DIAG, bool CRK, int W>
struct XVState {
    using X = XVLayout<DIAG, CRK>;
    using XS = XState<DIAG, CRK, W, false>;
    static constexpr unsigned kFull = DIAG ? 0x7ffu : 0x575u;
    static constexpr unsigned kXMinus = 0x92u & kFull;  // slots 1, 4, 7
    static constexpr unsigned kXPlus = 0x248u & kFull;  // slots 3, 6, 9

    const GridGeom& g;
    const PhysF& q;
    const AsmFields<float>& f;
    const float* kp;
    const float2* v;
    float* ring;
    int lane, k, nx, ny, nxy, kb, i0, ia, ib, ih;
    bool act, hl, hact, zm, zp;

    // window: row j (C), the halo cell of rows j and j-1, x-neighbours of
    // row j, the links and T of row j-1 into row j, v of rows j-1 and j
    CellPair Cc;
    CellVal<float> Ch, Ph, Cm, Cp;
    Link2 Uy, Uxy, Umxy;
    float2 Typ, Tppp, Tmpp;
    VRow2 vP, vC;

    __device__ __forceinline__ XVState(const GridGeom& g_, const PhysF& q_, const AsmFields<float>& f_,
                                       const float* kp_, const float2* v_, float* ring_, int lane_, int k_, int bx)
        : g(g_), q(q_), f(f_), kp(kp_), v(v_), ring(ring_), lane(lane_), k(k_) {
        nx = g.nx;
        ny = g.ny;
        nxy = nx * ny;
        kb = nxy * k;
        i0 = bx * 64;
        ia = i0 + 2 * lane;
        ib = ia + 1;
        act = ia < nx;  // nx even: then ib < nx too
        hl = lane == 31;
        ih = hl ? i0 + 64 : i0 - 1;
        hact = (lane == 0 || hl) && ih >= 0 && ih < nx;
        zm = k > 0;
        zp = k + 1 < g.nz;
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
        cpa8(Sl + X::P_K * 64, kp + c, a);
        if (CRK) cpa8(Sl + X::P_PHI * 64, f.phi0 + c, a);
        const int cm = zm ? c - nxy : c, cp = zp ? c + nxy : c;
        cpa8(Sl + X::P_PZM * 64, f.p + cm, a && zm);
        cpa8(Sl + X::P_ZZM * 64, f.z + cm, a && zm);
        cpa8(Sl + X::P_TZM * 64, f.Tz + cm, a && zm);
        cpa8(Sl + X::P_PZP * 64, f.p + cp, a && zp);
        cpa8(Sl + X::P_ZZP * 64, f.z + cp, a && zp);
        cpa16(S + X::OFF_MN + 4 * lane, f.mn + c, a);
        cpa16(S + X::OFF_V + 4 * lane, v + c, a);
        cpa16(S + X::OFF_VZM + 4 * lane, v + cm, a && zm);
        cpa16(S + X::OFF_VZP + 4 * lane, v + cp, a && zp);
        if (lane == 0 || hl) {
            const int side = hl ? 1 : 0;
            float* H = S + X::OFF_H;
            const int ch = kb + nx * (rv ? r : 0) + (hact ? ih : 0);
            cpa4(H + side, f.p + ch, rv && hact);
            cpa4(H + 2 + side, f.z + ch, rv && hact);
            // lane 0: Tx(i0-1, r) and Tpp(i0-1, r-1); lane 31: Tmp(i0+64, r-1)
            const bool t1 = rv && hact && !hl;
            cpa4(H + 4 + side, f.Tx + (t1 ? ch : 0), t1);
            if (DIAG) {
                const bool t2 = rv && hact && r > 0;
                cpa4(H + 6 + side, (hl ? f.Tmp : f.Tpp) + (t2 ? ch - nx : 0), t2);
            }
            cpa8(H + 8 + 2 * side, reinterpret_cast<const float*>(v + ch), rv && hact);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __device__ __forceinline__ float2 pair_at(int sl, int fld) const {
        return *reinterpret_cast<const float2*>(ring + sl * X::SLOT + fld * 64 + 2 * lane);
    }
    __device__ __forceinline__ float halo_at(int sl, int fld) const {
        return ring[sl * X::SLOT + X::OFF_H + 2 * fld + (hl ? 1 : 0)];
    }
    // v of the row in slot sl (own cells, and the halo cell at lanes 0 / 31)
    // with its x-neighbours: m = a - 1, p = b + 1
    __device__ __forceinline__ VRow2 vrow(int sl) const {
        const float4 t = *reinterpret_cast<const float4*>(ring + sl * X::SLOT + X::OFF_V + 4 * lane);
        const float2 h = *reinterpret_cast<const float2*>(ring + sl * X::SLOT + X::OFF_H + 8 + (hl ? 2 : 0));
        VRow2 r;
        r.hi = f2(t.x, t.z);
        r.lo = f2(t.y, t.w);
        r.mh = __shfl_up_sync(0xffffffffu, t.z, 1);
        r.ml = __shfl_up_sync(0xffffffffu, t.w, 1);
        r.ph = __shfl_down_sync(0xffffffffu, t.x, 1);
        r.pl = __shfl_down_sync(0xffffffffu, t.y, 1);
        if (lane == 0) r.mh = h.x, r.ml = h.y;
        if (hl) r.ph = h.x, r.pl = h.y;
        return r;
    }
    __device__ __forceinline__ void vz(int sl, int off, float2& hi, float2& lo) const {
        const float4 t = *reinterpret_cast<const float4*>(ring + sl * X::SLOT + off + 4 * lane);
        hi = f2(t.x, t.z);
        lo = f2(t.y, t.w);
    }
    __device__ __forceinline__ void cells_of(int sl, CellPair& Cr, CellVal<float>& Hr) const {
        const float2 pp = pair_at(sl, X::P_P), zz = pair_at(sl, X::P_Z);
        const CellVal<float> ca = make_cell(q, pp.x, zz.x), cb = make_cell(q, pp.y, zz.y);
        Cr = CellPair{pp, zz, f2(ca.rho, cb.rho), f2(ca.drho, cb.drho)};
        Hr = make_cell(q, halo_at(sl, 0), halo_at(sl, 1));
    }
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

    // Prologue of a march starting at row j0: rows j0-1 (slot 0) and j0
    // (slot 1), the links and T of row j0-1 into row j0; row j0+1 requested
    // into slot 2.
    __device__ __forceinline__ void start(int j0) {
        issue(j0 - 1, 0);
        issue(j0, 1);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        CellPair Pc;
        cells_of(0, Pc, Ph);
        cells_of(1, Cc, Ch);
        neighbours(Cc, Ch, Cm, Cp);
        Typ = pair_at(0, X::P_TY);
        Tppp = DIAG ? pair_at(0, X::P_TPP) : f2(0.f);
        Tmpp = DIAG ? pair_at(0, X::P_TMP) : f2(0.f);
        Uy = link_pp(q, Typ, Pc, Cc);
        if (DIAG) {
            Uxy = link_pp(q, Tppp, Pc, XS::shift_left(Cc, Cp));
            Umxy = link_pp(q, Tmpp, Pc, XS::shift_right(Cm, Cc));
        }
        vP = vrow(0);
        vC = vrow(1);
        issue(j0 + 1, 2);
    }

    // One slot's terms for both cells into the two Kahan pairs (g_p and
    // g_lnk), in slot order; va / vb: the slot exists for cell a / b (PATH 2:
    // always; PATH 1: x-slots of the boundary cells; PATH 0: per-cell masks).
    template <int PATH, int S>
    __device__ __forceinline__ void term(const XVSlot& s, float2 vch, float2 vcl, float2 inv2k, Kahan2& kpp,
                                         Kahan2& kkk, bool va, bool vb, bool& zero) const {
        if constexpr (!((kFull >> S) & 1u)) return;
        const float2 dv = __fadd2_rn(sub2(vch, s.vh), sub2(vcl, s.vl));
        const float2 ratio = __fmul2_rn(s.T, inv2k);  // s.T holds T (d/A) already
        const float2 tp = __fmul2_rn(s.Da, dv);
        const float2 tk = __fmul2_rn(__fmul2_rn(s.F, ratio), dv);
        if constexpr (PATH == 2) {
            kpp.add(tp);
            kkk.add(tk);
            zero = zero || s.F.x == 0.f || s.F.y == 0.f;
        } else {
            constexpr bool xm = (kXMinus >> S) & 1u, xp = (kXPlus >> S) & 1u;
            if (PATH == 1 && !xm && !xp) {
                kpp.add(tp);
                kkk.add(tk);
                zero = zero || s.F.x == 0.f || s.F.y == 0.f;
            } else {
                kahan2_masked(kpp, tp, va, vb);
                kahan2_masked(kkk, tk, va, vb);
                zero = zero || (va && s.F.x == 0.f) || (vb && s.F.y == 0.f);
            }
        }
    }

    // Row j: its inputs are in slot sD, row j+1's in slot sN; row j+2 is
    // requested into slot sI.  Writes g_p and g_lnk of cells a and b;
    // returns whether a link of the row had zero flux (warp-uniform).
    template <int PATH>
    __device__ __forceinline__ bool row(int j, int sD, int sN, int sI, const LinkGeo& lg, double* gP, double* gK,
                                        bool out16, unsigned int* status) {
        issue(j + 2, sI);
        CellPair Nc;
        CellVal<float> Nh;
        cells_of(sN, Nc, Nh);
        const VRow2 vN = vrow(sN);
        const float2 Tx = pair_at(sD, X::P_TX), Ty = pair_at(sD, X::P_TY), Tz = pair_at(sD, X::P_TZ);
        const float2 Tpp = DIAG ? pair_at(sD, X::P_TPP) : f2(0.f), Tmp = DIAG ? pair_at(sD, X::P_TMP) : f2(0.f);
        const float2 kk = pair_at(sD, X::P_K);
        const float hT1 = halo_at(sD, 2), hT2 = DIAG ? halo_at(sD, 3) : 0.f;

        // validity of the x-slots (PATH 1) or of every slot (PATH 0)
        unsigned ma = kFull, mb = kFull;
        if constexpr (PATH == 1) {
            if (ia == 0) ma &= ~kXMinus;
            if (ib == nx - 1) mb &= ~kXPlus;
        } else if constexpr (PATH == 0) {
            ma = slot_mask(g, act ? ia : 0, j, k);
            mb = slot_mask(g, act ? ib : 1, j, k);
        }
        const float2 inv2k = f2(kk.x > 0.f ? __fdiv_rn(0.5f, kk.x) : 0.f, kk.y > 0.f ? __fdiv_rn(0.5f, kk.y) : 0.f);
        Kahan2 kpp, kkk;
        bool zero = false;
        const float2 gz = f2(lg.cz), gy = f2(lg.cy), gx = f2(lg.cx), gd = f2(lg.cd);
#define XV_TERM(S_, slot_) \
    term<PATH, S_>(slot_, vC.hi, vC.lo, inv2k, kpp, kkk, (ma >> S_) & 1u, (mb >> S_) & 1u, zero)

        // slot 0: -z
        {
            const float2 pzm = pair_at(sD, X::P_PZM), zzm = pair_at(sD, X::P_ZZM), tzm = pair_at(sD, X::P_TZM);
            float2 vzmh, vzml;
            vz(sD, X::OFF_VZM, vzmh, vzml);
            CellPair Zm;
            {
                const CellVal<float> a0 = make_cell(q, pzm.x, zzm.x), b0 = make_cell(q, pzm.y, zzm.y);
                Zm = XS::pair2(a0, b0);
            }
            const Link2 L = link_pp(q, tzm, Cc, Zm);
            XV_TERM(0, (XVSlot{L.F, L.Da, __fmul2_rn(tzm, gz), vzmh, vzml}));
        }
        // the segment's halo links: lane 0 -> a's -x (halo of row j) and -x-y
        // (halo of row j-1); lane 31 -> b's +x-y (halo of row j-1)
        Link2 LH;
        {
            const CellVal<float> own = hl ? CellVal<float>{Cc.p.y, Cc.z.y, Cc.rho.y, Cc.drho.y}
                                          : CellVal<float>{Cc.p.x, Cc.z.x, Cc.rho.x, Cc.drho.x};
            LH = link_pp(q, hl ? f2(hT2, 0.f) : f2(hT1, hT2), XS::pair2(own, own), XS::pair2(hl ? Ph : Ch, Ph));
        }
        if (DIAG) {  // slot 1: -x-y
            const float f1 = __shfl_up_sync(0xffffffffu, Uxy.F.y, 1), b1 = __shfl_up_sync(0xffffffffu, Uxy.Db.y, 1);
            const float t1 = __shfl_up_sync(0xffffffffu, Tppp.y, 1);
            const float Fa = lane == 0 ? LH.F.y : -f1, Da = lane == 0 ? LH.Da.y : -b1;
            const float Ta = lane == 0 ? hT2 : t1;
            XV_TERM(1, (XVSlot{f2(Fa, -Uxy.F.x), f2(Da, -Uxy.Db.x), __fmul2_rn(f2(Ta, Tppp.x), gd), f2(vP.mh, vP.hi.x),
                               f2(vP.ml, vP.lo.x)}));
        }
        // slot 2: -y
        XV_TERM(2, (XVSlot{neg2(Uy.F), neg2(Uy.Db), __fmul2_rn(Typ, gy), vP.hi, vP.lo}));
        if (DIAG) {  // slot 3: +x-y
            const float f3 = __shfl_down_sync(0xffffffffu, Umxy.F.x, 1),
                        b3 = __shfl_down_sync(0xffffffffu, Umxy.Db.x, 1);
            const float t3 = __shfl_down_sync(0xffffffffu, Tmpp.x, 1);
            const float Fb = hl ? LH.F.x : -f3, Db = hl ? LH.Da.x : -b3;
            const float Tb = hl ? hT2 : t3;
            XV_TERM(3, (XVSlot{f2(-Umxy.F.y, Fb), f2(-Umxy.Db.y, Db), __fmul2_rn(f2(Tmpp.y, Tb), gd),
                               f2(vP.hi.y, vP.ph), f2(vP.lo.y, vP.pl)}));
        }
        const Link2 LX_ = link_pp(q, Tx, Cc, XS::shift_left(Cc, Cp));
        {  // slot 4: -x
            const float f4 = __shfl_up_sync(0xffffffffu, LX_.F.y, 1), b4 = __shfl_up_sync(0xffffffffu, LX_.Db.y, 1);
            const float t4 = __shfl_up_sync(0xffffffffu, Tx.y, 1);
            const float Fa = lane == 0 ? LH.F.x : -f4, Da = lane == 0 ? LH.Da.x : -b4;
            const float Ta = lane == 0 ? hT1 : t4;
            XV_TERM(4, (XVSlot{f2(Fa, -LX_.F.x), f2(Da, -LX_.Db.x), __fmul2_rn(f2(Ta, Tx.x), gx), f2(vC.mh, vC.hi.x),
                               f2(vC.ml, vC.lo.x)}));
        }
        // slot 6: +x
        XV_TERM(6, (XVSlot{LX_.F, LX_.Da, __fmul2_rn(Tx, gx), f2(vC.hi.y, vC.ph), f2(vC.lo.y, vC.pl)}));
        CellVal<float> Nm, Np;
        neighbours(Nc, Nh, Nm, Np);
        Link2 LMXY, LXY;
        if (DIAG) {  // slot 7: -x+y
            LMXY = link_pp(q, Tmp, Cc, XS::shift_right(Nm, Nc));
            XV_TERM(7, (XVSlot{LMXY.F, LMXY.Da, __fmul2_rn(Tmp, gd), f2(vN.mh, vN.hi.x), f2(vN.ml, vN.lo.x)}));
        }
        // slot 8: +y
        const Link2 LY = link_pp(q, Ty, Cc, Nc);
        XV_TERM(8, (XVSlot{LY.F, LY.Da, __fmul2_rn(Ty, gy), vN.hi, vN.lo}));
        if (DIAG) {  // slot 9: +x+y
            LXY = link_pp(q, Tpp, Cc, XS::shift_left(Nc, Np));
            XV_TERM(9, (XVSlot{LXY.F, LXY.Da, __fmul2_rn(Tpp, gd), f2(vN.hi.y, vN.ph), f2(vN.lo.y, vN.pl)}));
        }
        {  // slot 10: +z
            const float2 pzp = pair_at(sD, X::P_PZP), zzp = pair_at(sD, X::P_ZZP);
            float2 vzph, vzpl;
            vz(sD, X::OFF_VZP, vzph, vzpl);
            CellPair Zp;
            {
                const CellVal<float> a1 = make_cell(q, pzp.x, zzp.x), b1 = make_cell(q, pzp.y, zzp.y);
                Zp = XS::pair2(a1, b1);
            }
            const Link2 L = link_pp(q, Tz, Cc, Zp);
            XV_TERM(10, (XVSlot{L.F, L.Da, __fmul2_rn(Tz, gz), vzph, vzpl}));
        }
#undef XV_TERM
        const bool fix = __any_sync(0xffffffffu, act && zero);

        // the cells' own terms v_i dA_i/dp_i (one fused FP32 product of the
        // pair), then the FP64 combinations
        const float2 pn = pair_at(sD, X::P_PN), phi = CRK ? pair_at(sD, X::P_PHI) : f2(0.f);
        const double2 mn = *reinterpret_cast<const double2*>(ring + sD * X::SLOT + X::OFF_MN + 4 * lane);
        const AccF acc_a = accumulation<CRK>(q, Cc.p.x, pn.x, mn.x, Cc.rho.x, phi.x);
        const AccF acc_b = accumulation<CRK>(q, Cc.p.y, pn.y, mn.y, Cc.rho.y, phi.y);
        const float2 dA = f2(acc_a.dA, acc_b.dA);
        kpp.add(__ffma2_rn(vC.hi, dA, __fmul2_rn(vC.lo, dA)));
        if (act) {
            const double gpa = __dadd_rn(__dadd_rn(widen(kpp.s.x), -widen(kpp.c.x)), 0.0);
            const double gpb = __dadd_rn(__dadd_rn(widen(kpp.s.y), -widen(kpp.c.y)), 0.0);
            const double gka = __dadd_rn(widen(kkk.s.x), -widen(kkk.c.x));
            const double gkb = __dadd_rn(widen(kkk.s.y), -widen(kkk.c.y));
            const int c = kb + nx * j + ia;
            if (out16) {
                *reinterpret_cast<double2*>(gP + c) = make_double2(gpa, gpb);
                if (gK) *reinterpret_cast<double2*>(gK + c) = make_double2(gka, gkb);
            } else {
                gP[c] = gpa, gP[c + 1] = gpb;
                if (gK) gK[c] = gka, gK[c + 1] = gkb;
            }
            if (nonfinite(gpa) || nonfinite(gpb) || nonfinite(gka) || nonfinite(gkb)) atomicOr(status, STATUS_NONFINITE);
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
        Typ = Ty;
        Tppp = Tpp;
        Tmpp = Tmp;
        vP = vC;
        vC = vN;
        return fix;
    }
};

}  // namespace tpfa
