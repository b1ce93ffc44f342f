// tpfa_ymarch.cuh -- the production assembly kernel (sm_103a).
//
// A warp owns a 32-cell x-segment (cells i0 .. i0+31) of one z-plane k and
// marches along y over a run of JY rows; a block stacks W warps on W
// consecutive planes (their vertical neighbours then hit in L1).  Per row j
// each lane assembles row (i, j, k) of Algorithm 1 / Eq. vk:
//
//   * rows j-1, j, j+1 of (p, z, rho, rho') live in registers ({c, m, p} =
//     the lane's cell and its x-neighbours, obtained by shuffles; lanes 0 and
//     31 carry the halo cells i0-1 and i0+32), so each density is evaluated
//     once per row it enters;
//   * seven links are evaluated from the lane's own side: -z, -x, +x, the
//     three links into row j+1 (-x+y, +y, +x+y) and +z;
//   * the three links into row j-1 are the negations of the previous step's
//     links into row j (the lane's own +y, the left neighbour's +x+y and the
//     right neighbour's -x+y, fetched by shuffles): F_LK = -F_KL and the two
//     derivatives swap and change sign, bit for bit.  Lanes 0 and 31 evaluate
//     the one such link whose far end lies in the halo.  An exact tie
//     dPhi == 0 breaks that symmetry (each end takes the other cell as
//     upstream), so a warp that meets one re-evaluates those links directly;
//   * rows with all ten neighbours (the interior) take a path with fixed slot
//     positions; rows of a segment at an x boundary (j and k interior) take a
//     path whose masks and offsets differ only in the edge lanes; the other
//     boundary rows use per-slot validity masks;
//   * the warp's Jacobian rows form one contiguous CSR segment whose offset is
//     a closed form of (i0, j, k) (the y-row part advanced incrementally along
//     the march); values are staged in shared memory at their
//     offsets and written with 16-byte stores;
//   * every input of row j+2 is requested with cp.async into a per-warp
//     shared-memory ring at the start of step j, so loads are in flight a
//     whole step ahead without holding registers.  Registers are capped at
//     128 for FP32 (16 warps per SM) and 255 for FP64 (whose bound is the
//     FP64 pipe, not latency).
//
// Every value goes through the same link()/accumulation() arithmetic and the
// same summation order as assemble_row(), so this kernel and the naive one
// produce identical bits.
//
// The same march also drives the matrix-free Jacobian-vector product of the
// mixed path (JV = true, tpfa_jvp.cu): w joins the prefetched row inputs and
// each row emits (J w)_K instead of a CSR row.
#pragma once

#include <type_traits>

#include "tpfa_row.cuh"
#include "tpfa_tma.cuh"

namespace tpfa {

template <typename Real>
struct YRow {
    CellVal<Real> c, m, p;  // cells (i, j), (i-1, j), (i+1, j) of this lane
};

template <typename Real>
struct YIn {  // inputs of one row other than p and z
    Real Tx, Ty, Tz, Tpp, Tmp, pn, phi0;
    double mn;
    Real p_zm, z_zm, p_zp, z_zp, Tz_m;
    Real hT1, hT2;  // lane 0: Tx(i0-1, j), Tpp(i0-1, j-1); lane 31: Tmp(i0+32, j-1)
};

template <typename Real>
struct YUp {  // a link from row j-1 into row j, seen from row j-1
    LinkOut<Real> y, xy, mxy;  // to (i, j), (i+1, j), (i-1, j)
    bool tie;                  // any of the three had dPhi == 0 exactly
};

template <typename Real>
__device__ __forceinline__ Real vshfl_up(Real v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename Real>
__device__ __forceinline__ Real vshfl_down(Real v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

__device__ __forceinline__ float drho_of(const PhysF& q, float rho) { return __fmul_rn(q.c_f, rho); }
__device__ __forceinline__ double drho_of(const PhysD& q, double rho) { return __dmul_rn(q.c_f, rho); }

// A link and whether it may be an exact tie: dPhi == 0 forces F == 0, so
// F == 0 on a link with T != 0 flags every tie (and, harmlessly, fluxes that
// underflow to zero).
template <typename Real, typename Phys>
__device__ __forceinline__ LinkOut<Real> link_t(const Phys& q, Real T, const CellVal<Real>& a,
                                                const CellVal<Real>& b, bool& tie) {
    const LinkOut<Real> r = link(q, T, a, b);
    tie = (r.F == Real(0)) && (T != Real(0));
    return r;
}

// w of one row for the Jacobian-vector product (FP32): the lane's cell and
// its x-neighbours.
struct YW {
    float c, m, p;
};

// v of one row for the adjoint as split doubles (hi + lo): the lane's cell
// and the lane's halo cell (lanes 0 and 31); x-neighbours by shuffles where
// used.
struct YV {
    F2Split c, h;
};

template <typename Real, bool DIAG, bool CRK, bool JAC, int W, bool JV = false, bool VJ = false>
struct YMarch {
    static_assert(!JV || (sizeof(Real) == 4 && !JAC), "the J w march is the mixed path's, without CSR values");
    static_assert(!VJ || (sizeof(Real) == 4 && !JAC && !JV), "the adjoint march is the mixed path's");
    using Phys = typename PhysOf<Real>::type;
    static constexpr int VEC = 16 / (int)sizeof(Real);  // elements per 16-byte store

    const GridGeom& g;
    const Phys& q;
    const AsmFields<Real>& f;
    const AsmOut<Real>& o;
    int lane, i0, i, k, nx, ny, nxy, kb, ih;
    bool act, hact, zm, zp, xint, v16;
    long long base_k;
    int rowA, rowB;  // CSR entries per y-row of plane k: rowA + (y links of the row) rowB
    int X2;          // offset of this segment within a y-row whose j and k are interior
    int Sx0, ez;

    __device__ __forceinline__ YMarch(const GridGeom& g_, const Phys& q_, const AsmFields<Real>& f_,
                                      const AsmOut<Real>& o_, int lane_, int i0_, int k_)
        : g(g_), q(q_), f(f_), o(o_), lane(lane_), i0(i0_), i(i0_ + lane_), k(k_) {
        nx = g.nx;
        ny = g.ny;
        nxy = nx * ny;
        kb = nxy * k;
        act = i < nx;
        ih = lane == 0 ? i0 - 1 : (lane == 31 ? i0 + 32 : -1);
        hact = ih >= 0 && ih < nx;
        zm = k > 0;
        zp = k + 1 < g.nz;
        xint = i0 > 0 && i0 + 32 < nx;
        v16 = (reinterpret_cast<uintptr_t>(o.vals) & 15u) == 0;
        const long long Ex = 2LL * (nx - 1), Ey = 2LL * (ny - 1), D = g.diag;
        const long long plane = (long long)nx * ny + Ex * ny + (long long)nx * Ey + D * Ex * Ey;
        ez = axis_links(k, g.nz);
        base_k = (long long)k * plane + (long long)nxy * axis_links_before(k, g.nz);
        rowA = (int)(nx + Ex + (long long)nx * ez);
        rowB = (int)(nx + D * Ex);
        Sx0 = (int)axis_links_before(i0, nx);
        X2 = i0 * (3 + ez) + Sx0 * (int)(1 + 2 * D);
    }

    // CSR offset of row (0, j, k) relative to the plane's first row (one
    // plane's rows number fewer than 2^31: the grid has fewer than 2^31 / 11
    // cells per plane whenever its pattern is addressable).
    __device__ __forceinline__ int row_base(int j) const {
        return j * rowA + (int)axis_links_before(j, ny) * rowB;
    }
    __device__ __forceinline__ int row_base_step(int j) const { return rowA + axis_links(j, ny) * rowB; }

    // Row kinds: 2 = every neighbour exists (interior x-segment, j and k
    // interior); 1 = j and k interior in a segment that touches an x boundary
    // (the lanes at i = 0 and i = nx - 1 lack their -x or +x links); 0 = any
    // other row.
    static constexpr unsigned kFullMask = DIAG ? 0x7ffu : 0x575u;
    static constexpr unsigned kXMinus = 0x92u;   // slots 1, 4, 7
    static constexpr unsigned kXPlus = 0x248u;   // slots 3, 6, 9
    template <int PATH>
    __device__ __forceinline__ unsigned row_mask(int j) const {
        if constexpr (PATH == 2) {
            return kFullMask;
        } else if constexpr (PATH == 1) {
            unsigned m = kFullMask;
            if (i == 0) m &= ~kXMinus;
            if (i == nx - 1) m &= ~kXPlus;
            return m;
        } else {
            return slot_mask(g, i, j, k);
        }
    }

    // ---- row inputs, prefetched into a per-warp shared-memory ring of RING
    // rows with cp.async (4- or 8-byte copies by each lane; lanes whose value
    // does not exist copy nothing and get zeros).  Field f of the row in ring
    // slot s for lane l lives at ring[s * NF * 32 + f * 32 + l]; m^n at
    // ringm[s * 32 + l].  Slots rotate explicitly (no modulo per access).
    static constexpr int RING = 3;
    enum { F_P, F_Z, F_HP, F_HZ, F_TX, F_TY, F_TZ, F_TPP, F_TMP, F_PN, F_PHI, F_PZM, F_ZZM, F_TZM, F_PZP, F_ZZP,
           F_HT1, F_HT2, F_K };
    static constexpr int NF = VJ ? F_K + 1 : F_K;  // the adjoint also prefetches the cell's k
    Real* ring;      // RING * NF * 32 values
    double* ringm;   // RING * 32 values of m^n
    // J w mode: RING * NW * 32 values of w (own, halo, z-1, z+1), the
    // direction w and the output
    static constexpr int NW = 4;
    double* ringw = nullptr;
    const double* wv = nullptr;
    double* Jw = nullptr;
    // adjoint mode: k of the field type, the link geometry, the two gradients
    const Real* kperm = nullptr;
    LinkGeo lg{};
    double* gP = nullptr;
    double* gK = nullptr;

    __device__ __forceinline__ void cp4(Real* dst, const Real* src, bool valid) const {
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
        const int n = valid ? (int)sizeof(Real) : 0;
        if constexpr (sizeof(Real) == 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    }
    __device__ __forceinline__ void cp8(double* dst, const double* src, bool valid) const {
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
    }
    // Request every input of row r into ring slot sl (a row outside the grid
    // requests nothing).
    __device__ __forceinline__ void issue_row(int r, int sl) const {
        Real* R = ring + sl * (NF * 32) + lane;
        const bool rv = r >= 0 && r < ny;
        const int c = kb + nx * (rv ? r : 0) + (act ? i : 0);
        const bool a = rv && act;
        cp4(R + F_P * 32, f.p + c, a);
        cp4(R + F_Z * 32, f.z + c, a);
        const int ch = kb + nx * (rv ? r : 0) + (hact ? ih : 0);
        cp4(R + F_HP * 32, f.p + ch, rv && hact);
        cp4(R + F_HZ * 32, f.z + ch, rv && hact);
        cp4(R + F_TX * 32, f.Tx + c, a);
        cp4(R + F_TY * 32, f.Ty + c, a);
        cp4(R + F_TZ * 32, f.Tz + c, a);
        if (DIAG) {
            cp4(R + F_TPP * 32, f.Tpp + c, a);
            cp4(R + F_TMP * 32, f.Tmp + c, a);
        }
        cp4(R + F_PN * 32, f.pn + c, a);
        if (CRK) cp4(R + F_PHI * 32, f.phi0 + c, a);
        cp4(R + F_PZM * 32, f.p + (zm ? c - nxy : c), a && zm);
        cp4(R + F_ZZM * 32, f.z + (zm ? c - nxy : c), a && zm);
        cp4(R + F_TZM * 32, f.Tz + (zm ? c - nxy : c), a && zm);
        cp4(R + F_PZP * 32, f.p + (zp ? c + nxy : c), a && zp);
        cp4(R + F_ZZP * 32, f.z + (zp ? c + nxy : c), a && zp);
        const bool h1 = rv && lane == 0 && i0 > 0;
        cp4(R + F_HT1 * 32, f.Tx + (h1 ? c - 1 : c), h1);
        if (DIAG) {
            const bool h2l = h1 && r > 0, h2r = rv && lane == 31 && hact && r > 0;
            cp4(R + F_HT2 * 32, h2l ? f.Tpp + (c - nx - 1) : f.Tmp + (h2r ? c - nx + 1 : c), h2l || h2r);
        }
        cp8(ringm + sl * 32 + lane, f.mn + c, a);
        if constexpr (VJ) cp4(R + F_K * 32, kperm + c, a);
        if constexpr (JV || VJ) {
            double* Wr = ringw + sl * (NW * 32) + lane;
            cp8(Wr, wv + c, a);
            cp8(Wr + 32, wv + ch, rv && hact);
            cp8(Wr + 64, wv + (zm ? c - nxy : c), a && zm);
            cp8(Wr + 96, wv + (zp ? c + nxy : c), a && zp);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // Wait until every requested row but the most recent one has arrived
    // (each lane reads back only what it copied itself).
    __device__ __forceinline__ void wait_all_but_newest() const {
        asm volatile("cp.async.wait_group 1;" ::: "memory");
    }
    __device__ __forceinline__ YIn<Real> read_in(int sl) const {
        const Real* R = ring + sl * (NF * 32) + lane;
        YIn<Real> D;
        D.Tx = R[F_TX * 32];
        D.Ty = R[F_TY * 32];
        D.Tz = R[F_TZ * 32];
        D.Tpp = DIAG ? R[F_TPP * 32] : Real(0);
        D.Tmp = DIAG ? R[F_TMP * 32] : Real(0);
        D.pn = R[F_PN * 32];
        D.phi0 = CRK ? R[F_PHI * 32] : Real(0);
        D.mn = ringm[sl * 32 + lane];
        D.p_zm = R[F_PZM * 32];
        D.z_zm = R[F_ZZM * 32];
        D.Tz_m = R[F_TZM * 32];
        D.p_zp = R[F_PZP * 32];
        D.z_zp = R[F_ZZP * 32];
        D.hT1 = R[F_HT1 * 32];
        D.hT2 = DIAG ? R[F_HT2 * 32] : Real(0);
        return D;
    }
    __device__ __forceinline__ YRow<Real> row_cells(int sl) const {
        const Real* R = ring + sl * (NF * 32) + lane;
        return make_row(R[F_P * 32], R[F_Z * 32], R[F_HP * 32], R[F_HZ * 32]);
    }

    // ---- the same row inputs delivered by TMA (the mixed assembly march on
    // grids whose x-rows are 16-byte multiples): the block's W warps own W
    // consecutive x-segments of one plane and share a ring of TRING slots
    // (TmaSlot<W>), each with a "full" mbarrier (one arrival plus the
    // transaction bytes) and an "empty" one (one arrival per warp).  Thread
    // (0, 0) of the block issues every copy; every lane waits on "full".
    static constexpr int TRING = 3;  // slots: rows j-1 (until its refill), j, j+1, ...
    using TS = TmaSlot<W>;
    unsigned char* tring = nullptr;  // the block's first slot (128-byte aligned)
    uint32_t tslot0 = 0, tfull0 = 0, tempty0 = 0;  // shared addresses: first slot, first full / empty barrier
    const TmaMaps* tm = nullptr;
    unsigned tphase = 0u;  // per slot: parity of its next "full" completion
    unsigned ephase = 0u;  // per slot: parity of its next "empty" completion (issuing thread)
    unsigned tpend = 0u;   // per slot: requested and not yet awaited
    int xo = 0;            // this warp's segment within the block's boxes (cells)
    int hx = 0;            // index in a halo box row of the value this lane takes as its x-halo
    bool issuer = false;   // thread (0, 0) of the block

    // Set up the shared ring (slots, TRING full then TRING empty barriers);
    // every thread of the block calls it (it ends with a block barrier).
    __device__ __forceinline__ void tma_init(unsigned char* slots, uint64_t* bars, const TmaMaps* maps, int w) {
        tring = slots;
        tslot0 = smem_u32(slots);
        tfull0 = smem_u32(bars);
        tempty0 = tfull0 + 8u * TRING;
        tm = maps;
        xo = 32 * w;
        hx = xo + (lane == 0 ? 3 : (lane == 31 ? 36 : 4 + lane));
        issuer = w == 0 && lane == 0;
        if (issuer) {
            for (int s = 0; s < TRING; ++s) {
                mbar_init(tfull0 + 8u * s, 1u);
                mbar_init(tempty0 + 8u * s, (unsigned)W);
            }
            mbar_fence_init();
        }
        __syncthreads();
    }
    // Thread (0, 0): request every box of row r (block x-range from X0, plane
    // k) into slot sl; with `refill`, first wait until every warp has
    // released the slot.  False if that wait ran out (nothing is issued).
    __device__ __forceinline__ bool tma_issue(int r, int sl, int X0, bool refill) {
        if (refill) {
            if (!mbar_wait_bounded(tempty0 + 8u * sl, (ephase >> sl) & 1u)) return false;
            ephase ^= 1u << sl;
        }
        const uint32_t d = tslot0 + (uint32_t)(sl * TS::BYTES), b = tfull0 + 8u * sl;
        const int xh = X0 - 4;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(b, TS::tx_bytes(DIAG, CRK));
        tma_load_3d(d + TS::P, &tm->p, xh, r, k - 1, b);
        tma_load_3d(d + TS::Z, &tm->z, xh, r, k - 1, b);
        tma_load_3d(d + TS::TX, &tm->Tx, xh, r, k, b);
        tma_load_3d(d + TS::TY, &tm->Ty, X0, r, k, b);
        tma_load_3d(d + TS::TZ, &tm->Tz, X0, r, k - 1, b);
        if (DIAG) {
            tma_load_3d(d + TS::TPP, &tm->Tpp, xh, r, k, b);
            tma_load_3d(d + TS::TMP, &tm->Tmp, xh, r, k, b);
        }
        tma_load_3d(d + TS::PN, &tm->pn, X0, r, k, b);
        if (CRK) tma_load_3d(d + TS::PHI, &tm->phi, X0, r, k, b);
        tma_load_3d(d + TS::MN, &tm->mn, X0, r, k, b);
        return true;
    }
    // Every warp: the row requested into slot sl is now expected.
    __device__ __forceinline__ void tma_requested(int sl) { tpend |= 1u << sl; }
    // This warp is done with slot sl.
    __device__ __forceinline__ void tma_release(int sl) const {
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8u * sl);
    }
    // Wait for slot sl's row; false (for the whole warp) if the wait ran out.
    __device__ __forceinline__ bool tma_wait(int sl) {
        bool ok = mbar_wait_bounded(tfull0 + 8u * sl, (tphase >> sl) & 1u);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
            tphase ^= 1u << sl;
            tpend &= ~(1u << sl);
        }
        return ok;
    }
    // Wait (bounded) for every slot still expected; false if one ran out.
    __device__ __forceinline__ bool tma_drain() {
        bool ok = true;
        for (int s = 0; s < TRING; ++s)
            if ((tpend >> s) & 1u) ok = tma_wait(s) && ok;
        return ok;
    }
    __device__ __forceinline__ const float* tma_slot(int sl) const {
        return reinterpret_cast<const float*>(tring + sl * TS::BYTES);
    }
    __device__ __forceinline__ YRow<Real> tma_row_cells(int sl) const {
        const float* S = tma_slot(sl);
        constexpr int P1 = TS::P / 4 + TS::HX, Z1 = TS::Z / 4 + TS::HX;  // plane k
        return make_row(S[P1 + xo + 4 + lane], S[Z1 + xo + 4 + lane], S[P1 + hx], S[Z1 + hx]);
    }
    // The diagonal-link T of lanes 0 and 31 into row r - 1 (Tpp(i0 - 1, r - 1)
    // and Tmp(i0 + 32, r - 1)), read from the slot of row r - 1 before it is
    // refilled; 0 in the other lanes.
    __device__ __forceinline__ Real tma_h2(int sl) const {
        if (!DIAG) return Real(0);
        const float* S = tma_slot(sl);
        const float t = lane == 31 ? S[TS::TMP / 4 + xo + 36] : S[TS::TPP / 4 + xo + 3];
        return (lane == 0 || lane == 31) ? t : 0.f;
    }
    __device__ __forceinline__ YIn<Real> tma_read_in(int sl, Real hT2) const {
        const float* S = tma_slot(sl);
        constexpr int P0 = TS::P / 4, Z0 = TS::Z / 4, B = TS::HX;
        const int o = xo + lane, oh = o + 4;  // the lane's cell in a plain box row and in a halo box row
        YIn<Real> D;
        D.Tx = S[TS::TX / 4 + oh];
        D.Ty = S[TS::TY / 4 + o];
        D.Tz = S[TS::TZ / 4 + TS::SX + o];
        D.Tpp = DIAG ? S[TS::TPP / 4 + oh] : Real(0);
        D.Tmp = DIAG ? S[TS::TMP / 4 + oh] : Real(0);
        D.pn = S[TS::PN / 4 + o];
        D.phi0 = CRK ? S[TS::PHI / 4 + o] : Real(0);
        D.mn = reinterpret_cast<const double*>(tring + sl * TS::BYTES + TS::MN)[o];
        D.p_zm = S[P0 + oh];
        D.z_zm = S[Z0 + oh];
        D.Tz_m = S[TS::TZ / 4 + o];
        D.p_zp = S[P0 + 2 * B + oh];
        D.z_zp = S[Z0 + 2 * B + oh];
        D.hT1 = lane == 0 ? S[TS::TX / 4 + xo + 3] : Real(0);  // Tx(i0 - 1, r)
        D.hT2 = hT2;
        return D;
    }

    // w of the row in ring slot sl, narrowed to FP32 on the integer pipe
    // (truncation, below one float ulp), x-neighbours by shuffles.
    __device__ __forceinline__ YW w_row(int sl) const {
        const double* Wr = ringw + sl * (NW * 32) + lane;
        YW r;
        r.c = narrow_rz(Wr[0]);
        const float h = narrow_rz(Wr[32]);
        r.m = vshfl_up(r.c);
        r.p = vshfl_down(r.c);
        if (lane == 0) r.m = h;
        if (lane == 31) r.p = h;
        return r;
    }

    // v of the row in ring slot sl as FP32 pairs (own and halo): in the
    // adjoint mode the ring's 8-byte entries hold the pairs (hi, lo) of the
    // split cotangent, not doubles.
    __device__ __forceinline__ F2Split v_at(int sl, int e) const {
        const float2 t = reinterpret_cast<const float2*>(ringw + sl * (NW * 32) + lane)[32 * e];
        return F2Split{t.x, t.y};
    }
    __device__ __forceinline__ YV v_row(int sl) const { return YV{v_at(sl, 0), v_at(sl, 1)}; }
    __device__ __forceinline__ F2Split v_minus(const YV& v) const {
        F2Split t{__shfl_up_sync(0xffffffffu, v.c.hi, 1), __shfl_up_sync(0xffffffffu, v.c.lo, 1)};
        return lane == 0 ? v.h : t;
    }
    __device__ __forceinline__ F2Split v_plus(const YV& v) const {
        F2Split t{__shfl_down_sync(0xffffffffu, v.c.hi, 1), __shfl_down_sync(0xffffffffu, v.c.lo, 1)};
        return lane == 31 ? v.h : t;
    }

    __device__ __forceinline__ YRow<Real> make_row(Real po, Real zo, Real ph, Real zh) const {
        YRow<Real> R;
        R.c = make_cell(q, po, zo);
        const CellVal<Real> h = make_cell(q, ph, zh);
        R.m.p = vshfl_up(R.c.p);
        R.m.z = vshfl_up(R.c.z);
        R.m.rho = vshfl_up(R.c.rho);
        R.p.p = vshfl_down(R.c.p);
        R.p.z = vshfl_down(R.c.z);
        R.p.rho = vshfl_down(R.c.rho);
        if (lane == 0) R.m = h;
        if (lane == 31) R.p = h;
        R.m.drho = drho_of(q, R.m.rho);
        R.p.drho = drho_of(q, R.p.rho);
        return R;
    }
    // Links from row r into row r+1, seen from row r (cells of rows r and r+1).
    __device__ __forceinline__ YUp<Real> up_links(const YRow<Real>& R, const YRow<Real>& Nx, Real Ty, Real Tpp,
                                                  Real Tmp) const {
        YUp<Real> U;
        bool t0, t1 = false, t2 = false;
        U.y = link_t(q, Ty, R.c, Nx.c, t0);
        if (DIAG) {
            U.xy = link_t(q, Tpp, R.c, Nx.p, t1);
            U.mxy = link_t(q, Tmp, R.c, Nx.m, t2);
        }
        U.tie = t0 || t1 || t2;
        return U;
    }

    // The ten links of row j (slot order), and the links from row j into
    // row j+1 for the next step.  The links into row j-1 are the negations of
    // the previous step's, exact except at a tie dPhi == 0 (where each end
    // takes the other cell as upstream): U.tie flags those, and the marches
    // recompute the affected rows afterwards.
    __device__ __forceinline__ void eval_links(const YRow<Real>& P, const YRow<Real>& C, const YRow<Real>& N,
                                               const YIn<Real>& D, const YUp<Real>& Uprev,
                                               LinkOut<Real> (&S)[NSLOT], YUp<Real>& U) const {
        Real Tx_m = vshfl_up(D.Tx);
        if (lane == 0) Tx_m = D.hT1;
        const CellVal<Real> zmc = make_cell(q, D.p_zm, D.z_zm);
        const CellVal<Real> zpc = make_cell(q, D.p_zp, D.z_zp);

        // slot order: 0 (0,0,-1) 1 (-1,-1) 2 (0,-1) 3 (+1,-1) 4 (-1,0) 5 self
        //             6 (+1,0) 7 (-1,+1) 8 (0,+1) 9 (+1,+1) 10 (0,0,+1)
        LinkOut<Real> E;  // lane 0: its (-1,-1) link; lane 31: its (+1,-1) link
        if constexpr (sizeof(Real) == 4) {
            // eight links as four FP32x2 pairs
            const Link2 x = link2(q, f2(Tx_m, D.Tx), C.c, C.m, C.p);
            const Link2 yz = link2(q, f2(D.Ty, D.Tz), C.c, N.c, zpc);
            S[4] = LinkOut<float>{x.F.x, x.Da.x, x.Db.x};
            S[6] = LinkOut<float>{x.F.y, x.Da.y, x.Db.y};
            S[8] = LinkOut<float>{yz.F.x, yz.Da.x, yz.Db.x};
            S[10] = LinkOut<float>{yz.F.y, yz.Da.y, yz.Db.y};
            if (DIAG) {
                const Link2 d = link2(q, f2(D.Tmp, D.Tpp), C.c, N.m, N.p);
                const Link2 ze = link2(q, f2(D.Tz_m, D.hT2), C.c, zmc, lane == 0 ? P.m : P.p);
                S[7] = LinkOut<float>{d.F.x, d.Da.x, d.Db.x};
                S[9] = LinkOut<float>{d.F.y, d.Da.y, d.Db.y};
                S[0] = LinkOut<float>{ze.F.x, ze.Da.x, ze.Db.x};
                E = LinkOut<float>{ze.F.y, ze.Da.y, ze.Db.y};
            } else {
                S[0] = link(q, D.Tz_m, C.c, zmc);
            }
        } else {
            S[0] = link(q, D.Tz_m, C.c, zmc);
            S[4] = link(q, Tx_m, C.c, C.m);
            S[6] = link(q, D.Tx, C.c, C.p);
            S[8] = link(q, D.Ty, C.c, N.c);
            S[10] = link(q, D.Tz, C.c, zpc);
            if (DIAG) {
                S[7] = link(q, D.Tmp, C.c, N.m);
                S[9] = link(q, D.Tpp, C.c, N.p);
                E = link(q, D.hT2, C.c, lane == 0 ? P.m : P.p);
            }
        }
        U.y = S[8];
        U.xy = S[9];
        U.mxy = S[7];
        U.tie = (S[8].F == Real(0) && D.Ty != Real(0)) ||
                (DIAG && ((S[9].F == Real(0) && D.Tpp != Real(0)) || (S[7].F == Real(0) && D.Tmp != Real(0))));

        // links into row j-1: negations of Uprev (own +y, left's +x+y, right's -x+y)
        S[2] = LinkOut<Real>{-Uprev.y.F, -Uprev.y.Db, -Uprev.y.Da};
        if (DIAG) {
            const Real f1 = vshfl_up(Uprev.xy.F), a1 = vshfl_up(Uprev.xy.Da), b1 = vshfl_up(Uprev.xy.Db);
            const Real f3 = vshfl_down(Uprev.mxy.F), a3 = vshfl_down(Uprev.mxy.Da), b3 = vshfl_down(Uprev.mxy.Db);
            S[1] = LinkOut<Real>{-f1, -b1, -a1};
            S[3] = LinkOut<Real>{-f3, -b3, -a3};
            if (lane == 0) S[1] = E;
            if (lane == 31) S[3] = E;
        }
    }

    // Assemble row j.  P, C, N: rows j-1, j, j+1.  Uprev: links from row j-1
    // into row j.  buf: this step's staging buffer.  Returns the links from
    // row j into row j+1.
    template <int PATH>
    __device__ __forceinline__ YUp<Real> row(int j, const YRow<Real>& P, const YRow<Real>& C, const YRow<Real>& N,
                                             const YIn<Real>& D, const YUp<Real>& Uprev, Real* buf,
                                             int rowbase) const {
        constexpr bool FULL = PATH == 2, INJK = PATH >= 1;
        constexpr int L = DIAG ? 11 : 7, LX = DIAG ? 3 : 1;  // interior row length; x links per side
        const int ey = INJK ? 2 : axis_links(j, ny);
        const unsigned mask = row_mask<PATH>(j);
        LinkOut<Real> S[NSLOT];
        YUp<Real> U;
        eval_links(P, C, N, D, Uprev, S, U);

        // offsets of this row's CSR segment and of this lane's row in it
        const int per = 1 + ey + ez, perx = 1 + g.diag * ey;
        int lane_off;
        if constexpr (FULL) lane_off = lane * L;
        else if constexpr (INJK) lane_off = lane * L - ((i0 == 0 && lane > 0) ? LX : 0);
        else lane_off = (i - i0) * per + (int)(axis_links_before(i, nx) - Sx0) * perx;
        const long long seg = base_k + (rowbase + (INJK ? X2 : i0 * per + Sx0 * perx));
        const int aoff = JAC ? (int)(seg & (VEC - 1)) : 0;

        const RowSums out = sum_row(S, mask, C.c, D, buf + aoff + lane_off);
        const int c = kb + nx * j + i;
        if (act) {
            if (o.R) o.R[c] = out.R;
            if (JAC && o.diag64) o.diag64[c] = out.diag64;
            if (out.bad) atomicOr(o.status, STATUS_NONFINITE);
        }
        if (JAC) {
            const int iend = min(i0 + 32, nx);
            int seg_len;
            if constexpr (FULL) seg_len = 32 * L;
            else if constexpr (INJK) seg_len = (iend - i0) * L - (i0 == 0 ? LX : 0) - (iend == nx ? LX : 0);
            else seg_len = (iend - i0) * per + (int)(axis_links_before(iend, nx) - Sx0) * perx;
            write_segment(buf, seg, aoff, seg_len);
        }
        return U;
    }

    // J w (and R when o.R is set) of row j: wP, wC, wN hold w of rows j-1,
    // j, j+1; wzm, wzp the vertical neighbours'.  Per link the term
    // dF/dp_K w_K + dF/dp_L w_L is one FP32 fma; the terms and the residual's
    // fluxes share one FP32x2 Kahan sum in slot order, then dA/dp w_K.
    template <int PATH>
    __device__ __forceinline__ YUp<Real> row_jvp(int j, const YRow<Real>& P, const YRow<Real>& C,
                                                 const YRow<Real>& N, const YIn<Real>& D, const YUp<Real>& Uprev,
                                                 const YW& wP, const YW& wC, const YW& wN, float wzm,
                                                 float wzp) const {
        const unsigned mask = row_mask<PATH>(j);
        LinkOut<Real> S[NSLOT];
        YUp<Real> U;
        eval_links(P, C, N, D, Uprev, S, U);
        const float ws[NSLOT] = {wzm, wP.m, wP.c, wP.p, wC.m, 0.f, wC.p, wN.m, wN.c, wN.p, wzp};
        Kahan2 ks;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s == SLOT_SELF) continue;
            if (mask & (1u << s)) ks.add(f2(S[s].F, __fmaf_rn(S[s].Da, wC.c, __fmul_rn(S[s].Db, ws[s]))));
        }
        const AccF acc = accumulation<CRK>(q, C.c.p, D.pn, D.mn, C.c.rho, D.phi0);
        Kahan32 js{ks.s.y, ks.c.y};
        js.add(__fmul_rn(acc.dA, wC.c));
        const double jw = __dadd_rn(widen(js.s), -widen(js.c));
        if (act) {
            const int c = kb + nx * j + i;
            Jw[c] = jw;
            double r = 0.0;
            if (o.R) {
                r = __dadd_rn(__dadd_rn(acc.A, widen(ks.s.x)), -widen(ks.c.x));
                o.R[c] = r;
            }
            if (nonfinite(jw) || nonfinite(r)) atomicOr(o.status, STATUS_NONFINITE);
        }
        return U;
    }

    // Adjoint of row j (tpfa_vjp.cu states the formulation): vP, vC, vN hold
    // v of rows j-1, j, j+1 split into FP32 pairs, vzm, vzp the vertical
    // neighbours' pairs, kC the cell's k.  Per link, with dv = v_K - v_L
    // (FP32 from the split pairs), the terms dF_KL/dp_K dv and F_KL (k_L / (k_K +
    // k_L)) dv share one FP32x2 Kahan sum in slot order; k_L / (k_K + k_L) =
    // Upsilon_KL (d/A) / (2 k_K) for the harmonic two-point transmissibility.
    // The links into row j-1 are reused by negation, which is exact except
    // at a tie; a tie has zero flux, so `fix` reports (warp-uniformly) a row
    // where any link had F == 0, and the caller recomputes it after the march
    // with the full formulation (which adds the tie terms).
    template <int PATH>
    __device__ __forceinline__ YUp<Real> row_vjp(int j, const YRow<Real>& P, const YRow<Real>& C,
                                                 const YRow<Real>& N, const YIn<Real>& D, const YUp<Real>& Uprev,
                                                 Real Ty_prev, Real Tpp_prev, Real Tmp_prev, const YV& vP,
                                                 const YV& vC, const YV& vN, const F2Split& vzm, const F2Split& vzp,
                                                 float kC, bool& fix) const {
        const unsigned mask = row_mask<PATH>(j);
        LinkOut<Real> S[NSLOT];
        YUp<Real> U;
        eval_links(P, C, N, D, Uprev, S, U);
        Real Tx_m = vshfl_up(D.Tx), Tl = vshfl_up(Tpp_prev), Tr = vshfl_down(Tmp_prev);
        if (lane == 0) Tx_m = D.hT1, Tl = D.hT2;
        if (lane == 31) Tr = D.hT2;
        const float Ts[NSLOT] = {D.Tz_m, Tl, Ty_prev, Tr, Tx_m, 0.f, D.Tx, D.Tmp, D.Ty, D.Tpp, D.Tz};
        const float gs[NSLOT] = {lg.cz, lg.cd, lg.cy, lg.cd, lg.cx, 0.f, lg.cx, lg.cd, lg.cy, lg.cd, lg.cz};
        const F2Split vs[NSLOT] = {F2Split{}, v_minus(vP), vP.c, v_plus(vP), v_minus(vC), F2Split{}, v_plus(vC),
                                   v_minus(vN), vN.c, v_plus(vN), F2Split{}};
        const float inv2k = kC > 0.f ? __fdiv_rn(0.5f, kC) : 0.f;
        Kahan2 ks;
        bool zero_flux = false;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s == SLOT_SELF || !(mask & (1u << s))) continue;
            const float dv = diff_f2(vC.c, s == 0 ? vzm : (s == 10 ? vzp : vs[s]));
            const float ratio = __fmul_rn(__fmul_rn(Ts[s], gs[s]), inv2k);
            ks.add(f2(__fmul_rn(S[s].Da, dv), __fmul_rn(__fmul_rn(S[s].F, ratio), dv)));
            zero_flux |= S[s].F == 0.f;
        }
        fix = __any_sync(0xffffffffu, zero_flux);
        const AccF acc = accumulation<CRK>(q, C.c.p, D.pn, D.mn, C.c.rho, D.phi0);
        if (act) {
            const int c = kb + nx * j + i;
            // the diagonal's own term v_i dA_i/dp_i joins the compensated FP32
            // sum last; + 0.0 is the twin's tie correction when no link has
            // zero flux (it turns a -0 into +0 as that addition does)
            Kahan32 kp{ks.s.x, ks.c.x};
            kp.add(__fmaf_rn(vC.c.hi, acc.dA, __fmul_rn(vC.c.lo, acc.dA)));
            const double gp = __dadd_rn(__dadd_rn(widen(kp.s), -widen(kp.c)), 0.0);
            const double gk = __dadd_rn(widen(ks.s.y), -widen(ks.c.y));
            gP[c] = gp;
            if (gK) gK[c] = gk;
            if (nonfinite(gp) || nonfinite(gk)) atomicOr(o.status, STATUS_NONFINITE);
        }
        return U;
    }

    // Slot values go to rowbuf; residual and diagonal sums in slot order.
    // FP32: one FP32x2 Kahan sum carries (residual, diagonal); FP64: plain sums.
    __device__ __forceinline__ RowSums sum_row(const LinkOut<Real> (&S)[NSLOT], unsigned mask, const CellVal<Real>& me,
                                               const YIn<Real>& D, Real* rowbuf) const {
        if constexpr (sizeof(Real) == 4) {
            Kahan2 ks;
#pragma unroll
            for (int s = 0; s < NSLOT; ++s) {
                if (s == SLOT_SELF) continue;
                if (mask & (1u << s)) {
                    ks.add(f2(S[s].F, JAC ? S[s].Da : 0.f));
                    if (JAC && act) rowbuf[slot_pos(mask, s)] = S[s].Db;
                }
            }
            const AccF acc = accumulation<CRK>(q, me.p, D.pn, D.mn, me.rho, D.phi0);
            RowSums out;
            out.R = __dadd_rn(__dadd_rn(acc.A, widen(ks.s.x)), -widen(ks.c.x));
            out.diag64 = 0.0;
            if (JAC) {
                Kahan32 ds{ks.s.y, ks.c.y};
                ds.add(acc.dA);
                out.diag64 = __dadd_rn(widen(ds.s), -widen(ds.c));
                if (act) rowbuf[slot_pos(mask, SLOT_SELF)] = __fsub_rn(ds.s, ds.c);
            }
            out.bad = nonfinite(out.R) || (JAC && nonfinite(out.diag64));
            return out;
        } else {
            double rs = 0.0, ds = 0.0;
#pragma unroll
            for (int s = 0; s < NSLOT; ++s) {
                if (s == SLOT_SELF) continue;
                if (mask & (1u << s)) {
                    rs = __dadd_rn(rs, S[s].F);
                    if (JAC) {
                        ds = __dadd_rn(ds, S[s].Da);
                        if (act) rowbuf[slot_pos(mask, s)] = S[s].Db;
                    }
                }
            }
            const AccD acc = accumulation<CRK>(q, me.p, D.pn, D.mn, me.rho, D.phi0);
            RowSums out;
            out.R = __dadd_rn(rs, acc.A);
            out.diag64 = 0.0;
            if (JAC) {
                ds = __dadd_rn(ds, acc.dA);
                out.diag64 = ds;
                if (act) rowbuf[slot_pos(mask, SLOT_SELF)] = ds;
            }
            out.bad = nonfinite(out.R) || (JAC && nonfinite(out.diag64));
            return out;
        }
    }

    // Wait until the bulk store issued from this buffer two steps ago has
    // read it (lane 0 issued it), so the buffer can be refilled.
    // (every lane waits: the other lanes have no bulk groups, so their wait
    // returns at once, and the warp does not branch)
    __device__ __forceinline__ void buffer_ready() const {
        if (JAC && v16) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
    }

    // Copy buf[aoff .. aoff+len) to vals[seg .. seg+len).  The 16-byte-aligned
    // middle goes out as one bulk shared->global copy (issued by lane 0,
    // tracked as a bulk async-group); the at most 2 (VEC - 1) elements at the
    // ends are stored by single lanes.
    __device__ __forceinline__ void write_segment(Real* buf, long long seg, int aoff, int len) const {
        Real* dst = o.vals + (seg - aoff);  // 16-byte aligned when v16
        const int span = aoff + len;
        if (v16) {
            const int qlo = (aoff + VEC - 1) / VEC, qhi = span / VEC;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (qhi > qlo) {
                {  // issued and committed by lane 0 (a guard predicate, no branch)
                    const uint32_t src = (uint32_t)__cvta_generic_to_shared(buf + qlo * VEC);
                    const uint32_t bytes = (uint32_t)(qhi - qlo) * 16u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %3, 0;\n\t"
                                 "@p cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
                                 "@p cp.async.bulk.commit_group;\n\t}" ::"l"(dst + qlo * VEC), "r"(src), "r"(bytes),
                                 "r"(lane)
                                 : "memory");
                }
                const int nh = qlo * VEC - aoff, nt = span - qhi * VEC;  // each < VEC
                if (lane >= 1 && lane <= nh) dst[aoff + lane - 1] = buf[aoff + lane - 1];
                if (lane >= 8 && lane < 8 + nt) dst[qhi * VEC + lane - 8] = buf[qhi * VEC + lane - 8];
            } else {
                if (lane < len) dst[aoff + lane] = buf[aoff + lane];
            }
        } else {
            __syncwarp();
            for (int e = aoff + lane; e < span; e += 32) dst[e] = buf[e];
            __syncwarp();
        }
    }

    // All bulk stores complete before the block exits.
    __device__ __forceinline__ void drain() const {
        if (JAC && v16 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
};

// Dynamic shared memory of one block of W warps: per warp two CSR staging
// buffers, the RING x NF input ring and the RING m^n values.
template <typename Real, int W>
constexpr int ymarch_smem_bytes() {
    return W * (2 * (32 * NSLOT + 16 / (int)sizeof(Real)) * (int)sizeof(Real) +
                3 * 18 * 32 * (int)sizeof(Real) + 3 * 32 * (int)sizeof(double));
}

// One block's work: x-segment bx, y-run by, z-block bz of one grid.  Shared
// by the single-grid kernel and the persistent ensemble kernel (whose blocks
// call it once per tile they claim), so both produce identical rows.
// Runs step(path, j) over the rows j0 .. j1-1 of a march: the boundary rows
// (j = 0, j = ny - 1, and every row of a boundary plane) on path 0, the
// interior rows in one loop whose path is fixed for the warp (2: interior
// x-segment, 1: a segment at an x boundary) instead of a choice per row.
// `path` is a std::integral_constant, so the step is compiled per path.
template <class Step>
__device__ __forceinline__ void march_rows(int j0, int j1, int ny, bool zint, bool xint, Step&& step) {
    int j = j0;
    if (zint) {
        if (j == 0 && j < j1) step(std::integral_constant<int, 0>{}, j++);
        const int jend = min(j1, ny - 1);
        if (xint) {
#pragma unroll 1
            for (; j < jend; ++j) step(std::integral_constant<int, 2>{}, j);
        } else {
#pragma unroll 1
            for (; j < jend; ++j) step(std::integral_constant<int, 1>{}, j);
        }
    }
#pragma unroll 1
    for (; j < j1; ++j) step(std::integral_constant<int, 0>{}, j);
}

// SPLIT: run the rows through march_rows (one loop per path).  Measured at
// 160 x 160 x 80 and on the 64-model ensemble: the ensemble's persistent
// kernel gains 5 % with it, the single-grid kernel loses 4 %, so only the
// ensemble uses it.
template <typename Real, bool DIAG, bool CRK, bool JAC, int W, bool SPLIT = false>
__device__ __forceinline__ void ymarch_tile(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                            const AsmFields<Real>& f, const AsmOut<Real>& o, int JY, int bx, int by,
                                            int bz, unsigned char* smem, int kbase = 0, int kend = -1) {
    using M_t = YMarch<Real, DIAG, CRK, JAC, W>;
    constexpr int BUF = 32 * NSLOT + 16 / (int)sizeof(Real);
    const int lane = threadIdx.x, w = threadIdx.y;
    const int k = kbase + bz * W + w;  // planes [kbase, kend) of the grid (all by default)
    if (k >= (kend < 0 ? g.nz : kend)) return;  // warp-uniform
    // per warp: two staging buffers, then the input ring, then the m^n ring
    Real* stage = reinterpret_cast<Real*>(smem) + w * 2 * BUF;
    Real* ring = reinterpret_cast<Real*>(smem) + W * 2 * BUF + w * M_t::RING * M_t::NF * 32;
    double* ringm = reinterpret_cast<double*>(reinterpret_cast<Real*>(smem) + W * 2 * BUF +
                                              W * M_t::RING * M_t::NF * 32) + w * M_t::RING * 32;
    M_t M(g, q, f, o, lane, bx * 32, k);
    M.ring = ring;
    M.ringm = ringm;
    const int j0 = by * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;

    // prologue: rows j0-1, j0, j0+1 into ring slots 0, 1, 2; cells of rows
    // j0-1 and j0 and the links of row j0-1 into row j0 (unused when j0 == 0)
    M.issue_row(j0 - 1, 0);
    M.issue_row(j0, 1);
    M.issue_row(j0 + 1, 2);
    M.wait_all_but_newest();
    YRow<Real> P = M.row_cells(0);
    YRow<Real> C = M.row_cells(1);
    Real Ty_prev, Tpp_prev, Tmp_prev;
    {
        const YIn<Real> Dp = M.read_in(0);
        Ty_prev = Dp.Ty;
        Tpp_prev = Dp.Tpp;
        Tmp_prev = Dp.Tmp;
    }
    YUp<Real> U = M.up_links(P, C, Ty_prev, Tpp_prev, Tmp_prev);
    int s0 = 1, s1 = 2, s2 = 0;  // ring slots of rows j, j+1, j+2
    int rowbase = M.row_base(j0);
    // rows whose links into the previous row (reused by negation) met an
    // exact tie dPhi == 0: recomputed after the march (bit j - j0; JY <= 64)
    unsigned long long tie_rows = 0ull;

    if constexpr (SPLIT) {
        march_rows(j0, j1, M.ny, zint, M.xint, [&](auto path, int j) {
            constexpr int PATH = decltype(path)::value;
            // row j+2 is requested now and used two steps later; row j+1 arrived
            M.issue_row(j + 2, s2);
            M.wait_all_but_newest();
            const YRow<Real> N = M.row_cells(s1);
            const YIn<Real> D = M.read_in(s0);
            const int st = s0;
            s0 = s1;
            s1 = s2;
            s2 = st;
            Real* buf = stage + ((j - j0) & 1) * BUF;
            M.buffer_ready();
            if (__any_sync(0xffffffffu, U.tie)) tie_rows |= 1ull << (j - j0);
            U = M.template row<PATH>(j, P, C, N, D, U, buf, rowbase);
            rowbase += M.row_base_step(j);
            P = C;
            C = N;
        });
    } else {
        for (int j = j0; j < j1; ++j) {
            // row j+2 is requested now and used two steps later; row j+1 arrived
            M.issue_row(j + 2, s2);
            M.wait_all_but_newest();
            const YRow<Real> N = M.row_cells(s1);
            const YIn<Real> D = M.read_in(s0);
            const int st = s0;
            s0 = s1;
            s1 = s2;
            s2 = st;
            Real* buf = stage + ((j - j0) & 1) * BUF;
            M.buffer_ready();
            if (__any_sync(0xffffffffu, U.tie)) tie_rows |= 1ull << (j - j0);
            const bool injk = zint && j > 0 && j + 1 < M.ny;
            if (injk && M.xint) U = M.template row<2>(j, P, C, N, D, U, buf, rowbase);
            else if (injk) U = M.template row<1>(j, P, C, N, D, U, buf, rowbase);
            else U = M.template row<0>(j, P, C, N, D, U, buf, rowbase);
            rowbase += M.row_base_step(j);
            P = C;
            C = N;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    M.drain();
    if (tie_rows) {  // warp-uniform; every bulk store of the warp has completed
        __syncwarp();
        for (int b = 0; b < 64; ++b)
            if ((tie_rows >> b) & 1ull) naive_row<Real, CRK, JAC>(g, q, f, o, M.act, M.i, j0 + b, k);
    }
}

// Dynamic shared memory of one block of the TMA march: the shared ring of
// TRING slots, per warp two CSR staging buffers, 2 TRING mbarriers, and
// slack to align the ring to 128 bytes.
template <int W, int TRING>
constexpr int ymarch_tma_smem_bytes() {
    return 128 + TRING * TmaSlot<W>::BYTES + W * 2 * (32 * NSLOT + 4) * 4 + 2 * TRING * 8;
}

// The march with its row inputs delivered by TMA (mixed path): block (bx,
// by, k) runs the W x-segments bx W .. bx W + W - 1 of plane k over the
// y-run by, one warp per segment, all warps stepping through a shared ring.
// Every row is computed by the same code as in ymarch_tile, so the results
// are bit-identical.  Warps whose segment lies past the grid's x-extent only
// keep the ring's protocol.  A barrier wait that runs out sets
// STATUS_TIMEOUT and ends the march (after a bounded wait for the copies
// still in flight).
template <bool DIAG, bool CRK, bool JAC, int W>
__device__ __forceinline__ void ymarch_tile_tma(const GridGeom& g, const PhysF& q, const AsmFields<float>& f,
                                                const AsmOut<float>& o, const TmaMaps* maps, int JY, int bx,
                                                int by, int k, unsigned char* smem) {
    using M_t = YMarch<float, DIAG, CRK, JAC, W>;
    using TS = TmaSlot<W>;
    constexpr int BUF = 32 * NSLOT + 4, TR = M_t::TRING;
    const int lane = threadIdx.x, w = threadIdx.y;
    unsigned char* base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    float* stage = reinterpret_cast<float*>(base + TR * TS::BYTES) + w * 2 * BUF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + TR * TS::BYTES + W * 2 * BUF * 4);
    const int X0 = bx * 32 * W;
    M_t M(g, q, f, o, lane, X0 + 32 * w, k);
    M.tma_init(base, bars, maps, w);
    const bool live = M.i0 < g.nx;  // warp-uniform
    const int j0 = by * JY;
    const int j1 = min(j0 + JY, g.ny);
    const bool zint = M.zm && M.zp;

    bool ok = true;
    if (M.issuer) {
        for (int s = 0; s < TR; ++s) M.tma_issue(j0 - 1 + s, s, X0, false);
    }
    for (int s = 0; s < TR; ++s) M.tma_requested(s);
    ok = M.tma_wait(0);
    ok = ok && M.tma_wait(1);
    unsigned long long tie_rows = 0ull;
    if (ok) {
        YRow<float> P = M.tma_row_cells(0);
        YRow<float> C = M.tma_row_cells(1);
        YUp<float> U;
        {
            const YIn<float> Dp = M.tma_read_in(0, 0.f);
            U = M.up_links(P, C, Dp.Ty, Dp.Tpp, Dp.Tmp);
        }
        int sp = 0;  // slot of row j-1; rows j, j+1, ... follow in the next slots (mod TR)
        int rowbase = M.row_base(j0);
        for (int j = j0; j < j1; ++j) {
            const int s0 = sp + 1 == TR ? 0 : sp + 1;
            const int s1 = s0 + 1 == TR ? 0 : s0 + 1;
            const float hT2 = M.tma_h2(sp);  // slot sp holds row j-1 until the refill below
            M.tma_release(sp);
            if (M.issuer && !M.tma_issue(j + TR - 1, sp, X0, true)) atomicOr(o.status, STATUS_TIMEOUT);
            M.tma_requested(sp);
            if (!M.tma_wait(s1)) {
                ok = false;
                break;
            }
            const YRow<float> N = M.tma_row_cells(s1);
            const YIn<float> D = M.tma_read_in(s0, hT2);
            sp = s0;
            if (live) {
                float* buf = stage + ((j - j0) & 1) * BUF;
                M.buffer_ready();
                if (__any_sync(0xffffffffu, U.tie)) tie_rows |= 1ull << (j - j0);
                const bool injk = zint && j > 0 && j + 1 < M.ny;
                if (injk && M.xint) U = M.template row<2>(j, P, C, N, D, U, buf, rowbase);
                else if (injk) U = M.template row<1>(j, P, C, N, D, U, buf, rowbase);
                else U = M.template row<0>(j, P, C, N, D, U, buf, rowbase);
                rowbase += M.row_base_step(j);
            }
            P = C;
            C = N;
        }
    }
    ok = M.tma_drain() && ok;
    M.drain();
    if (!ok) {
        if (lane == 0) atomicOr(o.status, STATUS_TIMEOUT);
        return;
    }
    if (tie_rows) {  // warp-uniform; every bulk store of the warp has completed
        __syncwarp();
        for (int b = 0; b < 64; ++b)
            if ((tie_rows >> b) & 1ull) naive_row<float, CRK, JAC>(g, q, f, o, M.act, M.i, j0 + b, k);
    }
}

template <bool DIAG, bool CRK, bool JAC, int W>
__global__ void __launch_bounds__(32 * W, 16 / W)
    k_assemble_ymarch_tma(GridGeom g, PhysF q, AsmFields<float> f, AsmOut<float> o, const __grid_constant__ TmaMaps tm,
                          int JY, int k0) {
    extern __shared__ __align__(16) unsigned char smem[];
    ymarch_tile_tma<DIAG, CRK, JAC, W>(g, q, f, o, &tm, JY, blockIdx.x, blockIdx.y, k0 + (int)blockIdx.z, smem);
}

template <typename Real, bool DIAG, bool CRK, bool JAC, int W>
__global__ void __launch_bounds__(32 * W, (sizeof(Real) == 4 ? 16 : 8) / W)
    k_assemble_ymarch(GridGeom g, typename PhysOf<Real>::type q, AsmFields<Real> f, AsmOut<Real> o, int JY,
                      int k0, int k1) {
    extern __shared__ __align__(16) unsigned char smem[];
    ymarch_tile<Real, DIAG, CRK, JAC, W>(g, q, f, o, JY, blockIdx.x, blockIdx.y, blockIdx.z, smem, k0, k1);
}

}  // namespace tpfa
