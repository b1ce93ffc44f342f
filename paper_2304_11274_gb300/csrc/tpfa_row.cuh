// tpfa_row.cuh -- assembly of one Jacobian row and one residual entry.
//
// Algorithm 1 of arXiv 2304.11274 for cell K: the flux of every link K -> L,
// L in adj(K), is added to r_K; Eq. vk adds the accumulation term.  The
// Jacobian row holds dR_K/dp_L for L in adj(K) and the diagonal dR_K/dp_K.
//
// Slots of a row, in ascending column order (offsets in cells):
//   0 (0,0,-1)  1 (-1,-1,0)  2 (0,-1,0)  3 (+1,-1,0)  4 (-1,0,0)  5 self
//   6 (+1,0,0)  7 (-1,+1,0)  8 (0,+1,0)  9 (+1,+1,0) 10 (0,0,+1)
// Slots 1, 3, 7, 9 exist only with 10-point connectivity.  Both the residual
// and the diagonal are summed over the slots in this order, then the
// accumulation term, in every kernel; so all kernels give identical bits.
#pragma once

#include "tpfa_common.cuh"

namespace tpfa {

constexpr int SLOT_SELF = 5;
constexpr int NSLOT = 11;

// Validity mask of the slots of row (i, j, k).
__device__ __forceinline__ unsigned slot_mask(const GridGeom& g, int i, int j, int k) {
    const bool xm = i > 0, xp = i + 1 < g.nx, ym = j > 0, yp = j + 1 < g.ny;
    const bool zm = k > 0, zp = k + 1 < g.nz;
    unsigned m = (1u << SLOT_SELF);
    m |= (unsigned)zm << 0;
    m |= (unsigned)ym << 2;
    m |= (unsigned)xm << 4;
    m |= (unsigned)xp << 6;
    m |= (unsigned)yp << 8;
    m |= (unsigned)zp << 10;
    if (g.diag) {
        m |= (unsigned)(xm && ym) << 1;
        m |= (unsigned)(xp && ym) << 3;
        m |= (unsigned)(xm && yp) << 7;
        m |= (unsigned)(xp && yp) << 9;
    }
    return m;
}

// Position of slot s within its row.
__device__ __forceinline__ int slot_pos(unsigned mask, int s) { return __popc(mask & ((1u << s) - 1u)); }

template <typename Real>
struct PhysOf;
template <>
struct PhysOf<float> {
    using type = PhysF;
};
template <>
struct PhysOf<double> {
    using type = PhysD;
};

// Row result.  Mixed path: R = A + (s - c) of an FP32 Kahan sum combined in
// FP64; diag64 likewise.  FP64 path: plain FP64 sums.
struct RowSums {
    double R;
    double diag64;
    bool bad;
};

// FP32 (mixed) row.  `sink(pos, value)` receives every Jacobian value.
template <bool CRK, bool JAC, typename Sink>
__device__ __forceinline__ RowSums assemble_row(const PhysF& q, const CellVal<float>& me,
                                                const CellVal<float> (&nb)[NSLOT], const float (&T)[NSLOT],
                                                unsigned mask, float pn, double mn, float phi0, Sink&& sink) {
    Kahan32 rs, ds;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        if (s == SLOT_SELF) continue;
        if (mask & (1u << s)) {
            const LinkOut<float> L = link(q, T[s], me, nb[s]);
            rs.add(L.F);
            if (JAC) {
                ds.add(L.Da);
                sink(slot_pos(mask, s), L.Db);
            }
        }
    }
    const AccF acc = accumulation<CRK>(q, me.p, pn, mn, me.rho, phi0);
    RowSums out;
    out.R = __dadd_rn(__dadd_rn(acc.A, widen(rs.s)), -widen(rs.c));
    out.diag64 = 0.0;
    if (JAC) {
        ds.add(acc.dA);
        out.diag64 = __dadd_rn(widen(ds.s), -widen(ds.c));
        sink(slot_pos(mask, SLOT_SELF), __fsub_rn(ds.s, ds.c));
    }
    out.bad = nonfinite(out.R) || (JAC && nonfinite(out.diag64));
    return out;
}

// FP64 row.
template <bool CRK, bool JAC, typename Sink>
__device__ __forceinline__ RowSums assemble_row(const PhysD& q, const CellVal<double>& me,
                                                const CellVal<double> (&nb)[NSLOT], const double (&T)[NSLOT],
                                                unsigned mask, double pn, double mn, double phi0, Sink&& sink) {
    double rs = 0.0, ds = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        if (s == SLOT_SELF) continue;
        if (mask & (1u << s)) {
            const LinkOut<double> L = link(q, T[s], me, nb[s]);
            rs = __dadd_rn(rs, L.F);
            if (JAC) {
                ds = __dadd_rn(ds, L.Da);
                sink(slot_pos(mask, s), L.Db);
            }
        }
    }
    const AccD acc = accumulation<CRK>(q, me.p, pn, mn, me.rho, phi0);
    RowSums out;
    out.R = __dadd_rn(rs, acc.A);
    out.diag64 = 0.0;
    if (JAC) {
        ds = __dadd_rn(ds, acc.dA);
        out.diag64 = ds;
        sink(slot_pos(mask, SLOT_SELF), ds);
    }
    out.bad = nonfinite(out.R) || (JAC && nonfinite(out.diag64));
    return out;
}

}  // namespace tpfa
