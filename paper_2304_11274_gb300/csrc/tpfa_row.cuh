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

// Row (i, j, k) read straight from global memory and written out: the cell
// and its neighbours, densities recomputed per neighbour as in Algorithm 1.
// The naive kernel runs it for every cell; the tiled kernel runs it for the
// rows whose reused links met an exact tie.  A lane with act == false works
// on cell (0, j, k) with no links and stores nothing, so every address formed
// stays inside the arrays.
template <typename Real, bool CRK, bool JAC>
__device__ __forceinline__ void naive_row(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                          const AsmFields<Real>& f, const AsmOut<Real>& o, bool act, int i, int j,
                                          int k) {
    const long long nx = g.nx, nxy = nx * g.ny;
    const long long c = (act ? (long long)i + nx * j : 0) + nxy * k;
    const unsigned mask = act ? slot_mask(g, i, j, k) : (1u << SLOT_SELF);
    const long long off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
    const CellVal<Real> me = make_cell(q, f.p[c], f.z[c]);
    CellVal<Real> nb[NSLOT];
    Real T[NSLOT];
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        nb[s] = me;
        T[s] = Real(0);
        const bool valid = s != SLOT_SELF && (mask & (1u << s));
        const long long d = valid ? c + off[s] : c;  // in range even if a load is hoisted
        if (valid) nb[s] = make_cell(q, f.p[d], f.z[d]);
    }
    if (mask & (1u << 0)) T[0] = f.Tz[(mask & 1u) ? c - nxy : c];
    if (mask & (1u << 1)) T[1] = f.Tpp[(mask & 2u) ? c - nx - 1 : c];
    if (mask & (1u << 2)) T[2] = f.Ty[(mask & 4u) ? c - nx : c];
    if (mask & (1u << 3)) T[3] = f.Tmp[(mask & 8u) ? c - nx + 1 : c];
    if (mask & (1u << 4)) T[4] = f.Tx[(mask & 16u) ? c - 1 : c];
    if (mask & (1u << 6)) T[6] = f.Tx[c];
    if (mask & (1u << 7)) T[7] = f.Tmp[c];
    if (mask & (1u << 8)) T[8] = f.Ty[c];
    if (mask & (1u << 9)) T[9] = f.Tpp[c];
    if (mask & (1u << 10)) T[10] = f.Tz[c];
    const long long rs = act ? row_start(g, i, j, k) : 0;
    Real* vals = o.vals;
    auto sink = [&](int pos, Real v) {
        if (act) vals[rs + pos] = v;
    };
    const RowSums r = assemble_row<CRK, JAC>(q, me, nb, T, mask, f.pn[c], f.mn[c], CRK ? f.phi0[c] : Real(0), sink);
    if (!act) return;
    if (o.R) o.R[c] = r.R;
    if (JAC && o.diag64) o.diag64[c] = r.diag64;
    if (r.bad) atomicOr(o.status, STATUS_NONFINITE);
}

}  // namespace tpfa
