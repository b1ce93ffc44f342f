// tpfa_assemble.cu -- residual + Jacobian assembly kernels (sm_103a).
//
// Two kernels compute the same rows (see tpfa_row.cuh for the row layout and
// summation order), so their outputs are bit-identical:
//
//   k_assemble_naive  -- one thread per cell; the cell and its 10 neighbours
//                        read from global memory, densities recomputed per
//                        neighbour as in Algorithm 1.  The correctness
//                        baseline.
//   k_assemble_ymarch -- the production kernel.  A warp owns a 32-cell
//                        x-segment of one z-plane and marches along y over a
//                        run of rows, keeping rows j-1, j, j+1 in registers:
//                        each cell's density is evaluated once per row it
//                        enters, x-neighbours come from warp shuffles (the
//                        two halo cells ride in lanes 0 and 31), y- and
//                        diagonal neighbours from the register window, and
//                        the next rows' loads are issued one or two rows
//                        ahead.  Each warp's Jacobian rows form one
//                        contiguous CSR segment, staged in shared memory and
//                        written with coalesced stores.
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"

namespace tpfa {

// ------------------------------------------------------------------ naive

template <typename Real, bool CRK, bool JAC>
__global__ void __launch_bounds__(256) k_assemble_naive(GridGeom g, typename PhysOf<Real>::type q,
                                                        AsmFields<Real> f, AsmOut<Real> o) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long nx = g.nx, nxy = nx * g.ny;
    const long long c = (long long)i + nx * j + nxy * k;
    const unsigned mask = slot_mask(g, i, j, k);
    const long long off[NSLOT] = {-nxy, -nx - 1, -nx, -nx + 1, -1, 0, 1, nx - 1, nx, nx + 1, nxy};
    const CellVal<Real> me = make_cell(q, f.p[c], f.z[c]);
    CellVal<Real> nb[NSLOT];
    Real T[NSLOT];
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        nb[s] = me;
        T[s] = Real(0);
        if (s != SLOT_SELF && (mask & (1u << s))) {
            const long long d = c + off[s];
            nb[s] = make_cell(q, f.p[d], f.z[d]);
        }
    }
    if (mask & (1u << 0)) T[0] = f.Tz[c - nxy];
    if (mask & (1u << 1)) T[1] = f.Tpp[c - nx - 1];
    if (mask & (1u << 2)) T[2] = f.Ty[c - nx];
    if (mask & (1u << 3)) T[3] = f.Tmp[c - nx + 1];
    if (mask & (1u << 4)) T[4] = f.Tx[c - 1];
    if (mask & (1u << 6)) T[6] = f.Tx[c];
    if (mask & (1u << 7)) T[7] = f.Tmp[c];
    if (mask & (1u << 8)) T[8] = f.Ty[c];
    if (mask & (1u << 9)) T[9] = f.Tpp[c];
    if (mask & (1u << 10)) T[10] = f.Tz[c];
    const long long rs = row_start(g, i, j, k);
    Real* vals = o.vals;
    auto sink = [&](int pos, Real v) { vals[rs + pos] = v; };
    const RowSums r = assemble_row<CRK, JAC>(q, me, nb, T, mask, f.pn[c], f.mn[c], CRK ? f.phi0[c] : Real(0), sink);
    if (o.R) o.R[c] = r.R;
    if (JAC && o.diag64) o.diag64[c] = r.diag64;
    if (r.bad) atomicOr(o.status, STATUS_NONFINITE);
}

// ------------------------------------------------------------------ y-march

template <typename Real>
struct Row3 {
    CellVal<Real> m, c, p;  // cells i-1, i, i+1 of one grid row, for this lane
};

template <typename Real>
__device__ __forceinline__ CellVal<Real> shfl_cell(const CellVal<Real>& v, int delta, bool up,
                                                   const typename PhysOf<Real>::type& q) {
    CellVal<Real> r;
    if (up) {
        r.p = __shfl_up_sync(0xffffffffu, v.p, delta);
        r.z = __shfl_up_sync(0xffffffffu, v.z, delta);
        r.rho = __shfl_up_sync(0xffffffffu, v.rho, delta);
    } else {
        r.p = __shfl_down_sync(0xffffffffu, v.p, delta);
        r.z = __shfl_down_sync(0xffffffffu, v.z, delta);
        r.rho = __shfl_down_sync(0xffffffffu, v.rho, delta);
    }
    // the same product make_cell forms, so shuffled and local cells agree bitwise
    if constexpr (sizeof(Real) == 4) r.drho = __fmul_rn(q.c_f, r.rho);
    else r.drho = __dmul_rn(q.c_f, r.rho);
    return r;
}

// Per-row inputs other than p and z.
template <typename Real>
struct RowData {
    Real Tx, Ty, Tz, Tpp, Tmp, pn, phi0;
    double mn;
    Real p_zm, z_zm, p_zp, z_zp, Tz_m;  // cells (i, j, k-1), (i, j, k+1) and the link to k-1
    Real hT1, hT2;  // lane 0: Tx(i0-1, j), Tpp(i0-1, j-1); lane 31: -, Tmp(i0+32, j-1)
};

template <typename Real, bool DIAG, bool CRK, bool JAC, int W>
__global__ void __launch_bounds__(32 * W) k_assemble_ymarch(GridGeom g, typename PhysOf<Real>::type q,
                                                            AsmFields<Real> f, AsmOut<Real> o, int JY) {
    using Phys = typename PhysOf<Real>::type;
    __shared__ Real stage[JAC ? W : 1][JAC ? 32 * NSLOT : 1];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int i0 = blockIdx.x * 32, i = i0 + lane;
    const int k = blockIdx.z * W + w;
    if (k >= g.nz) return;  // warp-uniform
    const int j0 = blockIdx.y * JY;
    const int j1 = min(j0 + JY, g.ny);
    const long long nx = g.nx, nxy = nx * (long long)g.ny;
    const long long kb = nxy * k;
    const bool act = i < g.nx;
    const int ih = lane == 0 ? i0 - 1 : (lane == 31 ? i0 + 32 : -1);  // halo cell this lane carries
    const bool hact = ih >= 0 && ih < g.nx;
    const bool zm = k > 0, zp = k + 1 < g.nz;
    const Phys& Q = q;

    auto load_pz = [&](int r, Real& po, Real& zo, Real& ph, Real& zh) {
        po = Real(Q.p_ref);
        zo = Real(0);
        ph = Real(Q.p_ref);
        zh = Real(0);
        if (r >= 0 && r < g.ny) {
            const long long rb = kb + nx * r;
            if (act) {
                po = __ldg(f.p + rb + i);
                zo = __ldg(f.z + rb + i);
            }
            if (hact) {
                ph = __ldg(f.p + rb + ih);
                zh = __ldg(f.z + rb + ih);
            }
        }
    };
    auto make_row = [&](Real po, Real zo, Real ph, Real zh) {
        Row3<Real> R;
        R.c = make_cell(Q, po, zo);
        const CellVal<Real> h = make_cell(Q, ph, zh);
        R.m = shfl_cell(R.c, 1, true, Q);
        R.p = shfl_cell(R.c, 1, false, Q);
        if (lane == 0) R.m = h;
        if (lane == 31) R.p = h;
        return R;
    };
    auto load_data = [&](int r) {
        RowData<Real> D;
        D.Tx = D.Ty = D.Tz = D.Tpp = D.Tmp = D.pn = D.phi0 = Real(0);
        D.mn = 0.0;
        D.p_zm = D.p_zp = Real(Q.p_ref);
        D.z_zm = D.z_zp = D.Tz_m = Real(0);
        D.hT1 = D.hT2 = Real(0);
        if (r < g.ny) {
            const long long c = kb + nx * r + i;
            if (act) {
                D.Tx = __ldg(f.Tx + c);
                D.Ty = __ldg(f.Ty + c);
                D.Tz = __ldg(f.Tz + c);
                if (DIAG) {
                    D.Tpp = __ldg(f.Tpp + c);
                    D.Tmp = __ldg(f.Tmp + c);
                }
                D.pn = __ldg(f.pn + c);
                D.mn = __ldg(f.mn + c);
                if (CRK) D.phi0 = __ldg(f.phi0 + c);
                if (zm) {
                    D.p_zm = __ldg(f.p + c - nxy);
                    D.z_zm = __ldg(f.z + c - nxy);
                    D.Tz_m = __ldg(f.Tz + c - nxy);
                }
                if (zp) {
                    D.p_zp = __ldg(f.p + c + nxy);
                    D.z_zp = __ldg(f.z + c + nxy);
                }
            }
            if (lane == 0 && i0 > 0) {
                D.hT1 = __ldg(f.Tx + c - 1);
                if (DIAG && r > 0) D.hT2 = __ldg(f.Tpp + c - nx - 1);
            }
            if (DIAG && lane == 31 && hact && r > 0) D.hT2 = __ldg(f.Tmp + c - nx + 1);
        }
        return D;
    };

    // prologue: rows j0-1, j0, j0+1 and the data of row j0
    Row3<Real> P, C, N;
    {
        Real a, b, c2, d;
        load_pz(j0 - 1, a, b, c2, d);
        P = make_row(a, b, c2, d);
        load_pz(j0, a, b, c2, d);
        C = make_row(a, b, c2, d);
        load_pz(j0 + 1, a, b, c2, d);
        N = make_row(a, b, c2, d);
    }
    RowData<Real> D = load_data(j0);
    Real Ty_prev = Real(0), Tpp_prev = Real(0), Tmp_prev = Real(0);
    if (j0 > 0 && act) {
        const long long c = kb + nx * (j0 - 1) + i;
        Ty_prev = __ldg(f.Ty + c);
        if (DIAG) {
            Tpp_prev = __ldg(f.Tpp + c);
            Tmp_prev = __ldg(f.Tmp + c);
        }
    }

    for (int j = j0; j < j1; ++j) {
        // issue the loads of the rows needed next
        Real a2, b2, c2, d2;
        load_pz(j + 2, a2, b2, c2, d2);
        const RowData<Real> Dn = load_data(j + 1);

        // neighbour transmissibilities owned by the cells to the left and below
        Real Tx_m = __shfl_up_sync(0xffffffffu, D.Tx, 1);
        Real Tpp_pm = Real(0), Tmp_pp = Real(0);
        if (DIAG) {
            Tpp_pm = __shfl_up_sync(0xffffffffu, Tpp_prev, 1);
            Tmp_pp = __shfl_down_sync(0xffffffffu, Tmp_prev, 1);
        }
        if (lane == 0) {
            Tx_m = D.hT1;
            Tpp_pm = D.hT2;
        }
        if (lane == 31) Tmp_pp = D.hT2;

        const unsigned mask = slot_mask(g, i, j, k);
        CellVal<Real> nb[NSLOT];
        nb[0] = zm ? make_cell(Q, D.p_zm, D.z_zm) : C.c;
        nb[1] = P.m;
        nb[2] = P.c;
        nb[3] = P.p;
        nb[4] = C.m;
        nb[5] = C.c;
        nb[6] = C.p;
        nb[7] = N.m;
        nb[8] = N.c;
        nb[9] = N.p;
        nb[10] = zp ? make_cell(Q, D.p_zp, D.z_zp) : C.c;
        Real T[NSLOT];
        T[0] = D.Tz_m;
        T[1] = Tpp_pm;
        T[2] = Ty_prev;
        T[3] = Tmp_pp;
        T[4] = Tx_m;
        T[5] = Real(0);
        T[6] = D.Tx;
        T[7] = D.Tmp;
        T[8] = D.Ty;
        T[9] = D.Tpp;
        T[10] = D.Tz;

        // CSR segment of this warp's row run (cells i0 .. min(i0+32, nx)-1 of row j)
        const int ez = axis_links(k, g.nz), ey = axis_links(j, g.ny);
        const int per = 1 + ey + ez, perx = 1 + g.diag * ey;
        const int lane_off = (i - i0) * per + (int)(axis_links_before(i, g.nx) - axis_links_before(i0, g.nx)) * perx;
        Real* buf = stage[JAC ? w : 0];
        auto sink = [&](int pos, Real v) {
            if (JAC && act) buf[lane_off + pos] = v;
        };
        const RowSums r = assemble_row<CRK, JAC>(Q, C.c, nb, T, mask, D.pn, D.mn, D.phi0, sink);
        const long long c = kb + nx * j + i;
        if (act) {
            if (o.R) o.R[c] = r.R;
            if (JAC && o.diag64) o.diag64[c] = r.diag64;
            if (r.bad) atomicOr(o.status, STATUS_NONFINITE);
        }
        if (JAC) {
            __syncwarp();
            const int iend = min(i0 + 32, g.nx);
            const int seg_len = (iend - i0) * per + (int)(axis_links_before(iend, g.nx) - axis_links_before(i0, g.nx)) * perx;
            const long long seg = row_start(g, i0, j, k);
            Real* dst = o.vals + seg;
            for (int t = lane; t < seg_len; t += 32) dst[t] = buf[t];
            __syncwarp();
        }

        // rotate the window
        Ty_prev = D.Ty;
        Tpp_prev = D.Tpp;
        Tmp_prev = D.Tmp;
        P = C;
        C = N;
        N = make_row(a2, b2, c2, d2);
        D = Dn;
    }
}

// ------------------------------------------------------------------ launchers

template <typename Real, bool CRK, bool JAC>
static cudaError_t launch_naive_t(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                  const AsmFields<Real>& f, const AsmOut<Real>& o, cudaStream_t st) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    k_assemble_naive<Real, CRK, JAC><<<grid, block, 0, st>>>(g, q, f, o);
    return cudaGetLastError();
}

template <typename Real, bool DIAG, bool CRK, bool JAC>
static cudaError_t launch_ymarch_t(const GridGeom& g, const typename PhysOf<Real>::type& q,
                                   const AsmFields<Real>& f, const AsmOut<Real>& o, int JY,
                                   cudaStream_t st) {
    constexpr int W = 4;
    dim3 block(32, W, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + JY - 1) / JY, (g.nz + W - 1) / W);
    k_assemble_ymarch<Real, DIAG, CRK, JAC, W><<<grid, block, 0, st>>>(g, q, f, o, JY);
    return cudaGetLastError();
}

template <typename Real>
static cudaError_t dispatch(AsmKernel kern, const GridGeom& g, const typename PhysOf<Real>::type& q,
                            bool crk, const AsmFields<Real>& f, const AsmOut<Real>& o, int JY,
                            cudaStream_t st) {
    const bool jac = o.vals != nullptr;
    if (kern == AsmKernel::Naive) {
        if (crk) return jac ? launch_naive_t<Real, true, true>(g, q, f, o, st) : launch_naive_t<Real, true, false>(g, q, f, o, st);
        return jac ? launch_naive_t<Real, false, true>(g, q, f, o, st) : launch_naive_t<Real, false, false>(g, q, f, o, st);
    }
    if (g.diag) {
        if (crk) return jac ? launch_ymarch_t<Real, true, true, true>(g, q, f, o, JY, st)
                            : launch_ymarch_t<Real, true, true, false>(g, q, f, o, JY, st);
        return jac ? launch_ymarch_t<Real, true, false, true>(g, q, f, o, JY, st)
                   : launch_ymarch_t<Real, true, false, false>(g, q, f, o, JY, st);
    }
    if (crk) return jac ? launch_ymarch_t<Real, false, true, true>(g, q, f, o, JY, st)
                        : launch_ymarch_t<Real, false, true, false>(g, q, f, o, JY, st);
    return jac ? launch_ymarch_t<Real, false, false, true>(g, q, f, o, JY, st)
               : launch_ymarch_t<Real, false, false, false>(g, q, f, o, JY, st);
}

cudaError_t launch_assemble_mixed(AsmKernel kern, const GridGeom& g, const PhysF& q, bool crk,
                                  const AsmFields<float>& f, const AsmOut<float>& o, int JY,
                                  cudaStream_t st) {
    return dispatch<float>(kern, g, q, crk, f, o, JY, st);
}

cudaError_t launch_assemble_fp64(AsmKernel kern, const GridGeom& g, const PhysD& q, bool crk,
                                 const AsmFields<double>& f, const AsmOut<double>& o, int JY,
                                 cudaStream_t st) {
    return dispatch<double>(kern, g, q, crk, f, o, JY, st);
}

}  // namespace tpfa
