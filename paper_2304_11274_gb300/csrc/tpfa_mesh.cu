// tpfa_mesh.cu -- residual and Jacobian of Eq. vk on a general mesh given as a
// list of connections (K, L, Upsilon_KL), the extension to arbitrary mesh
// topologies (corner-point grids with faults, unstructured meshes) that the
// paper names as future work (Section 8).  sm_103a.
//
// Gather form: one thread per row K walks row K of the pattern (columns
// ascending) and evaluates every link from K's side with the same link() and
// accumulation() arithmetic as the structured kernels, so a structured grid
// passed as a connection list sums in the same (ascending-column) order.  No
// atomics: each link is evaluated once from each side (bit-exact
// antisymmetry of F).  A block's 128 rows own one contiguous stretch of the
// CSR values, staged in shared memory and written out with consecutive-lane
// stores (rows longer than the staging buffer fall back to direct stores).
// Neighbour gathers go through a checked load.
#include <cuda_runtime.h>

#include "tpfa_impl.h"
#include "tpfa_row.cuh"

namespace tpfa {

namespace {

constexpr int kRows = 128;
constexpr int kStage = kRows * 16;  // staged CSR values per block

template <typename T>
__device__ __forceinline__ T ldm(const T* p, long long idx, long long n, unsigned int* status) {
    if (idx < 0 || idx >= n) {
        atomicOr(status, STATUS_DEVICE_CHECK);
        return T(0);
    }
    return __ldg(p + idx);
}

template <typename Real, bool CRK, bool JAC>
__global__ void __launch_bounds__(kRows) k_mesh_assemble(MeshFields<Real> f, long long n,
                                                         typename PhysOf<Real>::type q, AsmOut<Real> o) {
    __shared__ Real stage[kStage];
    const long long r0 = (long long)blockIdx.x * kRows;
    const long long r = r0 + threadIdx.x;
    const long long rl = min(r0 + kRows, n);
    const long long e0 = f.row_ptr[r0], e1 = f.row_ptr[rl];
    const bool staged = JAC && (e1 - e0) <= kStage;
    auto put = [&](long long e, Real v) {
        if (staged) stage[e - e0] = v;
        else o.vals[e] = v;
    };
    if (r < n) {
        const long long rs = f.row_ptr[r], re = f.row_ptr[r + 1];
        const long long nnz = f.row_ptr[n];
        const CellVal<Real> me = make_cell(q, f.p[r], f.z[r]);
        long long dpos = rs;
        RowSums out;
        if constexpr (sizeof(Real) == 4) {
            Kahan32 rsum, dsum;
            for (long long e = rs; e < re; ++e) {
                const long long c = ldm(f.col, e, nnz, o.status);
                if (c == r) {
                    dpos = e;
                    continue;
                }
                const CellVal<float> nb = make_cell(q, ldm(f.p, c, n, o.status), ldm(f.z, c, n, o.status));
                const LinkOut<float> L = link(q, ldm(f.Tc, e, nnz, o.status), me, nb);
                rsum.add(L.F);
                if (JAC) {
                    dsum.add(L.Da);
                    put(e, L.Db);
                }
            }
            const AccF acc = accumulation<CRK>(q, me.p, f.pn[r], f.mn[r], me.rho, CRK ? f.phi0[r] : 0.f);
            out.R = __dadd_rn(__dadd_rn(acc.A, widen(rsum.s)), -widen(rsum.c));
            out.diag64 = 0.0;
            if (JAC) {
                dsum.add(acc.dA);
                out.diag64 = __dadd_rn(widen(dsum.s), -widen(dsum.c));
                put(dpos, __fsub_rn(dsum.s, dsum.c));
            }
        } else {
            double rsum = 0.0, dsum = 0.0;
            for (long long e = rs; e < re; ++e) {
                const long long c = ldm(f.col, e, nnz, o.status);
                if (c == r) {
                    dpos = e;
                    continue;
                }
                const CellVal<double> nb = make_cell(q, ldm(f.p, c, n, o.status), ldm(f.z, c, n, o.status));
                const LinkOut<double> L = link(q, ldm(f.Tc, e, nnz, o.status), me, nb);
                rsum = __dadd_rn(rsum, L.F);
                if (JAC) {
                    dsum = __dadd_rn(dsum, L.Da);
                    put(e, L.Db);
                }
            }
            const AccD acc = accumulation<CRK>(q, me.p, f.pn[r], f.mn[r], me.rho, CRK ? f.phi0[r] : 0.0);
            out.R = __dadd_rn(rsum, acc.A);
            out.diag64 = 0.0;
            if (JAC) {
                dsum = __dadd_rn(dsum, acc.dA);
                out.diag64 = dsum;
                put(dpos, dsum);
            }
        }
        if (o.R) o.R[r] = out.R;
        if (JAC && o.diag64) o.diag64[r] = out.diag64;
        if (nonfinite(out.R) || (JAC && nonfinite(out.diag64))) atomicOr(o.status, STATUS_NONFINITE);
    }
    if (staged) {  // block-uniform
        __syncthreads();
        for (long long e = e0 + threadIdx.x; e < e1; e += kRows) o.vals[e] = stage[e - e0];
    }
}

// (V / dt) phi0 per cell in FP64, and in the field type when c_r != 0.
template <typename Real>
__global__ void k_mesh_vphi(long long n, double inv_dt, const double* __restrict__ V, const double* __restrict__ poro,
                            double* vphi_d, Real* vphi_r) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double v = (V[c] * inv_dt) * poro[c];
        vphi_d[c] = v;
        if (vphi_r) vphi_r[c] = (Real)v;
    }
}

unsigned blocks_of(long long n, int per) {
    long long b = (n + per - 1) / per;
    return (unsigned)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

template <typename Real>
cudaError_t launch_mesh_t(const MeshFields<Real>& f, long long n, const typename PhysOf<Real>::type& q, bool crk,
                          const AsmOut<Real>& o, cudaStream_t st) {
    const unsigned nb = (unsigned)((n + kRows - 1) / kRows);
    const bool jac = o.vals != nullptr;
    if (crk) {
        if (jac) k_mesh_assemble<Real, true, true><<<nb, kRows, 0, st>>>(f, n, q, o);
        else k_mesh_assemble<Real, true, false><<<nb, kRows, 0, st>>>(f, n, q, o);
    } else {
        if (jac) k_mesh_assemble<Real, false, true><<<nb, kRows, 0, st>>>(f, n, q, o);
        else k_mesh_assemble<Real, false, false><<<nb, kRows, 0, st>>>(f, n, q, o);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mesh_vphi(long long n, double dt, bool mixed, const double* V, const double* poro,
                             double* vphi_d, void* vphi_r, cudaStream_t st) {
    if (mixed)
        k_mesh_vphi<float><<<blocks_of(n, 256), 256, 0, st>>>(n, 1.0 / dt, V, poro, vphi_d, (float*)vphi_r);
    else
        k_mesh_vphi<double><<<blocks_of(n, 256), 256, 0, st>>>(n, 1.0 / dt, V, poro, vphi_d, (double*)vphi_r);
    return cudaGetLastError();
}

cudaError_t launch_mesh_mixed(const MeshFields<float>& f, long long n, const PhysF& q, bool crk,
                              const AsmOut<float>& o, cudaStream_t st) {
    return launch_mesh_t<float>(f, n, q, crk, o, st);
}

cudaError_t launch_mesh_fp64(const MeshFields<double>& f, long long n, const PhysD& q, bool crk,
                             const AsmOut<double>& o, cudaStream_t st) {
    return launch_mesh_t<double>(f, n, q, crk, o, st);
}

}  // namespace tpfa
