// tpfa_static.cu -- residual + Jacobian assembly that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose own
// pooled allocator has reserved the GPU's memory up front, processes with a
// hard device-memory budget enforced outside the CUDA runtime, or code that
// runs where a new allocation is not allowed.  tpfa_assemble_jacobian_static
// serves them.  It runs the same setup and assembly kernels as the handle
// API, but every intermediate array (the owned transmissibilities, the FP32
// depth, m^n and the error word) lives in one fixed workspace: a file-scope
// __device__ array of TPFA_STATIC_WORKSPACE_BYTES, which every GPU that loads
// the library holds until the process exits.  The caller passes all inputs
// and outputs.
//
// The workspace is shared by every call and keeps the last call's contents;
// each call overwrites what it reads and clears its error word first.  Calls
// whose work overlaps on the GPU (different streams, or different host
// threads, without ordering between them) race on the workspace.
//
// Host code cannot use the array's name as a device address, so each call
// asks the runtime for the array's device address on the current device
// (cudaGetSymbolAddress) and keeps it per device.  While the stream is being
// captured into a CUDA graph the kept address is used instead of a new
// query, so the first call on a device must come before any capture.  A
// call outside capture always queries afresh: after cudaDeviceReset the
// library's module is loaded again, possibly elsewhere, and an address kept
// from before would point at freed memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "tpfa_common.cuh"
#include "tpfa_impl.h"

using namespace tpfa;

namespace {

constexpr size_t kWorkspaceBytes = (size_t)TPFA_STATIC_WORKSPACE_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_workspace[kWorkspaceBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_workspace on device `dev` (current): queried on every
// call outside stream capture, the kept one during capture.
cudaError_t workspace_address(int dev, cudaStream_t st, unsigned char** out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_addr[dev]) {
        if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;  // no address kept yet
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_workspace);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout: the error word in the first 256 bytes, then each array
// from a 256-byte boundary: the owned transmissibilities (3 or 5, field
// type), on the mixed path the FP32 depth (and the FP32 phi0 when c_r != 0),
// then m^n (FP64).  Returns the bytes used.
struct Layout {
    size_t T[5] = {0, 0, 0, 0, 0};
    size_t z = 0, phi = 0, mn = 0;
};
size_t layout(long long N, int connectivity, bool mixed, bool crk, Layout* L) {
    const size_t rs = mixed ? sizeof(float) : sizeof(double);
    const int nT = connectivity == 10 ? 5 : 3;
    size_t off = 256;
    for (int t = 0; t < nT; ++t) {
        L->T[t] = off;
        off += align256(rs * (size_t)N);
    }
    if (mixed) {
        L->z = off;
        off += align256(rs * (size_t)N);
        if (crk) {
            L->phi = off;
            off += align256(rs * (size_t)N);
        }
    }
    L->mn = off;
    off += align256(sizeof(double) * (size_t)N);
    return off;
}

}  // namespace

extern "C" int tpfa_assemble_jacobian_static(int nx, int ny, int nz, const tpfa_params* prm, tpfa_precision prec,
                                             const double* perm_dev, const double* poro_dev, const double* depth_dev,
                                             const void* p_dev, const void* p_prev_dev, double* R_dev, void* vals_dev,
                                             double* diag64_dev, unsigned int* status_dev, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !prm || (prm->connectivity != 6 && prm->connectivity != 10) ||
        (prec != TPFA_FP64 && prec != TPFA_MIXED) || !(prm->mu > 0.0) || !(prm->dt > 0.0) || !(prm->dx > 0.0) ||
        !(prm->dy > 0.0) || !(prm->dz > 0.0))
        return report_error(TPFA_ERR_INVALID_ARG, "static assembly: bad grid size, parameters or precision");
    if (!perm_dev || !poro_dev || !depth_dev || !p_dev || !p_prev_dev || !vals_dev)
        return report_error(TPFA_ERR_INVALID_ARG, "static assembly: an input or the values pointer is NULL");
    if (prec == TPFA_FP64 && diag64_dev)
        return report_error(TPFA_ERR_INVALID_ARG, "static assembly: diag64 must be NULL on the FP64 path");
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31)) return report_error(TPFA_ERR_TOO_LARGE, "static assembly: N exceeds 2^31 - 1");

    const bool mixed = prec == TPFA_MIXED;
    const bool crk = prm->c_r != 0.0;
    Layout L;
    const size_t need = layout(N, prm->connectivity, mixed, crk, &L);
    if (need > kWorkspaceBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "static assembly: a %d x %d x %d grid needs %zu bytes of workspace, more than the fixed %zu "
                 "(use the handle API for larger grids)", nx, ny, nz, need, kWorkspaceBytes);
        return report_error(TPFA_ERR_TOO_LARGE, msg);
    }
    const int nT = prm->connectivity == 10 ? 5 : 3;
    const size_t* offT = L.T;
    const size_t offZ = L.z, offPhi = L.phi, offM = L.mn;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report_error(TPFA_ERR_CUDA, "static assembly: no usable current device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* ws = nullptr;
    cudaError_t ea = workspace_address(dev, st, &ws);
    if (ea != cudaSuccess) return report_error(TPFA_ERR_CUDA, cudaGetErrorString(ea));

    unsigned int* status = status_dev ? status_dev : reinterpret_cast<unsigned int*>(ws);
    const GridGeom g{nx, ny, nz, prm->connectivity == 10 ? 1 : 0};
    const double V_dt = prm->dx * prm->dy * prm->dz / prm->dt;
    const SetupPhys sp{prm->dx, prm->dy, prm->dz, prm->rho_ref, prm->p_ref, prm->c_f, prm->c_r, V_dt};
    void* T[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int t = 0; t < nT; ++t) T[t] = ws + offT[t];
    double* mn = reinterpret_cast<double*>(ws + offM);

    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned int), st);
    if (mixed) {
        float* z = reinterpret_cast<float*>(ws + offZ);
        float* phi = crk ? reinterpret_cast<float*>(ws + offPhi) : z;  // read only when c_r != 0; never NULL
        if (e == cudaSuccess)
            e = launch_transmissibility_f32(g, sp, perm_dev, (float*)T[0], (float*)T[1], (float*)T[2], (float*)T[3],
                                            (float*)T[4], st);
        if (e == cudaSuccess) e = launch_convert_f32(depth_dev, z, N, st);
        if (e == cudaSuccess && crk) e = launch_convert_f32(poro_dev, phi, N, st);
        if (e == cudaSuccess) e = launch_prev_mass_f32(sp, (const float*)p_prev_dev, poro_dev, mn, N, st);
        if (e == cudaSuccess) {
            const PhysF q{(float)prm->rho_ref, (float)prm->p_ref, (float)prm->c_f, (float)(1.0 / prm->mu),
                          (float)prm->g, (float)(0.5 * prm->g), (float)V_dt, (float)prm->c_r};
            AsmFields<float> f{(const float*)p_dev, (const float*)p_prev_dev, mn, z, phi,
                               (const float*)T[0], (const float*)T[1], (const float*)T[2],
                               (const float*)(T[3] ? T[3] : T[0]), (const float*)(T[4] ? T[4] : T[0])};
            AsmOut<float> o{R_dev, (float*)vals_dev, diag64_dev, status};
            e = launch_assemble_mixed(AsmKernel::YMarch, g, q, crk, f, o, 32, 4, st);
        }
    } else {
        if (e == cudaSuccess)
            e = launch_transmissibility_f64(g, sp, perm_dev, (double*)T[0], (double*)T[1], (double*)T[2],
                                            (double*)T[3], (double*)T[4], st);
        if (e == cudaSuccess) e = launch_prev_mass_f64(sp, (const double*)p_prev_dev, poro_dev, mn, N, st);
        if (e == cudaSuccess) {
            const PhysD q{prm->rho_ref, prm->p_ref, prm->c_f, 1.0 / prm->mu, prm->g, 0.5 * prm->g, V_dt, prm->c_r};
            AsmFields<double> f{(const double*)p_dev, (const double*)p_prev_dev, mn, depth_dev, poro_dev,
                                (const double*)T[0], (const double*)T[1], (const double*)T[2],
                                (const double*)(T[3] ? T[3] : T[0]), (const double*)(T[4] ? T[4] : T[0])};
            AsmOut<double> o{R_dev, (double*)vals_dev, nullptr, status};
            e = launch_assemble_fp64(AsmKernel::YMarch, g, q, crk, f, o, 32, 4, st);
        }
    }
    if (e != cudaSuccess) return report_error(TPFA_ERR_CUDA, cudaGetErrorString(e));
    return TPFA_OK;
}

extern "C" long long tpfa_static_workspace_bytes(int nx, int ny, int nz, int connectivity, tpfa_precision prec,
                                                 int rock_compressible) {
    if (nx < 1 || ny < 1 || nz < 1 || (connectivity != 6 && connectivity != 10) ||
        (prec != TPFA_FP64 && prec != TPFA_MIXED))
        return report_error(TPFA_ERR_INVALID_ARG, "static workspace size: bad grid size, connectivity or precision");
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31)) return report_error(TPFA_ERR_TOO_LARGE, "static workspace size: N exceeds 2^31 - 1");
    Layout L;
    return (long long)layout(N, connectivity, prec == TPFA_MIXED, rock_compressible != 0, &L);
}
