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
// Host code cannot use the array's name as a device address, so the first
// call on each device asks the runtime for the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it.
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

// Device address of g_workspace on the current device (set up once per device).
cudaError_t workspace_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_workspace);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

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

    // Workspace layout: error word, owned transmissibilities, and for the
    // mixed path the FP32 depth (and FP32 phi0 when c_r != 0); then m^n.
    const bool mixed = prec == TPFA_MIXED;
    const bool crk = prm->c_r != 0.0;
    const size_t rs = mixed ? sizeof(float) : sizeof(double);
    const int nT = prm->connectivity == 10 ? 5 : 3;
    size_t off = 256;  // the error word sits in the first 256 bytes
    size_t offT[5] = {0, 0, 0, 0, 0};
    for (int t = 0; t < nT; ++t) {
        offT[t] = off;
        off += align256(rs * (size_t)N);
    }
    size_t offZ = 0, offPhi = 0;
    if (mixed) {
        offZ = off;
        off += align256(rs * (size_t)N);
        if (crk) {
            offPhi = off;
            off += align256(rs * (size_t)N);
        }
    }
    const size_t offM = off;
    off += align256(sizeof(double) * (size_t)N);
    if (off > kWorkspaceBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "static assembly: a %d x %d x %d grid needs %zu bytes of workspace, more than the fixed %zu "
                 "(use the handle API for larger grids)", nx, ny, nz, off, kWorkspaceBytes);
        return report_error(TPFA_ERR_TOO_LARGE, msg);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report_error(TPFA_ERR_CUDA, "static assembly: no usable current device");
    unsigned char* ws = nullptr;
    cudaError_t ea = workspace_address(dev, &ws);
    if (ea != cudaSuccess) return report_error(TPFA_ERR_CUDA, cudaGetErrorString(ea));

    cudaStream_t st = static_cast<cudaStream_t>(stream);
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
        float* phi = crk ? reinterpret_cast<float*>(ws + offPhi) : nullptr;
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
