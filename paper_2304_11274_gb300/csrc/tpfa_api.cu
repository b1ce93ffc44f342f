// tpfa_api.cu -- the C ABI declared in include/tpfa.h.
//
// Host logic only: argument checks, device memory of the handle, launches.
// Every computation runs in the kernels of tpfa_setup.cu / tpfa_assemble.cu;
// there is no host fallback.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "tpfa_common.cuh"
#include "tpfa_impl.h"

using namespace tpfa;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(TPFA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// TPFA_FAULT_INJECT=alloc makes every device allocation of the library fail,
// so the out-of-memory path (error code, nothing leaked) can be tested
// without exhausting a GPU.
bool alloc_fault_injected() {
    const char* v = getenv("TPFA_FAULT_INJECT");
    return v != nullptr && strcmp(v, "alloc") == 0;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes > 0 ? bytes : 1);
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace tpfa {
// Error reporting for entry points defined in other translation units.
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }

cudaError_t ensure_smem_limit(const void* func, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;  // (kernel, device) pairs whose limit is raised
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({func, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({func, dev});
    return e;
}
}  // namespace tpfa

struct tpfa_grid {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    tpfa_precision prec = TPFA_FP64;
    tpfa_params prm{};
    GridGeom geom{};
    PhysF qf{};
    PhysD qd{};
    SetupPhys sp{};
    bool crk = false;
    size_t real_size = 8;
    void* T[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // Tx, Ty, Tz, Tpp, Tmp
    void* z = nullptr;
    void* kperm = nullptr;  // permeability in the field type (adjoint)
    float2* vsplit = nullptr;  // the mixed adjoint's cotangent as FP32 pairs (allocated on first use)
    LinkGeo lg{};           // distance / area per link direction (adjoint)
    double* phi0_d = nullptr;
    void* phi0_r = nullptr;  // phi0 in the field type (mixed path with c_r != 0)
    double* mn = nullptr;
    unsigned int* status = nullptr;
    long long* row_ptr = nullptr;
    int* col_idx = nullptr;
    long long nnz = 0;
    const void* p = nullptr;
    const void* pn = nullptr;
    bool has_state = false;
    int JY = 32;  // rows per warp march (tpfa_autotune may change it)
    int sms = 0;  // multiprocessors of the grid's device
    int W = 4;    // warps (z-planes) per block
    // a z-slab of a larger grid (tpfa_create_slab): the handle's planes are
    // the slab and its one-plane halos; assemblies write the rows of the
    // owned planes [own0, own1) only
    bool slab = false;
    int own0 = 0, own1 = 0;       // owned planes, local numbering
    int slab_k0 = 0, slab_k1 = 0; // owned planes, the larger grid's numbering
    int slab_nz = 0;              // planes of the larger grid
    // tensor maps of the TMA march (mixed path): the library-owned fields'
    // maps are encoded once (tm_static: 0 not yet, 1 done, -1 impossible),
    // those of p and p^n whenever the bound pointers change
    TmaMaps tm{};
    int tm_static = 0;
    bool tm_state = false;
    const void* tm_p = nullptr;
    const void* tm_pn = nullptr;
    // buffers of the host-memory entry point, allocated on first use
    void* h_p = nullptr;
    double* h_R = nullptr;
    void* h_vals = nullptr;
    double* h_diag = nullptr;
    // the host-buffer pipeline's copy streams and per-slab events
    static constexpr int kMaxSlabs = 16;
    cudaStream_t h_up = nullptr, h_down = nullptr;
    cudaEvent_t h_ev[2 * kMaxSlabs + 2] = {};
    // Newton / Krylov workspace, allocated on first use
    void* kv_vals = nullptr;
    double* kv_diag = nullptr;
    double* kv_R = nullptr;
    double* kv_vec[12] = {};  // x, r, r^, p, p^, v, s, s^, t, M^-1 (and z-line multipliers, super-diagonal)
    float* kv_f32[4] = {};    // p^ and s^ split into FP32 pairs (mixed path)
    double* kv_part = nullptr;
    KrylovScalars* kv_S = nullptr;
    KrylovScalars* kv_S_host = nullptr;  // pinned
    // the solve's batches of iterations as one CUDA graph, launched on a
    // library stream that follows the caller's stream through events
    cudaStream_t kv_stream = nullptr;
    cudaEvent_t kv_ev[2] = {};
    cudaGraphExec_t kv_exec = nullptr;
    const double* kv_exec_x = nullptr;  // what the graph was captured for
    int kv_exec_every = 0;
    bool kv_exec_line = false;

    void release() {
        for (auto& ev : h_ev) {
            if (ev) cudaEventDestroy(ev);
            ev = nullptr;
        }
        if (h_up) cudaStreamDestroy(h_up);
        if (h_down) cudaStreamDestroy(h_down);
        h_up = h_down = nullptr;
        dev_free(kv_vals);
        dev_free(kv_diag);
        dev_free(kv_R);
        for (auto& v : kv_vec) dev_free(v), v = nullptr;
        for (auto& v : kv_f32) dev_free(v), v = nullptr;
        dev_free(kv_part);
        dev_free(kv_S);
        if (kv_S_host) cudaFreeHost(kv_S_host);
        kv_vals = nullptr, kv_diag = nullptr, kv_R = nullptr, kv_part = nullptr, kv_S = nullptr, kv_S_host = nullptr;
        if (kv_exec) cudaGraphExecDestroy(kv_exec);
        for (auto& ev : kv_ev)
            if (ev) cudaEventDestroy(ev), ev = nullptr;
        if (kv_stream) cudaStreamDestroy(kv_stream);
        kv_exec = nullptr, kv_stream = nullptr;
        for (auto& t : T) dev_free(t), t = nullptr;
        dev_free(z);
        dev_free(kperm);
        dev_free(vsplit);
        vsplit = nullptr;
        dev_free(phi0_d);
        dev_free(phi0_r);
        dev_free(mn);
        dev_free(status);
        dev_free(row_ptr);
        dev_free(col_idx);
        dev_free(h_p);
        dev_free(h_R);
        dev_free(h_vals);
        dev_free(h_diag);
        z = nullptr, kperm = nullptr, phi0_d = nullptr, phi0_r = nullptr, mn = nullptr, status = nullptr;
        row_ptr = nullptr, col_idx = nullptr, h_p = nullptr, h_R = nullptr, h_vals = nullptr, h_diag = nullptr;
    }
};

namespace {

bool finite_pos(double x) { return x > 0.0 && x < 1e300; }

int check_params(const tpfa_params* prm) {
    if (!prm) return fail(TPFA_ERR_INVALID_ARG, "params is NULL");
    if (prm->connectivity != 6 && prm->connectivity != 10)
        return fail(TPFA_ERR_INVALID_ARG, "connectivity must be 6 or 10 (got %d)", prm->connectivity);
    if (!finite_pos(prm->mu)) return fail(TPFA_ERR_INVALID_ARG, "mu must be > 0");
    if (!(prm->dt > 0.0)) return fail(TPFA_ERR_INVALID_ARG, "dt must be > 0");
    if (!finite_pos(prm->dx) || !finite_pos(prm->dy) || !finite_pos(prm->dz))
        return fail(TPFA_ERR_INVALID_ARG, "cell sizes must be > 0");
    if (!(prm->rho_ref > 0.0)) return fail(TPFA_ERR_INVALID_ARG, "rho_ref must be > 0");
    return TPFA_OK;
}

template <typename Real>
AsmFields<Real> fields_of(const tpfa_grid* h) {
    AsmFields<Real> f;
    f.p = static_cast<const Real*>(h->p);
    f.pn = static_cast<const Real*>(h->pn);
    f.mn = h->mn;
    f.z = static_cast<const Real*>(h->z);
    // phi0 in the field type exists only when c_r != 0 (the only case that
    // reads it); otherwise the pointer names the depth array, so that no
    // kernel ever receives a NULL field pointer
    f.phi0 = static_cast<const Real*>(h->phi0_r ? h->phi0_r : h->z);
    f.Tx = static_cast<const Real*>(h->T[0]);
    f.Ty = static_cast<const Real*>(h->T[1]);
    f.Tz = static_cast<const Real*>(h->T[2]);
    // 6-point grids have no diagonal links; their pointers still name a valid
    // array so that no load, even one a compiler hoists out of its guard, can
    // dereference NULL.
    f.Tpp = static_cast<const Real*>(h->T[3] ? h->T[3] : h->T[0]);
    f.Tmp = static_cast<const Real*>(h->T[4] ? h->T[4] : h->T[0]);
    return f;
}

// Whether the TMA march can run at the bound state (mixed path, nx a
// multiple of 4, every field 16-byte aligned); encodes the tensor maps it
// needs.
bool tma_ready(tpfa_grid* h) {
    if (h->prec != TPFA_MIXED || !h->has_state) return false;
    if (h->tm_static == 0) h->tm_static = tma_encode_static(&h->tm, h->geom, fields_of<float>(h), h->crk) ? 1 : -1;
    if (h->tm_static < 0) return false;
    if (h->tm_p != h->p || h->tm_pn != h->pn) {
        h->tm_state = tma_encode_state(&h->tm, h->geom, static_cast<const float*>(h->p),
                                       static_cast<const float*>(h->pn));
        h->tm_p = h->p;
        h->tm_pn = h->pn;
    }
    return h->tm_state;
}

// The library's choice of assembly kernel: the march with two cells per lane
// on grids at least 256 cells wide, or 128 or 192 wide (whole 64-cell
// segments), else the one-cell march (the dispatch runs the one-cell march
// where the two-cell one does not apply: residual-only calls, the FP64 path,
// odd nx, fields not pair-aligned).  A ragged last segment leaves lanes idle
// and the x-boundary segments cost their lanes masked sums, so narrow grids
// whose width is not a multiple of 64 do better one cell per lane: measured
// (G cells/s, one-cell vs two-cell, best rows per march each) 26.4 vs 28.3 at
// 128^3, 26.9 vs 24.7 at 160 x 160 x 80, 28.5 vs 29.2 at 192 x 160 x 80, 22.3
// vs 18.1 at 224 x 96 x 48, 11.5 vs 10.4 at 64^3, 33.4 vs 36.3 at
// 256 x 256 x 128, 38.0 vs 46.4 at 512 x 512 x 256.  (The TMA march gives the
// same bits but measured 8 % slower than the one-cell march at
// 512 x 512 x 256: its row waits stall where the per-lane prefetch does not.)
AsmKernel auto_kernel(tpfa_grid* h) {
    const int nx = h->nx;
    return nx >= 256 || nx == 128 || nx == 192 ? AsmKernel::XMarch : AsmKernel::YMarch;
}

int launch(tpfa_grid* h, AsmKernel kern, double* R, void* vals, double* diag64, cudaStream_t st, int k0 = 0,
           int k1 = -1) {
    cudaError_t e;
    if (h->slab) {  // a slab assembles its owned planes only
        if (kern == AsmKernel::Naive) kern = AsmKernel::YMarch;
        k0 = h->own0;
        k1 = h->own1;
    }
    if (kern == AsmKernel::YMarchTma && !tma_ready(h))
        return fail(TPFA_ERR_INVALID_ARG,
                    "the TMA march needs the mixed path, nx a multiple of 4 and 16-byte aligned p and p^n");
    if (h->prec == TPFA_MIXED) {
        AsmOut<float> o{R, static_cast<float*>(vals), diag64, h->status};
        if (kern == AsmKernel::YMarchTma)
            e = launch_assemble_mixed_tma(h->geom, h->qf, h->crk, fields_of<float>(h), o, h->tm, h->JY, h->W, st, k0,
                                          k1);
        else
            e = launch_assemble_mixed(kern, h->geom, h->qf, h->crk, fields_of<float>(h), o, h->JY, h->W, st, k0, k1);
    } else {
        AsmOut<double> o{R, static_cast<double*>(vals), nullptr, h->status};
        e = launch_assemble_fp64(kern, h->geom, h->qd, h->crk, fields_of<double>(h), o, h->JY, h->W, st, k0, k1);
    }
    if (e != cudaSuccess) return cuda_fail(e, "assembly launch");
    return TPFA_OK;
}

// The adjoint's kernel for TPFA_KERNEL_AUTO: the one-cell march.  The
// two-cell adjoint march issues 18 % fewer instructions per cell but needs
// 168 registers (12 warps per multiprocessor, a few spilled values) against
// 119 (16 warps): measured (G cells/s per call, one-cell vs two-cell) 21.4
// vs 17.2 at 128^3, 28.4 vs 26.2 at 256 x 256 x 128, 32.7 vs 32.5 at
// 512 x 512 x 256.
AsmKernel vjp_auto_kernel(tpfa_grid*) { return AsmKernel::YMarch; }

int check_handle(tpfa_handle h) {
    if (!h) return fail(TPFA_ERR_INVALID_ARG, "handle is NULL");
    return TPFA_OK;
}

// Rows per march for the J w and adjoint marches: the grid's tiling, halved
// (down to 8) until the launch has at least four blocks per multiprocessor,
// so that small grids still fill the GPU.
int march_rows(const tpfa_grid* h) {
    int jy = h->JY;
    const long long bx = (h->nx + 31) / 32, bz = (h->nz + h->W - 1) / h->W;
    while (jy > 8 && h->sms > 0 && bx * ((h->ny + jy - 1) / jy) * bz < 4LL * h->sms) jy /= 2;
    return jy;
}

// The same for the two-cell marches (64-cell x-segments, three blocks of
// four warps per multiprocessor).
int march_rows2(const tpfa_grid* h) {
    int jy = h->JY;
    const long long bx = (h->nx + 63) / 64, bz = (h->nz + h->W - 1) / h->W;
    while (jy > 8 && h->sms > 0 && bx * ((h->ny + jy - 1) / jy) * bz < 3LL * h->sms) jy /= 2;
    return jy;
}

// Newton / Krylov workspace: the assembled Jacobian, R, twelve FP64 vectors,
// the partial sums and the scalar record (device and pinned host copies).
int krylov_workspace(tpfa_grid* h) {
    if (h->kv_S_host) return TPFA_OK;
    const size_t nb = sizeof(double) * (size_t)h->N;
    bool ok = dev_alloc(&h->kv_vals, h->real_size * (size_t)h->nnz) == cudaSuccess;
    if (ok && h->prec == TPFA_MIXED) ok = dev_alloc((void**)&h->kv_diag, nb) == cudaSuccess;
    ok = ok && dev_alloc((void**)&h->kv_R, nb) == cudaSuccess;
    for (auto& v : h->kv_vec) ok = ok && dev_alloc((void**)&v, nb) == cudaSuccess;
    if (h->prec == TPFA_MIXED)
        for (auto& v : h->kv_f32) ok = ok && dev_alloc((void**)&v, sizeof(float) * (size_t)h->N) == cudaSuccess;
    ok = ok && dev_alloc((void**)&h->kv_part, sizeof(double) * 2 * (size_t)krylov_partials(h->geom, h->N)) ==
                   cudaSuccess;
    ok = ok && dev_alloc((void**)&h->kv_S, sizeof(KrylovScalars)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&h->kv_S_host, sizeof(KrylovScalars)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dev_free(h->kv_vals);
        dev_free(h->kv_diag);
        dev_free(h->kv_R);
        for (auto& v : h->kv_vec) dev_free(v), v = nullptr;
        for (auto& v : h->kv_f32) dev_free(v), v = nullptr;
        dev_free(h->kv_part);
        dev_free(h->kv_S);
        if (h->kv_S_host) cudaFreeHost(h->kv_S_host);
        h->kv_vals = nullptr, h->kv_diag = nullptr, h->kv_R = nullptr, h->kv_part = nullptr, h->kv_S = nullptr;
        h->kv_S_host = nullptr;
        return fail(TPFA_ERR_OOM, "device allocation failed for the Newton/Krylov workspace");
    }
    return TPFA_OK;
}

// Solve J x = sign * b with the Jacobian held in the workspace.
int krylov_solve(tpfa_grid* h, const double* b, double sign, double* x, const tpfa_krylov_opts* opts,
                 tpfa_krylov_stats* stats, cudaStream_t st) {
    const int max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 1000;
    const double rtol = (opts && opts->rtol > 0.0) ? opts->rtol : 1e-8;
    const int every = (opts && opts->check_every > 0) ? opts->check_every : 8;
    const bool line = !(opts && opts->preconditioner == TPFA_PRECOND_JACOBI);
    const bool mixed = h->prec == TPFA_MIXED;
    KrylovWork w;
    w.x = x;
    w.r = h->kv_vec[1];
    w.rh = h->kv_vec[2];
    w.p = h->kv_vec[3];
    w.ph = h->kv_vec[4];
    w.v = h->kv_vec[5];
    w.s = h->kv_vec[6];
    w.sh = h->kv_vec[7];
    w.t = h->kv_vec[8];
    w.dinv = h->kv_vec[9];
    w.lmul = h->kv_vec[10];
    w.up = h->kv_vec[11];
    w.phh = h->kv_f32[0];
    w.phl = h->kv_f32[1];
    w.shh = h->kv_f32[2];
    w.shl = h->kv_f32[3];
    w.part = h->kv_part;
    w.S = h->kv_S;
    KrylovScalars* Sh = h->kv_S_host;
    *Sh = KrylovScalars{};
    Sh->tol2 = rtol * rtol;
    Sh->max_iters = max_iters;
    // The iterations run on the library's stream as CUDA-graph launches of
    // `every` iterations each (ten kernels per iteration: one launch per
    // batch instead of ten per iteration); that stream waits for `st`
    // before the solve and `st` for it after.  A stream that is being
    // captured gets the plain launches instead.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    bool graph = cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    if (graph && !h->kv_stream) {
        graph = cudaStreamCreateWithFlags(&h->kv_stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&h->kv_ev[0], cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&h->kv_ev[1], cudaEventDisableTiming) == cudaSuccess;
        if (!graph) {
            cudaGetLastError();
            for (auto& ev : h->kv_ev)
                if (ev) cudaEventDestroy(ev), ev = nullptr;
            if (h->kv_stream) cudaStreamDestroy(h->kv_stream), h->kv_stream = nullptr;
        }
    }
    cudaGetLastError();
    cudaStream_t ks = st;
    cudaError_t e = cudaSuccess;
    // `st` waits for the library stream on every return after the fork, the
    // error returns included, so that nothing the caller queues next on `st`
    // overlaps iterations still in flight
    auto join = [&]() -> cudaError_t {
        if (ks == st) return cudaSuccess;
        cudaError_t j = cudaEventRecord(h->kv_ev[1], ks);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(st, h->kv_ev[1], 0);
        return j;
    };
    if (graph) {
        e = cudaEventRecord(h->kv_ev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->kv_stream, h->kv_ev[0], 0);
        if (e != cudaSuccess) return cuda_fail(e, "Krylov stream");
        ks = h->kv_stream;
        if (h->kv_exec && (h->kv_exec_x != x || h->kv_exec_every != every || h->kv_exec_line != line)) {
            cudaGraphExecDestroy(h->kv_exec);
            h->kv_exec = nullptr;
        }
        if (!h->kv_exec) {  // capture one batch of iterations
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(ks, cudaStreamCaptureModeThreadLocal);
            cudaError_t el = cudaSuccess;
            for (int q = 0; q < every && e == cudaSuccess && el == cudaSuccess; ++q)
                el = krylov_iteration(h->geom, h->N, mixed, h->kv_vals, h->kv_diag, w, line, ks);
            if (e == cudaSuccess) e = cudaStreamEndCapture(ks, &gr);
            if (e == cudaSuccess) e = el;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->kv_exec, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            if (e != cudaSuccess) {
                h->kv_exec = nullptr;
                join();
                return cuda_fail(e, "Krylov graph");
            }
            h->kv_exec_x = x;
            h->kv_exec_every = every;
            h->kv_exec_line = line;
        }
    }
    e = cudaMemcpyAsync(w.S, Sh, sizeof(KrylovScalars), cudaMemcpyHostToDevice, ks);
    if (e == cudaSuccess) e = krylov_dinv(h->geom, mixed, h->kv_vals, h->kv_diag, w.dinv, w.lmul, w.up, line, ks);
    if (e == cudaSuccess) e = krylov_start(h->geom, h->N, b, sign, w, ks);
    if (e != cudaSuccess) {
        join();
        return cuda_fail(e, "Krylov start");
    }
    // every kernel returns at entry once `done` is set, so batches of
    // `every` iterations may overshoot the stopping point harmlessly; the
    // device stops at max_iters, so this loop ends after at most
    // max_iters / every + 1 polls
    for (int it = 0; it <= max_iters + every; it += every) {
        if (graph) e = cudaGraphLaunch(h->kv_exec, ks);
        for (int q = 0; !graph && q < every && e == cudaSuccess; ++q)
            e = krylov_iteration(h->geom, h->N, mixed, h->kv_vals, h->kv_diag, w, line, ks);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Sh, w.S, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, ks);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ks);
        if (e != cudaSuccess) {
            join();
            return cuda_fail(e, "Krylov iteration");
        }
        if (Sh->done) break;
    }
    e = join();
    if (e != cudaSuccess) return cuda_fail(e, "Krylov stream");
    const bool converged = Sh->done && !Sh->breakdown && Sh->rr <= Sh->tol2 * Sh->bb;
    if (stats) {
        stats->iterations = Sh->iter;
        stats->converged = converged ? 1 : 0;
        stats->breakdown = Sh->breakdown;
        stats->b_norm = sqrt(Sh->bb);
        stats->rel_residual = Sh->bb > 0.0 ? sqrt(Sh->rr / Sh->bb) : 0.0;
    }
    if (!converged)
        return fail(TPFA_ERR_NO_CONVERGENCE, "BiCGStab stopped after %d iterations at relative residual %.3e%s",
                    Sh->iter, Sh->bb > 0.0 ? sqrt(Sh->rr / Sh->bb) : 0.0, Sh->breakdown ? " (breakdown)" : "");
    return TPFA_OK;
}

}  // namespace

// A general mesh: the pattern built from the connection list, per-entry
// transmissibilities, cell fields and the bound state.
struct tpfa_mesh_s {
    int device = 0;
    long long N = 0, nc = 0, nnz = 0;
    tpfa_precision prec = TPFA_MIXED;
    PhysF qf{};
    PhysD qd{};
    SetupPhys sp{};
    bool crk = false;
    size_t real_size = 4;
    long long* row_ptr = nullptr;
    int* col_idx = nullptr;
    void* Tc = nullptr;
    void* z = nullptr;
    double* vphi_d = nullptr;
    void* vphi_r = nullptr;
    double* mn = nullptr;
    unsigned int* status = nullptr;
    const void* p = nullptr;
    const void* pn = nullptr;
    bool has_state = false;

    void release() {
        dev_free(row_ptr);
        dev_free(col_idx);
        dev_free(Tc);
        dev_free(z);
        dev_free(vphi_d);
        dev_free(vphi_r);
        dev_free(mn);
        dev_free(status);
        row_ptr = nullptr, col_idx = nullptr, Tc = nullptr, z = nullptr, vphi_d = nullptr, vphi_r = nullptr;
        mn = nullptr, status = nullptr;
    }
};

namespace {

template <typename Real>
MeshFields<Real> mesh_fields(const tpfa_mesh_s* m) {
    MeshFields<Real> f;
    f.row_ptr = m->row_ptr;
    f.col = m->col_idx;
    f.Tc = static_cast<const Real*>(m->Tc);
    f.p = static_cast<const Real*>(m->p);
    f.pn = static_cast<const Real*>(m->pn);
    f.mn = m->mn;
    f.z = static_cast<const Real*>(m->z);
    f.phi0 = static_cast<const Real*>(m->vphi_r ? m->vphi_r : m->z);  // never NULL; read only when c_r != 0
    return f;
}

// Host-side CSR of a connection list: row K = K and its neighbours, columns
// ascending; Tc[e] the entry's transmissibility (0 on the diagonal).
int build_mesh_pattern(long long n, long long nc, const std::vector<int>& ci, const std::vector<int>& cj,
                       const std::vector<double>& T, std::vector<long long>& row_ptr, std::vector<int>& col,
                       std::vector<double>& Tc) {
    for (long long c = 0; c < nc; ++c) {
        if (ci[c] < 0 || ci[c] >= n || cj[c] < 0 || cj[c] >= n)
            return fail(TPFA_ERR_INVALID_ARG, "connection %lld joins cells %d and %d outside [0, %lld)", c, ci[c],
                        cj[c], n);
        if (ci[c] == cj[c]) return fail(TPFA_ERR_INVALID_ARG, "connection %lld joins cell %d to itself", c, ci[c]);
        if (!(T[c] >= 0.0) || !(T[c] < 1e300))
            return fail(TPFA_ERR_INVALID_ARG, "connection %lld has transmissibility %g", c, T[c]);
    }
    row_ptr.assign(n + 1, 0);
    for (long long c = 0; c < nc; ++c) {
        row_ptr[ci[c] + 1] += 1;
        row_ptr[cj[c] + 1] += 1;
    }
    for (long long K = 0; K < n; ++K) row_ptr[K + 1] += row_ptr[K] + 1;
    const long long nnz = row_ptr[n];
    if (nnz >= (1LL << 31)) return fail(TPFA_ERR_TOO_LARGE, "the pattern has %lld entries (>= 2^31)", nnz);
    col.assign(nnz, 0);
    Tc.assign(nnz, 0.0);
    std::vector<long long> fill(n);
    for (long long K = 0; K < n; ++K) {
        col[row_ptr[K]] = (int)K;
        fill[K] = row_ptr[K] + 1;
    }
    for (long long c = 0; c < nc; ++c) {
        long long e = fill[ci[c]]++;
        col[e] = cj[c];
        Tc[e] = T[c];
        e = fill[cj[c]]++;
        col[e] = ci[c];
        Tc[e] = T[c];
    }
    std::vector<std::pair<int, double>> row;
    for (long long K = 0; K < n; ++K) {
        const long long a = row_ptr[K], b = row_ptr[K + 1];
        row.clear();
        for (long long e = a; e < b; ++e) row.emplace_back(col[e], Tc[e]);
        std::sort(row.begin(), row.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
            return x.first < y.first;
        });
        for (long long e = a; e < b; ++e) {
            col[e] = row[e - a].first;
            Tc[e] = row[e - a].second;
            if (e > a && col[e] == col[e - 1])
                return fail(TPFA_ERR_INVALID_ARG, "cells %lld and %d are connected more than once", K, col[e]);
        }
    }
    return TPFA_OK;
}

}  // namespace

extern "C" {

int tpfa_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* tpfa_last_error_string(void) { return g_err.c_str(); }

int tpfa_math_eval(tpfa_math_fn fn, const double* x_dev, double* y_dev, long long n, void* stream) {
    g_err.clear();
    if (fn != TPFA_MATH_EXP_FP64 && fn != TPFA_MATH_EXPM1_FP64 && fn != TPFA_MATH_EXPM1_FP32)
        return fail(TPFA_ERR_INVALID_ARG, "bad math function %d", (int)fn);
    if (n < 0) return fail(TPFA_ERR_INVALID_ARG, "n must be >= 0");
    if (n > 0 && (!x_dev || !y_dev)) return fail(TPFA_ERR_INVALID_ARG, "x and y must be non-NULL");
    const cudaError_t e = launch_math_eval((int)fn, x_dev, y_dev, n, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "math launch");
    return TPFA_OK;
}

int tpfa_create_grid(tpfa_handle* out, int nx, int ny, int nz, const tpfa_params* prm, tpfa_precision prec,
                     const double* perm_dev, const double* poro_dev, const double* depth_dev, void* stream) {
    g_err.clear();
    if (!out) return fail(TPFA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(TPFA_ERR_INVALID_ARG, "grid sizes must be >= 1 (%d %d %d)", nx, ny, nz);
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31)) return fail(TPFA_ERR_TOO_LARGE, "N = %lld cells exceeds 2^31 - 1", N);
    // the assembly kernels address one z-plane's CSR entries in 32 bits
    if ((long long)nx * ny * 11 >= (1LL << 31))
        return fail(TPFA_ERR_TOO_LARGE, "a %d x %d z-plane has too many Jacobian entries (limit 11 nx ny < 2^31)",
                    nx, ny);
    int rc = check_params(prm);
    if (rc) return rc;
    if (prec != TPFA_FP64 && prec != TPFA_MIXED) return fail(TPFA_ERR_INVALID_ARG, "bad precision %d", (int)prec);
    if (!perm_dev || !poro_dev || !depth_dev) return fail(TPFA_ERR_INVALID_ARG, "perm/poro/depth must be non-NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    tpfa_grid* h = new tpfa_grid();
    h->device = dev;
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        h->sms = 0;
    }
    h->nx = nx, h->ny = ny, h->nz = nz, h->N = N;
    h->prec = prec;
    h->prm = *prm;
    h->geom = GridGeom{nx, ny, nz, prm->connectivity == 10 ? 1 : 0};
    h->crk = prm->c_r != 0.0;
    h->real_size = prec == TPFA_MIXED ? sizeof(float) : sizeof(double);
    const double V_dt = prm->dx * prm->dy * prm->dz / prm->dt;
    h->qd = PhysD{prm->rho_ref, prm->p_ref, prm->c_f, 1.0 / prm->mu, prm->g, 0.5 * prm->g, V_dt, prm->c_r};
    h->qf = PhysF{(float)prm->rho_ref, (float)prm->p_ref, (float)prm->c_f, (float)(1.0 / prm->mu),
                  (float)prm->g, (float)(0.5 * prm->g), (float)V_dt, (float)prm->c_r};
    h->sp = SetupPhys{prm->dx, prm->dy, prm->dz, prm->rho_ref, prm->p_ref, prm->c_f, prm->c_r, V_dt};
    h->lg = LinkGeo{(float)(prm->dx / (prm->dy * prm->dz)), (float)(prm->dy / (prm->dx * prm->dz)),
                    (float)(prm->dz / (prm->dx * prm->dy)),
                    (float)((prm->dx * prm->dx + prm->dy * prm->dy) / (prm->dz * prm->dx * prm->dy))};
    h->nnz = total_nnz(h->geom);

    const size_t rb = h->real_size * (size_t)N;
    const int nT = h->geom.diag ? 5 : 3;
    bool ok = true;
    for (int t = 0; t < nT && ok; ++t) ok = dev_alloc(&h->T[t], rb) == cudaSuccess;
    ok = ok && dev_alloc(&h->z, rb) == cudaSuccess;
    ok = ok && dev_alloc(&h->kperm, rb) == cudaSuccess;
    ok = ok && dev_alloc((void**)&h->phi0_d, sizeof(double) * (size_t)N) == cudaSuccess;
    if (ok && h->crk) ok = dev_alloc(&h->phi0_r, rb) == cudaSuccess;
    ok = ok && dev_alloc((void**)&h->mn, sizeof(double) * (size_t)N) == cudaSuccess;
    ok = ok && dev_alloc((void**)&h->status, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        h->release();
        delete h;
        return fail(TPFA_ERR_OOM, "device allocation failed for a %d x %d x %d grid", nx, ny, nz);
    }
    e = cudaMemsetAsync(h->status, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        if (prec == TPFA_MIXED)
            e = launch_transmissibility_f32(h->geom, h->sp, perm_dev, (float*)h->T[0], (float*)h->T[1], (float*)h->T[2],
                                            (float*)h->T[3], (float*)h->T[4], st);
        else
            e = launch_transmissibility_f64(h->geom, h->sp, perm_dev, (double*)h->T[0], (double*)h->T[1],
                                            (double*)h->T[2], (double*)h->T[3], (double*)h->T[4], st);
    }
    if (e == cudaSuccess)
        e = prec == TPFA_MIXED ? launch_convert_f32(depth_dev, (float*)h->z, N, st)
                               : launch_copy_f64(depth_dev, (double*)h->z, N, st);
    if (e == cudaSuccess)
        e = prec == TPFA_MIXED ? launch_store_perm_f32(perm_dev, (float*)h->kperm, N, st)
                               : launch_store_perm_f64(perm_dev, (double*)h->kperm, N, st);
    if (e == cudaSuccess) e = launch_copy_f64(poro_dev, h->phi0_d, N, st);
    if (e == cudaSuccess && h->crk)
        e = prec == TPFA_MIXED ? launch_convert_f32(poro_dev, (float*)h->phi0_r, N, st)
                               : launch_copy_f64(poro_dev, (double*)h->phi0_r, N, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        h->release();
        delete h;
        return cuda_fail(e, "grid setup");
    }
    *out = h;
    return TPFA_OK;
}

int tpfa_set_state(tpfa_handle h, const void* p_dev, const void* p_prev_dev, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!p_dev || !p_prev_dev) return fail(TPFA_ERR_INVALID_ARG, "p and p_prev must be non-NULL");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = h->prec == TPFA_MIXED
                        ? launch_prev_mass_f32(h->sp, (const float*)p_prev_dev, h->phi0_d, h->mn, h->N, st)
                        : launch_prev_mass_f64(h->sp, (const double*)p_prev_dev, h->phi0_d, h->mn, h->N, st);
    if (e != cudaSuccess) return cuda_fail(e, "set_state launch");
    h->p = p_dev;
    h->pn = p_prev_dev;
    h->has_state = true;
    return TPFA_OK;
}

int tpfa_set_pressure(tpfa_handle h, const void* p_dev) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!p_dev) return fail(TPFA_ERR_INVALID_ARG, "p must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    h->p = p_dev;
    return TPFA_OK;
}

int tpfa_assemble_residual(tpfa_handle h, double* R_dev, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!R_dev) return fail(TPFA_ERR_INVALID_ARG, "R must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    DeviceGuard dg(h->device);
    return launch(h, auto_kernel(h), R_dev, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

int tpfa_assemble_jacobian_kernel(tpfa_handle h, tpfa_kernel kern, double* R_dev, void* vals_dev,
                                  double* diag64_dev, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!vals_dev) return fail(TPFA_ERR_INVALID_ARG, "vals must be non-NULL");
    if (h->prec == TPFA_FP64 && diag64_dev) return fail(TPFA_ERR_INVALID_ARG, "diag64 must be NULL on the FP64 path");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    AsmKernel k;
    switch (kern) {
        case TPFA_KERNEL_AUTO: k = auto_kernel(h); break;
        case TPFA_KERNEL_TILED: k = AsmKernel::YMarch; break;
        case TPFA_KERNEL_TILED_TMA: k = AsmKernel::YMarchTma; break;
        case TPFA_KERNEL_TILED2: k = AsmKernel::XMarch; break;
        case TPFA_KERNEL_NAIVE: k = AsmKernel::Naive; break;
        default: return fail(TPFA_ERR_INVALID_ARG, "bad kernel variant %d", (int)kern);
    }
    DeviceGuard dg(h->device);
    return launch(h, k, R_dev, vals_dev, diag64_dev, static_cast<cudaStream_t>(stream));
}

int tpfa_resolve_kernel(tpfa_handle h, tpfa_kernel kern, int* resolved) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!resolved) return fail(TPFA_ERR_INVALID_ARG, "resolved must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    AsmKernel k;
    switch (kern) {
        case TPFA_KERNEL_AUTO: k = auto_kernel(h); break;
        case TPFA_KERNEL_TILED: k = AsmKernel::YMarch; break;
        case TPFA_KERNEL_TILED_TMA: k = AsmKernel::YMarchTma; break;
        case TPFA_KERNEL_TILED2: k = AsmKernel::XMarch; break;
        case TPFA_KERNEL_NAIVE: k = AsmKernel::Naive; break;
        default: return fail(TPFA_ERR_INVALID_ARG, "bad kernel variant %d", (int)kern);
    }
    // the same fall-backs as launch() and the mixed dispatch
    if (h->slab && k == AsmKernel::Naive) k = AsmKernel::YMarch;
    if (k == AsmKernel::YMarchTma && !tma_ready(h))
        return fail(TPFA_ERR_INVALID_ARG,
                    "the TMA march needs the mixed path, nx a multiple of 4 and 16-byte aligned p and p^n");
    if (k == AsmKernel::XMarch && (h->prec != TPFA_MIXED || !xmarch_ok(h->geom, fields_of<float>(h))))
        k = AsmKernel::YMarch;
    switch (k) {
        case AsmKernel::Naive: *resolved = TPFA_KERNEL_NAIVE; break;
        case AsmKernel::YMarch: *resolved = TPFA_KERNEL_TILED; break;
        case AsmKernel::YMarchTma: *resolved = TPFA_KERNEL_TILED_TMA; break;
        case AsmKernel::XMarch: *resolved = TPFA_KERNEL_TILED2; break;
    }
    return TPFA_OK;
}

int tpfa_assemble_jacobian(tpfa_handle h, double* R_dev, void* vals_dev, double* diag64_dev, void* stream) {
    return tpfa_assemble_jacobian_kernel(h, TPFA_KERNEL_AUTO, R_dev, vals_dev, diag64_dev, stream);
}

int tpfa_assemble_jacobian_host(tpfa_handle h, const void* p_host, double* R_host, void* vals_host,
                                double* diag64_host, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!p_host) return fail(TPFA_ERR_INVALID_ARG, "p_host must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    if (h->slab) return fail(TPFA_ERR_INVALID_ARG, "this call is not available on a slab handle (assembly only)");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t pb = h->real_size * (size_t)h->N;
    const size_t vb = h->real_size * (size_t)h->nnz;
    bool ok = true;
    if (!h->h_p) ok = dev_alloc(&h->h_p, pb) == cudaSuccess;
    if (ok && !h->h_R) ok = dev_alloc((void**)&h->h_R, sizeof(double) * (size_t)h->N) == cudaSuccess;
    if (ok && !h->h_vals) ok = dev_alloc(&h->h_vals, vb) == cudaSuccess;
    if (ok && h->prec == TPFA_MIXED && !h->h_diag)
        ok = dev_alloc((void**)&h->h_diag, sizeof(double) * (size_t)h->N) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(TPFA_ERR_OOM, "device allocation failed for the host-buffer entry point");
    }
    cudaError_t e = cudaSuccess;
    if (!h->h_up) {
        e = cudaStreamCreateWithFlags(&h->h_up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->h_down, cudaStreamNonBlocking);
        for (auto& ev : h->h_ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
    }
    // Pipeline over slabs of whole z-planes (a multiple of 8 planes, so of
    // either block height): the upload of slab s+1's pressure, the assembly
    // of slab s and the download of slab s-1's outputs overlap on three
    // streams.  A slab reads the pressure of its planes and of the plane
    // below its last one; planes are uploaded once, in order.
    const int nz = h->nz;
    int slab = ((nz + tpfa_grid::kMaxSlabs / 2 - 1) / (tpfa_grid::kMaxSlabs / 2) + 7) / 8 * 8;
    if (slab < 8) slab = 8;
    const int nslab = (nz + slab - 1) / slab;
    const size_t plane = (size_t)h->nx * h->ny;
    cudaEvent_t* ev_up = h->h_ev;
    cudaEvent_t* ev_cmp = h->h_ev + tpfa_grid::kMaxSlabs;
    cudaEvent_t ev_start = h->h_ev[2 * tpfa_grid::kMaxSlabs], ev_done = h->h_ev[2 * tpfa_grid::kMaxSlabs + 1];
    e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->h_up, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->h_down, ev_start, 0);
    const void* saved = h->p;
    h->p = h->h_p;
    int up_to = 0;
    for (int s = 0; s < nslab && e == cudaSuccess && rc == TPFA_OK; ++s) {
        const int k0 = s * slab, k1 = std::min(nz, k0 + slab);
        const int need = std::min(nz, k1 + 1);
        if (need > up_to) {
            const size_t off = h->real_size * plane * (size_t)up_to;
            e = cudaMemcpyAsync(static_cast<char*>(h->h_p) + off, static_cast<const char*>(p_host) + off,
                                h->real_size * plane * (size_t)(need - up_to), cudaMemcpyHostToDevice, h->h_up);
            up_to = need;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_up[s], h->h_up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_up[s], 0);
        if (e != cudaSuccess) break;
        rc = launch(h, auto_kernel(h), h->h_R, h->h_vals, h->prec == TPFA_MIXED ? h->h_diag : nullptr, st, k0, k1);
        if (rc) break;
        e = cudaEventRecord(ev_cmp[s], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->h_down, ev_cmp[s], 0);
        const size_t r0 = plane * (size_t)k0, rn = plane * (size_t)(k1 - k0);
        const long long v0 = row_start(h->geom, 0, 0, k0), v1 = k1 == nz ? h->nnz : row_start(h->geom, 0, 0, k1);
        if (e == cudaSuccess && R_host)
            e = cudaMemcpyAsync(R_host + r0, h->h_R + r0, sizeof(double) * rn, cudaMemcpyDeviceToHost, h->h_down);
        if (e == cudaSuccess && vals_host)
            e = cudaMemcpyAsync(static_cast<char*>(vals_host) + h->real_size * (size_t)v0,
                                static_cast<char*>(h->h_vals) + h->real_size * (size_t)v0,
                                h->real_size * (size_t)(v1 - v0), cudaMemcpyDeviceToHost, h->h_down);
        if (e == cudaSuccess && diag64_host && h->prec == TPFA_MIXED)
            e = cudaMemcpyAsync(diag64_host + r0, h->h_diag + r0, sizeof(double) * rn, cudaMemcpyDeviceToHost,
                                h->h_down);
    }
    h->p = saved;
    // whatever was enqueued completes before the call returns
    cudaError_t e2 = cudaEventRecord(ev_done, h->h_down);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, ev_done, 0);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->h_up);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (rc) return rc;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "host-buffer pipeline");
    return TPFA_OK;
}

namespace {
int set_perm(tpfa_handle h, const double* perm_dev, void* stream, bool log_k) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!perm_dev) return fail(TPFA_ERR_INVALID_ARG, "perm must be non-NULL");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (h->prec == TPFA_MIXED) {
        e = launch_transmissibility_f32(h->geom, h->sp, perm_dev, (float*)h->T[0], (float*)h->T[1], (float*)h->T[2],
                                        (float*)h->T[3], (float*)h->T[4], st, log_k);
        if (e == cudaSuccess) e = launch_store_perm_f32(perm_dev, (float*)h->kperm, h->N, st, log_k);
    } else {
        e = launch_transmissibility_f64(h->geom, h->sp, perm_dev, (double*)h->T[0], (double*)h->T[1],
                                        (double*)h->T[2], (double*)h->T[3], (double*)h->T[4], st, log_k);
        if (e == cudaSuccess) e = launch_store_perm_f64(perm_dev, (double*)h->kperm, h->N, st, log_k);
    }
    if (e != cudaSuccess) return cuda_fail(e, "set_permeability launch");
    return TPFA_OK;
}
}  // namespace

int tpfa_set_permeability(tpfa_handle h, const double* perm_dev, void* stream) {
    return set_perm(h, perm_dev, stream, false);
}

int tpfa_set_log_permeability(tpfa_handle h, const double* log_perm_dev, void* stream) {
    return set_perm(h, log_perm_dev, stream, true);
}

int tpfa_vjp_kernel(tpfa_handle h, tpfa_kernel kern, const double* v_dev, double* g_p_dev, double* g_lnk_dev,
                    void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!v_dev || !g_p_dev) return fail(TPFA_ERR_INVALID_ARG, "v and g_p must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    if (h->slab) return fail(TPFA_ERR_INVALID_ARG, "this call is not available on a slab handle (assembly only)");
    AsmKernel k;
    switch (kern) {
        case TPFA_KERNEL_AUTO: k = vjp_auto_kernel(h); break;
        case TPFA_KERNEL_TILED: k = AsmKernel::YMarch; break;
        case TPFA_KERNEL_TILED2: k = AsmKernel::XMarch; break;
        case TPFA_KERNEL_NAIVE: k = AsmKernel::Naive; break;
        default: return fail(TPFA_ERR_INVALID_ARG, "bad kernel variant %d", (int)kern);
    }
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (h->prec == TPFA_MIXED && !h->vsplit) {
        if (dev_alloc((void**)&h->vsplit, sizeof(float2) * (size_t)h->N) != cudaSuccess) {
            cudaGetLastError();
            h->vsplit = nullptr;
            return fail(TPFA_ERR_OOM, "device allocation failed for the adjoint's workspace");
        }
    }
    if (h->prec == TPFA_MIXED)
        e = launch_vjp_mixed(k, h->geom, h->qf, h->crk, fields_of<float>(h), (const float*)h->kperm, h->lg, v_dev,
                             h->vsplit, g_p_dev, g_lnk_dev, h->status,
                             k == AsmKernel::XMarch ? march_rows2(h) : march_rows(h), h->W, st);
    else
        e = launch_vjp_fp64(h->geom, h->qd, h->crk, fields_of<double>(h), (const double*)h->kperm, v_dev, g_p_dev,
                            g_lnk_dev, h->status, st);
    if (e != cudaSuccess) return cuda_fail(e, "vjp launch");
    return TPFA_OK;
}

int tpfa_vjp(tpfa_handle h, const double* v_dev, double* g_p_dev, double* g_lnk_dev, void* stream) {
    return tpfa_vjp_kernel(h, TPFA_KERNEL_AUTO, v_dev, g_p_dev, g_lnk_dev, stream);
}

int tpfa_jvp_kernel(tpfa_handle h, tpfa_kernel kern, const double* w_dev, double* Jw_dev, double* R_dev,
                    void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!w_dev || !Jw_dev) return fail(TPFA_ERR_INVALID_ARG, "w and Jw must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    if (h->slab) return fail(TPFA_ERR_INVALID_ARG, "this call is not available on a slab handle (assembly only)");
    AsmKernel k;
    switch (kern) {
        case TPFA_KERNEL_AUTO:
        case TPFA_KERNEL_TILED: k = AsmKernel::YMarch; break;
        case TPFA_KERNEL_NAIVE: k = AsmKernel::Naive; break;
        default: return fail(TPFA_ERR_INVALID_ARG, "bad kernel variant %d", (int)kern);
    }
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (h->prec == TPFA_MIXED)
        e = launch_jvp_mixed(k, h->geom, h->qf, h->crk, fields_of<float>(h), w_dev, Jw_dev, R_dev, h->status,
                             march_rows(h), h->W, st);
    else
        e = launch_jvp_fp64(h->geom, h->qd, h->crk, fields_of<double>(h), w_dev, Jw_dev, R_dev, h->status, st);
    if (e != cudaSuccess) return cuda_fail(e, "jvp launch");
    return TPFA_OK;
}

int tpfa_jvp(tpfa_handle h, const double* w_dev, double* Jw_dev, double* R_dev, void* stream) {
    return tpfa_jvp_kernel(h, TPFA_KERNEL_AUTO, w_dev, Jw_dev, R_dev, stream);
}

int tpfa_linear_solve(tpfa_handle h, const double* b_dev, double* x_dev, const tpfa_krylov_opts* opts,
                      tpfa_krylov_stats* stats, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!b_dev || !x_dev) return fail(TPFA_ERR_INVALID_ARG, "b and x must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    if (h->slab) return fail(TPFA_ERR_INVALID_ARG, "this call is not available on a slab handle (assembly only)");
    DeviceGuard dg(h->device);
    rc = krylov_workspace(h);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = launch(h, auto_kernel(h), nullptr, h->kv_vals, h->prec == TPFA_MIXED ? h->kv_diag : nullptr, st);
    if (rc) return rc;
    return krylov_solve(h, b_dev, 1.0, x_dev, opts, stats, st);
}

int tpfa_newton_step(tpfa_handle h, void* p_dev, const tpfa_krylov_opts* opts, tpfa_krylov_stats* stats,
                     double* R_dev, double* delta_dev, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!p_dev) return fail(TPFA_ERR_INVALID_ARG, "p must be non-NULL");
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    if (h->slab) return fail(TPFA_ERR_INVALID_ARG, "this call is not available on a slab handle (assembly only)");
    DeviceGuard dg(h->device);
    rc = krylov_workspace(h);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    h->p = p_dev;
    double* R = R_dev ? R_dev : h->kv_R;
    double* x = delta_dev ? delta_dev : h->kv_vec[0];
    rc = launch(h, auto_kernel(h), R, h->kv_vals, h->prec == TPFA_MIXED ? h->kv_diag : nullptr, st);
    if (rc) return rc;
    rc = krylov_solve(h, R, -1.0, x, opts, stats, st);
    if (rc) return rc;
    cudaError_t e = krylov_add_delta(h->N, h->prec == TPFA_MIXED, p_dev, x, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "Newton update");
    return TPFA_OK;
}

int tpfa_get_pattern(tpfa_handle h, const long long** row_ptr_dev, const int** col_idx_dev, long long* nnz,
                     void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard dg(h->device);
    if (!h->row_ptr) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        void *rp = nullptr, *ci = nullptr;
        if (dev_alloc(&rp, sizeof(long long) * (size_t)(h->N + 1)) != cudaSuccess ||
            dev_alloc(&ci, sizeof(int) * (size_t)h->nnz) != cudaSuccess) {
            cudaGetLastError();
            dev_free(rp);
            dev_free(ci);
            return fail(TPFA_ERR_OOM, "device allocation failed for the pattern (nnz %lld)", h->nnz);
        }
        cudaError_t e = launch_pattern(h->geom, (long long*)rp, (int*)ci, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            dev_free(rp);
            dev_free(ci);
            return cuda_fail(e, "pattern build");
        }
        h->row_ptr = (long long*)rp;
        h->col_idx = (int*)ci;
    }
    if (row_ptr_dev) *row_ptr_dev = h->row_ptr;
    if (col_idx_dev) *col_idx_dev = h->col_idx;
    if (nnz) *nnz = h->nnz;
    return TPFA_OK;
}

long long tpfa_nnz(int nx, int ny, int nz, int connectivity) {
    if (nx < 1 || ny < 1 || nz < 1 || (connectivity != 6 && connectivity != 10))
        return fail(TPFA_ERR_INVALID_ARG, "bad grid size or connectivity");
    return total_nnz(GridGeom{nx, ny, nz, connectivity == 10 ? 1 : 0});
}

int tpfa_copy_pattern(tpfa_handle h, long long* row_ptr_out_dev, int* col_idx_out_dev, void* stream) {
    int rc = tpfa_get_pattern(h, nullptr, nullptr, nullptr, stream);
    if (rc) return rc;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (row_ptr_out_dev)
        e = cudaMemcpyAsync(row_ptr_out_dev, h->row_ptr, sizeof(long long) * (size_t)(h->N + 1),
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && col_idx_out_dev)
        e = cudaMemcpyAsync(col_idx_out_dev, h->col_idx, sizeof(int) * (size_t)h->nnz, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "pattern copy");
    return TPFA_OK;
}

int tpfa_grid_info(tpfa_handle h, int* nx, int* ny, int* nz, int* connectivity, long long* nnz, int* precision) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (nx) *nx = h->nx;
    if (ny) *ny = h->ny;
    if (nz) *nz = h->nz;
    if (connectivity) *connectivity = h->prm.connectivity;
    if (nnz) *nnz = h->nnz;
    if (precision) *precision = (int)h->prec;
    return TPFA_OK;
}

int tpfa_get_transmissibility(tpfa_handle h, int which, void* out_dev, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (which < 0 || which > 4 || !out_dev) return fail(TPFA_ERR_INVALID_ARG, "bad transmissibility index or NULL output");
    if (which >= 3 && !h->geom.diag) return fail(TPFA_ERR_INVALID_ARG, "diagonal links need 10-point connectivity");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemcpyAsync(out_dev, h->T[which], h->real_size * (size_t)h->N, cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "transmissibility copy");
    return TPFA_OK;
}

int tpfa_slab_bounds(int nz, int parts, int part, int* k0, int* k1, int* e0, int* e1) {
    if (nz < 1 || parts < 1 || part < 0 || part >= parts || parts > nz)
        return fail(TPFA_ERR_INVALID_ARG, "slab bounds: need 1 <= parts <= nz and 0 <= part < parts (nz %d, parts %d, "
                    "part %d)", nz, parts, part);
    // balanced: the first nz % parts slabs hold one plane more
    const int base = nz / parts, extra = nz % parts;
    const int a = part * base + (part < extra ? part : extra);
    const int b = a + base + (part < extra ? 1 : 0);
    if (k0) *k0 = a;
    if (k1) *k1 = b;
    if (e0) *e0 = a > 0 ? a - 1 : 0;
    if (e1) *e1 = b < nz ? b + 1 : nz;
    return TPFA_OK;
}

int tpfa_create_slab(tpfa_handle* out, int nx, int ny, int nz, int k0, int k1, const tpfa_params* prm,
                     tpfa_precision prec, const double* perm_dev, const double* poro_dev, const double* depth_dev,
                     void* stream) {
    g_err.clear();
    if (!out) return fail(TPFA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nz < 1 || k0 < 0 || k1 > nz || k0 >= k1)
        return fail(TPFA_ERR_INVALID_ARG, "slab planes [%d, %d) are not a non-empty range of [0, %d)", k0, k1, nz);
    const int e0 = k0 > 0 ? k0 - 1 : 0, e1 = k1 < nz ? k1 + 1 : nz;
    tpfa_handle h = nullptr;
    int rc = tpfa_create_grid(&h, nx, ny, e1 - e0, prm, prec, perm_dev, poro_dev, depth_dev, stream);
    if (rc) return rc;
    h->slab = true;
    h->own0 = k0 - e0;
    h->own1 = k1 - e0;
    h->slab_k0 = k0;
    h->slab_k1 = k1;
    h->slab_nz = nz;
    *out = h;
    return TPFA_OK;
}

int tpfa_slab_info(tpfa_handle h, int* k0, int* k1, int* own0, int* own1, long long* row0, long long* row1,
                   long long* entry0, long long* entry1) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->slab) return fail(TPFA_ERR_INVALID_ARG, "not a slab handle");
    const long long nxy = (long long)h->nx * h->ny;
    if (k0) *k0 = h->slab_k0;
    if (k1) *k1 = h->slab_k1;
    if (own0) *own0 = h->own0;
    if (own1) *own1 = h->own1;
    if (row0) *row0 = nxy * h->own0;
    if (row1) *row1 = nxy * h->own1;
    if (entry0) *entry0 = row_start(h->geom, 0, 0, h->own0);
    if (entry1) *entry1 = h->own1 == h->nz ? h->nnz : row_start(h->geom, 0, 0, h->own1);
    return TPFA_OK;
}

int tpfa_slab_exchange(tpfa_handle lower, void* p_lower_dev, tpfa_handle upper, void* p_upper_dev, void* stream) {
    int rc = check_handle(lower);
    if (rc) return rc;
    rc = check_handle(upper);
    if (rc) return rc;
    if (!lower->slab || !upper->slab || lower->slab_k1 != upper->slab_k0 || lower->slab_nz != upper->slab_nz ||
        lower->nx != upper->nx || lower->ny != upper->ny || lower->prec != upper->prec)
        return fail(TPFA_ERR_INVALID_ARG, "slab exchange: the handles are not adjacent slabs of one grid");
    if (!p_lower_dev || !p_upper_dev) return fail(TPFA_ERR_INVALID_ARG, "slab exchange: NULL pressure array");
    const size_t plane = lower->real_size * (size_t)lower->nx * (size_t)lower->ny;
    char* pl = static_cast<char*>(p_lower_dev);
    char* pu = static_cast<char*>(p_upper_dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceGuard dg(upper->device);
    // the lower slab's last owned plane -> the upper slab's bottom halo (its plane 0);
    // the upper slab's first owned plane -> the lower slab's top halo (its last plane)
    cudaError_t e = cudaMemcpyPeerAsync(pu, upper->device, pl + plane * (size_t)(lower->own1 - 1), lower->device,
                                        plane, st);
    if (e == cudaSuccess)
        e = cudaMemcpyPeerAsync(pl + plane * (size_t)lower->own1, lower->device, pu + plane * (size_t)upper->own0,
                                upper->device, plane, st);
    if (e != cudaSuccess) return cuda_fail(e, "slab exchange");
    return TPFA_OK;
}

int tpfa_sync_status(tpfa_handle h, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int s = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&s, h->status, sizeof s, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s) e = cudaMemset(h->status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (s & STATUS_TIMEOUT) return fail(TPFA_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (s & STATUS_DEVICE_CHECK) return fail(TPFA_ERR_DEVICE_CHECK, "a device-side bounds check failed");
    if (s & STATUS_NONFINITE) return fail(TPFA_ERR_NONFINITE, "a residual or Jacobian value was NaN or Inf");
    return TPFA_OK;
}

int tpfa_destroy(tpfa_handle h) {
    if (!h) return TPFA_OK;
    {
        DeviceGuard dg(h->device);
        cudaDeviceSynchronize();
        h->release();
    }
    delete h;
    return TPFA_OK;
}

int tpfa_create_mesh(tpfa_mesh* out, long long n_cells, long long n_conn, const tpfa_params* prm,
                     tpfa_precision prec, const int* conn_i_dev, const int* conn_j_dev, const double* trans_dev,
                     const double* volume_dev, const double* poro_dev, const double* depth_dev, void* stream) {
    g_err.clear();
    if (!out) return fail(TPFA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_cells < 1) return fail(TPFA_ERR_INVALID_ARG, "a mesh needs at least one cell");
    if (n_cells >= (1LL << 31)) return fail(TPFA_ERR_TOO_LARGE, "%lld cells exceed 2^31 - 1", n_cells);
    if (n_conn < 0) return fail(TPFA_ERR_INVALID_ARG, "negative connection count");
    if (!prm) return fail(TPFA_ERR_INVALID_ARG, "params is NULL");
    if (!(prm->mu > 0.0) || !(prm->dt > 0.0)) return fail(TPFA_ERR_INVALID_ARG, "mu and dt must be > 0");
    if (prec != TPFA_FP64 && prec != TPFA_MIXED) return fail(TPFA_ERR_INVALID_ARG, "bad precision %d", (int)prec);
    if (!volume_dev || !poro_dev || !depth_dev || (n_conn > 0 && (!conn_i_dev || !conn_j_dev || !trans_dev)))
        return fail(TPFA_ERR_INVALID_ARG, "mesh arrays must be non-NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // the connection list comes to the host once for the pattern build
    std::vector<int> ci(n_conn), cj(n_conn);
    std::vector<double> T(n_conn);
    if (n_conn > 0) {
        e = cudaMemcpyAsync(ci.data(), conn_i_dev, sizeof(int) * n_conn, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cj.data(), conn_j_dev, sizeof(int) * n_conn, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T.data(), trans_dev, sizeof(double) * n_conn, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "connection list download");
    }
    std::vector<long long> row_ptr;
    std::vector<int> col;
    std::vector<double> Tc;
    int rc = build_mesh_pattern(n_cells, n_conn, ci, cj, T, row_ptr, col, Tc);
    if (rc) return rc;

    tpfa_mesh_s* m = new tpfa_mesh_s();
    m->device = dev;
    m->N = n_cells;
    m->nc = n_conn;
    m->nnz = row_ptr[n_cells];
    m->prec = prec;
    m->crk = prm->c_r != 0.0;
    m->real_size = prec == TPFA_MIXED ? sizeof(float) : sizeof(double);
    // the cell volume is folded into m^n and into (V/dt) phi0, so V_dt = 1
    m->qd = PhysD{prm->rho_ref, prm->p_ref, prm->c_f, 1.0 / prm->mu, prm->g, 0.5 * prm->g, 1.0, prm->c_r};
    m->qf = PhysF{(float)prm->rho_ref, (float)prm->p_ref, (float)prm->c_f, (float)(1.0 / prm->mu), (float)prm->g,
                  (float)(0.5 * prm->g), 1.0f, (float)prm->c_r};
    m->sp = SetupPhys{1.0, 1.0, 1.0, prm->rho_ref, prm->p_ref, prm->c_f, prm->c_r, 1.0};
    const size_t rb = m->real_size * (size_t)n_cells;
    double* Tc_d = nullptr;
    bool ok = dev_alloc((void**)&m->row_ptr, sizeof(long long) * (size_t)(n_cells + 1)) == cudaSuccess;
    ok = ok && dev_alloc((void**)&m->col_idx, sizeof(int) * (size_t)m->nnz) == cudaSuccess;
    ok = ok && dev_alloc(&m->Tc, m->real_size * (size_t)m->nnz) == cudaSuccess;
    ok = ok && dev_alloc((void**)&Tc_d, sizeof(double) * (size_t)m->nnz) == cudaSuccess;
    ok = ok && dev_alloc(&m->z, rb) == cudaSuccess;
    ok = ok && dev_alloc((void**)&m->vphi_d, sizeof(double) * (size_t)n_cells) == cudaSuccess;
    if (ok && m->crk) ok = dev_alloc(&m->vphi_r, rb) == cudaSuccess;
    ok = ok && dev_alloc((void**)&m->mn, sizeof(double) * (size_t)n_cells) == cudaSuccess;
    ok = ok && dev_alloc((void**)&m->status, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dev_free(Tc_d);
        m->release();
        delete m;
        return fail(TPFA_ERR_OOM, "device allocation failed for a mesh of %lld cells", n_cells);
    }
    e = cudaMemcpyAsync(m->row_ptr, row_ptr.data(), sizeof(long long) * (n_cells + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->col_idx, col.data(), sizeof(int) * m->nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Tc_d, Tc.data(), sizeof(double) * m->nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        if (prec == TPFA_MIXED) {
            e = launch_convert_f32(Tc_d, (float*)m->Tc, m->nnz, st);
            if (e == cudaSuccess) e = launch_convert_f32(depth_dev, (float*)m->z, n_cells, st);
        } else {
            e = launch_copy_f64(Tc_d, (double*)m->Tc, m->nnz, st);
            if (e == cudaSuccess) e = launch_copy_f64(depth_dev, (double*)m->z, n_cells, st);
        }
    }
    if (e == cudaSuccess)
        e = launch_mesh_vphi(n_cells, prm->dt, prec == TPFA_MIXED, volume_dev, poro_dev, m->vphi_d, m->vphi_r, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(Tc_d);
    if (e != cudaSuccess) {
        m->release();
        delete m;
        return cuda_fail(e, "mesh setup");
    }
    *out = m;
    return TPFA_OK;
}

int tpfa_mesh_set_state(tpfa_mesh m, const void* p_dev, const void* p_prev_dev, void* stream) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    if (!p_dev || !p_prev_dev) return fail(TPFA_ERR_INVALID_ARG, "p and p_prev must be non-NULL");
    DeviceGuard dg(m->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = m->prec == TPFA_MIXED
                        ? launch_prev_mass_f32(m->sp, (const float*)p_prev_dev, m->vphi_d, m->mn, m->N, st)
                        : launch_prev_mass_f64(m->sp, (const double*)p_prev_dev, m->vphi_d, m->mn, m->N, st);
    if (e != cudaSuccess) return cuda_fail(e, "previous-step mass");
    m->p = p_dev;
    m->pn = p_prev_dev;
    m->has_state = true;
    return TPFA_OK;
}

int tpfa_mesh_set_pressure(tpfa_mesh m, const void* p_dev) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    if (!p_dev) return fail(TPFA_ERR_INVALID_ARG, "p must be non-NULL");
    if (!m->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_mesh_set_state has not been called");
    m->p = p_dev;
    return TPFA_OK;
}

int tpfa_mesh_assemble(tpfa_mesh m, double* R_dev, void* vals_dev, double* diag64_dev, void* stream) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    if (!R_dev && !vals_dev) return fail(TPFA_ERR_INVALID_ARG, "nothing to assemble (R and vals NULL)");
    if (m->prec == TPFA_FP64 && diag64_dev) return fail(TPFA_ERR_INVALID_ARG, "diag64 must be NULL on the FP64 path");
    if (!m->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_mesh_set_state has not been called");
    DeviceGuard dg(m->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (m->prec == TPFA_MIXED) {
        AsmOut<float> o{R_dev, static_cast<float*>(vals_dev), diag64_dev, m->status};
        e = launch_mesh_mixed(mesh_fields<float>(m), m->N, m->qf, m->crk, o, st);
    } else {
        AsmOut<double> o{R_dev, static_cast<double*>(vals_dev), nullptr, m->status};
        e = launch_mesh_fp64(mesh_fields<double>(m), m->N, m->qd, m->crk, o, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mesh assembly launch");
    return TPFA_OK;
}

int tpfa_mesh_copy_pattern(tpfa_mesh m, long long* row_ptr_out_dev, int* col_idx_out_dev, void* stream) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (row_ptr_out_dev)
        e = cudaMemcpyAsync(row_ptr_out_dev, m->row_ptr, sizeof(long long) * (size_t)(m->N + 1),
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && col_idx_out_dev)
        e = cudaMemcpyAsync(col_idx_out_dev, m->col_idx, sizeof(int) * (size_t)m->nnz, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "pattern copy");
    return TPFA_OK;
}

int tpfa_mesh_info(tpfa_mesh m, long long* n_cells, long long* n_conn, long long* nnz, int* precision) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    if (n_cells) *n_cells = m->N;
    if (n_conn) *n_conn = m->nc;
    if (nnz) *nnz = m->nnz;
    if (precision) *precision = (int)m->prec;
    return TPFA_OK;
}

int tpfa_mesh_sync_status(tpfa_mesh m, void* stream) {
    if (!m) return fail(TPFA_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int s = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&s, m->status, sizeof s, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s) e = cudaMemset(m->status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (s & STATUS_DEVICE_CHECK) return fail(TPFA_ERR_DEVICE_CHECK, "a device-side bounds check failed");
    if (s & STATUS_NONFINITE) return fail(TPFA_ERR_NONFINITE, "a residual or Jacobian value was NaN or Inf");
    return TPFA_OK;
}

int tpfa_destroy_mesh(tpfa_mesh m) {
    if (!m) return TPFA_OK;
    {
        DeviceGuard dg(m->device);
        cudaDeviceSynchronize();
        m->release();
    }
    delete m;
    return TPFA_OK;
}

}  // extern "C"

// ===================================================================== tiling, autotuning, ensembles

#include <stdint.h>

#include <map>
#include <vector>

#include "tpfa_batch.h"

namespace {

// Autotune cache: a text file of "key JY W" lines (a header line starts with '#').
std::map<std::string, std::pair<int, int>> cache_read(const char* path) {
    std::map<std::string, std::pair<int, int>> m;
    if (!path) return m;
    FILE* fp = fopen(path, "r");
    if (!fp) return m;
    char key[256];
    int jy, w;
    char line[512];
    while (fgets(line, sizeof line, fp)) {
        if (line[0] == '#') continue;
        if (sscanf(line, "%255s %d %d", key, &jy, &w) == 3 && jy >= 1 && jy <= 64 && (w == 4 || w == 8))
            m[key] = {jy, w};
    }
    fclose(fp);
    return m;
}

bool cache_write(const char* path, const std::map<std::string, std::pair<int, int>>& m) {
    if (!path) return true;
    std::string tmp = std::string(path) + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "w");
    if (!fp) return false;
    fprintf(fp, "# tpfa autotune cache v1: key rows_per_march warps_per_block\n");
    for (const auto& kv : m) fprintf(fp, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
    fclose(fp);
    return rename(tmp.c_str(), path) == 0;
}

std::string device_tag(int dev) {
    int maj = 0, mnr = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    char b[32];
    snprintf(b, sizeof b, "sm%d%d", maj, mnr);
    return b;
}

int log2_bucket(long long n) {
    int b = 0;
    while ((1LL << (b + 1)) <= n) ++b;
    return b;
}

const int kTuneJY[] = {8, 16, 24, 32, 40, 48, 64};
const int kTuneW[] = {4, 8};

}  // namespace

struct tpfa_ensemble_s {
    int device = 0;
    int M = 0;
    std::vector<tpfa_handle> grids;
    bool diag = false, crk = false;
    std::vector<double*> R;
    std::vector<float*> vals;
    std::vector<double*> diag64;
    BatchModel* d_models = nullptr;
    BatchModel* h_stage = nullptr;  // pinned upload buffer
    std::vector<BatchModel> last;   // the table last uploaded
    cudaEvent_t upload_done = nullptr;
    unsigned long long* ticket = nullptr;
    long long total = 0;
    int JY = 32, W = 4;
    int blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // parameters the graph's kernel node was built with
    int g_JY = 0, g_W = 0, g_blocks = 0;
    long long g_total = -1;

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (upload_done) cudaEventDestroy(upload_done);
        dev_free(d_models);
        dev_free(ticket);
        if (h_stage) cudaFreeHost(h_stage);
        exec = nullptr, graph = nullptr, upload_done = nullptr, d_models = nullptr, ticket = nullptr, h_stage = nullptr;
    }
};

namespace {

int build_table(tpfa_ensemble e, std::vector<BatchModel>& tab) {
    tab.resize(e->M);
    long long first = 0;
    // tiles are numbered (and claimed) largest model first, so the launch
    // ends on the small models' tiles
    std::vector<int> order(e->M);
    for (int m = 0; m < e->M; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e->grids[a]->N > e->grids[b]->N; });
    for (int t = 0; t < e->M; ++t) {
        const int m = order[t];
        tpfa_grid* h = e->grids[m];
        if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "ensemble model %d has no state (tpfa_set_state)", m);
        if (!e->vals[m]) return fail(TPFA_ERR_INVALID_ARG, "ensemble model %d has no outputs (tpfa_ensemble_set_outputs)", m);
        BatchModel bm;
        memset(&bm, 0, sizeof bm);
        bm.g = h->geom;
        bm.q = h->qf;
        bm.f = fields_of<float>(h);
        bm.o = AsmOut<float>{e->R[m], e->vals[m], e->diag64[m], h->status};
        bm.tx = (h->nx + 31) / 32;
        bm.ty = (h->ny + e->JY - 1) / e->JY;
        bm.tz = (h->nz + e->W - 1) / e->W;
        bm.crk = h->crk ? 1 : 0;
        bm.first = first;
        first += (long long)bm.tx * bm.ty * bm.tz;
        tab[t] = bm;
    }
    e->total = first;
    return TPFA_OK;
}

int ensure_graph(tpfa_ensemble e) {
    int bps = 0;
    cudaError_t ce = batch_blocks_per_sm(e->diag, e->crk, e->W, &bps);
    if (ce != cudaSuccess) return cuda_fail(ce, "ensemble kernel occupancy");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
    e->blocks = (int)std::min<long long>((long long)sms * (bps > 0 ? bps : 1), e->total > 0 ? e->total : 1);
    if (e->exec && e->g_JY == e->JY && e->g_W == e->W && e->g_total == e->total && e->g_blocks == e->blocks)
        return TPFA_OK;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    const void* func = nullptr;
    int smem = 0;
    ce = batch_kernel(e->diag, e->crk, e->W, &func, &smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "ensemble kernel");
    ce = cudaGraphCreate(&e->graph, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphCreate");
    // node 1: reset the tile ticket; node 2: the persistent kernel
    cudaMemsetParams mp;
    memset(&mp, 0, sizeof mp);
    mp.dst = e->ticket;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    cudaGraphNode_t n_reset, n_kernel;
    ce = cudaGraphAddMemsetNode(&n_reset, e->graph, nullptr, 0, &mp);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph memset node");
    const BatchModel* models = e->d_models;
    int M = e->M;
    long long total = e->total;
    int JY = e->JY;
    unsigned long long* ticket = e->ticket;
    void* args[] = {&models, &M, &total, &JY, &ticket};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = const_cast<void*>(func);
    kp.gridDim = dim3(e->blocks, 1, 1);
    kp.blockDim = dim3(32, e->W, 1);
    kp.sharedMemBytes = smem;
    kp.kernelParams = args;
    ce = cudaGraphAddKernelNode(&n_kernel, e->graph, &n_reset, 1, &kp);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph kernel node");
    ce = cudaGraphInstantiate(&e->exec, e->graph, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    e->g_JY = e->JY, e->g_W = e->W, e->g_total = e->total, e->g_blocks = e->blocks;
    return TPFA_OK;
}

}  // namespace

extern "C" {

int tpfa_set_tiling(tpfa_handle h, int rows_per_march, int warps_per_block) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (rows_per_march < 1 || rows_per_march > 64 || (warps_per_block != 4 && warps_per_block != 8))
        return fail(TPFA_ERR_INVALID_ARG, "rows_per_march must be in [1, 64] and warps_per_block 4 or 8");
    h->JY = rows_per_march;
    h->W = warps_per_block;
    return TPFA_OK;
}

int tpfa_get_tiling(tpfa_handle h, int* rows_per_march, int* warps_per_block) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (rows_per_march) *rows_per_march = h->JY;
    if (warps_per_block) *warps_per_block = h->W;
    return TPFA_OK;
}

int tpfa_autotune(tpfa_handle h, const char* cache_path, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->has_state) return fail(TPFA_ERR_NO_STATE, "tpfa_set_state has not been called");
    DeviceGuard dg(h->device);
    char key[256];
    snprintf(key, sizeof key, "grid/%s/%s/c%d/r%d/n%d", device_tag(h->device).c_str(),
             h->prec == TPFA_MIXED ? "mixed" : "fp64", h->prm.connectivity, h->crk ? 1 : 0, log2_bucket(h->N));
    auto cache = cache_read(cache_path);
    auto it = cache.find(key);
    if (it != cache.end()) {
        h->JY = it->second.first;
        h->W = it->second.second;
        return TPFA_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *R = nullptr, *vals = nullptr, *diag = nullptr;
    cudaError_t e = cudaMallocAsync(&R, sizeof(double) * (size_t)h->N, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&vals, h->real_size * (size_t)h->nnz, st);
    if (e == cudaSuccess && h->prec == TPFA_MIXED) e = cudaMallocAsync(&diag, sizeof(double) * (size_t)h->N, st);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    int bj = h->JY, bw = h->W;
    for (int jy : kTuneJY) {
        for (int w : kTuneW) {
            if (e != cudaSuccess) break;
            h->JY = jy;
            h->W = w;
            for (int r = 0; r < 2 && !rc; ++r) rc = launch(h, auto_kernel(h), (double*)R, vals, (double*)diag, st);
            if (rc) break;
            cudaEventRecord(a, st);
            for (int r = 0; r < 5 && !rc; ++r) rc = launch(h, auto_kernel(h), (double*)R, vals, (double*)diag, st);
            cudaEventRecord(b, st);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && ms < best) best = ms, bj = jy, bw = w;
        }
        if (rc) break;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (R) cudaFreeAsync(R, st);
    if (vals) cudaFreeAsync(vals, st);
    if (diag) cudaFreeAsync(diag, st);
    cudaStreamSynchronize(st);
    h->JY = bj;
    h->W = bw;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    cache[key] = {bj, bw};
    if (!cache_write(cache_path, cache)) return fail(TPFA_ERR_INVALID_ARG, "cannot write autotune cache %s", cache_path);
    return TPFA_OK;
}

int tpfa_create_ensemble(tpfa_ensemble* out, int M, const tpfa_handle* grids) {
    if (!out) return fail(TPFA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (M < 1 || !grids) return fail(TPFA_ERR_INVALID_ARG, "an ensemble needs M >= 1 grids");
    for (int m = 0; m < M; ++m) {
        if (!grids[m]) return fail(TPFA_ERR_INVALID_ARG, "grid %d is NULL", m);
        if (grids[m]->prec != TPFA_MIXED) return fail(TPFA_ERR_INVALID_ARG, "ensembles use the mixed path (grid %d is FP64)", m);
        if (grids[m]->geom.diag != grids[0]->geom.diag || grids[m]->crk != grids[0]->crk)
            return fail(TPFA_ERR_INVALID_ARG, "grid %d differs from grid 0 in connectivity or in c_r == 0", m);
        if (grids[m]->device != grids[0]->device) return fail(TPFA_ERR_INVALID_ARG, "grid %d is on another device", m);
        if (grids[m]->slab) return fail(TPFA_ERR_INVALID_ARG, "grid %d is a slab handle", m);
    }
    tpfa_ensemble e = new tpfa_ensemble_s();
    e->device = grids[0]->device;
    e->M = M;
    e->grids.assign(grids, grids + M);
    e->diag = grids[0]->geom.diag != 0;
    e->crk = grids[0]->crk;
    e->R.assign(M, nullptr);
    e->vals.assign(M, nullptr);
    e->diag64.assign(M, nullptr);
    DeviceGuard dg(e->device);
    void* dm = nullptr;
    void* tk = nullptr;
    cudaError_t ce = dev_alloc(&dm, sizeof(BatchModel) * (size_t)M);
    if (ce == cudaSuccess) ce = dev_alloc(&tk, sizeof(unsigned long long));
    e->d_models = (BatchModel*)dm;
    e->ticket = (unsigned long long*)tk;
    if (ce == cudaSuccess && !alloc_fault_injected()) ce = cudaMallocHost((void**)&e->h_stage, sizeof(BatchModel) * (size_t)M);
    else if (ce == cudaSuccess) ce = cudaErrorMemoryAllocation;
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->upload_done, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        e->release();
        delete e;
        return fail(TPFA_ERR_OOM, "ensemble allocation failed");
    }
    *out = e;
    return TPFA_OK;
}

int tpfa_ensemble_set_outputs(tpfa_ensemble e, int m, double* R_dev, void* vals_dev, double* diag64_dev) {
    if (!e) return fail(TPFA_ERR_INVALID_ARG, "ensemble is NULL");
    if (m < 0 || m >= e->M) return fail(TPFA_ERR_INVALID_ARG, "model index %d out of range", m);
    if (!vals_dev) return fail(TPFA_ERR_INVALID_ARG, "vals must be non-NULL");
    e->R[m] = R_dev;
    e->vals[m] = static_cast<float*>(vals_dev);
    e->diag64[m] = diag64_dev;
    return TPFA_OK;
}

int tpfa_assemble_batch(tpfa_ensemble e, void* stream) {
    if (!e) return fail(TPFA_ERR_INVALID_ARG, "ensemble is NULL");
    DeviceGuard dg(e->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<BatchModel> tab;
    int rc = build_table(e, tab);
    if (rc) return rc;
    if (e->last.size() != tab.size() || memcmp(e->last.data(), tab.data(), sizeof(BatchModel) * tab.size()) != 0) {
        cudaError_t ce = cudaEventSynchronize(e->upload_done);  // the staging buffer is free again
        if (ce == cudaSuccess) {
            memcpy(e->h_stage, tab.data(), sizeof(BatchModel) * tab.size());
            ce = cudaMemcpyAsync(e->d_models, e->h_stage, sizeof(BatchModel) * tab.size(), cudaMemcpyHostToDevice, st);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e->upload_done, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ensemble table upload");
        e->last = tab;
    }
    rc = ensure_graph(e);
    if (rc) return rc;
    cudaError_t ce = cudaGraphLaunch(e->exec, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphLaunch");
    return TPFA_OK;
}

int tpfa_ensemble_tiling(tpfa_ensemble e, int* rows_per_march, int* warps_per_block, long long* tiles, int* blocks) {
    if (!e) return fail(TPFA_ERR_INVALID_ARG, "ensemble is NULL");
    if (rows_per_march) *rows_per_march = e->JY;
    if (warps_per_block) *warps_per_block = e->W;
    if (tiles) *tiles = e->total;
    if (blocks) *blocks = e->blocks;
    return TPFA_OK;
}

int tpfa_ensemble_autotune(tpfa_ensemble e, const char* cache_path, void* stream) {
    if (!e) return fail(TPFA_ERR_INVALID_ARG, "ensemble is NULL");
    DeviceGuard dg(e->device);
    long long cells = 0;
    for (auto h : e->grids) cells += h->N;
    char key[256];
    snprintf(key, sizeof key, "ensemble/%s/M%d/c%d/r%d/n%d", device_tag(e->device).c_str(), e->M,
             e->diag ? 10 : 6, e->crk ? 1 : 0, log2_bucket(cells));
    auto cache = cache_read(cache_path);
    auto it = cache.find(key);
    if (it != cache.end()) {
        e->JY = it->second.first;
        e->W = it->second.second;
        return TPFA_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&b);
    float best = 1e30f;
    int bj = e->JY, bw = e->W, rc = TPFA_OK;
    for (int jy : kTuneJY) {
        for (int w : kTuneW) {
            if (ce != cudaSuccess || rc) break;
            e->JY = jy;
            e->W = w;
            rc = tpfa_assemble_batch(e, stream);
            if (rc) break;
            cudaEventRecord(a, st);
            for (int r = 0; r < 3 && !rc; ++r) rc = tpfa_assemble_batch(e, stream);
            cudaEventRecord(b, st);
            ce = cudaEventSynchronize(b);
            float ms = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
            if (ce == cudaSuccess && ms < best) best = ms, bj = jy, bw = w;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    e->JY = bj;
    e->W = bw;
    if (rc) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "ensemble autotune");
    cache[key] = {bj, bw};
    if (!cache_write(cache_path, cache)) return fail(TPFA_ERR_INVALID_ARG, "cannot write autotune cache %s", cache_path);
    return TPFA_OK;
}

int tpfa_destroy_ensemble(tpfa_ensemble e) {
    if (!e) return TPFA_OK;
    {
        DeviceGuard dg(e->device);
        cudaDeviceSynchronize();
        e->release();
    }
    delete e;
    return TPFA_OK;
}

}  // extern "C"
