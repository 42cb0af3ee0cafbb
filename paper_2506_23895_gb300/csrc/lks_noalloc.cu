// lks_step_noalloc: one LKS step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they want a step: code that runs while
// a CUDA stream is being captured into a graph, code inside a host framework that owns all device
// memory through its own pool, or a real-time loop that must not block on the driver's
// allocator.  For them this file runs the plain per-node step (f^eq into scratch planes, then the
// gather, Brinkman update and boundary writes) with the scratch planes in one file-scope
// device array instead of a workspace.  The caller passes only its inputs and outputs.
//
// The array is created when the library is loaded on a device and stays until the process exits.
// Host code cannot use its name as a device address (on the host the symbol is only a stand-in),
// so a call looks up its address with cudaGetSymbolAddress while that device is current.  A call
// made while cfg->stream is being captured does not look it up (it reuses the address the last
// uncaptured call on that device found), so make the first call on each device before any stream
// capture begins; every uncaptured call looks it up again, so a device reset or a re-created
// primary context (after which the module may load elsewhere) is picked up by the next
// uncaptured call.
// All calls share the one array: calls whose kernels overlap on the GPU (two streams, or two
// host threads) race on it and must be serialised by the caller.  Every call overwrites all of
// the scratch it reads, so nothing has to be cleared between calls.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lks.h"
#include "lks_internal.h"

using namespace lks;

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB: Q f^eq planes of one step
static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

void put_err(char* err, size_t len, const char* msg) {
    if (err && len > 0) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
}

// Fill the kernels' geometry from the configuration; the footprint box is the whole grid when
// kappa/u_S are given per node, empty otherwise.
Geom geom_from(const lks_config* cfg, bool with_body) {
    Geom g;
    std::memset(&g, 0, sizeof(g));
    g.dim = cfg->dim;
    g.n[0] = cfg->nx;
    g.n[1] = cfg->ny;
    g.n[2] = cfg->dim == 3 ? cfg->nz : 1;
    for (int a = 0; a < 3; ++a) g.periodic[a] = (a >= cfg->dim) || cfg->bc[2 * a] == LKS_BC_PERIODIC;
    g.nodes = (long long)g.n[0] * g.n[1] * g.n[2];
    for (int f = 0; f < 6; ++f) {
        g.bc[f] = cfg->bc[f];
        for (int k = 0; k < 4; ++k) g.bcv[f][k] = cfg->bc_val[f][k];
    }
    g.rho0 = cfg->rho0;
    g.A = cfg->A;
    for (int a = 0; a < 3; ++a) g.body[a] = cfg->body_force[a];
    if (with_body) {
        for (int a = 0; a < 3; ++a) {
            g.blo[a] = 0;
            g.bn[a] = g.n[a];
        }
        g.boxN = g.nodes;
    }
    return g;
}

}  // namespace

extern "C" lks_status lks_step_noalloc(const lks_config* cfg, const void* state_in,
                                       void* state_out, const void* kappa_us, char* err,
                                       size_t err_len) {
    put_err(err, err_len, "");
    if (!cfg || !state_in || !state_out) {
        put_err(err, err_len, "lks_step_noalloc: null configuration or state pointer");
        return LKS_ERR_ARG;
    }
    {
        // an error left pending by earlier work on this thread is reported as such, not as a
        // failure of this call's launches
        const cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess) {
            char msg[256];
            std::snprintf(msg, sizeof(msg),
                          "lks_step_noalloc: a CUDA error was pending before this call: %s",
                          cudaGetErrorString(pending));
            put_err(err, err_len, msg);
            return LKS_ERR_CUDA;
        }
    }
    if (lks_workspace_bytes(cfg) == 0) {
        put_err(err, err_len, "lks_step_noalloc: invalid configuration");
        return LKS_ERR_ARG;
    }
    const size_t tsz = cfg->precision == LKS_FP64 ? 8 : 4;
    {
        // the kernels move one node record (4 values) per vector access
        const uintptr_t rec = 4 * tsz;
        if ((uintptr_t)state_in % rec || (uintptr_t)state_out % rec ||
            (uintptr_t)kappa_us % rec) {
            char msg[160];
            std::snprintf(msg, sizeof(msg),
                          "lks_step_noalloc: state_in, state_out and kappa_us must be aligned "
                          "to one node record (%zu bytes)",
                          (size_t)rec);
            put_err(err, err_len, msg);
            return LKS_ERR_ARG;
        }
    }
    const int Q = cfg->dim == 3 ? 15 : 9;
    const long long nodes = (long long)cfg->nx * cfg->ny * (cfg->dim == 3 ? cfg->nz : 1);
    const size_t need = (size_t)nodes * Q * tsz;
    if (need > kScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "lks_step_noalloc: grid needs %zu bytes of scratch, limit is %zu "
                      "(%lld nodes x %d directions x %zu bytes)",
                      need, kScratchBytes, nodes, Q, tsz);
        put_err(err, err_len, msg);
        return LKS_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        put_err(err, err_len, "lks_step_noalloc: no usable current device");
        return LKS_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cfg->stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        put_err(err, err_len, "lks_step_noalloc: cfg->stream is not a usable stream");
        return LKS_ERR_ARG;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                put_err(err, err_len, "lks_step_noalloc: cudaGetSymbolAddress failed");
                return LKS_ERR_CUDA;
            }
            g_scratch_ptr[dev] = p;
        } else if (!g_scratch_ptr[dev]) {
            put_err(err, err_len,
                    "lks_step_noalloc: the first call on a device must come before stream "
                    "capture");
            return LKS_ERR_ORDER;
        }
        scratch = g_scratch_ptr[dev];
    }
    const Geom g = geom_from(cfg, kappa_us != nullptr);
    if (cfg->precision == LKS_FP64) {
        launch_feq<double>(g, (const V4<double>*)state_in, (double*)scratch, st);
        launch_gather<double>(g, (const double*)scratch, (const V4<double>*)kappa_us,
                              (V4<double>*)state_out, st);
    } else {
        launch_feq<float>(g, (const V4<float>*)state_in, (float*)scratch, st);
        launch_gather<float>(g, (const float*)scratch, (const V4<float>*)kappa_us,
                             (V4<float>*)state_out, st);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_err(err, err_len, cudaGetErrorString(e));
        return LKS_ERR_CUDA;
    }
    return LKS_OK;
}
