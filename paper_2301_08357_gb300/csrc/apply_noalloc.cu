// ps_pressure_apply_noalloc: the operator apply y = A x without any device
// allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// apply the operator -- for example a host framework whose caching allocator
// has already reserved the device memory it is allowed to use (a fresh
// cudaMalloc would fail or push it over its budget), or a solver loop that
// must not let an allocation implicitly synchronise the device between time
// steps.  ps_pressure_apply allocates its workspace (permuted copies of x and
// y, partial sums of shared nodes) on first use; this variant instead carves
// that scratch out of one file-scope __device__ array, which every GPU that
// loads the library holds until the process exits.
//
// The array's host-side name is only a stand-in; the device address is looked
// up once per device with cudaGetSymbolAddress (that device current) when a
// context is created on it (ps_ctx_create calls noalloc_setup): the lookup
// loads this file's module, which commits the array's device memory then and
// not inside a later apply.  The cached address assumes the device's primary
// context lives until the process exits (no cudaDeviceReset in between).
// Every call shares the array and it keeps the last call's contents; nothing
// in it needs to start at zero because a call that completes writes every
// entry it later reads.  (If a bounded device wait gives up, the kernel
// leaves its chunk unwritten: y is then undefined, and the context's error
// flag reports PS_ETIMEOUT at its next synchronising call.)  Calls whose work
// overlaps on the GPU (different streams, or different meshes at the same
// time) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/pressure.h"
#include "internal.h"

using namespace ps;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the scratch array on `device` (which must be current).
int scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            ps_set_last_error(e == cudaSuccess ? "no device address for the allocation-free scratch"
                                               : cudaGetErrorString(e));
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? PS_ENOMEM : PS_ECUDA;
        }
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return PS_OK;
}

}  // namespace

// Called by ps_ctx_create with `device` current: looks the scratch array up
// (loading this module and committing its memory) once per device.
int ps::noalloc_setup(int device) {
    void *p = nullptr;
    return scratch_address(device, &p);
}

extern "C" int ps_pressure_apply_noalloc(ps_mesh *m, const void *x, void *y, int prec, void *stream) {
    if (!m || !x || !y || (prec != PS_F32 && prec != PS_F64) || x == y) return PS_EINVAL;
    if (!m->coeff_ok) return PS_ESTATE;
    const size_t esz = prec == PS_F32 ? 4 : 8;
    const int64_t np = m->dev.n_pad;
    const int64_t sh = m->prep.sh_total > 0 ? m->prep.sh_total : 1;
    const size_t need = 2 * align256((size_t)np * esz) + align256((size_t)sh * esz);
    if (need > kScratchBytes) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "mesh too large for ps_pressure_apply_noalloc: needs %zu bytes of scratch, limit %zu",
                 need, kScratchBytes);
        ps_set_last_error(msg);
        return PS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(m->ctx->mu);
    cudaError_t e = cudaSetDevice(m->ctx->device);
    if (e != cudaSuccess) {
        ps_set_last_error(cudaGetErrorString(e));
        return PS_ECUDA;
    }
    void *base = nullptr;
    int rc = scratch_address(m->ctx->device, &base);
    if (rc != PS_OK) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    void *xi = b;
    void *yi = b + align256((size_t)np * esz);
    void *part = b + 2 * align256((size_t)np * esz);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = m->dev.n_nodes, nu = m->prep.n_nodes;   // unknowns, caller's vertices
    const int g = grid_for(n, m->ctx->sms), gu = grid_for(nu, m->ctx->sms);
    if (prec == PS_F32) {
        k_perm_in<float, float><<<g, kChunkThreads, 0, s>>>(n, (const float *)x, (float *)xi, m->d_old_of_new, m->dev.dirichlet);
        VecArgs<float> a;
        std::memset(&a, 0, sizeof(a));
        a.x = (const float *)xi;
        a.y = (float *)yi;
        a.partial = (float *)part;
        rc = launch_pass<float, kApply>(m, a, s);
        if (rc != PS_OK) return rc;
        k_perm_out<float, float><<<gu, kChunkThreads, 0, s>>>(nu, (const float *)yi, (float *)y, m->d_new_of_old);
    } else {
        k_perm_in<double, double><<<g, kChunkThreads, 0, s>>>(n, (const double *)x, (double *)xi, m->d_old_of_new,
                                                    m->dev.dirichlet);
        VecArgs<double> a;
        std::memset(&a, 0, sizeof(a));
        a.x = (const double *)xi;
        a.y = (double *)yi;
        a.partial = (double *)part;
        rc = launch_pass<double, kApply>(m, a, s);
        if (rc != PS_OK) return rc;
        k_perm_out<double, double><<<gu, kChunkThreads, 0, s>>>(nu, (const double *)yi, (double *)y, m->d_new_of_old);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ps_set_last_error(cudaGetErrorString(e));
        return PS_ECUDA;
    }
    return PS_OK;
}
