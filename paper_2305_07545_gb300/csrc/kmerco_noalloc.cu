// Classification over caller-owned device buffers that allocates nothing.
//
// Some callers cannot call cudaMalloc: a process whose device memory is all
// reserved up front by its own pool allocator (a serving stack, a framework
// that owns the GPU), a plug-in living inside such a host, or a latency-bound
// path that must not pay for cudaMalloc/cudaFree, which can synchronise the
// whole device.  kmerco_classify_noalloc() serves them: the caller passes the
// countBF, the keys and every output buffer, and the only scratch the split
// needs -- one trusted-key count per 4096-key tile -- lives in the fixed
// device array below.  Every GPU that loads this library holds that array
// (512 KiB + 8 bytes) until the process exits.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/kmerco.h"
#include "kmerco_internal.cuh"

namespace countbf {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr uint64_t kTile = (uint64_t)kThreads * kPerThread;   // keys per split tile
constexpr uint64_t kMaxTiles = KMERCO_NOALLOC_MAX_KEYS / kTile;
static_assert(kMaxTiles * kTile == KMERCO_NOALLOC_MAX_KEYS, "whole tiles");

// Tile counts, then (after the scan) tile prefixes; the last slot holds the
// number of trusted keys.  Each call overwrites the slots it uses before
// reading them, so nothing has to start at zero.
static __device__ __align__(256) unsigned long long g_split_scratch[kMaxTiles + 1];


__global__ void __launch_bounds__(kThreads) count_kernel(const uint32_t *est, uint64_t n,
                                                         uint32_t tau, unsigned long long *scratch) {
    const uint64_t base = blockIdx.x * kTile + threadIdx.x * (uint64_t)kPerThread;
    unsigned long long c = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) c += (base + j < n) && est[base + j] > tau;
    unsigned long long tot;
    block_exclusive_scan<unsigned long long, kThreads>(c, tot);
    if (threadIdx.x == 0) scratch[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) scan_kernel(unsigned long long *scratch,
                                                        uint64_t ntiles) {
    unsigned long long carry = 0;
    for (uint64_t s0 = 0; s0 < ntiles; s0 += kThreads) {
        const uint64_t i = s0 + threadIdx.x;
        unsigned long long v = i < ntiles ? scratch[i] : 0ull, tot;
        const unsigned long long pre = block_exclusive_scan<unsigned long long, kThreads>(v, tot) + carry;
        if (i < ntiles) scratch[i] = pre;
        carry += tot;
    }
    if (threadIdx.x == 0) scratch[kMaxTiles] = carry;
}

template <int KW>
__global__ void __launch_bounds__(kThreads) scatter_kernel(const uint64_t *keys, const uint32_t *est,
                                                           uint64_t n, uint32_t tau,
                                                           const unsigned long long *scratch,
                                                           uint64_t *out) {
    const uint64_t tile0 = blockIdx.x * kTile;
    const uint64_t base = tile0 + threadIdx.x * (uint64_t)kPerThread;
    unsigned flags = 0;
    unsigned long long c = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const bool t = (base + j < n) && est[base + j] > tau;
        flags |= (unsigned)t << j;
        c += t;
    }
    unsigned long long tot;
    const unsigned long long pre = block_exclusive_scan<unsigned long long, kThreads>(c, tot);
    const uint64_t T = scratch[kMaxTiles];
    const uint64_t tile_trusted = scratch[blockIdx.x];
    uint64_t tpos = tile_trusted + pre;
    uint64_t epos = T + (tile0 - tile_trusted) + ((base < n ? base - tile0 : 0) - pre);
    for (int j = 0; j < kPerThread; ++j) {
        const uint64_t i = base + j;
        if (i >= n) break;
        const uint64_t o = (flags >> j) & 1u ? tpos++ : epos++;
#pragma unroll
        for (int w = 0; w < KW; ++w) out[o * KW + w] = keys[i * KW + w];
    }
}

// Device address of g_split_scratch on the current device.  In host code
// the array's name only stands for the device object; the runtime has to
// translate it, which is done once per device and CUDA context: the address
// is cached with the identity of the context it was taken in, so that after
// cudaDeviceReset (a new context on the same device) it is looked up again
// instead of reusing an address of the destroyed context.
std::mutex g_mutex;
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long *ptr;
    unsigned long long ctx;   // cuCtxGetId of the context it was taken in; 0 unknown
};
ScratchAddr g_scratch[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **ctx);                       // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);     // cuCtxGetId
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// Unique id of the calling thread's current CUDA context, 0 when there is
// none or the driver does not tell (the caller then looks the address up
// again).  The driver functions are reached through the runtime's entry
// point query, so the library needs no link to the driver library.
unsigned long long current_context_id() {
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_id = (CtxGetIdFn)f;
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

int scratch_on_current_device(unsigned long long **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return KMERCO_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    ScratchAddr &a = g_scratch[dev];
    if (!a.ptr || ctx == 0 || a.ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_split_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return KMERCO_ECUDA;
        }
        a.ptr = (unsigned long long *)p;
        a.ctx = current_context_id();   // the lookup made the device's context current
    }
    *out = a.ptr;
    return KMERCO_OK;
}

}  // namespace
}  // namespace countbf

using namespace countbf;

extern "C" int kmerco_classify_noalloc(const uint64_t *cells, uint64_t m, int k, int counter_bits,
                                       int nhash, uint32_t threshold, const uint64_t *keys,
                                       uint64_t n, uint32_t *est, uint64_t *out,
                                       uint64_t *n_trusted, void *stream) {
    if (!n_trusted) return KMERCO_EINVAL;
    if (k < 1 || k > 64 || counter_bits < 1 || counter_bits > 32 || nhash < 1 || nhash > 32)
        return KMERCO_EINVAL;
    const uint64_t eta = 64 / (uint64_t)counter_bits;
    const uint64_t maxc = (1ull << counter_bits) - 1;
    if (m < 1 || m % eta != 0 || (uint64_t)threshold >= maxc) return KMERCO_EINVAL;
    if (n > KMERCO_NOALLOC_MAX_KEYS) return KMERCO_EINVAL;
    if (n == 0) {
        *n_trusted = 0;
        return KMERCO_OK;
    }
    if (!cells || !keys || !est || !out) return KMERCO_EINVAL;
    unsigned long long *scratch = nullptr;
    int status = scratch_on_current_device(&scratch);
    if (status != KMERCO_OK) return status;

    Geometry G = make_geometry(m / eta, 0, 0, counter_bits, nhash);
    G.cells = const_cast<uint64_t *>(cells);
    const int kw = k <= 32 ? 1 : 2;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t ntiles = (n + kTile - 1) / kTile;

    cudaError_t e = launch_query(keys, n, kw, k, G, est, s);
    if (e == cudaSuccess) {
        count_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(est, n, threshold, scratch);
        scan_kernel<<<1, kThreads, 0, s>>>(scratch, ntiles);
        if (kw == 1)
            scatter_kernel<1><<<(unsigned)ntiles, kThreads, 0, s>>>(keys, est, n, threshold, scratch, out);
        else
            scatter_kernel<2><<<(unsigned)ntiles, kThreads, 0, s>>>(keys, est, n, threshold, scratch, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n_trusted, scratch + kMaxTiles, sizeof(uint64_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KMERCO_ECUDA;
    }
    return KMERCO_OK;
}
