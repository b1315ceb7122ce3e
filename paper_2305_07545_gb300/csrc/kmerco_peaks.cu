// Random-access rate microbenchmarks (include/kmerco_peaks.h): the
// ceilings of the countBF update (random 64-bit read + compare-and-swap)
// and of the query (random 8-byte reads) on this device.
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/kmerco.h"
#include "../../include/kmerco_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;   // independent operations in flight per thread

// SplitMix64's output function: a bijective 64-bit mix of a counter.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void fill_kernel(uint64_t *buf, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        buf[i] = mix64(i) & 0x0F0F0F0F0F0F0F0Full;
}

// rounds x kPerThread operations per thread: all loads of a round first,
// then all compare-and-swaps (the atomic update design issues its first
// attempts the same way).
__global__ void __launch_bounds__(kThreads) cas_kernel(uint64_t *buf, uint64_t mask,
                                                       uint32_t rounds, uint64_t seed) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint32_t r = 0; r < rounds; ++r) {
        uint64_t idx[kPerThread], cur[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            idx[j] = mix64(seed ^ (t * (uint64_t)(rounds * kPerThread) + r * kPerThread + j)) & mask;
            cur[j] = __ldcg(buf + idx[j]);
        }
#pragma unroll
        for (int j = 0; j < kPerThread; ++j)
            atomicCAS((unsigned long long *)(buf + idx[j]), (unsigned long long)cur[j],
                      (unsigned long long)(cur[j] + 1));
    }
}

__global__ void __launch_bounds__(kThreads) read_kernel(const uint64_t *buf, uint64_t mask,
                                                        uint32_t rounds, uint64_t seed,
                                                        uint64_t *sink) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t acc = 0;
    for (uint32_t r = 0; r < rounds; ++r) {
        uint64_t v[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const uint64_t idx =
                mix64(seed ^ (t * (uint64_t)(rounds * kPerThread) + r * kPerThread + j)) & mask;
            v[j] = __ldcg(buf + idx);
        }
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) acc += v[j];
    }
    if (acc == 0x5A5A5A5A5A5A5A5Aull) sink[0] = acc;   // keeps the loads; practically never true
}

struct DeviceScope {
    int prev = -1, want = -1;
    explicit DeviceScope(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        want = d < 0 ? prev : d;
        if (want >= 0 && want != prev) cudaSetDevice(want);
    }
    ~DeviceScope() {
        if (prev >= 0 && want != prev) cudaSetDevice(prev);
    }
};

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return KMERCO_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KMERCO_ENOMEM : KMERCO_ECUDA;
}

// Shared driver: buffer, fill, one warm-up and one timed launch of the
// chosen kernel.  cas != 0 selects the read-modify-write kernel.
int measure(uint64_t bytes, uint64_t ops, int device, int cas, double *rate) {
    if (!rate || ops == 0 || bytes < 4096 || (bytes & (bytes - 1))) return KMERCO_EINVAL;
    DeviceScope scope(device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, scope.want < 0 ? 0 : scope.want) !=
            cudaSuccess || sms <= 0)
        return KMERCO_ECUDA;
    const uint64_t words = bytes / 8;
    const uint64_t threads = (uint64_t)sms * 8 * kThreads;   // 8 blocks of 256 per SM
    uint64_t rounds = (ops + threads * kPerThread - 1) / (threads * kPerThread);
    if (rounds < 1) rounds = 1;
    if (rounds > (1u << 20)) return KMERCO_EINVAL;
    uint64_t *buf = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = KMERCO_OK;
    do {
        if ((st = status_of(cudaMalloc(&buf, bytes)))) break;
        if ((st = status_of(cudaMalloc(&sink, 8)))) break;
        if ((st = status_of(cudaEventCreate(&e0)))) break;
        if ((st = status_of(cudaEventCreate(&e1)))) break;
        fill_kernel<<<sms * 4, kThreads>>>(buf, words);
        const unsigned grid = (unsigned)(threads / kThreads);
        for (int rep = 0; rep < 2; ++rep) {   // warm-up, then timed
            if (rep == 1 && (st = status_of(cudaEventRecord(e0)))) break;
            if (cas)
                cas_kernel<<<grid, kThreads>>>(buf, words - 1, (uint32_t)rounds, 0x1234ull + rep);
            else
                read_kernel<<<grid, kThreads>>>(buf, words - 1, (uint32_t)rounds, 0x1234ull + rep, sink);
            if ((st = status_of(cudaGetLastError()))) break;
        }
        if (st) break;
        if ((st = status_of(cudaEventRecord(e1)))) break;
        if ((st = status_of(cudaEventSynchronize(e1)))) break;
        float ms = 0.f;
        if ((st = status_of(cudaEventElapsedTime(&ms, e0, e1)))) break;
        *rate = (double)(threads * kPerThread * rounds) / (ms / 1000.0);
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return st;
}

}  // namespace

extern "C" {

int kmerco_peak_random_cas(uint64_t bytes, uint64_t ops, int device, double *rate) {
    return measure(bytes, ops, device, 1, rate);
}

int kmerco_peak_random_read(uint64_t bytes, uint64_t ops, int device, double *rate) {
    return measure(bytes, ops, device, 0, rate);
}

}  // extern "C"
