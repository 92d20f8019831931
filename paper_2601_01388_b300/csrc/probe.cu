// Random-access read probe: the bandwidth of independent random 32-byte sector
// reads over a caller-provided device buffer (chosen far larger than L2), the
// memory pattern that bounds the sampler's gathers and searches.
#include "agis_internal.h"

namespace agis {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    // splitmix64 finaliser (Steele, Lea & Flood, OOPSLA'14)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Every thread reads `per_thread` 8-byte words, each at the start of a random
// 32-byte sector among the first sector_mask + 1 (a power of two); the xor of the
// words goes to sink so the loads stay.
__global__ void k_random_read(const uint64_t *buf, uint64_t sector_mask, uint64_t per_thread, uint64_t seed,
                              unsigned long long *sink)
{
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t acc = 0;
    uint64_t h = mix64(seed ^ (tid * 0xD1B54A32D192ED03ull));
    constexpr int kInFlight = 8;
    for (uint64_t k = 0; k < per_thread; k += kInFlight) {
        uint64_t v[kInFlight];
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) {
            h = mix64(h);
            v[j] = __ldcg(buf + (h & sector_mask) * 4);
        }
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) acc ^= v[j];
    }
    if (acc == 0x123456789abcdefull) atomicAdd(sink, 1ull);
}

}  // namespace
}  // namespace agis

extern "C" int agis_probe_random_read(const void *buf, uint64_t bytes, uint64_t reads, uint64_t seed,
                                      void *cuda_stream, void *sink)
{
    using namespace agis;
    if (!buf || !sink || bytes < 4096 || reads == 0) return AGIS_ERR_ARG;
    int device = 0, sms = 0;
    AGIS_CUDA_TRY(cudaGetDevice(&device));
    AGIS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const uint64_t threads = (uint64_t)sms * 2048;
    uint64_t per = (reads + threads - 1) / threads;
    per = (per + 7) / 8 * 8;
    uint64_t sectors = 1;
    while (sectors * 2 <= bytes / 32) sectors *= 2;
    count_launch();
    k_random_read<<<(unsigned)(threads / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        (const uint64_t *)buf, sectors - 1, per, seed, (unsigned long long *)sink);
    return cuda_status(cudaGetLastError());
}
