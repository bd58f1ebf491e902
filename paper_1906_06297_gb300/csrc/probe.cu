// probe.cu -- throughput probes for the integer ceiling of the sweep.  Not
// steps of the method: they measure what bounds it.  The sweep draws its
// random numbers inside the kernel (Sec. 3.3 of the paper: no pre-filled
// random array), so its rate is set by Philox4x32-10, whose rounds are
// 32 x 32 -> 64-bit multiplies and three-input XORs.
//
//   mulwide_probe_kernel  the wide multiply alone: independent chains of
//                         dependent mad.wide.u32, no memory traffic, a full
//                         grid; its rate is the machine's wide-multiply peak.
//   rng_probe_kernel      Philox alone, shaped like the sweep: each thread
//                         step makes 8 blocks that share counter words 1..3
//                         (as a lane's 8 blocks in one row of the sweep do),
//                         with 32-bit indices and a full grid, and counts the
//                         draws below a threshold with the sweep's predicated
//                         adds.  Its rate is the sweep's ceiling with the
//                         lattice traffic and the neighbour sums taken away.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace ising {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kMulChains = 16;
constexpr int kMulUnroll = 4;

// FORM 0 (the form of a Philox round): d = x * M, M an immediate, no addend;
//        the chain continues with x = hi(d) ^ lo(d) (one XOR on the logic
//        pipe per multiply, as a round has).
// FORM 1: a = hi(a) * m + a, a 64-bit multiply-add with a register addend.
// In both, every multiply depends on the previous one of its chain and both
// halves of every product reach the next step.
template <int FORM>
__global__ void __launch_bounds__(kProbeThreads) mulwide_probe_kernel(uint32_t iters, uint32_t m,
                                                                      unsigned long long *sink)
{
    const uint32_t tid = blockIdx.x * kProbeThreads + threadIdx.x;
    uint64_t a[kMulChains];
    uint32_t x[kMulChains];
#pragma unroll
    for (int c = 0; c < kMulChains; ++c) {
        a[c] = ((uint64_t)tid << 8) | (uint64_t)(2 * c + 1);
        x[c] = (tid << 5) ^ (uint32_t)(2 * c + 1);
    }
#pragma unroll kMulUnroll
    for (uint32_t k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kMulChains; ++c) {
            if (FORM == 0) {
                asm("{\n\t"
                    ".reg .u32 lo, hi;\n\t"
                    ".reg .u64 d;\n\t"
                    "mul.wide.u32 d, %0, 0xD2511F53;\n\t"
                    "mov.b64 {lo, hi}, d;\n\t"
                    "xor.b32 %0, lo, hi;\n\t"
                    "}"
                    : "+r"(x[c]));
            } else {
                asm("{\n\t"
                    ".reg .u32 lo, hi;\n\t"
                    "mov.b64 {lo, hi}, %0;\n\t"
                    "mad.wide.u32 %0, hi, %1, %0;\n\t"
                    "}"
                    : "+l"(a[c])
                    : "r"(m));
            }
        }
    }
    uint64_t y = 0;
#pragma unroll
    for (int c = 0; c < kMulChains; ++c) y ^= FORM == 0 ? (uint64_t)x[c] * 0x100000001ull : a[c];
    // depends on both halves of every chain (FORM 1) or on every chain
    // (FORM 0), so none of them is dead; the store is rare
    if (FORM == 0 ? (uint32_t)y == 0x5bd1e995u : (uint32_t)y == (uint32_t)(y >> 32)) atomicAdd(sink, 1ull);
}

// Counts a draw below T3 with one compare and one predicated add into a
// counter, the form each of the sweep's two threshold marks takes.
__device__ __forceinline__ void count_below(uint32_t &cnt, uint32_t u, uint32_t T3)
{
    asm("{\n\t"
        ".reg .pred p;\n\t"
        "setp.lt.u32 p, %1, %2;\n\t"
        "@p add.u32 %0, %0, 1;\n\t"
        "}"
        : "+r"(cnt)
        : "r"(u), "r"(T3));
}

__global__ void __launch_bounds__(kProbeThreads) rng_probe_kernel(uint32_t n_groups, uint32_t tail,
                                                                  const __grid_constant__ RoundKeys rk,
                                                                  uint32_t c2, uint32_t c3, uint32_t T3,
                                                                  unsigned long long *count)
{
    // group g holds blocks 8g .. 8g+7 (q = 8g + b: counter words 0 and 1 are
    // the low and high halves of q); the last group holds `tail` blocks when
    // tail != 0
    uint32_t cnt = 0;
    const uint32_t step = gridDim.x * kProbeThreads;
    const uint32_t full = tail ? n_groups - 1 : n_groups;
    for (uint32_t g = blockIdx.x * kProbeThreads + threadIdx.x; g < full; g += step) {
        const uint32_t c0 = g << 3, c1 = g >> 29;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint4 u = philox(c0 | (uint32_t)b, c1, c2, c3, rk);
            count_below(cnt, u.x, T3);
            count_below(cnt, u.y, T3);
            count_below(cnt, u.z, T3);
            count_below(cnt, u.w, T3);
        }
    }
    if (tail && blockIdx.x == 0 && threadIdx.x < tail) {
        const uint32_t g = n_groups - 1;
        const uint4 u = philox((g << 3) | threadIdx.x, g >> 29, c2, c3, rk);
        count_below(cnt, u.x, T3);
        count_below(cnt, u.y, T3);
        count_below(cnt, u.z, T3);
        count_below(cnt, u.w, T3);
    }
    long long total = cnt, zero = 0;
    __shared__ long long buf[2];
    if (threadIdx.x == 0) buf[0] = buf[1] = 0;
    __syncthreads();
    block_reduce_add2<kProbeThreads>(total, zero, buf);
    __syncthreads();
    if (threadIdx.x == 0 && buf[0] != 0) atomicAdd(count, (unsigned long long)buf[0]);
}

struct ProbeOccupancy {
    std::mutex mu;
    int mul[128] = {}, rng[64] = {};
};
ProbeOccupancy g_probe_occ;

// Resident blocks of `kernel` per SM on the current device (cached).
template <typename K>
int blocks_per_sm(K kernel, int *cache)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(g_probe_occ.mu);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kProbeThreads, 0) != cudaSuccess || n < 1) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

}  // namespace

cudaError_t mulwide_probe(int form, uint32_t iters, unsigned long long *sink, uint64_t *multiplies, cudaStream_t s)
{
    DeviceInfo info;
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return e;
    const int per_sm = form == 0 ? blocks_per_sm(mulwide_probe_kernel<0>, g_probe_occ.mul)
                                 : blocks_per_sm(mulwide_probe_kernel<1>, g_probe_occ.mul + 64);
    const unsigned blocks = (unsigned)info.sm_count * (unsigned)per_sm;
    *multiplies = (uint64_t)blocks * kProbeThreads * (uint64_t)iters * kMulChains;
    if (form == 0) mulwide_probe_kernel<0><<<blocks, kProbeThreads, 0, s>>>(iters, 0xD2511F53u, sink);
    else mulwide_probe_kernel<1><<<blocks, kProbeThreads, 0, s>>>(iters, 0x9E3779B9u, sink);
    return cudaGetLastError();
}

cudaError_t rng_probe(uint64_t n_blocks, const RoundKeys &rk, uint32_t c2, uint32_t c3, uint32_t T3,
                      unsigned long long *count, cudaStream_t s)
{
    DeviceInfo info;
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return e;
    const uint32_t n_groups = (uint32_t)((n_blocks + 7) >> 3), tail = (uint32_t)(n_blocks & 7);
    const int per_sm = blocks_per_sm(rng_probe_kernel, g_probe_occ.rng);
    const int64_t want = ((int64_t)n_groups + kProbeThreads - 1) / kProbeThreads;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)info.sm_count * per_sm));
    rng_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(n_groups, tail, rk, c2, c3, T3, count);
    return cudaGetLastError();
}

}  // namespace ising
