// common.cuh -- device helpers shared by the libising kernels: the keyed
// Philox4x32-10 block function and the launch parameter blocks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11, Sec. 3.3).  One round: the 64-bit products of counter
// words 0 and 2 with two fixed multipliers are split into halves and mixed as
//   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)).
// The round keys are precomputed on the host (key + r * Weyl constant) and
// arrive in the kernel parameter block, so every launch reads them from the
// constant bank instead of re-deriving them per block.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct RoundKeys {
    uint32_t k[20];  // k[2r], k[2r+1]: key words of round r
};

inline RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const RoundKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k[2 * r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k[2 * r + 1];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Counter word 3: colour in bit 0, purpose in bits 1-2, sweep index bits
// 32.. in bits 8..31.
__host__ __device__ __forceinline__ uint32_t counter_word3(int colour, int purpose, uint64_t t)
{
    return (uint32_t)colour | ((uint32_t)purpose << 1) | ((uint32_t)(t >> 32) << 8);
}

enum Purpose { kPurposeMetropolis = 0, kPurposeInit = 1, kPurposeExchange = 2, kPurposeLearned = 3 };

// ---------------------------------------------------------------------------
// Acceptance, in the form the kernels consume.  For beta >= 0, T[0..2] = 2^32
// (always flip); T3 / T4 are the 32-bit thresholds for a = 3 / a = 4, and
// `always` stands in for a threshold of 2^32 (beta = 0, where T3 = T4 = 2^32).
// ---------------------------------------------------------------------------
struct Accept {
    uint32_t T3, T4;  // 32-bit thresholds (meaningful when below 2^32)
    uint32_t always;  // 1 when T3 = T4 = 2^32 (beta = 0): every spin flips
    uint32_t zero;    // 0 (a value the compiler cannot see)
    uint64_t T3_64, T4_64;
};

// ---------------------------------------------------------------------------
// Launch parameter blocks (passed by value: they live in the constant bank).
// ---------------------------------------------------------------------------
// The planes hold `rows` target rows (local rows 0 .. rows-1, global rows
// row0 .. row0+rows-1 of the L x L lattice).  Source rows are addressed by
// local index too: for the whole periodic lattice (rows = L, row0 = 0) the
// row above row 0 is row L-1 and the row below row L-1 is row 0; for a slab
// with halo rows, local rows -1 and `rows` are the halos and nothing wraps.
// wrap_row / wrap_to say where the downward walk over source rows jumps back
// (L -> 0 for the periodic lattice; rows+1 -> -1 for a slab, a row that is
// fetched but never used), first_up is the source row above local row 0.
struct Msc4SweepParams {
    uint64_t *tgt;        // target plane, local row 0
    const uint64_t *src;  // source plane (other colour), local row 0
    int64_t L;            // side of the whole lattice
    int64_t rows;         // target rows in this plane
    int64_t row0;         // global row of local row 0
    int64_t wrap_row, wrap_to, first_up;
    int64_t wpr;          // words per row = L / 32
    int64_t stride;       // row stride in words
    int64_t qrow;         // Philox blocks per plane row = L / 8
    int64_t total;        // work units: (64-word chunk column) x (row)
    uint32_t c2, c3;      // counter words 2 and 3 of this half-sweep
    Accept acc;
    RoundKeys rk;
    long long *obs;       // {sum s, sum bonds} accumulators or nullptr
    int32_t spare_sms = 0;  // host side: SMs the launch leaves without a block
};

struct Int8SweepParams {
    int8_t *tgt;
    const int8_t *src;
    int64_t L;
    int64_t half;    // L / 2 spins per plane row
    int64_t stride;  // bytes
    int64_t nblk;    // Philox blocks per plane = ceil(L * half / 4)
    uint32_t c2, c3;
    Accept acc;
    RoundKeys rk;
    long long *obs;
};

constexpr uint32_t kNibbleLsb = 0x11111111u;

// The 16 spins of an MSC4 word as 16 bits (bit k = the low bit of nibble k,
// 1 for an up spin) and back: the bit-packed format holds a plane row's spins
// in the same order at one bit each.
__device__ __forceinline__ uint32_t msc4_word_to_bits(uint64_t w)
{
    uint64_t v = w & 0x1111111111111111ull;
    v = (v | (v >> 3)) & 0x0303030303030303ull;
    v = (v | (v >> 6)) & 0x000F000F000F000Full;
    v = (v | (v >> 12)) & 0x000000FF000000FFull;
    return (uint32_t)((v | (v >> 24)) & 0xFFFFull);
}

__device__ __forceinline__ uint64_t bits_to_msc4_word(uint32_t x)
{
    uint64_t v = x & 0xFFFFull;
    v = (v | (v << 24)) & 0x000000FF000000FFull;
    v = (v | (v << 12)) & 0x000F000F000F000Full;
    v = (v | (v << 6)) & 0x0303030303030303ull;
    return (v | (v << 3)) & 0x1111111111111111ull;
}

// ---------------------------------------------------------------------------
// Block-wide reduction of two int64 partial sums and one atomic per block.
// ---------------------------------------------------------------------------
template <int kThreads>
__device__ __forceinline__ void block_reduce_add2(long long a, long long b, long long *out)
{
    constexpr int kWarps = kThreads / 32;
    __shared__ long long sa[kWarps], sb[kWarps];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < kWarps ? sa[lane] : 0;
        b = lane < kWarps ? sb[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(out), (unsigned long long)a);
            atomicAdd(reinterpret_cast<unsigned long long *>(out + 1), (unsigned long long)b);
        }
    }
}

}  // namespace ising
