// bits.cu -- conversions between MSC4 colour planes and the bit-packed I/O
// format of the host-resident sweep (one bit per spin in the order of the
// MSC4 nibbles, L/16 bytes per plane row).  Not part of the paper's method:
// MSC4 (Sec. 3.3) spends four bits per spin on the bit-parallel neighbour
// sums; storage and host transfers need one.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "common.cuh"
#include "launch.h"

namespace ising {

// ---------------------------------------------------------------------------
// MSC4 plane rows <-> the bit-packed format (one bit per spin, L/16 bytes per
// row, dense rows): a thread converts V pairs of words (32 spins each) <-> V
// uint32, V = 4 on rows of 4 pairs or more, else 1.  One launch converts up
// to kMaxConvJobs row ranges (bands of different planes); blockIdx.x covers
// (row of the concatenated ranges, chunk of the row).  MSC4 -> bits: a
// thread's pairs are adjacent (one 16-byte store of bits, where the row
// length and the buffers' alignment allow it); bits -> MSC4: a thread's pairs
// are 256 apart, so that each warp store is part of 512 contiguous bytes.
// ---------------------------------------------------------------------------
struct ConvParams {
    const void *src[kMaxConvJobs];
    void *dst[kMaxConvJobs];
    unsigned row_end[kMaxConvJobs];  // cumulative rows of the ranges
    int n;
};

__device__ __forceinline__ int conv_job(const ConvParams &c, unsigned g, unsigned &r)
{
    int j = 0;
    while (j + 1 < c.n && g >= c.row_end[j]) ++j;
    r = g - (j ? c.row_end[j - 1] : 0u);
    return j;
}

template <int V>
__global__ void __launch_bounds__(256) msc4_to_bits_kernel(const __grid_constant__ ConvParams c, int64_t stride_words,
                                                           int64_t pairs, unsigned chunks)
{
    const unsigned g = blockIdx.x / chunks;
    const int64_t p = ((int64_t)(blockIdx.x - g * chunks) * 256 + threadIdx.x) * V;
    if (p >= pairs) return;
    unsigned r;
    const int j = conv_job(c, g, r);
    const ulonglong2 *src =
        reinterpret_cast<const ulonglong2 *>((const uint64_t *)c.src[j] + (int64_t)r * stride_words + 2 * p);
    uint32_t out[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const ulonglong2 w = src[v];
        out[v] = msc4_word_to_bits(w.x) | (msc4_word_to_bits(w.y) << 16);
    }
    uint32_t *dst = (uint32_t *)c.dst[j] + (int64_t)r * pairs + p;
    if constexpr (V == 4)
        *reinterpret_cast<uint4 *>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
    else
        dst[0] = out[0];
}

template <int V>
__global__ void __launch_bounds__(256) bits_to_msc4_kernel(const __grid_constant__ ConvParams c, int64_t stride_words,
                                                           int64_t pairs, unsigned chunks)
{
    const unsigned g = blockIdx.x / chunks;
    const int64_t p0 = (int64_t)(blockIdx.x - g * chunks) * 256 * V + threadIdx.x;
    unsigned r;
    const int j = conv_job(c, g, r);
    const uint32_t *src = (const uint32_t *)c.src[j] + (int64_t)r * pairs;
    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>((uint64_t *)c.dst[j] + (int64_t)r * stride_words);
    uint32_t b[V];
#pragma unroll
    for (int v = 0; v < V; ++v) b[v] = p0 + 256 * v < pairs ? src[p0 + 256 * v] : 0u;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (p0 + 256 * v < pairs)
            dst[p0 + 256 * v] = make_ulonglong2(bits_to_msc4_word(b[v] & 0xFFFFu), bits_to_msc4_word(b[v] >> 16));
}

namespace {

// collects the jobs' ranges; false if there are too many rows for the grid
bool conv_params(const ConvJob *jobs, int n, ConvParams &c, int64_t &rows)
{
    c = ConvParams{};
    rows = 0;
    for (int j = 0; j < n; ++j) {
        c.src[j] = jobs[j].src;
        c.dst[j] = jobs[j].dst;
        rows += jobs[j].rows;
        c.row_end[j] = (unsigned)rows;
    }
    c.n = n;
    return rows < (int64_t(1) << 31);
}

}  // namespace

cudaError_t msc4_to_bits_multi(const ConvJob *jobs, int n, int64_t stride_words, int64_t L, cudaStream_t s)
{
    if (n <= 0 || n > kMaxConvJobs) return n == 0 ? cudaSuccess : cudaErrorInvalidValue;
    ConvParams c;
    int64_t rows = 0;
    if (!conv_params(jobs, n, c, rows)) return cudaErrorInvalidConfiguration;
    if (rows == 0) return cudaSuccess;
    const int64_t pairs = L / 64;
    // MSC4 -> bits with V = 4 needs a multiple of 4 pairs per row and 16-byte aligned bit rows
    bool wide = pairs % 4 == 0;
    for (int j = 0; j < n; ++j) wide = wide && (uintptr_t)jobs[j].dst % 16 == 0;
    const int V = wide ? 4 : 1;
    const unsigned chunks = (unsigned)((pairs / V + 255) / 256);
    if (rows * (int64_t)chunks > INT32_MAX) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)(rows * chunks);
    if (V == 4)
        msc4_to_bits_kernel<4><<<grid, 256, 0, s>>>(c, stride_words, pairs, chunks);
    else
        msc4_to_bits_kernel<1><<<grid, 256, 0, s>>>(c, stride_words, pairs, chunks);
    return cudaGetLastError();
}

cudaError_t bits_to_msc4_multi(const ConvJob *jobs, int n, int64_t stride_words, int64_t L, cudaStream_t s)
{
    if (n <= 0 || n > kMaxConvJobs) return n == 0 ? cudaSuccess : cudaErrorInvalidValue;
    ConvParams c;
    int64_t rows = 0;
    if (!conv_params(jobs, n, c, rows)) return cudaErrorInvalidConfiguration;
    if (rows == 0) return cudaSuccess;
    const int64_t pairs = L / 64;
    const int V = pairs >= 4 ? 4 : 1;
    const unsigned chunks = (unsigned)((pairs + 256 * V - 1) / (256 * V));
    if (rows * (int64_t)chunks > INT32_MAX) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)(rows * chunks);
    if (V == 4)
        bits_to_msc4_kernel<4><<<grid, 256, 0, s>>>(c, stride_words, pairs, chunks);
    else
        bits_to_msc4_kernel<1><<<grid, 256, 0, s>>>(c, stride_words, pairs, chunks);
    return cudaGetLastError();
}

cudaError_t msc4_to_bits(const uint64_t *plane, int64_t stride_words, uint32_t *bits, int64_t L, int64_t rows,
                         cudaStream_t s)
{
    const ConvJob job{plane, bits, rows};
    return msc4_to_bits_multi(&job, 1, stride_words, L, s);
}

cudaError_t bits_to_msc4(const uint32_t *bits, uint64_t *plane, int64_t stride_words, int64_t L, int64_t rows,
                         cudaStream_t s)
{
    const ConvJob job{bits, plane, rows};
    return bits_to_msc4_multi(&job, 1, stride_words, L, s);
}

}  // namespace ising
