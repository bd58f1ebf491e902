// launch.h -- host-side launchers implemented by the kernel translation units
// and called by the C ABI in api.cu.  Every launcher returns the cudaError_t of
// its launch (cudaGetLastError right after it).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ising {

struct DeviceInfo {
    int sm_count;
};

// Multi-spin-coded (4 bits per spin) lattice.
// Rows row0 .. row0+rows-1 of an L x L lattice's plane of one colour; `plane`
// points at the first of them.
cudaError_t msc4_init(uint64_t *plane, int colour, int64_t L, int64_t rows, int64_t row0, int64_t stride_words,
                      int mode, uint64_t seed, cudaStream_t s);
cudaError_t msc4_half_sweep(const Msc4SweepParams &p, int colour, cudaStream_t s);
// Copies n rows of `words` uint64 each: row k from src[k] to dst[k] (n <= kMaxHaloRows).
constexpr int kMaxHaloRows = 128;
struct HaloCopy {
    const uint64_t *src[kMaxHaloRows];
    uint64_t *dst[kMaxHaloRows];
};
cudaError_t msc4_copy_rows(const HaloCopy &c, int n, int64_t words, cudaStream_t s);
cudaError_t msc4_observables(const uint64_t *black, const uint64_t *white, int64_t L,
                             int64_t stride_words, long long *out, cudaStream_t s);
cudaError_t msc4_pack(const int8_t *src, int64_t src_stride, uint64_t *dst, int64_t dst_stride_words,
                      int64_t L, cudaStream_t s);
cudaError_t msc4_unpack(const uint64_t *src, int64_t src_stride_words, int8_t *dst, int64_t dst_stride,
                        int64_t L, cudaStream_t s);
// `rows` rows of an MSC4 plane (row stride in words) <-> the same rows in the
// bit-packed format (L/16 bytes per row, dense); L % 64 == 0.  The _multi
// forms convert up to kMaxConvJobs row ranges (source, destination, rows) of
// the same L and stride in one launch.
constexpr int kMaxConvJobs = 4;
struct ConvJob {
    const void *src;
    void *dst;
    int64_t rows;
};
cudaError_t msc4_to_bits_multi(const ConvJob *jobs, int n, int64_t stride_words, int64_t L, cudaStream_t s);
cudaError_t bits_to_msc4_multi(const ConvJob *jobs, int n, int64_t stride_words, int64_t L, cudaStream_t s);
cudaError_t msc4_to_bits(const uint64_t *plane, int64_t stride_words, uint32_t *bits, int64_t L, int64_t rows,
                         cudaStream_t s);
cudaError_t bits_to_msc4(const uint32_t *bits, uint64_t *plane, int64_t stride_words, int64_t L, int64_t rows,
                         cudaStream_t s);

// One int8 per spin.
cudaError_t int8_init(int8_t *plane, int colour, int64_t L, int64_t stride, int mode, uint64_t seed,
                      cudaStream_t s);
cudaError_t int8_half_sweep(const Int8SweepParams &p, int colour, cudaStream_t s);
cudaError_t int8_observables(const int8_t *black, const int8_t *white, int64_t L, int64_t stride,
                             long long *out, cudaStream_t s);

// Throughput probes (probe.cu): the generator alone, shaped like the sweep
// (n_blocks <= 2^34), and the 32 x 32 -> 64-bit multiply alone (*multiplies
// receives the number the launch performs).
cudaError_t rng_probe(uint64_t n_blocks, const RoundKeys &rk, uint32_t c2, uint32_t c3, uint32_t T3,
                      unsigned long long *count, cudaStream_t s);
cudaError_t mulwide_probe(int form, uint32_t iters, unsigned long long *sink, uint64_t *multiplies, cudaStream_t s);

// ISING_OK if [ptr, ptr + bytes) is device memory of the current device inside
// one allocation; else ISING_EINVAL with the reason in ising_last_error().
int check_device_range(const void *ptr, size_t bytes, const char *name);

// Cached per-device facts (SM count), for the device current on this thread.
cudaError_t device_info(DeviceInfo *info);

}  // namespace ising
