// msc4.cu -- kernels on the multi-spin-coded lattice: 16 spins of one colour
// per uint64, 4 bits per spin, -1/+1 stored as 0/1 (Sec. 3.3 of the paper).
//
// Plane layout: L rows of L/32 words; compacted column j sits in word j/16 at
// bits 4*(j%16) .. +3.  Site (i, c) is black iff (i + c) is even and has
// compacted column j = c/2 (Sec. 3.1, Fig. 1).
//
// Neighbours of the target word (i, w) in the source plane (Sec. 3.3, Fig. 3):
// the words (i-1, w), (i, w), (i+1, w) give the vertical and one horizontal
// neighbour of all 16 spins; the other horizontal neighbour comes from the
// centre word shifted by one spin, with the missing spin shifted in from the
// word on the left (black on even rows, white on odd rows) or on the right
// (black on odd rows, white on even rows).  With spins as 0/1 nibbles, the
// four neighbour words add nibble-wise without carries (each sum is 0..4).
//
// Sweep kernel design (GB300, sm_103a):
//   * Each warp owns a 64-word column chunk (lane l holds words 2l, 2l+1, one
//     128-bit load per plane row) and marches down a contiguous range of rows,
//     keeping rows i-1, i, i+1 of the source plane in registers: every source
//     word is read from memory once per half-sweep (plus one halo row at each
//     end of the range).
//   * The side word is the neighbouring lane's centre word (one warp shuffle);
//     only the chunk edges read a single extra word.
//   * Work is split evenly: the (chunk, row) units of the plane are cut into
//     one contiguous range per resident warp of a persistent grid.
//   * Random numbers: one Philox4x32-10 block per 4 sites, keyed by
//     (seed, sweep, colour, site), compared as uint32 with the a = 3 / a = 4
//     thresholds; everything else is bit-parallel over nibbles.
//   * Observables (white half-sweep): after the update, each white site adds
//     s * (sum of its 4 black neighbours), which visits every bond once; the
//     black centre words already in registers give the black magnetisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace ising {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMinRowsPerWarp = 16;

__device__ __forceinline__ ulonglong2 ld128(const uint64_t *p)
{
    return *reinterpret_cast<const ulonglong2 *>(p);
}

__device__ __forceinline__ void st128(uint64_t *p, uint64_t x, uint64_t y)
{
    *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x, y);
}

// New values of 8 spins (one 32-bit half word).  s: spins, k: neighbour sums
// (nibble-wise 0..4); blocks c0 and c0+1 give the 8 draws (spin n uses word
// n%4 of block c0 + n/4).  With OBS, adds the anti-aligned counts after the
// update into the byte lanes of dbytes.
template <bool OBS>
__device__ __forceinline__ uint32_t update_half(uint32_t s, uint32_t k, uint32_t c0, uint32_t c1,
                                                const Msc4SweepParams &p, uint32_t &dbytes)
{
    uint32_t r3 = 0, r4 = 0;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const uint4 u = philox(c0 + b, c1, p.c2, p.c3, p.rk);
        const int sh = 16 * b;
        r3 |= ((uint32_t)(u.x < p.acc.T3) << sh) | ((uint32_t)(u.y < p.acc.T3) << (sh + 4)) |
              ((uint32_t)(u.z < p.acc.T3) << (sh + 8)) | ((uint32_t)(u.w < p.acc.T3) << (sh + 12));
        r4 |= ((uint32_t)(u.x < p.acc.T4) << sh) | ((uint32_t)(u.y < p.acc.T4) << (sh + 4)) |
              ((uint32_t)(u.z < p.acc.T4) << (sh + 8)) | ((uint32_t)(u.w < p.acc.T4) << (sh + 12));
    }
    // d = number of anti-aligned neighbours (4 - a): k for a down spin,
    // 4 - k for an up spin.
    const uint32_t m = s * 15u;
    const uint32_t k4 = 0x44444444u - k;
    const uint32_t d = (k & ~m) | (k4 & m);
    const uint32_t t1 = d >> 1;
    const uint32_t ge2 = (t1 | (t1 >> 1)) & kNibbleLsb;  // d >= 2: dE <= 0, always flip
    const uint32_t eq1 = d & ~ge2 & kNibbleLsb;          // d == 1: a = 3
    const uint32_t eq0 = ~(d | ge2) & kNibbleLsb;        // d == 0: a = 4
    const uint32_t flip = ge2 | (eq1 & (r3 | p.acc.A3)) | (eq0 & (r4 | p.acc.A4));
    const uint32_t ns = s ^ flip;
    if (OBS) {
        const uint32_t m2 = ns * 15u;
        const uint32_t d2 = (k & ~m2) | (k4 & m2);
        dbytes += (d2 & 0x0F0F0F0Fu) + ((d2 >> 4) & 0x0F0F0F0Fu);
    }
    return ns;
}

template <bool OBS>
__device__ __forceinline__ uint64_t update_word(uint64_t s, uint64_t k, uint64_t q0, const Msc4SweepParams &p,
                                                uint32_t &dbytes)
{
    // q0 is a multiple of 4, so the low counter word of its 4 blocks never carries.
    const uint32_t c0 = (uint32_t)q0, c1 = (uint32_t)(q0 >> 32);
    const uint32_t lo = update_half<OBS>((uint32_t)s, (uint32_t)k, c0, c1, p, dbytes);
    const uint32_t hi = update_half<OBS>((uint32_t)(s >> 32), (uint32_t)(k >> 32), c0 + 2, c1, p, dbytes);
    return ((uint64_t)hi << 32) | lo;
}

template <int COLOR, bool OBS>
__global__ void __launch_bounds__(kThreads) msc4_sweep_kernel(const __grid_constant__ Msc4SweepParams p)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    const int64_t begin = gw * p.total / nw;
    const int64_t end = (gw + 1) * p.total / nw;

    long long ones = 0, dsum = 0, nrows = 0;

    for (int64_t lin = begin; lin < end;) {
        const int64_t chunk = lin / p.L;
        const int64_t r0 = lin - chunk * p.L;
        const int64_t r1 = min(p.L, r0 + (end - lin));
        lin += r1 - r0;

        const int64_t w0 = chunk * 64 + 2 * lane;
        const bool valid = w0 < p.wpr;
        // chunk-edge lanes read the one side word that no lane of this warp holds
        const bool edge_right = valid && (lane == 31 || w0 + 2 >= p.wpr);
        const int64_t w_left = (w0 == 0 ? p.wpr : w0) - 1;
        const int64_t w_right = (w0 + 2 >= p.wpr) ? 0 : w0 + 2;

        auto load_row = [&](int64_t r) {
            return valid ? ld128(p.src + r * p.stride + w0) : make_ulonglong2(0, 0);
        };
        auto load_edge = [&](int64_t r) -> uint64_t {
            const bool left = ((r + COLOR) & 1) == 0;
            if (left) return lane == 0 ? p.src[r * p.stride + w_left] : 0;
            return edge_right ? p.src[r * p.stride + w_right] : 0;
        };

        ulonglong2 up = load_row(r0 == 0 ? p.L - 1 : r0 - 1);
        ulonglong2 cur = load_row(r0);
        uint64_t edge = load_edge(r0);

        for (int64_t r = r0; r < r1; ++r) {
            const int64_t rdn = (r + 1 == p.L) ? 0 : r + 1;
            const ulonglong2 dn = load_row(rdn);
            const uint64_t edge_dn = load_edge(rdn);
            uint64_t *trow = p.tgt + r * p.stride;
            const ulonglong2 tg = valid ? ld128(trow + w0) : make_ulonglong2(0, 0);

            // side word: the source spin on the far side of each target spin
            uint64_t sx, sy;
            if (((r + COLOR) & 1) == 0) {  // left neighbour word
                const uint64_t prev = __shfl_up_sync(0xffffffffu, cur.y, 1);
                const uint64_t W = lane == 0 ? edge : prev;
                sx = (cur.x << 4) | (W >> 60);
                sy = (cur.y << 4) | (cur.x >> 60);
            } else {  // right neighbour word
                const uint64_t next = __shfl_down_sync(0xffffffffu, cur.x, 1);
                const uint64_t E = edge_right ? edge : next;
                sx = (cur.x >> 4) | (cur.y << 60);
                sy = (cur.y >> 4) | (E << 60);
            }
            // nibble-wise neighbour sums, 0..4: no carry ever leaves a nibble
            const uint64_t kx = up.x + dn.x + cur.x + sx;
            const uint64_t ky = up.y + dn.y + cur.y + sy;

            const uint64_t q0 = (uint64_t)r * (uint64_t)p.qrow + 4 * (uint64_t)w0;
            uint32_t dbytes = 0;
            const uint64_t nx = update_word<OBS>(tg.x, kx, q0, p, dbytes);
            const uint64_t ny = update_word<OBS>(tg.y, ky, q0 + 4, p, dbytes);
            if (valid) st128(trow + w0, nx, ny);

            if (OBS && valid) {
                dsum += (dbytes * 0x01010101u) >> 24;
                ones += __popcll(nx) + __popcll(ny) + __popcll(cur.x) + __popcll(cur.y);
                nrows += 1;
            }
            up = cur;
            cur = dn;
            edge = edge_dn;
        }
    }
    if (OBS) {
        // per lane and row: 32 white + 32 black spins; 32 white sites x 4 bonds
        const long long sum_s = 2 * ones - 64 * nrows;
        const long long sum_b = 128 * nrows - 2 * dsum;
        block_reduce_add2<kThreads>(sum_s, sum_b, p.obs);
    }
}

struct Occupancy {
    std::mutex mu;
    int blocks[64][4] = {};  // per device: colour x obs
};
Occupancy g_occ;

template <int COLOR, bool OBS>
int sweep_blocks_per_sm()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(g_occ.mu);
    int &b = g_occ.blocks[dev][COLOR * 2 + (OBS ? 1 : 0)];
    if (b == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, msc4_sweep_kernel<COLOR, OBS>, kThreads, 0) !=
                cudaSuccess ||
            n < 1)
            n = 1;
        b = n;
    }
    return b;
}

template <int COLOR, bool OBS>
cudaError_t launch_sweep(const Msc4SweepParams &p, cudaStream_t s)
{
    DeviceInfo info;
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return e;
    const int64_t max_warps = (int64_t)info.sm_count * sweep_blocks_per_sm<COLOR, OBS>() * kWarps;
    const int64_t want = std::max<int64_t>(1, (p.total + kMinRowsPerWarp - 1) / kMinRowsPerWarp);
    const int64_t warps = std::min(max_warps, want);
    const int64_t blocks = (warps + kWarps - 1) / kWarps;
    msc4_sweep_kernel<COLOR, OBS><<<(unsigned)blocks, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial state: thread per word.  Random: spin n of word (i, w) has plane site
// i*L/2 + 16w + n and is +1 iff its purpose-1 draw at t = 0 is below 2^31.
// ---------------------------------------------------------------------------
__global__ void msc4_init_kernel(uint64_t *plane, int64_t L, int64_t stride, int mode, uint32_t c3,
                                 const __grid_constant__ RoundKeys rk)
{
    const int64_t wpr = L / 32, qrow = L / 8;
    const int64_t n = L * wpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / wpr, w = idx - i * wpr;
        uint64_t word;
        if (mode == 1) {
            word = 0x1111111111111111ull;
        } else if (mode == 2) {
            word = 0;
        } else {
            word = 0;
            const uint64_t q0 = (uint64_t)i * qrow + 4 * (uint64_t)w;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint4 u = philox((uint32_t)q0 + b, (uint32_t)(q0 >> 32), 0u, c3, rk);
                const int sh = 16 * b;
                word |= ((uint64_t)(u.x < 0x80000000u) << sh) | ((uint64_t)(u.y < 0x80000000u) << (sh + 4)) |
                        ((uint64_t)(u.z < 0x80000000u) << (sh + 8)) | ((uint64_t)(u.w < 0x80000000u) << (sh + 12));
            }
        }
        plane[i * stride + w] = word;
    }
}

// ---------------------------------------------------------------------------
// Observables without an update: thread per white word.  Same neighbour rule
// as the white half-sweep; each white site contributes s * (sum of its black
// neighbours) = 4 - 2d (d = anti-aligned count), each site its spin.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) msc4_obs_kernel(const uint64_t *black, const uint64_t *white, int64_t L,
                                                       int64_t stride, long long *out)
{
    const int64_t wpr = L / 32;
    const int64_t n = L * wpr;
    long long ones = 0, dsum = 0, cnt = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / wpr, w = idx - i * wpr;
        const int64_t iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
        const uint64_t C = black[i * stride + w];
        uint64_t side;
        if ((i & 1) == 1) {  // white, odd row: left word
            const uint64_t W = black[i * stride + (w == 0 ? wpr - 1 : w - 1)];
            side = (C << 4) | (W >> 60);
        } else {
            const uint64_t E = black[i * stride + (w + 1 == wpr ? 0 : w + 1)];
            side = (C >> 4) | (E << 60);
        }
        const uint64_t k = black[iu * stride + w] + black[id * stride + w] + C + side;
        const uint64_t s = white[i * stride + w];
        const uint64_t m = s * 15ull;
        const uint64_t d = (k & ~m) | ((0x4444444444444444ull - k) & m);
        const uint64_t nib = (d & 0x0F0F0F0F0F0F0F0Full) + ((d >> 4) & 0x0F0F0F0F0F0F0F0Full);
        dsum += (long long)((nib * 0x0101010101010101ull) >> 56);
        ones += __popcll(s) + __popcll(C);
        cnt += 1;
    }
    block_reduce_add2<256>(2 * ones - 32 * cnt, 64 * cnt - 2 * dsum, out);
}

// ---------------------------------------------------------------------------
// Layout conversion: thread per word; int8 column j <-> word j/16, nibble j%16.
// ---------------------------------------------------------------------------
__global__ void msc4_pack_kernel(const int8_t *src, int64_t sstride, uint64_t *dst, int64_t dstride, int64_t L)
{
    const int64_t wpr = L / 32, n = L * wpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / wpr, w = idx - i * wpr;
        const int8_t *row = src + i * sstride + 16 * w;
        uint64_t word = 0;
#pragma unroll
        for (int t = 0; t < 16; ++t) word |= (uint64_t)(row[t] > 0) << (4 * t);
        dst[i * dstride + w] = word;
    }
}

__global__ void msc4_unpack_kernel(const uint64_t *src, int64_t sstride, int8_t *dst, int64_t dstride, int64_t L)
{
    const int64_t wpr = L / 32, n = L * wpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / wpr, w = idx - i * wpr;
        const uint64_t word = src[i * sstride + w];
        int8_t *row = dst + i * dstride + 16 * w;
#pragma unroll
        for (int t = 0; t < 16; ++t) row[t] = ((word >> (4 * t)) & 1) ? 1 : -1;
    }
}

unsigned grid_for(int64_t n, int threads)
{
    DeviceInfo info{1};
    device_info(&info);
    const int64_t cap = (int64_t)info.sm_count * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (n + threads - 1) / threads));
}

}  // namespace

cudaError_t msc4_half_sweep(const Msc4SweepParams &p, int colour, cudaStream_t s)
{
    const bool obs = p.obs != nullptr;
    if (colour == 0) return obs ? launch_sweep<0, true>(p, s) : launch_sweep<0, false>(p, s);
    return obs ? launch_sweep<1, true>(p, s) : launch_sweep<1, false>(p, s);
}

cudaError_t msc4_init(uint64_t *plane, int colour, int64_t L, int64_t stride_words, int mode, uint64_t seed,
                      cudaStream_t s)
{
    const RoundKeys rk = make_round_keys(seed);
    const int64_t n = L * (L / 32);
    msc4_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(plane, L, stride_words, mode,
                                                      counter_word3(colour, kPurposeInit, 0), rk);
    return cudaGetLastError();
}

cudaError_t msc4_observables(const uint64_t *black, const uint64_t *white, int64_t L, int64_t stride_words,
                             long long *out, cudaStream_t s)
{
    const int64_t n = L * (L / 32);
    msc4_obs_kernel<<<grid_for(n, 256), 256, 0, s>>>(black, white, L, stride_words, out);
    return cudaGetLastError();
}

cudaError_t msc4_pack(const int8_t *src, int64_t src_stride, uint64_t *dst, int64_t dst_stride_words, int64_t L,
                      cudaStream_t s)
{
    const int64_t n = L * (L / 32);
    msc4_pack_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, src_stride, dst, dst_stride_words, L);
    return cudaGetLastError();
}

cudaError_t msc4_unpack(const uint64_t *src, int64_t src_stride_words, int8_t *dst, int64_t dst_stride, int64_t L,
                        cudaStream_t s)
{
    const int64_t n = L * (L / 32);
    msc4_unpack_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, src_stride_words, dst, dst_stride, L);
    return cudaGetLastError();
}

}  // namespace ising
