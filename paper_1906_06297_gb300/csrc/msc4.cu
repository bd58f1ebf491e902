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
//     16-byte copy per plane row) and marches down a contiguous range of rows.
//     Rows i-1, i, i+1 of the source plane, the target row and the next rows
//     in flight sit in a per-warp ring in shared memory, filled by cp.async
//     two rows ahead: every source word is read from memory once per
//     half-sweep (plus one halo row at each end of the range), and moving to
//     the next row changes which slot is read instead of moving registers
//     (register moves would compete with Philox for the multiply-add pipe).
//   * The side word is the neighbouring lane's centre word (one warp shuffle);
//     only the chunk edges read a single extra word.
//   * Work is split evenly: the (chunk, row) units of the plane are cut into
//     one contiguous range per resident warp of a persistent grid.
//   * Random numbers: one Philox4x32-10 block per 4 sites, keyed by
//     (seed, sweep, colour, site), compared as uint32 with the a = 3 / a = 4
//     thresholds; everything else is bit-parallel over nibbles.
//   * Observables (white half-sweep): after the update, each white site adds
//     s * (sum of its 4 black neighbours), which visits every bond once; the
//     black centre words already loaded give the black magnetisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "sweep_core.cuh"

namespace ising {

namespace {

// Launch shape of the sweep kernel (compile-time; the defaults are the tuned
// values for GB300).
#ifndef ISING_MSC4_THREADS
#define ISING_MSC4_THREADS 512
#endif
#ifndef ISING_MSC4_MIN_BLOCKS
#define ISING_MSC4_MIN_BLOCKS 1
#endif
constexpr int kThreads = ISING_MSC4_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kMinRowsPerWarp = 16;

__device__ __forceinline__ void st128(uint64_t *p, uint4 v)
{
    *reinterpret_cast<uint4 *>(p) = v;
}

// Each warp keeps its lanes' rows in a ring in shared memory: 4 source rows
// (r-1, r, r+1 and the row r+2 being fetched), 2 target rows and the 4 edge
// words that belong to the source rows.  A lane only ever reads the slots it
// filled itself, so no lane waits for another.
constexpr int kRing = 4;
struct WarpRing {
    uint4 src[kRing][32];
    uint4 tgt[2][32];
    uint32_t edge[kRing][32];
};
constexpr size_t kRingBytes = sizeof(WarpRing) * kWarps;

// Asynchronous global -> shared copies of 16 / 4 bytes that only lanes with
// `pred` issue (cp.async: no registers hold the data in flight).
__device__ __forceinline__ void cp16_if(void *smem, const void *gmem, bool pred)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("{\n\t"
                 ".reg .pred q;\n\t"
                 "setp.ne.b32 q, %2, 0;\n\t"
                 "@q cp.async.cg.shared.global [%0], [%1], 16;\n\t"
                 "}" ::"r"(s), "l"(gmem), "r"((int)pred) : "memory");
}

__device__ __forceinline__ void cp4_if(void *smem, const void *gmem, bool pred)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("{\n\t"
                 ".reg .pred q;\n\t"
                 "setp.ne.b32 q, %2, 0;\n\t"
                 "@q cp.async.ca.shared.global [%0], [%1], 4;\n\t"
                 "}" ::"r"(s), "l"(gmem), "r"((int)pred) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all groups but the most recent one have landed (and are visible to this thread)
__device__ __forceinline__ void cp_wait_all_but_last() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Q64: the Philox counter q = site / 4 needs 64 bits (L above 185363);
// otherwise its high word is 0 and only the low word is carried per row.
template <int COLOR, bool OBS, bool ALWAYS, bool Q64>
__global__ void __launch_bounds__(kThreads, ISING_MSC4_MIN_BLOCKS)
    msc4_sweep_kernel(const __grid_constant__ Msc4SweepParams p)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    WarpRing &ring = reinterpret_cast<WarpRing *>(ring_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    const int64_t begin = gw * p.total / nw;
    const int64_t end = (gw + 1) * p.total / nw;
    const int64_t R = p.rows, stride = p.stride;
    // row r (local) has the neighbour word on the left iff r + pofs is even
    const int64_t pofs = p.row0 + COLOR;
    // local row indices fit 32 bits (rows <= L <= 2^18)
    const int32_t wrap_row = (int32_t)p.wrap_row, wrap_to = (int32_t)p.wrap_to;

    uint32_t ones = 0, dsum = 0, nrows = 0;

    for (int64_t lin = begin; lin < end;) {
        const int64_t chunk = lin / R;
        const int32_t r0 = (int32_t)(lin - chunk * R);
        const int32_t r1 = (int32_t)min(R, r0 + (end - lin));
        lin += r1 - r0;

        const int64_t w0 = chunk * 64 + 2 * lane;
        const bool valid = w0 < p.wpr;
        // chunk-edge lanes read the one side word that no lane of this warp
        // holds: lane 0 the high half of the word on the left, the last valid
        // lane the low half of the word on the right (periodic in the row);
        // offsets in 32-bit units from this lane's first word
        const bool edge_right = valid && (lane == 31 || w0 + 2 >= p.wpr);
        const int64_t off_left = 2 * ((w0 == 0 ? p.wpr : w0) - 1 - w0) + 1;
        const int64_t off_right = 2 * ((w0 + 2 >= p.wpr ? 0 : w0 + 2) - w0);
        const bool edge_left = lane == 0;
        const uint64_t *col = p.src + w0;  // this lane's column of the source plane
        // source row `row` (local index, wrapped) and its edge word into slot k
        auto fetch_src = [&](const uint64_t *rowp, int32_t row, int k) {
            cp16_if(&ring.src[k][lane], rowp, valid);
            const bool left = ((row + pofs) & 1) == 0;
            const uint32_t *h = reinterpret_cast<const uint32_t *>(rowp) + (left ? off_left : off_right);
            cp4_if(&ring.edge[k][lane], h, left ? edge_left : edge_right);
        };

        // rows r0-1, r0, r0+1 of the source and row r0 of the target, then in
        // each iteration the source row two ahead and the next target row
        int32_t rn = r0 + 2 >= wrap_row ? r0 + 2 - wrap_row + wrap_to : r0 + 2;
        const uint64_t *pn = col + (int64_t)rn * stride;
        {
            const int64_t ru = r0 == 0 ? p.first_up : r0 - 1;
            const int32_t rd = r0 + 1 == wrap_row ? wrap_to : r0 + 1;
            cp16_if(&ring.src[(r0 + 3) & 3][lane], col + ru * stride, valid);
            fetch_src(col + (int64_t)r0 * stride, r0, r0 & 3);
            fetch_src(col + (int64_t)rd * stride, r0 + 1, (r0 + 1) & 3);
            cp16_if(&ring.tgt[r0 & 1][lane], p.tgt + w0 + (int64_t)r0 * stride, valid);
            cp_commit();
        }
        uint64_t *tp = p.tgt + w0 + (int64_t)r0 * stride;  // target row r
        uint64_t q0 = (uint64_t)(p.row0 + r0) * (uint64_t)p.qrow + 4 * (uint64_t)w0;
        uint32_t q32 = (uint32_t)q0;

        for (int32_t r = r0; r < r1; ++r) {
            const int k = r & 3;
            fetch_src(pn, rn, (k + 2) & 3);
            cp16_if(&ring.tgt[(k + 1) & 1][lane], tp + stride, valid && r + 1 < r1);
            cp_commit();
            cp_wait_all_but_last();  // rows r-1 .. r+1, target row r and the edge of row r
            const uint4 up = ring.src[(k + 3) & 3][lane];
            const uint4 cur = ring.src[k][lane];
            const uint4 dn = ring.src[(k + 1) & 3][lane];
            const uint4 tg = ring.tgt[k & 1][lane];
            const uint32_t edge = ring.edge[k][lane];

            // side words, as 32-bit halves: .x/.y = lo/hi of word w0, .z/.w of w0+1
            uint4 sd;
            if (((r + pofs) & 1) == 0) {  // left neighbour word: shift up one spin
                const uint32_t prev = __shfl_up_sync(0xffffffffu, cur.w, 1);
                const uint32_t W = edge_left ? edge : prev;
                sd.x = __funnelshift_l(W, cur.x, 4);
                sd.y = __funnelshift_l(cur.x, cur.y, 4);
                sd.z = __funnelshift_l(cur.y, cur.z, 4);
                sd.w = __funnelshift_l(cur.z, cur.w, 4);
            } else {  // right neighbour word: shift down one spin
                const uint32_t next = __shfl_down_sync(0xffffffffu, cur.x, 1);
                const uint32_t E = edge_right ? edge : next;
                sd.x = __funnelshift_r(cur.x, cur.y, 4);
                sd.y = __funnelshift_r(cur.y, cur.z, 4);
                sd.z = __funnelshift_r(cur.z, cur.w, 4);
                sd.w = __funnelshift_r(cur.w, E, 4);
            }
            // Philox blocks q0 .. q0+7 cover the lane's 32 sites; q0 % 8 == 0,
            // so the low counter word never carries within them
            const uint32_t c0 = Q64 ? (uint32_t)q0 : q32, c1 = Q64 ? (uint32_t)(q0 >> 32) : 0u;
            uint32_t dacc = 0;
            uint4 ns;
            // nibble-wise neighbour sums stay in 0..4: no carry leaves a nibble
            const DrawCtx dc{p.c2, p.c3, p.acc.T3, p.acc.T4, p.acc.zero};
            ns.x = update_half<OBS, ALWAYS>(tg.x, up.x + dn.x + cur.x, sd.x, c0, c1, dc, p.rk, dacc);
            ns.y = update_half<OBS, ALWAYS>(tg.y, up.y + dn.y + cur.y, sd.y, c0 | 2, c1, dc, p.rk, dacc);
            ns.z = update_half<OBS, ALWAYS>(tg.z, up.z + dn.z + cur.z, sd.z, c0 | 4, c1, dc, p.rk, dacc);
            ns.w = update_half<OBS, ALWAYS>(tg.w, up.w + dn.w + cur.w, sd.w, c0 | 6, c1, dc, p.rk, dacc);
            if (valid) st128(tp, ns);

            if (OBS && valid) {
                // up-spin counts of the 32 white and 32 black sites, nibble-wise
                // (at most 8 per nibble), then folded to bytes
                const uint32_t n8 = ns.x + ns.y + ns.z + ns.w + cur.x + cur.y + cur.z + cur.w;
                const uint32_t sb = (n8 & 0x0F0F0F0Fu) + ((n8 >> 4) & 0x0F0F0F0Fu);
                ones += (sb * 0x01010101u) >> 24;    // 4 byte lanes of at most 16
                dsum += (dacc * 0x01010101u) >> 24;  // 4 byte lanes of at most 32
                nrows += 1;
            }
            tp += stride;
            if (Q64) q0 += (uint64_t)p.qrow;
            else q32 += (uint32_t)p.qrow;
            pn += stride;
            if (++rn == wrap_row) {
                rn = wrap_to;
                pn = col + (int64_t)rn * stride;
            }
        }
        // the last group (the unused prefetch) lands before the slots serve
        // the next range
        cp_wait_all();
    }
    if (OBS) {
        // per lane and row: 32 white + 32 black spins; 32 white sites x 4 bonds
        const long long sum_s = 2 * (long long)ones - 64 * (long long)nrows;
        const long long sum_b = 128 * (long long)nrows - 2 * (long long)dsum;
        block_reduce_add2<kThreads>(sum_s, sum_b, p.obs);
    }
}

struct Occupancy {
    std::mutex mu;
    int blocks[64][16] = {};  // per device: colour x obs x always x q64
};
Occupancy g_occ;

template <int COLOR, bool OBS, bool ALWAYS, bool Q64>
int sweep_blocks_per_sm()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(g_occ.mu);
    int &b = g_occ.blocks[dev][COLOR * 8 + (OBS ? 4 : 0) + (ALWAYS ? 2 : 0) + (Q64 ? 1 : 0)];
    if (b == 0) {
        auto k = msc4_sweep_kernel<COLOR, OBS, ALWAYS, Q64>;
        int n = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads, kRingBytes) != cudaSuccess || n < 1)
            n = 1;
        b = n;
    }
    return b;
}

template <int COLOR, bool OBS, bool ALWAYS, bool Q64>
cudaError_t launch_sweep(const Msc4SweepParams &p, cudaStream_t s)
{
    DeviceInfo info;
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return e;
    const int per_sm = sweep_blocks_per_sm<COLOR, OBS, ALWAYS, Q64>();
    const int64_t sms = std::max<int64_t>(1, (int64_t)info.sm_count - p.spare_sms);
    const int64_t max_warps = sms * per_sm * kWarps;
    const int64_t want = std::max<int64_t>(1, (p.total + kMinRowsPerWarp - 1) / kMinRowsPerWarp);
    const int64_t warps = std::min(max_warps, want);
    const int64_t blocks = (warps + kWarps - 1) / kWarps;
    msc4_sweep_kernel<COLOR, OBS, ALWAYS, Q64><<<(unsigned)blocks, kThreads, kRingBytes, s>>>(p);
    return cudaGetLastError();
}

template <int COLOR, bool OBS, bool ALWAYS>
cudaError_t launch_sweep_q(const Msc4SweepParams &p, cudaStream_t s)
{
    // the Philox counter of the last row's blocks fits 32 bits up to L = 185363
    const bool q64 = (uint64_t)(p.row0 + p.rows + 1) * (uint64_t)p.qrow > 0xFFFFFFFFull;
    return q64 ? launch_sweep<COLOR, OBS, ALWAYS, true>(p, s) : launch_sweep<COLOR, OBS, ALWAYS, false>(p, s);
}

template <int COLOR>
cudaError_t launch_sweep_colour(const Msc4SweepParams &p, cudaStream_t s)
{
    const bool obs = p.obs != nullptr, always = p.acc.always != 0;
    if (always) return obs ? launch_sweep_q<COLOR, true, true>(p, s) : launch_sweep_q<COLOR, false, true>(p, s);
    return obs ? launch_sweep_q<COLOR, true, false>(p, s) : launch_sweep_q<COLOR, false, false>(p, s);
}

// ---------------------------------------------------------------------------
// Initial state: thread per word.  Random: spin n of word (i, w) has plane site
// i*L/2 + 16w + n and is +1 iff its purpose-1 draw at t = 0 is below 2^31.
// ---------------------------------------------------------------------------
__global__ void msc4_init_kernel(uint64_t *plane, int64_t L, int64_t rows, int64_t row0, int64_t stride, int mode,
                                 uint32_t c3, const __grid_constant__ RoundKeys rk)
{
    const int64_t wpr = L / 32, qrow = L / 8;
    const int64_t n = rows * wpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / wpr, w = idx - i * wpr;  // local row i = global row row0 + i
        uint64_t word;
        if (mode == 1) {
            word = 0x1111111111111111ull;
        } else if (mode == 2) {
            word = 0;
        } else {
            word = 0;
            const uint64_t q0 = (uint64_t)(row0 + i) * qrow + 4 * (uint64_t)w;
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
    return colour == 0 ? launch_sweep_colour<0>(p, s) : launch_sweep_colour<1>(p, s);
}

cudaError_t msc4_init(uint64_t *plane, int colour, int64_t L, int64_t rows, int64_t row0, int64_t stride_words,
                      int mode, uint64_t seed, cudaStream_t s)
{
    const RoundKeys rk = make_round_keys(seed);
    const int64_t n = rows * (L / 32);
    msc4_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(plane, L, rows, row0, stride_words, mode,
                                                      counter_word3(colour, kPurposeInit, 0), rk);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Halo rows of slabs: block k copies row k (16-byte aligned, an even number of
// words) with 128-bit accesses.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) msc4_copy_rows_kernel(const __grid_constant__ HaloCopy c, int64_t words)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(c.src[blockIdx.x]);
    uint4 *dst = reinterpret_cast<uint4 *>(c.dst[blockIdx.x]);
    for (int64_t v = threadIdx.x; v < words / 2; v += blockDim.x) dst[v] = src[v];
}

cudaError_t msc4_copy_rows(const HaloCopy &c, int n, int64_t words, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    msc4_copy_rows_kernel<<<n, 256, 0, s>>>(c, words);
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
