// batch.cu -- many independent multi-spin-coded lattices swept in one
// persistent launch, with replica exchange (parallel tempering) between the
// temperatures of each ladder of lattices.  Not in the paper: this is the
// batched form of its checkerboard Metropolis sweep (Sec. 2, Sec. 3.3).
//
// Layout.  Lattice i (side L_i, a multiple of 32) stores each colour plane as
// L_i rows of L_i/32 words (the MSC4 layout of a single lattice) at word
// offset word_off[i] of one black and one white buffer.  Lattices of equal
// side that are adjacent in the batch form a group; group g is cut into work
// items of wpt_g consecutive words of one row, 32 items to a chunk, and every
// chunk lies inside one lattice.  Groups whose side is a power of two from
// 128 to 2048 are swept by the row-marching path instead (see march_rows):
// items of 2 words, a chunk is a warp's worth of whole rows, and a warp's
// chunks are marched row after row by its lane groups.
//
// Draws.  Lattice i uses Philox4x32-10 with the batch seed as key and i added
// to counter word 1 (its "stream"); lattice 0 of a batch therefore follows
// the same trajectory as the single-lattice entry points with the same seed.
// The exchange draw of slot pair (k, k+1) of ladder l at sweep t is the
// purpose-2 draw of site k in stream l.
//
// Schedule (one cooperative launch, grid-wide barriers between phases):
//   for each sweep t:  black half-sweep | barrier | white half-sweep
//   (with per-lattice observables when t is a record sweep) | barrier |
//   on record sweeps: record and exchange | barrier.
// Every barrier wait is bounded: after `timeout_cycles` the block sets the
// error flag to ISING_ETIMEOUT and the whole grid returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "common.cuh"
#include "launch.h"
#include "sweep_core.cuh"

// Size of the fixed scratch array of ising_batch_run_noalloc (4 MiB).
#define ISING_NOALLOC_SCRATCH_BYTES (4u << 20)


namespace ising {

namespace {

constexpr int kMaxGroups = 16;
constexpr int kMarchMinL = 128;  // smallest side of the row-marching path

struct BatchGroup {
    int64_t first;        // first lattice id of the group
    int64_t count;        // lattices in the group
    int64_t word_base;    // word offset of the first lattice's plane
    int64_t chunk_begin;  // first chunk (32 items) of the group
    int64_t items;        // items per lattice = L * wpr / wpt
    int64_t weight_begin; // cumulative work weight of the groups before this one
    int32_t L, wpr, wpt, gpr;  // side, words per row, words per item, items per row
    int32_t weight;       // work weight of one chunk: wpt + kappa
    int32_t march;        // 1: rows marched by lane groups (side a power of two, 128 .. 2048)
};

struct BatchParams {
    uint64_t *black, *white;
    BatchGroup g[kMaxGroups];
    int32_t n_groups;
    int32_t S;            // ladder size
    int64_t n;            // lattices
    int64_t n_ladders;
    int64_t n_chunks;
    int64_t plane_words;  // words of one colour plane over all lattices
    int64_t total_weight; // sum of the chunk weights
    int32_t *slot_of;     // [n] slot of each lattice
    int32_t *lattice_at;  // [n_ladders * S] lattice at each (ladder, slot)
    const uint32_t *thr;  // [S][2] (T3, T4) of each slot's beta
    const int64_t *swap_off, *swap_len;  // [S - 1] exchange threshold tables
    const uint64_t *swap_tab;
    long long *acc;       // [n][2] observables accumulators
    long long *trace;     // [events][n][2] or nullptr
    unsigned *bar;        // [0] arrivals, [1] generation
    int *err;
    int64_t n_sweeps;
    uint64_t t0;
    int64_t event_first;
    int32_t record_every, swaps;
    long long timeout_cycles;
    int32_t expect_blocks;  // blocks a barrier waits for (gridDim.x; larger only in the self-test)
    RoundKeys rk;
};

// ---------------------------------------------------------------------------
// Grid-wide barrier with a bounded wait.  Thread 0 of each block arrives on a
// counter; the last arrival resets it and bumps the generation word, which
// the others poll.  Returns false (in every thread) once any block has set
// the error flag; the caller then returns.
// ---------------------------------------------------------------------------
__device__ bool grid_sync(const BatchParams &p)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = p.bar + 1;
        volatile int *err = p.err;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(p.bar, 1u) + 1;
        if (arrived == (unsigned)p.expect_blocks) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 1, 1u);
        } else {
            const long long start = clock64();
            while (*gen == g0) {
                if (*err != 0) break;
                if (clock64() - start > p.timeout_cycles) {
                    atomicCAS(p.err, 0, (int)ISING_ETIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = (*err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// One work item: `WPT` consecutive words of row r of one lattice.
template <int WPT, bool OBS>
__device__ __forceinline__ void sweep_item(const uint64_t *__restrict__ src, uint64_t *__restrict__ tgt, int L,
                                           int wpr, int r, int w0, int colour, uint32_t stream, const DrawCtx &dc,
                                           const RoundKeys &rk, uint32_t &ones, uint32_t &dsum)
{
    const int ru = r == 0 ? L - 1 : r - 1, rd = r + 1 == L ? 0 : r + 1;
    const uint64_t *rc = src + (int64_t)r * wpr, *ra = src + (int64_t)ru * wpr, *rb = src + (int64_t)rd * wpr;
    uint64_t *rt = tgt + (int64_t)r * wpr;
    uint64_t C[WPT], U[WPT], D[WPT], T[WPT];
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
        C[j] = rc[w0 + j];
        U[j] = ra[w0 + j];
        D[j] = rb[w0 + j];
        T[j] = rt[w0 + j];
    }
    const bool left = ((r + colour) & 1) == 0;
    const uint64_t edge = left ? rc[(w0 == 0 ? wpr : w0) - 1] : rc[(w0 + WPT == wpr) ? 0 : w0 + WPT];
    const uint64_t q0 = (uint64_t)r * (uint64_t)(L / 8) + 4 * (uint64_t)w0;
    uint32_t dacc = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
        uint64_t side;
        if (left) {
            const uint64_t W = j == 0 ? edge : C[j - 1];
            side = (C[j] << 4) | (W >> 60);
        } else {
            const uint64_t E = j == WPT - 1 ? edge : C[j + 1];
            side = (C[j] >> 4) | (E << 60);
        }
        const uint64_t tsum = U[j] + D[j] + C[j];
        const uint32_t c0 = (uint32_t)(q0 + 4 * j);
        const uint32_t c1 = (uint32_t)((q0 + 4 * j) >> 32) + stream;
        const uint32_t lo = update_half<OBS, false>((uint32_t)T[j], (uint32_t)tsum, (uint32_t)side, c0, c1, dc, rk, dacc);
        const uint32_t hi = update_half<OBS, false>((uint32_t)(T[j] >> 32), (uint32_t)(tsum >> 32),
                                                    (uint32_t)(side >> 32), c0 | 2, c1, dc, rk, dacc);
        const uint64_t ns = ((uint64_t)hi << 32) | lo;
        rt[w0 + j] = ns;
        if (OBS) ones += __popcll(ns) + __popcll(C[j]);
    }
    if (OBS) dsum += (dacc & 0xFFu) + ((dacc >> 8) & 0xFFu) + ((dacc >> 16) & 0xFFu) + (dacc >> 24);
}

// ---------------------------------------------------------------------------
// Row-marching path for lattices whose side L is a power of two from 128 to
// 2048.  A row of L/32 words is held whole by a group of L/64 lanes, 2 words
// (16 bytes) per lane, so a warp holds 32 / (L/64) rows side by side.  The
// chunks a warp owns in such a group are consecutive rows of the group's row
// space (lattice-major); they are cut into one run of consecutive rows per lane
// group, and each lane group marches down its run as the single-lattice kernel
// does: each lane copies its 16 bytes of the source row two ahead and of the
// next target row into a per-warp ring in shared memory with cp.async, and
// reads rows r-1, r, r+1 back from its own slots.  The side word comes from the
// neighbouring lane of the same row (periodic within the lane group), so no lane
// loads an edge word.  At the start of each lattice of its run a lane group
// refetches rows L-1, 0, 1 of that lattice (the rows before do not belong to
// it) and takes the lattice's stream and thresholds.
// ---------------------------------------------------------------------------
struct MarchRing {
    uint4 src[4][32];
    uint4 tgt[2][32];
};

__device__ __forceinline__ void cp16_if(void *smem, const void *gmem, bool pred)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("{\n\t"
                 ".reg .pred q;\n\t"
                 "setp.ne.b32 q, %2, 0;\n\t"
                 "@q cp.async.cg.shared.global [%0], [%1], 16;\n\t"
                 "}" ::"r"(sa), "l"(gmem), "r"((int)pred) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_last() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Adds a lane group's observables of one lattice: per lane and row 32 white
// sites (4 bonds each) and 32 black centres were counted, `ones` of them up.
template <bool OBS>
__device__ __forceinline__ void march_flush(const BatchParams &p, int64_t lat, unsigned gmask, int lpr, int j,
                                            uint32_t &ones, uint32_t &dsum, uint32_t &nrows)
{
    if (!OBS) return;
    long long a = ones, b = dsum, c = nrows;
    for (int off = lpr >> 1; off > 0; off >>= 1) {
        a += __shfl_xor_sync(gmask, a, off);
        b += __shfl_xor_sync(gmask, b, off);
        c += __shfl_xor_sync(gmask, c, off);
    }
    if (j == 0 && c > 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p.acc + 2 * lat), (unsigned long long)(2 * a - 64 * c));
        atomicAdd(reinterpret_cast<unsigned long long *>(p.acc + 2 * lat + 1), (unsigned long long)(128 * c - 2 * b));
    }
    ones = dsum = nrows = 0;
}

// Chunks [c0, c1) (relative to the group) of march group G: rows
// [c0 P, c1 P) of the group's row space, P = rows per warp, as P runs of
// n = c1 - c0 rows, run k for lane group k.
template <bool OBS>
__device__ void march_rows(const BatchParams &p, const BatchGroup &G, int64_t c0, int64_t c1, int colour,
                           uint64_t t, MarchRing &ring)
{
    const int lane = threadIdx.x & 31;
    const int lpr = G.gpr;  // lanes per row
    const int P = 32 / lpr;
    const int grp = lane / lpr, j = lane - grp * lpr;
    const unsigned gmask = lpr == 32 ? 0xffffffffu : ((1u << lpr) - 1u) << (grp * lpr);
    const int n = (int)(c1 - c0);
    const int L = G.L, wpr = G.wpr;
    const int64_t rho = c0 * P + (int64_t)grp * n;  // first row of this lane group's run
    int64_t li = rho / L;
    int r = (int)(rho - li * L);
    const int64_t lat_words = (int64_t)L * wpr;
    const uint64_t *src_all = (colour == 0 ? p.white : p.black) + G.word_base + 2 * j;
    uint64_t *tgt_all = (colour == 0 ? p.black : p.white) + G.word_base + 2 * j;
    const int left_lane = grp * lpr + (j == 0 ? lpr - 1 : j - 1);
    const int right_lane = grp * lpr + (j + 1 == lpr ? 0 : j + 1);
    // Philox block of the lane's first site: q = r * L/8 + 4 * (2j), below 2^19
    const uint32_t qrow = (uint32_t)(L / 8), qlane = 8u * (uint32_t)j;
    DrawCtx dc{(uint32_t)t, counter_word3(colour, kPurposeMetropolis, t), 0u, 0u, 0u};
    const uint64_t *src = src_all;
    uint64_t *tgt = tgt_all;
    // row addresses carried from row to row (no multiply per row): the target
    // row r and the source row (r + 2) mod L; q = r L/8 + 8 j
    const uint64_t *src2 = src_all;
    uint64_t *tgt_r = tgt_all;
    uint32_t q = 0;
    int64_t lat = 0;
    uint32_t stream = 0, ones = 0, dsum = 0, nrows = 0;
    // lattice li from row r on, for step s: its stream and thresholds, and
    // source rows r-1, r, r+1 and target row r into the slots of step s
    auto enter = [&](int s) {
        lat = G.first + li;
        src = src_all + li * lat_words;
        tgt = tgt_all + li * lat_words;
        tgt_r = tgt + (int64_t)r * wpr;
        src2 = src + (int64_t)(r + 2 >= L ? r + 2 - L : r + 2) * wpr;
        q = (uint32_t)r * qrow + qlane;
        const int slot = p.slot_of[lat];
        dc.T3 = p.thr[2 * slot];
        dc.T4 = p.thr[2 * slot + 1];
        stream = (uint32_t)lat;
        const int ru = r == 0 ? L - 1 : r - 1, rd = r + 1 == L ? 0 : r + 1;
        cp16_if(&ring.src[(s + 3) & 3][lane], src + (int64_t)ru * wpr, true);
        cp16_if(&ring.src[s & 3][lane], src + (int64_t)r * wpr, true);
        cp16_if(&ring.src[(s + 1) & 3][lane], src + (int64_t)rd * wpr, true);
        cp16_if(&ring.tgt[s & 1][lane], tgt + (int64_t)r * wpr, true);
        cp_commit();
    };
    if (n > 0) enter(0);
    for (int s = 0; s < n; ++s) {
        const bool last_row = r + 1 == L, more = s + 1 < n;
        // rows two ahead (source) and one ahead (target) of the same lattice;
        // none after its last row, where the next step enters a new lattice
        const bool ahead = more && !last_row;
        cp16_if(&ring.src[(s + 2) & 3][lane], src2, ahead);
        cp16_if(&ring.tgt[(s + 1) & 1][lane], tgt_r + wpr, ahead);
        cp_commit();
        cp_wait_all_but_last();
        const uint4 up = ring.src[(s + 3) & 3][lane];
        const uint4 cur = ring.src[s & 3][lane];
        const uint4 dn = ring.src[(s + 1) & 3][lane];
        const uint4 tg = ring.tgt[s & 1][lane];
        const uint32_t prev = __shfl_sync(0xffffffffu, cur.w, left_lane);
        const uint32_t next = __shfl_sync(0xffffffffu, cur.x, right_lane);
        uint4 sd;  // side words as 32-bit halves
        if (((r + colour) & 1) == 0) {  // left neighbour word: shift up one spin
            sd.x = __funnelshift_l(prev, cur.x, 4);
            sd.y = __funnelshift_l(cur.x, cur.y, 4);
            sd.z = __funnelshift_l(cur.y, cur.z, 4);
            sd.w = __funnelshift_l(cur.z, cur.w, 4);
        } else {  // right neighbour word: shift down one spin
            sd.x = __funnelshift_r(cur.x, cur.y, 4);
            sd.y = __funnelshift_r(cur.y, cur.z, 4);
            sd.z = __funnelshift_r(cur.z, cur.w, 4);
            sd.w = __funnelshift_r(cur.w, next, 4);
        }
        uint32_t dacc = 0;
        uint4 ns;
        ns.x = update_half<OBS, false>(tg.x, up.x + dn.x + cur.x, sd.x, q, stream, dc, p.rk, dacc);
        ns.y = update_half<OBS, false>(tg.y, up.y + dn.y + cur.y, sd.y, q | 2, stream, dc, p.rk, dacc);
        ns.z = update_half<OBS, false>(tg.z, up.z + dn.z + cur.z, sd.z, q | 4, stream, dc, p.rk, dacc);
        ns.w = update_half<OBS, false>(tg.w, up.w + dn.w + cur.w, sd.w, q | 6, stream, dc, p.rk, dacc);
        *reinterpret_cast<uint4 *>(tgt_r) = ns;
        if (OBS) {
            const uint32_t n8 = ns.x + ns.y + ns.z + ns.w + cur.x + cur.y + cur.z + cur.w;
            const uint32_t sb = (n8 & 0x0F0F0F0Fu) + ((n8 >> 4) & 0x0F0F0F0Fu);
            ones += (sb * 0x01010101u) >> 24;
            dsum += (dacc * 0x01010101u) >> 24;
            nrows += 1;
        }
        ++r;
        tgt_r += wpr;
        q += qrow;
        src2 = r + 2 == L ? src : src2 + wpr;
        if (last_row) {
            march_flush<OBS>(p, lat, gmask, lpr, j, ones, dsum, nrows);
            ++li;
            r = 0;
            if (more) enter(s + 1);
        }
    }
    if (n > 0 && r != 0) march_flush<OBS>(p, lat, gmask, lpr, j, ones, dsum, nrows);
    cp_wait_all();
}

// One half-sweep of every lattice.  Each chunk carries a work weight wpt +
// kappa (its words plus a fixed per-chunk cost, kappa chosen by the
// autotuner); warp gw owns the contiguous chunks whose starting weight lies in
// [gw * W / nw, (gw + 1) * W / nw) of the total W.  Observables are flushed
// with one pair of atomics whenever the warp moves to another lattice.
template <bool OBS>
__device__ void batch_half(const BatchParams &p, int colour, uint64_t t, MarchRing &ring)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto chunk_at = [&](int64_t w) -> int64_t {
        if (w >= p.total_weight) return p.n_chunks;
        int g = 0;
        while (g + 1 < p.n_groups && p.g[g + 1].weight_begin <= w) ++g;
        const int64_t per = p.g[g].weight;
        return p.g[g].chunk_begin + (w - p.g[g].weight_begin + per - 1) / per;
    };
    const int64_t cb = chunk_at(gw * p.total_weight / nw), ce = chunk_at((gw + 1) * p.total_weight / nw);
    const uint64_t *src = colour == 0 ? p.white : p.black;
    uint64_t *tgt = colour == 0 ? p.black : p.white;
    DrawCtx dc{(uint32_t)t, counter_word3(colour, kPurposeMetropolis, t), 0u, 0u, 0u};

    int gi = 0;
    int64_t cur_lat = -1;
    uint32_t ones = 0, dsum = 0, nitems = 0;
    auto flush = [&]() {
        if (OBS && cur_lat >= 0) {
            long long a = ones, b = dsum, c = nitems;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, off);
                b += __shfl_xor_sync(0xffffffffu, b, off);
                c += __shfl_xor_sync(0xffffffffu, c, off);
            }
            if (lane == 0) {
                // c white sites and c black centres were counted, a of them up;
                // each white site adds 4 - 2d over its 4 bonds
                atomicAdd(reinterpret_cast<unsigned long long *>(p.acc + 2 * cur_lat),
                          (unsigned long long)(2 * a - 2 * c));
                atomicAdd(reinterpret_cast<unsigned long long *>(p.acc + 2 * cur_lat + 1),
                          (unsigned long long)(4 * c - 2 * b));
            }
        }
        ones = dsum = nitems = 0;
    };
    // this lane's item as (lattice li of the group, row r, item q of the row):
    // derived by division at a group's first chunk, then stepped 32 items per
    // chunk (a warp's chunks are consecutive) with one carry into the row and
    // at most one wrap into the next lattice
    int cur_g = -1;
    int64_t li = 0;
    int r = 0, q = 0, dr = 0, dq = 0;
    for (int64_t c = cb; c < ce; ++c) {
        while (gi + 1 < p.n_groups && c >= p.g[gi + 1].chunk_begin) ++gi;
        const BatchGroup &G = p.g[gi];
        if (G.march) {
            // this warp's chunks of the group, all at once (warp-uniform)
            const int64_t gend = gi + 1 < p.n_groups ? p.g[gi + 1].chunk_begin : p.n_chunks;
            const int64_t c1 = ce < gend ? ce : gend;
            flush();
            cur_lat = -1;
            march_rows<OBS>(p, G, c - G.chunk_begin, c1 - G.chunk_begin, colour, t, ring);
            c = c1 - 1;
            cur_g = -1;
            continue;
        }
        if (gi != cur_g) {
            cur_g = gi;
            const int64_t item = (c - G.chunk_begin) * 32 + lane;
            li = item / G.items;
            const int64_t within = item - li * G.items;
            r = (int)(within / G.gpr);
            q = (int)(within - (int64_t)r * G.gpr);
            dr = 32 / G.gpr;
            dq = 32 - dr * G.gpr;
        } else {
            q += dq;
            r += dr;
            if (q >= G.gpr) {
                q -= G.gpr;
                ++r;
            }
            if (r >= G.L) {
                r -= G.L;
                ++li;
            }
        }
        const int64_t lat = G.first + li;
        if (lat != cur_lat) {
            flush();
            cur_lat = lat;
        }
        const int w0 = q * G.wpt;
        const int64_t base = G.word_base + li * (int64_t)G.L * G.wpr;
        const int slot = p.slot_of[lat];
        dc.T3 = p.thr[2 * slot];
        dc.T4 = p.thr[2 * slot + 1];
        const uint32_t stream = (uint32_t)lat;
        if (G.wpt == 4)
            sweep_item<4, OBS>(src + base, tgt + base, G.L, G.wpr, r, w0, colour, stream, dc, p.rk, ones, dsum);
        else if (G.wpt == 2)
            sweep_item<2, OBS>(src + base, tgt + base, G.L, G.wpr, r, w0, colour, stream, dc, p.rk, ones, dsum);
        else
            sweep_item<1, OBS>(src + base, tgt + base, G.L, G.wpr, r, w0, colour, stream, dc, p.rk, ones, dsum);
        // per item: 16 * wpt white sites (4 bonds each) and as many black centres
        nitems += 16 * G.wpt;
    }
    flush();
}

// Record and exchange: warp gw handles ladders gw, gw + nw, ...
__device__ void batch_exchange(const BatchParams &p, uint64_t t)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t e = (int64_t)((t + 1) / (uint64_t)p.record_every) - 1;
    for (int64_t l = gw; l < p.n_ladders; l += nw) {
        int32_t *at = p.lattice_at + l * p.S;
        if (p.trace != nullptr) {
            long long *row = p.trace + 2 * ((e - p.event_first) * p.n + l * p.S);
            for (int k = lane; k < p.S; k += 32) {
                const int32_t x = at[k];
                row[2 * k] = p.acc[2 * x];
                row[2 * k + 1] = p.acc[2 * x + 1];
            }
        }
        __syncwarp();
        if (p.swaps) {
            for (int k = (int)(e & 1) + 2 * lane; k + 1 < p.S; k += 64) {
                const int32_t a = at[k], b = at[k + 1];
                const long long D = p.acc[2 * a + 1] - p.acc[2 * b + 1];  // E_b - E_a
                bool swap = D >= 0;
                if (!swap) {
                    if ((D & 3) != 0) atomicCAS(p.err, 0, (int)ISING_EINVAL);
                    const int64_t m = -D;
                    const uint64_t TS = m < p.swap_len[k] ? p.swap_tab[p.swap_off[k] + m] : 0ull;
                    const uint32_t site = (uint32_t)k;
                    const uint4 u4 = philox(site >> 2, (uint32_t)l, (uint32_t)t,
                                            counter_word3(0, kPurposeExchange, t), p.rk);
                    const uint32_t w = (site & 3) == 0 ? u4.x : (site & 3) == 1 ? u4.y : (site & 3) == 2 ? u4.z : u4.w;
                    swap = (uint64_t)w < TS;
                }
                if (swap) {
                    at[k] = b;
                    at[k + 1] = a;
                    p.slot_of[a] = k + 1;
                    p.slot_of[b] = k;
                }
            }
        }
        __syncwarp();
        for (int k = lane; k < p.S; k += 32) {
            const int32_t x = at[k];
            p.acc[2 * x] = 0;
            p.acc[2 * x + 1] = 0;
        }
    }
}

// One 512-thread block per SM may use up to 128 registers: the march path's
// Philox blocks then stay in flight together (measured: 127 registers, 1285
// flips/ns on the replica-exchange batch, against 1216 at the compiler's own
// choice of 95 and 1236 at 64 with two blocks per SM).
__global__ void __launch_bounds__(512, 1) batch_kernel(const __grid_constant__ BatchParams p)
{
    // one MarchRing per warp (dynamic shared memory)
    extern __shared__ __align__(16) unsigned char batch_smem[];
    MarchRing &ring = reinterpret_cast<MarchRing *>(batch_smem)[threadIdx.x >> 5];
    for (int64_t s = 0; s < p.n_sweeps; ++s) {
        const uint64_t t = p.t0 + (uint64_t)s;
        const bool rec = p.record_every > 0 && (t + 1) % (uint64_t)p.record_every == 0;
        batch_half<false>(p, 0, t, ring);
        if (!grid_sync(p)) return;
        if (rec)
            batch_half<true>(p, 1, t, ring);
        else
            batch_half<false>(p, 1, t, ring);
        if (!grid_sync(p)) return;
        if (rec) {
            batch_exchange(p, t);
            if (!grid_sync(p)) return;
        }
    }
}

// Initial state: thread per word; lattice i draws in stream i (purpose 1, t = 0).
__global__ void batch_init_kernel(const __grid_constant__ BatchParams p, int mode)
{
    int64_t total = 0;
    for (int gi = 0; gi < p.n_groups; ++gi) total += p.g[gi].count * (int64_t)p.g[gi].L * p.g[gi].wpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int gi = 0;
        int64_t off = idx;
        while (off >= p.g[gi].count * (int64_t)p.g[gi].L * p.g[gi].wpr) {
            off -= p.g[gi].count * (int64_t)p.g[gi].L * p.g[gi].wpr;
            ++gi;
        }
        const BatchGroup &G = p.g[gi];
        const int64_t per = (int64_t)G.L * G.wpr;
        const int64_t li = off / per, w_in = off - li * per;
        const int64_t r = w_in / G.wpr, w = w_in - r * G.wpr;
        const uint32_t stream = (uint32_t)(G.first + li);
        const int64_t word = G.word_base + off;
        for (int colour = 0; colour < 2; ++colour) {
            uint64_t v = 0;
            if (mode == 1) {
                v = 0x1111111111111111ull;
            } else if (mode == 0) {
                const uint64_t q0 = (uint64_t)r * (uint64_t)(G.L / 8) + 4 * (uint64_t)w;
                const uint32_t c3 = counter_word3(colour, kPurposeInit, 0);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint4 u = philox((uint32_t)(q0 + b), (uint32_t)((q0 + b) >> 32) + stream, 0u, c3, p.rk);
                    const int sh = 16 * b;
                    v |= ((uint64_t)(u.x < 0x80000000u) << sh) | ((uint64_t)(u.y < 0x80000000u) << (sh + 4)) |
                         ((uint64_t)(u.z < 0x80000000u) << (sh + 8)) | ((uint64_t)(u.w < 0x80000000u) << (sh + 12));
                }
            }
            (colour == 0 ? p.black : p.white)[word] = v;
        }
    }
}

// Identity slot assignment and cleared accumulators.
__global__ void batch_reset_kernel(const __grid_constant__ BatchParams p)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
        p.slot_of[i] = (int32_t)(i % p.S);
        p.lattice_at[i] = (int32_t)i;
        p.acc[2 * i] = 0;
        p.acc[2 * i + 1] = 0;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace ising

// ---------------------------------------------------------------------------
// Host side: the handle, the workspace layout, graph capture and autotuning.
// ---------------------------------------------------------------------------
struct ising_batch {
    int64_t n = 0;
    int32_t S = 0;
    std::vector<int64_t> L, word_off;
    std::vector<double> beta;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t plane_words = 0;
    // workspace offsets
    size_t o_black, o_white, o_slot, o_at, o_thr, o_soff, o_slen, o_stab, o_acc, o_bar, o_tune, total;
    std::vector<int64_t> swap_len;
    int32_t threads = 512;
    int32_t wpt_max = 4;
    int32_t kappa = 4;
    int device = 0;
    // captured graph of the persistent launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    int32_t graph_threads = 0, graph_blocks = 0;
};

namespace ising {
namespace {

thread_local char g_batch_error[256] = "";

int bfail(int status, const char *msg)
{
    snprintf(g_batch_error, sizeof(g_batch_error), "%s", msg);
    return status;
}

// Exchange threshold tables: for slot pair (k, k+1), entry m (m = -D >= 0) is
// floor(2^32 exp(-(beta[k+1] - beta[k]) * m)), 2^32 when exp(...) >= 1, up to
// the first zero.  Only multiples of 4 are ever read; the table is indexed by
// m itself for clarity.
void swap_tables(const std::vector<double> &beta, std::vector<int64_t> &len, std::vector<uint64_t> *tab)
{
    const int S = (int)beta.size();
    len.assign(S > 1 ? S - 1 : 0, 0);
    for (int k = 0; k + 1 < S; ++k) {
        int64_t m = 0;
        for (;; ++m) {
            const double x = (beta[k + 1] - beta[k]) * (double)m;
            const double pr = std::exp(-x);
            const uint64_t T = pr >= 1.0 ? (uint64_t(1) << 32) : (uint64_t)std::floor(std::ldexp(pr, 32));
            if (tab) tab->push_back(T);
            if (T == 0) break;
            if (m > (int64_t(1) << 24)) break;  // guarded by the minimum spacing check
        }
        len[k] = m + 1;
    }
}

int layout(ising_batch_t *b)
{
    b->word_off.assign(b->n + 1, 0);
    for (int64_t i = 0; i < b->n; ++i) b->word_off[i + 1] = b->word_off[i] + b->L[i] * (b->L[i] / 32);
    b->plane_words = (size_t)b->word_off[b->n];
    swap_tables(b->beta, b->swap_len, nullptr);
    size_t ntab = 0;
    for (int64_t v : b->swap_len) ntab += (size_t)v;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    b->o_black = take(b->plane_words * 8);
    b->o_white = take(b->plane_words * 8);
    b->o_slot = take((size_t)b->n * 4);
    b->o_at = take((size_t)b->n * 4);
    b->o_thr = take((size_t)b->S * 8);
    b->o_soff = take((size_t)std::max(1, b->S - 1) * 8);
    b->o_slen = take((size_t)std::max(1, b->S - 1) * 8);
    b->o_stab = take(std::max<size_t>(1, ntab) * 8);
    b->o_acc = take((size_t)b->n * 16);
    b->o_bar = take(64);
    b->o_tune = take(2 * b->plane_words * 8);
    b->total = o;
    return ISING_OK;
}

int build_groups(const ising_batch_t *b, int wpt_max, int kappa, BatchParams &p)
{
    int ng = 0;
    int64_t chunk = 0, weight = 0;
    for (int64_t i = 0; i < b->n;) {
        int64_t j = i;
        while (j < b->n && b->L[j] == b->L[i]) ++j;
        if (ng == kMaxGroups) return bfail(ISING_EINVAL, "too many runs of equal lattice size (max 16)");
        BatchGroup &G = p.g[ng++];
        G.first = i;
        G.count = j - i;
        G.word_base = b->word_off[i];
        G.L = (int32_t)b->L[i];
        G.wpr = G.L / 32;
        // marching pays from 128 up (64: one lane per row, 1239 against 1285
        // flips/ns on the replica-exchange batch; starting at 256: 1206)
        G.march = (G.L & (G.L - 1)) == 0 && G.L >= kMarchMinL && G.L <= 2048;
        G.wpt = 1;
        if (G.march) {
            G.wpt = 2;  // 16 bytes of a row per lane
        } else {
            for (int w : {4, 2}) {
                if (w <= wpt_max && G.wpr % w == 0) {
                    G.wpt = w;
                    break;
                }
            }
        }
        G.gpr = G.wpr / G.wpt;
        G.items = (int64_t)G.L * G.gpr;
        G.chunk_begin = chunk;
        G.weight = G.wpt + kappa;
        G.weight_begin = weight;
        chunk += G.count * G.items / 32;
        weight += G.count * G.items / 32 * G.weight;
        i = j;
    }
    p.n_groups = ng;
    p.n_chunks = chunk;
    p.plane_words = b->word_off[b->n];
    p.total_weight = weight;
    return ISING_OK;
}

BatchParams base_params(const ising_batch_t *b)
{
    BatchParams p;
    memset(&p, 0, sizeof(p));
    p.black = (uint64_t *)(b->ws + b->o_black);
    p.white = (uint64_t *)(b->ws + b->o_white);
    p.S = b->S;
    p.n = b->n;
    p.n_ladders = b->n / b->S;
    p.slot_of = (int32_t *)(b->ws + b->o_slot);
    p.lattice_at = (int32_t *)(b->ws + b->o_at);
    p.thr = (const uint32_t *)(b->ws + b->o_thr);
    p.swap_off = (const int64_t *)(b->ws + b->o_soff);
    p.swap_len = (const int64_t *)(b->ws + b->o_slen);
    p.swap_tab = (const uint64_t *)(b->ws + b->o_stab);
    p.acc = (long long *)(b->ws + b->o_acc);
    p.bar = (unsigned *)(b->ws + b->o_bar);
    p.err = (int *)(b->ws + b->o_bar + 16);
    return p;
}

// Dynamic shared memory of a launch: one MarchRing per warp.
size_t smem_for(int threads) { return (size_t)(threads / 32) * sizeof(MarchRing); }

int blocks_for(int threads, int *blocks)
{
    DeviceInfo info{1};
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    // allow the largest ring (16 warps) beside the kernel's static shared memory
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(512));
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, threads, smem_for(threads));
    if (e != cudaSuccess || per_sm < 1) return bfail(ISING_ECUDA, "batch kernel does not fit on an SM");
    *blocks = info.sm_count * per_sm;
    return ISING_OK;
}

cudaError_t launch_coop(const BatchParams &p, int blocks, int threads, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem_for(threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel, p);
}

}  // namespace
}  // namespace ising

using namespace ising;

extern "C" {

ISING_API const char *ising_batch_last_error(void) { return g_batch_error; }

static int check_batch_args(int64_t n, const int64_t *L, int32_t S, const double *beta)
{
    if (n <= 0 || L == nullptr || beta == nullptr) return bfail(ISING_EINVAL, "empty batch or NULL arrays");
    if (S <= 0 || n % S != 0) return bfail(ISING_EINVAL, "the batch size must be a multiple of the ladder size");
    for (int64_t i = 0; i < n; ++i)
        if (L[i] < 32 || L[i] % 32 != 0 || L[i] > 65536)
            return bfail(ISING_EINVAL, "every side must be a multiple of 32 in [32, 65536]");
    for (int64_t l = 0; l < n / S; ++l)
        for (int32_t k = 1; k < S; ++k)
            if (L[l * S + k] != L[l * S]) return bfail(ISING_EINVAL, "lattices of one ladder must have equal sides");
    for (int32_t k = 0; k < S; ++k) {
        if (!std::isfinite(beta[k]) || beta[k] < 0.0) return bfail(ISING_EINVAL, "betas must be finite and >= 0");
        if (k > 0 && !(beta[k] - beta[k - 1] >= 1e-4))
            return bfail(ISING_EINVAL, "betas must increase by at least 1e-4");
    }
    if (beta[0] <= 0.0) return bfail(ISING_EINVAL, "beta = 0 is not supported in a batch");
    // The batched decision compares each draw with T3 and T4 as 32-bit words
    // (flip iff d >= [u >= T3] + [u >= T4]); a threshold of 2^32 (p = 1, the
    // Metropolis rule of Sec. 2 flipping always) has no 32-bit form there.
    // exp(-4 beta) rounds to 1 in FP64 for beta below about 1.4e-17, so such
    // betas are refused rather than run with a truncated table.
    for (int32_t k = 0; k < S; ++k) {
        uint64_t T[5];
        if (ising_thresholds(beta[k], T) != ISING_OK) return bfail(ISING_EINVAL, "bad beta");
        if (T[3] >= (uint64_t(1) << 32) || T[4] >= (uint64_t(1) << 32))
            return bfail(ISING_EINVAL, "beta too small for a batch: exp(-4 beta) rounds to 1 (use beta >= 1e-16)");
    }
    return ISING_OK;
}

ISING_API int ising_batch_bytes(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta, size_t *bytes)
{
    int rc = check_batch_args(n, L, ladder_size, beta);
    if (rc) return rc;
    if (bytes == nullptr) return bfail(ISING_EINVAL, "bytes is NULL");
    ising_batch_t tmp;
    tmp.n = n;
    tmp.S = ladder_size;
    tmp.L.assign(L, L + n);
    tmp.beta.assign(beta, beta + ladder_size);
    layout(&tmp);
    *bytes = tmp.total;
    return ISING_OK;
}

ISING_API int ising_batch_create(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta,
                                 void *workspace_dev, size_t workspace_bytes, ising_batch_t **out)
{
    int rc = check_batch_args(n, L, ladder_size, beta);
    if (rc) return rc;
    if (out == nullptr || workspace_dev == nullptr) return bfail(ISING_EINVAL, "NULL workspace or output");
    if ((uintptr_t)workspace_dev % 256 != 0) return bfail(ISING_EINVAL, "workspace must be 256-byte aligned");
    ising_batch_t *b = new (std::nothrow) ising_batch_t;
    if (!b) return bfail(ISING_EINVAL, "out of host memory");
    b->n = n;
    b->S = ladder_size;
    b->L.assign(L, L + n);
    b->beta.assign(beta, beta + ladder_size);
    layout(b);
    if (workspace_bytes < b->total) {
        delete b;
        return bfail(ISING_EINVAL, "workspace is smaller than ising_batch_bytes");
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, workspace_dev) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        delete b;
        return bfail(ISING_EINVAL, "workspace is not device memory");
    }
    cudaGetDevice(&b->device);
    b->ws = (char *)workspace_dev;
    b->ws_bytes = workspace_bytes;
    // tables: thresholds per slot, exchange tables
    std::vector<uint32_t> thr(2 * (size_t)ladder_size);
    for (int k = 0; k < ladder_size; ++k) {
        uint64_t T[5];
        ising_thresholds(beta[k], T);
        thr[2 * k] = (uint32_t)T[3];
        thr[2 * k + 1] = (uint32_t)T[4];
    }
    std::vector<uint64_t> tab;
    std::vector<int64_t> len;
    swap_tables(b->beta, len, &tab);
    std::vector<int64_t> off(len.size());
    int64_t acc_off = 0;
    for (size_t k = 0; k < len.size(); ++k) {
        off[k] = acc_off;
        acc_off += len[k];
    }
    cudaError_t e = cudaMemset(b->ws + b->o_slot, 0, b->o_tune - b->o_slot);
    if (e == cudaSuccess) e = cudaMemcpy(b->ws + b->o_thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !len.empty())
        e = cudaMemcpy(b->ws + b->o_soff, off.data(), off.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !len.empty())
        e = cudaMemcpy(b->ws + b->o_slen, len.data(), len.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tab.empty())
        e = cudaMemcpy(b->ws + b->o_stab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete b;
        return bfail(ISING_ECUDA, cudaGetErrorString(e));
    }
    *out = b;
    return ISING_OK;
}

ISING_API int ising_batch_destroy(ising_batch_t *b)
{
    if (b == nullptr) return ISING_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return ISING_OK;
}

ISING_API int ising_batch_planes(const ising_batch_t *b, void **black_dev, void **white_dev, int64_t *word_offsets)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    if (black_dev) *black_dev = b->ws + b->o_black;
    if (white_dev) *white_dev = b->ws + b->o_white;
    if (word_offsets) memcpy(word_offsets, b->word_off.data(), (size_t)(b->n + 1) * 8);
    return ISING_OK;
}

ISING_API int ising_batch_state(const ising_batch_t *b, int32_t **slot_of_dev, int32_t **lattice_at_dev)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    if (slot_of_dev) *slot_of_dev = (int32_t *)(b->ws + b->o_slot);
    if (lattice_at_dev) *lattice_at_dev = (int32_t *)(b->ws + b->o_at);
    return ISING_OK;
}

ISING_API int ising_batch_init(ising_batch_t *b, int32_t init, uint64_t seed, ising_stream_t stream)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    if (init < ISING_INIT_RANDOM || init > ISING_INIT_DOWN) return bfail(ISING_EINVAL, "unknown init mode");
    BatchParams p = base_params(b);
    int rc = build_groups(b, b->wpt_max, b->kappa, p);
    if (rc) return rc;
    p.rk = make_round_keys(seed);
    cudaStream_t s = (cudaStream_t)stream;
    DeviceInfo info{1};
    device_info(&info);
    batch_init_kernel<<<info.sm_count * 4, 256, 0, s>>>(p, init);
    batch_reset_kernel<<<info.sm_count, 256, 0, s>>>(p);
    cudaError_t e = cudaMemsetAsync(b->ws + b->o_bar, 0, 64, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : bfail(ISING_ECUDA, cudaGetErrorString(e));
}

static int run_impl(ising_batch_t *b, uint64_t *black, uint64_t *white, int64_t n_sweeps, uint64_t seed,
                    uint64_t off, int32_t record_every, int32_t swaps, int64_t *trace, int32_t use_graph,
                    cudaStream_t s)
{
    BatchParams p = base_params(b);
    if (black) {
        p.black = black;
        p.white = white;
    }
    int rc = build_groups(b, b->wpt_max, b->kappa, p);
    if (rc) return rc;
    p.n_sweeps = n_sweeps;
    p.t0 = off;
    p.record_every = record_every;
    p.swaps = swaps;
    p.trace = (long long *)trace;
    p.event_first = record_every > 0 ? (int64_t)(off / (uint64_t)record_every) : 0;
    p.rk = make_round_keys(seed);
    p.timeout_cycles = (long long)4e9;  // ~2 s at 2 GHz
    int blocks = 0;
    rc = blocks_for(b->threads, &blocks);
    if (rc) return rc;
    p.expect_blocks = blocks;
    if (n_sweeps == 0) return ISING_OK;
    if (!use_graph) {
        cudaError_t e = launch_coop(p, blocks, b->threads, s);
        return e == cudaSuccess ? ISING_OK : bfail(ISING_ECUDA, cudaGetErrorString(e));
    }
    if (b->exec == nullptr || b->graph_threads != b->threads || b->graph_blocks != blocks) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = launch_coop(p, blocks, b->threads, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        size_t nn = 1;
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, &node, &nn);
        if (e != cudaSuccess || nn != 1) {
            if (g) cudaGraphDestroy(g);
            return bfail(ISING_ECUDA, "graph capture of the batch launch failed");
        }
        b->graph = g;
        b->node = node;
        b->graph_threads = b->threads;
        b->graph_blocks = blocks;
    }
    cudaKernelNodeParams kp = {};
    void *args[1] = {&p};
    kp.func = (void *)batch_kernel;
    kp.gridDim = dim3((unsigned)blocks);
    kp.blockDim = dim3((unsigned)b->threads);
    kp.sharedMemBytes = (unsigned)smem_for(b->threads);
    kp.kernelParams = args;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(b->exec, b->node, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? ISING_OK : bfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_batch_run(ising_batch_t *b, int64_t n_sweeps, uint64_t seed, uint64_t sweep_offset,
                              int32_t record_every, int32_t swaps, int64_t *trace_dev, int32_t use_graph,
                              ising_stream_t stream)
{
    if (b == nullptr || n_sweeps < 0 || record_every < 0) return bfail(ISING_EINVAL, "bad batch run arguments");
    if (swaps && record_every == 0) return bfail(ISING_EINVAL, "exchanges happen on record sweeps: set record_every");
    if (trace_dev != nullptr && record_every > 0) {
        const int64_t events = (int64_t)((sweep_offset + (uint64_t)n_sweeps) / (uint64_t)record_every) -
                               (int64_t)(sweep_offset / (uint64_t)record_every);
        if (events > 0 && check_device_range(trace_dev, (size_t)events * (size_t)b->n * 16, "trace") != ISING_OK)
            return bfail(ISING_EINVAL, "trace must be device memory of events x n x 2 int64");
    }
    return run_impl(b, nullptr, nullptr, n_sweeps, seed, sweep_offset, record_every, swaps, trace_dev, use_graph,
                    (cudaStream_t)stream);
}

ISING_API int ising_batch_check(ising_batch_t *b, ising_stream_t stream)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    int err = 0;
    e = cudaMemcpy(&err, b->ws + b->o_bar + 16, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    if (err != 0) {
        cudaMemset(b->ws + b->o_bar, 0, 64);
        return bfail(err, err == ISING_ETIMEOUT ? "a grid barrier wait timed out" : "device-side check failed");
    }
    return ISING_OK;
}

ISING_API int ising_batch_config(ising_batch_t *b, int32_t threads, int32_t words_per_thread)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    if ((threads != 256 && threads != 512) || (words_per_thread != 1 && words_per_thread != 2 && words_per_thread != 4))
        return bfail(ISING_EINVAL, "threads must be 256 or 512 and words_per_thread 1, 2 or 4");
    b->threads = threads;
    b->wpt_max = words_per_thread;
    return ISING_OK;
}

ISING_API int ising_batch_get_config(const ising_batch_t *b, int32_t *threads, int32_t *words_per_thread)
{
    if (b == nullptr) return bfail(ISING_EINVAL, "NULL batch");
    if (threads) *threads = b->threads;
    if (words_per_thread) *words_per_thread = b->wpt_max;
    return ISING_OK;
}

ISING_API int ising_batch_autotune(ising_batch_t *b, int64_t n_sweeps, ising_stream_t stream)
{
    if (b == nullptr || n_sweeps <= 0) return bfail(ISING_EINVAL, "bad autotune arguments");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *tb = (uint64_t *)(b->ws + b->o_tune);
    uint64_t *tw = tb + b->plane_words;
    cudaError_t e = cudaMemcpyAsync(tb, b->ws + b->o_black, b->plane_words * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tw, b->ws + b->o_white, b->plane_words * 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int32_t bt = b->threads, bw = b->wpt_max;
    b->kappa = 1 << 20;  // chunk-count split while tuning the shape
    const int32_t threads_c[2] = {256, 512}, wpt_c[3] = {1, 2, 4};
    for (int32_t th : threads_c) {
        for (int32_t w : wpt_c) {
            b->threads = th;
            b->wpt_max = w;
            // one untimed pass (warms caches and the occupancy query), then the timed one
            int rc = run_impl(b, tb, tw, 1, 0x5eed, 0, 0, 0, nullptr, 0, s);
            if (rc == ISING_OK) {
                cudaEventRecord(e0, s);
                rc = run_impl(b, tb, tw, n_sweeps, 0x5eed, 1, 0, 0, nullptr, 0, s);
                cudaEventRecord(e1, s);
            }
            if (rc != ISING_OK) continue;
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = th;
                bw = w;
            }
        }
    }
    b->threads = bt;
    b->wpt_max = bw;
    // then the per-chunk weight of the work split
    int32_t bk = b->kappa;
    for (int32_t kap : {0, 1, 2, 4, 8, 1 << 20}) {
        b->kappa = kap;
        int rc = run_impl(b, tb, tw, 1, 0x5eed, 0, 0, 0, nullptr, 0, s);
        if (rc == ISING_OK) {
            cudaEventRecord(e0, s);
            rc = run_impl(b, tb, tw, n_sweeps, 0x5eed, 1, 0, 0, nullptr, 0, s);
            cudaEventRecord(e1, s);
        }
        if (rc != ISING_OK) continue;
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bk = kap;
        }
    }
    b->kappa = bk;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best < 1e30f ? ISING_OK : bfail(ISING_ECUDA, "no autotune candidate ran");
}

// Self-test of the bounded barrier: one launch whose barrier waits for one
// block more than the grid has, so every wait runs out; the kernel must
// return and report ISING_ETIMEOUT through the batch's error flag.
ISING_API int ising_batch_barrier_selftest(ising_batch_t *b, int64_t timeout_cycles, ising_stream_t stream)
{
    if (b == nullptr || timeout_cycles <= 0) return bfail(ISING_EINVAL, "bad self-test arguments");
    BatchParams p = base_params(b);
    int rc = build_groups(b, b->wpt_max, b->kappa, p);
    if (rc) return rc;
    int blocks = 0;
    rc = blocks_for(b->threads, &blocks);
    if (rc) return rc;
    p.n_sweeps = 1;
    p.rk = make_round_keys(0);
    p.timeout_cycles = timeout_cycles;
    p.expect_blocks = blocks + 1;
    cudaStream_t s = (cudaStream_t)stream;
    // the run sweeps the tuning copy, not the lattices
    p.black = (uint64_t *)(b->ws + b->o_tune);
    p.white = p.black + b->plane_words;
    cudaError_t e = cudaMemsetAsync(b->ws + b->o_bar, 0, 64, s);
    if (e == cudaSuccess) e = launch_coop(p, blocks, b->threads, s);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    return ising_batch_check(b, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched run.
//
// For callers that must not allocate device memory themselves -- for example
// code running under another framework's memory manager, which owns the
// device budget and does not let plug-ins call cudaMalloc, or a latency-bound
// loop where an allocation could synchronise the device -- this entry point
// keeps the batch kernel's scratch (threshold tables, exchange tables,
// per-lattice accumulators, barrier words) in the fixed array below instead
// of a caller-provided workspace.  Every GPU that loads the library holds the
// array until the process exits.  Its address is looked up once per device
// (cudaGetSymbolAddress, with that device current) by the first call on the
// device.  All calls share the array, so calls that overlap on the GPU race;
// each call clears what must start at zero (accumulators, barrier words).
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[ISING_NOALLOC_SCRATCH_BYTES];

namespace ising {
namespace {

struct NoallocScratch {
    std::mutex mu;
    void *addr[64] = {};
};
NoallocScratch g_noalloc;

int noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return bfail(ISING_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc.mu);
    if (g_noalloc.addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return bfail(ISING_ECUDA, "cudaGetSymbolAddress of the scratch failed");
        g_noalloc.addr[dev] = p;
    }
    *out = g_noalloc.addr[dev];
    return ISING_OK;
}

}  // namespace
}  // namespace ising

extern "C" ISING_API int ising_batch_run_noalloc(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta,
                                                 void *black_dev, void *white_dev, int32_t *slot_of_dev,
                                                 int32_t *lattice_at_dev, int64_t n_sweeps, uint64_t seed,
                                                 uint64_t sweep_offset, int32_t record_every, int32_t swaps,
                                                 int64_t *trace_dev, ising_stream_t stream)
{
    int rc = check_batch_args(n, L, ladder_size, beta);
    if (rc) return rc;
    if (n_sweeps < 0 || record_every < 0) return bfail(ISING_EINVAL, "bad batch run arguments");
    if (swaps && record_every == 0) return bfail(ISING_EINVAL, "exchanges happen on record sweeps: set record_every");
    // host-side layout of the planes (the same as ising_batch_create's)
    ising_batch_t lay;
    lay.n = n;
    lay.S = ladder_size;
    lay.L.assign(L, L + n);
    lay.beta.assign(beta, beta + ladder_size);
    layout(&lay);
    // scratch layout inside the fixed array
    std::vector<uint32_t> thr(2 * (size_t)ladder_size);
    for (int k = 0; k < ladder_size; ++k) {
        uint64_t T[5];
        ising_thresholds(beta[k], T);
        thr[2 * k] = (uint32_t)T[3];
        thr[2 * k + 1] = (uint32_t)T[4];
    }
    std::vector<uint64_t> tab;
    std::vector<int64_t> len;
    swap_tables(lay.beta, len, &tab);
    std::vector<int64_t> off(len.size());
    int64_t o_acc_tab = 0;
    for (size_t k = 0; k < len.size(); ++k) {
        off[k] = o_acc_tab;
        o_acc_tab += len[k];
    }
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t s_thr = take(thr.size() * 4), s_off = take(std::max<size_t>(1, off.size()) * 8),
                 s_len = take(std::max<size_t>(1, len.size()) * 8), s_tab = take(std::max<size_t>(1, tab.size()) * 8),
                 s_acc = take((size_t)n * 16), s_bar = take(64);
    if (o > (size_t)ISING_NOALLOC_SCRATCH_BYTES) {
        char msg[160];
        snprintf(msg, sizeof(msg), "needs %zu bytes of scratch; the allocation-free entry point holds %zu",
                 o, (size_t)ISING_NOALLOC_SCRATCH_BYTES);
        return bfail(ISING_EINVAL, msg);
    }
    // the caller's buffers must be aligned for the kernel's accesses and cover
    // what the kernel touches
    if (((uintptr_t)black_dev | (uintptr_t)white_dev) % 16 != 0)
        return bfail(ISING_EINVAL, "black_dev and white_dev must be 16-byte aligned");
    if (((uintptr_t)slot_of_dev | (uintptr_t)lattice_at_dev) % 4 != 0)
        return bfail(ISING_EINVAL, "slot_of_dev and lattice_at_dev must be 4-byte aligned");
    if ((uintptr_t)trace_dev % 8 != 0) return bfail(ISING_EINVAL, "trace_dev must be 8-byte aligned");
    const size_t plane = lay.plane_words * 8;
    if (check_device_range(black_dev, plane, "black") || check_device_range(white_dev, plane, "white") ||
        check_device_range(slot_of_dev, (size_t)n * 4, "slot_of") ||
        check_device_range(lattice_at_dev, (size_t)n * 4, "lattice_at"))
        return bfail(ISING_EINVAL, "planes and slot arrays must be device memory of the batch's sizes");
    if (trace_dev != nullptr && record_every > 0) {
        const int64_t events = (int64_t)((sweep_offset + (uint64_t)n_sweeps) / (uint64_t)record_every) -
                               (int64_t)(sweep_offset / (uint64_t)record_every);
        if (events > 0 && check_device_range(trace_dev, (size_t)events * (size_t)n * 16, "trace") != ISING_OK)
            return bfail(ISING_EINVAL, "trace must be device memory of events x n x 2 int64");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // The kernel indexes its tables and the planes with the slot state, which
    // here is the caller's (ising_batch_run fills its own): read it back and
    // check that it is a valid state before anything is launched.
    {
        std::vector<int32_t> slot((size_t)n), at((size_t)n);
        cudaError_t ce = cudaMemcpyAsync(slot.data(), slot_of_dev, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(at.data(), lattice_at_dev, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(ce));
        for (int64_t i = 0; i < n; ++i)
            if (slot[(size_t)i] < 0 || slot[(size_t)i] >= ladder_size)
                return bfail(ISING_EINVAL, "slot_of holds a slot outside [0, ladder_size)");
        for (int64_t l = 0; l < n / ladder_size; ++l)
            for (int32_t k = 0; k < ladder_size; ++k) {
                const int64_t a = at[(size_t)(l * ladder_size + k)];
                if (a < l * ladder_size || a >= (l + 1) * ladder_size || slot[(size_t)a] != k)
                    return bfail(ISING_EINVAL, "lattice_at is not the inverse of slot_of within each ladder");
            }
    }
    void *scr = nullptr;
    rc = noalloc_scratch(&scr);
    if (rc) return rc;
    char *sc = (char *)scr;
    cudaError_t e = cudaMemcpyAsync(sc + s_thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !len.empty())
        e = cudaMemcpyAsync(sc + s_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !len.empty())
        e = cudaMemcpyAsync(sc + s_len, len.data(), len.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !tab.empty())
        e = cudaMemcpyAsync(sc + s_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc + s_acc, 0, (s_bar + 64) - s_acc, s);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));

    BatchParams p;
    memset(&p, 0, sizeof(p));
    p.black = (uint64_t *)black_dev;
    p.white = (uint64_t *)white_dev;
    rc = build_groups(&lay, 4, 4, p);
    if (rc) return rc;
    p.S = ladder_size;
    p.n = n;
    p.n_ladders = n / ladder_size;
    p.slot_of = slot_of_dev;
    p.lattice_at = lattice_at_dev;
    p.thr = (const uint32_t *)(sc + s_thr);
    p.swap_off = (const int64_t *)(sc + s_off);
    p.swap_len = (const int64_t *)(sc + s_len);
    p.swap_tab = (const uint64_t *)(sc + s_tab);
    p.acc = (long long *)(sc + s_acc);
    p.bar = (unsigned *)(sc + s_bar);
    p.err = (int *)(sc + s_bar + 16);
    p.n_sweeps = n_sweeps;
    p.t0 = sweep_offset;
    p.record_every = record_every;
    p.swaps = swaps;
    p.trace = (long long *)trace_dev;
    p.event_first = record_every > 0 ? (int64_t)(sweep_offset / (uint64_t)record_every) : 0;
    p.rk = make_round_keys(seed);
    p.timeout_cycles = (long long)4e9;
    int blocks = 0;
    rc = blocks_for(512, &blocks);
    if (rc) return rc;
    p.expect_blocks = blocks;
    if (n_sweeps > 0) {
        e = launch_coop(p, blocks, 512, s);
        if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    }
    // synchronous: report a timed-out barrier wait before returning
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    int err = 0;
    e = cudaMemcpy(&err, sc + s_bar + 16, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(ISING_ECUDA, cudaGetErrorString(e));
    if (err != 0) return bfail(err, err == ISING_ETIMEOUT ? "a grid barrier wait timed out" : "device-side check failed");
    return ISING_OK;
}
