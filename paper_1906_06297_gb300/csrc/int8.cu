// int8.cu -- kernels on the one-byte-per-spin lattice (Sec. 3.1 of the paper):
// two colour planes of L rows x L/2 int8 spins (+1 / -1), compacted along rows.
//
// The per-site update is the basic kernel of Fig. 2: the three vertically and
// horizontally aligned source sites (i-1, j), (i, j), (i+1, j) plus the side
// site (i, joff), where joff = j+1 for black on odd rows and white on even
// rows, j-1 otherwise (periodic), and an acceptance test equivalent to
// rand < exp(-2 beta nn s).  Here the random number is the site's keyed
// Philox draw and the test is the exact integer form u < T[a].
//
// Each thread owns one Philox block, i.e. 4 consecutive sites of the plane in
// row-major order (they may straddle a row end when L/2 is not a multiple
// of 4), so every block is computed exactly once.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ising {

namespace {

constexpr int kThreads = 256;

template <int COLOR, bool OBS>
__global__ void __launch_bounds__(kThreads) int8_sweep_kernel(const __grid_constant__ Int8SweepParams p)
{
    const int64_t nsites = p.L * p.half;
    long long sum_s = 0, sum_b = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p.nblk;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint4 u4 = philox((uint32_t)q, (uint32_t)((uint64_t)q >> 32), p.c2, p.c3, p.rk);
        const uint32_t us[4] = {u4.x, u4.y, u4.z, u4.w};
        const int64_t site0 = 4 * q;
        int64_t i = site0 / p.half;
        int64_t j = site0 - i * p.half;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (site0 + k < nsites) {
                const int64_t iu = i == 0 ? p.L - 1 : i - 1;
                const int64_t id = i + 1 == p.L ? 0 : i + 1;
                const int64_t jl = j == 0 ? p.half - 1 : j - 1;
                const int64_t jr = j + 1 == p.half ? 0 : j + 1;
                const bool odd = (i & 1) != 0;
                const int64_t joff = (COLOR == 0) ? (odd ? jr : jl) : (odd ? jl : jr);
                const int8_t *srow = p.src + i * p.stride;
                const int centre = srow[j];
                const int nn = p.src[iu * p.stride + j] + p.src[id * p.stride + j] + centre + srow[joff];
                int8_t *tp = p.tgt + i * p.stride + j;
                const int s = *tp;
                const int a = (4 + s * nn) >> 1;  // aligned neighbours
                const uint64_t u = us[k];
                const bool flip = a <= 2 || (a == 3 ? u < p.acc.T3_64 : u < p.acc.T4_64);
                const int ns = flip ? -s : s;
                if (flip) *tp = (int8_t)ns;
                if (OBS) {
                    sum_s += ns + centre;
                    sum_b += ns * nn;
                }
            }
            if (++j == p.half) {
                j = 0;
                ++i;
            }
        }
    }
    if (OBS) block_reduce_add2<kThreads>(sum_s, sum_b, p.obs);
}

__global__ void int8_init_kernel(int8_t *plane, int64_t L, int64_t stride, int mode, uint32_t c3,
                                 const __grid_constant__ RoundKeys rk)
{
    const int64_t half = L / 2, nsites = L * half, nblk = (nsites + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nblk;
         q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t us[4] = {0, 0, 0, 0};
        if (mode == 0) {
            const uint4 u4 = philox((uint32_t)q, (uint32_t)((uint64_t)q >> 32), 0u, c3, rk);
            us[0] = u4.x; us[1] = u4.y; us[2] = u4.z; us[3] = u4.w;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t site = 4 * q + k;
            if (site < nsites) {
                const int64_t i = site / half, j = site - i * half;
                int8_t v = mode == 1 ? 1 : (mode == 2 ? -1 : (us[k] < 0x80000000u ? 1 : -1));
                plane[i * stride + j] = v;
            }
        }
    }
}

// Thread per white site: s_w * (sum of its 4 black neighbours) visits every
// bond once; s_w + s_b(i, j) visits every site once.
__global__ void __launch_bounds__(256) int8_obs_kernel(const int8_t *black, const int8_t *white, int64_t L,
                                                       int64_t stride, long long *out)
{
    const int64_t half = L / 2, nsites = L * half;
    long long sum_s = 0, sum_b = 0;
    for (int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; site < nsites;
         site += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = site / half, j = site - i * half;
        const int64_t iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
        const int64_t joff = (i & 1) ? (j == 0 ? half - 1 : j - 1) : (j + 1 == half ? 0 : j + 1);
        const int centre = black[i * stride + j];
        const int nn = black[iu * stride + j] + black[id * stride + j] + centre + black[i * stride + joff];
        const int s = white[i * stride + j];
        sum_s += s + centre;
        sum_b += s * nn;
    }
    block_reduce_add2<256>(sum_s, sum_b, out);
}

unsigned grid_for(int64_t n, int threads, int per_sm)
{
    DeviceInfo info{1};
    device_info(&info);
    const int64_t cap = (int64_t)info.sm_count * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (n + threads - 1) / threads));
}

}  // namespace

cudaError_t int8_half_sweep(const Int8SweepParams &p, int colour, cudaStream_t s)
{
    const unsigned g = grid_for(p.nblk, kThreads, 8);
    const bool obs = p.obs != nullptr;
    if (colour == 0) {
        if (obs) int8_sweep_kernel<0, true><<<g, kThreads, 0, s>>>(p);
        else int8_sweep_kernel<0, false><<<g, kThreads, 0, s>>>(p);
    } else {
        if (obs) int8_sweep_kernel<1, true><<<g, kThreads, 0, s>>>(p);
        else int8_sweep_kernel<1, false><<<g, kThreads, 0, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t int8_init(int8_t *plane, int colour, int64_t L, int64_t stride, int mode, uint64_t seed,
                      cudaStream_t s)
{
    const RoundKeys rk = make_round_keys(seed);
    const int64_t nblk = (L * (L / 2) + 3) / 4;
    int8_init_kernel<<<grid_for(nblk, 256, 8), 256, 0, s>>>(plane, L, stride, mode,
                                                            counter_word3(colour, kPurposeInit, 0), rk);
    return cudaGetLastError();
}

cudaError_t int8_observables(const int8_t *black, const int8_t *white, int64_t L, int64_t stride, long long *out,
                             cudaStream_t s)
{
    int8_obs_kernel<<<grid_for(L * (L / 2), 256, 8), 256, 0, s>>>(black, white, L, stride, out);
    return cudaGetLastError();
}

}  // namespace ising
