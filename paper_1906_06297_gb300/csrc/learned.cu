// learned.cu -- the learned block-proposal move: a small convolutional network
// proposes which 8 x 8 block of a lattice to flip, and an exact
// Metropolis-Hastings test accepts or rejects the flip.  Not in the paper: a
// proposal move layered on its checkerboard sweep (Sec. 2, Sec. 3.3), which
// stays the fallback and the ergodic part of the chain.
//
// Chains.  C lattices of side L (multiple of 32; blocks of 8 x 8) in the
// batched MSC4 layout: lattice c's colour planes start at word c * L * L/32 of
// one black and one white buffer (as a batch of equal sides).
//
// Network (3 x 3 periodic cross-correlations, 32 channels; weights rounded to
// bfloat16 for every use, products accumulated in FP32):
//   a1 = gelu(conv(spins; W1, b1)), a2 = gelu(conv(a1; W2, b2)),
//   a3 = gelu(conv(a2; W3, b3)), z4 = conv(a3; W4, b4) (one channel),
//   logit of block b = mean of z4 over the block; q(b) = softmax(logits)_b.
// gelu(z) = z * Phi(z).  Parameters are one FP32 vector in the order
// W1[32][9], b1[32], W2[32][32][9], b2[32], W3[32][32][9], b3[32], W4[32][9], b4[1].
// Activations are NHWC FP32 (32 channels per pixel).  All reductions have a
// fixed order, so a forward pass is a deterministic function of the state.
//
// Move.  Block b is drawn by inverse CDF of q_x (purpose-3 draw, site 0, in
// the chain's stream) or uniformly; x' = x with block b flipped; the flip is
// accepted iff the purpose-3 draw of site 1 is below
// floor(2^32 min(1, exp(-beta dE + log q_x'(b) - log q_x(b)))), dE the exact
// integer energy change (twice the boundary bond sum).  Softmax sums run in
// block order in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/ising.h"
#include "common.cuh"
#include "launch.h"

namespace ising {

namespace {

constexpr int kCh = 32;
constexpr int kBlk = 8;
constexpr int kN1 = kCh * 9, kNb = kCh, kN2 = kCh * kCh * 9;
constexpr int kOffW1 = 0, kOffB1 = kN1, kOffW2 = kOffB1 + kNb, kOffB2 = kOffW2 + kN2, kOffW3 = kOffB2 + kNb,
              kOffB3 = kOffW3 + kN2, kOffW4 = kOffB3 + kNb, kOffB4 = kOffW4 + kN1, kParams = kOffB4 + 1;
constexpr int kThreads = 256;

__device__ __forceinline__ float bf16r(float x)
{
    // round to the nearest bfloat16, ties to even (finite inputs)
    uint32_t u = __float_as_uint(x);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(u);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct Chains {
    const uint64_t *black, *white;
    int L, wpr;
};

// Spin (+1/-1) at row y, column x of chain c, with block `flip` (or -1) negated.
__device__ __forceinline__ float spin_at(const Chains &ch, int64_t c, int y, int x, int flip)
{
    const int colour = (y + x) & 1;
    const int j = x >> 1;
    const uint64_t *plane = colour ? ch.white : ch.black;
    const uint64_t w = plane[c * (int64_t)ch.L * ch.wpr + (int64_t)y * ch.wpr + (j >> 4)];
    float s = ((w >> (4 * (j & 15))) & 1) ? 1.0f : -1.0f;
    if (flip >= 0) {
        const int nb = ch.L / kBlk;
        const int by = flip / nb, bx = flip - by * nb;
        if ((y >> 3) == by && (x >> 3) == bx) s = -s;
    }
    return s;
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
// Layer 1: thread per pixel.  z stored when z_out != nullptr.
__global__ void __launch_bounds__(kThreads) l1_kernel(Chains ch, int64_t C, const int32_t *flip, const float *params,
                                                      float *z_out, float *a_out)
{
    __shared__ float W[kN1], Bs[kCh];
    for (int i = threadIdx.x; i < kN1; i += blockDim.x) W[i] = bf16r(params[kOffW1 + i]);
    for (int i = threadIdx.x; i < kCh; i += blockDim.x) Bs[i] = bf16r(params[kOffB1 + i]);
    __syncthreads();
    const int L = ch.L;
    const int64_t npix = C * (int64_t)L * L;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ((int64_t)L * L);
        const int yx = (int)(p - c * (int64_t)L * L);
        const int y = yx / L, x = yx - y * L;
        const int fb = flip ? flip[c] : -1;
        float s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = (y + k / 3 - 1 + L) % L, xx = (x + k % 3 - 1 + L) % L;
            s[k] = spin_at(ch, c, yy, xx, fb);
        }
        float *zo = z_out ? z_out + p * kCh : nullptr;
        float *ao = a_out + p * kCh;
#pragma unroll 4
        for (int o = 0; o < kCh; ++o) {
            float z = Bs[o];
#pragma unroll
            for (int k = 0; k < 9; ++k) z = fmaf(W[o * 9 + k], s[k], z);
            if (zo) zo[o] = z;
            ao[o] = gelu(z);
        }
    }
}

// Layers 2 and 3: thread per pixel, 32 accumulators; weights in shared memory
// as Ws[k][i][o] so that a tap and input channel give 32 contiguous outputs.
__global__ void __launch_bounds__(kThreads) conv32_kernel(int L, int64_t C, const float *params, int w_off, int b_off,
                                                          const float *a_in, float *z_out, float *a_out)
{
    extern __shared__ float Ws[];  // 9 * 32 * 32
    __shared__ float Bs[kCh];
    for (int i = threadIdx.x; i < kN2; i += blockDim.x) {
        const int o = i / (kCh * 9), rem = i - o * kCh * 9, ci = rem / 9, k = rem - ci * 9;
        Ws[(k * kCh + ci) * kCh + o] = bf16r(params[w_off + i]);
    }
    for (int i = threadIdx.x; i < kCh; i += blockDim.x) Bs[i] = bf16r(params[b_off + i]);
    __syncthreads();
    const int64_t npix = C * (int64_t)L * L;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ((int64_t)L * L);
        const int yx = (int)(p - c * (int64_t)L * L);
        const int y = yx / L, x = yx - y * L;
        float acc[kCh];
#pragma unroll
        for (int o = 0; o < kCh; ++o) acc[o] = Bs[o];
        for (int k = 0; k < 9; ++k) {
            const int yy = (y + k / 3 - 1 + L) % L, xx = (x + k % 3 - 1 + L) % L;
            const float4 *src = reinterpret_cast<const float4 *>(a_in + ((c * L + yy) * (int64_t)L + xx) * kCh);
#pragma unroll
            for (int q = 0; q < kCh / 4; ++q) {
                const float4 v = src[q];
                const float in4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float *w = Ws + (k * kCh + 4 * q + r) * kCh;
#pragma unroll
                    for (int o = 0; o < kCh; ++o) acc[o] = fmaf(w[o], in4[r], acc[o]);
                }
            }
        }
        float *zo = z_out ? z_out + p * kCh : nullptr;
        float4 *ao = reinterpret_cast<float4 *>(a_out + p * kCh);
#pragma unroll
        for (int q = 0; q < kCh / 4; ++q) {
            if (zo) reinterpret_cast<float4 *>(zo)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            ao[q] = make_float4(gelu(acc[4 * q]), gelu(acc[4 * q + 1]), gelu(acc[4 * q + 2]), gelu(acc[4 * q + 3]));
        }
    }
}

// Layer 4 and the block mean: warp per (chain, block), two pixels per lane,
// lane sums in a fixed order then a fixed shuffle tree.
__global__ void __launch_bounds__(kThreads) l4_pool_kernel(int L, int64_t C, const float *params, const float *a3,
                                                           float *logits)
{
    __shared__ float W[kN1];
    __shared__ float b4;
    for (int i = threadIdx.x; i < kN1; i += blockDim.x) W[i] = bf16r(params[kOffW4 + i]);
    if (threadIdx.x == 0) b4 = bf16r(params[kOffB4]);
    __syncthreads();
    const int nb1 = L / kBlk, nb = nb1 * nb1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < C * nb; wi += nw) {
        const int64_t c = wi / nb;
        const int b = (int)(wi - c * nb), by = b / nb1, bx = b - by * nb1;
        float part = 0.0f;
        for (int e = 0; e < 2; ++e) {
            const int pix = lane + 32 * e;  // 0..63 within the block
            const int y = by * kBlk + pix / kBlk, x = bx * kBlk + pix % kBlk;
            float z = b4;
            for (int k = 0; k < 9; ++k) {
                const int yy = (y + k / 3 - 1 + L) % L, xx = (x + k % 3 - 1 + L) % L;
                const float *src = a3 + ((c * L + yy) * (int64_t)L + xx) * kCh;
#pragma unroll
                for (int i = 0; i < kCh; ++i) z = fmaf(W[i * 9 + k], src[i], z);
            }
            part += z;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) logits[c * nb + b] = part * (1.0f / (kBlk * kBlk));
    }
}

// ---------------------------------------------------------------------------
// Backward (uses z1..z3, a1..a3 stored by a training forward)
// ---------------------------------------------------------------------------
// dz3 = gelu'(z3) * sum_k W4[i][k] * d4(p - off_k),  d4(p) = dlogit(block of p) / 64.
__global__ void __launch_bounds__(kThreads) l4_bwd_data_kernel(int L, int64_t C, const float *params,
                                                               const float *dlogits, const float *z3, float *dz3)
{
    __shared__ float W[kN1];
    for (int i = threadIdx.x; i < kN1; i += blockDim.x) W[i] = bf16r(params[kOffW4 + i]);
    __syncthreads();
    const int nb1 = L / kBlk;
    const int64_t npix = C * (int64_t)L * L;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ((int64_t)L * L);
        const int yx = (int)(p - c * (int64_t)L * L);
        const int y = yx / L, x = yx - y * L;
        float d[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            // output pixel q = p - off_k used input p through tap k
            const int yy = (y - (k / 3 - 1) + L) % L, xx = (x - (k % 3 - 1) + L) % L;
            d[k] = dlogits[c * nb1 * nb1 + (yy / kBlk) * nb1 + xx / kBlk] * (1.0f / (kBlk * kBlk));
        }
        for (int i = 0; i < kCh; ++i) {
            float g = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) g = fmaf(W[i * 9 + k], d[k], g);
            dz3[p * kCh + i] = g * gelu_grad(z3[p * kCh + i]);
        }
    }
}

// dz_prev = gelu'(z_prev) * sum_{k, o} W[o][i][k] * dz(p - off_k)[o]; weights
// as Wt[k][o][i] (32 contiguous inputs per tap and output).
__global__ void __launch_bounds__(kThreads) conv32_bwd_data_kernel(int L, int64_t C, const float *params, int w_off,
                                                                   const float *dz, const float *z_prev, float *dz_prev)
{
    extern __shared__ float Wt[];
    for (int i = threadIdx.x; i < kN2; i += blockDim.x) {
        const int o = i / (kCh * 9), rem = i - o * kCh * 9, ci = rem / 9, k = rem - ci * 9;
        Wt[(k * kCh + o) * kCh + ci] = bf16r(params[w_off + i]);
    }
    __syncthreads();
    const int64_t npix = C * (int64_t)L * L;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ((int64_t)L * L);
        const int yx = (int)(p - c * (int64_t)L * L);
        const int y = yx / L, x = yx - y * L;
        float acc[kCh];
#pragma unroll
        for (int i = 0; i < kCh; ++i) acc[i] = 0.0f;
        for (int k = 0; k < 9; ++k) {
            const int yy = (y - (k / 3 - 1) + L) % L, xx = (x - (k % 3 - 1) + L) % L;
            const float4 *src = reinterpret_cast<const float4 *>(dz + ((c * L + yy) * (int64_t)L + xx) * kCh);
#pragma unroll
            for (int q = 0; q < kCh / 4; ++q) {
                const float4 v = src[q];
                const float g4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float *w = Wt + (k * kCh + 4 * q + r) * kCh;
#pragma unroll
                    for (int i = 0; i < kCh; ++i) acc[i] = fmaf(w[i], g4[r], acc[i]);
                }
            }
        }
        const float *zp = z_prev + p * kCh;
        float *out = dz_prev + p * kCh;
#pragma unroll
        for (int i = 0; i < kCh; ++i) out[i] = acc[i] * gelu_grad(zp[i]);
    }
}

// Weight gradients as per-CTA partial sums (fixed order).  The pixels are cut
// into tiles of 8 rows x 32 columns of one chain; CTA j handles tiles j,
// j + gridDim.x, ... in order.  A tile's output gradients dz (and the layer's
// input a, with a one-pixel halo) are staged in shared memory; thread (oq, iq)
// of 16 x 16 accumulates the 2 x 2 (output, input) channel pairs 2 oq + {0, 1}
// x 2 iq + {0, 1} for all 9 taps, and threads with iq = 0 the bias sums.
// partial[cta][e]: e = (o * CIN + i) * 9 + k for weights, then the biases.
constexpr int kTy = 8, kTx = 32;

template <int CIN, int COUT>
__device__ __forceinline__ void wgrad_stage(const Chains &ch, const float *a_prev, const float *dz,
                                            const float *dlogits, int64_t c, int y0, int x0, float *sa, float *sd)
{
    const int L = ch.L, nb1 = L / kBlk;
    // input tile with halo: (kTy + 2) x (kTx + 2) pixels x CIN channels
    for (int e = threadIdx.x; e < (kTy + 2) * (kTx + 2) * CIN; e += blockDim.x) {
        const int pix = e / CIN, i = e - pix * CIN;
        const int ty = pix / (kTx + 2), tx = pix - ty * (kTx + 2);
        int y = y0 + ty - 1, x = x0 + tx - 1;
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        x = x < 0 ? x + L : (x >= L ? x - L : x);
        sa[e] = CIN == 1 ? spin_at(ch, c, y, x, -1) : a_prev[((c * L + y) * (int64_t)L + x) * CIN + i];
    }
    for (int e = threadIdx.x; e < kTy * kTx * COUT; e += blockDim.x) {
        const int pix = e / COUT, o = e - pix * COUT;
        const int y = y0 + pix / kTx, x = x0 + pix % kTx;
        sd[e] = COUT == 1 ? dlogits[c * nb1 * nb1 + (y / kBlk) * nb1 + x / kBlk] * (1.0f / (kBlk * kBlk))
                          : dz[((c * L + y) * (int64_t)L + x) * COUT + o];
    }
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_kernel(Chains ch, int64_t C, const float *a_prev, const float *dz,
                                                    const float *dlogits, float *partial)
{
    extern __shared__ float smem[];
    float *sa = smem;                                 // (kTy+2) (kTx+2) CIN
    float *sd = smem + (kTy + 2) * (kTx + 2) * CIN;   // kTy kTx COUT
    constexpr int NE = COUT * CIN * 9 + COUT;
    const int L = ch.L;
    const int tiles_x = L / kTx, tiles_y = L / kTy;
    const int64_t n_tiles = C * tiles_x * tiles_y;
    // thread roles: oq, iq in 0..15 cover output / input channel pairs; for
    // CIN == 1 or COUT == 1 the unused index collapses
    constexpr int OQ = COUT == 1 ? 1 : COUT / 2, IQ = CIN == 1 ? 1 : CIN / 2;
    constexpr int OPT = COUT == 1 ? 1 : 2, IPT = CIN == 1 ? 1 : 2;
    const int role = threadIdx.x;
    const bool active = role < OQ * IQ;
    const int oq = active ? role / IQ : 0, iq = active ? role - (role / IQ) * IQ : 0;
    float acc[OPT][IPT][9];
    float bacc[OPT];
#pragma unroll
    for (int a = 0; a < OPT; ++a) {
        bacc[a] = 0.0f;
#pragma unroll
        for (int b = 0; b < IPT; ++b)
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[a][b][k] = 0.0f;
    }
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t c = tile / (tiles_x * tiles_y);
        const int rem = (int)(tile - c * tiles_x * tiles_y);
        const int y0 = (rem / tiles_x) * kTy, x0 = (rem % tiles_x) * kTx;
        __syncthreads();
        wgrad_stage<CIN, COUT>(ch, a_prev, dz, dlogits, c, y0, x0, sa, sd);
        __syncthreads();
        if (active) {
            for (int pix = 0; pix < kTy * kTx; ++pix) {
                const int ty = pix / kTx, tx = pix - ty * kTx;
                float g[OPT];
#pragma unroll
                for (int a = 0; a < OPT; ++a) g[a] = sd[pix * COUT + OPT * oq + a];
#pragma unroll
                for (int a = 0; a < OPT; ++a) bacc[a] += g[a];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int hp = (ty + k / 3) * (kTx + 2) + (tx + k % 3);
#pragma unroll
                    for (int b = 0; b < IPT; ++b) {
                        const float av = sa[hp * CIN + IPT * iq + b];
#pragma unroll
                        for (int a = 0; a < OPT; ++a) acc[a][b][k] = fmaf(g[a], av, acc[a][b][k]);
                    }
                }
            }
        }
    }
    if (active) {
        float *out = partial + (int64_t)blockIdx.x * NE;
#pragma unroll
        for (int a = 0; a < OPT; ++a)
#pragma unroll
            for (int b = 0; b < IPT; ++b)
#pragma unroll
                for (int k = 0; k < 9; ++k) out[((OPT * oq + a) * CIN + IPT * iq + b) * 9 + k] = acc[a][b][k];
        if (iq == 0)
#pragma unroll
            for (int a = 0; a < OPT; ++a) out[COUT * CIN * 9 + OPT * oq + a] = bacc[a];
    }
}

// grad[off + e] = sum over ctas (in order) of partial[cta][e]; weights come
// first (W[o][i][k] order), then the biases.
__global__ void reduce_partials_kernel(const float *partial, int64_t n_cta, int ne, int nw, float *grad, int w_off,
                                       int b_off)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int64_t k = 0; k < n_cta; ++k) s += partial[k * ne + e];
        if (e < nw)
            grad[w_off + e] = s;
        else
            grad[b_off + (e - nw)] = s;
    }
}

// ---------------------------------------------------------------------------
// Targets, loss, optimiser
// ---------------------------------------------------------------------------
// Twice the boundary bond sum of block b of chain c: E(x') - E(x).
__device__ int block_delta_E(const Chains &ch, int64_t c, int b)
{
    const int L = ch.L, nb1 = L / kBlk;
    const int by = b / nb1, bx = b - by * nb1, y0 = by * kBlk, x0 = bx * kBlk;
    int d = 0;
    for (int t = 0; t < kBlk; ++t) {
        // top and bottom edges, left and right edges
        const int xt = x0 + t, yt = y0 + t;
        d += (int)spin_at(ch, c, y0, xt, -1) * (int)spin_at(ch, c, (y0 - 1 + L) % L, xt, -1);
        d += (int)spin_at(ch, c, y0 + kBlk - 1, xt, -1) * (int)spin_at(ch, c, (y0 + kBlk) % L, xt, -1);
        d += (int)spin_at(ch, c, yt, x0, -1) * (int)spin_at(ch, c, yt, (x0 - 1 + L) % L, -1);
        d += (int)spin_at(ch, c, yt, x0 + kBlk - 1, -1) * (int)spin_at(ch, c, yt, (x0 + kBlk) % L, -1);
    }
    return 2 * d;
}

// t_b = min(0, -beta dE_b); r = logit - t; dlogits = 2 r / (C nb); per-chain
// squared-residual sums for the loss.
__global__ void targets_loss_kernel(Chains ch, int64_t C, double beta, const float *logits, float *dlogits,
                                    float *chain_sq)
{
    const int nb1 = ch.L / kBlk, nb = nb1 * nb1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += nw) {
        float sq = 0.0f;
        for (int b = lane; b < nb; b += 32) {
            const int dE = block_delta_E(ch, c, b);
            const float t = (float)fmin(0.0, -beta * (double)dE);
            const float r = logits[c * nb + b] - t;
            dlogits[c * nb + b] = 2.0f * r / (float)(C * nb);
            sq += r * r;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
        if (lane == 0) chain_sq[c] = sq;
    }
}

__global__ void loss_reduce_kernel(const float *chain_sq, int64_t C, int nb, float *loss)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int64_t c = 0; c < C; ++c) s += chain_sq[c];
        *loss = (float)(s / (double)(C * nb));
    }
}

__global__ void adam_kernel(int n, float *params, const float *grad, float *m, float *v, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// The Metropolis-Hastings block move
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t move_draw(const RoundKeys &rk, uint32_t stream, uint32_t site, uint64_t t)
{
    const uint4 u = philox(site >> 2, stream, (uint32_t)t, counter_word3(0, kPurposeLearned, t), rk);
    const uint32_t w = site & 3;
    return w == 0 ? u.x : w == 1 ? u.y : w == 2 ? u.z : u.w;
}

// log of the softmax normaliser, summed in block order in FP64
__device__ double log_norm(const float *l, int nb)
{
    double m = l[0];
    for (int b = 1; b < nb; ++b) m = fmax(m, (double)l[b]);
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += exp((double)l[b] - m);
    return m + log(s);
}

__global__ void propose_kernel(int64_t C, int nb, const float *logits, const __grid_constant__ RoundKeys rk,
                               uint64_t t, int32_t *block)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = move_draw(rk, (uint32_t)c, 0, t);
        int b = nb - 1;
        if (logits == nullptr) {
            b = (int)(((uint64_t)u * (uint64_t)nb) >> 32);
        } else {
            const float *l = logits + c * nb;
            double m = l[0];
            for (int k = 1; k < nb; ++k) m = fmax(m, (double)l[k]);
            double total = 0.0;
            for (int k = 0; k < nb; ++k) total += exp((double)l[k] - m);
            const double target = ((double)u / 4294967296.0) * total;
            double acc = 0.0;
            for (int k = 0; k < nb; ++k) {
                acc += exp((double)l[k] - m);
                if (acc > target) {
                    b = k;
                    break;
                }
            }
        }
        block[c] = b;
    }
}

__global__ void accept_kernel(Chains ch, uint64_t *black, uint64_t *white, int64_t C, double beta, const float *lx,
                              const float *lxp, const int32_t *block, const __grid_constant__ RoundKeys rk, uint64_t t,
                              int32_t *accepted, int64_t *dE_out)
{
    const int L = ch.L, nb1 = L / kBlk, nb = nb1 * nb1;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int b = block[c];
        const int dE = block_delta_E(ch, c, b);
        double x = -beta * (double)dE;
        if (lx != nullptr) {
            const double logp_rev = (double)lxp[c * nb + b] - log_norm(lxp + c * nb, nb);
            const double logp_fwd = (double)lx[c * nb + b] - log_norm(lx + c * nb, nb);
            x = (x + logp_rev) - logp_fwd;
        }
        const uint64_t T = x >= 0.0 ? (uint64_t(1) << 32) : (uint64_t)floor(ldexp(exp(x), 32));
        const uint32_t u = move_draw(rk, (uint32_t)c, 1, t);
        const bool acc = (uint64_t)u < T;
        accepted[c] = acc ? 1 : 0;
        if (dE_out) dE_out[c] = dE;
        if (acc) {
            const int by = b / nb1, bx = b - by * nb1;
            // the block's 4 sites of each colour per row sit in nibbles 4 bx .. 4 bx + 3
            const int j0 = 4 * bx;
            const uint64_t mask = 0x1111ull << (4 * (j0 & 15));
            for (int r = 0; r < kBlk; ++r) {
                const int64_t w = c * (int64_t)L * ch.wpr + (int64_t)(by * kBlk + r) * ch.wpr + (j0 >> 4);
                black[w] ^= mask;
                white[w] ^= mask;
            }
        }
    }
}

unsigned grid1d(int64_t n, int threads)
{
    DeviceInfo info{1};
    device_info(&info);
    const int64_t cap = (int64_t)info.sm_count * 16;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (n + threads - 1) / threads));
}

thread_local char g_net_error[200] = "";

int nfail(int status, const char *msg)
{
    snprintf(g_net_error, sizeof(g_net_error), "%s", msg);
    return status;
}

int check_chains(int64_t L, int64_t C)
{
    if (L < 32 || L % 32 != 0 || L > 4096) return nfail(ISING_EINVAL, "L must be a multiple of 32 in [32, 4096]");
    if (C <= 0) return nfail(ISING_EINVAL, "C must be positive");
    return ISING_OK;
}

// Work layout: [z1 a1 z2 a2 z3 a3 d_a d_b] activations (8 x C L^2 32 floats)
// in training mode, [a1 a2] in inference mode, then weight-gradient partials.
struct NetWork {
    float *z1, *a1, *z2, *a2, *z3, *a3, *da, *db, *partial;
    int64_t n_cta;
    size_t bytes;
};

constexpr int64_t kWgradCtasPerSm = 2;  // persistent CTAs per SM in the weight-gradient kernels

NetWork net_layout(int64_t L, int64_t C, int train, char *base)
{
    NetWork w;
    memset(&w, 0, sizeof(w));
    const size_t act = (size_t)C * L * L * kCh * sizeof(float);
    size_t o = 0;
    auto take = [&](size_t n) {
        char *p = base ? base + o : nullptr;
        o += (n + 255) & ~size_t(255);
        return (float *)p;
    };
    if (train) {
        w.z1 = take(act); w.a1 = take(act); w.z2 = take(act); w.a2 = take(act);
        w.z3 = take(act); w.a3 = take(act); w.da = take(act); w.db = take(act);
        DeviceInfo info{152};
        device_info(&info);
        w.n_cta = (int64_t)info.sm_count * kWgradCtasPerSm;
        w.partial = take((size_t)w.n_cta * (kN2 + kCh) * sizeof(float));
    } else {
        w.a1 = take(act); w.a2 = take(act);
        w.a3 = w.a1;
    }
    w.bytes = o;
    return w;
}

}  // namespace
}  // namespace ising

using namespace ising;

extern "C" {

ISING_API int ising_net_param_count(void) { return kParams; }

ISING_API const char *ising_net_last_error(void) { return g_net_error; }

ISING_API int ising_net_workspace_bytes(int64_t L, int64_t C, int32_t train, size_t *bytes)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    if (!bytes) return nfail(ISING_EINVAL, "bytes is NULL");
    *bytes = net_layout(L, C, train, nullptr).bytes;
    return ISING_OK;
}

ISING_API int ising_net_forward(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                const int32_t *flip_block_dev, const float *params_dev, float *logits_dev,
                                void *work_dev, size_t work_bytes, int32_t train, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    NetWork w = net_layout(L, C, train, (char *)work_dev);
    if (work_dev == nullptr || work_bytes < w.bytes) return nfail(ISING_EINVAL, "work buffer too small");
    const size_t plane = (size_t)C * L * L / 32 * 8;
    if (check_device_range(black_dev, plane, "black") || check_device_range(white_dev, plane, "white") ||
        check_device_range(params_dev, kParams * 4, "params") ||
        check_device_range(logits_dev, (size_t)C * (L / 8) * (L / 8) * 4, "logits"))
        return nfail(ISING_EINVAL, "planes, params and logits must be device memory of their sizes");
    cudaStream_t s = (cudaStream_t)stream;
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    const int64_t npix = C * L * L;
    const unsigned g = grid1d(npix, kThreads);
    const size_t smem = (size_t)kN2 * sizeof(float);
    cudaFuncSetAttribute(conv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    l1_kernel<<<g, kThreads, 0, s>>>(ch, C, flip_block_dev, params_dev, train ? w.z1 : nullptr, w.a1);
    conv32_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW2, kOffB2, w.a1, train ? w.z2 : nullptr, w.a2);
    float *a3 = train ? w.a3 : w.a1;  // inference ping-pongs two buffers
    conv32_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW3, kOffB3, w.a2, train ? w.z3 : nullptr, a3);
    const int64_t warps = C * (L / 8) * (L / 8);
    l4_pool_kernel<<<grid1d(warps * 32, kThreads), kThreads, 0, s>>>((int)L, C, params_dev, a3, logits_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_net_backward(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                 const float *params_dev, const float *dlogits_dev, float *grad_dev, void *work_dev,
                                 size_t work_bytes, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    NetWork w = net_layout(L, C, 1, (char *)work_dev);
    if (work_dev == nullptr || work_bytes < w.bytes) return nfail(ISING_EINVAL, "work buffer too small (train mode)");
    if (check_device_range(grad_dev, kParams * 4, "grad") ||
        check_device_range(dlogits_dev, (size_t)C * (L / 8) * (L / 8) * 4, "dlogits"))
        return nfail(ISING_EINVAL, "grad and dlogits must be device memory of their sizes");
    cudaStream_t s = (cudaStream_t)stream;
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    const int64_t npix = C * L * L;
    const unsigned g = grid1d(npix, kThreads);
    const size_t smem = (size_t)kN2 * sizeof(float);
    const unsigned gw = (unsigned)w.n_cta;
    cudaFuncSetAttribute(conv32_bwd_data_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const size_t sm32 = (size_t)((kTy + 2) * (kTx + 2) * kCh + kTy * kTx * kCh) * sizeof(float);
    const size_t sm4 = (size_t)((kTy + 2) * (kTx + 2) * kCh + kTy * kTx) * sizeof(float);
    const size_t sm1 = (size_t)((kTy + 2) * (kTx + 2) + kTy * kTx * kCh) * sizeof(float);
    cudaFuncSetAttribute(wgrad_kernel<kCh, kCh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
    cudaFuncSetAttribute(wgrad_kernel<kCh, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4);
    cudaFuncSetAttribute(wgrad_kernel<1, kCh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    // layer 4
    wgrad_kernel<kCh, 1><<<gw, 256, sm4, s>>>(ch, C, w.a3, nullptr, dlogits_dev, w.partial);
    reduce_partials_kernel<<<4, 256, 0, s>>>(w.partial, w.n_cta, kN1 + 1, kN1, grad_dev, kOffW4, kOffB4);
    l4_bwd_data_kernel<<<g, kThreads, 0, s>>>((int)L, C, params_dev, dlogits_dev, w.z3, w.da);  // dz3
    // layer 3
    wgrad_kernel<kCh, kCh><<<gw, 256, sm32, s>>>(ch, C, w.a2, w.da, nullptr, w.partial);
    reduce_partials_kernel<<<40, 256, 0, s>>>(w.partial, w.n_cta, kN2 + kCh, kN2, grad_dev, kOffW3, kOffB3);
    conv32_bwd_data_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW3, w.da, w.z2, w.db);  // dz2
    // layer 2
    wgrad_kernel<kCh, kCh><<<gw, 256, sm32, s>>>(ch, C, w.a1, w.db, nullptr, w.partial);
    reduce_partials_kernel<<<40, 256, 0, s>>>(w.partial, w.n_cta, kN2 + kCh, kN2, grad_dev, kOffW2, kOffB2);
    conv32_bwd_data_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW2, w.db, w.z1, w.da);  // dz1
    // layer 1
    wgrad_kernel<1, kCh><<<gw, 256, sm1, s>>>(ch, C, nullptr, w.da, nullptr, w.partial);
    reduce_partials_kernel<<<4, 256, 0, s>>>(w.partial, w.n_cta, kN1 + kCh, kN1, grad_dev, kOffW1, kOffB1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_net_targets_loss(int64_t L, int64_t C, const void *black_dev, const void *white_dev, double beta,
                                     const float *logits_dev, float *dlogits_dev, float *chain_sq_dev,
                                     float *loss_dev, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    if (!(beta >= 0.0) || !std::isfinite(beta)) return nfail(ISING_EINVAL, "beta must be finite and >= 0");
    if (check_device_range(chain_sq_dev, (size_t)C * 4, "chain_sq") || check_device_range(loss_dev, 4, "loss"))
        return nfail(ISING_EINVAL, "chain_sq and loss must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    targets_loss_kernel<<<grid1d(C * 32, kThreads), kThreads, 0, s>>>(ch, C, beta, logits_dev, dlogits_dev,
                                                                      chain_sq_dev);
    loss_reduce_kernel<<<1, 32, 0, s>>>(chain_sq_dev, C, (int)((L / 8) * (L / 8)), loss_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_net_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int64_t step,
                             float lr, ising_stream_t stream)
{
    if (step <= 0 || !(lr > 0.0f)) return nfail(ISING_EINVAL, "step must be >= 1 and lr > 0");
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<grid1d(kParams, 256), 256, 0, (cudaStream_t)stream>>>(kParams, params_dev, grad_dev, m_dev, v_dev,
                                                                         lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_block_propose(int64_t L, int64_t C, const float *logits_dev, uint64_t seed, uint64_t t,
                                  int32_t *block_dev, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    if (check_device_range(block_dev, (size_t)C * 4, "block")) return nfail(ISING_EINVAL, "block must be device memory");
    const int nb = (int)((L / 8) * (L / 8));
    propose_kernel<<<grid1d(C, 128), 128, 0, (cudaStream_t)stream>>>(C, nb, logits_dev, make_round_keys(seed), t,
                                                                     block_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

ISING_API int ising_block_accept(int64_t L, int64_t C, void *black_dev, void *white_dev, double beta,
                                 const float *logits_x_dev, const float *logits_xp_dev, const int32_t *block_dev,
                                 uint64_t seed, uint64_t t, int32_t *accepted_dev, int64_t *dE_dev,
                                 ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    if (!(beta >= 0.0) || !std::isfinite(beta)) return nfail(ISING_EINVAL, "beta must be finite and >= 0");
    if ((logits_x_dev == nullptr) != (logits_xp_dev == nullptr))
        return nfail(ISING_EINVAL, "give both logits (network proposal) or neither (uniform)");
    const size_t plane = (size_t)C * L * L / 32 * 8;
    if (check_device_range(black_dev, plane, "black") || check_device_range(white_dev, plane, "white") ||
        check_device_range(accepted_dev, (size_t)C * 4, "accepted"))
        return nfail(ISING_EINVAL, "planes and accepted must be device memory of their sizes");
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    accept_kernel<<<grid1d(C, 128), 128, 0, (cudaStream_t)stream>>>(
        ch, (uint64_t *)black_dev, (uint64_t *)white_dev, C, beta, logits_x_dev, logits_xp_dev, block_dev,
        make_round_keys(seed), t, accepted_dev, dE_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
