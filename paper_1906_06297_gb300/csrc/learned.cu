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
// Network (3 x 3 periodic cross-correlations, 32 channels; a BF16 network:
// weights and the activations a1..a3 are bfloat16 (round to nearest even),
// products are accumulated in FP32):
//   a1 = gelu(conv(spins; W1, b1)), a2 = gelu(conv(a1; W2, b2)),
//   a3 = gelu(conv(a2; W3, b3)), z4 = conv(a3; W4, b4) (one channel),
//   logit of block b = mean of z4 over the block; q(b) = softmax(logits)_b.
// gelu(z) = z * Phi(z).  Parameters are one FP32 vector in the order
// W1[32][9], b1[32], W2[32][32][9], b2[32], W3[32][32][9], b3[32], W4[32][9], b4[1].
// Activations are bfloat16, 32 channels (64 bytes) per pixel, in rows of L + 2
// pixels: column 0 repeats pixel L - 1 and column L + 1 pixel 0 (the periodic
// halo, written by the producer), so that one rectangular copy fetches a row
// segment with both neighbours.  The pre-activations z kept for training and
// the gradients are NHWC FP32 without halo.
//
// Forward kernels: layer 1 by table lookup (l1_table_kernel, l1_kernel); the
// two 32 -> 32 layers on the tensor cores (tcgen05; conv32_ring_kernel for L
// a multiple of 128, conv32_tc_kernel otherwise), the second one also
// contracting layer 4's input channels (P, the 9 tap projections; reduced to
// row partials of z4 per 8-pixel block column where L is a multiple of 128);
// the tap sums and block means (pool_rows_kernel, pool_kernel).  Every
// reduction has a fixed order, so
// a forward pass is a deterministic function of the state.  Backward kernels,
// straight through the bfloat16 roundings: for L a multiple of 128 the data
// and weight gradients of the two 32 -> 32 layers on the tensor cores
// (conv32_ring_kernel in BWD mode, wgrad_tc_kernel), the rest in FP32 on the
// CUDA cores; weight gradients as fixed-order per-CTA partial sums.
//
// Move.  Block b is drawn by inverse CDF of q_x (purpose-3 draw, site 0, in
// the chain's stream) or uniformly; x' = x with block b flipped; the flip is
// accepted iff the purpose-3 draw of site 1 is below
// floor(2^32 min(1, exp(-beta dE + log q_x'(b) - log q_x(b)))), dE the exact
// integer energy change (twice the boundary bond sum).  Softmax sums run in
// block order in FP64.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ising.h"
#include "common.cuh"
#include "launch.h"
#include "tc.cuh"

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

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Eight FP32 values as two bfloat16 parts, packed in pairs: hi = bf16(v) and
// lo = bf16(v - hi) (v - hi is exact in FP32), so hi + lo equals v to about
// 2^-17 relative.
__device__ __forceinline__ void split_bf16(const float (&v)[8], uint32_t (&hi)[4], uint32_t (&lo)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        hi[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
        lo[j] = pack_bf16x2(v[2 * j] - bf16_lo(hi[j]), v[2 * j + 1] - bf16_hi(hi[j]));
    }
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// GELU z Phi(z), Phi(z) = erfc(-z / sqrt 2) / 2, with erfc from the Chebyshev
// fit of Numerical Recipes (Press et al., 2nd ed., Sec. 6.2, "erfcc"):
// erfc(x) = t exp(-x^2 + P(t)), t = 1 / (1 + x / 2), P of degree 9, fractional
// error below 1.2e-7 for every x >= 0, so Phi keeps its relative accuracy for
// negative z too.  Evaluated in FP32 with the hardware reciprocal and 2^x the
// relative error of gelu is about 5e-6 for |z| < 6 (the rounding of the
// exponent -x^2 + P), far below the bfloat16 step the result is rounded to.
// With h = Phi(-|z|), gelu(z) = max(z, 0) - |z| h for either sign of z (z (1 -
// h) for z >= 0, z h for z < 0), one multiply-add.
__device__ __forceinline__ float gelu(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.5f, x, 1.0f));
    float p = 0.17087277f;
    p = fmaf(p, t, -0.82215223f);
    p = fmaf(p, t, 1.48851587f);
    p = fmaf(p, t, -1.13520398f);
    p = fmaf(p, t, 0.27886807f);
    p = fmaf(p, t, -0.18628806f);
    p = fmaf(p, t, 0.09678418f);
    p = fmaf(p, t, 0.37409196f);
    p = fmaf(p, t, 1.00002368f);
    p = fmaf(p, t, -1.26551223f);
    // -|z| Phi(-|z|) = x (-sqrt(1/2)) t 2^((-x^2 + P) log2 e)
    const float nq = -0.70710678118654752f * t * ex2_approx(fmaf(-x, x, p) * 1.44269504088896341f);
    return fmaf(x, nq, fmaxf(z, 0.0f));
}

// The same GELU for two values at once: the FP32 multiplies and adds as
// packed pairs (fma.rn.f32x2 / mul.rn.f32x2, each half rounded like the
// scalar instruction, so the results equal gelu's bit for bit), the
// reciprocal and 2^x per value.  Halves the instructions of the polynomial.
__device__ __forceinline__ uint64_t f2_pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void f2_unpack(uint64_t v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t f2_splat(float c) { return f2_pack(c, c); }

__device__ __forceinline__ void gelu2(float &z0, float &z1)
{
    const uint64_t x = f2_mul(f2_pack(fabsf(z0), fabsf(z1)), f2_splat(0.70710678118654752f));
    float d0, d1;
    f2_unpack(f2_fma(f2_splat(0.5f), x, f2_splat(1.0f)), d0, d1);
    const uint64_t t = f2_pack(rcp_approx(d0), rcp_approx(d1));
    uint64_t p = f2_splat(0.17087277f);
    p = f2_fma(p, t, f2_splat(-0.82215223f));
    p = f2_fma(p, t, f2_splat(1.48851587f));
    p = f2_fma(p, t, f2_splat(-1.13520398f));
    p = f2_fma(p, t, f2_splat(0.27886807f));
    p = f2_fma(p, t, f2_splat(-0.18628806f));
    p = f2_fma(p, t, f2_splat(0.09678418f));
    p = f2_fma(p, t, f2_splat(0.37409196f));
    p = f2_fma(p, t, f2_splat(1.00002368f));
    p = f2_fma(p, t, f2_splat(-1.26551223f));
    float x0, x1;
    f2_unpack(x, x0, x1);
    float a0, a1;
    f2_unpack(f2_mul(f2_fma(f2_pack(-x0, -x1), x, p), f2_splat(1.44269504088896341f)), a0, a1);
    const uint64_t nq = f2_mul(f2_mul(f2_splat(-0.70710678118654752f), t), f2_pack(ex2_approx(a0), ex2_approx(a1)));
    f2_unpack(f2_fma(x, nq, f2_pack(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f))), z0, z1);
}

// gelu'(z) = Phi(z) + z phi(z), phi the normal density, with Phi from the
// same Numerical Recipes erfc fit as gelu and phi(z) = 2^(-x^2 log2 e) /
// sqrt(2 pi), x = |z| / sqrt 2; for two values at once (packed FP32 as in
// gelu2).  Relative error about 1e-6, far below the gradient tolerance.
__device__ __forceinline__ void gelu_grad2(float &z0, float &z1)
{
    const uint64_t x = f2_mul(f2_pack(fabsf(z0), fabsf(z1)), f2_splat(0.70710678118654752f));
    float d0, d1;
    f2_unpack(f2_fma(f2_splat(0.5f), x, f2_splat(1.0f)), d0, d1);
    const uint64_t t = f2_pack(rcp_approx(d0), rcp_approx(d1));
    uint64_t p = f2_splat(0.17087277f);
    p = f2_fma(p, t, f2_splat(-0.82215223f));
    p = f2_fma(p, t, f2_splat(1.48851587f));
    p = f2_fma(p, t, f2_splat(-1.13520398f));
    p = f2_fma(p, t, f2_splat(0.27886807f));
    p = f2_fma(p, t, f2_splat(-0.18628806f));
    p = f2_fma(p, t, f2_splat(0.09678418f));
    p = f2_fma(p, t, f2_splat(0.37409196f));
    p = f2_fma(p, t, f2_splat(1.00002368f));
    p = f2_fma(p, t, f2_splat(-1.26551223f));
    float x0, x1;
    f2_unpack(x, x0, x1);
    const uint64_t nx2 = f2_mul(f2_pack(-x0, -x1), x);  // -x^2
    float a0, a1, b0, b1;
    f2_unpack(f2_mul(f2_fma(f2_splat(1.0f), nx2, p), f2_splat(1.44269504088896341f)), a0, a1);
    f2_unpack(f2_mul(nx2, f2_splat(1.44269504088896341f)), b0, b1);
    float h0, h1, g0, g1;
    f2_unpack(f2_mul(f2_mul(f2_splat(0.5f), t), f2_pack(ex2_approx(a0), ex2_approx(a1))), h0, h1);  // Phi(-|z|)
    f2_unpack(f2_mul(f2_pack(ex2_approx(b0), ex2_approx(b1)), f2_splat(0.39894228040143268f)), g0, g1);  // phi(z)
    const float P0 = z0 >= 0.0f ? 1.0f - h0 : h0, P1 = z1 >= 0.0f ? 1.0f - h1 : h1;
    f2_unpack(f2_fma(f2_pack(z0, z1), f2_pack(g0, g1), f2_pack(P0, P1)), z0, z1);
}

__device__ __forceinline__ float gelu_grad(float z)
{
    float other = 0.0f;
    gelu_grad2(z, other);
    return z;
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
// Which rows a forward launch computes.  A full pass covers every row of every
// chain (flip == nullptr here).  A band pass, used for the flipped state of a
// block move, covers per chain `rows` consecutive rows starting `lead` rows
// above the first row of the chain's flipped block (periodically): the rows
// whose values can differ from the unflipped state's and that the recomputed
// logits need.
struct Band {
    int L;
    int rows;             // rows per chain (L for a full pass)
    int lead;             // band pass: first row = 8 by - lead (mod L)
    const int32_t *flip;  // band pass: the flipped block of each chain
    int64_t C;
};

__device__ __forceinline__ int band_row0(const Band &b, int64_t c)
{
    if (b.flip == nullptr) return 0;
    const int f = b.flip[c];
    const int by = f < 0 ? 0 : f / (b.L / kBlk);
    const int r = by * kBlk - b.lead;
    return r < 0 ? r + b.L : r;
}

// Pixel pb of the band (0 <= pb < C rows L) -> chain c and the offset yx =
// y L + x of its pixel within the chain.
__device__ __forceinline__ void band_pixel(const Band &b, int64_t pb, int64_t &c, int &yx)
{
    const int64_t per = (int64_t)b.rows * b.L;
    c = pb / per;
    const int r = (int)(pb - c * per);
    const int ry = r / b.L;
    int y = band_row0(b, c) + ry;
    if (y >= b.L) y -= b.L;
    yx = y * b.L + (r - ry * b.L);
}

__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Index of pixel (y, x), -1 <= x <= L, of chain c in an activation buffer
// (rows of L + 2 pixels with the periodic halo columns).
__device__ __forceinline__ int64_t apix(int L, int64_t c, int y, int x) { return (c * L + y) * (int64_t)(L + 2) + x + 1; }

// Stores one 16-byte part of pixel (y, x)'s activations and, for x = 0 or
// x = L - 1, its copy in the halo column.
__device__ __forceinline__ void store_act(__nv_bfloat16 *a, int L, int64_t c, int y, int x, int off, uint4 v)
{
    *reinterpret_cast<uint4 *>(a + apix(L, c, y, x) * kCh + off) = v;
    if (x == 0) *reinterpret_cast<uint4 *>(a + apix(L, c, y, L) * kCh + off) = v;
    if (x == L - 1) *reinterpret_cast<uint4 *>(a + apix(L, c, y, -1) * kCh + off) = v;
}

// Layer 1 (1 -> 32 channels) sees only the 3 x 3 spins around a pixel, so its
// output is a function of a 9-bit pattern (bit k set when the spin at tap k =
// 3 (dy + 1) + (dx + 1) is +1).  l1_table_kernel evaluates z1 and
// bf16(gelu(z1)) for all 512 patterns, with the arithmetic a direct evaluation
// would use (bias first, then the taps in order by fmaf); l1_kernel then reads
// each pixel's pattern and copies its row of the table.
constexpr int kPatterns = 512;
constexpr int kL1Threads = 128;

__global__ void l1_table_kernel(const float *params, float *tz, __nv_bfloat16 *ta)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // pattern * 32 + output channel
    if (e >= kPatterns * kCh) return;
    const int pat = e / kCh, o = e - pat * kCh;
    float v = bf16r(params[kOffB1 + o]);
#pragma unroll
    for (int k = 0; k < 9; ++k) v = fmaf(bf16r(params[kOffW1 + o * 9 + k]), ((pat >> k) & 1) ? 1.0f : -1.0f, v);
    tz[e] = v;
    ta[e] = __float2bfloat16_rn(gelu(v));
}

// 1 if the spin at row y, column x of chain c is +1 (block `flip`, or -1 for
// none, negated).
__device__ __forceinline__ uint32_t spin_up(const Chains &ch, int64_t c, int y, int x, int flip)
{
    const int j = x >> 1;
    const uint64_t *plane = ((y + x) & 1) ? ch.white : ch.black;
    uint32_t u = (uint32_t)(plane[c * (int64_t)ch.L * ch.wpr + (int64_t)y * ch.wpr + (j >> 4)] >> (4 * (j & 15))) & 1u;
    if (flip >= 0) {
        const int nb = ch.L / kBlk;
        const int by = flip / nb, bx = flip - by * nb;
        if ((y >> 3) == by && (x >> 3) == bx) u ^= 1u;
    }
    return u;
}

// Thread per pixel of the band; blockIdx.y walks the chains and blockIdx.x
// the 128-pixel tiles of a chain's band, so all index arithmetic is 32-bit.
// Writes a1 (bfloat16, from the table in shared memory) and, when z_out !=
// nullptr, z1 (FP32), each store instruction covering whole pixels.
__global__ void __launch_bounds__(kL1Threads) l1_kernel(Chains ch, Band bd, const int32_t *flip,
                                                        const __nv_bfloat16 *ta, const float *tz, float *z_out,
                                                        __nv_bfloat16 *a_out)
{
    __shared__ uint4 T[kPatterns * kCh * 2 / 16];  // ta, 32 KiB
    for (int i = threadIdx.x; i < kPatterns * kCh * 2 / 16; i += blockDim.x) T[i] = reinterpret_cast<const uint4 *>(ta)[i];
    __syncthreads();
    const int L = ch.L;
    const int per = bd.rows * L;  // band pixels per chain, a multiple of 128
    for (int64_t c = blockIdx.y; c < bd.C; c += gridDim.y) {
        const int row0 = band_row0(bd, c);
        const int fb = flip ? flip[c] : -1;
        for (int r = blockIdx.x * kL1Threads + threadIdx.x; r < per; r += gridDim.x * kL1Threads) {
            const int ry = r / L, x = r - ry * L;
            int y = row0 + ry;
            y = y >= L ? y - L : y;
            uint32_t pat = 0;
#pragma unroll
            for (int k = 0; k < 9; ++k) pat |= spin_up(ch, c, wrap(y + k / 3 - 1, L), wrap(x + k % 3 - 1, L), fb) << k;
            // the warp's 32 pixels are consecutive in one row: store round j
            // writes pixels 8j .. 8j+7 whole (512 contiguous bytes), lane l
            // the 16-byte part l % 4 of pixel 8j + l / 4
            const int lane = threadIdx.x & 31, x_first = x - lane;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int pp = 8 * j + (lane >> 2), g = lane & 3;
                const uint32_t pt = __shfl_sync(0xffffffffu, pat, pp);
                store_act(a_out, L, c, y, x_first + pp, 8 * g, T[pt * 4 + g]);
            }
            if (z_out) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int pp = 4 * j + (lane >> 3), g = lane & 7;
                    const uint32_t pt = __shfl_sync(0xffffffffu, pat, pp);
                    reinterpret_cast<float4 *>(z_out + ((c * L + y) * (int64_t)L + x_first + pp) * kCh)[g] =
                        __ldg(reinterpret_cast<const float4 *>(tz + pt * kCh) + g);
                }
            }
        }
    }
}

// Layers 2 and 3 (32 -> 32 channels) on the tensor cores, as an implicit GEMM
// per tile of 128 consecutive pixels of the band:
//   Z[m][o] = sum over taps k and input channels i of A_k[m][i] W[o][i][k],
// M = 128 pixels, N = 32 output channels, K = 9 taps x 32 channels = 18 MMA
// steps of K = 16 (tcgen05.mma kind::f16, BF16 operands, FP32 accumulator in
// tensor memory).  A_k, the input activations of the pixels shifted by tap k
// (periodic), is gathered into shared memory in the no-swizzle K-major layout:
// for tap k and channel group g (8 channels = 16 bytes) a plane of 128 pixel
// rows of 16 bytes, planes 2080 bytes apart, so one MMA step (two channel
// groups of one tap) reads core matrices of 8 pixels x 16 bytes at SBO = 128
// bytes along M and LBO = 2080 bytes along K.  This kernel serves any L (a
// multiple of 32); conv32_ring_kernel below is the one for L a multiple of 128.  The weights, B_k[o][i] =
// bf16(W[o][i][k]), sit the same way (planes of 32 rows, LBO = 512 bytes),
// staged once per CTA.  Persistent CTAs (one per SM) walk tiles j, j + grid,
// ...; the gather of tile n+1 and the epilogue of tile n-1 overlap the MMAs of
// tile n (two shared-memory stages, two accumulators of 32 TMEM columns).
// Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its pixels) and
// columns 16 (w / 4) .. + 15 (its output channels), adds the bias, and writes
// z (FP32, training) and bf16(gelu(z)).
constexpr int kTileM = 128;
constexpr int kConvThreads = 256;
constexpr int kTaps = 9;
constexpr int kGroups = kCh / 8;                                      // 16-byte channel groups per pixel
// One channel group of 128 (+2) pixel rows: 2080 bytes, so that the planes of
// the 4 channel groups start 32 bytes apart modulo the 128-byte bank row and
// 8 lanes storing 2 pixels x 4 groups hit 8 different 16-byte bank groups.
constexpr uint32_t kPlane = (kTileM + 2) * 16;
constexpr uint32_t kAStage = kTaps * kGroups * kPlane;                // 74880 bytes per stage
constexpr uint32_t kBBytes = kTaps * kGroups * kCh * 16;              // 18432 bytes
// + bias, barriers and the TMEM slot
constexpr uint32_t kConvSmem = 2 * kAStage + kBBytes + kCh * 4 + 64;
constexpr uint32_t kTmemCols = 64;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ int g_tc_error;  // set to 1 when a tensor-core wait gives up

struct ConvTc {
    const __nv_bfloat16 *a_in;  // NHWC, C L^2 x 32
    __nv_bfloat16 *a_out;
    float *z_out;  // nullable
    const float *params;
    int w_off, b_off;
    Band bd;
    int64_t tiles;  // C rows L / 128
};

__device__ __forceinline__ void tile_origin(const ConvTc &p, int64_t tile, int64_t &c, int &yx0)
{
    band_pixel(p.bd, tile * kTileM, c, yx0);
}

// Gathers A_k for the 9 taps of one tile.  Thread t moves channel group t % 4
// of pixels m0 = t / 4 and m0 + 64 for every tap.
__device__ __forceinline__ void conv_gather(const ConvTc &p, int64_t tile, uint8_t *sa)
{
    const int L = p.bd.L;
    int64_t c;
    int yx0;
    tile_origin(p, tile, c, yx0);
    const int g = threadIdx.x & 3, m0 = threadIdx.x >> 2;
    int py[2], px[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int yx = yx0 + m0 + 64 * h;
        py[h] = yx / L;
        px[h] = yx - py[h] * L;
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(p.a_in);
    uint4 v[2 * kTaps];
#pragma unroll
    for (int k = 0; k < kTaps; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int yy = wrap(py[h] + k / 3 - 1, L), xx = wrap(px[h] + k % 3 - 1, L);
            v[2 * k + h] = __ldg(src + apix(L, c, yy, xx) * kGroups + g);
        }
#pragma unroll
    for (int k = 0; k < kTaps; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<uint4 *>(sa + (k * kGroups + g) * kPlane + (m0 + 64 * h) * 16) = v[2 * k + h];
}

__device__ __forceinline__ void conv_epilogue(const ConvTc &p, int64_t tile, uint32_t tacc, const float *bias)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quad = warp & 3, half = warp >> 2;
    int64_t c;
    int yx0;
    tile_origin(p, tile, c, yx0);
    const int L = p.bd.L;
    const int yx = yx0 + quad * 32 + lane, y = yx / L, x = yx - y * L;
    const int64_t q = c * (int64_t)L * L + yx;
    float v[16];
    tc::tmem_ld16(tacc + (uint32_t)(half * 16) + ((uint32_t)(quad * 32) << 16), v);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += bias[half * 16 + j];
    if (p.z_out) {
        float4 *zo = reinterpret_cast<float4 *>(p.z_out + q * kCh + half * 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) zo[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float g0 = v[2 * j], g1 = v[2 * j + 1];
        gelu2(g0, g1);
        w[j] = pack_bf16x2(g0, g1);
    }
    store_act(p.a_out, L, c, y, x, half * 16, make_uint4(w[0], w[1], w[2], w[3]));
    store_act(p.a_out, L, c, y, x, half * 16 + 8, make_uint4(w[4], w[5], w[6], w[7]));
}

__global__ void __launch_bounds__(kConvThreads, 1) conv32_tc_kernel(const __grid_constant__ ConvTc p)
{
    extern __shared__ __align__(1024) uint8_t conv_smem[];
    uint8_t *sA = conv_smem;
    uint8_t *sB = conv_smem + 2 * kAStage;
    float *sBias = reinterpret_cast<float *>(sB + kBBytes);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sBias + kCh);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::fence_mbar_init();
    }
    // B[k][g][o] = the 8 input channels 8g .. 8g+7 of W[o][.][k], bfloat16
    for (int e = tid; e < kTaps * kGroups * kCh; e += blockDim.x) {
        const int k = e / (kGroups * kCh), r = e - k * (kGroups * kCh), g = r / kCh, o = r - g * kCh;
        const float *w = p.params + p.w_off + (o * kCh + 8 * g) * 9 + k;
        *reinterpret_cast<uint4 *>(sB + e * 16) =
            make_uint4(pack_bf16x2(w[0], w[9]), pack_bf16x2(w[18], w[27]), pack_bf16x2(w[36], w[45]),
                       pack_bf16x2(w[54], w[63]));
    }
    if (tid < kCh) sBias[tid] = bf16r(p.params[p.b_off + tid]);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(kTileM, kCh);
    const uint32_t a_u32 = tc::smem_u32(sA), b_u32 = tc::smem_u32(sB);

    bool ok = true;
    int committed = 0;  // tiles whose MMAs were issued
    for (int n = 0;; ++n) {
        const int64_t tile = blockIdx.x + (int64_t)n * gridDim.x;
        const bool has = tile < p.tiles;
        const int buf = n & 1;
        // stage `buf` was last read by the MMAs of tile n-2, waited for below at step n-1
        if (has) conv_gather(p, tile, sA + buf * kAStage);
        tc::fence_async_smem();
        __syncthreads();
        if (has && tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < 2 * kTaps; ++s) {
                const int k = s >> 1, g = 2 * (s & 1);
                const uint64_t ad =
                    tc::smem_desc(a_u32 + buf * kAStage + (k * kGroups + g) * kPlane, kPlane, 128);
                const uint64_t bd = tc::smem_desc(b_u32 + (k * kGroups + g) * kCh * 16, kCh * 16, 128);
                tc::mma_bf16(tmem + (uint32_t)(buf * kCh), ad, bd, idesc, s > 0 ? 1u : 0u);
            }
            tc::mma_commit(&mbar[buf]);
        }
        if (has) committed = n + 1;
        if (n >= 1) {
            const int pn = n - 1, pb = pn & 1;
            // ok stays warp-uniform: the TMEM loads below are warp-collective
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&mbar[pb], (uint32_t)((pn >> 1) & 1), kWaitCycles)))
                ok = false;
            tc::fence_after_sync();
            if (ok) conv_epilogue(p, blockIdx.x + (int64_t)pn * gridDim.x, tmem + (uint32_t)(pb * kCh), sBias);
            tc::fence_before_sync();
        }
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (!has) break;
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(&g_tc_error, 1);
            // let the MMAs of the last issued tile finish before the TMEM is freed
            if (committed > 0) {
                const int ln = committed - 1;
                tc::mbar_wait(&mbar[ln & 1], (uint32_t)((ln >> 1) & 1), kWaitCycles);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// Layers 2 and 3 for L a multiple of 128: the same implicit GEMM per tile (one
// 128-pixel row segment), fed from a ring of staged input rows.  A work unit
// is up to kUnitRows consecutive output rows of one (chain, 128-column
// segment); it stages its rows r0 - 1 .. r0 + n once each, as a halo row of
// 130 pixels (x0 - 1 .. x0 + 128, periodic) in 4 channel-group planes of
// kRingPlane bytes, so the operand of tap (dy, dx) is the staged row y + dy
// offset by (1 + dx) x 16 bytes (LBO = kRingPlane, SBO = 128).
// Warp roles, linked by mbarriers (every wait bounded):
//   warp 0: loader -- lane 0 fetches each row with four tensor copies (TMA),
//           one per channel group: a box of 8 channels x 130 pixels of the
//           padded row (its halo columns included), completing on full[slot];
//           or, in the first layer of an inference pass (FUSED), the warp
//           builds the row of a1 itself: 18 lanes turn 3 spin rows x 6
//           32-column chunks around the segment into bit vectors (a chunk is
//           one black and one white MSC4 word, nibbles compressed and
//           interleaved by the row's colour parity), each pixel's 3 x 3
//           pattern comes from them by shuffles, and its layer-1 output is
//           the pattern's row of the table (l1_table_kernel); the lanes then
//           fence the async proxy and lane 0 arrives on full[slot]: a1 never
//           goes through global memory;
//   warp 1: lane 0 issues the MMAs row-stationary: each staged row, once
//           per (dx, K half), times the weights of the three dy taps stacked
//           along N = 96, into the accumulator blocks of the three output
//           rows it feeds (a ring of kAcc blocks in descending row order, so
//           the three are adjacent; two MMAs where the window wraps): 6-8
//           MMAs per row where a tile-at-a-time schedule needs 18 of N = 32
//           (the tensor core spends ~45 cycles on an N = 32 MMA and ~56 on an
//           N = 96 one).  It then commits to empty[slot] of the row (no later
//           MMA reads it) and to accf[block] of the output row that row
//           completed;
//   warps 2-9: epilogue, warp w on TMEM lanes 32 (w % 4) .. + 31 (its 32
//           pixels) and columns 16 h .. 16 h + 15, h = (w - 2) / 4 (its 16
//           channels): loads them, sets them to the bias (every MMA
//           accumulates, so the next row's sum starts from its bias; zero in
//           BWD), frees the block (acce, 8 arrivals) and writes z (training)
//           and a = bf16(gelu(z)).  (Adding the bias in the epilogue and
//           gelu as z (1 - h) or z h by sign instead of max(z, 0) - |z| h:
//           1.438 instead of 1.383 ms per full forward of 1024 chains.)
//           Two warps per TMEM lane quadrant, four per SM sub-partition with
//           two CTAs per SM, hide the latency of the GELU arithmetic.
// PROJ (the last 32-channel layer): layer 4's channel contraction is done
// here, on the tensor cores, as P[m][k] = sum_i a[m][i] W4[i][k] for the 9
// taps k (N padded to 16): the epilogue stages the tile's a in shared memory
// (a3full), lane 0 of a warp of its own (warp 10) multiplies it by W4^T into
// 16 more TMEM columns (pfull, a3empty), and four more warps (11-14, one per
// TMEM lane quadrant) read P out (pempty) and reduce it to row partials of z4
// (see pool_rows_kernel).  Then a3 itself need not reach global memory (it
// still does when training, for the backward pass).  Measured per full
// forward of 1024 chains of 128^2: these MMAs on the row MMA thread, which
// then waits for each tile's a3, 1.383 ms; on their own warp with P stored as
// 9 planes by the epilogue warps of the first channel half 1.371; stored by
// the four P warps 1.366 (1.400 with three a3 tiles, planes 2048 bytes
// apart); reduced to row partials as here 1.272.
// BWD (the data gradient of a 32 -> 32 layer in the training backward pass):
// the same contraction with the incoming gradient dz (bfloat16, halo columns)
// as the staged rows and the weights transposed and tap-flipped, B_k[i][o] =
// W[o][i][8 - k], since dz_prev(p)[i] = gelu'(z_prev(p)[i]) sum_k sum_o
// W[o][i][k] dz(p - off_k)[o] and -off_k = off_{8-k}; the epilogue multiplies
// by gelu'(z_prev) and writes dz_prev in FP32 (and in bfloat16 with halo
// columns when a_out is set, for the next data gradient).
// Dependencies: the MMAs of staged row i wait on the epilogue of output rows
// up to i + 1 - kAcc only, the epilogue of row t on the MMAs of staged rows up
// to t + 1 only, so no wait can close a cycle.
constexpr int kRing = 8;        // staged rows (a power of two)
constexpr int kAcc = 7;         // accumulator blocks of 32 TMEM columns, one per output row in flight
// output rows per work unit: each unit stages 2 halo rows and restarts the
// pipeline; 32 rows per unit measured 1.66 ms per full forward of 1024
// chains of 128^2 against 1.73 (16), 1.72 (64), 1.75 (128), 1.89 (24)
constexpr int kUnitRows = 32;
constexpr int kEpiWarps = 8;
constexpr int kRingThreads = 64 + 32 * kEpiWarps;
// one more warp: the second loader of the fused first conv, or the issuer of
// the layer-4 projection MMAs (PROJ)
constexpr int kRingExtra = 2 + kEpiWarps;
// PROJ: four more warps (kRingExtra + 1 .. + 4, one per TMEM lane quadrant)
// read the tap projections P out of tensor memory and reduce them to row
// partials of z4
constexpr int kProjWarps = 4;
template <bool PROJ, bool FUSED>
constexpr int ring_threads() { return PROJ ? kRingThreads + 32 * (1 + kProjWarps) : (FUSED ? kRingThreads + 32 : kRingThreads); }
constexpr int kProjN = 16;      // the 9 taps of layer 4, padded to an MMA N
// channel-group planes 2176 bytes apart: each tensor copy lands on a 128-byte
// boundary; 130 of its 136 16-byte entries are used
constexpr uint32_t kRingPlane = 17 * 128;
constexpr uint32_t kRowBytes = kGroups * kRingPlane;   // one staged row, or one a3 tile
constexpr uint32_t kW4Bytes = kGroups * kProjN * 16;   // 1024
constexpr int kRingBars = 2 * kRing + 2 * kAcc + 8 + 2;
// Shared-memory layout: the staged rows, then (only in the kernel that
// projects onto layer 4) two a3 tiles, the weights, (PROJ) W4^T, the bias,
// (STAGE) the epilogue warps' staging tiles and the barriers.  Without the a3 tiles two CTAs take 173 KB, so the SM keeps
// ~60 KB of L1 (a 196 KB carveout), enough for layer 1's 32 KB table that the
// fused first layer reads for every pixel (with the a3 tiles: 28 KB, and about
// 40% of its table reads missed L1).
//
// The data-gradient kernel (BWD) and the training forward of the first
// 32 -> 32 layer also hold a 2 KB staging tile per epilogue warp: their FP32
// loads and stores and their bfloat16 stores of a row go through it, so that
// every global access of a warp covers whole sectors of a few lines (a lane's
// own pixel is 64 or 128 bytes apart from its neighbour's).
constexpr uint32_t kStageBytes = 32 * 16 * 4;  // 32 pixels x 16 FP32 channels
template <bool PROJ, bool STAGE = false>
struct RingLayout {
    static constexpr uint32_t ring = 0;
    static constexpr uint32_t a3 = ring + kRing * kRowBytes;
    static constexpr uint32_t b = PROJ ? a3 + 2 * kRowBytes : a3;
    static constexpr uint32_t w4 = b + kBBytes;
    static constexpr uint32_t bias = PROJ ? w4 + kW4Bytes : w4;
    static constexpr uint32_t stage = bias + kCh * 4;
    static constexpr uint32_t bar = STAGE ? stage + kEpiWarps * kStageBytes : stage;
    static constexpr uint32_t bytes = bar + kRingBars * 8 + 16;
};
constexpr uint32_t kRingTmemCols = 256;  // 7 x 32 accumulator + 2 x 16 projection columns
constexpr int kStackN = 3 * kCh;         // the weights of the three dy taps stacked along N
// accumulator block of output row t (counted over a CTA's units, 32-bit: the
// MMA thread does this arithmetic for every row): descending, so that rows
// t + 1, t, t - 1 sit in consecutive blocks; and the parity of its use
__device__ __forceinline__ int ring_blk(uint32_t t) { return kAcc - 1 - (int)(t % (uint32_t)kAcc); }
__device__ __forceinline__ uint32_t ring_use(uint32_t t) { return t / (uint32_t)kAcc; }
static_assert((kRing & (kRing - 1)) == 0 && kRing >= 6, "ring of a power-of-two rows, 3 in use and 3 ahead");
static_assert(2 * RingLayout<true>::bytes <= 228 * 1024, "two CTAs per SM");
static_assert(2 * RingLayout<false>::bytes + 2048 <= 196 * 1024, "two CTAs per SM in a 196 KB carveout");
static_assert(2 * RingLayout<false, true>::bytes <= 228 * 1024 && RingLayout<false, true>::stage % 16 == 0,
              "two data-gradient CTAs per SM");

// A warp's staging tile: 32 pixels (lane = pixel in the per-pixel accesses) x
// 64 bytes.  FP32 tiles: chunk cc (4 channels, 16 bytes) of pixel pp at 16-byte
// slot 4 pp + (cc ^ ((pp >> 1) & 3)); the coalesced accesses take lane =
// 4 (pixel % 8) + chunk.  bfloat16 tiles (32 bytes per pixel): chunk cc (8
// channels) at slot 2 pp + (cc ^ ((pp >> 2) & 1)), coalesced lane = 2 (pixel %
// 16) + chunk.  Either way the eight lanes of each 128-bit shared-memory phase
// hit eight different 16-byte slots of a 128-byte window: no bank conflicts.
__device__ __forceinline__ int stage_slot32(int pp, int cc) { return 4 * pp + (cc ^ ((pp >> 1) & 3)); }
__device__ __forceinline__ int stage_slot16(int pp, int cc) { return 2 * pp + (cc ^ ((pp >> 2) & 1)); }

// v[16] = this lane's 16 FP32 channels of the tile at g (pixel pp at g + pp kCh).
__device__ __forceinline__ void tile_load_f32(const float *g, float4 *stg, int lane, float (&v)[16])
{
    __syncwarp();
    float4 t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        t[k] = __ldg(reinterpret_cast<const float4 *>(g + (8 * k + (lane >> 2)) * kCh + 4 * (lane & 3)));
#pragma unroll
    for (int k = 0; k < 4; ++k) stg[stage_slot32(8 * k + (lane >> 2), lane & 3)] = t[k];
    __syncwarp();
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const float4 x = stg[stage_slot32(lane, cc)];
        v[4 * cc] = x.x;
        v[4 * cc + 1] = x.y;
        v[4 * cc + 2] = x.z;
        v[4 * cc + 3] = x.w;
    }
}

// The tile at g = this lane's 16 FP32 channels v[16] (pixel pp at g + pp kCh).
__device__ __forceinline__ void tile_store_f32(float *g, float4 *stg, int lane, const float (&v)[16])
{
    __syncwarp();
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
        stg[stage_slot32(lane, cc)] = make_float4(v[4 * cc], v[4 * cc + 1], v[4 * cc + 2], v[4 * cc + 3]);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k)
        *reinterpret_cast<float4 *>(g + (8 * k + (lane >> 2)) * kCh + 4 * (lane & 3)) =
            stg[stage_slot32(8 * k + (lane >> 2), lane & 3)];
}

// 16 bfloat16 channels per pixel (first8 = channels off .. off + 7, last8 =
// off + 8 .. off + 15, packed) into activations `a`, pixels x0 .. x0 + 31 of
// row y of chain c, with the halo column copies of pixels 0 and L - 1.
__device__ __forceinline__ void tile_store_bf16(__nv_bfloat16 *a, int L, int64_t c, int y, int x0, int off,
                                                uint4 *stg, int lane, uint4 first8, uint4 last8)
{
    __syncwarp();
    stg[stage_slot16(lane, 0)] = first8;
    stg[stage_slot16(lane, 1)] = last8;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int pp = 16 * k + (lane >> 1), cc = lane & 1;
        store_act(a, L, c, y, x0 + pp, off + 8 * cc, stg[stage_slot16(pp, cc)]);
    }
}
static_assert(kAcc * kCh + 2 * kProjN <= (int)kRingTmemCols && 2 * kRingTmemCols <= 512, "TMEM columns");

struct RingConv {
    CUtensorMap tmap[kGroups];  // a_in viewed as (8 channels, L + 2 pixels, L rows, C chains), channel group g
    const __nv_bfloat16 *a_in;
    __nv_bfloat16 *a_out;  // nullable when PROJ
    __nv_bfloat16 *a_lo;   // BWD, nullable: bf16(dz_prev - bf16(dz_prev)) beside a_out (for the weight gradient)
    float *z_out;          // nullable
    float *P;              // PROJ: 9 planes of C L^2
    const float *zg;       // BWD: z of the layer below (FP32, NHWC) for gelu'
    float *d_out;          // BWD: dz of the layer below (FP32, NHWC)
    Chains ch;             // FUSED: the spins (flip[c], or -1, negated)
    const int32_t *flip;
    const __nv_bfloat16 *ta;  // FUSED: layer 1's table, 512 patterns x 32 channels
    const float *params;
    int w_off, b_off;
    Band bd;
    int segs;           // L / 128
    int units_per_col;  // ceil(bd.rows / kUnitRows)
    int64_t units;      // C segs units_per_col
    int withhold;       // self-test: never signal the first accumulator, so its wait runs out
};

struct RingUnit {
    int64_t c;
    int x0, r0, nrows;
};

__device__ __forceinline__ RingUnit ring_unit(const RingConv &p, int64_t u)
{
    RingUnit w;
    const int64_t col = u / p.units_per_col;
    const int rb = (int)(u - col * p.units_per_col);
    w.c = col / p.segs;
    w.x0 = (int)(col - w.c * p.segs) * kTileM;
    w.r0 = rb * kUnitRows;
    w.nrows = min(kUnitRows, p.bd.rows - w.r0);
    return w;
}

// Lattice row of band row r (-1 <= r <= rows) of chain c.
__device__ __forceinline__ int ring_row(const RingConv &p, int64_t c, int r)
{
    const int L = p.bd.L;
    int y = band_row0(p.bd, c) + r;
    y = y < 0 ? y + L : y;
    return y >= L ? y - L : y;
}

// Bit t of x (16 bits) moved to bit 2t.
__device__ __forceinline__ uint32_t bit_spread(uint32_t x)
{
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    return (x | (x << 1)) & 0x55555555u;
}

// Columns 32 b .. 32 b + 31 of spin row r of chain c as bits (1 = up), with
// block `flip` (or -1) negated.  Both planes' word b covers these columns:
// in row r the black spins sit at the columns of r's parity.
// The raw words behind spin_chunk: loaded one row ahead of their decoding in
// the fused loader, so that their latency overlaps the building of a row.
struct ChunkWords {
    uint64_t b, w;
    int r, blk;
};

__device__ __forceinline__ ChunkWords chunk_words(const Chains &ch, int64_t c, int r, int b)
{
    const int64_t at = (c * ch.L + r) * (int64_t)ch.wpr + b;
    return ChunkWords{ch.black[at], ch.white[at], r, b};
}

__device__ __forceinline__ uint32_t chunk_bits(const Chains &ch, const ChunkWords &k, int flip)
{
    const uint32_t kb = bit_spread(msc4_word_to_bits(k.b)), kw = bit_spread(msc4_word_to_bits(k.w));
    uint32_t v = (k.r & 1) ? (kw | (kb << 1)) : (kb | (kw << 1));
    if (flip >= 0) {
        const int nb = ch.L / kBlk, by = flip / nb, bx = flip - by * nb;
        if ((k.r >> 3) == by && ((bx * kBlk) >> 5) == k.blk) v ^= 0xFFu << ((bx * kBlk) & 31);
    }
    return v;
}

template <bool PROJ, bool BWD, bool FUSED>
__global__ void __launch_bounds__(ring_threads<PROJ, FUSED>(), 2) conv32_ring_kernel(const __grid_constant__ RingConv p)
{
    extern __shared__ __align__(1024) uint8_t ring_smem[];
    // the data-gradient kernel and the training forward of the first 32 -> 32
    // layer (neither fused with layer 1 nor projecting) stage their epilogue I/O
    constexpr bool STAGE = BWD || (!PROJ && !FUSED);
    using Lay = RingLayout<PROJ, STAGE>;
    uint8_t *ring = ring_smem + Lay::ring;
    uint8_t *a3s = ring_smem + Lay::a3;
    uint8_t *sB = ring_smem + Lay::b;
    uint8_t *sW4 = ring_smem + Lay::w4;
    float *sBias = reinterpret_cast<float *>(ring_smem + Lay::bias);
    uint64_t *full = reinterpret_cast<uint64_t *>(ring_smem + Lay::bar);
    uint64_t *empty = full + kRing, *accf = empty + kRing, *acce = accf + kAcc;
    uint64_t *a3full = acce + kAcc, *a3empty = a3full + 2, *pfull = a3empty + 2, *pempty = pfull + 2;
    uint64_t *drain = pempty + 2, *pdrain = drain + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(pdrain + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = p.bd.L;

    if (warp == 1) tc::tmem_alloc(tslot, kRingTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < kAcc; ++a) {
            tc::mbar_init(&accf[a], 1);
            tc::mbar_init(&acce[a], kEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&a3full[b], kEpiWarps);
            tc::mbar_init(&a3empty[b], 1);
            tc::mbar_init(&pfull[b], 1);
            tc::mbar_init(&pempty[b], 4);
        }
        tc::mbar_init(drain, 1);
        tc::mbar_init(pdrain, 1);
        tc::fence_mbar_init();
    }
    for (int e = tid; e < kTaps * kGroups * kCh; e += blockDim.x) {
        const int k = e / (kGroups * kCh), r = e - k * (kGroups * kCh), g = r / kCh, n = r - g * kCh;
        // forward: row n = output channel o, K = input channels 8g .. 8g+7 of tap k;
        // BWD: row n = input channel i, K = output channels 8g .. 8g+7 of tap 8 - k
        const int st = BWD ? kCh * 9 : 9;
        const float *w = p.params + p.w_off + (BWD ? ((8 * g) * kCh + n) * 9 + (8 - k) : (n * kCh + 8 * g) * 9 + k);
        // stacked operand of (dx, K half h): N = 96 rows, row 32 (dy + 1) + n,
        // K = channel groups 2h and 2h + 1 (LBO = 96 x 16 bytes, SBO = 128)
        const int dyi = k / 3, dxi = k % 3, h = g >> 1, gl = g & 1;
        *reinterpret_cast<uint4 *>(sB + ((((dxi * 2 + h) * 2 + gl) * kStackN) + kCh * dyi + n) * 16) =
            make_uint4(pack_bf16x2(w[0], w[st]), pack_bf16x2(w[2 * st], w[3 * st]),
                       pack_bf16x2(w[4 * st], w[5 * st]), pack_bf16x2(w[6 * st], w[7 * st]));
    }
    if (PROJ) {
        // W4^T as an N = 16 x K = 32 operand: row n = tap n (zero for n >= 9),
        // channel group g = input channels 8g .. 8g+7; W4[i][k] at kOffW4 + 9 i + k
        for (int e = tid; e < kGroups * kProjN; e += blockDim.x) {
            const int g = e / kProjN, n = e - g * kProjN;
            uint32_t u[4] = {0u, 0u, 0u, 0u};
            if (n < 9) {
                const float *w = p.params + kOffW4 + (8 * g) * 9 + n;
                for (int j = 0; j < 4; ++j) u[j] = pack_bf16x2(w[(2 * j) * 9], w[(2 * j + 1) * 9]);
            }
            *reinterpret_cast<uint4 *>(sW4 + e * 16) = make_uint4(u[0], u[1], u[2], u[3]);
        }
    }
    if (tid < kCh) sBias[tid] = BWD ? 0.0f : bf16r(p.params[p.b_off + tid]);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tproj = tmem + (uint32_t)(kAcc * kCh);
    // every accumulator block starts at the bias (zero in BWD), so that all
    // MMAs accumulate onto it
    if (warp >= 2 && warp < 2 + kEpiWarps) {
        const int quad = warp & 3, half = (warp - 2) >> 2;
        float bias[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) bias[i] = sBias[16 * half + i];
        for (int a = 0; a < kAcc; ++a) tc::tmem_st16(tmem + (uint32_t)(a * kCh + 16 * half) + ((uint32_t)(quad * 32) << 16), bias);
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    bool ok = true;

    if ((warp == 0 || warp == kRingExtra) && FUSED) {
        // two loader warps building the rows of a1 from the spins: warp 0 the
        // rows of even ring index, the other warp those of odd index (one
        // warp building rows is a chain of shuffles, table loads and stores
        // that the MMA thread outpaces)
        const uint32_t parity = warp == 0 ? 0u : 1u;
        uint32_t n = 0;  // ring index of the unit's first row
        const uint4 *ta = reinterpret_cast<const uint4 *>(p.ta);
        const int nw = L / 32;
        for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
            const RingUnit w = ring_unit(p, u);
            const int fb = p.flip ? p.flip[w.c] : -1;
            // lane 6 d + q (d < 3, q < 6): chunk x0 / 32 - 1 + q (periodic) of spin row y - 1 + d
            auto fetch = [&](int j) {
                ChunkWords k{0, 0, 0, 0};
                if (lane < 18) {
                    const int y = ring_row(p, w.c, w.r0 + j);
                    const int d = lane / 6, q = lane - 6 * d;
                    k = chunk_words(p.ch, w.c, wrap(y - 1 + d, L), (w.x0 / 32 - 1 + q + nw) % nw);
                }
                return k;
            };
            // this warp's rows j of the unit: ring index n + j + 1 of its parity
            const int j0 = -1 + (int)((parity - n) & 1u);
            ChunkWords next = j0 <= w.nrows ? fetch(j0) : ChunkWords{0, 0, 0, 0};
            for (int j = j0; j <= w.nrows; j += 2) {
                const uint32_t nn = n + (uint32_t)(j + 1);
                const uint32_t s = nn & (kRing - 1);
                const ChunkWords cur = next;
                if (j + 2 <= w.nrows) next = fetch(j + 2);  // in flight while row j is built
                if (nn >= kRing &&
                    !__all_sync(0xffffffffu, tc::mbar_wait(&empty[s], ((nn / kRing) + 1) & 1, kWaitCycles))) {
                    ok = false;
                    break;
                }
                const uint32_t bits = lane < 18 ? chunk_bits(p.ch, cur, fb) : 0u;
                uint8_t *dst = ring + s * kRowBytes;
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const int e = lane + 32 * i;   // entry e is column x0 - 1 + e
                    const int o = e + 30;          // column x0 - 2 + e relative to the window start x0 - 32
                    const int wi = o >> 5, sh = o & 31;
                    uint32_t pat = 0;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const uint32_t lo = __shfl_sync(0xffffffffu, bits, 6 * d + min(wi, 5));
                        const uint32_t hi = __shfl_sync(0xffffffffu, bits, 6 * d + min(wi + 1, 5));
                        const uint32_t trip = (uint32_t)((((uint64_t)hi << 32) | lo) >> sh) & 7u;
                        pat |= trip << (3 * d);
                    }
                    if (e < kTileM + 2) {
#pragma unroll
                        for (int g = 0; g < kGroups; ++g)
                            *reinterpret_cast<uint4 *>(dst + g * kRingPlane + e * 16) = __ldg(ta + pat * kGroups + g);
                    }
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&full[s]);
            }
            n += (uint32_t)(w.nrows + 2);
        }
    } else if (warp == 0) {
        // loader
        if (lane == 0) {
            uint32_t n = 0;  // rows staged so far
            for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
                const RingUnit w = ring_unit(p, u);
                for (int j = -1; j <= w.nrows; ++j, ++n) {
                    const uint32_t s = n & (kRing - 1);
                    if (n >= kRing && !tc::mbar_wait(&empty[s], ((n / kRing) + 1) & 1, kWaitCycles)) {
                        ok = false;
                        break;
                    }
                    const int y = ring_row(p, w.c, w.r0 + j);
                    tc::mbar_arrive_expect_tx(&full[s], kGroups * (kTileM + 2) * 16);
                    uint8_t *dst = ring + s * kRowBytes;
#pragma unroll
                    for (int g = 0; g < kGroups; ++g)
                        tc::tma_load_4d(dst + g * kRingPlane, &p.tmap[g], 0, w.x0, y, (int)w.c, &full[s]);
                }
            }
            // on a failure no copy may still be writing into shared memory when the CTA exits:
            // wait (bounded) for the last rows issued
            if (!ok)
                for (uint32_t m = n > kRing ? n - kRing : 0; m < n; ++m)
                    tc::mbar_wait(&full[m & (kRing - 1)], (m / kRing) & 1, kWaitCycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // N = 32, 64 or 96: one, two or three accumulator blocks per MMA
            // (the N field holds N / 8 from bit 17)
            const uint32_t idesc0 = tc::idesc_bf16_f32(kTileM, 0);
            const uint32_t ring_u32 = tc::smem_u32(ring), b_u32 = tc::smem_u32(sB);
            // descriptors of the ring's first byte and of the stacked weights'
            // first byte, as 32-bit words (the MMAs add offsets to the low words)
            const uint64_t a_desc0 = tc::smem_desc(ring_u32, kRingPlane, 128);
            const uint64_t b_desc0 = tc::smem_desc(b_u32, kStackN * 16, 128);
            const uint32_t a_lo0 = (uint32_t)a_desc0, a_hi = (uint32_t)(a_desc0 >> 32);
            const uint32_t b_lo0 = (uint32_t)b_desc0, b_hi = (uint32_t)(b_desc0 >> 32);
            // Row-stationary: staged input row i of a unit is multiplied once,
            // for each (dx, K half), by the three dy taps stacked along N, into
            // the accumulator blocks of the output rows it feeds, i + 1 (dy =
            // -1), i and i - 1 (dy = +1), those of them inside the unit.  Output
            // row t (counted over the units) has block kAcc - 1 - t % kAcc, so
            // rows i + 1, i, i - 1 have consecutive blocks and one MMA covers
            // them, two where the window passes the last block.  Every output
            // element still accumulates its 18 K steps in the order dy, dx, K.
            // (One M128 x N96 MMA costs a third of three N32 ones: the tensor
            // core takes ~45 cycles per N32 MMA and ~56 per N96 one.)
            uint32_t n0 = 0, t = 0, ready = 0;  // n0: ring index of the unit's row -1; t: rows of the units before
            for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
                const RingUnit w = ring_unit(p, u);
                for (int i = -1; i <= w.nrows && ok; ++i) {
                    while (ready < n0 + (uint32_t)(i + 2) && ok) {
                        if (!tc::mbar_wait(&full[ready & (kRing - 1)], (ready / kRing) & 1u, kWaitCycles)) ok = false;
                        ++ready;
                    }
                    // row i + 1 enters its block now: the block's last row must be read out
                    if (ok && i + 1 < w.nrows) {
                        const uint32_t tn = t + (uint32_t)(i + 1);
                        if (tn >= (uint32_t)kAcc &&
                            !tc::mbar_wait(&acce[ring_blk(tn)], (ring_use(tn) + 1u) & 1u, kWaitCycles))
                            ok = false;
                    }
                    if (!ok) break;
                    tc::fence_after_sync();
                    const int o_hi = min(i + 1, w.nrows - 1), o_lo = max(i - 1, 0);
                    const int cnt = o_hi - o_lo + 1;                    // blocks of the window (1 .. 3)
                    const int b0 = ring_blk(t + (uint32_t)o_hi);        // its first block
                    const int len0 = min(cnt, kAcc - b0);               // blocks before the wrap
                    const uint32_t dy0 = (uint32_t)(i - o_hi + 1);      // dy + 1 of the first block
                    const uint32_t row_lo = a_lo0 + (((n0 + (uint32_t)(i + 1)) & (kRing - 1)) * kRowBytes >> 4);
                    const uint32_t idesc_a = idesc0 | ((uint32_t)(len0 * kCh / 8) << 17);
                    const uint32_t idesc_b = idesc0 | ((uint32_t)((cnt - len0) * kCh / 8) << 17);
#pragma unroll
                    for (int st = 0; st < 6; ++st) {
                        const int dxi = st >> 1, h = st & 1;
                        const uint32_t a_lo = row_lo + ((2 * h * kRingPlane + dxi * 16) >> 4);
                        const uint32_t b_lo =
                            b_lo0 + ((uint32_t)((dxi * 2 + h) * 2 * kStackN * 16) >> 4) + dy0 * (kCh * 16 >> 4);
                        tc::mma_bf16_w(tmem + (uint32_t)(b0 * kCh), a_lo, a_hi, b_lo, b_hi, idesc_a, 1u);
                        if (len0 < cnt)
                            tc::mma_bf16_w(tmem, a_lo, a_hi, b_lo + (uint32_t)len0 * (kCh * 16 >> 4), b_hi, idesc_b, 1u);
                    }
                    tc::mma_commit(&empty[(n0 + (uint32_t)(i + 1)) & (kRing - 1)]);  // no later MMA reads row i
                    if (i >= 1) {
                        const uint32_t td = t + (uint32_t)(i - 1);  // row i - 1 has all 18 steps now
                        if (!(p.withhold && td == 0)) tc::mma_commit(&accf[ring_blk(td)]);
                    }
                }
                n0 += (uint32_t)(w.nrows + 2);
                t += (uint32_t)w.nrows;
            }
            // every MMA has completed before the TMEM is freed
            tc::mma_commit(drain);
            tc::mbar_wait(drain, 0, kWaitCycles);
        }
        __syncwarp();
    } else if (PROJ && warp == kRingExtra) {
        if (lane == 0) {
            // layer 4's channel contraction of every output row s, in order,
            // once the epilogue has staged its a3 (a3full) and read the P of
            // row s - 2 out of the same TMEM columns (pempty)
            const uint32_t idesc_p = tc::idesc_bf16_f32(kTileM, kProjN);
            const uint32_t a3_u32 = tc::smem_u32(a3s), w4_u32 = tc::smem_u32(sW4);
            int64_t rows = 0;
            for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) rows += ring_unit(p, u).nrows;
            for (int64_t s = 0; s < rows && ok; ++s) {
                const int b = (int)(s & 1);
                if (!tc::mbar_wait(&a3full[b], (uint32_t)((s >> 1) & 1), kWaitCycles) ||
                    (s >= 2 && !tc::mbar_wait(&pempty[b], (uint32_t)(((s >> 1) + 1) & 1), kWaitCycles))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ad = tc::smem_desc(a3_u32 + b * kRowBytes + 2 * h * kRingPlane, kRingPlane, 128);
                    const uint64_t bd = tc::smem_desc(w4_u32 + 2 * h * kProjN * 16, kProjN * 16, 128);
                    tc::mma_bf16(tproj + (uint32_t)(b * kProjN), ad, bd, idesc_p, h > 0 ? 1u : 0u);
                }
                tc::mma_commit(&pfull[b]);
                tc::mma_commit(&a3empty[b]);
            }
            // its MMAs have completed before the TMEM is freed
            tc::mma_commit(pdrain);
            tc::mbar_wait(pdrain, 0, kWaitCycles);
        }
        __syncwarp();
    } else if (warp < 2 + kEpiWarps) {
        const int quad = warp & 3, half = (warp - 2) >> 2, m = quad * 32 + lane;
        // STAGE: this warp's staging tile
        float4 *stg = reinterpret_cast<float4 *>(ring_smem + Lay::stage + (uint32_t)(warp - 2) * kStageBytes);
        uint4 *st16 = reinterpret_cast<uint4 *>(stg);
        const int xw = 32 * quad;  // the warp's first pixel in the tile (add w.x0)
        float bias[16];  // this warp's 16 channels (zero in BWD)
#pragma unroll
        for (int i = 0; i < 16; ++i) bias[i] = sBias[16 * half + i];
        int64_t t = 0;
        for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
            const RingUnit w = ring_unit(p, u);
            for (int j = 0; j < w.nrows; ++j, ++t) {
                const int a = ring_blk((uint32_t)t);
                const int y = ring_row(p, w.c, w.r0 + j);
                const int64_t q = (w.c * L + y) * (int64_t)L + w.x0 + m;
                // BWD: gelu'(z_prev) of this row does not depend on the
                // accumulator; load (through the warp's tile: q0 is the
                // warp's first pixel) and evaluate it while the MMAs run
                const int64_t q0 = q - lane;
                float gz[16];
                if constexpr (BWD) {
                    tile_load_f32(p.zg + q0 * kCh + 16 * half, stg, lane, gz);
#pragma unroll
                    for (int i = 0; i < 16; i += 2) gelu_grad2(gz[i], gz[i + 1]);
                }
                if (!__all_sync(0xffffffffu, tc::mbar_wait(&accf[a], ring_use((uint32_t)t) & 1u, kWaitCycles))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                float v[16];
                const uint32_t ta = tmem + (uint32_t)(a * kCh + 16 * half) + ((uint32_t)(quad * 32) << 16);
                tc::tmem_ld16(ta, v);
                // the block's next row accumulates onto the bias
                tc::tmem_st16(ta, bias);
                tc::tmem_wait_st();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acce[a]);
                if constexpr (BWD) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] *= gz[i];
                    tile_store_f32(p.d_out + q0 * kCh + 16 * half, stg, lane, v);
                    if (p.a_out) {
                        uint32_t hb[2][4], rb[2][4];
#pragma unroll
                        for (int h8 = 0; h8 < 2; ++h8) {
                            float v8[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) v8[i] = v[8 * h8 + i];
                            split_bf16(v8, hb[h8], rb[h8]);
                        }
                        tile_store_bf16(p.a_out, L, w.c, y, w.x0 + xw, 16 * half, st16, lane,
                                        make_uint4(hb[0][0], hb[0][1], hb[0][2], hb[0][3]),
                                        make_uint4(hb[1][0], hb[1][1], hb[1][2], hb[1][3]));
                        if (p.a_lo)
                            tile_store_bf16(p.a_lo, L, w.c, y, w.x0 + xw, 16 * half, st16, lane,
                                            make_uint4(rb[0][0], rb[0][1], rb[0][2], rb[0][3]),
                                            make_uint4(rb[1][0], rb[1][1], rb[1][2], rb[1][3]));
                    }
                } else {
                    if (p.z_out) {
                        if constexpr (STAGE) {
                            tile_store_f32(p.z_out + q0 * kCh + 16 * half, stg, lane, v);
                        } else {
                            float4 *zo = reinterpret_cast<float4 *>(p.z_out + q * kCh + 16 * half);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                zo[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                        }
                    }
                    uint32_t pk[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float g0 = v[2 * i], g1 = v[2 * i + 1];
                        gelu2(g0, g1);
                        pk[i] = pack_bf16x2(g0, g1);
                    }
                    if (p.a_out) {
                        if constexpr (STAGE) {
                            tile_store_bf16(p.a_out, L, w.c, y, w.x0 + xw, 16 * half, st16, lane,
                                            make_uint4(pk[0], pk[1], pk[2], pk[3]), make_uint4(pk[4], pk[5], pk[6], pk[7]));
                        } else {
                            store_act(p.a_out, L, w.c, y, w.x0 + m, 16 * half, make_uint4(pk[0], pk[1], pk[2], pk[3]));
                            store_act(p.a_out, L, w.c, y, w.x0 + m, 16 * half + 8,
                                      make_uint4(pk[4], pk[5], pk[6], pk[7]));
                        }
                    }
                    if (PROJ) {
                        const int b = (int)(t & 1);
                        if (t >= 2 && !__all_sync(0xffffffffu, tc::mbar_wait(&a3empty[b], (uint32_t)(((t >> 1) + 1) & 1),
                                                                              kWaitCycles))) {
                            ok = false;
                            break;
                        }
                        uint8_t *dst = a3s + b * kRowBytes + 2 * half * kRingPlane + m * 16;
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4 *>(dst + kRingPlane) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        tc::fence_async_smem();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&a3full[b]);
                    }
                }
            }
        }
    } else if (PROJ && warp > kRingExtra && warp <= kRingExtra + kProjWarps) {
        // P of every output row, pixel lane 32 quad + lane: waits for the
        // projection (pfull), reads its 16 TMEM columns, frees them (pempty,
        // four arrivals) and stores the 9 taps as FP32 planes P[k][pixel]
        const int quad = warp & 3, m = quad * 32 + lane;
        int64_t s = 0;
        for (int64_t u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
            const RingUnit w = ring_unit(p, u);
            for (int j = 0; j < w.nrows; ++j, ++s) {
                const int b = (int)(s & 1);
                if (!__all_sync(0xffffffffu, tc::mbar_wait(&pfull[b], (uint32_t)((s >> 1) & 1), kWaitCycles))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                float pv[16];
                tc::tmem_ld16(tproj + (uint32_t)(b * kProjN) + ((uint32_t)(quad * 32) << 16), pv);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&pempty[b]);
                // row partials of z4 (see pool_rows_kernel): P_k of this pixel
                // (y, x), tap k = 3 (dy + 1) + (dx + 1), goes to z4 at (y - dy,
                // x - dx); per dy, the part that stays in the pixel's 8 x 8
                // block column is summed over the block's 8 pixels (xor tree),
                // the block's first pixel sends its dx = +1 part to the block on
                // the left and its last pixel its dx = -1 part to the right
                const int y = ring_row(p, w.c, w.r0 + j);
                const int x = w.x0 + m, u = lane & 7, bx = x / kBlk, nb1 = L / kBlk;
                float *Rrow = p.P + (w.c * L + y) * (int64_t)(9 * nb1) + bx;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    float own = pv[3 * d + 1];
                    if (u != 0) own += pv[3 * d + 2];
                    if (u != 7) own += pv[3 * d];
                    own += __shfl_xor_sync(0xffffffffu, own, 1);
                    own += __shfl_xor_sync(0xffffffffu, own, 2);
                    own += __shfl_xor_sync(0xffffffffu, own, 4);
                    if (u == 0) {
                        Rrow[(3 * d + 0) * nb1] = own;
                        Rrow[(3 * d + 1) * nb1] = pv[3 * d + 2];
                    }
                    if (u == 7) Rrow[(3 * d + 2) * nb1] = pv[3 * d];
                }
            }
        }
    }
    if (!ok) atomicExch(&g_tc_error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kRingTmemCols);
    }
}

// Layer 4's channel contraction for the general conv kernel: thread per pixel
// of the band, P[k][q] = sum_i W4[i][k] a3(q)[i] (i in order).
__global__ void __launch_bounds__(kThreads) l4_project_kernel(Band bd, const float *params, const __nv_bfloat16 *a3,
                                                              float *P)
{
    __shared__ float W[kN1];  // W4[i][k] at 9 i + k
    for (int i = threadIdx.x; i < kN1; i += blockDim.x) W[i] = bf16r(params[kOffW4 + i]);
    __syncthreads();
    const int L = bd.L;
    const int64_t npix = bd.C * (int64_t)L * L;
    const int64_t n = bd.C * (int64_t)bd.rows * L;
    for (int64_t pb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pb < n; pb += (int64_t)gridDim.x * blockDim.x) {
        int64_t c;
        int yx;
        band_pixel(bd, pb, c, yx);
        const int64_t q = c * (int64_t)L * L + yx;
        const int y = yx / L;
        const uint4 *src = reinterpret_cast<const uint4 *>(a3 + apix(L, c, y, yx - y * L) * kCh);
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint4 v = __ldg(src + g);
            const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float lo = bf16_lo(u[j]), hi = bf16_hi(u[j]);
                const int i = 8 * g + 2 * j;
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = fmaf(W[(i + 1) * 9 + k], hi, fmaf(W[i * 9 + k], lo, acc[k]));
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k * npix + q] = acc[k];
    }
}

// Layer 4 and the block mean from the projections: z4(y, x) = b4 + sum over
// taps k of P[k](y + dy_k, x + dx_k).  Warp per (chain, block row, group of 4
// blocks) over `brows` block rows per chain (all of them in a full pass; in a
// band pass the flipped block's row and its two neighbours): lane l owns
// pixel column 8 b + l of the group and walks the block's 8 rows (taps in
// order, rows in order), so every load of a tap plane is 32 consecutive
// floats; the 8 lanes of a block then add up in a fixed shuffle tree.
__global__ void __launch_bounds__(kThreads) pool_kernel(int L, int64_t C, int brows, const int32_t *flip,
                                                        const float *params, const float *P, float *logits)
{
    const float b4 = bf16r(params[kOffB4]);
    const int nb1 = L / kBlk, nb = nb1 * nb1, groups = nb1 / 4;
    const int lane = threadIdx.x & 31;
    const int64_t npix = C * (int64_t)L * L;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int per = brows * groups;
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < C * per; wi += nw) {
        const int64_t c = wi / per;
        const int r = (int)(wi - c * per), rb = r / groups, bg = r - rb * groups;
        int by = rb;
        if (flip) {
            const int f = flip[c];
            by = wrap((f < 0 ? 0 : f / nb1) - 1 + rb, nb1);
        }
        const float *Pc = P + c * (int64_t)L * L;
        const int x = bg * 32 + lane;
        const int xs[3] = {wrap(x - 1, L), x, wrap(x + 1, L)};
        float part = 0.0f;
        // unrolled: the loads of all 8 rows are issued before the sums (same order of additions)
#pragma unroll
        for (int yy = by * kBlk; yy < by * kBlk + kBlk; ++yy) {
            const int ys[3] = {wrap(yy - 1, L), yy, wrap(yy + 1, L)};
            float z = b4;
#pragma unroll
            for (int k = 0; k < 9; ++k) z += __ldg(Pc + k * npix + ys[k / 3] * (int64_t)L + xs[k % 3]);
            part += z;
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if ((lane & 7) == 0) logits[c * nb + by * nb1 + 4 * bg + (lane >> 3)] = part * (1.0f / (kBlk * kBlk));
    }
}

// The block logits from the row partials the projecting ring kernel writes
// (L a multiple of 128): R[c][y][3 dy' + j][bx], dy' = dy + 1, holds for the
// P values of row y with tap row dy (they feed z4 in row y - dy)
//   j = 0: the sum over block column bx of the parts that stay in it,
//   j = 1: the dx = +1 part of the block's first pixel (feeds block bx - 1),
//   j = 2: the dx = -1 part of the block's last pixel (feeds block bx + 1),
// so that sum over the block of z4 = 64 b4 + sum over its 8 rows y' and the
// three dy of R[y' + dy][dy'][0][bx] + R[..][dy'][2][bx - 1] + R[..][dy'][1][bx + 1]
// (periodic), added in that fixed order.  Thread per logit.
__global__ void __launch_bounds__(kThreads) pool_rows_kernel(int L, int64_t C, int brows, const int32_t *flip,
                                                             const float *params, const float *R, float *logits)
{
    const float b4 = bf16r(params[kOffB4]);
    const int nb1 = L / kBlk, nb = nb1 * nb1;
    const int64_t n = C * brows * nb1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / (brows * nb1);
        const int r = (int)(e - c * brows * nb1), rb = r / nb1, bx = r - rb * nb1;
        int by = rb;
        if (flip) {
            const int f = flip[c];
            by = wrap((f < 0 ? 0 : f / nb1) - 1 + rb, nb1);
        }
        const int bl = bx == 0 ? nb1 - 1 : bx - 1, br = bx + 1 == nb1 ? 0 : bx + 1;
        float sum = 0.0f;
#pragma unroll
        for (int yy = 0; yy < kBlk; ++yy) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int y = wrap(by * kBlk + yy + d - 1, L);  // the source row of tap row dy = d - 1
                const float *Rr = R + (c * L + y) * (int64_t)(9 * nb1) + 3 * d * nb1;
                sum += __ldg(Rr + bx) + __ldg(Rr + 2 * nb1 + bl) + __ldg(Rr + nb1 + br);
            }
        }
        logits[c * nb + by * nb1 + bx] = b4 + sum * (1.0f / (kBlk * kBlk));
    }
}

// ---------------------------------------------------------------------------
// Backward (uses z1..z3, a1..a3 stored by a training forward)
// ---------------------------------------------------------------------------
// dz3 = gelu'(z3) * sum_k W4[i][k] * d4(p - off_k),  d4(p) = dlogit(block of p) / 64.
__global__ void __launch_bounds__(kThreads) l4_bwd_data_kernel(int L, int64_t C, const float *params,
                                                               const float *dlogits, const float *z3, float *dz3,
                                                               __nv_bfloat16 *dz3b, __nv_bfloat16 *dz3r)
{
    __shared__ float W[kN1];
    for (int i = threadIdx.x; i < kN1; i += blockDim.x) W[i] = bf16r(params[kOffW4 + i]);
    __syncthreads();
    const int nb1 = L / kBlk;
    const int64_t npix = C * (int64_t)L * L;
    // four threads per pixel, 8 channels each: a warp reads and writes 8
    // pixels' 1 KB of z3 / dz3 contiguously
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 4 * npix;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e >> 2;
        const int i8 = (int)(e & 3) * 8;
        const int64_t c = p / ((int64_t)L * L);
        const int yx = (int)(p - c * (int64_t)L * L);
        const int y = yx / L, x = yx - y * L;
        float d[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            // output pixel q = p - off_k used input p through tap k
            int yy = y - (k / 3 - 1), xx = x - (k % 3 - 1);
            yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
            xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
            d[k] = dlogits[c * nb1 * nb1 + (yy / kBlk) * nb1 + xx / kBlk] * (1.0f / (kBlk * kBlk));
        }
        const float4 *zp = reinterpret_cast<const float4 *>(z3 + p * kCh + i8);
        const float4 za = zp[0], zb = zp[1];
        const float z[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        float v[8], gz[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) gz[i] = z[i];
#pragma unroll
        for (int i = 0; i < 8; i += 2) gelu_grad2(gz[i], gz[i + 1]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float g = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) g = fmaf(W[(i8 + i) * 9 + k], d[k], g);
            v[i] = g * gz[i];
        }
        float4 *out = reinterpret_cast<float4 *>(dz3 + p * kCh + i8);
        out[0] = make_float4(v[0], v[1], v[2], v[3]);
        out[1] = make_float4(v[4], v[5], v[6], v[7]);
        // bfloat16 copy with halo columns: the operand of the next data gradient on the tensor cores
        // (and, with the rounding of its remainder, of the weight gradient)
        if (dz3b) {
            uint32_t hb[4], rb[4];
            split_bf16(v, hb, rb);
            store_act(dz3b, L, c, y, x, i8, make_uint4(hb[0], hb[1], hb[2], hb[3]));
            if (dz3r) store_act(dz3r, L, c, y, x, i8, make_uint4(rb[0], rb[1], rb[2], rb[3]));
        }
    }
}

// dz_prev = gelu'(z_prev) * sum_{k, o} W[o][i][k] * bf16(dz(p - off_k)[o]);
// weights as Wt[k][o][i] (32 contiguous inputs per tap and output).  The
// incoming gradient is rounded to bfloat16, as on the tensor-core path.
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
                const float g4[4] = {bf16r(v.x), bf16r(v.y), bf16r(v.z), bf16r(v.w)};
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

// Weight gradients of a 32 -> 32 layer on the CUDA cores (L not a multiple of
// 128; wgrad_tc_kernel below serves the others), as per-CTA partial sums
// (fixed order).  The pixels are cut into tiles of 8 rows x 32 columns of one
// chain; CTA j handles tiles j, j + gridDim.x, ... in order.  A tile's output
// gradients dz (and the layer's input a, with a one-pixel halo) are staged in
// shared memory; thread (oq, iq) of 16 x 16 accumulates the 2 x 2 (output,
// input) channel pairs 2 oq + {0, 1} x 2 iq + {0, 1} for all 9 taps, and
// threads with iq = 0 the bias sums.  partial[cta][e]: e = (o * 32 + i) * 9 + k
// for weights, then the biases.
constexpr int kTy = 8, kTx = 32;

__device__ __forceinline__ void wgrad_stage(const Chains &ch, const __nv_bfloat16 *a_prev, const float *dz, int64_t c,
                                            int y0, int x0, float *sa, float *sd)
{
    const int L = ch.L;
    // input tile with halo: (kTy + 2) x (kTx + 2) pixels x 32 channels, as four
    // 16-byte loads of 8 bfloat16 per pixel
    constexpr int kOct = kCh / 8;
    for (int e = threadIdx.x; e < (kTy + 2) * (kTx + 2) * kOct; e += blockDim.x) {
        const int pix = e / kOct, q = e - pix * kOct;
        const int ty = pix / (kTx + 2), tx = pix - ty * (kTx + 2);
        int y = y0 + ty - 1, x = x0 + tx - 1;
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        x = x < 0 ? x + L : (x >= L ? x - L : x);
        const uint4 v = *reinterpret_cast<const uint4 *>(a_prev + apix(L, c, y, x) * kCh + 8 * q);
        float4 *dst = reinterpret_cast<float4 *>(sa + pix * kCh + 8 * q);
        dst[0] = make_float4(bf16_lo(v.x), bf16_hi(v.x), bf16_lo(v.y), bf16_hi(v.y));
        dst[1] = make_float4(bf16_lo(v.z), bf16_hi(v.z), bf16_lo(v.w), bf16_hi(v.w));
    }
    // output gradients of the tile: a tile row of 32 pixels x 32 channels is
    // contiguous, loaded as float4
    for (int e = threadIdx.x; e < kTy * kTx * kCh / 4; e += blockDim.x) {
        const int row = e / (kTx * kCh / 4), v = e - row * (kTx * kCh / 4);
        const float4 *src = reinterpret_cast<const float4 *>(dz + ((c * L + y0 + row) * (int64_t)L + x0) * kCh);
        reinterpret_cast<float4 *>(sd)[e] = src[v];
    }
}

__global__ void __launch_bounds__(256) wgrad_kernel(Chains ch, int64_t C, const __nv_bfloat16 *a_prev, const float *dz,
                                                    float *partial)
{
    extern __shared__ float smem[];
    float *sa = smem;                                 // (kTy+2) (kTx+2) 32
    float *sd = smem + (kTy + 2) * (kTx + 2) * kCh;   // kTy kTx 32
    constexpr int NE = kN2 + kCh;
    const int L = ch.L;
    const int tiles_x = L / kTx, tiles_y = L / kTy;
    const int64_t n_tiles = C * tiles_x * tiles_y;
    const int oq = threadIdx.x >> 4, iq = threadIdx.x & 15;  // channel pairs 2 oq, 2 oq + 1 and 2 iq, 2 iq + 1
    float acc[2][2][9];
    float bacc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[a][b][k] = 0.0f;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t c = tile / (tiles_x * tiles_y);
        const int rem = (int)(tile - c * tiles_x * tiles_y);
        const int y0 = (rem / tiles_x) * kTy, x0 = (rem % tiles_x) * kTx;
        __syncthreads();
        wgrad_stage(ch, a_prev, dz, c, y0, x0, sa, sd);
        __syncthreads();
        // pixels in row order; along a tile row the 3 x 3 input window slides
        // in registers, so each pixel loads one new column per dy (channel
        // pairs as float2)
        for (int ty = 0; ty < kTy; ++ty) {
            float2 win[3][3];  // [dy][dx], input channels 2 iq, 2 iq + 1
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx)
                    win[dy][dx] = *reinterpret_cast<const float2 *>(sa + ((ty + dy) * (kTx + 2) + dx) * kCh + 2 * iq);
#pragma unroll
            for (int tx = 0; tx < kTx; ++tx) {
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
                    win[dy][2] = *reinterpret_cast<const float2 *>(sa + ((ty + dy) * (kTx + 2) + tx + 2) * kCh + 2 * iq);
                const float2 g2 = *reinterpret_cast<const float2 *>(sd + (ty * kTx + tx) * kCh + 2 * oq);
                const float g[2] = {g2.x, g2.y};
#pragma unroll
                for (int a = 0; a < 2; ++a) bacc[a] += g[a];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float2 wv = win[k / 3][k % 3];
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        acc[a][0][k] = fmaf(g[a], wv.x, acc[a][0][k]);
                        acc[a][1][k] = fmaf(g[a], wv.y, acc[a][1][k]);
                    }
                }
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    win[dy][0] = win[dy][1];
                    win[dy][1] = win[dy][2];
                }
            }
        }
    }
    float *out = partial + (int64_t)blockIdx.x * NE;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int k = 0; k < 9; ++k) out[((2 * oq + a) * kCh + 2 * iq + b) * 9 + k] = acc[a][b][k];
    if (iq == 0)
#pragma unroll
        for (int a = 0; a < 2; ++a) out[kN2 + 2 * oq + a] = bacc[a];
}

// Weight gradients of the layers with one input or one output channel, warp
// per run of rows, lane per channel:
//   layer 1 (spins -> 32): dW1[o][k] = sum_p dz1(p)[o] s(p + off_k),
//                          db1[o] = sum_p dz1(p)[o]                (lane o);
//   layer 4 (32 -> 1):     dW4[i][k] = sum_q a3(q)[i] d4(q - off_k),
//                          db4 = sum_p d4(p), d4(p) = dlogit(block of p) / 64
//                                                                 (lane i).
// Per pixel q the lane's value v (dz1(q)[o] or a3(q)[i]) multiplies a 3 x 3
// window of a field that is the same for all lanes (the spins, or d4).  A
// warp walks its rows in order, each in chunks of 32 pixels: lane j holds the
// field at column x0 + j of rows y - 1, y, y + 1, the halo columns are loaded
// by every lane, and the window slides along the chunk by one shuffle per row
// and pixel.  Per pixel and lane: one load, three shuffles, nine FMAs.  The
// CTA's warps are added in warp order and written as the CTA's partial sums
// (layout of wgrad_kernel), summed by reduce_partials_kernel.  (wgrad_kernel
// gives these layers 16 busy threads per CTA.)
constexpr int kThinWarps = 8;

template <bool L4>
__device__ __forceinline__ float thin_field(const Chains &ch, const float *dlogits, int64_t c, int y, int x)
{
    const int L = ch.L;
    y = wrap(y, L);
    x = wrap(x, L);
    if constexpr (L4) {
        const int nb1 = L / kBlk;
        return dlogits[c * nb1 * nb1 + (y / kBlk) * nb1 + x / kBlk] * (1.0f / (kBlk * kBlk));
    } else {
        return spin_at(ch, c, y, x, -1);
    }
}

template <bool L4>
__global__ void __launch_bounds__(32 * kThinWarps, 2) wgrad_thin_kernel(Chains ch, int64_t C, const float *dz1,
                                                                      const __nv_bfloat16 *a3, const float *dlogits,
                                                                      float *partial)
{
    constexpr int NE = L4 ? kN1 + 1 : kN1 + kCh;
    __shared__ float red[kThinWarps][32][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = ch.L;
    const int64_t rows = C * L;
    const int64_t nw = (int64_t)gridDim.x * kThinWarps, gw = (int64_t)blockIdx.x * kThinWarps + warp;
    const int64_t r0 = gw * rows / nw, r1 = (gw + 1) * rows / nw;
    float acc[9], bacc = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    for (int64_t gr = r0; gr < r1; ++gr) {
        const int64_t c = gr / L;
        const int y = (int)(gr - c * L);
        for (int x0 = 0; x0 < L; x0 += 32) {
            float f[3], hl[3], hr[3], w[3][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                f[d] = thin_field<L4>(ch, dlogits, c, y - 1 + d, x0 + lane);
                hl[d] = thin_field<L4>(ch, dlogits, c, y - 1 + d, x0 - 1);
                hr[d] = thin_field<L4>(ch, dlogits, c, y - 1 + d, x0 + 32);
                w[d][0] = hl[d];
                w[d][1] = __shfl_sync(0xffffffffu, f[d], 0);
                w[d][2] = __shfl_sync(0xffffffffu, f[d], 1);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float v;
                if constexpr (L4) {
                    v = __bfloat162float(a3[apix(L, c, y, x0 + j) * kCh + lane]);
                    bacc += w[1][1];  // d4 of the pixel itself
                } else {
                    v = dz1[((c * L + y) * (int64_t)L + x0 + j) * kCh + lane];
                    bacc += v;
                }
                // window entry (d, e) is the field at (y - 1 + d, x + e - 1): tap
                // 3 d + e of layer 1 (p + off_k), tap 8 - 3 d - e of layer 4 (q - off_k)
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int k = L4 ? 8 - 3 * d - e : 3 * d + e;
                        acc[k] = fmaf(v, w[d][e], acc[k]);
                    }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    w[d][0] = w[d][1];
                    w[d][1] = w[d][2];
                    w[d][2] = j + 2 < 32 ? __shfl_sync(0xffffffffu, f[d], (j + 2) & 31) : hr[d];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) red[warp][lane][k] = acc[k];
    red[warp][lane][9] = bacc;
    __syncthreads();
    float *out = partial + (int64_t)blockIdx.x * NE;
    for (int t = threadIdx.x; t < 32 * 10; t += blockDim.x) {
        const int l = t / 10, k = t - 10 * l;
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < kThinWarps; ++q) sum += red[q][l][k];
        if (k < 9)
            out[l * 9 + k] = sum;  // layer 1: (o, k); layer 4: (i, k)
        else if (!L4)
            out[kN1 + l] = sum;    // db1[o]
        else if (l == 0)
            out[kN1] = sum;        // db4 (every lane summed the same d4)
    }
}

// grad[off + e] = sum over ctas of partial[cta][e] in a fixed order: warp w
// of a block sums the w-th eighth of the CTA range (in order) for 32
// consecutive e, then the eight warp sums are added in warp order.  Weights
// come first (W[o][i][k] order), then the biases.  Launch: ceil(ne / 32)
// blocks of 256 threads.
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(32 * kReduceWarps) reduce_partials_kernel(const float *partial, int64_t n_cta,
                                                                            int ne, int nw, float *grad, int w_off,
                                                                            int b_off)
{
    __shared__ float part[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int64_t k0 = n_cta * warp / kReduceWarps, k1 = n_cta * (warp + 1) / kReduceWarps;
    float s = 0.0f;
    if (e < ne)
        for (int64_t k = k0; k < k1; ++k) s += partial[k * ne + e];
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && e < ne) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < kReduceWarps; ++w) t += part[w][lane];
        if (e < nw)
            grad[w_off + e] = t;
        else
            grad[b_off + (e - nw)] = t;
    }
}

// Weight gradients of a 32 -> 32 layer on the tensor cores (L a multiple of
// 128).  With a the layer's input (bfloat16, halo columns) and dz the gradient
// of its pre-activations,
//   dW[o][i][k] = sum_p dz(p)[o] a(p + off_k)[i],   db[o] = sum_p dz(p)[o],
// off_k = (dy - 1, dx - 1) for tap k = 3 dy + dx.  Input row y' meets the
// gradient rows y' + 1, y', y' - 1 (dy = 0, 1, 2), so per 128-pixel row
// segment of input row y' there is one GEMM over the segment's 128 pixels (K):
//   D[m][n] += sum_x A_y'[m][x] B_y'[n][x]
// with M = 128 rows, of which rows m = 32 dx + i (dx = 0..2) are the input row
// shifted by dx - 1 and rows 96..127 are not used, and N = 192 columns
// n = 64 b + 32 h + o for the gradient rows y' - 1, y', y' + 1 (b = 0, 1, 2:
// dy = 2 - b), each as two bfloat16 parts, h = 0 its rounding and h = 1 the
// rounding of the remainder, so that a x (hi + lo) carries dz to about 2^-17
// and the FP32 accumulation sees the unrounded gradient to that accuracy
// (dW = D[.][64 b + o] + D[.][64 b + 32 + o]).  Eight MMAs of M128 x N192 x
// K16 per input row segment.
// Both operands are MN-major and come straight from the NHWC buffers: a
// tensor copy of 128 whole pixels (32 channels, 64 bytes each) with the
// 64-byte swizzle is the MN-major 64-byte-swizzled operand form: 8 K rows
// (pixels) of 64 bytes per 512-byte atom, SBO = 512 bytes between the 8-row
// groups along K, LBO = 8 KB between the 32-channel groups along M (or N).
// So every sector a copy fetches is used whole.  A staged input row is three
// such copies, of the row starting at pixels x0 - 1 + dx; the unused M rows
// 96..127 read the 8 KB after it (the next slot, or the first gradient slot
// after the last one), whose products land in TMEM lanes no one reads.  A
// staged gradient row is two copies (hi, lo) in a slot of a ring whose first
// two slots are also copied behind its last one, so that any three
// consecutive gradient rows lie at one stride (the N operand).
// Work: the (chain, segment, row) lines of all chains are cut into one
// contiguous range per CTA (ranges differ by at most one row); a range is
// walked as runs of consecutive gradient rows r0 .. r0 + n - 1 of one
// (chain, segment).  A run stages the input rows r0 - 1 .. r0 + n and the
// gradient rows r0 - 2 .. r0 + n + 1, those outside the run as zeros (tensor
// copies of a row past the lattice's last, which the copy fills with zeros),
// so that every (input row, gradient row) pair is counted by exactly one CTA.
// The accumulators (192 TMEM columns) collect the CTA's whole range; at the
// end they are written as the CTA's partial sums in the weight-gradient
// layout (e = (o CIN + i) 9 + k, then the biases).
// Warp roles (bounded mbarrier waits): warp 0 lane 0 issues the tensor
// copies; warp 1 lane 0 the MMAs; warps 2..5 add up every staged gradient row
// for the bias sums (fixed order; the zero rows add nothing) and, after the
// last MMA, read the accumulators.  A gradient slot is free once the MMAs of
// its last input row have completed and the four bias warps have read it.
constexpr int kWgActSlots = 3;                      // staged input rows
constexpr int kWgDzSlots = 4;                       // staged gradient rows (3 in use, 1 ahead)
constexpr int kWgDzMirror = 2;                      // slots 0, 1 repeated after the last
constexpr int kWgBiasWarps = 4;
constexpr uint32_t kWgBox = kTileM * kCh * 2;      // 128 pixels x 32 channels, bfloat16, 64-byte swizzled
constexpr uint32_t kWgActBytes = 3 * kWgBox;        // dx = 0, 1, 2
constexpr uint32_t kWgDzBytes = 2 * kWgBox;         // hi, lo
constexpr uint32_t kWgDz0 = kWgActSlots * kWgActBytes;
constexpr uint32_t kWgBias = kWgDz0 + (kWgDzSlots + kWgDzMirror) * kWgDzBytes;  // per bias warp 32 sums
constexpr uint32_t kWgBar = kWgBias + kWgBiasWarps * kCh * 4;
constexpr uint32_t kWgSmem = kWgBar + (2 * kWgActSlots + 2 * kWgDzSlots + 1) * 8 + 16;
constexpr int kWgThreads = 64 + 32 * kWgBiasWarps;
constexpr int kWgN = 6 * kCh;                       // three gradient rows, hi and lo
constexpr uint32_t kWgTmemCols = 256;               // 192 used
static_assert(kWgDz0 >= kWgActBytes + kWgBox && kWgSmem <= 227 * 1024 && kWgActBytes % 1024 == 0 &&
                  kWgDz0 % 1024 == 0,
              "the unused M rows of the last input slot read the gradient slots; one CTA per SM");

struct WgradTc {
    CUtensorMap act;  // a: (32 channels, L + 2 pixels, L rows, C chains), boxes 32 x 128 x 1 x 1, 64-byte swizzle
    CUtensorMap hi;   // bf16(dz), same layout
    CUtensorMap lo;   // bf16(dz - bf16(dz)), same layout
    float *partial;   // [gridDim.x][kN2 + kCh]
    int L, segs;
    int64_t lines;    // C segs L
};

// The run of this CTA's range that starts at line `lin`: chain, segment, first
// row and row count.
__device__ __forceinline__ RingUnit wg_run(const WgradTc &p, int64_t lin, int64_t end)
{
    RingUnit w;
    const int64_t col = lin / p.L;
    w.r0 = (int)(lin - col * p.L);
    w.nrows = (int)min((int64_t)(p.L - w.r0), end - lin);
    w.c = col / p.segs;
    w.x0 = (int)(col - w.c * p.segs) * kTileM;
    return w;
}

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_tc_kernel(const __grid_constant__ WgradTc p)
{
    extern __shared__ __align__(1024) uint8_t wg_smem[];
    float *bias_part = reinterpret_cast<float *>(wg_smem + kWgBias);
    uint64_t *afull = reinterpret_cast<uint64_t *>(wg_smem + kWgBar);
    uint64_t *aempty = afull + kWgActSlots, *dfull = aempty + kWgActSlots, *dempty = dfull + kWgDzSlots;
    uint64_t *drain = dempty + kWgDzSlots;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(drain + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = p.L;
    const int64_t begin = blockIdx.x * p.lines / gridDim.x, end = (blockIdx.x + 1) * p.lines / gridDim.x;

    if (warp == 1) tc::tmem_alloc(tslot, kWgTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kWgActSlots; ++s) {
            tc::mbar_init(&afull[s], 1);
            tc::mbar_init(&aempty[s], 1);
        }
        for (int s = 0; s < kWgDzSlots; ++s) {
            tc::mbar_init(&dfull[s], 1);
            tc::mbar_init(&dempty[s], 1 + kWgBiasWarps);
        }
        tc::mbar_init(drain, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t na = 0, nd = 0;  // input and gradient rows staged so far
            auto stage_act = [&](const RingUnit &w, int r) -> bool {
                const uint32_t s = na % kWgActSlots;
                if (na >= kWgActSlots && !tc::mbar_wait(&aempty[s], ((na / kWgActSlots) + 1) & 1, kWaitCycles))
                    return false;
                const int y = wrap(r, L);
                tc::mbar_arrive_expect_tx(&afull[s], kWgActBytes);
                uint8_t *dst = wg_smem + s * kWgActBytes;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) tc::tma_load_4d(dst + dx * kWgBox, &p.act, 0, w.x0 + dx, y, (int)w.c, &afull[s]);
                ++na;
                return true;
            };
            // gradient row r of the run, or zeros (row L, past the lattice) when r is outside it
            auto stage_dz = [&](const RingUnit &w, int r) -> bool {
                const uint32_t s = nd % kWgDzSlots;
                if (nd >= kWgDzSlots && !tc::mbar_wait(&dempty[s], ((nd / kWgDzSlots) + 1) & 1, kWaitCycles))
                    return false;
                const int y = (r >= w.r0 && r < w.r0 + w.nrows) ? r : L;
                const int copies = s < (uint32_t)kWgDzMirror ? 2 : 1;
                tc::mbar_arrive_expect_tx(&dfull[s], copies * kWgDzBytes);
                for (int k = 0; k < copies; ++k) {
                    uint8_t *dst = wg_smem + kWgDz0 + (s + k * kWgDzSlots) * kWgDzBytes;
                    tc::tma_load_4d(dst, &p.hi, 0, w.x0 + 1, y, (int)w.c, &dfull[s]);
                    tc::tma_load_4d(dst + kWgBox, &p.lo, 0, w.x0 + 1, y, (int)w.c, &dfull[s]);
                }
                ++nd;
                return true;
            };
            for (int64_t lin = begin; lin < end && ok;) {
                const RingUnit w = wg_run(p, lin, end);
                lin += w.nrows;
                // gradient rows r0 - 2, r0 - 1, then per input row r0 - 1 + a that row and gradient row r0 + a
                ok = stage_dz(w, w.r0 - 2) && stage_dz(w, w.r0 - 1);
                for (int a = 0; a < w.nrows + 2 && ok; ++a) ok = stage_act(w, w.r0 - 1 + a) && stage_dz(w, w.r0 + a);
            }
            // on a failure no copy may still be writing into shared memory when the CTA exits
            if (!ok) {
                for (uint32_t m = na > kWgActSlots ? na - kWgActSlots : 0; m < na; ++m)
                    tc::mbar_wait(&afull[m % kWgActSlots], (m / kWgActSlots) & 1, kWaitCycles);
                for (uint32_t m = nd > kWgDzSlots ? nd - kWgDzSlots : 0; m < nd; ++m)
                    tc::mbar_wait(&dfull[m % kWgDzSlots], (m / kWgDzSlots) & 1, kWaitCycles);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32_mn(kTileM, kWgN);
            const uint64_t a_desc0 = tc::smem_desc_sw64(tc::smem_u32(wg_smem), kWgBox, 512);
            const uint64_t b_desc0 = tc::smem_desc_sw64(tc::smem_u32(wg_smem + kWgDz0), kWgBox, 512);
            const uint32_t a_lo0 = (uint32_t)a_desc0, a_hi = (uint32_t)(a_desc0 >> 32);
            const uint32_t b_lo0 = (uint32_t)b_desc0, b_hi = (uint32_t)(b_desc0 >> 32);
            uint32_t ma = 0, md = 0, dready = 0;  // input rows consumed; first gradient row of the run; gradient rows landed
            bool first = true;
            for (int64_t lin = begin; lin < end && ok;) {
                const RingUnit w = wg_run(p, lin, end);
                lin += w.nrows;
                for (int a = 0; a < w.nrows + 2 && ok; ++a) {
                    // input row r0 - 1 + a meets gradient rows r0 - 2 + a .. r0 + a (indices md + a .. md + a + 2)
                    while (dready < md + (uint32_t)a + 3 && ok) {
                        if (!tc::mbar_wait(&dfull[dready % kWgDzSlots], (dready / kWgDzSlots) & 1u, kWaitCycles))
                            ok = false;
                        ++dready;
                    }
                    const uint32_t as = ma % kWgActSlots;
                    if (ok && !tc::mbar_wait(&afull[as], (ma / kWgActSlots) & 1u, kWaitCycles)) ok = false;
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t a_row = a_lo0 + ((as * kWgActBytes) >> 4);
                    const uint32_t b_row = b_lo0 + ((((md + (uint32_t)a) % kWgDzSlots) * kWgDzBytes) >> 4);
#pragma unroll
                    for (int ks = 0; ks < kTileM / 16; ++ks)  // 16 pixels = two 512-byte atoms
                        tc::mma_bf16_w(tmem, a_row + (uint32_t)(ks * 64), a_hi, b_row + (uint32_t)(ks * 64), b_hi, idesc,
                                       (first && ks == 0) ? 0u : 1u);
                    first = false;
                    tc::mma_commit(&aempty[as]);
                    ++ma;
                    tc::mma_commit(&dempty[(md + (uint32_t)a) % kWgDzSlots]);  // gradient row r0 - 2 + a: last use
                }
                if (!ok) break;
                tc::mma_commit(&dempty[(md + (uint32_t)w.nrows + 2) % kWgDzSlots]);
                tc::mma_commit(&dempty[(md + (uint32_t)w.nrows + 3) % kWgDzSlots]);
                md += (uint32_t)w.nrows + 4;
            }
            // every MMA has completed before the accumulators are read and the TMEM is freed
            tc::mma_commit(drain);
            if (!tc::mbar_wait(drain, 0, kWaitCycles)) ok = false;
        }
        __syncwarp();
    } else {
        // bias sums: bias warp q adds pixels 32 q .. 32 q + 31 of every staged
        // gradient row (the zero rows add nothing); lane = 4 p8 + g holds
        // channels 8 g .. 8 g + 7 of the pixels 32 q + 8 it + p8 (it = 0..3),
        // hi + lo.  In the 64-byte swizzle, channel group g of pixel px is the
        // 16-byte chunk g ^ ((px >> 1) & 3) of the pixel's 64 bytes.
        const int q = warp - 2, g = lane & 3, p8 = lane >> 2;
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
        int64_t staged = 0;  // gradient rows staged for this CTA: n + 4 per run
        for (int64_t lin = begin; lin < end;) {
            const RingUnit w = wg_run(p, lin, end);
            lin += w.nrows;
            staged += w.nrows + 4;
        }
        for (int64_t md = 0; md < staged; ++md) {
            const uint32_t ds = (uint32_t)(md % kWgDzSlots);
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&dfull[ds], (uint32_t)(md / kWgDzSlots) & 1u, kWaitCycles))) {
                ok = false;
                break;
            }
            const uint8_t *dz = wg_smem + kWgDz0 + ds * kWgDzBytes;
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int px = 32 * q + 8 * it + p8;
                const uint32_t at = px * 64 + ((g ^ ((px >> 1) & 3)) << 4);
                const uint4 h = *reinterpret_cast<const uint4 *>(dz + at);
                const uint4 l = *reinterpret_cast<const uint4 *>(dz + kWgBox + at);
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[2 * j] += bf16_lo(hw[j]) + bf16_lo(lw[j]);
                    acc[2 * j + 1] += bf16_hi(hw[j]) + bf16_hi(lw[j]);
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&dempty[ds]);
        }
        // lanes of one channel group (lane ^ 4, ^ 8, ^ 16), then the four warps in order
#pragma unroll
        for (int sh = 4; sh < 32; sh <<= 1)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], sh);
        if (lane < 4)
#pragma unroll
            for (int j = 0; j < 8; ++j) bias_part[q * kCh + 8 * g + j] = acc[j];
    }
    if (__syncthreads_or(!ok)) ok = false;
    tc::fence_after_sync();
    if (warp >= 2 && ok) {
        // TMEM lane m = 32 quad + lane: input channel i = lane of tap column
        // dx = quad (quad < 3); lanes 96..127 are not used.  Column block b
        // holds tap row dy = 2 - b.
        const int quad = warp & 3;
        float *out = p.partial + (int64_t)blockIdx.x * (kN2 + kCh);
#pragma unroll 1
        for (int b = 0; b < 3; ++b) {
#pragma unroll 1
            for (int oh = 0; oh < 2; ++oh) {
                float vh[16], vl[16];
                const uint32_t ta = tmem + (uint32_t)(64 * b + 16 * oh) + ((uint32_t)(quad * 32) << 16);
                tc::tmem_ld16(ta, vh);
                tc::tmem_ld16(ta + (uint32_t)kCh, vl);
                if (quad < 3)
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        out[((16 * oh + j) * kCh + lane) * 9 + 3 * (2 - b) + quad] = vh[j] + vl[j];
            }
        }
        if (warp == 2)
            out[kN2 + lane] = ((bias_part[lane] + bias_part[kCh + lane]) + bias_part[2 * kCh + lane]) +
                              bias_part[3 * kCh + lane];
    }
    if (!ok && tid == 0) atomicExch(&g_tc_error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kWgTmemCols);
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
// CTA per chain (kThreads threads): thread t takes blocks t, t + kThreads,
// ...; the squared residuals are summed in a fixed order (per thread, then a
// warp tree, then the warps in order).
__global__ void __launch_bounds__(kThreads) targets_loss_kernel(Chains ch, int64_t C, double beta,
                                                                const float *logits, float *dlogits, float *chain_sq)
{
    __shared__ float part[kThreads / 32];
    const int nb1 = ch.L / kBlk, nb = nb1 * nb1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < C; c += gridDim.x) {
        float sq = 0.0f;
        for (int b = threadIdx.x; b < nb; b += kThreads) {
            const int dE = block_delta_E(ch, c, b);
            const float t = (float)fmin(0.0, -beta * (double)dE);
            const float r = logits[c * nb + b] - t;
            dlogits[c * nb + b] = 2.0f * r / (float)(C * nb);
            sq += r * r;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
        __syncthreads();  // the previous chain's sums have been read
        if (lane == 0) part[warp] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.0f;
#pragma unroll
            for (int q = 0; q < kThreads / 32; ++q) tot += part[q];
            chain_sq[c] = tot;
        }
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

// The move kernels run one warp per chain.  FP64 arithmetic is slow on this
// GPU, so the lanes compute the exponentials of a chunk of 256 blocks in
// parallel into shared memory and lane 0 adds them up in block order: every
// FP64 operation, and so every decision, is the one of a sequential loop.
constexpr int kMoveWarps = 4;   // chains per 128-thread CTA
constexpr int kChunk = 256;     // blocks per chunk

__device__ __forceinline__ double warp_max_logit(const float *l, int nb)
{
    double m = -INFINITY;
    for (int b = (threadIdx.x & 31); b < nb; b += 32) m = fmax(m, (double)l[b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    return m;
}

// exp(l[b] - m) of the blocks base .. base + n - 1 into e[0 .. n-1]
__device__ __forceinline__ void chunk_exp(const float *l, double m, int base, int n, double *e)
{
    for (int j = (threadIdx.x & 31); j < n; j += 32) e[j] = exp((double)l[base + j] - m);
    __syncwarp();
}

// sum over b of exp(l[b] - m) in block order (the value is lane 0's)
__device__ double warp_exp_sum(const float *l, int nb, double m, double *e)
{
    double total = 0.0;
    for (int base = 0; base < nb; base += kChunk) {
        const int n = min(kChunk, nb - base);
        chunk_exp(l, m, base, n, e);
        if ((threadIdx.x & 31) == 0)
            for (int j = 0; j < n; ++j) total += e[j];
        __syncwarp();
    }
    return total;
}

__global__ void __launch_bounds__(32 * kMoveWarps) propose_kernel(int64_t C, int nb, const float *logits,
                                                                   const __grid_constant__ RoundKeys rk, uint64_t t,
                                                                   int32_t *block)
{
    __shared__ double ebuf[kMoveWarps][kChunk];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    double *e = ebuf[wl];
    const int64_t nwarps = (int64_t)gridDim.x * kMoveWarps;
    for (int64_t c = (int64_t)blockIdx.x * kMoveWarps + wl; c < C; c += nwarps) {
        const uint32_t u = move_draw(rk, (uint32_t)c, 0, t);
        int b = nb - 1;
        if (logits == nullptr) {
            b = (int)(((uint64_t)u * (uint64_t)nb) >> 32);
        } else {
            // inverse CDF: the first block whose cumulative weight exceeds u / 2^32 of the total
            const float *l = logits + c * nb;
            const double m = warp_max_logit(l, nb);
            const double target = ((double)u / 4294967296.0) * warp_exp_sum(l, nb, m, e);
            double acc = 0.0;
            int found = -1;
            for (int base = 0; base < nb && found < 0; base += kChunk) {
                const int n = min(kChunk, nb - base);
                chunk_exp(l, m, base, n, e);
                if (lane == 0)
                    for (int j = 0; j < n; ++j) {
                        acc += e[j];
                        if (acc > target) {
                            found = base + j;
                            break;
                        }
                    }
                found = __shfl_sync(0xffffffffu, found, 0);
            }
            if (found >= 0) b = found;
        }
        if (lane == 0) block[c] = b;
    }
}

__global__ void __launch_bounds__(32 * kMoveWarps) accept_kernel(Chains ch, uint64_t *black, uint64_t *white,
                                                                  int64_t C, double beta, const float *lx,
                                                                  const float *lxp, const int32_t *block,
                                                                  const __grid_constant__ RoundKeys rk, uint64_t t,
                                                                  int32_t *accepted, int64_t *dE_out)
{
    __shared__ double ebuf[kMoveWarps][kChunk];
    const int L = ch.L, nb1 = L / kBlk, nb = nb1 * nb1;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    double *e = ebuf[wl];
    const int64_t nwarps = (int64_t)gridDim.x * kMoveWarps;
    for (int64_t c = (int64_t)blockIdx.x * kMoveWarps + wl; c < C; c += nwarps) {
        const int b = block[c];
        const int by = b / nb1, bx = b - by * nb1, y0 = by * kBlk, x0 = bx * kBlk;
        // twice the boundary bond sum: lane = (edge, position along it)
        const int pos = lane & 7, edge = lane >> 3;
        int yi, xi, yo, xo;
        if (edge == 0) { yi = y0; xi = x0 + pos; yo = (y0 - 1 + L) % L; xo = xi; }
        else if (edge == 1) { yi = y0 + kBlk - 1; xi = x0 + pos; yo = (y0 + kBlk) % L; xo = xi; }
        else if (edge == 2) { yi = y0 + pos; xi = x0; yo = yi; xo = (x0 - 1 + L) % L; }
        else { yi = y0 + pos; xi = x0 + kBlk - 1; yo = yi; xo = (x0 + kBlk) % L; }
        int d = (int)spin_at(ch, c, yi, xi, -1) * (int)spin_at(ch, c, yo, xo, -1);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
        const int dE = 2 * d;
        double x = -beta * (double)dE;
        if (lx != nullptr) {
            // log q(b) = l_b - (max + log sum exp(l - max)), sums in block order
            const float *lr = lxp + c * nb, *lf = lx + c * nb;
            const double mr = warp_max_logit(lr, nb);
            const double sr = warp_exp_sum(lr, nb, mr, e);
            const double mf = warp_max_logit(lf, nb);
            const double sf = warp_exp_sum(lf, nb, mf, e);
            const double logp_rev = (double)lr[b] - (mr + log(sr));
            const double logp_fwd = (double)lf[b] - (mf + log(sf));
            x = (x + logp_rev) - logp_fwd;
        }
        if (lane == 0) {
            const uint64_t T = x >= 0.0 ? (uint64_t(1) << 32) : (uint64_t)floor(ldexp(exp(x), 32));
            const uint32_t u = move_draw(rk, (uint32_t)c, 1, t);
            const bool acc = (uint64_t)u < T;
            accepted[c] = acc ? 1 : 0;
            if (dE_out) dE_out[c] = dE;
            if (acc) {
                // the block's 4 sites of each colour per row sit in nibbles 4 bx .. 4 bx + 3
                const int j0 = 4 * bx;
                const uint64_t mask = 0x1111ull << (4 * (j0 & 15));
                for (int r = 0; r < kBlk; ++r) {
                    const int64_t w = c * (int64_t)L * ch.wpr + (int64_t)(y0 + r) * ch.wpr + (j0 >> 4);
                    black[w] ^= mask;
                    white[w] ^= mask;
                }
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

// Work layout: training keeps z1 z2 z3 (FP32), a1 a2 a3 (bfloat16) and two
// FP32 gradient buffers, then the weight-gradient partials; inference keeps
// a1 and a2 (bfloat16; where a3 is written at all it reuses a1's buffer).
// Both end with room for the 9 FP32 planes P of layer 4's tap projections
// (for L a multiple of 128 it holds the row partials of z4 instead, 9 values
// per row and 8-pixel block column).
struct NetWork {
    float *z1, *z2, *z3, *da, *db, *partial, *P, *tz;
    __nv_bfloat16 *a1, *a2, *a3, *ta, *gb1, *gb2;  // gb: bfloat16 gradients with halo columns (training)
    __nv_bfloat16 *gr1, *gr2;                      // the bfloat16 roundings of their remainders
    int64_t n_cta;
    size_t bytes;
};

constexpr int64_t kWgradCtasPerSm = 3;  // persistent CTAs per SM in the weight-gradient kernels

NetWork net_layout(int64_t L, int64_t C, int train, char *base)
{
    NetWork w;
    memset(&w, 0, sizeof(w));
    const size_t pix = (size_t)C * L * L * kCh;        // FP32 buffers
    const size_t apx = (size_t)C * L * (L + 2) * kCh;  // activation buffers (halo columns)
    size_t o = 0;
    auto take = [&](size_t n) {
        char *p = base ? base + o : nullptr;
        o += (n + 255) & ~size_t(255);
        return (void *)p;
    };
    if (train) {
        w.z1 = (float *)take(pix * 4); w.z2 = (float *)take(pix * 4); w.z3 = (float *)take(pix * 4);
        w.a1 = (__nv_bfloat16 *)take(apx * 2); w.a2 = (__nv_bfloat16 *)take(apx * 2);
        w.a3 = (__nv_bfloat16 *)take(apx * 2);
        w.da = (float *)take(pix * 4); w.db = (float *)take(pix * 4);
        w.gb1 = (__nv_bfloat16 *)take(apx * 2); w.gb2 = (__nv_bfloat16 *)take(apx * 2);
        if (L % kTileM == 0) {
            w.gr1 = (__nv_bfloat16 *)take(apx * 2); w.gr2 = (__nv_bfloat16 *)take(apx * 2);
        }
        DeviceInfo info{152};
        device_info(&info);
        w.n_cta = (int64_t)info.sm_count * kWgradCtasPerSm;
        w.partial = (float *)take((size_t)w.n_cta * (kN2 + kCh) * sizeof(float));
    } else {
        w.a1 = (__nv_bfloat16 *)take(apx * 2); w.a2 = (__nv_bfloat16 *)take(apx * 2);
        w.a3 = w.a1;
    }
    w.P = (float *)take((size_t)C * L * L * 9 * sizeof(float));
    w.tz = (float *)take((size_t)kPatterns * kCh * sizeof(float));
    w.ta = (__nv_bfloat16 *)take((size_t)kPatterns * kCh * 2);
    w.bytes = o;
    return w;
}

// Rows of each layer in a band pass.  Layer 4 recomputes the logits of block
// rows by - 1 .. by + 1, i.e. z4 on rows 8 by - 8 .. 8 by + 15; every 3 x 3
// layer below needs one more row on each side: a3 8 by - 9 .. 8 by + 16, a2
// 8 by - 10 .. 8 by + 17, a1 8 by - 11 .. 8 by + 18.  No value outside these
// rows (nor any logit outside those block rows) depends on the flipped block,
// whose rows are 8 by .. 8 by + 7: its influence reaches 4 rows (4 layers).
constexpr int kBandRows[4] = {30, 28, 26, 3};  // a1, a2, a3 rows; logit block rows
constexpr int kBandLead[3] = {11, 10, 9};

bool band_supported(int64_t L) { return L % kTileM == 0 && L >= 128; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link libcuda).
EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// The ring kernel's view of an activation buffer, one tensor map per channel
// group g: (8 channels at 8g, L + 2 pixels of 64 bytes, L rows, C chains),
// boxes of 8 x 130 x 1 x 1.
bool encode_rows(CUtensorMap (&m)[kGroups], const __nv_bfloat16 *a, int L, int64_t C)
{
    EncodeTiledFn fn = encode_tiled_fn();
    if (fn == nullptr) return false;
    const cuuint64_t dims[4] = {8, (cuuint64_t)L + 2, (cuuint64_t)L, (cuuint64_t)C};
    const cuuint64_t strides[3] = {(cuuint64_t)kCh * 2, (cuuint64_t)(L + 2) * kCh * 2,
                                   (cuuint64_t)L * (L + 2) * kCh * 2};
    const cuuint32_t box[4] = {8, kTileM + 2, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int g = 0; g < kGroups; ++g)
        if (fn(&m[g], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a + 8 * g), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    return true;
}

// The data gradient of a 32 -> 32 layer (weights at w_off) on the tensor
// cores: dz_prev = gelu'(zg) * conv^T(in), in the bfloat16 gradient with halo
// columns; writes d_out (FP32) and, if given, a_out (bfloat16, halo columns)
// and a_lo (the bfloat16 rounding of d_out - a_out).
int launch_ring_bwd(int L, int64_t C, const float *params, int w_off, const __nv_bfloat16 *in, const float *zg,
                    float *d_out, __nv_bfloat16 *a_out, __nv_bfloat16 *a_lo, cudaStream_t s)
{
    DeviceInfo info{152};
    device_info(&info);
    RingConv p{};
    if (!encode_rows(p.tmap, in, L, C)) return nfail(ISING_ECUDA, "cuTensorMapEncodeTiled failed");
    p.a_in = in;
    p.a_out = a_out;
    p.a_lo = a_lo;
    p.zg = zg;
    p.d_out = d_out;
    p.params = params;
    p.w_off = w_off;
    p.b_off = 0;
    p.bd.L = L;
    p.bd.C = C;
    p.bd.rows = L;
    p.bd.lead = 0;
    p.bd.flip = nullptr;
    p.segs = L / kTileM;
    p.units_per_col = (L + kUnitRows - 1) / kUnitRows;
    p.units = C * p.segs * p.units_per_col;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(p.units, 2 * info.sm_count));
    cudaFuncSetAttribute(conv32_ring_kernel<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)RingLayout<false, true>::bytes);
    conv32_ring_kernel<false, true, false><<<grid, kRingThreads, RingLayout<false, true>::bytes, s>>>(p);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

// The weight gradients of a 32 -> 32 layer on the tensor cores (L a multiple
// of 128): the layer's input a (bfloat16, halo columns) and its gradient as
// hi = bf16(dz), lo = bf16(dz - hi) (same layout); one CTA per SM writes its
// partial sums into partial[cta][kN2 + kCh].  Returns the number of CTAs.
int launch_wgrad_tc(int L, int64_t C, const __nv_bfloat16 *a, const __nv_bfloat16 *hi, const __nv_bfloat16 *lo,
                    float *partial, int64_t max_ctas, cudaStream_t s, int64_t *n_cta)
{
    EncodeTiledFn fn = encode_tiled_fn();
    if (fn == nullptr) return nfail(ISING_ECUDA, "cuTensorMapEncodeTiled is not available");
    DeviceInfo info{152};
    device_info(&info);
    WgradTc p{};
    const cuuint64_t dims[4] = {(cuuint64_t)kCh, (cuuint64_t)L + 2, (cuuint64_t)L, (cuuint64_t)C};
    const cuuint64_t strides[3] = {(cuuint64_t)kCh * 2, (cuuint64_t)(L + 2) * kCh * 2,
                                   (cuuint64_t)L * (L + 2) * kCh * 2};
    const cuuint32_t box[4] = {kCh, kTileM, 1, 1};  // whole pixels, 64 bytes: the 64-byte swizzle
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const __nv_bfloat16 *src[3] = {a, hi, lo};
    CUtensorMap *maps[3] = {&p.act, &p.hi, &p.lo};
    for (int t = 0; t < 3; ++t)
        if (fn(maps[t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)src[t], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return nfail(ISING_ECUDA, "cuTensorMapEncodeTiled failed");
    p.partial = partial;
    p.L = L;
    p.segs = L / kTileM;
    p.lines = C * p.segs * L;
    // every CTA gets at least one row, so every partial row is written
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({(int64_t)info.sm_count, max_ctas, p.lines}));
    cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    wgrad_tc_kernel<<<(unsigned)grid, kWgThreads, kWgSmem, s>>>(p);
    *n_cta = grid;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

int launch_forward(const Chains &ch, int64_t C, const int32_t *flip, bool band, const float *params,
                   float *logits, const NetWork &w, int train, cudaStream_t s, bool withhold = false)
{
    const int L = ch.L;
    DeviceInfo info{152};
    device_info(&info);
    Band bd[3];
    for (int l = 0; l < 3; ++l) {
        bd[l].L = L;
        bd[l].C = C;
        bd[l].rows = band ? kBandRows[l] : L;
        bd[l].lead = band ? kBandLead[l] : 0;
        bd[l].flip = band ? flip : nullptr;
    }
    {
        // enough CTAs for ~16 per SM, tiles of a chain first, then chains
        const int64_t tiles = (int64_t)bd[0].rows * L / kL1Threads;
        const int64_t want = (int64_t)info.sm_count * 16;
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, want));
        const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>({C, 65535, (want + gx - 1) / gx}));
        l1_table_kernel<<<kPatterns * kCh / 256, 256, 0, s>>>(params, w.tz, w.ta);
        // an inference pass of the row-ring kernels forms layer 1 inside the first conv
        if (train || L % kTileM != 0)
            l1_kernel<<<dim3(gx, gy), kL1Threads, 0, s>>>(ch, bd[0], flip, w.ta, w.tz, train ? w.z1 : nullptr,
                                                           w.a1);
    }
    const int off[2][2] = {{kOffW2, kOffB2}, {kOffW3, kOffB3}};
    const __nv_bfloat16 *ins[2] = {w.a1, w.a2};
    float *zs[2] = {train ? w.z2 : nullptr, train ? w.z3 : nullptr};
    if (L % kTileM == 0) {
        // row-ring kernels; the second one also projects onto layer 4's taps
        cudaFuncSetAttribute(conv32_ring_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RingLayout<false>::bytes);
        cudaFuncSetAttribute(conv32_ring_kernel<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RingLayout<false, true>::bytes);
        cudaFuncSetAttribute(conv32_ring_kernel<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RingLayout<true>::bytes);
        // shared memory for two CTAs of the first conv, the rest as L1 for the layer-1 table
        cudaFuncSetAttribute(conv32_ring_kernel<false, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             86);
        __nv_bfloat16 *outs[2] = {w.a2, train ? w.a3 : nullptr};
        for (int l = 0; l < 2; ++l) {
            RingConv p{};
            const bool fused = l == 0 && !train;
            if (!fused && !encode_rows(p.tmap, ins[l], L, C)) return nfail(ISING_ECUDA, "cuTensorMapEncodeTiled failed");
            p.ch = ch;
            p.flip = flip;
            p.ta = w.ta;
            p.a_in = ins[l];
            p.a_out = outs[l];
            p.z_out = zs[l];
            p.P = w.P;
            p.params = params;
            p.w_off = off[l][0];
            p.b_off = off[l][1];
            p.bd = bd[l + 1];
            p.segs = L / kTileM;
            p.units_per_col = (bd[l + 1].rows + kUnitRows - 1) / kUnitRows;
            p.units = C * p.segs * p.units_per_col;
            p.withhold = withhold && l == 0;
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(p.units, 2 * info.sm_count));
            if (fused)
                conv32_ring_kernel<false, false, true><<<grid, ring_threads<false, true>(), RingLayout<false>::bytes, s>>>(p);
            else if (l == 0)
                conv32_ring_kernel<false, false, false><<<grid, kRingThreads, RingLayout<false, true>::bytes, s>>>(p);
            else
                conv32_ring_kernel<true, false, false><<<grid, ring_threads<true, false>(), RingLayout<true>::bytes, s>>>(p);
        }
    } else {
        cudaFuncSetAttribute(conv32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
        __nv_bfloat16 *outs[2] = {w.a2, w.a3};  // inference: a3 reuses a1's buffer
        for (int l = 0; l < 2; ++l) {
            ConvTc p;
            p.a_in = ins[l];
            p.a_out = outs[l];
            p.z_out = zs[l];
            p.params = params;
            p.w_off = off[l][0];
            p.b_off = off[l][1];
            p.bd = bd[l + 1];
            p.tiles = C * (int64_t)bd[l + 1].rows * L / kTileM;
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(p.tiles, info.sm_count));
            conv32_tc_kernel<<<grid, kConvThreads, kConvSmem, s>>>(p);
        }
        l4_project_kernel<<<grid1d(C * (int64_t)bd[2].rows * L, kThreads), kThreads, 0, s>>>(bd[2], params, w.a3,
                                                                                             w.P);
    }
    const int brows = band ? kBandRows[3] : L / kBlk;
    if (L % kTileM == 0) {
        // the projecting ring kernel left row partials of z4 in w.P
        pool_rows_kernel<<<grid1d(C * brows * (L / kBlk), kThreads), kThreads, 0, s>>>(
            L, C, brows, band ? flip : nullptr, params, w.P, logits);
    } else {
        const int64_t warps = C * brows * (L / kBlk / 4);
        pool_kernel<<<grid1d(warps * 32, kThreads), kThreads, 0, s>>>(L, C, brows, band ? flip : nullptr, params, w.P,
                                                                      logits);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
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
        check_device_range(logits_dev, (size_t)C * (L / 8) * (L / 8) * 4, "logits") ||
        check_device_range(work_dev, w.bytes, "work"))
        return nfail(ISING_EINVAL, "planes, params, logits and work must be device memory of their sizes");
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    return launch_forward(ch, C, flip_block_dev, false, params_dev, logits_dev, w, train, (cudaStream_t)stream);
}

ISING_API int ising_net_forward_flipped(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                        const int32_t *flip_block_dev, const float *params_dev,
                                        const float *logits_x_dev, float *logits_dev, void *work_dev,
                                        size_t work_bytes, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    NetWork w = net_layout(L, C, 0, (char *)work_dev);
    if (work_dev == nullptr || work_bytes < w.bytes) return nfail(ISING_EINVAL, "work buffer too small");
    const size_t plane = (size_t)C * L * L / 32 * 8;
    const size_t lbytes = (size_t)C * (L / 8) * (L / 8) * 4;
    if (check_device_range(black_dev, plane, "black") || check_device_range(white_dev, plane, "white") ||
        check_device_range(params_dev, kParams * 4, "params") || check_device_range(logits_dev, lbytes, "logits") ||
        check_device_range(logits_x_dev, lbytes, "logits_x") || check_device_range(flip_block_dev, (size_t)C * 4, "flip") ||
        check_device_range(work_dev, w.bytes, "work"))
        return nfail(ISING_EINVAL, "planes, params, logits, flip and work must be device memory of their sizes");
    if (logits_x_dev == logits_dev) return nfail(ISING_EINVAL, "logits_x and logits must differ");
    cudaStream_t s = (cudaStream_t)stream;
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    if (!band_supported(L)) return launch_forward(ch, C, flip_block_dev, false, params_dev, logits_dev, w, 0, s);
    cudaError_t e = cudaMemcpyAsync(logits_dev, logits_x_dev, lbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return nfail(ISING_ECUDA, cudaGetErrorString(e));
    return launch_forward(ch, C, flip_block_dev, true, params_dev, logits_dev, w, 0, s);
}

ISING_API int ising_net_wait_selftest(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                     const float *params_dev, float *logits_dev, void *work_dev, size_t work_bytes,
                                     ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    if (L % kTileM != 0) return nfail(ISING_EINVAL, "the self-test runs the row-ring kernel: L must be a multiple of 128");
    NetWork w = net_layout(L, C, 0, (char *)work_dev);
    if (work_dev == nullptr || work_bytes < w.bytes) return nfail(ISING_EINVAL, "work buffer too small");
    const size_t plane = (size_t)C * L * L / 32 * 8;
    if (check_device_range(black_dev, plane, "black") || check_device_range(white_dev, plane, "white") ||
        check_device_range(params_dev, kParams * 4, "params") ||
        check_device_range(logits_dev, (size_t)C * (L / 8) * (L / 8) * 4, "logits") ||
        check_device_range(work_dev, w.bytes, "work"))
        return nfail(ISING_EINVAL, "planes, params, logits and work must be device memory of their sizes");
    Chains ch{(const uint64_t *)black_dev, (const uint64_t *)white_dev, (int)L, (int)(L / 32)};
    return launch_forward(ch, C, nullptr, false, params_dev, logits_dev, w, 0, (cudaStream_t)stream, true);
}

ISING_API int ising_net_check(ising_stream_t stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    int flag = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&flag, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return nfail(ISING_ECUDA, cudaGetErrorString(e));
    if (flag) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
        return nfail(ISING_ETIMEOUT, "a tensor-core kernel gave up waiting for its MMAs");
    }
    return ISING_OK;
}

ISING_API int ising_net_backward(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                 const float *params_dev, const float *dlogits_dev, float *grad_dev, void *work_dev,
                                 size_t work_bytes, ising_stream_t stream)
{
    int rc = check_chains(L, C);
    if (rc) return rc;
    NetWork w = net_layout(L, C, 1, (char *)work_dev);
    if (work_dev == nullptr || work_bytes < w.bytes) return nfail(ISING_EINVAL, "work buffer too small (train mode)");
    if (check_device_range(work_dev, w.bytes, "work")) return nfail(ISING_EINVAL, "work must be device memory of its size");
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
    cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
    auto reduce = [&](int ne, int nw, int w_off, int b_off, int64_t n_cta) {
        reduce_partials_kernel<<<(unsigned)((ne + 31) / 32), 32 * kReduceWarps, 0, s>>>(w.partial, n_cta, ne, nw,
                                                                                       grad_dev, w_off, b_off);
    };
    // layer 4
    // the thin weight gradients: one wave of two CTAs per SM
    DeviceInfo info{152};
    device_info(&info);
    const int64_t n_thin = std::min<int64_t>(w.n_cta, 2 * (int64_t)info.sm_count);
    wgrad_thin_kernel<true><<<(unsigned)n_thin, 32 * kThinWarps, 0, s>>>(ch, C, nullptr, w.a3, dlogits_dev, w.partial);
    reduce(kN1 + 1, kN1, kOffW4, kOffB4, n_thin);
    // for L a multiple of 128 the data and weight gradients of the 32 -> 32
    // layers run on the tensor cores; their gradients are then also kept as
    // bfloat16 parts (gb: the rounding, gr: the rounding of the remainder)
    const bool ring = L % kTileM == 0;
    l4_bwd_data_kernel<<<grid1d(4 * npix, kThreads), kThreads, 0, s>>>((int)L, C, params_dev, dlogits_dev, w.z3,
                                                                     w.da, ring ? w.gb1 : nullptr,
                                                                     ring ? w.gr1 : nullptr);  // dz3
    // layer 3
    int64_t n_tc = 0;
    if (ring) {
        rc = launch_wgrad_tc((int)L, C, w.a2, w.gb1, w.gr1, w.partial, w.n_cta, s, &n_tc);
        if (rc) return rc;
        reduce(kN2 + kCh, kN2, kOffW3, kOffB3, n_tc);
        rc = launch_ring_bwd((int)L, C, params_dev, kOffW3, w.gb1, w.z2, w.db, w.gb2, w.gr2, s);  // dz2
        if (rc) return rc;
    } else {
        wgrad_kernel<<<gw, 256, sm32, s>>>(ch, C, w.a2, w.da, w.partial);
        reduce(kN2 + kCh, kN2, kOffW3, kOffB3, w.n_cta);
        conv32_bwd_data_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW3, w.da, w.z2, w.db);  // dz2
    }
    // layer 2
    if (ring) {
        rc = launch_wgrad_tc((int)L, C, w.a1, w.gb2, w.gr2, w.partial, w.n_cta, s, &n_tc);
        if (rc) return rc;
        reduce(kN2 + kCh, kN2, kOffW2, kOffB2, n_tc);
        rc = launch_ring_bwd((int)L, C, params_dev, kOffW2, w.gb2, w.z1, w.da, nullptr, nullptr, s);  // dz1
        if (rc) return rc;
    } else {
        wgrad_kernel<<<gw, 256, sm32, s>>>(ch, C, w.a1, w.db, w.partial);
        reduce(kN2 + kCh, kN2, kOffW2, kOffB2, w.n_cta);
        conv32_bwd_data_kernel<<<g, kThreads, smem, s>>>((int)L, C, params_dev, kOffW2, w.db, w.z1, w.da);  // dz1
    }
    // layer 1
    wgrad_thin_kernel<false><<<(unsigned)n_thin, 32 * kThinWarps, 0, s>>>(ch, C, w.da, nullptr, nullptr, w.partial);
    reduce(kN1 + kCh, kN1, kOffW1, kOffB1, n_thin);
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
    targets_loss_kernel<<<(unsigned)std::min<int64_t>(C, 1 << 30), kThreads, 0, s>>>(ch, C, beta, logits_dev,
                                                                                     dlogits_dev, chain_sq_dev);
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
    propose_kernel<<<grid1d(C * 32, 32 * kMoveWarps), 32 * kMoveWarps, 0, (cudaStream_t)stream>>>(
        C, nb, logits_dev, make_round_keys(seed), t, block_dev);
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
    accept_kernel<<<grid1d(C * 32, 32 * kMoveWarps), 32 * kMoveWarps, 0, (cudaStream_t)stream>>>(
        ch, (uint64_t *)black_dev, (uint64_t *)white_dev, C, beta, logits_x_dev, logits_xp_dev, block_dev,
        make_round_keys(seed), t, accepted_dev, dE_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISING_OK : nfail(ISING_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
