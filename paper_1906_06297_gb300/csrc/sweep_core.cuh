// sweep_core.cuh -- the per-word arithmetic of a multi-spin-coded half-sweep,
// shared by the single-lattice and the batched sweep kernels: the threshold
// marks of the keyed draws and the bit-parallel Metropolis decision.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace ising {

// Per-call inputs of the draws and the decision: Philox counter words 2 and 3
// (sweep index and colour), the thresholds for a = 3 / a = 4, and a runtime
// zero (see mark_ge).
struct DrawCtx {
    uint32_t c2, c3;
    uint32_t T3, T4;
    uint32_t zero;
};

// Counts, at the nibble given by `bit`, how many of the two thresholds the
// draw u fails: [u >= T3] + [u >= T4] (0..2).  Two compares and two predicated
// updates per draw.  Where the updates run is a compile-time choice, because
// the logic pipe and the multiply-add pipe share the load of this kernel:
//   ISING_MSC4_MARK 0: two predicated adds into one counter (the compiler puts
//                      them on the multiply-add pipe, next to Philox),
//   ISING_MSC4_MARK 1: g3 by a predicated OR (logic pipe), g4 by an add,
//   ISING_MSC4_MARK 2: both by predicated ORs (logic pipe).
// The OR forms start from a runtime zero (Accept::zero), which keeps the
// compiler from rewriting them as adds.  ncu on GB300: form 0 is fastest.
#ifndef ISING_MSC4_MARK
#define ISING_MSC4_MARK 0
#endif
__device__ __forceinline__ void mark_ge(uint32_t &g3, uint32_t &g4, uint32_t u, uint32_t T3, uint32_t T4,
                                        uint32_t bit)
{
#if ISING_MSC4_MARK == 0
    asm("{\n\t"
        ".reg .pred p3, p4;\n\t"
        "setp.ge.u32 p3, %1, %3;\n\t"
        "setp.ge.u32 p4, %1, %4;\n\t"
        "@p3 add.u32 %0, %0, %2;\n\t"
        "@p4 add.u32 %0, %0, %2;\n\t"
        "}"
        : "+r"(g3)
        : "r"(u), "r"(bit), "r"(T3), "r"(T4));
    (void)g4;
#elif ISING_MSC4_MARK == 1
    asm("{\n\t"
        ".reg .pred p3, p4;\n\t"
        "setp.ge.u32 p3, %2, %4;\n\t"
        "setp.ge.u32 p4, %2, %5;\n\t"
        "@p3 or.b32 %0, %0, %3;\n\t"
        "@p4 add.u32 %1, %1, %3;\n\t"
        "}"
        : "+r"(g3), "+r"(g4)
        : "r"(u), "r"(bit), "r"(T3), "r"(T4));
#else
    asm("{\n\t"
        ".reg .pred p3, p4;\n\t"
        "setp.ge.u32 p3, %2, %4;\n\t"
        "setp.ge.u32 p4, %2, %5;\n\t"
        "@p3 or.b32 %0, %0, %3;\n\t"
        "@p4 or.b32 %1, %1, %3;\n\t"
        "}"
        : "+r"(g3), "+r"(g4)
        : "r"(u), "r"(bit), "r"(T3), "r"(T4));
#endif
}

// New values of 8 spins (one 32-bit half word).
//   s     spins (0/1 per nibble)
//   t, e  neighbour words: t = up + down + centre (nibble-wise), e = side word
//   c0,c1 Philox blocks c0 and c0+1 give the 8 draws (spin n uses word n%4 of
//         block c0 + n/4); c0 is even
//
// With d = number of anti-aligned neighbours (0..4) and G = [u >= T3] +
// [u >= T4] (T4 <= T3), the Metropolis decision "flip iff u < T[4 - d]"
// (always for d >= 2) is exactly "flip iff d >= G": for d = 1 it reads
// u < T3, for d = 0 it reads u < T4.  Per nibble d + 8 - G lies in 6..12, so
// bit 3 of the nibble is the flip bit and no carry crosses nibbles.  d + 8 is
// selected from k + 8 (down spin) and 12 - k (up spin), k = t + e.
//
// ALWAYS (beta = 0: every threshold is 2^32) flips every spin; the draws are
// then irrelevant and not computed.
//
// With OBS, the anti-aligned counts after the update are added to the byte
// lanes of dacc.
template <bool OBS, bool ALWAYS>
__device__ __forceinline__ uint32_t update_half(uint32_t s, uint32_t t, uint32_t e, uint32_t c0, uint32_t c1,
                                                const DrawCtx &dc, const RoundKeys &rk, uint32_t &dacc)
{
    const uint32_t a8 = t + e + 0x88888888u;  // 8 + k
    const uint32_t b8 = 0xCCCCCCCCu - t - e;  // 12 - k
    uint32_t ns;
    if (ALWAYS) {
        ns = s ^ kNibbleLsb;
    } else {
#if ISING_MSC4_MARK == 0
        uint32_t g3 = 0, g4 = 0;  // g3 holds G, g4 stays 0
#else
        uint32_t g3 = dc.zero, g4 = dc.zero;
#endif
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const uint4 u = philox(c0 | b, c1, dc.c2, dc.c3, rk);
            mark_ge(g3, g4, u.x, dc.T3, dc.T4, 1u << (16 * b));
            mark_ge(g3, g4, u.y, dc.T3, dc.T4, 1u << (16 * b + 4));
            mark_ge(g3, g4, u.z, dc.T3, dc.T4, 1u << (16 * b + 8));
            mark_ge(g3, g4, u.w, dc.T3, dc.T4, 1u << (16 * b + 12));
        }
        const uint32_t m = s * 15u;               // nibble mask of the up spins
        const uint32_t d8 = (a8 & ~m) | (b8 & m);  // 8 + d
        const uint32_t x = d8 - g3 - g4;
        ns = s ^ ((x >> 3) & kNibbleLsb);
    }
    if (OBS) {
        // both selections have bit 3 set (k <= 4), so masking with 7 leaves d
        const uint32_t m2 = ns * 15u;
        const uint32_t d2 = (a8 & ~m2) | (b8 & m2);
        dacc += (d2 & 0x07070707u) + ((d2 >> 4) & 0x07070707u);
    }
    return ns;
}

}  // namespace ising
