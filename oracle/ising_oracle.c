/*
 * ising_oracle.c -- plain CPU oracle for the checkerboard Metropolis sweep of
 * the two-dimensional ferromagnetic Ising model (J = 1, h = 0, periodic L x L).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator with
 * the CUDA library; it is written from the paper and from the definitions
 * below, plainly and slowly, so that a reader can check it by eye.
 *
 * What it computes (Romero, Bisson, Fatica, Bernaschi, "A Performance study of
 * the 2D Ising model on GPUs", arXiv:1906.06297):
 *   - Hamiltonian H = -sum_<ij> sigma_i sigma_j over the 4 nearest neighbours
 *     (Sec. 2, Eq. 1, with J_ij = J = 1).
 *   - Metropolis rule: flip a spin; accept if dE < 0, else with probability
 *     exp(-beta dE) (Sec. 2, the three-step Metropolis description).
 *   - Checkerboard decomposition: all spins of one colour are updated with the
 *     other colour held fixed, then the other colour (Sec. 2, last paragraph on
 *     parallel updates; Sec. 3.3, two launches per step, black then white).
 *   - Colour and neighbour convention of the basic kernel (Sec. 3.1, Fig. 2):
 *     site (i, c) is black iff (i + c) is even; its compacted plane column is
 *     c / 2; the acceptance test is exp(-2 beta * nn_sum * s).
 *
 * Readings where the paper leaves a choice (each is listed with its reason in
 * the design notes of the repository):
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
 *     "Parallel random numbers: as easy as 1, 2, 3"), keyed by
 *       key     = (seed & 0xffffffff, seed >> 32)
 *       counter = (q_lo, q_hi, t_lo, colour | purpose << 1 | t_hi << 8)
 *     with site = i * (L/2) + c/2 (index in the colour plane), q = site >> 2,
 *     t = sweep index, and the draw is output word (site & 3).  purpose 0 is
 *     the Metropolis draw, purpose 1 the random initial state.
 *     (Sec. 3.2 uses cuRAND's per-thread Philox4_32_10 sequences; the counter
 *     is keyed to the site here so that results do not depend on launch shape.)
 *   - acceptance: with a = number of the 4 neighbours equal to the spin,
 *     dE = 4a - 8 and p_a = min(1, exp(-beta dE)); the threshold table is
 *     T[a] = 2^32 if p_a >= 1 else floor(p_a * 2^32), built in double with
 *     exp(); the spin flips iff (uint64) u < T[a], so P(flip) = T[a] / 2^32.
 *   - random initial state: spin = +1 iff the init draw (t = 0, purpose 1)
 *     is below 2^31.
 *
 * Per site the oracle recomputes a whole Philox block and keeps one word of
 * it: four times the work of sharing a block between four sites, but with no
 * blocking to get wrong.  Rows of one colour are independent, so a half-sweep
 * may run its rows in parallel (OpenMP) and stay bit-exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 as defined in Salmon et al. (SC'11), Sec. 3.3 ("Philox"):     */
/* each round multiplies counter words 0 and 2 by two fixed 32-bit constants,  */
/* takes the 64-bit products apart into hi and lo halves, and forms            */
/*   (hi(M1*x2) ^ x1 ^ k0,  lo(M1*x2),  hi(M0*x0) ^ x3 ^ k1,  lo(M0*x0));      */
/* the key is bumped by the Weyl constants between rounds.                     */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x[1] ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x[3] ^ k1;
        uint32_t y3 = lo0;
        x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/*
 * The 32-bit draw for one site of one colour plane at sweep t.  `stream`
 * separates the lattices of a batch (and the ladders of its replica swaps):
 * it is added to counter word 1, which is q_hi for a single lattice.
 */
uint32_t oracle_draw_stream(uint64_t seed, uint32_t stream, uint64_t site, uint64_t t, int colour, int purpose)
{
    uint64_t q = site >> 2;
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)(q & 0xffffffffu);
    ctr[1] = (uint32_t)(q >> 32) + stream;
    ctr[2] = (uint32_t)(t & 0xffffffffu);
    ctr[3] = (uint32_t)colour | ((uint32_t)purpose << 1) | ((uint32_t)(t >> 32) << 8);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[site & 3];
}

uint32_t oracle_draw(uint64_t seed, uint64_t site, uint64_t t, int colour, int purpose)
{
    return oracle_draw_stream(seed, 0, site, t, colour, purpose);
}

/* ------------------------------------------------------------------------- */
/* Acceptance table.  With a aligned neighbours out of 4, flipping the spin    */
/* changes the energy by dE = 2 * s * (sum of neighbours) = 4a - 8; Metropolis */
/* accepts with min(1, exp(-beta dE)) (Sec. 2).                                */
/* ------------------------------------------------------------------------- */
int oracle_thresholds(double beta, uint64_t T[5])
{
    if (!(beta >= 0.0) || isinf(beta)) return 1;
    for (int a = 0; a <= 4; a++) {
        double dE = 4.0 * a - 8.0;
        double p = exp(-beta * dE);
        if (p >= 1.0)
            T[a] = (uint64_t)1 << 32;
        else
            T[a] = (uint64_t)floor(ldexp(p, 32));
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Full-lattice helpers.  s is an L x L row-major array of int8 spins (+1/-1). */
/* ------------------------------------------------------------------------- */
static inline int64_t wrap(int64_t x, int64_t L) { return (x % L + L) % L; }

static inline int colour_of(int64_t i, int64_t c) { return (int)((i + c) & 1); }

static inline uint64_t plane_site(int64_t L, int64_t i, int64_t c)
{
    return (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(c / 2);
}

/* Initial state of row i: mode 0 = keyed random, 1 = all +1, 2 = all -1. */
void oracle_init_row_stream(int64_t L, int64_t i, int8_t *row, int mode, uint64_t seed, uint32_t stream)
{
    for (int64_t c = 0; c < L; c++) {
        int8_t v;
        if (mode == 1) {
            v = 1;
        } else if (mode == 2) {
            v = -1;
        } else {
            uint32_t u = oracle_draw_stream(seed, stream, plane_site(L, i, c), 0, colour_of(i, c), 1);
            v = (u < 0x80000000u) ? 1 : -1;
        }
        row[c] = v;
    }
}

void oracle_init_row(int64_t L, int64_t i, int8_t *row, int mode, uint64_t seed)
{
    oracle_init_row_stream(L, i, row, mode, seed, 0);
}

int oracle_init(int64_t L, int8_t *s, int mode, uint64_t seed)
{
    if (L <= 0 || (L & 1)) return 1;
    for (int64_t i = 0; i < L; i++) oracle_init_row(L, i, s + i * L, mode, seed);
    return 0;
}

/*
 * Update the sites of one colour in row i, given rows i-1 ("above") and i+1
 * ("below") of the full lattice.  The row is updated in place; sites of the
 * other colour in it are only read (they are the horizontal neighbours).
 */
void oracle_update_row_stream(int64_t L, const int8_t *above, int8_t *row, const int8_t *below, int64_t i,
                              int colour, const uint64_t T[5], uint64_t seed, uint64_t t, uint32_t stream)
{
    for (int64_t c = 0; c < L; c++) {
        if (colour_of(i, c) != colour) continue;
        int nb = above[c] + below[c] + row[wrap(c - 1, L)] + row[wrap(c + 1, L)];
        int s = row[c];
        int a = (4 + s * nb) / 2; /* aligned neighbours: s*nb = a - (4 - a) */
        uint32_t u = oracle_draw_stream(seed, stream, plane_site(L, i, c), t, colour, 0);
        if ((uint64_t)u < T[a]) row[c] = (int8_t)(-s);
    }
}

void oracle_update_row(int64_t L, const int8_t *above, int8_t *row, const int8_t *below, int64_t i, int colour,
                       const uint64_t T[5], uint64_t seed, uint64_t t)
{
    oracle_update_row_stream(L, above, row, below, i, colour, T, seed, t, 0);
}

/* One half-sweep: every site of one colour, rows in parallel. */
void oracle_half_sweep_stream(int64_t L, int8_t *s, int colour, const uint64_t T[5], uint64_t seed, uint64_t t,
                              uint32_t stream, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    /* threads only pay off on large lattices; small ones run serially */
#pragma omp parallel for schedule(static) num_threads(nthreads) if (L >= 256)
#endif
    for (int64_t i = 0; i < L; i++) {
        const int8_t *above = s + wrap(i - 1, L) * L;
        const int8_t *below = s + wrap(i + 1, L) * L;
        oracle_update_row_stream(L, above, s + i * L, below, i, colour, T, seed, t, stream);
    }
    (void)nthreads;
}

void oracle_half_sweep(int64_t L, int8_t *s, int colour, const uint64_t T[5], uint64_t seed, uint64_t t,
                       int nthreads)
{
    oracle_half_sweep_stream(L, s, colour, T, seed, t, 0, nthreads);
}

/*
 * Observables: out[0] = sum of spins, out[1] = sum over bonds of s_i s_j, each
 * bond counted once (the right and the down bond of every site).  The energy
 * is E = -out[1] (Eq. 1 with J = 1).
 */
void oracle_observables(int64_t L, const int8_t *s, int64_t out[2])
{
    int64_t m = 0, b = 0;
    for (int64_t i = 0; i < L; i++) {
        for (int64_t c = 0; c < L; c++) {
            int v = s[i * L + c];
            m += v;
            b += v * s[i * L + wrap(c + 1, L)];
            b += v * s[wrap(i + 1, L) * L + c];
        }
    }
    out[0] = m;
    out[1] = b;
}

/*
 * n sweeps starting at sweep index off: for each sweep, black then white.
 * trace (nullable) receives {sum s, sum bonds} after each sweep.
 */
int oracle_run(int64_t L, int8_t *s, double beta, int64_t n, uint64_t seed, uint64_t off,
               int64_t *trace, int nthreads)
{
    uint64_t T[5];
    if (L <= 0 || (L & 1) || n < 0) return 1;
    if (oracle_thresholds(beta, T)) return 1;
    for (int64_t k = 0; k < n; k++) {
        uint64_t t = off + (uint64_t)k;
        oracle_half_sweep(L, s, 0, T, seed, t, nthreads);
        oracle_half_sweep(L, s, 1, T, seed, t, nthreads);
        if (trace) oracle_observables(L, s, trace + 2 * k);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The two storage layouts of the colour planes, decoded and encoded here from */
/* their definition (own code; the CUDA library has its own):                  */
/*  int8: plane[colour] is L rows x (L/2) bytes, row stride `stride` bytes;    */
/*        site (i, c) of that colour sits at column c/2 (Sec. 3.1, Fig. 1).     */
/*  msc4: plane row of L/2 spins = L/32 uint64 words, row stride `stride`      */
/*        words; compacted column j is word j/16, bits 4*(j%16) .. +3, value    */
/*        0 for -1 and 1 for +1 (Sec. 3.3, 4 bits per spin, -1/1 -> 0/1).      */
/* ------------------------------------------------------------------------- */
void oracle_row_to_planes_int8(int64_t L, int64_t i, const int8_t *row, int8_t *black_row,
                               int8_t *white_row)
{
    for (int64_t c = 0; c < L; c++) {
        int8_t *dst = colour_of(i, c) == 0 ? black_row : white_row;
        dst[c / 2] = row[c];
    }
}

void oracle_row_from_planes_int8(int64_t L, int64_t i, const int8_t *black_row,
                                 const int8_t *white_row, int8_t *row)
{
    for (int64_t c = 0; c < L; c++) {
        const int8_t *src = colour_of(i, c) == 0 ? black_row : white_row;
        row[c] = src[c / 2];
    }
}

void oracle_row_to_planes_msc4(int64_t L, int64_t i, const int8_t *row, uint64_t *black_row,
                               uint64_t *white_row)
{
    int64_t words = L / 32;
    for (int64_t w = 0; w < words; w++) {
        black_row[w] = 0;
        white_row[w] = 0;
    }
    for (int64_t c = 0; c < L; c++) {
        uint64_t *dst = colour_of(i, c) == 0 ? black_row : white_row;
        int64_t j = c / 2;
        if (row[c] > 0) dst[j / 16] |= (uint64_t)1 << (4 * (j % 16));
    }
}

void oracle_row_from_planes_msc4(int64_t L, int64_t i, const uint64_t *black_row,
                                 const uint64_t *white_row, int8_t *row)
{
    for (int64_t c = 0; c < L; c++) {
        const uint64_t *src = colour_of(i, c) == 0 ? black_row : white_row;
        int64_t j = c / 2;
        uint64_t nib = (src[j / 16] >> (4 * (j % 16))) & 0xF;
        row[c] = nib == 1 ? 1 : (nib == 0 ? -1 : 0); /* 0 marks a corrupt nibble */
    }
}

void oracle_to_planes_int8(int64_t L, const int8_t *s, int8_t *black, int8_t *white,
                           int64_t stride)
{
    for (int64_t i = 0; i < L; i++)
        oracle_row_to_planes_int8(L, i, s + i * L, black + i * stride, white + i * stride);
}

void oracle_from_planes_int8(int64_t L, const int8_t *black, const int8_t *white,
                             int64_t stride, int8_t *s)
{
    for (int64_t i = 0; i < L; i++)
        oracle_row_from_planes_int8(L, i, black + i * stride, white + i * stride, s + i * L);
}

void oracle_to_planes_msc4(int64_t L, const int8_t *s, uint64_t *black, uint64_t *white,
                           int64_t stride)
{
    for (int64_t i = 0; i < L; i++)
        oracle_row_to_planes_msc4(L, i, s + i * L, black + i * stride, white + i * stride);
}

void oracle_from_planes_msc4(int64_t L, const uint64_t *black, const uint64_t *white,
                             int64_t stride, int8_t *s)
{
    for (int64_t i = 0; i < L; i++)
        oracle_row_from_planes_msc4(L, i, black + i * stride, white + i * stride, s + i * L);
}

/* ------------------------------------------------------------------------- */
/* The bit-packed format (an I/O format of the library, not of the paper): a  */
/* colour plane row of L/2 spins as L/16 bytes, compacted column j at bit j%8 */
/* of byte j/8, 1 for +1 and 0 for -1; rows dense.                            */
/* ------------------------------------------------------------------------- */
void oracle_to_planes_bits(int64_t L, const int8_t *s, uint8_t *black, uint8_t *white)
{
    int64_t rb = L / 16;
    for (int64_t k = 0; k < L * rb; k++) {
        black[k] = 0;
        white[k] = 0;
    }
    for (int64_t i = 0; i < L; i++)
        for (int64_t c = 0; c < L; c++) {
            uint8_t *dst = (colour_of(i, c) == 0 ? black : white) + i * rb;
            int64_t j = c / 2;
            if (s[i * L + c] > 0) dst[j / 8] |= (uint8_t)(1u << (j % 8));
        }
}

void oracle_from_planes_bits(int64_t L, const uint8_t *black, const uint8_t *white, int8_t *s)
{
    int64_t rb = L / 16;
    for (int64_t i = 0; i < L; i++)
        for (int64_t c = 0; c < L; c++) {
            const uint8_t *src = (colour_of(i, c) == 0 ? black : white) + i * rb;
            int64_t j = c / 2;
            s[i * L + c] = ((src[j / 8] >> (j % 8)) & 1) ? 1 : -1;
        }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Batches of lattices with replica exchange (parallel tempering).            */
/*                                                                            */
/* Not in the paper: a batch of n independent lattices (sides L[i]) swept     */
/* together.  Lattice i draws with stream i.  Lattices [l*S, (l+1)*S) form    */
/* ladder l over S inverse temperatures beta[0] < ... < beta[S-1]; lattice i  */
/* sits at slot slot_of[i] and is swept at beta[slot_of[i]]; lattice_at[l*S+k] */
/* is the lattice at slot k of ladder l.                                       */
/*                                                                            */
/* After sweep t, when record_every > 0 and (t + 1) % record_every == 0, event */
/* e = (t + 1) / record_every - 1 happens: each lattice's {sum s, sum bonds}   */
/* is recorded at trace[e - e_first][l*S + k] for the lattice at (l, k), and,  */
/* with swaps on, adjacent slots (k, k+1), k = (e mod 2), (e mod 2) + 2, ...   */
/* exchange their lattices with the replica-exchange probability              */
/*   P = min(1, exp((beta[k+1] - beta[k]) (E_b - E_a))),  E = -sum bonds,      */
/* a at slot k, b at slot k+1: the ratio of the joint Boltzmann weights after  */
/* and before the exchange.  E_b - E_a = bonds_a - bonds_b = D is a multiple  */
/* of 4 on a periodic lattice with even sides; for D < 0 the threshold is      */
/*   TS = floor(2^32 exp(-x)),  x = (beta[k+1] - beta[k]) * (double)(-D)       */
/* (2^32 when exp(-x) >= 1) and the pair swaps iff its draw u < TS, u the      */
/* purpose-2 draw of site k in stream l at sweep t (colour 0).                 */
/* ------------------------------------------------------------------------- */
uint64_t oracle_swap_threshold(double beta_lo, double beta_hi, int64_t D)
{
    if (D >= 0) return (uint64_t)1 << 32;
    double x = (beta_hi - beta_lo) * (double)(-D);
    double p = exp(-x);
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

/*
 * lattice_base lets the oracle run a piece of a larger batch: its lattices
 * are lattices lattice_base .. lattice_base + n - 1 of that batch (streams
 * lattice_base + i; ladder streams lattice_base / S + l).
 */
int oracle_batch_run(int64_t n, const int64_t *L, int8_t *spins, int64_t S, const double *beta,
                     int32_t *slot_of, int32_t *lattice_at, int64_t n_sweeps, uint64_t seed, uint64_t off,
                     int64_t record_every, int swaps, int64_t *trace, int nthreads, int64_t lattice_base)
{
    if (n <= 0 || S <= 0 || n % S != 0 || n_sweeps < 0 || lattice_base < 0 || lattice_base % S != 0) return 1;
    int64_t n_ladders = n / S;
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *obs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * n));
    uint64_t (*T)[5] = malloc(sizeof(uint64_t[5]) * (size_t)S);
    if (!start || !obs || !T) return 2;
    start[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        if (L[i] <= 0 || (L[i] & 1)) return 1;
        start[i + 1] = start[i] + L[i] * L[i];
    }
    for (int64_t k = 0; k < S; k++)
        if (oracle_thresholds(beta[k], T[k])) return 1;
    int64_t e_first = -1;
    for (int64_t s = 0; s < n_sweeps; s++) {
        uint64_t t = off + (uint64_t)s;
        for (int64_t i = 0; i < n; i++) {
            const uint64_t *Ti = T[slot_of[i]];
            uint32_t stream = (uint32_t)(lattice_base + i);
            oracle_half_sweep_stream(L[i], spins + start[i], 0, Ti, seed, t, stream, nthreads);
            oracle_half_sweep_stream(L[i], spins + start[i], 1, Ti, seed, t, stream, nthreads);
        }
        if (record_every <= 0 || (t + 1) % (uint64_t)record_every != 0) continue;
        int64_t e = (int64_t)((t + 1) / (uint64_t)record_every) - 1;
        if (e_first < 0) e_first = e;
        for (int64_t i = 0; i < n; i++) oracle_observables(L[i], spins + start[i], obs + 2 * i);
        for (int64_t l = 0; l < n_ladders; l++) {
            if (trace) {
                for (int64_t k = 0; k < S; k++) {
                    int64_t x = lattice_at[l * S + k];
                    int64_t *dst = trace + 2 * ((e - e_first) * n + l * S + k);
                    dst[0] = obs[2 * x];
                    dst[1] = obs[2 * x + 1];
                }
            }
            if (!swaps) continue;
            for (int64_t k = e & 1; k + 1 < S; k += 2) {
                int32_t a = lattice_at[l * S + k], b = lattice_at[l * S + k + 1];
                int64_t D = obs[2 * a + 1] - obs[2 * b + 1];
                uint64_t TS = oracle_swap_threshold(beta[k], beta[k + 1], D);
                uint32_t u = oracle_draw_stream(seed, (uint32_t)(lattice_base / S + l), (uint64_t)k, t, 0, 2);
                if ((uint64_t)u < TS) {
                    lattice_at[l * S + k] = b;
                    lattice_at[l * S + k + 1] = a;
                    slot_of[a] = (int32_t)(k + 1);
                    slot_of[b] = (int32_t)k;
                }
            }
        }
    }
    free(start);
    free(obs);
    free(T);
    return 0;
}
