/*
 * ising.h -- C ABI of libising: checkerboard Metropolis sweeps of the 2D
 * ferromagnetic Ising model (J = 1, h = 0, periodic L x L) on one GPU.
 *
 * Method: Romero, Bisson, Fatica, Bernaschi, "A Performance study of the 2D
 * Ising model on GPUs" (arXiv:1906.06297).  Sec. 2 defines the model (Eq. 1),
 * the Metropolis rule and the checkerboard decomposition; Sec. 3.1 and Fig. 1
 * the two colour planes of N x N/2 spins compacted along rows; Fig. 2 the
 * per-site update (neighbour indexing by colour and row parity, acceptance
 * exp(-2 beta nn s)); Sec. 3.3 and Fig. 3 the multi-spin-coded lattice with
 * 4 bits per spin and one launch per colour per step.
 *
 * Conventions shared by every entry point
 *   - Site (i, c) (row i, column c, 0 <= i, c < L) is BLACK iff (i + c) is
 *     even, WHITE otherwise.  It lives in its colour's plane at row i,
 *     compacted column j = c / 2.  L must be even.
 *   - A sweep is a black half-sweep followed by a white half-sweep.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed_lo, seed_hi) and counter (q_lo, q_hi, t_lo,
 *     colour | purpose << 1 | t_hi << 8), where site = i * (L/2) + j,
 *     q = site >> 2, t = sweep index, and the site's draw is output word
 *     (site & 3).  purpose 0 = Metropolis, 1 = random initial state.  The
 *     result therefore depends only on (seed, t, colour, site), never on the
 *     launch shape.
 *   - Acceptance: a = number of the 4 neighbours equal to the spin,
 *     dE = 4a - 8, p_a = min(1, exp(-beta dE)); T[a] = 2^32 if p_a >= 1 else
 *     floor(p_a * 2^32) (built once per call on the host in FP64); the spin
 *     flips iff (uint64) u < T[a].
 *   - Layouts of one colour plane (rows of `row_stride_bytes` bytes):
 *       ISING_INT8: L rows x L/2 int8 spins (+1 / -1), Sec. 3.1.
 *       ISING_MSC4: L rows x L/32 uint64 words; column j is word j/16, bits
 *         4*(j%16) .. 4*(j%16)+3, value 1 for +1 and 0 for -1 (Sec. 3.3).
 *         Needs L % 64 == 0, 16-byte aligned planes and a row stride that is a
 *         multiple of 16 bytes.
 *   - Memory: every pointer argument named *_dev is device memory owned by
 *     the caller; the library allocates nothing.  Calls are asynchronous on
 *     the given stream (NULL = legacy default stream) unless stated.
 *   - Errors: every call returns an ising_status; arguments are checked before
 *     any work is queued, and nothing aborts the process.
 *   - Per-device state: streams, events, instantiated graphs and symbol
 *     addresses that some entry points create on first use are kept per
 *     device for the life of the process.  Do not use the library on a device
 *     after a cudaDeviceReset of that device.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ISING_API __attribute__((visibility("default")))
#else
#define ISING_API
#endif

/* Same object as cudaStream_t; declared here so this header needs no CUDA. */
typedef struct CUstream_st *ising_stream_t;

typedef enum {
    ISING_OK = 0,
    ISING_EINVAL = 1,   /* bad argument: see ising_strerror / the entry point */
    ISING_ECUDA = 2,    /* a CUDA runtime call or a launch failed */
    ISING_ETIMEOUT = 3, /* a bounded device wait gave up */
} ising_status;

typedef enum { ISING_INT8 = 0, ISING_MSC4 = 1 } ising_layout;

typedef enum { ISING_INIT_RANDOM = 0, ISING_INIT_UP = 1, ISING_INIT_DOWN = 2 } ising_init_mode;

/* A lattice: two caller-owned device planes.  Plain data; copy freely. */
typedef struct {
    void *black;              /* device pointer, colour 0 */
    void *white;              /* device pointer, colour 1 */
    int64_t L;                /* side length (even; MSC4: multiple of 64) */
    int32_t layout;           /* ising_layout */
    int32_t reserved;         /* must be 0 */
    int64_t row_stride_bytes; /* bytes between plane rows; >= the row size */
} ising_lattice_t;

/* Bytes of one colour plane row (`row_bytes`, the minimum row stride) and of
 * one dense plane (`plane_bytes` = L * row_bytes).  Either output may be NULL.
 * EINVAL: L <= 0, L odd, MSC4 with L % 64 != 0, unknown layout. */
ISING_API int ising_lattice_bytes(int64_t L, int32_t layout, size_t *row_bytes, size_t *plane_bytes);

/* Host, synchronous: the acceptance table for beta (Sec. 2, Metropolis rule)
 * exactly as the kernels use it.  EINVAL: beta < 0 or not finite, T NULL. */
ISING_API int ising_thresholds(double beta, uint64_t T[5]);

/* Fill both planes: ISING_INIT_RANDOM gives spin +1 iff the purpose-1 draw at
 * t = 0 is below 2^31; UP / DOWN give all +1 / all -1. */
ISING_API int ising_init_lattice(const ising_lattice_t *lat, int32_t init, uint64_t seed,
                                 ising_stream_t stream);

/* One half-sweep of colour `colour` (0 black, 1 white) at sweep index t
 * (Sec. 2 checkerboard; Fig. 2 per-site rule).  If obs_dev is not NULL the
 * kernel ADDS {sum of spins, sum over bonds s_i s_j} of the whole lattice
 * after the update to obs_dev[0..1] (int64, caller zeroes it); this is only
 * supported for colour 1, where every bond has exactly one white end. */
ISING_API int ising_half_sweep(const ising_lattice_t *lat, double beta, int32_t colour, uint64_t seed,
                               uint64_t t, int64_t *obs_dev, ising_stream_t stream);

/* n_sweeps sweeps with sweep indices sweep_offset .. sweep_offset+n_sweeps-1
 * (Sec. 3.3: two launches per step, black then white).  trace_dev, if not
 * NULL, receives n_sweeps x 2 int64 {sum of spins, sum over bonds} after each
 * sweep (the call zeroes it first).  Running a sweeps and then b sweeps with
 * offset a gives the same lattice as a + b sweeps in one call. */
ISING_API int ising_sweep(const ising_lattice_t *lat, double beta, int64_t n_sweeps, uint64_t seed,
                          uint64_t sweep_offset, int64_t *trace_dev, ising_stream_t stream);

/* Same as ising_sweep, for a lattice held in host memory: copies the dense
 * host planes (L rows of ising_lattice_bytes' row_bytes each) into the
 * caller's device lattice `dev`, runs the sweeps, and copies the planes and
 * the trace (if trace_host is not NULL; trace_dev is then required as device
 * staging of n_sweeps x 2 int64) back.  Pinned host memory makes the copies
 * asynchronous; the call does not synchronise the stream.  One sweep of an
 * MSC4 lattice runs in row bands (about 16 MiB of host plane each, smaller
 * first and last bands) on streams of the library's own: plane bands are
 * copied in in the order the half-sweeps need them and each is copied out as
 * soon as it is final, so that both directions of the host link are busy
 * while the bands are swept.  The schedule is captured and replayed on
 * `stream` as a CUDA graph (launched directly if capture fails); the work is
 * ordered on `stream` (it starts after the work queued on it and the stream
 * waits for all of it), and the result is that of ising_sweep.  Calls on one
 * device are serialised while they queue work. */
ISING_API int ising_sweep_host(const ising_lattice_t *dev, void *black_host, void *white_host, double beta,
                               int64_t n_sweeps, uint64_t seed, uint64_t sweep_offset, int64_t *trace_dev,
                               int64_t *trace_host, ising_stream_t stream);

/* Bit-packed format of an MSC4 lattice's colour planes (an I/O format, not
 * in the paper): L rows of L/2 bits, L/16 bytes per row, rows dense;
 * compacted column j of a row is bit j % 8 of the row's byte j / 8, 1 for an
 * up spin and 0 for a down spin.  These are the MSC4 plane's spins in the
 * same order at one bit each instead of four (Sec. 3.3 spends four bits per
 * spin for the bit-parallel neighbour sums, which storage and transfers do not
 * need), so a lattice crosses the host link in a quarter of the bytes.
 * L % 64 == 0.  *bytes_per_plane = L * L / 16. */
ISING_API int ising_bits_bytes(int64_t L, size_t *bytes_per_plane);

/* MSC4 device lattice -> bit planes in device memory (ising_bits_bytes each,
 * 4-byte aligned), and back.  Asynchronous on `stream`. */
ISING_API int ising_msc4_to_bits(const ising_lattice_t *msc4, void *black_bits, void *white_bits,
                                 ising_stream_t stream);
ISING_API int ising_bits_to_msc4(const void *black_bits, const void *white_bits, const ising_lattice_t *msc4,
                                 ising_stream_t stream);

/* ising_sweep_host for a lattice held in host memory in the bit-packed
 * format: black_host / white_host are bit planes (4-byte aligned; pinned for
 * asynchronous copies), `dev` an MSC4 device lattice of the same L that holds
 * the state during the call, stage_dev caller-owned device scratch of
 * 2 x ising_bits_bytes (16-byte aligned).  One sweep runs in row bands as in
 * ising_sweep_host, each band converted on the device after its copy in and
 * before its copy out; n_sweeps != 1 copies and converts whole planes.  The
 * result equals ising_sweep on the unpacked lattice, converted back. */
ISING_API int ising_sweep_host_bits(const ising_lattice_t *dev, void *black_host, void *white_host,
                                    void *stage_dev, double beta, int64_t n_sweeps, uint64_t seed,
                                    uint64_t sweep_offset, int64_t *trace_dev, int64_t *trace_host,
                                    ising_stream_t stream);

/* out_dev[0..1] = {sum of spins, sum over bonds s_i s_j}: magnetisation
 * M = out[0], energy E = -out[1] (Eq. 1 with J = 1). */
ISING_API int ising_observables(const ising_lattice_t *lat, int64_t *out_dev, ising_stream_t stream);

/* Convert between layouts (same L): int8 planes -> MSC4 planes and back. */
ISING_API int ising_pack(const ising_lattice_t *int8_src, const ising_lattice_t *msc4_dst, ising_stream_t stream);
ISING_API int ising_unpack(const ising_lattice_t *msc4_src, const ising_lattice_t *int8_dst, ising_stream_t stream);

/* The random stream alone, as the MSC4 sweep draws it: for q in [0, n_blocks)
 * compute the Philox block with counter (q_lo, q_hi, t_lo, colour | t_hi << 8)
 * and key (seed), compare each of its 4 words with threshold T3 and ADD the
 * number of words below it to *count_dev (uint64, caller zeroes it).  Used to
 * measure the generator's throughput ceiling and to check the stream.  The
 * kernel is shaped like the sweep's draws: each thread step makes 8 blocks
 * sharing counter words 1..3, with 32-bit indices, on a full grid.  EINVAL:
 * colour not 0 or 1, n_blocks > 2^34. */
ISING_API int ising_rng_probe(uint64_t n_blocks, uint64_t seed, uint64_t t, int32_t colour, uint32_t T3,
                              uint64_t *count_dev, ising_stream_t stream);

/* Throughput probe of the 32 x 32 -> 64-bit multiply that every Philox round
 * is built on (two per round, 20 per block of 4 draws; Sec. 3.3 draws the
 * random numbers inside the sweep kernel, so this multiply bounds it).  Not a
 * step of the method.  One launch on a full grid of the current device:
 * every thread runs 16 independent chains of `iters` dependent wide
 * multiplies, with no memory traffic.  form 0 is the multiply as a Philox
 * round issues it (by an immediate multiplier, no addend; the chain goes on
 * through the XOR of the product's halves); form 1 is a multiply-add with a
 * 64-bit register addend.  *multiplies (host) receives the number of wide
 * multiplies the launch performs; time the launch on `stream` to get the
 * rate.  sink_dev (one uint64, device) may be incremented: it keeps the
 * chains from being optimised away.  EINVAL: form not 0 or 1, iters == 0,
 * NULL pointers. */
ISING_API int ising_mulwide_probe(int32_t form, uint32_t iters, uint64_t *sink_dev, uint64_t *multiplies,
                                  ising_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Horizontal slabs (Sec. 4: the lattice is cut into horizontal slabs, each   */
/* kept in the single-GPU layout, and a slab's update needs only the boundary */
/* rows of the slabs above and below).  Here those boundary rows are staged   */
/* explicitly into halo rows: a slab holds rows row0 .. row0+rows-1 of the    */
/* L x L lattice plus, in each colour plane, one halo row above (global row   */
/* row0-1 mod L) and one below (row0+rows mod L).  The paper reaches the      */
/* neighbours' rows through unified memory instead; explicit halos give the   */
/* same reads and work within one process, across processes and across GPUs.  */
/* Because the random numbers are keyed by the global site, a lattice swept   */
/* as slabs is bit-identical to the same lattice swept whole.  MSC4 only.     */
/* ------------------------------------------------------------------------ */

/* One slab: two caller-owned device planes of rows + 2 rows each (plane row
 * 0 = halo above, rows 1 .. rows = the slab's own rows, row rows + 1 = halo
 * below), row stride row_stride_bytes (multiple of 16, planes 16-byte
 * aligned, as for an MSC4 lattice).  Plain data; copy freely. */
typedef struct {
    void *black;              /* device pointer, colour 0, halo row above first */
    void *white;              /* device pointer, colour 1 */
    int64_t L;                /* side of the whole lattice (multiple of 64) */
    int64_t row0;             /* global row of the first own row, 0 <= row0 < L */
    int64_t rows;             /* own rows, 1 <= rows, row0 + rows <= L */
    int32_t layout;           /* must be ISING_MSC4 */
    int32_t spare_sms;        /* SMs the half-sweep kernel leaves without a block
                                 (0: none; at most the device's SMs - 1), so that
                                 kernels of another stream, such as the halo
                                 messages of a multi-rank sweep, can run beside
                                 it */
    int64_t row_stride_bytes; /* bytes between plane rows; >= L / 4 */
} ising_slab_t;

/* Bytes of one slab plane row (`row_bytes` = L / 4) and of one dense slab
 * plane (`plane_bytes` = (rows + 2) * row_bytes).  Either output may be NULL.
 * EINVAL: bad L, rows < 1, layout other than MSC4. */
ISING_API int ising_slab_bytes(int64_t L, int64_t rows, int32_t layout, size_t *row_bytes, size_t *plane_bytes);

/* Fill the slab's own rows of both planes exactly as ising_init_lattice fills
 * those rows of the whole lattice; halo rows are not touched. */
ISING_API int ising_slab_init(const ising_slab_t *slab, int32_t init, uint64_t seed, ising_stream_t stream);

/* One half-sweep of colour `colour` over the slab's own rows at sweep index t
 * (same rule and random numbers as ising_half_sweep).  The halo rows of the
 * OTHER colour must hold the current neighbour rows (ising_slab_exchange, or
 * the caller's own transfer).  obs_dev (colour 1 only) receives ADDED
 * {sum of spins, sum over bonds} of the slab's own rows after the update,
 * counting each bond once at its white end: summed over the slabs of a
 * lattice they give the lattice's values. */
ISING_API int ising_slab_half_sweep(const ising_slab_t *slab, double beta, int32_t colour, uint64_t seed,
                                    uint64_t t, int64_t *obs_dev, ising_stream_t stream);

/* Make the colour-`colour` halo rows of n slabs current, for slabs on the
 * current device that together form one lattice: slab k covers the rows
 * right after slab k-1 (slab 0 starts at row 0, slab n-1 ends at row L-1).
 * The halo above slab k receives the last own row of slab k-1, the halo below
 * it the first own row of slab k+1 (periodic: slab 0's upper neighbour is
 * slab n-1; one slab is its own neighbour).  One launch, 2n row copies;
 * 1 <= n <= 64. */
ISING_API int ising_slab_exchange(const ising_slab_t *slabs, int32_t n, int32_t colour, ising_stream_t stream);

/* n_sweeps sweeps of the lattice held as n slabs (arranged as for
 * ising_slab_exchange): per sweep, white halos, every slab's black half-sweep,
 * black halos, every slab's white half-sweep.  trace_dev as for ising_sweep
 * (whole-lattice sums; the call zeroes it first).  The result equals
 * ising_sweep on the whole lattice, bit for bit. */
ISING_API int ising_slab_sweep(const ising_slab_t *slabs, int32_t n, double beta, int64_t n_sweeps, uint64_t seed,
                               uint64_t sweep_offset, int64_t *trace_dev, ising_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batches of lattices with replica exchange.  Not in the paper: the batched */
/* form of its sweep.  n lattices (sides L[i], multiples of 32 up to 65536,  */
/* MSC4 planes) are swept together in ONE persistent cooperative launch with */
/* grid-wide barriers (each wait bounded: a timeout sets ISING_ETIMEOUT,     */
/* read back by ising_batch_check).  Lattices [l*S, (l+1)*S) form ladder l   */
/* over S increasing inverse temperatures beta[0..S-1]; lattice i starts at  */
/* slot i mod S and is swept at the beta of its current slot.  Lattice i     */
/* draws in stream i (i added to Philox counter word 1), so lattice 0 follows */
/* the single-lattice trajectory for the same seed.                          */
/*                                                                           */
/* After sweep t with (t + 1) % record_every == 0 (event e = (t+1)/record_every */
/* - 1): every lattice's {sum s, sum bonds} goes to trace[e - e_first][l*S+k] */
/* for the lattice at slot k of ladder l (e_first = first event of the call) */
/* and, with swaps on, slot pairs (k, k+1), k = e mod 2, e mod 2 + 2, ...     */
/* exchange lattices iff u < floor(2^32 exp(-(beta[k+1]-beta[k]) m)), where  */
/* m = bonds_b - bonds_a if that is positive (else always), a at slot k, b at */
/* k+1, and u the purpose-2 draw of site k in stream l at sweep t: the       */
/* replica-exchange probability min(1, exp((beta[k+1]-beta[k])(E_b - E_a))). */
/*                                                                           */
/* All device memory is one caller-owned workspace (ising_batch_bytes); the  */
/* handle itself is host memory owned by the library until destroy.          */
/* ------------------------------------------------------------------------ */
typedef struct ising_batch ising_batch_t;

/* Workspace bytes for a batch.  EINVAL: n not a multiple of S, a side not a
 * multiple of 32 in [32, 65536], unequal sides within a ladder, betas not
 * increasing by >= 1e-4 or not > 0, or a beta so small (below about 1.4e-17)
 * that exp(-4 beta) rounds to 1: the batched decision holds the a = 3 and
 * a = 4 thresholds as 32-bit words and has no form for the always-flip
 * entry 2^32. */
ISING_API int ising_batch_bytes(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta,
                                size_t *bytes);

/* Lay a batch out in `workspace_dev` (device, 256-byte aligned, at least
 * ising_batch_bytes) and upload its tables (synchronous).  *out receives the
 * host handle. */
ISING_API int ising_batch_create(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta,
                                 void *workspace_dev, size_t workspace_bytes, ising_batch_t **out);
ISING_API int ising_batch_destroy(ising_batch_t *batch);

/* Initial planes (ISING_INIT_*; random: lattice i draws in stream i), identity
 * slots, cleared accumulators and barrier. */
ISING_API int ising_batch_init(ising_batch_t *batch, int32_t init, uint64_t seed, ising_stream_t stream);

/* n_sweeps sweeps with indices sweep_offset.. in one persistent launch
 * (replayed from a captured CUDA graph when use_graph != 0).  trace_dev
 * (nullable) receives events x n x 2 int64 as described above.  swaps needs
 * record_every > 0.  Asynchronous: ising_batch_check reports barrier
 * timeouts. */
ISING_API int ising_batch_run(ising_batch_t *batch, int64_t n_sweeps, uint64_t seed, uint64_t sweep_offset,
                              int32_t record_every, int32_t swaps, int64_t *trace_dev, int32_t use_graph,
                              ising_stream_t stream);

/* Synchronises `stream` and returns ISING_ETIMEOUT (or EINVAL for a device-side
 * consistency failure) if a launch of this batch reported one, clearing it. */
ISING_API int ising_batch_check(ising_batch_t *batch, ising_stream_t stream);

/* Device pointers of the concatenated planes and the word offset of each
 * lattice's plane (host array of n + 1), and of the slot state arrays. */
ISING_API int ising_batch_planes(const ising_batch_t *batch, void **black_dev, void **white_dev,
                                 int64_t *word_offsets);
ISING_API int ising_batch_state(const ising_batch_t *batch, int32_t **slot_of_dev, int32_t **lattice_at_dev);

/* Launch shape: 256 or 512 threads per block, 1, 2 or 4 words per thread (per
 * lattice the largest that divides its words per row).  Results do not depend
 * on it.  ising_batch_autotune times every shape for n_sweeps sweeps on a copy
 * of the planes (in the workspace) and keeps the fastest. */
ISING_API int ising_batch_config(ising_batch_t *batch, int32_t threads, int32_t words_per_thread);
ISING_API int ising_batch_get_config(const ising_batch_t *batch, int32_t *threads, int32_t *words_per_thread);
ISING_API int ising_batch_autotune(ising_batch_t *batch, int64_t n_sweeps, ising_stream_t stream);

/* Self-test of the bounded grid barrier: a launch on the workspace's tuning
 * copy whose barrier waits for one block more than the grid holds, so every
 * wait runs out after timeout_cycles SM clocks.  Returns ISING_ETIMEOUT when
 * the kernel gave up and returned as designed. */
ISING_API int ising_batch_barrier_selftest(ising_batch_t *batch, int64_t timeout_cycles, ising_stream_t stream);

/* Allocation-free form of ising_batch_run.  The paper has no counterpart.
 * For callers that may not allocate device memory themselves (code running
 * under another framework's memory manager, which owns the device budget and
 * does not let plug-ins call cudaMalloc; latency-bound loops where an
 * allocation could synchronise the device): the batch is described by its
 * arrays as in ising_batch_bytes, the caller passes the planes (black_dev,
 * white_dev: the concatenated MSC4 planes laid out as ising_batch_planes
 * reports, lattice i at word offset sum_{j<i} L_j^2/32), the slot state
 * (slot_of_dev, lattice_at_dev: n int32 each, e.g. the identity slot i mod S
 * and lattice i), and an optional trace; all other scratch (tables,
 * accumulators, barrier words) lives in a fixed 4 MiB array inside the
 * library, which every GPU that loads the library holds until exit.  Batches
 * whose scratch exceeds it are rejected with ISING_EINVAL and a message
 * giving the size.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process: do not use the library across a cudaDeviceReset.  Calls
 * share the array: calls that overlap on the GPU race.  Each call clears what
 * must start at zero.  Synchronous (it waits on `stream` and reads words back
 * to the host), so it can never be called on a capturing stream: returns
 * after the sweeps, with ISING_ETIMEOUT if a barrier wait ran out.  Before
 * any launch it checks the caller's buffers: planes 16-byte aligned, trace
 * 8-byte and slot arrays 4-byte aligned, each inside its device allocation;
 * the slot arrays are read back and must be a valid state (slot_of[i] in
 * [0, S), lattice_at[l*S + k] a lattice of ladder l, the two inverse to each
 * other), else ISING_EINVAL.  Results equal ising_batch_run's for the same
 * arguments. */
ISING_API int ising_batch_run_noalloc(int64_t n, const int64_t *L, int32_t ladder_size, const double *beta,
                                      void *black_dev, void *white_dev, int32_t *slot_of_dev,
                                      int32_t *lattice_at_dev, int64_t n_sweeps, uint64_t seed,
                                      uint64_t sweep_offset, int32_t record_every, int32_t swaps,
                                      int64_t *trace_dev, ising_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Learned block proposals.  Not in the paper: a Metropolis-Hastings move    */
/* that flips one 8 x 8 block, proposed by a small convolutional network,    */
/* layered on the checkerboard sweep.  Chains are C lattices of side L       */
/* (multiple of 32, at most 4096) laid out as a batch of equal sides:        */
/* lattice c's planes at word c * L * L/32 of the black and white buffers.    */
/* Network: three 3x3 periodic conv layers of 32 channels with GELU (the    */
/* first reads the spins), a 3x3 conv to one channel, and the mean over each  */
/* 8 x 8 block gives that block's logit (b = by * L/8 + bx).  A BF16 network: */
/* weights are rounded to bfloat16 for every use and each activation is      */
/* stored as bfloat16 (round to nearest even); products accumulate in FP32;  */
/* the 32 -> 32 layers run on the tensor cores.  Every reduction has a fixed  */
/* order, so logits are a deterministic function of the state.               */
/* Parameters: one FP32 vector of ising_net_param_count() values,            */
/* W1[32][9], b1[32], W2[32][32][9], b2[32], W3[32][32][9], b3[32], W4[32][9], */
/* b4[1] (tap k = 3 (dy + 1) + (dx + 1)).                                     */
/* ------------------------------------------------------------------------ */
ISING_API int ising_net_param_count(void);

/* Device work-buffer bytes of a forward (train = 0) or a forward + backward
 * (train = 1) over C chains of side L. */
ISING_API int ising_net_workspace_bytes(int64_t L, int64_t C, int32_t train, size_t *bytes);

/* logits_dev[c][b] for every chain; flip_block_dev (nullable, int32[C], -1 for
 * none) evaluates each chain with that block flipped.  train != 0 keeps the
 * activations in work_dev for ising_net_backward. */
ISING_API int ising_net_forward(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                const int32_t *flip_block_dev, const float *params_dev, float *logits_dev,
                                void *work_dev, size_t work_bytes, int32_t train, ising_stream_t stream);

/* The logits of the flipped states, the second network evaluation of a block
 * move: logits_dev[c] = the logits of chain c with block flip_block_dev[c]
 * flipped, given logits_x_dev = this network's logits of the unflipped chains
 * (same params, same planes; another buffer).  A flipped block changes the
 * activations only within 4 rows of it (four 3 x 3 layers), so for L a
 * multiple of 128 only a band of 30 rows per chain is recomputed and the
 * logits outside the block row and its two neighbours are copied from
 * logits_x_dev; the result equals ising_net_forward with flip_block_dev bit
 * for bit.  Other L compute the whole forward.  Inference workspace. */
ISING_API int ising_net_forward_flipped(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                        const int32_t *flip_block_dev, const float *params_dev,
                                        const float *logits_x_dev, float *logits_dev, void *work_dev,
                                        size_t work_bytes, ising_stream_t stream);

/* Synchronises `stream`, then reports ISING_ETIMEOUT (and clears the flag) if
 * a tensor-core kernel of the network gave up waiting for its MMAs since the
 * last check (each such wait is bounded at about 2 s), else ISING_OK. */
ISING_API int ising_net_check(ising_stream_t stream);

/* Failure-path self-test of the tensor-core kernels' bounded waits: runs one
 * forward (L a multiple of 128) in which the first 32-channel layer never
 * signals the completion of its first accumulator.  The waits that depend on
 * it give up after about 2 s, every CTA frees its tensor memory and returns,
 * and the next ising_net_check reports ISING_ETIMEOUT; the device stays usable.
 * logits_dev receives meaningless values.  Not part of the method. */
ISING_API int ising_net_wait_selftest(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                     const float *params_dev, float *logits_dev, void *work_dev, size_t work_bytes,
                                     ising_stream_t stream);

/* grad_dev = d(sum dlogits * logits)/d(params) for the last training forward
 * on the same chains and parameters (straight-through the bfloat16 rounding).
 * For L a multiple of 128 the data and weight gradients of the 32 -> 32
 * layers run on the tensor cores (the weight gradients see the output
 * gradient as two bfloat16 parts, its rounding and the rounding of the
 * remainder, which carry it to about 2^-17); a bounded wait that gives up there
 * is reported by the next ising_net_check.  Every weight gradient is a sum of
 * per-CTA partials in a fixed order: the result is deterministic. */
ISING_API int ising_net_backward(int64_t L, int64_t C, const void *black_dev, const void *white_dev,
                                 const float *params_dev, const float *dlogits_dev, float *grad_dev, void *work_dev,
                                 size_t work_bytes, ising_stream_t stream);

/* Regression of the block acceptance: t_b = min(0, -beta dE_b) from the exact
 * block energy changes; dlogits = 2 (logits - t) / (C nb) (the gradient of the
 * mean squared residual), chain_sq_dev[c] = that chain's squared residual sum,
 * *loss_dev = the mean squared residual. */
ISING_API int ising_net_targets_loss(int64_t L, int64_t C, const void *black_dev, const void *white_dev, double beta,
                                     const float *logits_dev, float *dlogits_dev, float *chain_sq_dev,
                                     float *loss_dev, ising_stream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected at `step`). */
ISING_API int ising_net_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int64_t step,
                             float lr, ising_stream_t stream);

/* Draw one block per chain: inverse CDF of softmax(logits) (FP64, block order)
 * with the purpose-3 draw of site 0 in stream c at step t, or uniformly
 * ((u * nb) >> 32) when logits_dev is NULL. */
ISING_API int ising_block_propose(int64_t L, int64_t C, const float *logits_dev, uint64_t seed, uint64_t t,
                                  int32_t *block_dev, ising_stream_t stream);

/* Accept or reject flipping block_dev[c] of each chain: dE = twice the sum of
 * the boundary bonds s_in s_out (exact); x = -beta dE + log q_x'(b) -
 * log q_x(b) (logits of the state and of the flipped state; both NULL for
 * uniform proposals); flip iff the purpose-3 draw of site 1 is below
 * floor(2^32 min(1, exp(x))).  accepted_dev[c] = 0/1, dE_dev (nullable) = dE. */
ISING_API int ising_block_accept(int64_t L, int64_t C, void *black_dev, void *white_dev, double beta,
                                 const float *logits_x_dev, const float *logits_xp_dev, const int32_t *block_dev,
                                 uint64_t seed, uint64_t t, int32_t *accepted_dev, int64_t *dE_dev,
                                 ising_stream_t stream);

/* Text of the last learned-proposal API failure seen by this thread. */
ISING_API const char *ising_net_last_error(void);

/* Text of the last batch-API failure seen by this thread. */
ISING_API const char *ising_batch_last_error(void);

/* Static description of a status code. */
ISING_API const char *ising_strerror(int status);

/* Text of the last EINVAL / ECUDA reason seen by this thread ("" if none). */
ISING_API const char *ising_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ISING_H */
