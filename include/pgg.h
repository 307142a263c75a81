/*
 * pgg.h -- C ABI of the GB300 (sm_103a) library for the spatial public goods game
 * Monte Carlo of Perc, "High-performance parallel computing in the classroom using
 * the public goods game as an example" (arXiv:1704.08098).
 *
 * The model (Section III): L x L periodic square lattice, strategies C (1) and D (0);
 * every player belongs to G = 5 overlapping groups (Fig. 1); in a group with N_C
 * cooperators a cooperator earns r N_C / 5 - 1 and a defector r N_C / 5 (Eq. (1)-(2),
 * c = 1); a player's payoff is the sum over its five groups. An elementary step lets a
 * player x adopt the strategy of a random nearest neighbour y with the Fermi
 * probability W = 1 / (1 + exp((P_x - P_y) / K)) (Eq. (3)); L^2 elementary steps are
 * one full Monte Carlo step (MCS). The observable is the cooperator fraction rho_C
 * (Eq. (4)).
 *
 * Parallel schedule: the random-sequential order of Section III is replaced by
 * sublattice steps. Step k updates, at once, every site (i, j) with
 * (i mod 4, j mod 4) equal to an offset drawn for step k; such sites are at least 4
 * apart and an update reads only sites within Manhattan distance 3 (Section IV,
 * Fig. 3), so the updates of one step are independent. 16 steps make one MCS.
 *
 * Randomness: Philox4x32-10 keyed by the 64-bit seed; every draw is a function of
 * (seed, step, site), so results do not depend on the launch configuration. The
 * counter layout is:
 *   init    (q_lo, q_hi, 0, 1<<24), q = (i*L + j) >> 2, word (i*L + j) & 3 < floor(p 2^32)
 *   offset  (m_lo, m_hi, 0, 2<<24), m = k >> 5, o = (word[(k>>3)&3] >> 4(k&7)) & 15,
 *           row offset o >> 2, column offset o & 3
 *   dir     (b >> 6, a, k_lo, k_hi | 3<<24), d = (word[(b>>4)&3] >> 2(b&15)) & 3,
 *           d = 0: (i, j+1), 1: (i, j-1), 2: (i+1, j), 3: (i-1, j)
 *   u       (b >> 2, a, k_lo, k_hi | 4<<24), u = word[b & 3]
 * where (a, b) are the sublattice coordinates of site (4a + row offset, 4b + column
 * offset) and k < 2^56 the step index. x adopts s_y iff s_x != s_y and u < T, with the
 * threshold T = floor(W 2^32) (2^32 - 1 when W >= 1) evaluated on the host in IEEE
 * double precision from P(s, S) = (r S)/5 - 5 s, S the sum of the cooperator counts of
 * the player's five groups.
 *
 * Conventions for every entry point:
 *   - Every function returns a pgg_status; no C++ exception crosses the ABI. On failure
 *     pgg_last_error() returns a message for the calling thread.
 *   - A context owns all device memory it allocates; host and device buffers passed
 *     in are borrowed for the duration of the call only (pgg_stage_lattice_packed: until
 *     its copy has completed, as stated there).
 *   - Work is enqueued on the CUDA stream given to pgg_create (borrowed, not owned;
 *     NULL = the legacy default stream). Calls are asynchronous on that stream unless
 *     stated otherwise. A context must not be used from two threads at once.
 *   - Lattices cross the ABI as L*L bytes, row-major, 1 = cooperator, 0 = defector, or,
 *     in the *_packed calls, as L rows of L/32 uint32 words (bit b of word w = column
 *     32w + b).
 */
#ifndef PGG_H
#define PGG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pgg_ctx pgg_ctx;

typedef enum {
    PGG_OK = 0,
    PGG_ERR_ARG = -1,     /* invalid argument; nothing was enqueued */
    PGG_ERR_CUDA = -2,    /* a CUDA call failed; the context may be unusable */
    PGG_ERR_OOM = -3,     /* device or pinned-host allocation failed */
    PGG_ERR_TIMEOUT = -4, /* a bounded device-side wait ran out; the kernel returned early */
    PGG_ERR_STATE = -5    /* call not valid in the current state */
} pgg_status;

/* Storage of the lattice on the device. */
typedef enum {
    PGG_U8 = 0,      /* one byte per site, L*L bytes; needs L % 4 == 0 */
    PGG_BITPACK = 1  /* one bit per site, 32 sites per uint32 along a row, bit b of
                        word w = column 32w + b; needs L % 32 == 0 */
} pgg_layout;

/* The game the lattice plays. */
typedef enum {
    PGG_GAME_GROUP = 0,   /* the public goods game in groups of five (Section III, Eq. (1)-(2));
                             the default */
    PGG_GAME_PAIRWISE = 1 /* a 2x2 matrix game with each of the four nearest neighbours, e.g.
                             the prisoner's dilemma (Section VI); an update reads one line
                             less in every direction (radius 2) */
} pgg_game;

/* Kernel family used by pgg_step_mcs. */
typedef enum {
    PGG_KERNEL_AUTO = 0,   /* the schedule pgg_autotune chose for (device, L, layout, game);
                              before any tuning: the resident kernel for L >= 2048 where it
                              fits, else the direct kernel (bit-packed, L % 256 == 0), else
                              the tiled kernel (L % 64 == 0), else the simple one */
    PGG_KERNEL_SIMPLE = 1, /* one launch per sublattice step, one thread per 8 sites,
                              operands from global memory; the plain baseline */
    PGG_KERNEL_TILED = 2,  /* shared-memory tiles with a 3k-site halo (2k for the pairwise
                              game), k sublattice
                              steps fused per launch (temporal blocking); k = 1 runs in
                              place, k > 1 ping-pongs between two lattice buffers */
    PGG_KERNEL_DIRECT = 3, /* bit-packed lattices with L % 256 == 0 only: one launch per
                              sublattice step, in place, operands straight from global
                              memory, tile_x = words per thread (4 or 8), tile_y = threads
                              per block (64, 128 or 256); the cooperator count is carried as
                              a running total */
    PGG_KERNEL_RESIDENT = 4 /* L % 256 == 0 with the bit-packed rows fitting the SMs'
                              shared memory: one cooperative launch per pgg_step_mcs call,
                              each CTA keeps a band of rows for all MCS and exchanges its
                              R s edge rows with its neighbours every s sublattice steps
                              (R = 3 group game, 2 pairwise; s = 1, 2 or 4, updating the
                              halo rows redundantly in between); only the active sites
                              (s_x != s_y) of a step are updated, gathered per warp; waits
                              are bounded (a time-out returns PGG_ERR_TIMEOUT at the next
                              synchronising call). A PGG_U8 lattice is packed as its bands
                              are staged and unpacked as they are written back */
} pgg_kernel;

/* Create a context for one L x L lattice with synergy factor r and noise K (Section III,
 * Eq. (1)-(3); G = 5, c = 1 fixed). Requires 4 <= L <= 32768, L % 4 == 0 (L % 32 == 0 for
 * PGG_BITPACK), r > 0, K > 0. Allocates the lattice and the 2x26x26 uint32 adoption
 * threshold table on the current CUDA device. The lattice starts all-defector with step 0
 * until pgg_seed or pgg_set_lattice. *out is set to NULL on failure. */
int pgg_create(pgg_ctx **out, int L, double r, double K, int layout, void *cuda_stream);

/* Change r and K (rebuilds the threshold table; the lattice is kept). Under
 * PGG_GAME_PAIRWISE, r is kept but unused. */
int pgg_set_params(pgg_ctx *ctx, double r, double K);

/* Choose the game (Section VI: the same parallel scheme for a game played pairwise).
 * PGG_GAME_GROUP ignores payoff (may be NULL). PGG_GAME_PAIRWISE needs payoff = {R, S, T, P}
 * (4 finite doubles, copied): the payoff of a cooperator meeting a cooperator (R) or a
 * defector (S), and of a defector meeting a cooperator (T) or a defector (P); the weak
 * prisoner's dilemma is {1, 0, b, 0}. A player with n cooperating neighbours then earns
 * n A + (4 - n) B, (A, B) = (R, S) for a cooperator and (T, P) for a defector, evaluated in
 * IEEE double precision without contraction; the adoption rule (Eq. (3), with the context's
 * K), the schedule and the random stream are those of the group game, and the threshold
 * table holds 2x5x5 entries indexed (s_x*5 + n_x)*5 + n_y. Every kernel family supports both
 * games; the batched and allocation-free entry points play the group game only. The
 * lattice and step counter are kept; autotuned choices are kept per game. */
int pgg_set_game(pgg_ctx *ctx, int game, const double payoff[4]);

/* The current game and (nullable) its payoff matrix (zeros for PGG_GAME_GROUP). */
int pgg_get_game(const pgg_ctx *ctx, int *game, double *payoff_out);

/* Initial condition of Section III: every site independently C with probability p
 * (p = 0.5: the even start of Section III), drawn from the Philox stream of `seed`; sets the step
 * counter to 0 and the seed used by later steps. 0 <= p <= 1. */
int pgg_seed(pgg_ctx *ctx, uint64_t seed, double p);

/* Advance the lattice by n_mcs full Monte Carlo steps (16 * n_mcs sublattice steps).
 * coop_per_mcs (nullable) receives n_mcs uint64 cooperator counts (numerator of
 * Eq. (4)), the count after each MCS; it may be device memory (written
 * asynchronously) or host memory (the call then synchronises the stream before
 * returning, and also reports a failed bounded wait or index check of this call's
 * kernels). n_mcs >= 0; n_mcs == 0 is a no-op. The first call on the resident kernel
 * allocates its exchange mailbox and count slots and, for the group game where the kernel
 * keeps one, a column-class copy of the lattice (L*L/8 bytes) that later resident calls
 * reuse while nothing else has written the lattice. */
int pgg_step_mcs(pgg_ctx *ctx, int64_t n_mcs, uint64_t *coop_per_mcs);

/* Number of cooperators now (numerator of Eq. (4)) into *out (host). Synchronises the
 * context's stream; reports a device-side failure flagged by earlier kernels. */
int pgg_count_coop(pgg_ctx *ctx, uint64_t *out);

/* Copy the lattice to host_out (L*L bytes, row-major, 1 = C) and the sublattice step
 * counter to *step_out (nullable; 16 per MCS). Synchronises the stream. */
int pgg_get_lattice(pgg_ctx *ctx, uint8_t *host_out, uint64_t *step_out);

/* Replace the lattice with host_in (L*L bytes, any non-zero byte = C) and set the step
 * counter (for tests and exact checkpoint/resume: (lattice, seed, step, r, K) is the
 * whole state). The seed is kept. Synchronises the stream. */
int pgg_set_lattice(pgg_ctx *ctx, const uint8_t *host_in, uint64_t step);

/* The same two transfers with the lattice bit-packed on the host: L rows of L/32 uint32 words,
 * bit b of word w of a row = column 32w + b (1 = C), the device layout of PGG_BITPACK, so a
 * checkpoint or an upload moves L*L/8 bytes instead of L*L. Need L % 32 == 0 (either layout;
 * a PGG_U8 context converts on the device through its staging buffer). Synchronise the
 * stream. */
int pgg_get_lattice_packed(pgg_ctx *ctx, uint32_t *host_words_out, uint64_t *step_out);
int pgg_set_lattice_packed(pgg_ctx *ctx, const uint32_t *host_words_in, uint64_t step);

/* Overlapped upload: queue the copy of host_words_in (bit-packed as above, L*L/8 bytes) on a
 * copy stream of the context's own and return without waiting, so that the copy runs while
 * work already queued on the context stream computes. The staged lattice and `step` replace the
 * context's lattice and step counter at the next call that reads or writes them (pgg_step_mcs,
 * pgg_count_coop, the get/set calls, pgg_seed, pgg_autotune, pgg_lattice_device_ptr), in stream
 * order: that call's work waits for the copy. pgg_get_state reports the staged step at once.
 * Two device buffers alternate, so a loop of stage / step calls overlaps the upload of the next
 * input with the current step. host_words_in should be pinned memory (from pageable memory the
 * copy cannot overlap) and must stay valid and unchanged until the copy has completed: at the
 * latest when a synchronising call after the applying call has returned, or when an event recorded
 * on the context stream after the applying call has completed. Need L % 32 == 0 and step < 2^56;
 * PGG_ERR_STATE if a staged lattice has not been applied yet. */
int pgg_stage_lattice_packed(pgg_ctx *ctx, const uint32_t *host_words_in, uint64_t step);

/* Current seed and step counter. */
int pgg_get_state(const pgg_ctx *ctx, uint64_t *seed_out, uint64_t *step_out);

/* Choose the kernel family, the number of sublattice steps fused per launch k
 * (1, 2, 4, 8 or 16; PGG_KERNEL_TILED only) and the tile size in sites (tile_x a
 * multiple of 64, tile_y a multiple of 4; 0 = default); for PGG_KERNEL_DIRECT tile_x is
 * the number of words per thread (4 or 8) and tile_y the block size (64, 128, 256), 0 =
 * default; for PGG_KERNEL_RESIDENT tile_y is the number of sublattice steps between halo
 * exchanges (1, 2 or 4; 0 = the largest whose halo rows fit) and tile_x is ignored (the
 * resolved schedule reports the number of bands there). PGG_KERNEL_AUTO restores the tuned
 * default. */
int pgg_set_schedule(pgg_ctx *ctx, int kernel, int steps_per_launch, int tile_x, int tile_y);

/* Autotuner: time every applicable schedule (direct words-per-thread x block size, tiled
 * k x tile shape, simple) for n_mcs MCS (1..1000) on a saved copy of this context's lattice,
 * restore the lattice, step counter and the caller's schedule, and remember the fastest
 * schedule for (device, L, layout) in a process-wide table that PGG_KERNEL_AUTO consults
 * from then on (for every context with that device, L and layout). The winner and its time
 * per MCS are returned through the (nullable) pointers. Synchronises the stream; allocates
 * one lattice-sized temporary. Results do not depend on the schedule. */
int pgg_autotune(pgg_ctx *ctx, int n_mcs, int *kernel, int *steps_per_launch, int *tile_x,
                 int *tile_y, float *ms_per_mcs);

/* Polls a CTA of PGG_KERNEL_RESIDENT makes on a neighbour's step counter before it gives up
 * and flags a time-out (default 1 << 22, about a second). 0 makes every wait fail at once,
 * for testing the failure path. */
int pgg_set_spin_limit(pgg_ctx *ctx, unsigned int limit);

/* Kernel timing, for measurement: with enable != 0 the context records a CUDA event pair on its
 * stream around every launch of its step kernel (resident, direct, tiled or simple; not the
 * conversions, counts or copies around it) from then on, dropping earlier records; enable == 0
 * stops and releases the events. Both synchronise the stream. pgg_kernel_time synchronises the
 * stream and returns the summed duration of the recorded launches in milliseconds and their
 * number (either pointer may be NULL). */
int pgg_set_kernel_timing(pgg_ctx *ctx, int enable);
int pgg_kernel_time(pgg_ctx *ctx, double *ms_total, int64_t *launches);

/* The schedule pgg_step_mcs will use (after AUTO resolution). Any pointer may be NULL. */
int pgg_get_schedule(const pgg_ctx *ctx, int *kernel, int *steps_per_launch, int *tile_x,
                     int *tile_y);

/* Copy the 2*26*26 adoption thresholds to host_out, index (s_x*26 + S_x)*26 + S_y with
 * s_y = 1 - s_x (entries with s_x == s_y are never used). Under PGG_GAME_PAIRWISE the first
 * 2*5*5 entries hold the table indexed (s_x*5 + n_x)*5 + n_y and the rest are zero. */
int pgg_get_threshold_table(const pgg_ctx *ctx, uint32_t *host_out);

/* The same table built on the host for the given game and parameters, without a context or a
 * device (the library's own statement of Eq. (3) and the payoff rules, callable anywhere):
 * game PGG_GAME_GROUP needs r > 0 (payoff ignored, may be NULL), PGG_GAME_PAIRWISE needs the 4
 * finite payoffs {R, S, T, P} (r ignored); K > 0. host_out receives 2*26*26 uint32 laid out as
 * above. */
int pgg_threshold_table(int game, double r, double K, const double payoff[4], uint32_t *host_out);

/* Device pointer of the lattice (layout as created) and its size in bytes, for callers
 * that hand the lattice to their own kernels on the same stream. The context may move its
 * lattice between two buffers (fused tiled schedules alternate them; an applied staged upload
 * of a bit-packed context takes over the staging buffer), so query the pointer again after any
 * call that steps or replaces the lattice. The caller may write the lattice through the pointer
 * until the context's next call: after this call the context treats the lattice as replaced
 * (the column-class copy a resident step keeps of it is rebuilt at the next such step). */
int pgg_lattice_device_ptr(pgg_ctx *ctx, void **dev_ptr, uint64_t *bytes);

/* Allocation-free variant of pgg_step_mcs, for callers that cannot allocate device memory:
 * plug-ins of a host application that hands out all device memory from its own pool (there a
 * cudaMalloc fails once the pool holds the device, or escapes the application's accounting),
 * and services that must not allocate after start-up (cudaMalloc may block on the whole device
 * for an unbounded time). The paper has no counterpart; it is a packaging of the fused tiled
 * kernel.
 *   lattice_in, lattice_out: device buffers in `layout` (PGG_U8: L*L bytes; PGG_BITPACK:
 *     L*L/8 bytes, see pgg_layout); they may be the same buffer.
 *   Runs n_mcs MCS of the model with (r, K, seed) starting at sublattice step step0
 *   (the state (lattice, seed, step, r, K) is the same as that of a context); the result is
 *   the one pgg_step_mcs gives, bit for bit.
 *   coop_per_mcs: NULL or a device buffer of n_mcs uint64 counts; it is cleared and filled.
 *   Requires L % 64 == 0, 64 <= L, and a lattice of at most 4 MiB (L <= 2048 for PGG_U8,
 *   L <= 4096 for PGG_BITPACK), and step0 + 16 n_mcs < 2^56; otherwise PGG_ERR_ARG with a
 *   message.
 * It calls no cudaMalloc, cudaFree or allocating routine: its scratch (a 4 MiB intermediate
 * lattice plus the threshold table, which reaches the device as a kernel parameter) is one
 * fixed device array in the library, held by every GPU that loads the library until the
 * process exits. The first call on a device resolves that array's address
 * (cudaGetSymbolAddress) with the device current; make that first call before any stream
 * capture. All calls share the array and each
 * overwrites what the last one left there: calls that overlap on the GPU (on different streams)
 * race and must be serialised by the caller. Asynchronous on cuda_stream. Not callable from a
 * host function enqueued on a stream (cudaLaunchHostFunc), where CUDA calls are not allowed. */
int pgg_step_mcs_noalloc(const void *lattice_in, void *lattice_out, int L, int layout, double r,
                         double K, uint64_t seed, uint64_t step0, int64_t n_mcs,
                         uint64_t *coop_per_mcs, void *cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Batched replicas: many independent lattices (each with its own L, r, K and seed) advanced
 * by one persistent kernel launch. The paper simulates many lattice sizes and lengths near
 * r_c (Section V); this runs such sets together. Every replica is bit-packed and kept in one
 * SM's shared memory for the whole call, so L must be 64, 128, 256, 512 or 1024. A replica's
 * trajectory is identical, bit for bit, to a pgg_ctx with the same (L, r, K, seed).
 * --------------------------------------------------------------------------------------- */
typedef struct pgg_batch pgg_batch;

/* Create n replicas (arrays of length n, copied). Allocates their lattices and threshold
 * tables on the current device; lattices start all-defector at step 0. */
int pgg_batch_create(pgg_batch **out, int n, const int *L, const double *r, const double *K,
                     const uint64_t *seeds, void *cuda_stream);

/* Every replica: Bernoulli(p) initial state from its own seed (as pgg_seed); steps := 0. */
int pgg_batch_seed(pgg_batch *b, double p);

/* Advance every replica by n_mcs MCS in one launch. counts (nullable) receives n * n_mcs
 * uint32 cooperator counts, replica-major ([i * n_mcs + m] = count of replica i after MCS m),
 * in device memory (asynchronous) or host memory (the call synchronises). */
int pgg_batch_step_mcs(pgg_batch *b, int n_mcs, uint32_t *counts);

/* Warps that advance one replica, per size class L = 64, 128, 256, 512, 1024 (5 entries,
 * each 1, 2, 4, 8, 16 or 32, at most the CTA's warps). Default {1, 1, 2, 4, 16}. Results do not
 * depend on it. */
int pgg_batch_set_team_warps(pgg_batch *b, const int *warps);
int pgg_batch_get_team_warps(const pgg_batch *b, int *warps);

/* Threads per persistent CTA: 512 (default) or 1024 (more warps, fewer registers each).
 * Setting 512 caps the team sizes at 16 warps. */
int pgg_batch_set_cta_threads(pgg_batch *b, int threads);
int pgg_batch_get_cta_threads(const pgg_batch *b, int *threads);

/* Autotuner: time candidate (CTA size, team sizes) for n_mcs MCS on a saved copy of the
 * replicas, restore them, keep the fastest; warps_out (nullable, 5 entries) and ms_out
 * (nullable) receive the choice and its time for the n_mcs MCS. Synchronises the stream. */
int pgg_batch_autotune(pgg_batch *b, int n_mcs, int *warps_out, float *ms_out);

/* pgg_batch_step_mcs captures its persistent launch in a CUDA graph (once per n_mcs) and
 * replays it (enable = 1, default), or launches directly (enable = 0). */
int pgg_batch_use_graph(pgg_batch *b, int enable);

/* Replica i's lattice (L*L bytes, 1 = C) and step counter, or replace them. Synchronise. */
int pgg_batch_get_lattice(pgg_batch *b, int i, uint8_t *host_out, uint64_t *step_out);
int pgg_batch_set_lattice(pgg_batch *b, int i, const uint8_t *host_in, uint64_t step);

/* Number of replicas. */
int pgg_batch_size(const pgg_batch *b, int *n);

/* Release the batch (NULL accepted). Synchronises the stream. */
void pgg_batch_destroy(pgg_batch *b);

/* ---------------------------------------------------------------------------------------
 * Surrogate network for the r_c search. The paper locates r_c from long runs (Section V,
 * Fig. 4); this small network reads the first 200 samples of rho_C(t) of a run plus its
 * normalised (r, K) and predicts P(absorbing) and the stationary rho_C, so that a bisection
 * can stop replicas early. 202 -> 128 (relu) -> 128 (relu) -> 2 (sigmoid heads); BF16
 * parameters rounded to nearest even from an FP32 master copy, FP32 accumulation; Adam
 * (beta 0.9 / 0.999, eps 1e-8, bias corrected). Parameters are packed W1 (128x202 row-major),
 * b1, W2 (128x128), b2, W3 (2x128), b3. X (B x 202), Y (B x 3: absorbed 0/1, stationary
 * rho, mask of the rho term) and outputs are row-major FP32 device buffers.
 * Loss = mean BCE(p, absorbed) + mean(mask * (rho - y_rho)^2).
 * --------------------------------------------------------------------------------------- */
typedef struct pgg_mlp pgg_mlp;

/* Layer sizes and parameter count (any pointer may be NULL). */
int pgg_mlp_info(int *n_in, int *n_hidden, int *n_out, int *n_params);

/* Network for batches of up to max_batch rows; parameters start at zero. */
int pgg_mlp_create(pgg_mlp **out, int max_batch, void *cuda_stream);

/* Load the FP32 master parameters from host memory (n_params floats); resets Adam. */
int pgg_mlp_set_params(pgg_mlp *n, const float *host_master);

/* Copy the FP32 master parameters and/or their BF16 image (raw uint16) to host memory. */
int pgg_mlp_get_params(pgg_mlp *n, float *host_master, uint16_t *host_bf16);

/* out[b] = (P(absorbing), stationary rho) for the B rows of X. Asynchronous. */
int pgg_mlp_forward(pgg_mlp *n, const float *X, int B, float *out);

/* Loss (1 float, nullable) and gradient (n_params floats, nullable) into device memory. */
int pgg_mlp_loss_grad(pgg_mlp *n, const float *X, const float *Y, int B, float *loss_out,
                      float *grad_out);

/* One Adam step with learning rate lr on the batch; loss of the batch before the step into
 * loss_out (device, nullable). Asynchronous. */
int pgg_mlp_train_step(pgg_mlp *n, const float *X, const float *Y, int B, float lr,
                       float *loss_out);

/* Release the network (NULL accepted). */
void pgg_mlp_destroy(pgg_mlp *n);

/* Release the context and its device memory. NULL is accepted. Synchronises the stream. */
void pgg_destroy(pgg_ctx *ctx);

/* Message describing the last failure on the calling thread ("" if none). */
const char *pgg_last_error(void);

/* Library version string. */
const char *pgg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PGG_H */
