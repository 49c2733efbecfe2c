/*
 * picasso.h -- C ABI of libpicasso, a B300 (sm_103a) implementation of the
 * round hot path of Picasso (Ferdous et al., arXiv 2401.06713): palette-based
 * list coloring of the commutation graph of n Pauli strings.
 *
 * One round (Alg. 1 of the paper) over the still-uncolored vertex set V_l:
 *   assign lists   every v in V_l draws L_l distinct colors of the round's
 *                  palette [base_l, base_l + P_l)   (Alg. 1, list assignment)
 *   build          the conflict graph G_c: u != v are adjacent iff they commute
 *                  (an edge of the complement graph G', Sec. II) and their
 *                  lists intersect (Sec. III-A)
 *   color          static Random order with first fit (Sec. III-B): in
 *                  ascending (priority, global id) order, v takes the smallest
 *                  color of its list not taken by a conflict neighbour that
 *                  comes earlier; if none is left v stays uncolored
 *   carry          the uncolored vertices form V_{l+1} (Alg. 1, end of an
 *                  iteration); the next round uses a fresh palette.
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers on the device that was current
 *     when picasso_init ran; h_* are host pointers.  The caller owns every
 *     buffer it passes in; the context owns (and frees in picasso_destroy)
 *     every buffer it hands out.
 *   - Strings are packed as symplectic words: a string of q <= 1024 qubits
 *     is 2W uint64 words [x_0 .. x_{W-1}, z_0 .. z_{W-1}], W = ceil(q / 64)
 *     (for q <= 64 the two words [x, z]); qubit i sets bit i % 64 of x_{i/64}
 *     for X and Y, of z_{i/64} for Z and Y.  Two strings commute iff the
 *     popcount of the XOR over w of (x_u,w & z_v,w) ^ (z_u,w & x_v,w) is
 *     even.  Every d_xz below is [n][2W] in this layout.
 *   - Character codes are 0=I 1=X 2=Y 3=Z.
 *   - Random numbers are Philox4x32-10 (Salmon et al., SC'11).  Draw i of the
 *     stream (seed, round, gid, tag) is word i%4 of the block with counter
 *     (gid_lo, gid_hi, round, tag<<24 | i/4) and key (seed_lo, seed_hi); tag 1
 *     draws lists (Floyd's sampling, a draw x maps to [0, j] as x*(j+1)>>32),
 *     tag 2 draws the priority (draw 0).
 *   - Every call returns a picasso_status; no call aborts the process.  A
 *     CUDA error is reported as PICASSO_ERR_CUDA and leaves the context
 *     unusable except for picasso_destroy.
 *   - All work is ordered on the stream given to picasso_init.  Calls that
 *     return sizes (build, carry, round, run) synchronise that stream.
 *   - Contexts allocate from one library-owned memory pool per device.  Freed
 *     blocks stay reserved for the next round or context (no page mapping on
 *     the hot path) until picasso_trim_memory returns them.
 */
#ifndef PICASSO_H
#define PICASSO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PICASSO_OK = 0,
  PICASSO_ERR_INVALID_ARG = 1, /* null pointer, size out of range, bad order */
  PICASSO_ERR_OOM = 2,         /* device allocation failed                   */
  PICASSO_ERR_CUDA = 3,        /* a CUDA call or kernel failed               */
  PICASSO_ERR_BUDGET = 4,      /* conflict graph larger than byte_budget     */
  PICASSO_ERR_TIMEOUT = 5,     /* a bounded device wait gave up              */
  PICASSO_ERR_INTERNAL = 6,    /* an internal consistency check failed       */
  PICASSO_ERR_UNSUPPORTED = 7, /* valid request outside this build's limits  */
  PICASSO_ERR_STATE = 8        /* call out of order for the context's state  */
} picasso_status;

/* Conflict-graph construction strategy.  Both produce the same CSR.  AUTO
 * tests all pairs in rounds of at most 2,048 vertices and otherwise joins
 * through buckets, unless a bucket exceeds 2,048 members or the round has
 * 2^21 or more colors.                                                      */
typedef enum {
  PICASSO_CONFLICT_AUTO = 0,
  PICASSO_CONFLICT_ALLPAIRS = 1, /* every pair tested (the paper's GPU kernel) */
  PICASSO_CONFLICT_BUCKET = 2    /* pairs joined through per-color buckets   */
} picasso_conflict_algo;

/* Launch schedule of the kernels whose shape changes no result (colors,
 * CSRs, rounds and stats other than times are the same under every
 * schedule): the small-round engine's grid, the rounds it gives to one
 * thread-block cluster and to one block, and the blocks per SM of the bit
 * pass and of the mask coloring.  All zero = the library's defaults.  picasso_autotune picks
 * one for a workload by timing candidates on it.  The paper has no
 * counterpart (its kernels have one launch shape).                          */
typedef struct {
  int32_t engine_blocks_per_sm; /* grid launch of the small-round engine:
                                   1 or 2 blocks of 256 threads per SM
                                   (0: 2)                                    */
  int32_t cluster_max_n;        /* engine rounds of at most this many
                                   vertices run in one thread-block cluster
                                   (0: 2048; -1: never; else 1 .. 16384)     */
  int32_t cluster_blocks;       /* blocks of that cluster: 2, 4, 8 or 16 (0:
                                   the largest that fits); more than fit is
                                   clamped to the largest that fits         */
  int32_t bits_blocks_per_sm;   /* bit pass of the build: 1 .. 4 blocks of 256
                                   threads per SM (0: the occupancy limit;
                                   more than the limit is clamped)           */
  int32_t color_blocks_per_sm;  /* mask coloring: 1 .. 8 blocks of 256 per SM
                                   (0: the occupancy limit; clamped to it)   */
  int32_t engine_max_n;         /* picasso_run hands the rounds to the small-
                                   round engine from a round of at most this
                                   many vertices (0: 16384; else 1 .. 16384) */
  int32_t block_max_n;          /* engine rounds of at most this many
                                   vertices run in one block of 256 threads
                                   (0: 64; -1: never; else 1 .. 16384)       */
} picasso_schedule;

typedef struct {
  uint64_t seed;         /* Philox key                                        */
  int64_t palette_num;   /* P_l = max(1, ceil(n_l * num / den))  (Table I)    */
  int64_t palette_den;
  double alpha;          /* L_l = min(P_l, max(1, ceil(alpha * ln n_l)))     */
  int32_t conflict_algo; /* picasso_conflict_algo                             */
  int32_t max_rounds;    /* picasso_run gives up with ERR_INTERNAL beyond it  */
  int64_t byte_budget;   /* max bytes of one round's conflict CSR, 8 (n_l + 1)
                            + 4 nnz; 0 = no limit                            */
  int32_t color_algo;    /* picasso_color_algo                                */
  int32_t csr_form;      /* picasso_csr_form                                  */
  int32_t small_engine;  /* picasso_small_engine                              */
  int32_t budget_mode;   /* picasso_budget_mode                               */
  int32_t wait_polls;    /* bounded device waits (the ordered coloring waiting
                            on an earlier neighbour, per-round pass and small-
                            round engine): polls of one wait before the kernel
                            gives up, reports it and the round is recolored by
                            the sweep kernel (per-round path) or handed back to
                            the per-round path (engine); same colors either
                            way.  0 = 1,048,576; 1 <= wait_polls <= 2^30    */
  picasso_schedule sched; /* launch schedule (all zero: defaults)            */
} picasso_config;

/* What picasso_round / picasso_run do with a round whose conflict CSR would
 * exceed cfg.byte_budget (single-set contexts; the explicit steps always
 * return PICASSO_ERR_BUDGET):
 *   FAIL  return PICASSO_ERR_BUDGET before allocating the CSR (Alg. 3 sizes
 *         the CSR first, too);
 *   CHUNK color the round in chunks of its coloring order, each chunk's CSR
 *         rows (8 bytes per row + 8, 4 per run entry) within the budget:
 *         emit the chunk's rows, color them, free them, next chunk.  In the
 *         EARLIER form a row lists only earlier neighbours, so the colors are
 *         those of the unchunked round.  ERR_BUDGET only if one vertex's rows
 *         alone exceed the budget.
 *   HOST  Alg. 3's fallback: the round's columns go to pinned host memory
 *         (mapped, so the emit pass writes them and the coloring reads them
 *         in place; row and run offsets stay on the device).  The host
 *         buffer grows to the largest such round; picasso_destroy keeps it
 *         for later contexts (picasso_trim_memory frees it).  Colors are
 *         those of the device round; picasso_build_conflicts then hands out
 *         d_col as a mapped host pointer (valid on the device, UVA).       */
typedef enum {
  PICASSO_BUDGET_FAIL = 0,
  PICASSO_BUDGET_CHUNK = 1,
  PICASSO_BUDGET_HOST = 2
} picasso_budget_mode;

/* Which half of G_c the conflict CSR stores.  The coloring step only reads a
 * vertex's earlier neighbours, so EARLIER (the default) keeps each pair once,
 * at its later endpoint, and halves the CSR; FULL keeps both directions.   */
typedef enum {
  PICASSO_CSR_EARLIER = 0, /* row u: neighbours ranked before u              */
  PICASSO_CSR_FULL = 1     /* row u: all neighbours                          */
} picasso_csr_form;

/* picasso_run on a single set hands the remaining rounds to one cooperative
 * launch (the small-round engine) once a round has at most 16384 vertices,
 * at most 4096 palette colors and lists of at most 64 colors, for strings
 * of at most 128 qubits, under the defaults AUTO / EARLIER / AUTO coloring.  The engine runs the same rounds
 * as picasso_round (same lists, CSR and colors) without a host round trip
 * per round; a round it cannot finish (CSR over its buffer or the byte
 * budget, a bounded wait that ran out) goes back to the per-round path.   */
typedef enum {
  PICASSO_SMALL_AUTO = 0,
  PICASSO_SMALL_OFF = 1
} picasso_small_engine;

/* Coloring strategy (AUTO and SWEEP give the same colors). */
typedef enum {
  PICASSO_COLOR_AUTO = 0,  /* ordered persistent pass; sweeps if it gives up */
  PICASSO_COLOR_SWEEP = 1, /* dependency sweeps only                         */
  PICASSO_COLOR_DYNAMIC = 2 /* Alg. 2's dynamic order (most constrained
                               first), parallel rule: each step colors every
                               uncolored vertex whose (remaining list size,
                               priority) is below all its uncolored
                               neighbours', with a color drawn from its
                               remaining list, and strikes those colors from
                               the neighbours' lists.  Not the static order's
                               colors; lists of at most 64; the build keeps
                               both directions of every pair (FULL).      */
} picasso_color_algo;

/* Conflict CSR of the current round, owned by the context and valid until
 * the next assign/build/carry or destroy.  Ids are round-local: vertex r is
 * the r-th of the round's coloring order, ascending (priority, global id)
 * (picasso_get_round maps them to global ids).  Rows are color-major: row u
 * lists, for each color c of u's list in ascending order (its "run"), the
 * neighbours v that also hold c, ascending in v -- with cfg.csr_form EARLIER
 * only those with v < u, with FULL all of them.  An edge of G_c whose two
 * lists share m colors appears in m runs of its row(s), so nnz = sum over
 * edges of m (EARLIER) or twice that (FULL); that is |E_c| (2|E_c|) when no
 * pair shares two colors.  The run of c is what the coloring step reads to
 * test color c.                                                             */
typedef struct {
  const int64_t* d_off; /* [n_rows + 1]                                      */
  const int32_t* d_col; /* [nnz]                                             */
  int64_t n_rows;
  int64_t nnz;
} picasso_csr;

/* Per-round record kept by the context (the last round's values). */
typedef struct {
  int32_t round;       /* current round number (1-based)                     */
  int64_t n_total;     /* N                                                  */
  int64_t n_round;     /* n_l, vertices of the current round                 */
  int64_t P;           /* P_l of the last assign (batch: sum over the sets)  */
  int32_t L;           /* L_l of the last assign (batch: the largest)        */
  int64_t base;        /* base_l of the last assign (batch: of set 0)        */
  int64_t nnz;         /* run entries of the last build (see picasso_csr)    */
  int64_t colored;     /* vertices colored by the last color step            */
  int64_t colors_used; /* base after the last carry = sum of P of done rounds */
  int64_t peak_bytes;  /* high-water mark of context-owned device memory      */
  int32_t conflict_algo_used;
  int32_t jp_sweeps;   /* sweeps of the last color step (0: ordered pass)    */
  int32_t ordered_fallbacks; /* rounds whose ordered pass gave up (sweeps ran) */
  int64_t max_bucket;  /* largest color bucket of the last build (0: all pairs) */
  /* cumulative since picasso_init (CUDA events on the context's stream) */
  int32_t rounds_done;
  double t_assign_ms;   /* list assignment                                   */
  double t_build_ms;    /* conflict build (buckets, count, scans, fill)      */
  double t_color_ms;    /* coloring sweeps + color write-back                */
  double t_carry_ms;    /* compaction of the uncolored vertices              */
  double t_pairs_ms;    /* the pair-test kernels alone (bucket join: mask
                           pass, or the bit pass; all pairs: count and
                           fill)                                            */
  int64_t pairs_launches;     /* launches of the pair-test kernels           */
  int64_t logical_pairs;      /* sum over builds of n_l (n_l - 1) / 2        */
  int64_t tested_pairs;       /* pair tests of the pair-test kernels: per
                                 build, bucket join sum_c s_c (s_c - 1) / 2
                                 (the mask pass tests each unordered pair of
                                 a bucket once), all pairs 2 n (n - 1)      */
  double t_emit_ms;           /* bucket join's emit pass (CSR writes); with the
                                 bit pass, that same kernel's time          */
  int64_t emit_launches;
  int64_t emit_bytes;         /* bytes the emit passes move: mask words read,
                                 CSR written, member ids and run offsets
                                 read; bit pass: 28 per list entry (member
                                 words and entry ids read, one word of row
                                 address, slot and run length written) and 4
                                 per word of bit rows written               */
  int64_t nnz_total;          /* run entries of all builds                  */
  /* the last color step's first 64 sweeps: vertices pending at the start,
   * vertices re-evaluated, and duration in microseconds (0 for the last) */
  int32_t sweep_pending[64];
  int32_t sweep_active[64];
  float sweep_us[64];
  int32_t small_rounds;       /* rounds the small-round engine ran          */
  int32_t small_stops;        /* engine launches that handed a round back   */
  double t_small_ms;          /* time in the small-round engine             */
  int32_t round_chunks;       /* chunks of the rounds colored by chunk      */
  int32_t host_csr_rounds;    /* rounds whose columns went to host memory   */
  int32_t barrier_timeout[4]; /* a grid barrier that gave up (4 s; the call
                                 returned PICASSO_ERR_TIMEOUT): kernel (1
                                 small-round engine, 2 sweep coloring, 3
                                 dynamic order; 0 none), its site, round or
                                 step, and the blocks that had arrived      */
} picasso_stats;

/* Fill *cfg with the defaults: seed 0, P = n/8, alpha = 2 (the paper's normal
 * mode, Sec. VI), AUTO, max_rounds 100000, no budget.                       */
int picasso_config_default(picasso_config* cfg);

/* Pack n strings of q character codes (row-major uint8 [n][q]) into
 * symplectic words d_xz [n][2W], W = ceil(q / 64) (1 <= q <= 1024; more is
 * PICASSO_ERR_UNSUPPORTED).  Sec. III-A encodes characters in bits; this is
 * the product's word form of that idea.  Asynchronous.                     */
int picasso_pack(const uint8_t* d_codes, int64_t n, int32_t q, uint64_t* d_xz,
                 void* stream);

/* Create a context over d_xz [n][2W] (read-only, must outlive the context;
 * 1 <= n < 2^30, 1 <= q <= 1024, W = ceil(q / 64)).  stream is a
 * cudaStream_t (NULL = legacy default stream).  Round 1 starts with V_1 =
 * all n strings, all colors -1.  Strings of q > 64 (Sec. VII's larger
 * systems) take the same rounds; their conflict pass forms each pair's
 * symplectic product over all words (no bit layout); the small-round
 * engine takes strings of up to 128 qubits.                                */
int picasso_init(void** ctx, const picasso_config* cfg, const uint64_t* d_xz,
                 int64_t n, int32_t q, void* stream);

/* A batch of independent string sets in one context (one launch per step
 * for the whole batch).  d_xz [N][2W] holds the sets back to back; set k is
 * the global ids h_set_offsets[k] .. h_set_offsets[k+1] (host array of
 * nsets + 1 entries, h_set_offsets[0] = 0, N = h_set_offsets[nsets] < 2^30).
 * Set k is colored exactly as picasso_init on its own strings with seed
 * h_seeds[k] (host, NULL: cfg.seed + k) would color it; its colors start at
 * 0 and are written at its global ids by picasso_run / picasso_get_colors.
 * All sets run their rounds together; a set that is done has no vertices.
 * picasso_round_params and picasso_assign_lists need a single-set context. */
int picasso_init_batch(void** ctx, const picasso_config* cfg,
                       const uint64_t* d_xz, const int64_t* h_set_offsets,
                       int32_t nsets, const uint64_t* h_seeds, int32_t q,
                       void* stream);

/* Parameters the configuration gives the current round: P_l, L_l, base_l
 * (Table I rule; base_l = sum of the earlier rounds' P).                    */
int picasso_round_params(void* ctx, int64_t* P, int32_t* L, int64_t* base);

/* Alg. 1 list assignment for V_l with explicit P, L (1 <= L <= min(P, 512))
 * and base.  Also draws the round's priorities.  Asynchronous.             */
int picasso_assign_lists(void* ctx, int64_t P, int32_t L, int64_t base);

/* Alg. 1 conflict-graph construction (Sec. III-A, Alg. 3's count / offsets /
 * fill structure).  Synchronises to size the CSR; returns ERR_BUDGET, before
 * allocating, if the CSR would exceed cfg.byte_budget.
 * With the EARLIER form, no byte budget, strings of at most 64 qubits and
 * color buckets of at most 512 members, one pass tests the pairs of every
 * color bucket and stores G_c as the bucket's lower blocks of pair bits (the
 * library's bit layout: bit t of row i's word W says whether member i
 * commutes with member 32 W + t < i; read by picasso_color).  The canonical
 * row-major CSR described by picasso_csr is made from it when asked for: by
 * a non-NULL out here, or by picasso_get_runs / picasso_copy_csr /
 * picasso_copy_runs (which then allocate it and synchronise).  out may be
 * NULL.                                                                     */
int picasso_build_conflicts(void* ctx, picasso_csr* out);

/* Alg. 1 coloring of the unconflicted vertices and of G_c (Sec. III-B static
 * Random order, first fit), run as a dependency-driven parallel sweep that
 * reproduces the sequential order exactly.  Synchronises.  Writes the
 * round's colors into the context's color array.                           */
int picasso_color(void* ctx, int64_t* n_colored);

/* Alg. 1 carry: V_{l+1} = uncolored vertices of V_l, next palette base, next
 * round.  Synchronises; *n_remaining = |V_{l+1}|.                           */
int picasso_carry(void* ctx, int64_t* n_remaining);

/* One whole round: params, assign, build, color, carry.                    */
int picasso_round(void* ctx, int64_t* n_remaining);

/* Rounds until every vertex is colored; then copies the global colors to
 * d_color_out [n] (may be NULL) and sets *n_rounds (may be NULL).          */
int picasso_run(void* ctx, int32_t* d_color_out, int32_t* n_rounds);

/* Alg. 1 end to end from host buffers (the problem statement of Alg. 1: the
 * strings in, a coloring out): copies n strings of q character codes
 * (h_codes, row-major uint8 [n][q], 0 = I, 1 = X, 2 = Y, 3 = Z) to the
 * device, packs them, runs every round as picasso_init + picasso_run would
 * (cfg as there; n >= 1, 1 <= q <= 1024) and copies the global colors to
 * h_colors [n] (int32); *n_rounds (may be NULL) gets the rounds run.  The
 * device memory comes from the library's pool and is returned before the
 * call ends.  Host buffers should be pinned (cudaHostAlloc) for full copy
 * speed; pageable ones work.  Synchronises stream.                         */
int picasso_color_host(const picasso_config* cfg, const uint8_t* h_codes, int64_t n, int32_t q,
                       int32_t* h_colors, int32_t* n_rounds, void* stream);

/* Autotuner of the launch schedule (picasso_schedule) for a workload of one
 * or many sets, given as picasso_init_batch takes them (nsets = 1 with
 * h_set_offsets = {0, n}: one set).  Starting from cfg->sched it tunes one
 * field at a time, in the order engine_max_n, engine_blocks_per_sm,
 * cluster_max_n, cluster_blocks, block_max_n, bits_blocks_per_sm,
 * color_blocks_per_sm, over that field's candidates (16384, 8192, 4096; 1,
 * 2; -1, 512, 2048, 8192; 16, 8; -1, 64, 256, 1024; 4, 3, 2; 6, 4, 3),
 * keeping the others at their best so far.  Each candidate is one whole
 * picasso_run of the workload after one untimed run, timed with CUDA events
 * on `stream`, the median of `reps` (1 .. 64) runs.  The fastest schedule
 * goes to *best, its time to *best_ms and the time of cfg->sched itself to
 * *start_ms (either may be NULL).  The colors of every run are compared
 * with the first run's; a difference is PICASSO_ERR_INTERNAL.  d_xz,
 * h_set_offsets, h_seeds, q: as picasso_init_batch.  Synchronises; the
 * device memory it takes comes from the library's pool.  Not in the paper:
 * it picks launch shapes of this library's kernels.                        */
int picasso_autotune(const picasso_config* cfg, const uint64_t* d_xz, const int64_t* h_set_offsets,
                     int32_t nsets, const uint64_t* h_seeds, int32_t q, int32_t reps,
                     picasso_schedule* best, double* best_ms, double* start_ms, void* stream);

/* Copy the global color array [n] (-1 = not yet colored) to d_out.         */
int picasso_get_colors(void* ctx, int32_t* d_out);

/* Inspection of the current round, for tests and tools, indexed by the
 * round-local id once lists are assigned (coloring order):
 *   d_gid   [n_l]    global ids (before assignment: V_l in ascending order)
 *   d_lists [E]      bucket colors (round-local color + the set's offset),
 *                    ascending per vertex
 *   d_prio  [n_l]    priorities (smaller = earlier)
 * Any pointer may be NULL.                                                  */
int picasso_get_round(void* ctx, int32_t* d_gid, int32_t* d_lists,
                      uint32_t* d_prio);

/* Run structure of the last build: d_runoff [E + 1] int64 (E = the round's
 * list entries; with one list length L, entry u*L+k) where the run of row
 * u's k-th color is col[runoff[e] .. runoff[e+1]) of the canonical CSR.
 * Owned by the context.                                                    */
int picasso_get_runs(void* ctx, const int64_t** d_runoff);

/* Copy the last build's CSR into caller-owned device buffers: d_off
 * [n_rows + 1] int64, d_col [nnz] int32 (either may be NULL).  Asynchronous. */
int picasso_copy_csr(void* ctx, int64_t* d_off, int32_t* d_col);

/* Copy the last build's run offsets (layout as in picasso_get_runs) into a
 * caller-owned buffer.  Asynchronous.                                      */
int picasso_copy_runs(void* ctx, int64_t* d_runoff);

int picasso_get_stats(void* ctx, picasso_stats* out);

/* Per-set results of a (batched) context, each array nsets long, host
 * memory owned by the caller, any may be NULL:
 *   h_colors[k]     colors set k has used so far: the sum of its finished
 *                   rounds' palette sizes, the paper's count C = sum_l P_l
 *                   (Sec. III-C);
 *   h_peak_bytes[k] largest conflict CSR set k had in one round so far,
 *                   counted like cfg.byte_budget: 8 (n_k + 1) + 4 nnz_k
 *                   bytes (row offsets, run entries);
 *   h_remaining[k]  set k's uncolored vertices.                            */
int picasso_get_set_stats(void* ctx, int64_t* h_colors, int64_t* h_peak_bytes,
                          int64_t* h_remaining);

/* Checkpoint of a context between rounds (after picasso_carry or before the
 * first round): the round number, every string's color so far, the global
 * ids of the uncolored strings and the per-set counters.  Lists, priorities
 * and palettes are functions of (seed, round, global id), so a context that
 * loads this state and runs on colors exactly as the uninterrupted one.
 * picasso_save_state writes *bytes_out = the size; with h_buf == NULL that is
 * all it does, with capacity < size it returns INVALID_ARG.  The buffer is
 * host memory owned by the caller; the call synchronises the stream.
 * picasso_load_state wants a fresh or between-round context over the same
 * strings, sets, seeds and parameters (INVALID_ARG otherwise, with nothing
 * changed); both return ERR_STATE in the middle of a round.  The paper has
 * no counterpart.                                                          */
int picasso_save_state(void* ctx, void* h_buf, int64_t capacity,
                       int64_t* bytes_out);
int picasso_load_state(void* ctx, const void* h_buf, int64_t bytes);

/* ---- Parameter prediction (Sec. V) -------------------------------------
 * Sec. V predicts (P' = P/n, alpha) from instance features with a regressor
 * trained on grid-search labels.  Here the regressor is a 5-64-64-2 MLP with
 * GELU, bf16 weights and fp32 accumulation; these entries are its device
 * kernels and the feature extraction.  All pointers are device memory owned
 * by the caller; all calls are asynchronous on `stream`.
 *
 * Parameter vector (fp32 master weights and their bf16 copy share it):
 *   W1[64][5] | b1[64] | W2[64][64] | b2[64] | W3[2][64] | b3[2]
 * row-major, y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3 with the exact
 * (erf) GELU; picasso_mlp_param_count() elements.                          */

/* Instance features of n packed strings: d_counts[0] = non-identity positions
 * over all strings, d_counts[1] = commuting pairs among `samples` pairs of
 * distinct strings drawn by Philox (key seed, round 0, tag 3, counter = pair
 * index; first string floor(r0 n / 2^32), second floor(r1 (n-1) / 2^32),
 * plus one when not below the first).  d_feat[0..4] = log2(ln n) - 3
 * (-3 when n = 1), q / 64, d_counts[0] / (n q), d_counts[1] / samples (1 when
 * samples = 0), log2(budget_bytes / n) / 4 - 3.  n >= 1, budget_bytes > 0. */
int picasso_features(const uint64_t* d_xz, int64_t n, int32_t q,
                     uint64_t seed, int64_t samples, double budget_bytes,
                     int64_t* d_counts, float* d_feat, void* stream);

/* The same features for the weighted objective of Eq. ml, min over (P, alpha)
 * of beta C + (1 - beta) |E_c|: d_feat[4] = 4 beta - 2 in place of the
 * budget term (0 <= beta <= 1; the other four and d_counts as above).      */
int picasso_features_beta(const uint64_t* d_xz, int64_t n, int32_t q,
                          uint64_t seed, int64_t samples, double beta,
                          int64_t* d_counts, float* d_feat, void* stream);

int32_t picasso_mlp_param_count(void);

/* d_y[b][0..1] = MLP(d_w, d_x[b][0..4]) for b < batch (fp32 in and out). */
int picasso_mlp_forward(const uint16_t* d_w, const float* d_x, int32_t batch,
                        float* d_y, void* stream);

/* Gradient of loss = (1/batch) sum_b sum_o weight_o (y_bo - d_t[b][o])^2 / 2
 * with respect to the parameters, written to d_grad (fp32, overwritten);
 * d_loss (may be NULL) receives the loss.  batch >= 1.                      */
int picasso_mlp_backward(const uint16_t* d_w, const float* d_x,
                         const float* d_t, float weight0, float weight1,
                         int32_t batch, float* d_grad, float* d_loss,
                         void* stream);

/* One AdamW step (decoupled weight decay; Loshchilov & Hutter) on the fp32
 * master weights with moments d_m, d_v; step >= 1 is the 1-based step used
 * for bias correction; d_w receives the rounded-to-nearest-even bf16 copy. */
int picasso_mlp_adamw(float* d_master, uint16_t* d_w, const float* d_grad,
                      float* d_m, float* d_v, float lr, float beta1,
                      float beta2, float eps, float weight_decay,
                      int32_t step, void* stream);

/* d_dst[i] = bf16(d_src[i]), round to nearest even, i < count. */
int picasso_mlp_to_bf16(const float* d_src, uint16_t* d_dst, int32_t count,
                        void* stream);

/* Fill d_out[i] with draw i0+i of stream (seed, round, gid, tag), i < count.
 * Exposes the device generator for parity checks against a CPU Philox.      */
int picasso_philox_draws(uint64_t seed, int32_t round, int64_t gid,
                         uint32_t tag, uint32_t i0, int32_t count,
                         uint32_t* d_out, void* stream);

/* Return cached pool memory of the current device to the driver, keeping at
 * most keep_bytes reserved, and free the pinned host read-back buffers that
 * destroyed contexts left for reuse.  Synchronises the device.             */
int picasso_trim_memory(int64_t keep_bytes);

/* Process-wide count of kernels this library has launched (all contexts). */
int picasso_kernel_launches(int64_t* out);

/* Process-wide count of the memory requests this library has made: memory
 * pool creations, device allocations from its pool, and pinned or mapped
 * host allocations (all contexts).  The paper has no counterpart.          */
int picasso_memory_requests(int64_t* out);

/* Whole run of Alg. 1 (as picasso_init + picasso_run + picasso_get_colors,
 * same colors) for a small set, with no device allocation at all.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc while they work -- services that give the GPU's memory to their
 * own fixed pool, or hosts that forbid allocation on their hot path because it
 * synchronises the device.  Every temporary buffer lives in one library-owned
 * static device array of about 12.1 MB; once this function has run on a GPU,
 * that GPU holds the array until the process exits.
 *   d_xz        [n][2] packed strings (caller-owned, read-only)
 *   d_color_out [n] int32, receives the global colors (caller-owned); it is
 *               set to -1 first and each round writes its colors as it ends,
 *               so a call that fails in a later round (for example
 *               PICASSO_ERR_UNSUPPORTED from that round's size check, or
 *               PICASSO_ERR_BUDGET) leaves the earlier rounds' colors there
 *               and -1 for the rest
 *   n_rounds    may be NULL
 * Fields of cfg it reads: seed, palette_num, palette_den, alpha, max_rounds,
 * color_algo (AUTO and SWEEP give the same colors; DYNAMIC returns
 * PICASSO_ERR_UNSUPPORTED), byte_budget with budget_mode FAIL (a round whose
 * CSR in cfg.csr_form would exceed it returns PICASSO_ERR_BUDGET; another
 * budget_mode with a nonzero budget returns PICASSO_ERR_UNSUPPORTED), and
 * wait_polls.  conflict_algo and small_engine do not change colors and are
 * not read: every round tests all pairs.
 * Limits: 1 <= n <= 2048, q <= 64, round-1 list size L <= 32, and at most
 * 2,621,440 run entries in any round, counted with both directions of every
 * pair (the array's conflict rows hold both, whatever cfg.csr_form says);
 * beyond them it returns PICASSO_ERR_UNSUPPORTED without touching the GPU
 * (the size checks of later rounds run after that round's count pass).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Calls
 * share the array: calls whose GPU work overlaps (other streams, other host
 * threads) race and must be serialised by the caller.  Synchronises stream. */
int picasso_run_small_static(const uint64_t* d_xz, int64_t n, int32_t q,
                             const picasso_config* cfg, int32_t* d_color_out,
                             int32_t* n_rounds, void* stream);

int picasso_destroy(void* ctx);

const char* picasso_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* PICASSO_H */
