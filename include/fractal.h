/*
 * fractal.h -- C ABI of the GB300 library for cellular automata on NBB
 * fractals kept in compact storage (Quezada & Navarro, "Accelerating Compact
 * Fractals with Tensor Core GPUs", 2021).
 *
 * Terms (all from the paper):
 *   NBB fractal F_n^{k,s} (Sec. 1): level m+1 is k translated, non-rotated,
 *     non-overlapping copies of level m on an s-times larger grid; level 0 is
 *     one cell.  At level r the bounding box has side n = s^r and the fractal
 *     has V = k^r cells (Eq. 1).
 *   transition table: offsets[j*dim + i] in [0,s) is the position, in units
 *     of s^m, of replica j along axis i; j is the replica ID of Sec. 3.1.
 *   compact index omega = sum_mu d_mu k^mu, where d_mu is the replica ID at
 *     level mu (mu = 0 is the finest level).  Compact state buffers hold one
 *     byte per cell in this order (k^r bytes).
 *   lambda(omega) (Sec. 1, Sec. 3): compact index -> embedded coordinate
 *     p = sum_mu s^mu offsets[d_mu].
 *   nu(p) (Sec. 3.1, Eqs. 2-8): embedded coordinate -> compact index, or -1
 *     ("outside") when p is off the fractal or outside the box.
 *   box: the n^dim bounding box, one byte per cell, x fastest, then y, z.
 *
 * Conventions for every call:
 *   - Return value: FR_OK (0) or a negative FR_E* code; a readable message
 *     for the calling thread is available from fractal_last_error().
 *   - Buffers passed as `dev` are device pointers that the caller allocates,
 *     owns and keeps alive until the call's work on `stream` has finished.
 *     Buffers passed as `host` are host pointers (pinned memory is fastest).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued asynchronously; errors raised by a
 *     kernel while it runs surface at the next call or at fractal_sync().
 *   - Input states: any nonzero byte is alive.  Output states are exactly
 *     0 or 1.
 *   - Rules are life-like: bit c of birth_mask (survive_mask) gives the new
 *     state of a dead (live) cell with c live Moore neighbours (8 in 2D, 26
 *     in 3D).  Neighbours outside the box or off the fractal are dead; there
 *     is no wrap-around.  B3/S23 is birth 0x8, survive 0xC.
 *   - Handles are not thread-safe: one host thread per handle at a time.
 *     Different handles may be used concurrently.
 */
#ifndef FRACTAL_H
#define FRACTAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FR_OK = 0,
    FR_EINVAL = -1,     /* bad argument (null pointer, aliasing, bad table) */
    FR_EOVERFLOW = -2,  /* k^r, s^r or n^dim beyond the supported range    */
    FR_ENOMEM = -3,     /* device or host allocation failed                */
    FR_ECUDA = -4,      /* a CUDA runtime call failed                      */
    FR_ETIMEOUT = -5,   /* a bounded device-side wait gave up              */
    FR_EBUSY = -6,      /* resource (server slot, memory budget) exhausted */
    FR_ENOTFOUND = -7   /* unknown request or instance id                  */
};

typedef struct fractal fractal_t;

/* Message describing the last error raised on the calling thread ("" if
 * none).  The pointer stays valid until the thread's next library call. */
const char *fractal_last_error(void);

/* Library version string. */
const char *fractal_version(void);

/* Build a fractal handle (Sec. 1 definition, Eq. 1 volume).
 *   k        number of replicas per level, 1 <= k <= s^dim
 *   s        growth ratio per level, 2 <= s <= 16, and s^dim <= 256
 *   r        scale level, r >= 0; requires s^r < 2^31 and k^r < 2^62
 *   dim      2 or 3
 *   offsets  host array of k*dim int32 values in [0,s), rows pairwise
 *            distinct; row j is replica j.  Copied; not retained.
 *   out      receives the handle (owned by the caller, freed by
 *            fractal_destroy).
 * Errors: FR_EINVAL for a bad table, FR_EOVERFLOW for sizes out of range. */
int fractal_create(int k, int s, int r, int dim, const int32_t *offsets,
                   fractal_t **out);

/* A fractal combined from a different NBB transition table at each scale
 * level (the combination the paper's conclusions propose as future work).
 * Level mu (mu = 0 the finest, mu < r) has ks[mu] replicas, 1 <= ks[mu] <=
 * s^dim, whose offsets are the ks[mu] rows of dim int32 values in [0,s)
 * that follow the rows of levels 0 .. mu-1 in `offsets`; s and dim are
 * common.  It has prod ks[mu] cells; the compact index is the mixed-radix
 * number omega = sum_mu d_mu (ks[0] ... ks[mu-1]) of the replica IDs, and
 * the compact coordinate (fractal_nu2d) gives level mu's ID the weight
 * prod ks[nu] over the earlier levels nu of the same axis (nu = mu mod dim).
 * Supported by every call on handles except the tensor-core maps, the
 * paper's approaches, the sharded step and temporal blocking (FR_EINVAL);
 * the step uses the generic per-cell policy (2D) or the box policy (3D).
 * Errors as fractal_create; r in [1, 62]. */
int fractal_create_mixed(int s, int r, int dim, const int32_t *ks, const int32_t *offsets,
                         fractal_t **out);

/* Free a handle and the device memory it owns (tables, scratch).  Waits for
 * the handle's outstanding work.  NULL is accepted. */
int fractal_destroy(fractal_t *f);

/* cells = k^r (Eq. 1), side = n = s^r; either pointer may be NULL. */
int fractal_info(const fractal_t *f, int64_t *cells, int64_t *side);

/* lambda (Sec. 3): coords_dev[e*dim + i] = axis i of lambda(omega_dev[e]),
 * for e < count.  An omega outside [0, k^r) gets the coordinates -1. */
int fractal_lambda(const fractal_t *f, const int64_t *omega_dev, int64_t count,
                   int32_t *coords_dev, void *stream);

/* nu (Sec. 3.1, Eqs. 2-8 with the inverse transition table as H):
 * omega_dev[e] = compact index of the cell at coords_dev[e*dim ..], or -1
 * when that cell is outside the box or off the fractal. */
int fractal_nu(const fractal_t *f, const int32_t *coords_dev, int64_t count,
               int64_t *omega_dev, void *stream);

/* The paper's multi-dimensional compact coordinate (Eqs. 6-8): component
 * (mu mod dim) gains H_mu * k^floor(mu/dim) at each level mu.  In 2D this is
 * (nu_x, nu_y) on a k^ceil(r/2) x k^floor(r/2) rectangle.  Outside cells give
 * -1 in every component.  compact_dev has count*dim entries. */
int fractal_nu2d(const fractal_t *f, const int32_t *coords_dev, int64_t count,
                 int64_t *compact_dev, void *stream);

/* The same maps with their sums over levels on the tensor cores (Sec. 3.1,
 * the tensor-core encoding of nu, made exact): per warp, 32 cells' replica
 * IDs (nu) or digit offsets (lambda) form a matrix A, the level weights
 * (k^mu, tau(k, mu), s^mu) split into 11-bit limbs form B, and
 * mma.sync.m16n8k16 with fp16 operands and fp32 accumulators computes A B;
 * every partial sum stays below 2^24, so the results equal fractal_nu /
 * fractal_nu2d / fractal_lambda exactly.  fractal_nu_tc writes nu to
 * omega_dev and, if compact_dev is not NULL, the compact coordinate of
 * fractal_nu2d to compact_dev (count*dim entries).  Limits: r <= 32 and
 * k <= 255 (nu), dim*r <= 64 (lambda), else FR_EINVAL. */
int fractal_nu_tc(const fractal_t *f, const int32_t *coords_dev, int64_t count,
                  int64_t *omega_dev, int64_t *compact_dev, void *stream);
int fractal_lambda_tc(const fractal_t *f, const int64_t *omega_dev, int64_t count,
                      int32_t *coords_dev, void *stream);

/* Seeded Bernoulli(p) compact state (not from the paper; synthetic input):
 * state_dev[omega] = 1 iff the top 53 bits of the omega-th SplitMix64 output
 * for `seed` (mix(seed + (omega+1)*0x9e3779b97f4a7c15)) are below
 * floor(p * 2^53).  p is clamped to [0,1].  state_dev has k^r bytes. */
int fractal_init_bernoulli(const fractal_t *f, uint8_t *state_dev,
                           uint64_t seed, double p, void *stream);

/* The stencil step of Sec. 3, repeated `steps` times (synchronous
 * generations, Sec. 4 benchmark): every compact cell omega takes
 * lambda(omega), counts its live Moore neighbours through nu, and applies
 * the rule.  in_dev and out_dev are k^r-byte compact states that must not
 * overlap; in_dev is never written.  steps = 0 copies (normalised to 0/1).
 * For steps > 1 the library ping-pongs through its own scratch buffer of k^r
 * bytes, allocated on first need and kept until fractal_destroy.  When the
 * step's plan is the bit3 policy (3D fractals with s = 3 and k a multiple of
 * 4 at tile depth 3, fractal_plan_info policy 15), steps > 1 keep the state
 * bit-packed between the first and the last generation instead, in two
 * buffers of 3136 bytes per level-3 tile (k^(r-3) tiles), likewise allocated
 * on first need and kept until fractal_destroy; the result is the same. */
int fractal_step(fractal_t *f, const uint8_t *in_dev, uint8_t *out_dev,
                 int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                 void *stream);

/* fractal_step without any device allocation (the paper has no counterpart).
 * It serves callers that cannot allocate device memory while they run:
 * applications whose device memory is handed out up front by their own pool
 * or by another framework that reserves it, and real-time loops in which
 * cudaMalloc/cudaFree are not acceptable because they may synchronise the
 * whole device.  Same arguments and results as fractal_step, but:
 *   - the ping-pong buffer for steps > 1 is a fixed 32 MiB device array
 *     inside the library (held on every GPU that loads the library until the
 *     process exits), so k^r must be at most 33,554,432 cells; larger states
 *     are rejected with FR_EINVAL;
 *   - the handle's tables must already exist: they are built (and
 *     allocated) by the handle's first fractal_step, fractal_autotune or
 *     fractal_get_tile_levels call; otherwise FR_EINVAL;
 *   - the first call on each device (and the first after that device's
 *     context changed, e.g. after cudaDeviceReset) looks up the array's
 *     device address in the current context (cudaGetSymbolAddress) and
 *     caches it; make that first call before any stream capture;
 *   - the array is shared by every call in the process and keeps the last
 *     call's contents (no call needs it to start at zero: each generation
 *     overwrites it completely before it is read); calls whose work overlaps
 *     on the GPU (other streams, other host threads) race on it and must be
 *     serialised by the caller. */
int fractal_step_noalloc(fractal_t *f, const uint8_t *in_dev, uint8_t *out_dev,
                         int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                         void *stream);

/* The bounding-box approach (Sec. 4, "BB"): the same rule applied to every
 * cell of the n^dim box.  Cells off the fractal count as dead whatever their
 * byte and are written as 0.  box_in_dev / box_out_dev: n^dim bytes each,
 * not overlapping.  Scratch for steps > 1 as in fractal_step (n^dim bytes). */
int fractal_bb_step(fractal_t *f, const uint8_t *box_in_dev, uint8_t *box_out_dev,
                    int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                    void *stream);

/* ---- The paper's own two approaches, as baselines (Sec. 4) -------------
 * rho_levels = l in [1, r] with rho = s^l and rho^dim <= 1024.
 *
 * "lambda(omega)": the state stays in the n^dim box (as for fractal_bb_step),
 * but only the blocks of threads the fractal needs run: block b covers the
 * rho^dim box cells of coarse cell lambda(b) of the level r - l fractal, and
 * threads on members read their neighbours straight from the box.  box_in_dev
 * must hold 0 on every cell off the fractal (as fractal_scatter_to_box
 * writes); box_out_dev's cells off the fractal are not written (keep them 0).
 * steps >= 1; for steps > 1 the library ping-pongs through a zeroed box. */
int fractal_lambda_box_step(fractal_t *f, int rho_levels, const uint8_t *box_in_dev,
                            uint8_t *box_out_dev, int64_t steps, uint32_t birth_mask,
                            uint32_t survive_mask, void *stream);
/* Blocked storage (Sec. 3, the blocked approach): k^(r-l) mini boxes of
 * rho^dim bytes, mini box b (coarse cell b in compact order) holding the
 * cells of the level-l sub-fractal b at their positions in its rho^dim box
 * (x fastest), 0 elsewhere.  fractal_blocked_info gives the layout's bytes;
 * pack / unpack convert from / to compact order (pack writes every byte). */
int fractal_blocked_info(fractal_t *f, int rho_levels, int64_t *bytes);
int fractal_blocked_pack(fractal_t *f, int rho_levels, const uint8_t *compact_dev,
                         uint8_t *blocked_dev, void *stream);
int fractal_blocked_unpack(fractal_t *f, int rho_levels, const uint8_t *blocked_dev,
                           uint8_t *compact_dev, void *stream);
/* "nu(omega)" on blocked storage: one block per mini box stages it in shared
 * memory and maps its 3^dim - 1 neighbouring coarse cells once (coarse lambda,
 * a Moore move, coarse nu); members read neighbours inside the block from
 * shared memory and across its edge from the neighbouring mini boxes.  in /
 * out: blocked layouts of the same rho, not overlapping. */
int fractal_blocked_step(fractal_t *f, int rho_levels, const uint8_t *in_dev, uint8_t *out_dev,
                         int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                         void *stream);

/* Compact <-> box views (through lambda).  scatter writes every box byte:
 * box_dev[lambda(omega)] = compact_dev[omega] != 0, and 0 off the fractal.
 * gather: compact_dev[omega] = box_dev[lambda(omega)] != 0. */
int fractal_scatter_to_box(const fractal_t *f, const uint8_t *compact_dev,
                           uint8_t *box_dev, void *stream);
int fractal_gather_from_box(const fractal_t *f, const uint8_t *box_dev,
                            uint8_t *compact_dev, void *stream);

/* End-to-end call from host memory: copies host_in (k^r bytes) to the device,
 * runs fractal_step for `steps` generations and copies the result to
 * host_out (k^r bytes), all on `stream`, and waits for it.  Device buffers
 * are owned by the handle (allocated on first use, reused, freed by
 * fractal_destroy). */
int fractal_run_host(fractal_t *f, const uint8_t *host_in, uint8_t *host_out,
                     int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                     void *stream);

/* Tile depth used by fractal_step: a tile is the k^L cells that share their
 * digits above level L (one subtree).  L = -1 restores the automatic choice.
 * fractal_get_tile_levels reports the depth the next step will use. */
int fractal_set_tile_levels(fractal_t *f, int levels);
int fractal_get_tile_levels(const fractal_t *f, int *levels);

/* Input pipeline depth of fractal_step: how many tiles each block has in
 * flight in shared memory (2, 3 or 4), or -1 for the policy's default.  More
 * stages keep more bytes in flight per block but fit fewer blocks per SM.
 * Results do not depend on it.  FR_EINVAL outside {-1, 2, 3, 4}; FR_EBUSY
 * (for a new value) while a server holds requests of the handle. */
int fractal_set_pipeline_stages(fractal_t *f, int stages);

/* Temporal blocking of fractal_step (and fractal_run_host): with
 * generations = g in [1, 9], every pass over the state advances it by up to
 * g generations (ceil(steps / g) passes), instead of one.  Each tile (a
 * level-L subtree) and the level-2 units of its neighbouring tiles that
 * touch it are loaded once, advanced in shared memory as a bitmap of the
 * embedded box with one bit per cell (a cell at distance d from the loaded
 * region's edge is exact for d generations; the tile's cells are 9 or more
 * cells in), and written back: HBM bytes per cell-update fall from 2 to
 * about (2 + halo) / g.  Results are those of single generations exactly.
 * Only for the Sierpinski carpet and the Vicsek fractal with the preset
 * offset tables (FR_EINVAL otherwise).  tile_levels: -1 = the deepest tile
 * whose shared memory stays within 100 KB, else in [2, r].  generations = 0
 * turns it off.  The batch, server and no-allocation calls are unaffected. */
int fractal_set_temporal_blocking(fractal_t *f, int generations, int tile_levels);

/* Launch plan of fractal_step for this handle (built, with its
 * allocations, if it does not exist yet, as by fractal_get_tile_levels).
 * info[0..n-1] receives, in order: the policy (0: cell by cell, 3 or 4:
 * groups of s^G x s^G cells, 9: 2D groups of 9 cells in a shared-memory
 * box, 10: the triangle's 81-cell units with taps, 11 / 12: the carpet's /
 * Vicsek fractal's level-2 units summed by rows, 13: the Vicsek fractal's
 * level-3 units summed in omega order, 14: a 3D tile's box summed by whole
 * rows, then gathered in omega order, 15: a 3D tile of depth 3 per warp,
 * its box bit-sliced), the tile depth L, threads per block, blocks per
 * launch, dynamic shared memory bytes per block, input pipeline stages (0:
 * none), and resident blocks per SM.  1 <= n <= 7, else FR_EINVAL. */
int fractal_plan_info(const fractal_t *f, int32_t *info, int n);

/* Autotuner of fractal_step: times one generation from in_dev into out_dev
 * (both k^r bytes; out_dev is overwritten) for each candidate tile depth
 * (the deepest whose shared-memory layout fits, and the three below) with
 * 2, 3 and 4 pipeline stages, keeps the fastest plan for this handle and
 * remembers it for every later handle of the same fractal and level on the
 * same GPU model in this process.  Waits for
 * `stream`.  *levels (if not NULL) receives the chosen depth. */
int fractal_autotune(fractal_t *f, const uint8_t *in_dev, uint8_t *out_dev,
                     uint32_t birth_mask, uint32_t survive_mask, void *stream,
                     int *levels);

/* ---- Batched execution of many independent instances ------------------
 * (not in the paper: it fuses the generations of many uneven instances so
 * that small instances do not pay one launch each per generation).
 *
 * A batch holds instances (handle, in, out, steps, rule).  fractal_batch_run
 * advances every instance by its own number of generations, exactly as
 * fractal_step(handle, in, out, steps, rule) would, but with one kernel
 * launch per generation for all instances that share a fractal and tile
 * depth, and the whole run captured into one CUDA graph that is launched on
 * `stream` (asynchronously).  The graph is kept and replayed by later runs
 * until instances are added or cleared.  Buffers stay owned by the caller and
 * must stay valid while a run is in flight; the batch owns a device arena for
 * its tables and for one k^r-byte ping-pong buffer per instance with
 * steps > 1.  Handles must outlive the batch's runs.  Before the first run
 * (and after any change) the batch builds its tables and the graph: that run
 * allocates and waits for the device, so make it before any stream capture. */
typedef struct fractal_batch fractal_batch_t;
int fractal_batch_create(fractal_batch_t **out);
int fractal_batch_destroy(fractal_batch_t *b);
/* Adds an instance; in_dev / out_dev: k^r bytes each, not overlapping.
 * *id (if not NULL) receives its index in the batch. */
int fractal_batch_add(fractal_batch_t *b, fractal_t *f, const uint8_t *in_dev,
                      uint8_t *out_dev, int64_t steps, uint32_t birth_mask,
                      uint32_t survive_mask, int64_t *id);
int fractal_batch_clear(fractal_batch_t *b);
int fractal_batch_run(fractal_batch_t *b, void *stream);
/* Cell updates and kernel launches of the last built run. */
int fractal_batch_stats(const fractal_batch_t *b, int64_t *updates, int64_t *launches);

/* ---- Serving: continuous batching of requests that arrive at any time ----
 * (not in the paper).  A server owns a worker thread and a stream on the
 * current device.  A request is (handle, seed and density of its Bernoulli
 * initial state, steps, rule, result destination).  The worker admits queued
 * requests in arrival order while their state (2 k^r bytes, stream-ordered
 * allocation) fits the HBM budget, then repeatedly advances every resident
 * request by up to `chunk` generations with one launch per group of
 * requests sharing a fractal and tile depth, so requests that arrive while
 * others run join the same launches.  A finished request's final state is
 * copied to `host_out` (k^r bytes, pinned memory recommended; it must stay
 * valid until the request is done) or, when host_out is NULL, reduced to its
 * live-cell count.  Its latency is the time from submit to the moment the
 * copy has landed.  The result equals fractal_step on the same initial state.
 *   hbm_budget_bytes  admission budget (<= 0: 90% of the free memory now);
 *                     a request needing more than the budget gets FR_EBUSY.
 *   chunk             generations per tick (>= 1).
 * Handles submitted to a server must outlive it.  While a server holds a
 * request of a handle that is not done, fractal_set_tile_levels (with a new
 * depth) and fractal_autotune on that handle return FR_EBUSY.  The first
 * submit of a handle builds its tables on the caller's thread. */
typedef struct fractal_server fractal_server_t;
int fractal_server_create(int64_t hbm_budget_bytes, int chunk, fractal_server_t **out);
int fractal_server_destroy(fractal_server_t *srv);   /* finishes all requests first */
int fractal_server_submit(fractal_server_t *srv, fractal_t *f, uint64_t seed, double p,
                          int64_t steps, uint32_t birth_mask, uint32_t survive_mask,
                          uint8_t *host_out, int64_t *request_id);
/* *done = 1 once the result has landed; then *latency_s = completion - submit
 * and *population = live cells (host_out == NULL only), else -1.  Any pointer
 * may be NULL.  FR_ENOTFOUND for an unknown id. */
int fractal_server_poll(fractal_server_t *srv, int64_t request_id, int *done,
                        double *latency_s, int64_t *population);
/* Blocks until every submitted request is done (or the server failed). */
int fractal_server_wait_all(fractal_server_t *srv);
int fractal_server_stats(fractal_server_t *srv, int64_t *completed, int64_t *queued,
                         int64_t *resident, int64_t *cell_updates, int64_t *launches,
                         int64_t *hbm_used);

/* Waits for `stream` and reports any asynchronous CUDA error. */
int fractal_sync(void *stream);

/* Waits for the device, then returns FR_ETIMEOUT if a kernel of this handle
 * gave up a bounded device-side wait since the last check (the outputs of
 * that call are then invalid), FR_OK otherwise.  Clears the flag. */
int fractal_check(fractal_t *f);

/* ---- One instance split over several shards (one per GPU) -------------
 * The paper's fractal is k replicas of the level below, each a contiguous
 * omega range filling its own sub-box (Sec. 1, Sec. 3), so an instance
 * splits into contiguous ranges of tiles (level-L subtrees of k^L cells):
 * shard g of G owns tiles [floor(g NT / G), floor((g+1) NT / G)), NT =
 * k^(r-L).  Each generation a shard needs, besides its own tiles, the
 * neighbouring tiles of other shards that its tiles' Moore neighbourhoods
 * reach (its halo).  A shard's buffer holds its own tiles (tile t0 + i at
 * cell i k^L), then its halo tiles grouped by owning shard in increasing
 * shard order, each group in increasing tile order.  One generation is:
 * every shard gathers, for each peer, the tiles that peer needs
 * (fractal_shard_pack) and the caller moves that send buffer into the
 * peer's buffer at the offset fractal_shard_sends reports (NCCL send/recv,
 * a peer copy, or a device copy when shards share a GPU); then every shard
 * runs fractal_shard_step.  Results equal fractal_step on the whole state.
 *
 * fractal_shard_plan computes the plan on the host (no GPU needed): the
 * fractal (as in fractal_create), the tile depth L in [0, r], the number of
 * shards G >= 1 and this shard's index.  FR_EINVAL for bad arguments or
 * fewer tiles than shards, FR_EOVERFLOW when NT (3^dim - 1) > 2^28. */
typedef struct fractal_shard fractal_shard_t;
int fractal_shard_plan(int k, int s, int r, int dim, const int32_t *offsets, int tile_levels,
                       int nshards, int shard, fractal_shard_t **out);
int fractal_shard_destroy(fractal_shard_t *p);
/* first_cell: omega of the shard's first own cell; local_cells: its own
 * cells; buffer_cells: own + halo cells (the size of its state buffers). */
int fractal_shard_info(const fractal_shard_t *p, int64_t *first_cell, int64_t *local_cells,
                       int64_t *buffer_cells);
/* The tiles (global tile indices, increasing) this shard sends to `peer`
 * each generation (tiles may be NULL to query *count; else capacity >=
 * *count), and *dst_cell, where that block starts in the peer's buffer.
 * The block is count * k^L bytes, tile after tile. */
int fractal_shard_sends(const fractal_shard_t *p, int peer, int64_t *tiles, int64_t capacity,
                        int64_t *count, int64_t *dst_cell);
/* The tiles this shard receives from `peer` and where they start in this
 * shard's buffer. */
int fractal_shard_recvs(const fractal_shard_t *p, int peer, int64_t *tiles, int64_t capacity,
                        int64_t *count, int64_t *dst_cell);
/* Host copy of the shard's neighbour table: for own tile i and Moore
 * direction d (dx, dy[, dz] in -1..1 with x fastest, the centre skipped),
 * table[i (3^dim - 1) + d] = the tile slot of the shard's buffer that holds
 * that neighbour (own tiles first, then the halo), or -1 if there is none. */
int fractal_shard_neighbours(const fractal_shard_t *p, int32_t *table, int64_t capacity);
/* Binds the plan to a handle of the same fractal on the current device: sets
 * the handle's tile depth to the plan's and uploads the shard's tables
 * (device allocations owned by the plan). */
int fractal_shard_attach(fractal_shard_t *p, fractal_t *f);
/* Gathers into send_dev (count * k^L bytes, see fractal_shard_sends) the
 * tiles `peer` needs, read from this shard's buffer_dev.  Asynchronous on
 * `stream`. */
int fractal_shard_pack(const fractal_shard_t *p, int peer, const uint8_t *buffer_dev,
                       uint8_t *send_dev, void *stream);
/* One generation (Sec. 3 stencil procedure) of the shard's own tiles:
 * in_dev is a full shard buffer (own tiles and a filled halo), out_dev a
 * buffer of the same size that does not overlap it; only its own-tile part
 * is written.  Asynchronous on `stream`. */
int fractal_shard_step(fractal_shard_t *p, const uint8_t *in_dev, uint8_t *out_dev,
                       uint32_t birth_mask, uint32_t survive_mask, void *stream);

/* Failure-detection test hook (not in the paper).  The next compact-step
 * kernel launch of this handle (the first generation of the next
 * fractal_step) arms each of its pipeline stages' barriers for extra_bytes
 * more bytes than it copies, so no stage ever completes, and each of its
 * bounded waits gives up after wait_tries tries (each try suspends for at
 * most about a microsecond) instead of the default ~4 million.  The kernel
 * then records the timeout, waits (bounded) for the copies it issued, and
 * returns without writing further results: that call's output is invalid and
 * the next fractal_check returns FR_ETIMEOUT.  Later launches are unaffected.
 * extra_bytes in [1, 4096], wait_tries in [1, 2^20], else FR_EINVAL. */
int fractal_test_arm_timeout(fractal_t *f, uint32_t extra_bytes, uint32_t wait_tries);

#ifdef __cplusplus
}
#endif

#endif /* FRACTAL_H */
