/*
 * pedsim.h - C ABI of the GB300 (sm_103a) bi-directional pedestrian cellular
 * automaton: the per-timestep update of the Least Effort Model (LEM) and of
 * the pheromone-guided Ant Colony Optimisation (ACO) variant of Dutta,
 * McLeod, Friesen, "GPU accelerated Nature Inspired Methods for Modelling
 * Large Scale Bi-Directional Pedestrian Movement".
 *
 * Model (Sec. III): two groups of agents on an H x W grid of cells (W, H
 * multiples of 16, Sec. IV.a).  Group A starts in the leftmost band_cols
 * columns and heads for the right edge (+x); group B starts in the rightmost
 * band_cols columns and heads for the left edge (-x).  Cells outside the grid
 * are never available.  One step (Sec. IV.b-d) is synchronous: every agent
 * reads the state at t and proposes a neighbouring empty cell (forward first,
 * else Eq. 1 for LEM or Eq. 2 for ACO); every empty cell then gathers the
 * agents that chose it from its eight neighbours and picks one (Sec. IV.d:
 * scatter turned into gather); pheromone evaporates (Eq. 3) and the movers
 * deposit into their own group's plane (Eq. 4, Eq. 5).  The default step
 * (PEDSIM_VARIANT_AGENT) resolves conflicts with no atomic operation; the
 * tiled and fused variants combine one tile's claims in shared memory with an
 * order-free bitwise OR.
 * Random numbers come from Philox4x64-10 keyed by (seed, cell, step, stream),
 * so results depend only on (W, H, params, seed, step count): not on the
 * stream, the launch shape, the tile shape or the batch a scenario runs in.
 *
 * Conventions for every call:
 *   - return value 0 on success or a negative PEDSIM_E* code; the message of
 *     the last failure of a handle is returned by sim_last_error() /
 *     sim_batch_last_error() / sim_pool_last_error();
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory of the current device;
 *   - calls on one handle are not thread-safe; distinct handles are
 *     independent.
 *
 * Grid layout in memory (all planes row-major, cell c = y * W + x):
 *   occ   uint8  W*H   0 = empty, 1 = group A agent, 2 = group B agent
 *   ids   uint32 W*H   agent id 1..2N at occupied cells, 0 at empty cells
 *   tauA  float  W*H   group A pheromone (ACO only)
 *   tauB  float  W*H   group B pheromone (ACO only)
 *   per-agent arrays have 2N+1 entries indexed by id (entry 0 unused):
 *   arrival uint32     step at which the agent first entered the opposite
 *                      placement band (0 = not yet), Sec. VI "throughput"
 *   tour    float      tour length L_k of Eq. 5 (deposit_mode 1)
 */
#ifndef PEDSIM_H
#define PEDSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PEDSIM_OK         0
#define PEDSIM_EINVAL   (-22)  /* bad argument: sizes, params, NULL handle   */
#define PEDSIM_ENOMEM   (-12)  /* device or host allocation failed           */
#define PEDSIM_ENOSPC   (-28)  /* HBM budget of a pool would be exceeded     */
#define PEDSIM_ECUDA    (-5)   /* a CUDA runtime call failed                 */
#define PEDSIM_ETIMEDOUT (-110)/* a bounded device wait gave up              */
#define PEDSIM_ENOENT   (-2)   /* no such scenario / slot                    */

#define PEDSIM_LEM 0u
#define PEDSIM_ACO 1u

/* Parameters of one scenario.
 * model        PEDSIM_LEM (Sec. II.A, Eq. 1) or PEDSIM_ACO (Sec. II.B, Eq. 2-5)
 * n_per_side   agents in each group (N); 0 is allowed (empty grid)
 * band_cols    width of each placement band; 1 <= band_cols, 2*band_cols <= W,
 *              n_per_side <= band_cols*H (Sec. III: agents confined to edge
 *              rows/columns at start)
 * rho          ACO evaporation rate of Eq. 3, 0 < rho <= 1
 * tau0         ACO initial pheromone on every cell, >= 0
 * deposit      ACO constant deposit per visit (deposit_mode 0), >= 0
 * alpha, beta  ACO exponents of Eq. 2, integers 0..4
 * deposit_mode 0 = constant `deposit`; 1 = 1/L_k of Eq. 5 with L_k the agent's
 *              tour length (1 per orthogonal move, fl(sqrt 2) per diagonal)
 * lem_sigma    standard deviation of the LEM normal rank draw, > 0          */
typedef struct {
    uint32_t model;
    uint32_t n_per_side;
    uint32_t band_cols;
    float    rho;
    float    tau0;
    float    deposit;
    uint32_t alpha;
    uint32_t beta;
    uint32_t deposit_mode;
    float    lem_sigma;
} sim_params;

/* Counters of one scenario.  agents/parked are counted from the grid when
 * read; crossed, moved and conflicts accumulate from step 0.
 * agents[g]    agents of group g on the grid (conserved)
 * crossed[g]   agents of group g that have entered the opposite band (Sec. VI)
 * parked[g]    agents of group g standing on their goal edge column
 * moved        total successful moves
 * conflicts    total (cell, step) pairs where >= 2 agents chose one cell    */
typedef struct {
    uint64_t step;
    uint32_t agents[2];
    uint32_t crossed[2];
    uint32_t parked[2];
    uint64_t moved;
    uint64_t conflicts;
} sim_stats_t;

typedef struct sim_s sim_t;

/* Fills *p with the defaults: LEM, N = 0, band 16, rho 0.05, tau0 1,
 * deposit 1, alpha = beta = 1, deposit_mode 0, lem_sigma 1.                  */
void sim_default_params(sim_params *p);

/* Checks (W, H, *p) against the rules above; PEDSIM_EINVAL if any fails.   */
int sim_validate(int W, int H, const sim_params *p);

/* Device bytes one scenario of this size needs (planes, per-agent arrays,
 * counters); the figure used by pool admission.                              */
size_t sim_device_bytes(int W, int H, const sim_params *p);

/* Creates a scenario on the current CUDA device and allocates its device
 * state (owned by the library, freed by sim_destroy).  The grid is empty
 * until sim_place() or sim_set_state().  *out receives the handle.           */
int sim_create(int W, int H, const sim_params *p, sim_t **out);

/* Routes all later work of this handle to `stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream); NULL = the legacy default stream.
 * The library never synchronises the device, only this stream.              */
int sim_set_stream(sim_t *s, void *stream);

/* Random uniform placement (Sec. IV.a): in each band the n_per_side cells
 * with the smallest Philox keys (seed, cell, step 0, stream 3) are filled;
 * group A gets ids 1..N and group B ids N+1..2N in increasing cell index.
 * Pheromone := tau0, arrival := 0, tour := 0, counters := 0, step := 0.
 * Asynchronous on the stream.                                                 */
int sim_place(sim_t *s, uint64_t seed);

/* Advances n >= 0 synchronous steps (Sec. IV.b-d), asynchronously on the
 * stream.  Long runs replay a captured CUDA graph.  A call with n < 16
 * issues plain kernel launches and may be captured into the caller's own
 * CUDA graph: every replay advances the step index kept on the device, which
 * sim_read_grid, sim_stats and sim_save take as the current step.            */
int sim_step(sim_t *s, int n);

/* Copies the grid at the current step into host buffers (any may be NULL);
 * ids are 0 at empty cells.  Synchronises the stream.                         */
int sim_read_grid(sim_t *s, uint8_t *occ, uint32_t *ids, float *tauA, float *tauB);

/* Copies the per-agent arrays (2N+1 entries each, may be NULL) to the host.
 * Synchronises the stream.                                                    */
int sim_read_agents(sim_t *s, uint32_t *arrival, float *tour);

/* Replaces the state with a host-provided one (the inputs of an end-to-end
 * run).  occ/ids must describe 2N agents with ids a permutation of 1..2N,
 * N = p->n_per_side of sim_create; tauA/tauB/arrival/tour may be NULL (tau0,
 * zero, zero).  step becomes the step index; counters are reset.  The seed
 * is the one used by later steps.  Asynchronous (host buffers are staged).   */
int sim_set_state(sim_t *s, uint64_t seed, uint64_t step, const uint8_t *occ,
                  const uint32_t *ids, const float *tauA, const float *tauB,
                  const uint32_t *arrival, const float *tour);

/* Counters at the current step (see sim_stats_t).  Synchronises the stream. */
int sim_stats(sim_t *s, sim_stats_t *out);

/* Checkpoint: serialises the complete state (params, seed, step, planes,
 * per-agent arrays, counters).  With buf == NULL, *len receives the size
 * needed.  sim_load restores a checkpoint written for the same W, H and
 * params; continuing from it is bit-identical to never having stopped.       */
int sim_save(sim_t *s, void *buf, size_t *len);
int sim_load(sim_t *s, const void *buf, size_t len);

/* Step implementations; all give bit-identical results.
 * PEDSIM_VARIANT_TILED    two kernels per step: TMA-staged
 *                         proposals of 128 x tile_h tiles into a 1-byte
 *                         proposal plane, then TMA-staged gather resolution
 *                         with streamed pheromone evaporation and deposit
 * PEDSIM_VARIANT_TWO_PASS the same two passes, one thread per cell, plain
 *                         loads (reference baseline of the tiled kernels)
 * PEDSIM_VARIANT_FUSED    one persistent kernel per step over TMA-staged
 *                         tiles with a 3-cell halo (proposals recomputed in
 *                         the halo instead of a proposal plane); only tiles
 *                         with an agent in or next to them take the full
 *                         rule, the others only evaporate
 * PEDSIM_VARIANT_AGENT    (default) two kernels per step: one thread per agent
 *                         computes its proposal (written at its own cell of a
 *                         code plane) while the other CTAs of the same kernel
 *                         stream the pheromone evaporation of most cells; then
 *                         one thread per agent gathers its target's claimants
 *                         from the codes of the target's neighbours and
 *                         applies the winner's move and deposit, while
 *                         further CTAs evaporate the remaining cells (skipping
 *                         the claimed ones, which their winners write), and
 *                         the last CTA advances the step index
 * PEDSIM_VARIANT_DEFERRED the agent step without the dense evaporation
 *                         stream (deferred evaporation): each cell keeps a
 *                         one-byte stamp, the step at which its stored
 *                         pheromone values are valid, and a value is brought
 *                         up to date, by repeating Eq. 3's multiplication once
 *                         per missed step, only where it is read (a blocked
 *                         agent's available neighbours, a winner's target) and
 *                         in a rolling refresh of 1/32 of the cells per step
 *                         (no value is ever more than 32 steps old).  The same
 *                         operations in the same order as evaporating every
 *                         cell every step, so the results are identical; the
 *                         dense traffic drops from 18 to 18/32 bytes per
 *                         cell-step.  Read-back and checkpoints bring the
 *                         planes up to the current step first.
 * Selecting a variant resets the tile shape to its default (tiled: 128 x 16;
 * fused: 64 x 16; the agent and deferred variants have none).                */
#define PEDSIM_VARIANT_TILED    0
#define PEDSIM_VARIANT_TWO_PASS 1
#define PEDSIM_VARIANT_FUSED    2
#define PEDSIM_VARIANT_AGENT    3
#define PEDSIM_VARIANT_DEFERRED 4
int sim_set_variant(sim_t *s, int variant);

/* Kernel launches that sim_step(s, 1) issues with the current variant into
 * *out (agent and deferred: 2; fused: 2; tiled and two-pass: 3, each counting
 * the step-index advance); PEDSIM_EINVAL for a null argument.                 */
int sim_launches_per_step(sim_t *s, int *out);

/* Tile shape of the current variant: tiled: tile_w = 128, tile_h in
 * {8, 16}; fused: (tile_w, tile_h) in {(32,16), (64,8), (64,16),
 * (128,8), (128,16)} plus CTAs per SM of its persistent grid (0 =
 * automatic; ignored by the tiled variant).  PEDSIM_EINVAL otherwise, and
 * always for the agent and two-pass variants.                                */
int sim_set_tiling(sim_t *s, int tile_w, int tile_h, int ctas_per_sm);

/* Sticky device error word of the handle: 0, or PEDSIM_ETIMEDOUT when a
 * bounded device wait gave up.  Synchronises the stream and clears it.       */
int sim_device_status(sim_t *s);

/* Failure-detection test hook (the paper has no counterpart: its single GPU
 * run has no failure handling).  wait_cycles bounds every wait of the tiled
 * variant (PEDSIM_VARIANT_TILED) on its TMA copies, in SM clock cycles
 * (0 = the default, about 2 s at the maximum clock).  With test_flags =
 * PEDSIM_TEST_SKIP_RESOLVE_LOADS the tiled resolution kernel issues none of
 * its TMA loads, so its wait runs out: every CTA returns without writing any
 * state, with nothing in flight, and the handle's device error word becomes
 * PEDSIM_ETIMEDOUT (sim_device_status).  The state of the handle is then
 * undefined (that step's resolution did not happen); destroy it.  No fault,
 * trap or unbounded wait is involved, so the CUDA context stays usable.
 * Takes effect from the next step; PEDSIM_EINVAL for unknown flags.           */
#define PEDSIM_TEST_SKIP_RESOLVE_LOADS 1u
int sim_set_wait_test(sim_t *s, uint64_t wait_cycles, uint32_t test_flags);

void sim_destroy(sim_t *s);
const char *sim_last_error(const sim_t *s);

/* ------------------------------------------------------------------------ */
/* Batched scenarios: many independent scenarios of uneven size, density and */
/* model advanced together, each step one persistent launch over all        */
/* (scenario, tile) work items, the step loop replayed as a CUDA graph.      */
/* Every scenario's results are bit-identical to running it alone.           */
/* ------------------------------------------------------------------------ */
typedef struct batch_s batch_t;

/* Creates n scenarios (W[i], H[i], params[i]) and places each with seeds[i]. */
int sim_batch_create(int n, const int *W, const int *H, const sim_params *params,
                     const uint64_t *seeds, batch_t **out);
int sim_batch_set_stream(batch_t *b, void *stream);
/* Advances every scenario by n steps (asynchronous).                         */
int sim_batch_step(batch_t *b, int n);
/* Counters / grid of scenario i (synchronise the stream).                    */
int sim_batch_stats(batch_t *b, int i, sim_stats_t *out);
int sim_batch_read_grid(batch_t *b, int i, uint8_t *occ, uint32_t *ids, float *tauA,
                        float *tauB);
/* Step variant (PEDSIM_VARIANT_TILED, _FUSED, _AGENT or _DEFERRED) and tile
 * shape of the batched launches (see sim_set_variant / sim_set_tiling).      */
int sim_batch_set_variant(batch_t *b, int variant);
int sim_batch_set_tiling(batch_t *b, int tile_w, int tile_h, int ctas_per_sm);
int sim_batch_device_status(batch_t *b);
void sim_batch_destroy(batch_t *b);
const char *sim_batch_last_error(const batch_t *b);

/* ------------------------------------------------------------------------ */
/* Serving pool: device-resident scenario slots admitted against an HBM      */
/* budget and stepped together (continuous batching: a slot that finishes   */
/* frees its memory and a waiting request can be admitted at once).          */
/* ------------------------------------------------------------------------ */
typedef struct pool_s pool_t;

/* hbm_budget_bytes bounds the sum of sim_device_bytes() of live slots;
 * max_slots bounds their number.  The slots are allocated from a CUDA memory
 * pool of the pool's own on the current device, which keeps up to
 * hbm_budget_bytes reserved while slots come and go (released to the system
 * by sim_pool_destroy).  PEDSIM_ECUDA if that pool cannot be created.         */
int sim_pool_create(size_t hbm_budget_bytes, int max_slots, pool_t **out);
int sim_pool_set_stream(pool_t *pl, void *stream);
/* Admits one request: allocates its state, places it with `seed` and
 * schedules `steps` steps.  *slot receives its slot id.  PEDSIM_ENOSPC when
 * the budget or the slot count would be exceeded (nothing is allocated).     */
int sim_pool_admit(pool_t *pl, int W, int H, const sim_params *p, uint64_t seed,
                   uint64_t steps, int *slot);
/* Advances every live, unfinished slot by up to n steps (a slot stops at its
 * own step count) in one graph-captured persistent launch per step.          */
int sim_pool_step(pool_t *pl, int n);
/* Lists finished slots (synchronises the stream): up to max ids into
 * done[], their number into *n_done.                                          */
int sim_pool_finished(pool_t *pl, int *done, int max, int *n_done);
int sim_pool_stats(pool_t *pl, int slot, sim_stats_t *out);
int sim_pool_read_grid(pool_t *pl, int slot, uint8_t *occ, uint32_t *ids, float *tauA,
                       float *tauB);
/* Frees a slot (finished or not) and its device memory.                       */
int sim_pool_release(pool_t *pl, int slot);
size_t sim_pool_bytes_in_use(const pool_t *pl);
int sim_pool_live(const pool_t *pl);
void sim_pool_destroy(pool_t *pl);
const char *sim_pool_last_error(const pool_t *pl);

/* ------------------------------------------------------------------------ */
/* Domain decomposition: one step of a column strip of a larger grid.        */
/* ------------------------------------------------------------------------ */
/* A W_global x H grid split into strips of columns (each on its own device
 * or stream) advances by one sim_step_strip call per strip and step, with
 * the strips' halos refreshed from their neighbours' interiors in between
 * (paper_1412_4933_gb300/domain.py does both).  The strip's buffers hold its
 * local columns: interior_lo .. interior_hi-1 are its own, the others (at most
 * three on each side, more are allowed but unused) a halo copied from the
 * neighbouring strips.  The state of a cell after one step depends only on
 * cells at most three columns away (Sec. IV.b-d: a claimant's proposal needs
 * its 3 x 3 neighbourhood, an agent's departure its target's other
 * claimants), so with three halo columns the interior comes out bit for bit
 * as in sim_step on the whole grid; the halo's own results are to be
 * replaced by the next exchange.  Random numbers, the goal edge and the
 * crossing line use global coordinates (x0 = global column of local column
 * 0); neighbours beyond the strip's local columns count as unavailable.
 *   W, H            local width (interior + halos) and height (= the grid's)
 *   x0, W_global    global column of local column 0; width of the whole grid
 *   interior_lo/hi  the strip's own local columns [lo, hi); only events whose
 *                   target cell lies there are added to `counters`
 *   p, seed, step   the whole grid's parameters (validated against
 *                   W_global x H), its seed and the step index being taken
 *   occ_in/occ_out, ids, tau*_in/out, arrival, tour, counters
 *                   as in sim_step_noalloc, all device memory of the caller,
 *                   W x H local cells (per-agent arrays: 2N+1 entries; an
 *                   agent's entries must be current whenever it stands in the
 *                   strip's local columns)
 *   scratch         device uint8 W*H owned by the caller (the proposal plane)
 *   stream          cudaStream_t, NULL = the legacy default stream
 * Asynchronous on the stream; allocates nothing.  PEDSIM_EINVAL for invalid
 * parameters, columns outside the grid, NULL buffers, or occ_in, occ_out
 * and scratch sharing bytes; PEDSIM_ECUDA when a launch fails.  The paper
 * runs one grid on one GPU (Sec. V); this call serves the decomposition of
 * one grid over several devices, which the paper does not address.          */
int sim_step_strip(int W, int H, int x0, int W_global, int interior_lo, int interior_hi,
                   const sim_params *p, uint64_t seed, uint64_t step, const uint8_t *occ_in,
                   uint8_t *occ_out, uint32_t *ids, const float *tauA_in, const float *tauB_in,
                   float *tauA_out, float *tauB_out, uint32_t *arrival, float *tour,
                   uint8_t *scratch, unsigned long long *counters, void *stream);

/* Halo exchange between two strips on one device (or on devices with peer
 * access): columns [src_col, src_col + ncols) of the source strip's local
 * planes (width src_W) are copied into columns [dst_col, dst_col + ncols) of
 * the destination's (width dst_W), both H rows -- occupancy, ids and, for
 * ACO, both pheromone planes of the step's parity -- and for every copied
 * cell holding agent id (1..n_agents) that agent's arrival step and tour
 * length are copied from the source's per-agent arrays into the
 * destination's (n_agents + 1 entries each; the tour pair may be NULL when
 * the scenario keeps none).  This is the exchange sim_step_strip expects
 * between steps.  All pointers are device memory of the caller; the tau
 * pointers are all NULL (LEM) or all set.  Asynchronous on `stream` (NULL =
 * the legacy default stream), one kernel, no allocation; PEDSIM_EINVAL for
 * columns outside either strip or inconsistent NULL pointers, PEDSIM_ECUDA
 * when the launch fails.                                                      */
int sim_strip_halo(int H, int ncols, uint32_t n_agents, const uint8_t *src_occ,
                   const uint32_t *src_ids, const float *src_tauA, const float *src_tauB,
                   const uint32_t *src_arrival, const float *src_tour, int src_W, int src_col,
                   uint8_t *dst_occ, uint32_t *dst_ids, float *dst_tauA, float *dst_tauB,
                   uint32_t *dst_arrival, float *dst_tour, int dst_W, int dst_col, void *stream);

/* ------------------------------------------------------------------------ */
/* Allocation-free step.  The paper has no counterpart: this entry point     */
/* exists for callers that cannot let a library allocate device memory while */
/* they run -- applications that reserve all device memory up front under a  */
/* fixed budget, frameworks whose caching allocator must account for every   */
/* byte, code that records work into CUDA graphs.  It performs no cudaMalloc, */
/* cudaFree or other allocation.                                             */
/* ------------------------------------------------------------------------ */
/* Advances the scenario (W, H, *p, seed) by one step, from step index `step`
 * to step + 1, on caller-owned device buffers, asynchronously on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Same rules and bit-exact
 * results as sim_step.
 *   occ_in / occ_out   device uint8 W*H, the occupancy at `step` / step+1
 *                      (distinct buffers)
 *   ids                device uint32 W*H, updated in place (valid at occupied
 *                      cells; stale values may remain at vacated cells)
 *   tauA_in, tauB_in / tauA_out, tauB_out
 *                      device float W*H pheromone at step / step+1 (ACO only;
 *                      may be NULL for LEM)
 *   arrival, tour      device per-agent arrays of 2N+1 entries, updated in
 *                      place (tour only for ACO with deposit_mode 1)
 *   counters           device uint64[4] to which the step ADDS moved,
 *                      conflicts, crossed[A], crossed[B]; may be NULL
 * Scratch: the one-byte proposal plane between the two passes lives in a
 * device array of the library sized for at most 16,777,216 (2^24) cells,
 * e.g. 4096 x 4096; larger grids give PEDSIM_EINVAL.  The array exists on
 * every GPU that loads the library until the library is unloaded.  It is
 * shared by all calls (every call rewrites the part it uses before reading
 * it), so calls whose work overlaps on the GPU -- on different streams or
 * from different threads -- race and must be serialised by the caller.  The
 * first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture; the cached address belongs to the device's context and must not
 * be used after a cudaDeviceReset of that device.  Returns PEDSIM_EINVAL for
 * invalid parameters or sizes, NULL buffers or occupancy buffers that share
 * any byte, PEDSIM_ECUDA when a launch fails.                                 */
int sim_step_noalloc(int W, int H, const sim_params *p, uint64_t seed, uint64_t step,
                     const uint8_t *occ_in, uint8_t *occ_out, uint32_t *ids,
                     const float *tauA_in, const float *tauB_in, float *tauA_out,
                     float *tauB_out, uint32_t *arrival, float *tour,
                     unsigned long long *counters, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PEDSIM_H */
