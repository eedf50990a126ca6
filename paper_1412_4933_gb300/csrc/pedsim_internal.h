// Internal interface between the kernel translation unit and the C-ABI host
// library.  Not installed; include/pedsim.h is the public boundary.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace pedsim {

// Per-scenario descriptor in device memory.  A single simulation is a batch
// of one; the batched and serving paths hold arrays of these (each handle's
// device descriptor then lives in that array, so the step index has a single
// home).
//
// The first kDescHeaderBytes hold everything a CTA needs besides the tensor
// maps, so one 16-byte-per-thread copy brings a scenario into shared memory.
//   step          step index at the start of the current launch group: a
//                 step kernel works on step t = step + t_off (t_off a kernel
//                 argument) and a one-thread-per-scenario kernel adds the
//                 group's step count at its end, so one captured graph
//                 replays at any step
//   end_step      the scenario does not advance past this step
//   occ[p]        uint8 occupancy plane of parity p (state at step t lives in
//                 occ[t & 1]; the agent-parallel variant updates occ[0] in
//                 place at every step)
//   prop          uint8 proposal plane (two-kernel variants)
//   tau[g][p]     float pheromone plane of group g (0 = A, 1 = B), parity p
//   ids           uint32 agent-id plane, updated in place (a move reads the
//                 source cell, occupied at t, and writes the target cell,
//                 empty at t: the two sets are disjoint within one step)
//   part          per-slot partial counters (moved, conflicts, crossed[A],
//                 crossed[B]) x n_slots: each tile (or CTA) adds its counts to
//                 its own slot, so no two writers share an address; totals
//                 are the slot sums
//   pos           uint32 cell index of every agent, indexed by id (agent-
//                 parallel variant; rebuilt from the planes whenever the
//                 state is set from outside it)
//   acode         uint8 per agent: proposal code of the current step | group
//                 << 4 (the group from the moment the positions are built),
//                 | 0x80 once the agent has moved (agent-parallel and
//                 deferred variants)
//   codes[q]      uint8 code planes of the agent-parallel variant: at step
//                 t, codes[t & 1] holds each agent's direction code (0 =
//                 stay) at its cell and 0 at every cell empty at t; the
//                 resolution gathers a target's claimants from its eight
//                 neighbours there
//   wait_cycles   SM clock cycles after which a bounded wait of the tiled
//                 variant gives up (0 = kWaitCycles, about 2 s)
//   stamp         uint8 per cell (ACO), deferred-evaporation variant: the low
//                 byte of the step at which the cell's values in tau[g][0]
//                 are valid (the variant keeps one plane per group, updated
//                 in place)
//   w_mul, w_shr  division of a cell index by W without a divide: with
//                 l = ceil(log2 W), w_mul = floor(2^(31+l) / W) + 1 and
//                 w_shr = l - 1, floor(c / W) = umulhi(c, w_mul) >> w_shr for
//                 every c < 2^31 (the round-up method of Granlund and
//                 Montgomery, 1994: w_mul * W exceeds 2^(31+l) by at most W)
//   test_flags    failure-detection test hook: with kTestSkipResolveLoads the
//                 tiled resolution kernel issues none of its TMA loads, so
//                 its bounded wait runs out and it returns without writing
//                 any state
constexpr int kDescHeaderBytes = 256;
constexpr uint32_t kTestSkipResolveLoads = 1u;

struct alignas(128) ScenarioDesc {
    unsigned long long step;
    unsigned long long end_step;
    unsigned long long seed;
    int W, H;
    int tiles_x, tiles_y;
    int tile_w, tile_h;
    uint32_t model, alpha, beta, deposit_mode;
    uint32_t band, n_per_side;
    float q;          // fl(1 - rho)
    float deposit;    // constant deposit (deposit_mode 0)
    float lem_scale;  // fl(2^-16 / sigma)
    float tau0;
    uint32_t n_slots; // entries of `part` (x kNumCounters)
    uint32_t pad0_;
    uint8_t *occ[2];
    uint8_t *prop;
    uint32_t *ids;
    float *tau[2][2];
    uint32_t *arrival;
    float *tour;
    unsigned long long *part;
    int *error;
    uint32_t *pos;
    uint8_t *acode;
    uint8_t *codes[2];
    unsigned long long wait_cycles;  // limit of the tiled variant's bounded waits (0 = default)
    uint32_t test_flags;             // kTestSkipResolveLoads (failure-detection test only)
    uint32_t pad1_;
    uint8_t *stamp;                  // deferred-evaporation stamps (ACO)
    uint32_t w_mul, w_shr;           // cell / W = umulhi(cell, w_mul) >> w_shr (cell < 2^31)
    uint8_t header_pad_[kDescHeaderBytes - 96 - 16 * 8 - 32];
    // TMA tensor maps; boxes follow the variant and tile shape:
    //   tiled two-kernel step: occ (tile_w + 32) x (tile_h + 2), occ_out and
    //   prop_out tile_w x tile_h, prop (tile_w + 32) x (tile_h + 4), tau
    //   tile_w x tile_h (loads and stores);
    //   fused step: occ (tile_w + 32) x (tile_h + 6), tau (tile_w + 8) x
    //   (tile_h + 6), tau_tile tile_w x tile_h (quiet tiles).
    CUtensorMap map_occ[2];
    CUtensorMap map_occ_out[2];
    CUtensorMap map_prop;
    CUtensorMap map_prop_out;
    CUtensorMap map_tau[2][2];       // [group][parity]
    CUtensorMap map_tau_tile[2][2];  // [group][parity]
};
static_assert(sizeof(ScenarioDesc) == kDescHeaderBytes + 14 * sizeof(CUtensorMap),
              "descriptor header layout");

// Tile-activity control block of one work list of the fused step (device
// memory).  It is followed by flags[3][ceil(total / 32)] (one bit per work
// item) and list[3][total] (work item indices), total being the work list's
// item count.  Launch k uses generation g = phase: flags[g] marks the active
// tiles and list[g][0 .. n_act[g]) enumerates them; it sets generation
// (g + 1) % 3 for the next launch and clears (g + 2) % 3.  All zero except
// `reset` = nonzero after the host changes the work list or a state: that
// launch treats every tile as active.
struct ActivityCtl {
    uint32_t ticket;    // elects the launch's last CTA (fused and agent variants)
    uint32_t work;      // next entry of the active list to hand out
    uint32_t phase;     // launch index mod 3
    uint32_t reset;
    uint32_t n_act[3];
    uint32_t work_nat;  // next work item of the natural-order pass
};
// The multiplier and shift of the division by W (see ScenarioDesc).
inline void division_by_width(int W, uint32_t *mul, uint32_t *shr)
{
    uint32_t l = 0;
    while ((1ull << l) < (unsigned long long)W) ++l;
    *mul = (uint32_t)(((1ull << (31 + l)) / (unsigned long long)W) + 1ull);
    *shr = l - 1;
}

inline size_t activity_bytes(uint32_t total)
{
    return sizeof(ActivityCtl) + 4 * (3 * (((size_t)total + 31) / 32) + 3 * (size_t)total);
}

// Counter slots.
enum { kMoved = 0, kConflicts = 1, kCrossedA = 2, kCrossedB = 3, kNumCounters = 4 };

// Grid read-back helpers: agents[A], agents[B], parked[A], parked[B].
enum { kGridCounts = 4 };

// Step-kernel variants.
enum { kVariantPipeline = 0, kVariantTwoPass = 1, kVariantFused = 2, kVariantAgent = 3,
       kVariantDeferred = 4 };

// Work units of the agent-parallel variant: cells per CTA of its streaming
// pass (8 per thread: measured best among 4, 8, 16 and 32 at 2048^2 and
// 8192^2), agents per CTA of its proposal and resolution passes.
#ifndef PEDSIM_CELL_BLOCK
#define PEDSIM_CELL_BLOCK 2048
#endif
constexpr int kCellBlock = PEDSIM_CELL_BLOCK;
constexpr int kAgentBlock = 256;

// Supported fused tile shapes (tile_w x tile_h).
bool tile_supported(int tile_w, int tile_h);

// ---- launchers (all asynchronous on `stream`) ----------------------------
// Clear planes, fill pheromone with tau0, zero per-agent arrays, counters and
// the error word of scenarios [0, n).
cudaError_t launch_init(const ScenarioDesc *d_descs, int n, int max_cells, int max_agents,
                        cudaStream_t stream);
// Random placement of both groups of scenarios [0, n).
cudaError_t launch_place(const ScenarioDesc *d_descs, int n, cudaStream_t stream);
// One fused step (t = step + t_off) over all (scenario, tile) items;
// tile_prefix[i] = first work item of scenario i, tile_prefix[n] = total.
// `act` is the work list's activity block (activity_bytes(total) bytes).
cudaError_t launch_fused_step(const ScenarioDesc *d_descs, const uint32_t *d_tile_prefix,
                              int n, uint32_t total_tiles, int t_off, int tile_w, int tile_h,
                              int grid, ActivityCtl *act, cudaStream_t stream);
// Tiled two-kernel step (K1 proposals, K2 resolution) over all (scenario,
// tile) items; tiles are 128 x tile_h.
bool pipeline_tile_supported(int tile_w, int tile_h);
cudaError_t launch_pipeline_step(const ScenarioDesc *d_descs, const uint32_t *d_tile_prefix, int n,
                                 uint32_t total_tiles, int t_off, int tile_h, cudaStream_t stream);
// Two-pass step of one scenario: proposal plane, then resolution.  Its grid
// never exceeds two_pass_grid(W, H) CTAs (one counter slot each).
int two_pass_grid(int W, int H);
cudaError_t launch_two_pass_step(const ScenarioDesc *d_desc, uint8_t *d_prop, int W, int H,
                                 int t_off, cudaStream_t stream);
// Agent-parallel step over scenarios [0, n) at each scenario's step index,
// which the step advances itself (no launch_advance for this variant):
// cell_prefix[i] / agent_prefix[i] = first cell / agent block of scenario i
// (ceil(W*H / kCellBlock) and ceil(2 n_per_side / kAgentBlock) per
// scenario), [n] = the totals.  ctl->ticket (zero between launches) elects
// the CTA that advances the step indices.
cudaError_t launch_agent_step(const ScenarioDesc *d_descs, const uint32_t *d_cell_prefix,
                              const uint32_t *d_agent_prefix, int n, uint32_t cell_blocks,
                              uint32_t agent_blocks, ActivityCtl *ctl, cudaStream_t stream);
// Deferred-evaporation step over scenarios [0, n) (the agent-parallel step
// without the dense stream; see pedsim_agent.cu): slice_prefix[i] = first
// refresh CTA of scenario i (deferred_slices(its cell blocks) each).
cudaError_t launch_deferred_step(const ScenarioDesc *d_descs, const uint32_t *d_cell_prefix,
                                 const uint32_t *d_agent_prefix, const uint32_t *d_slice_prefix,
                                 int n, uint32_t slices, uint32_t agent_blocks, ActivityCtl *ctl,
                                 cudaStream_t stream);
uint32_t deferred_slices(uint32_t cell_blocks);
// Brings one scenario's deferred pheromone planes up to its current step.
cudaError_t launch_deferred_catch_up(const ScenarioDesc *d_desc, int cells, cudaStream_t stream);
// Rebuilds pos[] of one scenario from its occupancy plane `plane` and clears
// its code planes and per-agent codes (agent-parallel variant).
cudaError_t launch_build_pos(const ScenarioDesc *d_desc, int cells, int plane,
                             cudaStream_t stream);
// step += k (clamped at end_step) for scenarios [0, n).
cudaError_t launch_advance(const ScenarioDesc *d_descs, int n, int k, cudaStream_t stream);
// out[0..3] = counter totals of one scenario (sums over its slots).
cudaError_t launch_sum_slots(const ScenarioDesc *d_desc, unsigned long long *d_out,
                             cudaStream_t stream);
// agents/parked per group of the plane of parity p of one scenario.
cudaError_t launch_grid_counts(const ScenarioDesc *d_desc, int parity, int cells,
                               unsigned int *d_out, cudaStream_t stream);
// Resident CTAs per SM of the fused kernel of this tile shape.
int fused_blocks_per_sm(int tile_w, int tile_h);
int fused_threads();

}  // namespace pedsim
