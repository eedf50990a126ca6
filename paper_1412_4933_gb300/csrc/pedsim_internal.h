// Internal interface between the kernel translation unit and the C-ABI host
// library.  Not installed; include/pedsim.h is the public boundary.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace pedsim {

// Per-scenario descriptor in device memory.  A single simulation is a batch
// of one; the batched and serving paths hold arrays of these.
//   occ[p]        uint8 occupancy plane of parity p (state at step t lives in
//                 occ[t & 1])
//   tau[g][p]     float pheromone plane of group g (0 = A, 1 = B), parity p
//   ids           uint32 agent-id plane, updated in place (a move reads the
//                 source cell, occupied at t, and writes the target cell,
//                 empty at t: the two sets are disjoint within one step)
//   counters      moved, conflicts, crossed[A], crossed[B]
//   step          current step index; every step kernel reads t = *step +
//                 t_off, so one captured graph replays at any step
//   end_step      the scenario does not advance past this step
struct alignas(128) ScenarioDesc {
    CUtensorMap map_occ[2];      // box (tile_w + 32) x (tile_h + 6), uint8
    CUtensorMap map_tau[2][2];   // [group][parity], box tile_w x tile_h, float
    uint8_t *occ[2];
    uint32_t *ids;
    float *tau[2][2];
    uint32_t *arrival;
    float *tour;
    unsigned long long *counters;
    unsigned long long *step;
    unsigned long long end_step;
    unsigned long long seed;
    int *error;
    int W, H;
    int tiles_x, tiles_y;
    uint32_t model, alpha, beta, deposit_mode;
    uint32_t band, n_per_side;
    float q;          // fl(1 - rho)
    float deposit;    // constant deposit (deposit_mode 0)
    float lem_scale;  // fl(2^-16 / sigma)
    float tau0;
    int tile_w, tile_h;
    int pad_[2];
};

// Counter slots.
enum { kMoved = 0, kConflicts = 1, kCrossedA = 2, kCrossedB = 3, kNumCounters = 4 };

// Grid read-back helpers: agents[A], agents[B], parked[A], parked[B].
enum { kGridCounts = 4 };

// Step-kernel variants.
enum { kVariantFused = 0, kVariantTwoPass = 1 };

// Supported fused tile shapes (tile_w x tile_h).
bool tile_supported(int tile_w, int tile_h);

// ---- launchers (all asynchronous on `stream`) ----------------------------
// Clear planes, fill pheromone with tau0, zero per-agent arrays, counters and
// the step index of scenarios [0, n).
cudaError_t launch_init(const ScenarioDesc *d_descs, int n, int max_cells, int max_agents,
                        cudaStream_t stream);
// Random placement of both groups of scenarios [0, n).
cudaError_t launch_place(const ScenarioDesc *d_descs, int n, cudaStream_t stream);
// One fused step (t = *step + t_off) over all (scenario, tile) items.
// tile_prefix[i] = first work item of scenario i, tile_prefix[n] = total.
cudaError_t launch_fused_step(const ScenarioDesc *d_descs, const uint32_t *d_tile_prefix,
                              int n, uint32_t total_tiles, int t_off, int tile_w,
                              int tile_h, int grid, cudaStream_t stream);
// Two-pass step of one scenario: proposal plane, then resolution.
cudaError_t launch_two_pass_step(const ScenarioDesc *d_desc, uint8_t *d_prop, int W, int H,
                                 int t_off, cudaStream_t stream);
// *step += k for scenarios [0, n) (clamped at end_step).
cudaError_t launch_advance(const ScenarioDesc *d_descs, int n, int k, cudaStream_t stream);
// agents/parked per group of the plane of parity p of one scenario.
cudaError_t launch_grid_counts(const ScenarioDesc *d_desc, int parity, int cells,
                               unsigned int *d_out, cudaStream_t stream);
// out[c] = occ[c] ? ids[c] : 0 for the plane of parity p.
cudaError_t launch_mask_ids(const ScenarioDesc *d_desc, int parity, int cells,
                            uint32_t *d_out, cudaStream_t stream);
// Resident CTAs per SM of the fused kernel of this tile shape.
int fused_blocks_per_sm(int tile_w, int tile_h);
int fused_threads();

}  // namespace pedsim
