// Agent-parallel step (PEDSIM_VARIANT_AGENT) of the pedestrian cellular
// automaton (sm_103a).  One synchronous step (Sec. IV.b-d) is split by
// access pattern instead of by tile:
//
//   agent_propose_kernel  one thread per agent: forward first, else the full
//                         rule (Eq. 1 LEM rank draw, Eq. 2 ACO roulette) from
//                         the occupancy and pheromone at t; the direction code
//                         goes to the agent's cell of the proposal plane
//   stream_kernel         every cell: occupancy copied to the plane of t+1,
//                         both pheromone planes evaporated (Eq. 3); a pure
//                         16-byte-vector stream, the HBM-bound part of the step
//   agent_resolve_kernel  one thread per agent with a proposal: the claimants
//                         of its target cell are read back from the proposal
//                         plane (codes are valid exactly at cells occupied at
//                         t), the winner is drawn as in Sec. IV.d, and the
//                         winning agent moves: occupancy, id, position, tour
//                         and arrival, and its deposit (Eq. 4/5) on top of the
//                         evaporated value
//
// The proposal and streaming passes touch disjoint outputs and run together:
// the three kernels are chained by programmatic dependent launch in the
// order propose -> stream -> resolve.  The proposal pass waits for the
// previous step and then releases the streaming pass, which therefore starts
// on a complete state; the streaming pass waits for the proposal pass at its
// end, so that the resolution pass, which waits for the streaming pass,
// sees both.
#include "pedsim_internal.h"
#include "pedsim_rules.cuh"
#include "pedsim_ptx.cuh"

namespace pedsim {

constexpr int kStreamThreads = kCellBlock / 16;  // 16 cells per thread

// Scenario of work block b (prefix[i] = first block of scenario i).
__device__ __forceinline__ int block_scenario(const uint32_t *__restrict__ prefix, int n,
                                              uint32_t b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kAgentBlock)
agent_propose_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ agent_prefix,
                     int n_scen, int t_off)
{
    // The state at t is the previous step's output: wait for it, then let
    // the streaming pass of this step start.
    pdl_wait();
    pdl_trigger();
    const int s = block_scenario(agent_prefix, n_scen, blockIdx.x);
    const ScenarioDesc &d = descs[s];
    const uint64_t t = d.step + (uint64_t)t_off;
    const uint32_t a = (blockIdx.x - __ldg(agent_prefix + s)) * kAgentBlock + threadIdx.x;
    if (t >= d.end_step || a >= 2u * d.n_per_side) return;
    const uint32_t id = a + 1u;
    const int W = d.W, H = d.H;
    // read-only cached loads: this kernel writes none of the planes it reads
    const uint32_t cell = __ldg(d.pos + id);
    const int x = (int)(cell % (uint32_t)W), y = (int)(cell / (uint32_t)W);
    const int p = (int)(t & 1);
    const uint8_t *occ = d.occ[p];
    const int g = __ldg(occ + cell);
    const float *tp = d.tau[g == 2 ? 1 : 0][p];
    const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
    const int code = propose(
        x, y, g, W, H, (uint64_t)cell, t, d.seed, rp,
        [&](int dx, int dy) { return (int)__ldg(occ + ((int64_t)cell + (int64_t)dy * W + dx)); },
        tp ? tp + cell : nullptr, W);
    // the plane serves the neighbours' claim tests, the per-agent byte the
    // agent's own resolution
    d.prop[cell] = (uint8_t)code;
    d.acode[id] = (uint8_t)(code | (g << 4));
}

__global__ void __launch_bounds__(kStreamThreads)
stream_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ cell_prefix,
              int n_scen, int t_off)
{
    // Started by the proposal pass after the previous step completed.  Reads
    // bypass L1 (.cg), so no line cached before that point is used.
    const int s = block_scenario(cell_prefix, n_scen, blockIdx.x);
    const ScenarioDesc &d = descs[s];
    const uint64_t t = d.step + (uint64_t)t_off;
    if (t < d.end_step) {
        const size_t cells = (size_t)d.W * (size_t)d.H;
        const size_t c0 = (size_t)(blockIdx.x - __ldg(cell_prefix + s)) * kCellBlock;
        const int p = (int)(t & 1);
        const bool aco = d.model == 1;
        // occupancy: 16 cells per thread; pheromone: 4 float4 per plane and
        // thread, consecutive threads on consecutive vectors
        const size_t co = c0 + 16 * (size_t)threadIdx.x;
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (co < cells) o = __ldcg(reinterpret_cast<const uint4 *>(d.occ[p] + co));
        float4 va[4], vb[4];
        if (aco) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const size_t c = c0 + 4 * ((size_t)k * kStreamThreads + threadIdx.x);
                if (c < cells) {
                    va[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[0][p] + c));
                    vb[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[1][p] + c));
                }
            }
        }
        if (co < cells) *reinterpret_cast<uint4 *>(d.occ[p ^ 1] + co) = o;
        if (aco) {
            const float q = d.q;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const size_t c = c0 + 4 * ((size_t)k * kStreamThreads + threadIdx.x);
                if (c < cells) {
                    const float4 a4 = va[k], b4 = vb[k];
                    *reinterpret_cast<float4 *>(d.tau[0][p ^ 1] + c) =
                        make_float4(__fmul_rn(a4.x, q), __fmul_rn(a4.y, q), __fmul_rn(a4.z, q),
                                    __fmul_rn(a4.w, q));
                    *reinterpret_cast<float4 *>(d.tau[1][p ^ 1] + c) =
                        make_float4(__fmul_rn(b4.x, q), __fmul_rn(b4.y, q), __fmul_rn(b4.z, q),
                                    __fmul_rn(b4.w, q));
                }
            }
        }
    }
    // Complete only after the proposal pass has completed: the resolution
    // pass waits for this kernel and then reads the proposals.
    pdl_wait();
}

__global__ void __launch_bounds__(kAgentBlock)
agent_resolve_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ agent_prefix,
                     int n_scen, int t_off)
{
    pdl_wait();  // streaming pass and, through it, proposal pass complete
    pdl_trigger();
    const int s = block_scenario(agent_prefix, n_scen, blockIdx.x);
    const ScenarioDesc &d = descs[s];
    const uint64_t t = d.step + (uint64_t)t_off;
    const uint32_t blk = blockIdx.x - __ldg(agent_prefix + s);
    const uint32_t a = blk * kAgentBlock + threadIdx.x;
    Counts cnt;
    if (t < d.end_step && a < 2u * d.n_per_side) {
        // Two dependent rounds of loads: the agent's own entries, then its
        // target's neighbourhood (every load of a round is in flight at once).
        // Nothing read here is written by this kernel before it is read (the
        // position and per-agent entries only by their own thread, after
        // reading), so the loads take the read-only cached path.
        const uint32_t id = a + 1u;
        const uint32_t cell = __ldg(d.pos + id);
        const int ac = __ldg(d.acode + id);
        const bool aco = d.model == 1;
        const bool tour_mode = aco && d.deposit_mode == 1;
        const float tour0 = tour_mode ? __ldg(d.tour + id) : 0.0f;
        const uint32_t arrived = __ldg(d.arrival + id);
        const int code = ac & 15, g = ac >> 4;
        if (code) {
            const int W = d.W, H = d.H;
            const int p = (int)(t & 1);
            const uint8_t *occ = d.occ[p];
            const int x = (int)(cell % (uint32_t)W), y = (int)(cell / (uint32_t)W);
            const int dx = kCodeDX[code], dy = kCodeDY[code];
            const int tx = x + dx, ty = y + dy;
            const int64_t target = (int64_t)cell + (int64_t)dy * W + dx;
            // the evaporated value of the target, recomputed from t (the
            // streaming pass wrote the same value)
            const float tau_t = aco ? __ldg(d.tau[g == 2 ? 1 : 0][p] + target) : 0.0f;
            // Claim mask of the target: bit j when its neighbour at scan
            // offset j is occupied at t and chose the target (code 8 - j).
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ex = kCodeDX[j + 1], ey = kCodeDY[j + 1];
                const int nx = tx + ex, ny = ty + ey;
                if ((unsigned)nx >= (unsigned)W || (unsigned)ny >= (unsigned)H) continue;
                const int64_t nc = target + (int64_t)ey * W + ex;
                const int on = __ldg(occ + nc), pn = __ldg(d.prop + nc);
                if (on != 0 && pn == 8 - j) m |= 1u << j;
            }
            const uint32_t k = (uint32_t)__popc(m);
            const uint32_t mine = 8u - (uint32_t)code;  // this agent's scan offset
            const uint32_t win =
                k == 1 ? mine : pick_claimant(m, k, (uint64_t)target, t, d.seed);
            if (win == mine) {
                d.occ[p ^ 1][target] = (uint8_t)g;
                d.occ[p ^ 1][cell] = 0;
                d.pos[id] = (uint32_t)target;
                d.ids[target] = id;
                float dep = d.deposit;
                if (tour_mode) {
                    // Eq. 5: the tour length grows by the step length, then 1/L_k
                    const float L = __fadd_rn(tour0, (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
                    d.tour[id] = L;
                    dep = __fdiv_rn(1.0f, L);
                }
                const bool in_band = g == 1 ? tx >= W - (int)d.band : tx < (int)d.band;
                if (in_band && arrived == 0) {
                    d.arrival[id] = (uint32_t)(t + 1);
                    if (g == 1) ++cnt.crossed_a; else ++cnt.crossed_b;
                }
                if (aco)
                    d.tau[g == 2 ? 1 : 0][p ^ 1][target] = __fadd_rn(__fmul_rn(tau_t, d.q), dep);
                ++cnt.moved;
                if (k >= 2) ++cnt.conflicts;
            }
        }
    }
    flush_counts(d, cnt, blk % d.n_slots);
}

__global__ void build_pos_kernel(const ScenarioDesc *__restrict__ dp)
{
    const ScenarioDesc &d = *dp;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const uint8_t *occ = d.occ[d.step & 1];
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x)
        if (occ[c]) d.pos[d.ids[c]] = (uint32_t)c;
}

cudaError_t launch_agent_step(const ScenarioDesc *d_descs, const uint32_t *d_cell_prefix,
                              const uint32_t *d_agent_prefix, int n, uint32_t cell_blocks,
                              uint32_t agent_blocks, int t_off, cudaStream_t stream)
{
    if (n <= 0 || cell_blocks == 0) return cudaSuccess;
    // with no agent the proposal pass is one CTA that only orders the stream
    cudaError_t e = launch_pdl(agent_propose_kernel, agent_blocks ? agent_blocks : 1u,
                               (unsigned)kAgentBlock, stream, d_descs, d_agent_prefix, n, t_off);
    if (e != cudaSuccess) return e;
    e = launch_pdl(stream_kernel, cell_blocks, (unsigned)kStreamThreads, stream, d_descs,
                   d_cell_prefix, n, t_off);
    if (e != cudaSuccess || agent_blocks == 0) return e;
    return launch_pdl(agent_resolve_kernel, agent_blocks, (unsigned)kAgentBlock, stream, d_descs,
                      d_agent_prefix, n, t_off);
}

cudaError_t launch_build_pos(const ScenarioDesc *d_desc, int cells, cudaStream_t stream)
{
    int blocks = (cells + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    build_pos_kernel<<<blocks, 256, 0, stream>>>(d_desc);
    return cudaGetLastError();
}

}  // namespace pedsim
