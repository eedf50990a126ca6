// Agent-parallel step (PEDSIM_VARIANT_AGENT) of the pedestrian cellular
// automaton (sm_103a).  One synchronous step (Sec. IV.b-d) is split by
// access pattern instead of by tile, in two kernels:
//
//   agent_stage1_kernel   two CTA roles, the proposal blocks first:
//     proposal blocks     one thread per agent: forward first, else the full
//                         rule (Eq. 1 LEM rank draw, Eq. 2 ACO roulette) from
//                         the occupancy and pheromone at t; the direction code
//                         goes to the agent's entry of `acode`, and its claim
//                         bit (its scan offset seen from the target) is OR-ed
//                         into the target's byte of the step's claim plane
//     stream blocks       every cell: both pheromone planes evaporated into
//                         the planes of t+1 (Eq. 3); a pure 16-byte-vector
//                         stream, the HBM-bound part of the step (ACO only)
//   agent_resolve_kernel  one thread per agent with a proposal: the claim
//                         mask of its target cell (all its claimants' bits),
//                         the winner drawn from it as in Sec. IV.d, and the
//                         winning agent moves: occupancy, id, position, tour
//                         and arrival, and its deposit (Eq. 4/5) on top of the
//                         evaporated value; beside the agent CTAs, stream CTAs
//                         evaporate the step's last cell blocks (as many as
//                         fill one resident wave), skipping the claimed cells,
//                         whose winners write both planes
//
// Occupancy lives in one plane, occ[0], updated in place: the proposals read
// it (state at t) in the first kernel, the moves are applied to it only in
// the second, and no other cell changes.  The two roles of the first kernel
// write disjoint outputs, so the proposals run inside the stream instead of
// before it.  The resolution kernel is chained by
// programmatic dependent launch: the first kernel releases it as soon as all
// of its CTAs have started, so its CTAs are resident before the first kernel
// ends, and it waits for the first kernel's completion.  The last CTA of
// the resolution kernel advances the step index itself, so a step is two
// launches and a captured graph replays at any step.
#include <atomic>

#include "pedsim_internal.h"
#include "pedsim_rules.cuh"
#include "pedsim_ptx.cuh"


namespace pedsim {

constexpr int kMaxDevices = 64;  // devices whose occupancy is cached


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

// Proposal of agent index a (id a + 1) at step t.  The agent's code goes
// to its per-agent byte, and its claim bit (scan offset 8 - code seen from
// the target) is OR-ed into the target's byte of claim plane t & 1.  The
// agent also clears, in the other plane (written next at step t + 1), the
// byte of the target it claimed at step t - 1: that target is its cell now
// if it moved, else its cell plus its previous direction.
__device__ __forceinline__ void propose_agent(const ScenarioDesc &d, uint32_t a, uint64_t t)
{
    const uint32_t id = a + 1u;
    const int W = d.W, H = d.H;
    const uint32_t cell = __ldg(d.pos + id);
    const int prev = __ldg(d.acode + id);
    const int x = (int)(cell % (uint32_t)W), y = (int)(cell / (uint32_t)W);
    const int p = (int)(t & 1);
    const uint8_t *occ = d.occ[0];
    const int g = __ldg(occ + cell);
    const float *tp = d.tau[g == 2 ? 1 : 0][p];
    const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
    const int code = propose(
        x, y, g, W, H, (uint64_t)cell, t, d.seed, rp,
        [&](int dx, int dy) { return (int)__ldg(occ + ((int64_t)cell + (int64_t)dy * W + dx)); },
        tp ? tp + cell : nullptr, W);
    const int pc = prev & 15;
    if (pc) {
        const int64_t old_target =
            (prev & 0x80) ? (int64_t)cell : (int64_t)cell + (int64_t)kCodeDY[pc] * W + kCodeDX[pc];
        d.claim[p ^ 1][old_target] = 0;
    }
    if (code) {
        const int64_t target = (int64_t)cell + (int64_t)kCodeDY[code] * W + kCodeDX[code];
        uint8_t *cb = d.claim[p] + target;
        const uintptr_t addr = reinterpret_cast<uintptr_t>(cb);
        atomicOr(reinterpret_cast<unsigned int *>(addr & ~(uintptr_t)3),
                 (1u << (8 - code)) << (8 * (unsigned)(addr & 3)));
    }
    d.acode[id] = (uint8_t)(code | (g << 4));
}

// Evaporation of cell block b (kCellBlock cells) of the work list's
// pheromone.  Reads bypass L1 (.cg): the data is streamed once.
constexpr int kStreamVec = kCellBlock / 4 / kAgentBlock;  // float4 per plane and thread
static_assert(kStreamVec * 4 * kAgentBlock == kCellBlock, "cell block covers whole float4 per thread");

__device__ __forceinline__ void stream_block(const ScenarioDesc *__restrict__ descs,
                                             const uint32_t *__restrict__ cell_prefix, int n_scen,
                                             uint32_t b)
{
    const int s = block_scenario(cell_prefix, n_scen, b);
    const ScenarioDesc &d = descs[s];
    const uint64_t t = d.step;
    if (t >= d.end_step) return;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const size_t c0 = (size_t)(b - __ldg(cell_prefix + s)) * kCellBlock;
    const int p = (int)(t & 1);
    // kStreamVec float4 per plane and thread, consecutive threads on
    // consecutive vectors; every load of the block is in flight before the
    // first store
    float4 va[kStreamVec], vb[kStreamVec];
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        if (c < cells) {
            va[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[0][p] + c));
            vb[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[1][p] + c));
        }
    }
    const float q = d.q;
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
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


// Six resident CTAs per SM (40 registers, a few bytes of spill in the
// proposal path): more stream loads in flight than at the 48 registers the
// compiler picks by itself (5 CTAs per SM), measured 1-2 % faster at 2048^2.
__global__ void __launch_bounds__(kAgentBlock, 6)
agent_stage1_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ cell_prefix,
                    const uint32_t *__restrict__ agent_prefix, int n_scen, uint32_t cell_blocks,
                    uint32_t agent_blocks, uint32_t front)
{
    // The state at t is the previous step's output: wait for it, then let
    // the resolution kernel be scheduled (it waits for this one).
    pdl_wait();
    pdl_trigger();
    // (cell_blocks here counts the blocks this kernel streams: the first
    // ones; the resolution kernel evaporates the rest)
    // CTAs 0 .. front-1 are the first proposal blocks (at most one resident
    // wave): proposal CTAs (latency chains, longer in congestion) start at
    // once and end before the stream's tail, which measured faster than an
    // even spread when all proposals fit in that wave.  The remaining R
    // proposal blocks are spread evenly over the remaining T CTAs (CTA
    // front + j holds one where floor(j R / T) steps up), so that on large
    // grids the stream does not wait behind waves of proposals.
    const uint32_t i = blockIdx.x;
    uint32_t b = i;   // proposal block of this CTA, or agent_blocks
    uint32_t sb = 0;  // stream block of this CTA otherwise
    if (i >= front) {
        const uint32_t j = i - front;
        const uint32_t rest = agent_blocks - front;
        if (rest == 0) {
            b = agent_blocks;
            sb = j;
        } else {
            const uint32_t ctas = cell_blocks + rest;
            const uint64_t lo = (uint64_t)j * rest, hi = lo + rest;
            // 32-bit divisions whenever the products fit (all single grids
            // up to 2^31 cells), 64-bit ones otherwise
            const uint32_t before = hi >> 32 ? (uint32_t)(lo / ctas) : (uint32_t)lo / ctas;
            const uint32_t after = hi >> 32 ? (uint32_t)(hi / ctas) : (uint32_t)hi / ctas;
            if (after > before) {
                b = front + before;
            } else {
                b = agent_blocks;
                sb = j - before;
            }
        }
    }
    if (b >= agent_blocks) {
        stream_block(descs, cell_prefix, n_scen, sb);
    } else {
        const int s = block_scenario(agent_prefix, n_scen, b);
        const ScenarioDesc &d = descs[s];
        const uint64_t t = d.step;
        const uint32_t a = (b - __ldg(agent_prefix + s)) * kAgentBlock + threadIdx.x;
        if (t < d.end_step && a < 2u * d.n_per_side) propose_agent(d, a, t);
    }
}

// Evaporation of cell block b in the resolution kernel, where the claims of
// the step are final: the loads of the planes of t (which the first kernel
// does not write) are issued before the wait for the first kernel, the
// claim bytes after it, and claimed cells are left to their winners.
__device__ __forceinline__ void stream_block_claimed(const ScenarioDesc *__restrict__ descs,
                                                     const uint32_t *__restrict__ cell_prefix,
                                                     int n_scen, uint32_t b)
{
    const int s = block_scenario(cell_prefix, n_scen, b);
    const ScenarioDesc &d = descs[s];
    const uint64_t t = d.step;
    const bool active = t < d.end_step;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const size_t c0 = (size_t)(b - __ldg(cell_prefix + s)) * kCellBlock;
    const int p = (int)(t & 1);
    float4 va[kStreamVec], vb[kStreamVec];
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        if (active && c < cells) {
            va[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[0][p] + c));
            vb[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[1][p] + c));
        }
    }
    pdl_wait();  // the claims of the step are in
    pdl_trigger();
    if (!active) return;
    uint32_t cw[kStreamVec];
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        cw[k] = c < cells ? __ldcg(reinterpret_cast<const unsigned int *>(d.claim[p] + c)) : 0u;
    }
    const float q = d.q;
    float *const na = d.tau[0][p ^ 1], *const nb = d.tau[1][p ^ 1];
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        if (c >= cells) continue;
        const float a_[4] = {va[k].x, va[k].y, va[k].z, va[k].w};
        const float b_[4] = {vb[k].x, vb[k].y, vb[k].z, vb[k].w};
        if (cw[k] == 0u) {
            *reinterpret_cast<float4 *>(na + c) =
                make_float4(__fmul_rn(a_[0], q), __fmul_rn(a_[1], q), __fmul_rn(a_[2], q),
                            __fmul_rn(a_[3], q));
            *reinterpret_cast<float4 *>(nb + c) =
                make_float4(__fmul_rn(b_[0], q), __fmul_rn(b_[1], q), __fmul_rn(b_[2], q),
                            __fmul_rn(b_[3], q));
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((cw[k] >> (8 * j)) & 0xffu) continue;  // the winner stores this cell
                na[c + j] = __fmul_rn(a_[j], q);
                nb[c + j] = __fmul_rn(b_[j], q);
            }
        }
    }
}

// Resolution work of one agent: its own entries (position, tour and arrival
// before the wait for the first kernel, its code after it) and its target's
// claim mask and pheromone (a second round).  Nothing read here is written
// by the resolution kernel before it is read (position and per-agent entries
// only by their own thread, after reading), and the rounds of several agents
// overlap.
struct Resolve {
    uint32_t id, cell;
    int code, g;
    float tour0;
    uint32_t arrived;
    int64_t target;
    uint32_t mask;
    float tau_t;  // own group's pheromone at the target, at t
    float tau_o;  // the other group's (targets in cell blocks evaporated late)
    bool late;    // the target's cell block is evaporated in the resolution kernel
};

// The agent's entries the first kernel does not write (written by the
// previous step's resolution, complete before the first kernel began):
// loaded before the wait for the first kernel.
__device__ __forceinline__ void resolve_load_own(const ScenarioDesc &d, uint32_t a, Resolve &r)
{
    r.id = a + 1u;
    r.cell = __ldcg(d.pos + r.id);
    r.tour0 = (d.model == 1 && d.deposit_mode == 1) ? __ldcg(d.tour + r.id) : 0.0f;
    r.arrived = __ldcg(d.arrival + r.id);
}

// This step's proposal code and the agent's group (first kernel's output).
__device__ __forceinline__ void resolve_load_code(const ScenarioDesc &d, Resolve &r)
{
    const int ac = __ldcg(d.acode + r.id);
    r.code = ac & 15;
    r.g = ac >> 4;
}

// Claim mask of the target (bit j: its claimant at scan offset j; every
// claimant's proposal pass has OR-ed its bit in) and the target's own-group
// pheromone at t.
// late_from: the scenario's first cell block evaporated in the resolution
// kernel (its cell blocks from there on skip claimed cells).
__device__ __forceinline__ void resolve_load_target(const ScenarioDesc &d, uint64_t t, Resolve &r,
                                                    uint32_t late_from)
{
    const int W = d.W;
    const int p = (int)(t & 1);
    r.target = (int64_t)r.cell + (int64_t)kCodeDY[r.code] * W + kCodeDX[r.code];
    r.late = (uint64_t)r.target / kCellBlock >= late_from;
    r.tau_t = d.model == 1 ? __ldg(d.tau[r.g == 2 ? 1 : 0][p] + r.target) : 0.0f;
    r.tau_o = d.model == 1 && r.late ? __ldg(d.tau[r.g == 2 ? 0 : 1][p] + r.target) : 0.0f;
    r.mask = __ldg(d.claim[p] + r.target);
}

// The winner of the target (Sec. IV.d) and, if it is this agent, its move.
__device__ __forceinline__ void resolve_apply(const ScenarioDesc &d, uint64_t t, const Resolve &r,
                                              Counts &cnt)
{
    const uint32_t k = (uint32_t)__popc(r.mask);
    const uint32_t mine = 8u - (uint32_t)r.code;  // this agent's scan offset
    const uint32_t win = k == 1 ? mine : pick_claimant(r.mask, k, (uint64_t)r.target, t, d.seed);
    if (win != mine) return;
    const int W = d.W;
    const int p = (int)(t & 1);
    const int g = r.g;
    const int dx = kCodeDX[r.code], dy = kCodeDY[r.code];
    const int tx = (int)(r.cell % (uint32_t)W) + dx;
    d.occ[0][r.target] = (uint8_t)g;
    d.occ[0][r.cell] = 0;
    d.pos[r.id] = (uint32_t)r.target;
    d.acode[r.id] = (uint8_t)(r.code | (g << 4) | 0x80);
    d.ids[r.target] = r.id;
    float dep = d.deposit;
    if (d.model == 1 && d.deposit_mode == 1) {
        // Eq. 5: the tour length grows by the step length, then 1/L_k
        const float L = __fadd_rn(r.tour0, (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
        d.tour[r.id] = L;
        dep = __fdiv_rn(1.0f, L);
    }
    const bool in_band = g == 1 ? tx >= W - (int)d.band : tx < (int)d.band;
    if (in_band && r.arrived == 0) {
        d.arrival[r.id] = (uint32_t)(t + 1);
        if (g == 1) ++cnt.crossed_a; else ++cnt.crossed_b;
    }
    // the own group's evaporated value plus the deposit; in a cell block
    // evaporated in the resolution kernel (which skips claimed cells) also
    // the other group's evaporated value
    if (d.model == 1) {
        d.tau[g == 2 ? 1 : 0][p ^ 1][r.target] = __fadd_rn(__fmul_rn(r.tau_t, d.q), dep);
        if (r.late) d.tau[g == 2 ? 0 : 1][p ^ 1][r.target] = __fmul_rn(r.tau_o, d.q);
    }
    ++cnt.moved;
    if (k >= 2) ++cnt.conflicts;
}

// Each CTA resolves kResolveBlocks consecutive agent blocks, one agent of
// each per thread, with the loads of all of them in flight together (1: 2
// and 4 were measured slower at 2048^2 and 8192^2).
constexpr int kResolveBlocks = 1;  // the resolution kernel's CTA indices assume 1

__global__ void __launch_bounds__(kAgentBlock)
agent_resolve_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ agent_prefix,
                     const uint32_t *__restrict__ cell_prefix, int n_scen, uint32_t agent_blocks,
                     uint32_t first_late, uint32_t late_blocks, ActivityCtl *__restrict__ ctl)
{
    if (blockIdx.x >= agent_blocks) {
        // CTAs past the agent blocks evaporate cell blocks first_late .. ;
        // every CTA takes a ticket once its threads hold the step index
        const uint32_t b = first_late + (blockIdx.x - agent_blocks);
        if (b < first_late + late_blocks) stream_block_claimed(descs, cell_prefix, n_scen, b);
        else {
            pdl_wait();
            pdl_trigger();
        }
        __syncthreads();
        unsigned int ticket = 0;
        if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket, 1u);
        if (threadIdx.x < 32) {
            const bool last = __shfl_sync(0xffffffffu, ticket == gridDim.x - 1, 0);
            if (last) {
                ScenarioDesc *md = const_cast<ScenarioDesc *>(descs);
                for (int i = threadIdx.x; i < n_scen; i += 32) {
                    const unsigned long long v = md[i].step;
                    if (v < md[i].end_step) md[i].step = v + 1;
                }
                if (threadIdx.x == 0) ctl->ticket = 0u;
            }
        }
        return;
    }
    const ScenarioDesc *dq[kResolveBlocks];
    uint32_t lb[kResolveBlocks];
    uint64_t tq[kResolveBlocks];
    uint32_t late_from[kResolveBlocks];
    bool live[kResolveBlocks];
    Resolve r[kResolveBlocks];
#pragma unroll
    for (int q = 0; q < kResolveBlocks; ++q) {
        const uint32_t b = blockIdx.x * kResolveBlocks + q;
        live[q] = false;
        dq[q] = descs;
        lb[q] = 0;
        tq[q] = 0;
        late_from[q] = 0;
        if (b >= agent_blocks) continue;
        const int s = block_scenario(agent_prefix, n_scen, b);
        dq[q] = descs + s;
        lb[q] = b - __ldg(agent_prefix + s);
        tq[q] = dq[q]->step;
        const uint32_t cp = __ldg(cell_prefix + s);
        late_from[q] = first_late > cp ? first_late - cp : 0u;
        const uint32_t a = lb[q] * kAgentBlock + threadIdx.x;
        live[q] = tq[q] < dq[q]->end_step && a < 2u * dq[q]->n_per_side;
        if (live[q]) resolve_load_own(*dq[q], a, r[q]);
    }
    pdl_wait();  // first kernel (proposals and stream) complete
    pdl_trigger();
#pragma unroll
    for (int q = 0; q < kResolveBlocks; ++q) {
        if (live[q]) resolve_load_code(*dq[q], r[q]);
        if (live[q] && r[q].code == 0) live[q] = false;
    }
    // Every thread of the CTA has read its step index: the CTA takes its
    // ticket now (the reply is needed only at the end).  The CTA holding the
    // last ticket advances the step index of every scenario of the work list
    // (clamped at its end) after its own work: by then every CTA has read it.
    __syncthreads();
    unsigned int ticket = 0;
    if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket, 1u);
#pragma unroll
    for (int q = 0; q < kResolveBlocks; ++q)
        if (live[q]) resolve_load_target(*dq[q], tq[q], r[q], late_from[q]);
#pragma unroll
    for (int q = 0; q < kResolveBlocks; ++q) {
        Counts cnt;
        if (live[q]) resolve_apply(*dq[q], tq[q], r[q], cnt);
        if (blockIdx.x * kResolveBlocks + q < agent_blocks)
            flush_counts(*dq[q], cnt, lb[q] % dq[q]->n_slots);
    }
    if (threadIdx.x < 32) {
        const bool last = __shfl_sync(0xffffffffu, ticket == gridDim.x - 1, 0);
        if (last) {
            ScenarioDesc *md = const_cast<ScenarioDesc *>(descs);
            for (int i = threadIdx.x; i < n_scen; i += 32) {
                const unsigned long long v = md[i].step;
                if (v < md[i].end_step) md[i].step = v + 1;
            }
            if (threadIdx.x == 0) ctl->ticket = 0u;
        }
    }
}


__global__ void build_pos_kernel(const ScenarioDesc *__restrict__ dp, int plane)
{
    const ScenarioDesc &d = *dp;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const uint8_t *occ = d.occ[plane];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
        d.claim[0][c] = 0;
        d.claim[1][c] = 0;
        if (occ[c]) d.pos[d.ids[c]] = (uint32_t)c;
    }
    const size_t agents = 2 * (size_t)d.n_per_side + 1;
    for (size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x; a < agents; a += stride)
        d.acode[a] = 0;
}

// Resident CTAs of one wave of a kernel on the current device (occupancy
// queried once per device and kernel; the queries also run when a scenario
// is placed or loaded, so that no first query falls inside a caller's
// stream capture).
template <class Kernel>
static uint32_t resident_wave(Kernel kernel, std::atomic<uint32_t> (&cache)[kMaxDevices])
{
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t wave = (unsigned)dev < (unsigned)kMaxDevices ? cache[dev].load() : 0u;
    if (!wave) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kAgentBlock, 0);
        wave = (uint32_t)(sms > 0 ? sms : 1) * (uint32_t)(per_sm > 0 ? per_sm : 1);
        if ((unsigned)dev < (unsigned)kMaxDevices) cache[dev].store(wave);
    }
    return wave;
}

static uint32_t stage1_wave()
{
    static std::atomic<uint32_t> cache[kMaxDevices];
    return resident_wave(agent_stage1_kernel, cache);
}

static uint32_t resolve_wave()
{
    static std::atomic<uint32_t> cache[kMaxDevices];
    return resident_wave(agent_resolve_kernel, cache);
}

// Cell blocks of a step evaporated in the resolution kernel: the free part
// of one resident wave of that kernel, at most all but one cell block (the
// first kernel must run whenever there are cell blocks: the resolution
// kernel's loads before its wait rely on the first kernel having waited for
// the previous step).
static uint32_t resolve_late_blocks(uint32_t cell_blocks, uint32_t agent_blocks)
{
    const uint32_t wave = resolve_wave();
    if (cell_blocks == 0 || agent_blocks >= wave) return 0;
    const uint32_t free = wave - agent_blocks;
    return free < cell_blocks - 1 ? free : cell_blocks - 1;
}

cudaError_t launch_agent_step(const ScenarioDesc *d_descs, const uint32_t *d_cell_prefix,
                              const uint32_t *d_agent_prefix, int n, uint32_t cell_blocks,
                              uint32_t agent_blocks, ActivityCtl *ctl, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    // Cell blocks evaporated in the resolution kernel (the claims are final
    // there, so they skip claimed cells): as many as fill that kernel up to
    // one resident wave beside its agent CTAs, which alone leave most of the
    // GPU idle at a few hundred CTAs, and never all of them (the first
    // kernel keeps at least one, see resolve_late_blocks).
    const uint32_t late = resolve_late_blocks(cell_blocks, agent_blocks);
    if (cell_blocks + agent_blocks) {
        const uint32_t wave = stage1_wave();
        const uint32_t front = agent_blocks < wave ? agent_blocks : wave;
        const uint32_t c1 = cell_blocks - late;
        if (c1 + agent_blocks) {
            cudaError_t e = launch_pdl(agent_stage1_kernel, c1 + agent_blocks,
                                       (unsigned)kAgentBlock, stream, d_descs, d_cell_prefix,
                                       d_agent_prefix, n, c1, agent_blocks, front);
            if (e != cudaSuccess) return e;
        }
    }
    // the resolution kernel also evaporates the last `late` cell blocks and
    // advances the step index: with no agent and no such block it is one CTA
    // that does only that
    const uint32_t g = agent_blocks + late > 0 ? agent_blocks + late : 1u;
    return launch_pdl(agent_resolve_kernel, g, (unsigned)kAgentBlock, stream, d_descs,
                      d_agent_prefix, d_cell_prefix, n, agent_blocks, cell_blocks - late, late,
                      ctl);
}

cudaError_t launch_build_pos(const ScenarioDesc *d_desc, int cells, int plane, cudaStream_t stream)
{
    (void)stage1_wave();  // the step's occupancy queries, outside any capture
    (void)resolve_wave();
    int blocks = (cells + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    build_pos_kernel<<<blocks, 256, 0, stream>>>(d_desc, plane);
    return cudaGetLastError();
}

}  // namespace pedsim
