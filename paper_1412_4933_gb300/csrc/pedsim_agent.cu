// Agent-parallel step (PEDSIM_VARIANT_AGENT) of the pedestrian cellular
// automaton (sm_103a), and its deferred-evaporation form
// (PEDSIM_VARIANT_DEFERRED).  One synchronous step (Sec. IV.b-d) is split by
// access pattern instead of by tile, in two kernels:
//
//   agent_stage1_kernel   two CTA roles, the proposal blocks first:
//     proposal blocks     one thread per agent: forward first, else the full
//                         rule (Eq. 1 LEM rank draw, Eq. 2 ACO roulette) from
//                         the occupancy and pheromone at t, the blocked agents
//                         compacted into full warps; the direction code goes
//                         to the agent's entry of `acode` and to its own cell
//                         of the step's code plane, a claimed flag to its
//                         target's byte
//     stream blocks       every cell: both pheromone planes evaporated into
//                         the planes of t+1 (Eq. 3); a pure 16-byte-vector
//                         stream, the HBM-bound part of the step (ACO only)
//   agent_resolve_kernel  one thread per agent with a proposal: the claim
//                         mask of its target cell gathered from the codes of
//                         the target's eight neighbours (Sec. IV.d: scatter
//                         turned into gather, no atomics), the winner drawn
//                         from it, and the winning agent moves: occupancy,
//                         id, position, tour and arrival, and its deposit
//                         (Eq. 4/5) on top of the evaporated value; beside the
//                         agent CTAs, stream CTAs evaporate the step's last
//                         cell blocks (as many as fill one resident wave),
//                         skipping the claimed cells (from the flags), whose
//                         winners write both planes
//
//   deferred_stage1_kernel / deferred_resolve_kernel
//                         the same without the stream: one pheromone plane per
//                         group updated in place and a per-cell stamp; values
//                         are brought up to date where they are read and in a
//                         rolling refresh of 1/kDeferPeriod of the cell blocks
//                         per step (bit-identical to evaporating every cell)
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
constexpr uint8_t kClaimed = 0x80;  // code-plane byte of an empty cell some agent proposed


// Row of cell c (< 2^31) of scenario d without a divide (see ScenarioDesc).
__device__ __forceinline__ uint32_t cell_row(const ScenarioDesc &d, uint32_t c)
{
    return __umulhi(c, d.w_mul) >> d.w_shr;
}

// Scenario of work block b (prefix[i] = first block of scenario i, non-
// decreasing, prefix[0] = 0): the largest i < n with prefix[i] <= b.  A
// 32-way search by the whole warp (b is the same in every lane): each round
// the lanes test 32 evenly spaced entries at once, so 256 scenarios take two
// rounds of loads instead of eight dependent ones.  Every lane of the warp
// must call it.
__device__ __forceinline__ int block_scenario(const uint32_t *__restrict__ prefix, int n,
                                              uint32_t b)
{
    const int lane = (int)(threadIdx.x & 31u);
    int lo = 0, hi = n;  // the answer lies in [lo, hi)
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + lane * step;
        const bool ok = idx < hi && __ldg(prefix + idx) <= b;
        const unsigned m = __ballot_sync(0xffffffffu, ok);  // lane 0 (idx = lo) always holds
        lo += (31 - __clz((int)m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Brings the fetched values of the available frame neighbours (tv[i], with
// stamps aux[i]) up to step `now`: fl(v * q) once per missed step, the
// neighbours' evaporation chains interleaved.
__device__ __forceinline__ void catch_up_frame(float (&tv)[9], const uint32_t (&aux)[9],
                                               unsigned avail, uint32_t now, float q)
{
    uint32_t age[9], most = 0;
#pragma unroll
    for (int i = 2; i <= 8; ++i) {
        age[i] = (avail & (1u << i)) ? (now - aux[i]) & 255u : 0u;
        most = age[i] > most ? age[i] : most;
    }
    for (uint32_t k = 0; k < most; ++k) {
#pragma unroll
        for (int i = 2; i <= 8; ++i)
            if (k < age[i]) tv[i] = __fmul_rn(tv[i], q);
    }
}

// Own-group pheromone of a blocked agent's neighbours, loaded together with
// its occupancy before it was known whether the forward cell is free (the
// blocked agents then skip a dependent round of loads): v[i] and, for the
// deferred step, stamp[i] of frame neighbour i (zero outside the grid).
struct PrefetchedTau {
    const float *v;
    const uint8_t *stamp;  // nullptr: the values are current
    uint32_t now;
    float q;
    __device__ __forceinline__ float fetch(int i, int, uint32_t &aux) const
    {
        aux = stamp ? stamp[i] : 0u;
        return v[i];
    }
    __device__ __forceinline__ void finish(float (&tv)[9], const uint32_t (&aux)[9],
                                           unsigned avail) const
    {
        if (stamp) catch_up_frame(tv, aux, avail, now, q);
    }
};

// The same read from the planes once the agent is known to be blocked: c and
// sc point at the agent's own cell of its group's plane and of the stamps
// (nullptr: the values are current).
struct GlobalTau {
    const float *c;
    const uint8_t *sc;
    int stride;
    uint32_t now;
    float q;
    __device__ __forceinline__ float fetch(int, int code, uint32_t &aux) const
    {
        const int off = kCodeDY[code] * stride + kCodeDX[code];
        aux = sc ? __ldg(sc + off) : 0u;
        return __ldg(c + off);
    }
    __device__ __forceinline__ void finish(float (&tv)[9], const uint32_t (&aux)[9],
                                           unsigned avail) const
    {
        if (sc) catch_up_frame(tv, aux, avail, now, q);
    }
};

// Loads issued where they stand (the compiler may not sink them into the
// blocked agents' branch, which would cost that branch a round trip).
__device__ __forceinline__ float ld_nc_f32(const float *p)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_nc_u8(const uint8_t *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// A forward-blocked agent waiting for the full rule (Eq. 1 / Eq. 2): its
// prefetched pheromone and stamps, cell, id and frame state.
struct BlockedAgent {
    float v[9];
    uint8_t stamp[12];
    uint32_t cell, id;
    uint32_t avail, g;
};

// Proposals of agent block lb (kAgentBlock agents, one per thread; every
// thread of the CTA calls this) at step t.  The agent's group is known from
// its per-agent byte (kept there from placement on), so its own-group
// pheromone around it (with the stamps, for the deferred step) is loaded in
// the same round as the occupancy.  Forward first (Sec. III) decides most
// agents at once; the blocked ones are compacted into a shared list (warp
// ballots and a scan over the CTA's warps) and take the full rule one per
// thread, so its heavy path (a Philox block, the roulette) runs in as few
// full warps as there are blocked agents instead of in every warp that has
// one.
//
// Code plane t & 1 after the proposals of step t: at every occupied cell its
// agent's direction code (0 = stay), kClaimed at every empty cell some agent
// proposed, 0 elsewhere.  (A cell is never both occupied and proposed at one
// step, so one byte holds either.)  The resolution gathers a target's
// claimants from its neighbours' codes; the claimed flags only let the
// streams skip the cells the winners write.  Every proposer of a cell writes
// the same flag with a plain store.  Keeping the plane clean: an agent
// overwrites its own cell every step; a winner clears its old cell in the
// plane of the next step (in the resolution, where no one reads that plane)
// and, at the next step's proposals, in the plane of the step it moved in
// (no one writes that plane then); a claimed cell always receives its
// winner, whose later overwrite or clear removes the flag.
//
// prefetch (a launch-wide choice): load every agent's neighbour pheromone
// with its occupancy, which shortens the blocked agents' chain of dependent
// loads when the launch's agents fit in one resident wave (latency-bound);
// without it only the blocked agents load theirs, in the compacted pass,
// which spends far fewer loads when a launch carries millions of agents
// (throughput-bound).
template <bool Deferred>
__device__ __forceinline__ void propose_block(const ScenarioDesc &d, uint32_t lb, uint64_t t,
                                              bool prefetch)
{
    __shared__ BlockedAgent blocked[kAgentBlock];
    __shared__ uint32_t warp_base[kAgentBlock / 32 + 1];
    const uint32_t a = lb * kAgentBlock + threadIdx.x;
    // the position and per-agent byte are loaded whatever the step index, so
    // that they share a round of loads with it (the callers read it from L2
    // after their wait)
    const bool in = a < 2u * d.n_per_side;
    uint32_t cell0 = 0, prev0 = 0;
    if (in) {
        cell0 = __ldg(d.pos + a + 1u);
        prev0 = __ldg(d.acode + a + 1u);
    }
    const bool live = in && t < d.end_step;
    const int W = d.W, H = d.H;
    const int p = (int)(t & 1);
    bool is_blocked = false;
    uint32_t id = 0, cell = 0, avail = 0;
    int g = 1;
    float pre[9];
    uint32_t pst[9];
    if (live) {
        id = a + 1u;
        cell = cell0;
        const int prev = (int)prev0;
        g = prev >> 4 & 3;
        const uint32_t yr = cell_row(d, cell);
        const int x = (int)(cell - yr * (uint32_t)W), y = (int)yr;
        const uint8_t *occ = d.occ[0];
        const float *tp = d.tau[g == 2 ? 1 : 0][Deferred ? 0 : p];
        const int side = g - 1;
        if (tp && prefetch) {
#pragma unroll
            for (int i = 1; i <= 8; ++i) {
                const int code = kFrameCode[side][i];
                const int nx = x + kCodeDX[code], ny = y + kCodeDY[code];
                const bool inside = (unsigned)nx < (unsigned)W && (unsigned)ny < (unsigned)H;
                const int64_t off = (int64_t)cell + (int64_t)kCodeDY[code] * W + kCodeDX[code];
                pre[i] = inside ? ld_nc_f32(tp + off) : 0.0f;
                pst[i] = Deferred && inside ? ld_nc_u8(d.stamp + off) : 0u;
            }
        }
        int code = 0;
        if (!parked(x, g, W)) {
            avail = frame_avail(x, y, g, W, H, [&](int dx, int dy) {
                return (int)__ldg(occ + ((int64_t)cell + (int64_t)dy * W + dx));
            });
            if (avail & 2u) code = kFrameCode[side][1];
            else is_blocked = true;
        }
        if (prev & 0x80) {
            const int pc = prev & 15;
            const int64_t old_cell = (int64_t)cell - ((int64_t)kCodeDY[pc] * W + kCodeDX[pc]);
            d.codes[p ^ 1][old_cell] = 0;  // its code of t - 1 there
        }
        if (!is_blocked) {
            d.codes[p][cell] = (uint8_t)code;
            if (code) d.codes[p][(int64_t)cell + (int64_t)kCodeDY[code] * W + kCodeDX[code]] = kClaimed;
            d.acode[id] = (uint8_t)(code | (g << 4));
        }
    }
    // compaction of the blocked agents: each warp's count, then every thread
    // sums the counts of the warps before its own (its warp's offset) and of
    // all warps (the list's length) -- independent shared-memory reads
    // instead of a serial scan and a second barrier
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned ballot = __ballot_sync(0xffffffffu, is_blocked);
    if (lane == 0) warp_base[warp] = (uint32_t)__popc(ballot);
    __syncthreads();
    uint32_t base = 0, nb = 0;
#pragma unroll
    for (unsigned w = 0; w < kAgentBlock / 32; ++w) {
        const uint32_t c = warp_base[w];
        base += w < warp ? c : 0u;
        nb += c;
    }
    if (is_blocked) {
        BlockedAgent &e = blocked[base + __popc(ballot & ((1u << lane) - 1u))];
        if (d.tau[0][0] && prefetch) {
#pragma unroll
            for (int i = 1; i <= 8; ++i) {
                e.v[i] = pre[i];
                if (Deferred) e.stamp[i] = (uint8_t)pst[i];
            }
        }
        e.cell = cell;
        e.id = id;
        e.avail = avail;
        e.g = (uint32_t)g;
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        const BlockedAgent &e = blocked[threadIdx.x];
        const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
        int code;
        if (prefetch || !d.tau[0][0]) {
            code = choose_blocked(e.avail, (int)e.g - 1,
                                  PrefetchedTau{e.v, Deferred ? e.stamp : nullptr, (uint32_t)t, d.q},
                                  (uint64_t)e.cell, t, d.seed, rp);
        } else {
            const float *tp = d.tau[e.g == 2 ? 1 : 0][Deferred ? 0 : p] + e.cell;
            code = choose_blocked(e.avail, (int)e.g - 1,
                                  GlobalTau{tp, Deferred ? d.stamp + e.cell : nullptr, W,
                                            (uint32_t)t, d.q},
                                  (uint64_t)e.cell, t, d.seed, rp);
        }
        d.codes[p][e.cell] = (uint8_t)code;
        if (code) d.codes[p][(int64_t)e.cell + (int64_t)kCodeDY[code] * W + kCodeDX[code]] = kClaimed;
        d.acode[e.id] = (uint8_t)(code | (e.g << 4));
    }
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
                    uint32_t agent_blocks, uint32_t front, int prefetch)
{
    __shared__ __align__(128) ScenarioDesc hdr;  // header part only (proposal CTAs)
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
    // The state at t is the previous step's output: each CTA waits for it,
    // then lets the resolution kernel be scheduled (it waits for this one).
    if (b >= agent_blocks) {
        pdl_wait();
        pdl_trigger();
        stream_block(descs, cell_prefix, n_scen, sb);
    } else {
        // A proposal CTA copies its scenario's descriptor header (constant
        // during the step but for the step index) before the wait; after
        // it, the step index (from L2: the previous step's resolution
        // advanced it) is read in one round with the agents' positions.
        const int s = block_scenario(agent_prefix, n_scen, b);
        const uint32_t lb = b - __ldg(agent_prefix + s);
        load_header(&hdr, descs + s);
        pdl_wait();
        pdl_trigger();
        __syncthreads();
        propose_block<false>(hdr, lb, __ldcg(&descs[s].step), prefetch != 0);
    }
}

// Evaporation of cell block b in the resolution kernel, where the proposals
// of the step are final: the loads of the planes of t (which the first
// kernel does not write) are issued before the wait for the first kernel,
// the neighbours' codes after it, and claimed cells are left to their
// winners.
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
    pdl_wait();  // the proposals of the step are in
    pdl_trigger();
    if (!active) return;
    uint32_t cw[kStreamVec];  // claimed flags of the thread's cells
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        cw[k] = c < cells
                    ? __ldcg(reinterpret_cast<const unsigned int *>(d.codes[p] + c)) & 0x80808080u
                    : 0u;
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
// neighbours' codes and pheromone (a second round).  Nothing read here is written
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

// Claim mask of target cell (tx, ty) (linear index target), gathered from
// its eight neighbours' codes in the step's code plane (bit j: the
// neighbour at scan offset j proposed the target, i.e. holds code 8 - j; no
// atomics, Sec. IV.d).  Each of the three rows is read with one or two
// aligned 8-byte loads (the plane holds a multiple of 256 cells, so an
// aligned word inside it never ends past it).
__device__ __forceinline__ uint32_t gather_claims(const uint8_t *__restrict__ codes, int W, int H,
                                                  int64_t target, int tx, int ty)
{
    const int64_t cells = (int64_t)W * H;
    const unsigned long long *w = reinterpret_cast<const unsigned long long *>(codes);
    // edge masks: no left neighbour in column 0, no right one in column W-1
    const uint32_t keep = (tx > 0 ? 0x0000FFu : 0u) | 0x00FF00u | (tx + 1 < W ? 0xFF0000u : 0u);
    uint32_t m = 0;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
        if ((unsigned)(ty + oy) >= (unsigned)H) continue;
        const int64_t base = target + (int64_t)oy * W - 1;  // cell (tx - 1, ty + oy)
        const int64_t lo = (base < 0 ? 0 : base) & ~(int64_t)7;
        const int off = (int)(base - lo);  // -1 only for tx = 0 in row 0
        const unsigned long long w0 = __ldg(w + lo / 8);
        const unsigned long long w1 = off > 5 && lo + 8 < cells ? __ldg(w + lo / 8 + 1) : 0ull;
        // bytes 0, 1, 2 of v: the left, middle and right cell of the row
        const unsigned long long v =
            off < 0 ? w0 << 8 : off == 0 ? w0 : (w0 >> (8 * off)) | (w1 << (64 - 8 * off));
        // codes of the moves into the target from the row's left, middle and
        // right cell (the target itself, in the middle of its own row, can
        // hold no code: 0xFF never matches)
        const uint32_t pat = oy < 0 ? 0x00060708u : oy == 0 ? 0x0004FF05u : 0x00010203u;
        const uint32_t eq = __vcmpeq4((uint32_t)v & keep & 0x00FFFFFFu, pat) & 0x00010101u;
        const uint32_t bits = (eq & 1u) | ((eq >> 7) & 2u) | ((eq >> 14) & 4u);
        m |= oy < 0 ? bits : oy == 0 ? ((bits & 1u) << 3) | ((bits & 4u) << 2) : bits << 5;
    }
    return m;
}

// The target's claim mask and its own-group pheromone at t.
// late_from: the scenario's first cell block evaporated in the resolution
// kernel (its cell blocks from there on skip claimed cells).
__device__ __forceinline__ void resolve_load_target(const ScenarioDesc &d, uint64_t t, Resolve &r,
                                                    uint32_t late_from)
{
    const int W = d.W, H = d.H;
    const int p = (int)(t & 1);
    const int dx = kCodeDX[r.code], dy = kCodeDY[r.code];
    r.target = (int64_t)r.cell + (int64_t)dy * W + dx;
    const uint32_t yr = cell_row(d, r.cell);
    const int tx = (int)(r.cell - yr * (uint32_t)W) + dx, ty = (int)yr + dy;
    r.late = (uint64_t)r.target / kCellBlock >= late_from;
    r.tau_t = d.model == 1 ? __ldg(d.tau[r.g == 2 ? 1 : 0][p] + r.target) : 0.0f;
    r.tau_o = d.model == 1 && r.late ? __ldg(d.tau[r.g == 2 ? 0 : 1][p] + r.target) : 0.0f;
    r.mask = gather_claims(d.codes[p], W, H, r.target, tx, ty);
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
    const int tx = (int)(r.cell - cell_row(d, r.cell) * (uint32_t)W) + dx;
    d.occ[0][r.target] = (uint8_t)g;
    d.occ[0][r.cell] = 0;
    d.codes[p ^ 1][r.cell] = 0;  // its old cell, in the plane of step t + 1
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

// Five resident CTAs per SM (48 registers): the gathered claim mask alone
// would take the compiler to 54 registers and four CTAs per SM, a smaller
// resident wave for the late cell blocks.
__global__ void __launch_bounds__(kAgentBlock, 5)
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
    // Every thread of the CTA has read its step index: the CTA takes its
    // ticket now, before the wait (the reply is needed only at the end).  The
    // CTA holding the last ticket advances the step index of every scenario
    // of the work list (clamped at its end) after its own work: by then
    // every CTA has read it.
    __syncthreads();
    unsigned int ticket = 0;
    if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket, 1u);
    pdl_wait();  // first kernel (proposals and stream) complete
    pdl_trigger();
#pragma unroll
    for (int q = 0; q < kResolveBlocks; ++q) {
        if (live[q]) resolve_load_code(*dq[q], r[q]);
        if (live[q] && r[q].code == 0) live[q] = false;
    }
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


// ---------------------------------------------------------------------------
// Deferred evaporation (PEDSIM_VARIANT_DEFERRED): the same agent-parallel
// step without the dense stream.  Each scenario keeps one pheromone plane per
// group, updated in place, and one byte per cell, the stamp: the low byte of
// the step at which the cell's two stored values are valid.  The value at a
// later step t is the stored value evaporated once per missed step, i.e.
// fl(v * q) applied (t - stamp) mod 256 times -- the very operations Eq. 3
// performs on the cell, in the same order -- so every value read, deposited
// on or copied out equals the every-step evaporation bit for bit.  A value
// is brought up to date only where it is read (the blocked agents' available
// neighbours, each winner's target) and, so that no value is ever more than
// kDeferPeriod steps old, in a rolling refresh: at step t the resolution
// kernel brings the cell blocks b with b = t (mod kDeferPeriod) up to step
// t + 1.  The dense traffic is then that of one full pass every
// kDeferPeriod steps: 18 / kDeferPeriod bytes per cell-step.
// ---------------------------------------------------------------------------
#ifndef PEDSIM_DEFER_PERIOD
#define PEDSIM_DEFER_PERIOD 32
#endif
constexpr uint32_t kDeferPeriod = PEDSIM_DEFER_PERIOD;
static_assert(kDeferPeriod >= 1 && kDeferPeriod <= 128, "stamp ages must stay below 256");

// v evaporated `age` times (Eq. 3 once per step).
__device__ __forceinline__ float evaporate_n(float v, uint32_t age, float q)
{
    for (uint32_t i = 0; i < age; ++i) v = __fmul_rn(v, q);
    return v;
}

// First kernel of the deferred step: the proposals only.  Two builds: with
// no register cap (four CTAs per SM) for launches whose proposal CTAs fit one
// resident wave, where each agent's chain of loads is the step's critical
// path; and capped at six CTAs per SM for larger launches, which are
// throughput-bound and gain from the occupancy.
template <int kMinBlocks>
__global__ void __launch_bounds__(kAgentBlock, kMinBlocks)
deferred_stage1_kernel(const ScenarioDesc *__restrict__ descs,
                       const uint32_t *__restrict__ agent_prefix, int n_scen, uint32_t agent_blocks,
                       int prefetch)
{
    __shared__ __align__(128) ScenarioDesc hdr;  // header part only
    const uint32_t b = blockIdx.x;
    if (b >= agent_blocks) {
        pdl_wait();
        pdl_trigger();
        return;
    }
    // the descriptor header before the wait, the step index after it (see
    // agent_stage1_kernel)
    const int s = block_scenario(agent_prefix, n_scen, b);
    const uint32_t lb = b - __ldg(agent_prefix + s);
    load_header(&hdr, descs + s);
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    propose_block<true>(hdr, lb, __ldcg(&descs[s].step), prefetch != 0);
}

// Rolling refresh of cell block b of scenario d at step t: every unclaimed
// cell is brought up to step t + 1 (its stamp becomes t + 1); claimed cells
// are left to their winners, which write both planes and the stamp.  The
// values and stamps (not written by the first kernel) are loaded before the
// wait for it, the neighbours' codes after it.
__device__ __forceinline__ void refresh_block(const ScenarioDesc &d, uint64_t t, uint32_t b)
{
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const size_t c0 = (size_t)b * kCellBlock;
    float4 va[kStreamVec], vb[kStreamVec];
    uint32_t sw[kStreamVec];
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        if (c < cells) {
            va[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[0][0] + c));
            vb[k] = __ldcg(reinterpret_cast<const float4 *>(d.tau[1][0] + c));
            sw[k] = __ldcg(reinterpret_cast<const unsigned int *>(d.stamp + c));
        }
    }
    pdl_wait();  // the proposals of the step are in
    pdl_trigger();
    const int p = (int)(t & 1);
    const uint32_t now = (uint32_t)t, next = (uint32_t)(t + 1) & 255u;
    const float q = d.q;
    // each 4-cell group brought up to step t + 1, the evaporation chains of
    // its eight values interleaved
#pragma unroll
    for (int k = 0; k < kStreamVec; ++k) {
        const size_t c = c0 + 4 * ((size_t)k * kAgentBlock + threadIdx.x);
        if (c >= cells) continue;
        float a0 = va[k].x, a1 = va[k].y, a2 = va[k].z, a3 = va[k].w;
        float b0 = vb[k].x, b1 = vb[k].y, b2 = vb[k].z, b3 = vb[k].w;
        const uint32_t g0 = ((now - sw[k]) & 255u) + 1u, g1 = ((now - (sw[k] >> 8)) & 255u) + 1u;
        const uint32_t g2 = ((now - (sw[k] >> 16)) & 255u) + 1u, g3 = ((now - (sw[k] >> 24)) & 255u) + 1u;
        const uint32_t most = max(max(g0, g1), max(g2, g3));
        for (uint32_t i = 0; i < most; ++i) {
            if (i < g0) { a0 = __fmul_rn(a0, q); b0 = __fmul_rn(b0, q); }
            if (i < g1) { a1 = __fmul_rn(a1, q); b1 = __fmul_rn(b1, q); }
            if (i < g2) { a2 = __fmul_rn(a2, q); b2 = __fmul_rn(b2, q); }
            if (i < g3) { a3 = __fmul_rn(a3, q); b3 = __fmul_rn(b3, q); }
        }
        // claimed flags of the four cells
        const uint32_t cw = __ldcg(reinterpret_cast<const unsigned int *>(d.codes[p] + c)) & 0x80808080u;
        if (cw == 0u) {
            *reinterpret_cast<float4 *>(d.tau[0][0] + c) = make_float4(a0, a1, a2, a3);
            *reinterpret_cast<float4 *>(d.tau[1][0] + c) = make_float4(b0, b1, b2, b3);
            *reinterpret_cast<unsigned int *>(d.stamp + c) = next * 0x01010101u;
        } else {
            // the winners write the claimed cells
            if (!(cw & 0xffu)) { d.tau[0][0][c] = a0; d.tau[1][0][c] = b0; d.stamp[c] = (uint8_t)next; }
            if (!(cw & 0xff00u)) { d.tau[0][0][c + 1] = a1; d.tau[1][0][c + 1] = b1; d.stamp[c + 1] = (uint8_t)next; }
            if (!(cw & 0xff0000u)) { d.tau[0][0][c + 2] = a2; d.tau[1][0][c + 2] = b2; d.stamp[c + 2] = (uint8_t)next; }
            if (!(cw & 0xff000000u)) { d.tau[0][0][c + 3] = a3; d.tau[1][0][c + 3] = b3; d.stamp[c + 3] = (uint8_t)next; }
        }
    }
}

// Second kernel of the deferred step.  CTAs 0 .. agent_blocks-1 resolve one
// agent per thread as agent_resolve_kernel does; a winner brings both of its
// target's values up to step t, then writes the other group's evaporated
// value, its own group's evaporated value plus the deposit (Eq. 4/5) and the
// stamp t + 1.  The CTAs after them refresh the step's slice of cell blocks:
// CTA j of scenario s (slice_prefix) takes block j * kDeferPeriod + t mod
// kDeferPeriod.  The CTA holding the last ticket advances the step indices.
// Two builds: four CTAs per SM (64 registers, no spills of the prefetched
// values) for launches that fit one resident wave of that build, five CTAs
// per SM (48 registers) for larger ones.
template <int kMinBlocks>
__global__ void __launch_bounds__(kAgentBlock, kMinBlocks)
deferred_resolve_kernel(const ScenarioDesc *__restrict__ descs,
                        const uint32_t *__restrict__ agent_prefix,
                        const uint32_t *__restrict__ cell_prefix,
                        const uint32_t *__restrict__ slice_prefix, int n_scen,
                        uint32_t agent_blocks, ActivityCtl *__restrict__ ctl, int prefetch)
{
    unsigned int ticket = 0;
    if (blockIdx.x >= agent_blocks) {
        const uint32_t j = blockIdx.x - agent_blocks;
        const int s = block_scenario(slice_prefix, n_scen, j);
        const ScenarioDesc &d = descs[s];
        const uint64_t t = d.step;
        const uint32_t b = (j - __ldg(slice_prefix + s)) * kDeferPeriod +
                           (uint32_t)(t % kDeferPeriod);
        const uint32_t blocks = __ldg(cell_prefix + s + 1) - __ldg(cell_prefix + s);
        if (t < d.end_step && b < blocks) {
            refresh_block(d, t, b);
        } else {
            pdl_wait();
            pdl_trigger();
        }
        __syncthreads();  // every thread has read the step index
        if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket, 1u);
    } else {
        const uint32_t bb = blockIdx.x;
        const int s = block_scenario(agent_prefix, n_scen, bb);
        const ScenarioDesc &d = descs[s];
        const uint32_t lb = bb - __ldg(agent_prefix + s);
        const uint64_t t = d.step;
        const uint32_t a = lb * kAgentBlock + threadIdx.x;
        bool live = t < d.end_step && a < 2u * d.n_per_side;
        const bool aco = d.model == 1;
        const int W = d.W, H = d.H;
        Resolve r;
        // Before the wait for the proposals: the agent's own entries and, with
        // `prefetch` (latency-bound launches), both groups' values and the
        // stamps of its eight neighbours (the first kernel writes none of
        // them): whichever neighbour it proposed, its target's are at hand
        // after the wait.  Without it the target's are loaded with its
        // neighbours' codes (throughput-bound launches: 3 loads per agent
        // instead of 24).
        float va[8], vb[8];
        uint32_t st[8];
        int x = 0, y = 0;
        if (live) {
            resolve_load_own(d, a, r);
            y = (int)cell_row(d, r.cell);
            x = (int)(r.cell - (uint32_t)y * (uint32_t)W);
        }
        if (prefetch) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ox = j < 3 ? j - 1 : j < 5 ? 2 * j - 7 : j - 6;  // scan offset j
                const int oy = j < 3 ? -1 : j < 5 ? 0 : 1;
                const bool ok = live && aco && (unsigned)(x + ox) < (unsigned)W &&
                                (unsigned)(y + oy) < (unsigned)H;
                const int64_t off = (int64_t)r.cell + (int64_t)oy * W + ox;
                va[j] = ok ? ld_nc_f32(d.tau[0][0] + off) : 0.0f;
                vb[j] = ok ? ld_nc_f32(d.tau[1][0] + off) : 0.0f;
                st[j] = ok ? ld_nc_u8(d.stamp + off) : 0u;
            }
        }
        __syncthreads();  // every thread has read the step index: the ticket
        if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket, 1u);
        pdl_wait();  // proposals complete
        pdl_trigger();
        if (live) {
            resolve_load_code(d, r);
            live = r.code != 0;
        }
        Counts cnt;
        if (live) {
            // the target's claimants from its neighbours' codes
            const int dx = kCodeDX[r.code], dy = kCodeDY[r.code];
            r.target = (int64_t)r.cell + (int64_t)dy * W + dx;
            const int tx = x + dx;
            float ta = 0.0f, tb = 0.0f;
            uint32_t ts = 0;
            if (aco && !prefetch) {
                ta = __ldg(d.tau[0][0] + r.target);
                tb = __ldg(d.tau[1][0] + r.target);
                ts = __ldg(d.stamp + r.target);
            }
            r.mask = gather_claims(d.codes[(int)(t & 1)], W, H, r.target, tx, y + dy);
            const uint32_t k = (uint32_t)__popc(r.mask);
            const uint32_t mine = 8u - (uint32_t)r.code;
            const uint32_t win =
                k == 1 ? mine : pick_claimant(r.mask, k, (uint64_t)r.target, t, d.seed);
            if (win == mine) {
                const int g = r.g;
                d.occ[0][r.target] = (uint8_t)g;
                d.occ[0][r.cell] = 0;
                d.codes[(int)(t & 1) ^ 1][r.cell] = 0;  // its old cell, in the plane of t + 1
                d.pos[r.id] = (uint32_t)r.target;
                d.acode[r.id] = (uint8_t)(r.code | (g << 4) | 0x80);
                d.ids[r.target] = r.id;
                float dep = d.deposit;
                if (aco && d.deposit_mode == 1) {
                    const float L = __fadd_rn(r.tour0, (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
                    d.tour[r.id] = L;
                    dep = __fdiv_rn(1.0f, L);
                }
                const bool in_band = g == 1 ? tx >= W - (int)d.band : tx < (int)d.band;
                if (in_band && r.arrived == 0) {
                    d.arrival[r.id] = (uint32_t)(t + 1);
                    if (g == 1) ++cnt.crossed_a; else ++cnt.crossed_b;
                }
                if (aco) {
                    // the target is this agent's neighbour at scan offset
                    // code - 1: its values at t (both groups' chains
                    // interleaved), then step t's evaporation and the deposit
                    if (prefetch) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j == r.code - 1) { ta = va[j]; tb = vb[j]; ts = st[j]; }
                    }
                    const float q = d.q;
                    const uint32_t age = (((uint32_t)t - ts) & 255u) + 1u;
                    for (uint32_t i = 0; i < age; ++i) {
                        ta = __fmul_rn(ta, q);
                        tb = __fmul_rn(tb, q);
                    }
                    if (g == 1) ta = __fadd_rn(ta, dep); else tb = __fadd_rn(tb, dep);
                    d.tau[0][0][r.target] = ta;
                    d.tau[1][0][r.target] = tb;
                    d.stamp[r.target] = (uint8_t)(t + 1);
                }
                ++cnt.moved;
                if (k >= 2) ++cnt.conflicts;
            }
        }
        flush_counts(d, cnt, lb % d.n_slots);
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

// Brings every cell of one scenario up to its current step (both planes,
// stamps := step): read-back, checkpoints and a change of step variant see
// plain planes.  Values do not change, only how old their stored form is.
__global__ void deferred_catch_up_kernel(const ScenarioDesc *__restrict__ dp)
{
    const ScenarioDesc &d = *dp;
    if (d.model != 1) return;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const uint32_t now = (uint32_t)d.step;
    const float q = d.q;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
        const uint32_t age = (now - (uint32_t)d.stamp[c]) & 255u;
        if (!age) continue;
        d.tau[0][0][c] = evaporate_n(d.tau[0][0][c], age, q);
        d.tau[1][0][c] = evaporate_n(d.tau[1][0][c], age, q);
        d.stamp[c] = (uint8_t)now;
    }
}

__global__ void build_pos_kernel(const ScenarioDesc *__restrict__ dp, int plane)
{
    const ScenarioDesc &d = *dp;
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const uint8_t *occ = d.occ[plane];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
        d.codes[0][c] = 0;
        d.codes[1][c] = 0;
        if (occ[c]) {
            // every agent stands on exactly one cell: its position and its
            // per-agent byte (group, no code yet) are written once
            const uint32_t id = d.ids[c];
            d.pos[id] = (uint32_t)c;
            d.acode[id] = (uint8_t)(occ[c] << 4);
        }
    }
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

static uint32_t deferred_stage1_wave()
{
    static std::atomic<uint32_t> cache[kMaxDevices];
    return resident_wave(deferred_stage1_kernel<6>, cache);
}

static uint32_t deferred_resolve_wave()
{
    static std::atomic<uint32_t> cache[kMaxDevices];
    return resident_wave(deferred_resolve_kernel<5>, cache);
}

static uint32_t deferred_resolve_wave4()
{
    static std::atomic<uint32_t> cache[kMaxDevices];
    return resident_wave(deferred_resolve_kernel<4>, cache);
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
        // speculative pheromone loads only while the agents fit in one wave
        const int prefetch = agent_blocks <= wave;
        if (c1 + agent_blocks) {
            cudaError_t e = launch_pdl(agent_stage1_kernel, c1 + agent_blocks,
                                       (unsigned)kAgentBlock, stream, d_descs, d_cell_prefix,
                                       d_agent_prefix, n, c1, agent_blocks, front, prefetch);
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

cudaError_t launch_deferred_step(const ScenarioDesc *d_descs, const uint32_t *d_cell_prefix,
                                 const uint32_t *d_agent_prefix, const uint32_t *d_slice_prefix,
                                 int n, uint32_t slices, uint32_t agent_blocks, ActivityCtl *ctl,
                                 cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    // the first kernel runs even with no agent: the refresh CTAs' loads
    // before their wait rely on it having waited for the previous step
    // speculative loads only while each kernel's CTAs fit in one resident
    // wave (latency-bound); a launch with more agents is throughput-bound
    const int pre1 = agent_blocks <= deferred_stage1_wave();
    const unsigned g1 = agent_blocks > 0 ? agent_blocks : 1u;
    cudaError_t e = pre1 ? launch_pdl(deferred_stage1_kernel<1>, g1, (unsigned)kAgentBlock, stream,
                                      d_descs, d_agent_prefix, n, agent_blocks, pre1)
                         : launch_pdl(deferred_stage1_kernel<6>, g1, (unsigned)kAgentBlock, stream,
                                      d_descs, d_agent_prefix, n, agent_blocks, pre1);
    if (e != cudaSuccess) return e;
    const uint32_t g = agent_blocks + slices > 0 ? agent_blocks + slices : 1u;
    if (g <= deferred_resolve_wave4())
        return launch_pdl(deferred_resolve_kernel<4>, g, (unsigned)kAgentBlock, stream, d_descs,
                          d_agent_prefix, d_cell_prefix, d_slice_prefix, n, agent_blocks, ctl, 1);
    const int pre2 = g <= deferred_resolve_wave();
    return launch_pdl(deferred_resolve_kernel<5>, g, (unsigned)kAgentBlock, stream, d_descs,
                      d_agent_prefix, d_cell_prefix, d_slice_prefix, n, agent_blocks, ctl, pre2);
}

uint32_t deferred_slices(uint32_t cell_blocks)
{
    return (cell_blocks + kDeferPeriod - 1) / kDeferPeriod;
}

cudaError_t launch_deferred_catch_up(const ScenarioDesc *d_desc, int cells, cudaStream_t stream)
{
    int blocks = (cells + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    deferred_catch_up_kernel<<<blocks, 256, 0, stream>>>(d_desc);
    return cudaGetLastError();
}

cudaError_t launch_build_pos(const ScenarioDesc *d_desc, int cells, int plane, cudaStream_t stream)
{
    (void)stage1_wave();  // the steps' occupancy queries, outside any capture
    (void)resolve_wave();
    (void)deferred_stage1_wave();
    (void)deferred_resolve_wave();
    (void)deferred_resolve_wave4();
    int blocks = (cells + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    build_pos_kernel<<<blocks, 256, 0, stream>>>(d_desc, plane);
    return cudaGetLastError();
}

}  // namespace pedsim
