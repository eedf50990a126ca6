// CUDA kernels of the GB300 pedestrian cellular automaton (sm_103a).
//
//   init_kernel        clear planes, fill pheromone with tau0, zero arrays and
//                      counters
//   place_kernel       random placement in the edge bands (Sec. IV.a)
//   fused_step_kernel  one synchronous step (Sec. IV.b-d) in a single pass:
//                      persistent CTAs (four consumer warps and a producer
//                      warp) walk the (scenario, tile) work list, tiles near
//                      agents first; for such a tile a TMA copy stages the
//                      occupancy with a 3-cell halo and the two pheromone tiles
//                      in shared memory (two stages behind mbarriers), the
//                      proposals of the tile plus a 2-cell ring are computed,
//                      then every tile cell resolves (gather), evaporates
//                      (Eq. 3), deposits (Eq. 4/5) and counts; a tile with no
//                      agent within reach only evaporates its pheromone
//   propose_tile_kernel + resolve_tile_kernel
//                      the same step as two kernels per tile through a
//                      proposal plane
//   propose_plane_kernel + resolve_plane_kernel
//                      the same step in two passes through a proposal plane in
//                      HBM (baseline and cross-check of the fused pass)
//   grid_counts_kernel agents / parked per group (read-back helper)
// advance_kernel adds the step count of a launch group to every step index.
#include "pedsim_internal.h"
#include "pedsim_rules.cuh"
#include "pedsim_ptx.cuh"

namespace pedsim {

constexpr int kThreads = 256;
// ---------------------------------------------------------------------------
// Shared per-cell resolution (Sec. IV.d), used by both step variants.
// occ_at(dx, dy): occupancy at t; prop_at(dx, dy): proposal code at t.
// Returns the occupancy byte at t+1 and reports the group of an agent that
// entered this cell (0 if none) plus the deposit it leaves.
// ---------------------------------------------------------------------------

template <class OccFn, class PropFn>
__device__ __forceinline__ int resolve_cell(const ScenarioDesc &d, int x, int y, uint64_t cell,
                                            uint64_t t, int o, OccFn occ_at, PropFn prop_at,
                                            Counts &cnt, int &incoming, float &dep)
{
    const int W = d.W, H = d.H;
    incoming = 0;
    dep = d.deposit;
    if (o == 0) {
        int k;
        const int w = resolve_winner(x, y, W, H, cell, t, d.seed, prop_at, &k);
        if (w < 0) return 0;
        const int dx = kCodeDX[w + 1], dy = kCodeDY[w + 1];
        incoming = occ_at(dx, dy);
        const uint64_t src = cell + (int64_t)dy * W + dx;
        const uint32_t id = d.ids[src];
        d.ids[cell] = id;
        ++cnt.moved;
        if (k >= 2) ++cnt.conflicts;
        if (d.model == 1 && d.deposit_mode == 1) {
            // Eq. 5: the tour length grows by the step length, then 1/L_k
            const float L = __fadd_rn(d.tour[id], (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
            d.tour[id] = L;
            dep = __fdiv_rn(1.0f, L);
        }
        const bool in_band = incoming == 1 ? x >= W - (int)d.band : x < (int)d.band;
        if (in_band && d.arrival[id] == 0) {
            d.arrival[id] = (uint32_t)(t + 1);
            if (incoming == 1) ++cnt.crossed_a; else ++cnt.crossed_b;
        }
        return incoming;
    }
    const int code = prop_at(0, 0);
    if (code == 0) return o;
    const int dx = kCodeDX[code], dy = kCodeDY[code];
    int k;
    const int w = resolve_winner(
        x + dx, y + dy, W, H, cell + (int64_t)dy * W + dx, t, d.seed,
        [&](int ex, int ey) { return prop_at(dx + ex, dy + ey); }, &k);
    return (w == 8 - code) ? 0 : o;
}

// ---------------------------------------------------------------------------
// init / placement
// ---------------------------------------------------------------------------
__global__ void init_kernel(const ScenarioDesc *__restrict__ descs)
{
    const ScenarioDesc &d = descs[blockIdx.y];
    const size_t cells = (size_t)d.W * (size_t)d.H;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
        d.occ[0][c] = 0;
        d.ids[c] = 0;
        if (d.model == 1) {
            d.tau[0][0][c] = d.tau0;
            d.tau[1][0][c] = d.tau0;
            d.stamp[c] = (uint8_t)d.step;  // plane 0 is valid at the step index
        }
    }
    const size_t agents = 2 * (size_t)d.n_per_side + 1;
    for (size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x; a < agents; a += stride) {
        d.arrival[a] = 0;
        if (d.tour) d.tour[a] = 0.0f;
    }
    const size_t slots = (size_t)d.n_slots * kNumCounters;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride)
        d.part[i] = 0;
    // (the step index is part of the descriptor the host uploads)
    if (blockIdx.x == 0 && threadIdx.x == 0) *d.error = 0;
}

// One CTA per (scenario, group): the n band cells with the smallest
// Philox keys (stream 3, step 0) by a block-wide 8-bit radix select over the
// 64-bit keys, then ids in increasing cell order by a block scan of the
// selection flags.  Keys are recomputed in every pass instead of stored.
__global__ void __launch_bounds__(1024) place_kernel(const ScenarioDesc *__restrict__ descs)
{
    const ScenarioDesc &d = descs[blockIdx.x >> 1];
    const int g = (int)(blockIdx.x & 1) + 1;
    const uint32_t n = d.n_per_side;
    if (n == 0) return;
    const int band = (int)d.band, W = d.W;
    const int x0 = g == 1 ? 0 : W - band;
    const uint32_t M = (uint32_t)band * (uint32_t)d.H;
    const uint64_t seed = d.seed;

    __shared__ uint32_t hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_need, s_eq, s_base;
    __shared__ uint32_t warp_incl[32];

    auto cell_of = [&](uint32_t j) {
        return (uint64_t)(j / (uint32_t)band) * (uint64_t)W + (uint64_t)x0 + (j % (uint32_t)band);
    };
    auto key_of = [&](uint32_t j) { return draw(seed, cell_of(j), 0, kStreamPlace).r0; };

    uint64_t prefix = 0, mask = 0;
    uint32_t need = n, eq_total = 0;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
            const uint64_t key = key_of(j);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cum = 0;
            for (int b = 0; b < 256; ++b) {
                if (cum + hist[b] >= need) {
                    s_prefix = prefix | ((uint64_t)b << shift);
                    s_need = need - cum;
                    s_eq = hist[b];
                    break;
                }
                cum += hist[b];
            }
        }
        __syncthreads();
        prefix = s_prefix;
        need = s_need;
        eq_total = s_eq;
        mask |= 0xFFull << shift;
        __syncthreads();
    }
    // prefix is now the n-th smallest key; `need` of the eq_total cells
    // carrying exactly that key are taken, the lowest cell indices first.
    const uint64_t kth = prefix;
    const uint32_t first_id = g == 1 ? 1u : n + 1u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (uint32_t chunk = 0; chunk < M; chunk += blockDim.x) {
        const uint32_t j = chunk + threadIdx.x;
        bool sel = false;
        if (j < M) {
            const uint64_t key = key_of(j);
            if (key < kth) {
                sel = true;
            } else if (key == kth) {
                if (need == eq_total) {
                    sel = true;
                } else {
                    uint32_t before = 0;
                    for (uint32_t jj = 0; jj < j; ++jj) before += key_of(jj) == kth;
                    sel = before < need;
                }
            }
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, sel);
        const uint32_t in_warp = __popc(ballot & ((1u << lane) - 1u));
        if (lane == 0) warp_incl[warp] = __popc(ballot);
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < nwarps ? warp_incl[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (lane < nwarps) warp_incl[lane] = v;
        }
        __syncthreads();
        if (sel) {
            const uint32_t before = warp == 0 ? 0u : warp_incl[warp - 1];
            const uint64_t c = cell_of(j);
            d.occ[0][c] = (uint8_t)g;
            d.ids[c] = first_id + s_base + before + in_warp;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += warp_incl[nwarps - 1];
        __syncthreads();
    }
}

// Appends `n` entries of this thread to a shared list with one shared atomic
// per warp; returns the first slot of this thread.  All 32 lanes must call.
__device__ __forceinline__ int warp_reserve(unsigned int *counter, int n)
{
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned int)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return (int)base + incl - n;
}

// Forward-first part of a proposal (Sec. III): 0 for an agent on its goal
// column, the forward code when the forward cell is in the grid and empty,
// -1 when the agent is blocked and needs the full rule.
template <class OccFn>
__device__ __forceinline__ int forward_first(int x, int y, int g, int W, int H, OccFn occ)
{
    if ((g == 1 && x == W - 1) || (g == 2 && x == 0)) return 0;
    const int code = kFrameCode[g - 1][1];
    const int dx = kCodeDX[code];
    const int nx = x + dx;
    if ((unsigned)nx < (unsigned)W && occ(dx, 0) == 0) return code;
    (void)y;
    (void)H;
    return -1;
}

// ---------------------------------------------------------------------------
// Fused single-pass step with tile activity tracking
//
// A tile is ACTIVE at a step when an agent stands in it or on a cell next to
// it: only then can one of its cells change occupancy or receive a deposit
// (agents move at most one cell per step, Sec. III).  Every other tile is
// QUIET: its pheromone only evaporates (Eq. 3) and its occupancy stays empty.
// An active tile that ends the step with agents marks itself and each
// neighbouring tile that one of those agents touches (its border rows and
// columns, its corner cells) active for the next step; a mark sets the
// tile's flag bit and the first mark appends the tile to the next step's
// list.  Quiet tiles never end a step with agents, so the marks are complete.
//
// Per work list (one scenario or a batch) an ActivityCtl block holds three
// generations of flags and lists; launch k reads generation k % 3, writes
// k + 1 and clears k + 2.  Work items of a launch: the active list first
// (dense tiles start at once instead of forming the tail), then every tile
// in natural order in chunks of kQuietChunk, where flagged tiles are skipped
// and the rest are quiet.  After the host changes a work list or a state it
// sets `reset`: that launch treats every tile as active.
//
// CTA organisation: four consumer warps work on one item at a time; a fifth,
// producer, warp claims and decodes work items and issues the TMA copies of
// an active tile into one of two shared-memory stages (full / empty
// mbarriers), so claims, list reads and copies overlap the consumers' work.
// Quiet chunks need no copy: the consumers stream their pheromone through
// registers, every load of the chunk in flight at once.
//
// Shared memory of one CTA.  The byte planes use the occupancy tile's column
// mapping (column cx <-> x = x0 - 16 + cx, row stride OW), so one index
// arithmetic serves all of them:
//   occ[stage]     (TH+6) x OW      uint8  TMA copy of rows y0-3 .. y0+TH+2
//   tau[stage][g]  (TH+6) x (TW+8)  float  TMA copy of x0-4 .. x0+TW+3,
//                                          rows y0-3 .. y0+TH+2 (ACO)
//   prop           (TH+4) x OW      uint8  proposal codes, rows y0-2 .. y0+TH+1
//   win            (TH+2) x OW      uint8  claim masks, then winners, rows
//                                          y0-1 .. y0+TH
//   agents         list of the occupied cells of the tile and its 2-ring
//   moves          list of the tile cells that receive an agent
//   dep            TH x TW float deposit left in each receiving cell (ACO);
//                  before that, the list of blocked agents, then the list of
//                  cells with two or more claimants
// A claim mask holds bit j when the neighbour at scan offset j chose the
// cell; bitwise OR makes it independent of the order claims arrive in.  The
// winner byte is (scan index + 1) | 0x10 when there were >= 2 claimants.
// List order never matters: every list entry's effects are independent.
// ---------------------------------------------------------------------------
constexpr int kFusedConsumers = 128;                  // threads working on a tile
constexpr int kFusedThreads = kFusedConsumers + 32;   // + the producer warp
constexpr int kStages = 2;
constexpr int kFusedMinBlocks = 4;  // resident CTAs per SM the register budget allows
constexpr int align_to(int v, int a) { return (v + a - 1) / a * a; }

enum : uint32_t { kItemEnd = 0, kItemQuiet = 1, kItemActive = 2 };

template <int TW, int TH>
struct FusedLayout {
    static constexpr int OW = TW + 32;
    static constexpr int OH = TH + 6;
    static constexpr int TWH = TW + 8;  // pheromone tile row (4-column halo each side)
    static constexpr int THH = TH + 6;  // 3-row halo above and below
    static constexpr int OCC_BYTES = align_to(OH * OW, 128);
    static constexpr int TAU_BOX_BYTES = THH * TWH * 4;
    static constexpr int TAU_BYTES = align_to(TAU_BOX_BYTES, 128);
    static constexpr int PROP_BYTES = align_to((TH + 4) * OW, 16);
    static constexpr int WIN_BYTES = align_to((TH + 2) * OW, 16);
    static constexpr int MAX_AGENTS = (TH + 4) * (TW + 4);
    static constexpr int MAX_MOVES = TH * TW;
    static constexpr int MAX_CONFLICTS = (TH + 2) * (TW + 2);
    static constexpr int OFF_TAU = kStages * OCC_BYTES;  // [stage][group]
    static constexpr int OFF_PROP = OFF_TAU + kStages * 2 * TAU_BYTES;
    static constexpr int OFF_WIN = OFF_PROP + PROP_BYTES;
    static constexpr int OFF_DEP = OFF_WIN + WIN_BYTES;
    static constexpr int OFF_AGENTS = OFF_DEP + TH * TW * 4;
    static constexpr int OFF_MOVES = OFF_AGENTS + align_to(MAX_AGENTS * 2, 16);
    static constexpr int OFF_MISC = OFF_MOVES + align_to(MAX_MOVES * 2, 16);  // list counters
    static constexpr int OFF_ITEM = OFF_MISC + 32;           // per stage: item, scenario|mask, kind
    static constexpr int OFF_BAR = OFF_ITEM + kStages * 16;  // full[stage], empty[stage]
    static constexpr int SMEM = OFF_BAR + 2 * kStages * 8 + 128;  // + slack to align the base
    // 32-bit word columns covering cx = 12 .. TW+19 (x0-4 .. x0+TW+3)
    static constexpr int WC0 = 3, NWC = TW / 4 + 2;
    static_assert(OW <= 256 && OH <= 256 && TWH <= 256 && THH <= 256, "TMA box limit");
    static_assert((TH + 6) * OW < 65536, "16-bit list entries");
    static_assert(MAX_AGENTS * 2 <= TH * TW * 4 && MAX_CONFLICTS * 2 <= TH * TW * 4,
                  "blocked and conflict lists fit the deposit array");
};

// Tiles per quiet work item: about 2048 cells, so that each consumer thread
// keeps 16 pheromone cells of both groups in flight.
template <int TW, int TH>
__host__ __device__ constexpr int quiet_chunk() { return TW * TH >= 2048 ? 1 : 2048 / (TW * TH); }

__device__ __forceinline__ int scenario_of(const uint32_t *__restrict__ prefix, int n,
                                           uint32_t item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Barrier 1 over the consumer warps only (the producer warp never joins).
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kFusedConsumers) : "memory");
}

__device__ __forceinline__ bool consumer_sync_and(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kFusedConsumers)
        : "memory");
    return r != 0;
}

// Per-agent bookkeeping of one move into `cell` from `src` (Sec. IV.d): the
// id follows the agent, Eq. 5 extends the tour length, the first entry into
// the opposite band is recorded (Sec. VI).  Returns the deposit's float bits
// in the low word and 1 << 32 when the agent crossed at this step.
// `id` is the moving agent's id, read from its source cell.
__device__ __forceinline__ uint64_t apply_move_id(const ScenarioDesc &d, uint64_t cell,
                                                  uint32_t id, int inc, int xc, bool diagonal,
                                                  uint64_t t)
{
    d.ids[cell] = id;
    float dep = d.deposit;
    if (d.model == 1 && d.deposit_mode == 1) {
        const float L = __fadd_rn(d.tour[id], diagonal ? kSqrt2 : 1.0f);
        d.tour[id] = L;
        dep = __fdiv_rn(1.0f, L);
    }
    uint64_t crossed = 0;
    const bool in_band = inc == 1 ? xc >= d.W - (int)d.band : xc < (int)d.band;
    if (in_band && d.arrival[id] == 0) {
        d.arrival[id] = (uint32_t)(t + 1);
        crossed = 1ull << 32;
    }
    return crossed | (uint64_t)__float_as_uint(dep);
}

__device__ __forceinline__ uint64_t apply_move(const ScenarioDesc &d, uint64_t cell,
                                               uint64_t src, int inc, int xc, bool diagonal,
                                               uint64_t t)
{
    return apply_move_id(d, cell, d.ids[src], inc, xc, diagonal, t);
}

template <int TW, int TH>
__global__ void __launch_bounds__(kFusedThreads, kFusedMinBlocks)
fused_step_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                  int n_scen, uint32_t total, int t_off, ActivityCtl *__restrict__ act)
{
    using Lay = FusedLayout<TW, TH>;
    constexpr int NT = kFusedConsumers;
    constexpr int OW = Lay::OW, NWC = Lay::NWC, WC0 = Lay::WC0, TWH = Lay::TWH;
    constexpr int GW = TW / 4;  // 4-cell groups per tile row
    constexpr int QC = quiet_chunk<TW, TH>();
    constexpr int QG = (TH * GW + NT - 1) / NT;  // 4-cell groups per thread per quiet tile
    static_assert(32 % QC == 0, "quiet chunks never straddle a flag word");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // TMA destinations need 128-byte alignment: align the base explicitly
    uint8_t *const smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint8_t *const Pp = smem + Lay::OFF_PROP;
    uint8_t *const Cw = smem + Lay::OFF_WIN;
    float *const depv = reinterpret_cast<float *>(smem + Lay::OFF_DEP);
    uint16_t *const blocked = reinterpret_cast<uint16_t *>(smem + Lay::OFF_DEP);
    uint16_t *const conflicts = reinterpret_cast<uint16_t *>(smem + Lay::OFF_DEP);
    uint16_t *const agents = reinterpret_cast<uint16_t *>(smem + Lay::OFF_AGENTS);
    uint16_t *const moves = reinterpret_cast<uint16_t *>(smem + Lay::OFF_MOVES);
    unsigned int *const misc = reinterpret_cast<unsigned int *>(smem + Lay::OFF_MISC);
    // misc[0] agents, misc[1] moves, misc[2] blocked agents, misc[3] conflicts,
    // misc[4] neighbourhood mark bits
    uint32_t *const item_hdr = reinterpret_cast<uint32_t *>(smem + Lay::OFF_ITEM);
    uint64_t *const full = reinterpret_cast<uint64_t *>(smem + Lay::OFF_BAR);
    uint64_t *const empty = full + kStages;
    auto occ_stage = [&](int st) { return smem + st * Lay::OCC_BYTES; };
    auto tau_stage = [&](int st, int g) {
        return reinterpret_cast<float *>(smem + Lay::OFF_TAU + (st * 2 + g) * Lay::TAU_BYTES);
    };

    // This launch's generation of the activity flags and lists.
    const uint32_t ph = act->phase;
    const bool all_active = act->reset != 0;
    const uint32_t n_act = all_active ? 0u : act->n_act[ph];
    const uint32_t nfw = (total + 31u) / 32u;
    uint32_t *const flag_base = reinterpret_cast<uint32_t *>(act + 1);
    const uint32_t *const F_cur = flag_base + ph * nfw;
    uint32_t *const F_next = flag_base + ((ph + 1u) % 3u) * nfw;
    uint32_t *const F_old = flag_base + ((ph + 2u) % 3u) * nfw;
    uint32_t *const list_base = flag_base + 3u * nfw;
    const uint32_t *const L_cur = list_base + ph * total;
    uint32_t *const L_next = list_base + ((ph + 1u) % 3u) * total;
    unsigned int *const n_next = &act->n_act[(ph + 1u) % 3u];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kFusedConsumers / 32);
        }
        fence_mbarrier_init();
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool failed = false;

    if (warp == kFusedConsumers / 32) {
        // ------------------------------ producer ------------------------------
        auto live = [&](uint32_t sc) {
            const ScenarioDesc *d = descs + sc;
            return d->step + (uint64_t)t_off < d->end_step;
        };
        bool list_left = n_act > 0;
        uint32_t pend_j0 = 0, pend_m = 0;  // quiet tiles of a claimed chunk not yet handed out
        // Next work item with work: an active tile (item, aux = its scenario)
        // or quiet tiles of one scenario within a chunk (item = the chunk's
        // first item, aux = scenario << 8 | bit q for each quiet tile item + q).
        // The natural-order pass also clears generation k + 2's flag words.
        auto quiet_group = [&](uint32_t &item, uint32_t &aux) {
            // the first pending tile's scenario and every pending tile of it
            const int q0 = __ffs(pend_m) - 1;
            const uint32_t sc = (uint32_t)scenario_of(tile_prefix, n_scen, pend_j0 + (uint32_t)q0);
            const uint32_t end = __ldg(tile_prefix + sc + 1);
            uint32_t m = 0;
            for (int q = q0; q < QC; ++q)
                if (((pend_m >> q) & 1u) && pend_j0 + (uint32_t)q < end) m |= 1u << q;
            pend_m &= ~m;
            item = pend_j0;
            aux = (sc << 8) | m;
        };
        auto claim = [&](uint32_t &item, uint32_t &aux) -> uint32_t {
            if (pend_m) {
                quiet_group(item, aux);
                return kItemQuiet;
            }
            while (list_left) {
                const uint32_t j = atomicAdd(&act->work, 1u);
                if (j >= n_act) {
                    list_left = false;
                    break;
                }
                item = L_cur[j];
                aux = (uint32_t)scenario_of(tile_prefix, n_scen, item);
                if (live(aux)) return kItemActive;
            }
            for (;;) {
                if (all_active) {
                    const uint32_t j = atomicAdd(&act->work_nat, 1u);
                    if (j >= total) return kItemEnd;
                    if ((j & 31u) == 0) F_old[j >> 5] = 0u;
                    item = j;
                    aux = (uint32_t)scenario_of(tile_prefix, n_scen, item);
                    if (live(aux)) return kItemActive;
                    continue;
                }
                const uint32_t j0 = atomicAdd(&act->work_nat, (uint32_t)QC);
                if (j0 >= total) return kItemEnd;
                if ((j0 & 31u) == 0) F_old[j0 >> 5] = 0u;
                const uint32_t fw = F_cur[j0 >> 5] >> (j0 & 31u);
                uint32_t m = 0;
                for (int q = 0; q < QC; ++q) {
                    const uint32_t it = j0 + (uint32_t)q;
                    if (it >= total || ((fw >> q) & 1u)) continue;
                    if (live((uint32_t)scenario_of(tile_prefix, n_scen, it))) m |= 1u << q;
                }
                if (m) {
                    pend_j0 = j0;
                    pend_m = m;
                    quiet_group(item, aux);
                    return kItemQuiet;
                }
            }
        };
        int st = 0;
        uint32_t ephase = 0;
        for (;;) {
            uint32_t item = 0, aux = 0, kind = 0;
            if (lane == 0) kind = claim(item, aux);
            kind = __shfl_sync(0xffffffffu, kind, 0);
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&empty[st], ((ephase >> st) & 1u) ^ 1u);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            ephase ^= 1u << st;
            if (!ok) {
                failed = true;
                break;
            }
            if (lane == 0) {
                item_hdr[4 * st + 0] = item;
                item_hdr[4 * st + 1] = aux;
                item_hdr[4 * st + 2] = kind;
                if (kind == kItemActive) {
                    const ScenarioDesc *d = descs + aux;
                    const uint64_t t = d->step + (uint64_t)t_off;
                    const int p = (int)(t & 1);
                    const uint32_t local = item - __ldg(tile_prefix + aux);
                    const int tiles_x = d->tiles_x;
                    const int ty = (int)(local / (uint32_t)tiles_x), tx = (int)(local % (uint32_t)tiles_x);
                    const bool aco = d->model == 1;
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&full[st], Lay::OH * OW + (aco ? 2 * Lay::TAU_BOX_BYTES : 0));
                    tma_load_2d(occ_stage(st), &d->map_occ[p], tx * TW - 16, ty * TH - 3, &full[st]);
                    if (aco) {
                        tma_load_2d(tau_stage(st, 0), &d->map_tau[0][p], tx * TW - 4, ty * TH - 3, &full[st]);
                        tma_load_2d(tau_stage(st, 1), &d->map_tau[1][p], tx * TW - 4, ty * TH - 3, &full[st]);
                    }
                } else {
                    mbar_arrive(&full[st]);  // quiet chunk or end: nothing to copy
                }
            }
            __syncwarp();
            if (kind == kItemEnd) break;
            st = (st + 1) % kStages;
        }
    } else {
        // ------------------------------ consumers -----------------------------
        Counts cnt;
        int st = 0;
        uint32_t fphase = 0;
        for (;;) {
            if (threadIdx.x == 0) {
#pragma unroll
                for (int i = 0; i < 5; ++i) misc[i] = 0;
            }
            bool ok = true;
            if (threadIdx.x == 0) ok = mbar_wait_bounded(&full[st], (fphase >> st) & 1u);
            ok = consumer_sync_and(ok);
            fphase ^= 1u << st;
            if (!ok) {
                failed = true;
                break;
            }
            const uint32_t item = item_hdr[4 * st + 0];
            const uint32_t aux = item_hdr[4 * st + 1];
            const uint32_t kind = item_hdr[4 * st + 2];
            if (kind == kItemEnd) break;

            if (kind == kItemQuiet) {
                // No agent within reach: the occupancy stays empty and the
                // pheromone evaporates (Eq. 3).  The stage holds nothing for
                // this item: release it at once.
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
                const ScenarioDesc &d = descs[aux >> 8];
                const uint32_t m = aux & 255u;
                const uint32_t first = item - __ldg(tile_prefix + (aux >> 8));
                const int W = d.W, H = d.H, tiles_x = d.tiles_x;
                const int p = (int)((d.step + (uint64_t)t_off) & 1);
                const bool aco = d.model == 1;
                // cell index of group k of tile q of the chunk, or -1
                auto cell_of = [&](int q, int k) -> int64_t {
                    const int gi = threadIdx.x + k * NT;
                    if (!((m >> q) & 1u) || gi >= TH * GW) return -1;
                    const uint32_t local = first + (uint32_t)q;
                    const int ty = (int)(local / (uint32_t)tiles_x), tx = (int)(local % (uint32_t)tiles_x);
                    const int iy = gi / GW, gx = gi - iy * GW;
                    const int x = tx * TW + 4 * gx, y = ty * TH + iy;
                    if (x >= W || y >= H) return -1;
                    return (int64_t)y * W + x;
                };
                if (aco) {
                    float4 va[QC][QG], vb[QC][QG];
                    const float *sA = d.tau[0][p], *sB = d.tau[1][p];
                    // every pheromone load of the chunk first ...
#pragma unroll
                    for (int q = 0; q < QC; ++q)
#pragma unroll
                        for (int k = 0; k < QG; ++k) {
                            const int64_t c = cell_of(q, k);
                            if (c < 0) continue;
                            va[q][k] = __ldcs(reinterpret_cast<const float4 *>(sA + c));
                            vb[q][k] = __ldcs(reinterpret_cast<const float4 *>(sB + c));
                        }
                    // ... then the evaporated values out
                    const float qf = d.q;
                    float *dA = d.tau[0][p ^ 1], *dB = d.tau[1][p ^ 1];
#pragma unroll
                    for (int q = 0; q < QC; ++q)
#pragma unroll
                        for (int k = 0; k < QG; ++k) {
                            const int64_t c = cell_of(q, k);
                            if (c < 0) continue;
                            const float4 a4 = va[q][k], b4 = vb[q][k];
                            __stcs(reinterpret_cast<float4 *>(dA + c),
                                   make_float4(__fmul_rn(a4.x, qf), __fmul_rn(a4.y, qf),
                                               __fmul_rn(a4.z, qf), __fmul_rn(a4.w, qf)));
                            __stcs(reinterpret_cast<float4 *>(dB + c),
                                   make_float4(__fmul_rn(b4.x, qf), __fmul_rn(b4.y, qf),
                                               __fmul_rn(b4.z, qf), __fmul_rn(b4.w, qf)));
                        }
                }
                uint8_t *occ_dst = d.occ[p ^ 1];
#pragma unroll
                for (int q = 0; q < QC; ++q)
#pragma unroll
                    for (int k = 0; k < QG; ++k) {
                        const int64_t c = cell_of(q, k);
                        if (c >= 0) *reinterpret_cast<uint32_t *>(occ_dst + c) = 0u;
                    }
                st = (st + 1) % kStages;
                continue;
            }

            const uint32_t sc = aux;
            const ScenarioDesc &d = descs[sc];
            const uint64_t t = d.step + (uint64_t)t_off;
            const int W = d.W, H = d.H;
            const uint32_t local = item - __ldg(tile_prefix + sc);
            const int tiles_x = d.tiles_x;
            const int ty = (int)(local / (uint32_t)tiles_x), tx = (int)(local % (uint32_t)tiles_x);
            const int x0 = tx * TW, y0 = ty * TH;
            const int p = (int)(t & 1);
            const bool aco = d.model == 1;
            const float *tA = tau_stage(st, 0);
            const float *tB = tau_stage(st, 1);
            const uint8_t *O = occ_stage(st);
            const bool const_deposit = !(aco && d.deposit_mode == 1);

            // Phase 0: clear the claim masks; list the agents of the tile and its
            // 2-ring (cells outside the grid read as empty: TMA zero fill).  A
            // warp reserves its list slots with one shared atomic.
            for (int i = threadIdx.x; i < Lay::WIN_BYTES / 16; i += NT)
                reinterpret_cast<uint4 *>(Cw)[i] = make_uint4(0u, 0u, 0u, 0u);
            for (int i0 = 0; i0 < (TH + 4) * NWC; i0 += NT) {
                const int i = i0 + threadIdx.x;
                uint32_t found = 0;  // bit b: byte b of this word is a listed agent
                int r = 0, wc = 0;
                if (i < (TH + 4) * NWC) {
                    r = i / NWC;
                    wc = WC0 + i % NWC;
                    const uint32_t o4 = *reinterpret_cast<const uint32_t *>(O + (r + 1) * OW + 4 * wc);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int cx = 4 * wc + b;
                        if (((o4 >> (8 * b)) & 255u) && cx >= 14 && cx <= TW + 17) found |= 1u << b;
                    }
                }
                int slot = warp_reserve(&misc[0], __popc(found));
                for (int b = 0; b < 4; ++b)
                    if (found & (1u << b)) agents[slot++] = (uint16_t)((r + 1) * OW + 4 * wc + b);
            }
            consumer_sync();

            // Phase 1 (Sec. IV.b-c), from shared memory only.  1a: forward
            // first for every listed agent; the blocked ones are listed.  1b:
            // the full rule for the blocked agents, one per thread, so the
            // random draws run with full warps.  Each proposal that targets
            // the tile or its 1-ring sets its claim bit there.  Proposal codes
            // are written for occupied cells only, the only cells whose codes
            // are read.
            auto claim_target = [&](int r, int cx, int code) {
                const int tr = r - 1 + kCodeDY[code];
                const int tcx = cx + kCodeDX[code];
                if (tr >= 0 && tr < TH + 2 && tcx >= 15 && tcx <= TW + 16) {
                    const int idx = tr * OW + tcx;
                    atomicOr(reinterpret_cast<unsigned int *>(Cw + (idx & ~3)),
                             (1u << (8 - code)) << (8 * (idx & 3)));
                }
            };
            {
                const int n_agents = (int)misc[0];
                for (int a0 = 0; a0 < n_agents; a0 += NT) {
                    const int a = a0 + threadIdx.x;
                    bool is_blocked = false;
                    int oi = 0;
                    if (a < n_agents) {
                        oi = agents[a];
                        const int r = oi / OW - 1, cx = oi - (oi / OW) * OW;
                        const int x = x0 - 16 + cx, y = y0 - 2 + r;
                        const int g = O[oi];
                        const int code = forward_first(x, y, g, W, H,
                                                       [&](int dx, int dy) { return (int)O[oi + dy * OW + dx]; });
                        if (code < 0) {
                            is_blocked = true;
                        } else {
                            Pp[r * OW + cx] = (uint8_t)code;
                            if (code) claim_target(r, cx, code);
                        }
                    }
                    const int slot = warp_reserve(&misc[2], is_blocked ? 1 : 0);
                    if (is_blocked) blocked[slot] = (uint16_t)oi;
                }
            }
            consumer_sync();
            {
                const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
                const int n_blocked = (int)misc[2];
                for (int a = threadIdx.x; a < n_blocked; a += NT) {
                    const int oi = blocked[a];
                    const int r = oi / OW - 1, cx = oi - (oi / OW) * OW;
                    const int x = x0 - 16 + cx, y = y0 - 2 + r;
                    const int g = O[oi];
                    const uint64_t cell = (uint64_t)y * (uint64_t)W + (uint64_t)x;
                    const float *tc = (g == 2 ? tB : tA) + (r + 1) * TWH + (cx - 12);
                    const int code = propose(
                        x, y, g, W, H, cell, t, d.seed, rp,
                        [&](int dx, int dy) { return (int)O[oi + dy * OW + dx]; }, tc, TWH);
                    Pp[r * OW + cx] = (uint8_t)code;
                    if (code) claim_target(r, cx, code);
                }
            }
            consumer_sync();

            // Phase 1c: one winner per claimed cell of the tile and its 1-ring
            // (Sec. IV.d).  A single claimant wins at once; cells with k >= 2
            // claimants are listed and draw claimant floor(r * k / 2^32) in scan
            // order from Philox stream 2 at the target cell, one cell per
            // thread.  Tile cells that receive an agent go to the move list.
            for (int i0 = 0; i0 < (TH + 2) * NWC; i0 += NT) {
                const int i = i0 + threadIdx.x;
                uint32_t into = 0;   // bit b: byte b is a tile cell receiving an agent
                uint32_t multi = 0;  // bit b: byte b has two or more claimants
                int r = 0, wc = 0;
                if (i < (TH + 2) * NWC) {
                    r = i / NWC;
                    wc = WC0 + i % NWC;
                    uint32_t *cp = reinterpret_cast<uint32_t *>(Cw + r * OW + 4 * wc);
                    const uint32_t m4 = *cp;
                    if (m4) {
                        uint32_t w4 = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const uint32_t m = (m4 >> (8 * b)) & 255u;
                            if (!m) continue;
                            const int cx = 4 * wc + b;
                            if (m & (m - 1u)) {
                                multi |= 1u << b;
                                w4 |= m << (8 * b);  // resolved below
                            } else {
                                w4 |= (uint32_t)__ffs(m) << (8 * b);
                            }
                            if (r >= 1 && r <= TH && cx >= 16 && cx < TW + 16) into |= 1u << b;
                        }
                        *cp = w4;
                    }
                }
                int slot = warp_reserve(&misc[1], __popc(into));
                for (int b = 0; b < 4; ++b)
                    if (into & (1u << b)) moves[slot++] = (uint16_t)((r - 1) * TW + 4 * wc + b - 16);
                slot = warp_reserve(&misc[3], __popc(multi));
                for (int b = 0; b < 4; ++b)
                    if (multi & (1u << b)) conflicts[slot++] = (uint16_t)(r * OW + 4 * wc + b);
            }
            consumer_sync();
            {
                const int n_conf = (int)misc[3];
                for (int ci = threadIdx.x; ci < n_conf; ci += NT) {
                    const int idx = conflicts[ci];
                    const int r = idx / OW, cx = idx - r * OW;
                    const uint32_t m = Cw[idx];
                    const uint32_t k = (uint32_t)__popc(m);
                    const int x = x0 - 16 + cx, y = y0 - 1 + r;
                    const uint32_t j =
                        pick_claimant(m, k, (uint64_t)y * (uint64_t)W + (uint64_t)x, t, d.seed);
                    Cw[idx] = (uint8_t)((j + 1u) | 0x10u);
                }
            }
            consumer_sync();

            // Phase 2a: per-agent bookkeeping of the moves into tile cells (ids,
            // tour length, arrival), one move per thread.  Within a step a cell
            // that is read as a source (occupied at t) is never written as a
            // target (empty at t), so the id loads may take the non-coherent
            // path and all of them are in flight together.  With a constant
            // deposit nothing below depends on this pass; with Eq. 5 the
            // deposits go to shared memory first.
            {
                const int n_moves = (int)misc[1];
                for (int mi = threadIdx.x; mi < n_moves; mi += NT) {
                    const int li = moves[mi];
                    const int iy = li / TW, ix = li - iy * TW;
                    const int x = x0 + ix, y = y0 + iy;
                    const int w = Cw[(iy + 1) * OW + ix + 16];
                    const int j = (w & 15) - 1;
                    const int dx = kCodeDX[j + 1], dy = kCodeDY[j + 1];
                    const int inc = O[(iy + 3 + dy) * OW + ix + 16 + dx];
                    const uint64_t cell = (uint64_t)y * (uint64_t)W + (uint64_t)x;
                    const uint32_t id = __ldg(d.ids + cell + (int64_t)dy * W + dx);
                    const uint64_t rv = apply_move_id(d, cell, id, inc, x, dx != 0 && dy != 0, t);
                    ++cnt.moved;
                    cnt.conflicts += (w >> 4) & 1;
                    const unsigned crossed = (unsigned)(rv >> 32);
                    if (inc == 1) cnt.crossed_a += crossed; else cnt.crossed_b += crossed;
                    if (!const_deposit) depv[li] = __uint_as_float((uint32_t)rv);
                }
            }
            if (!const_deposit) consumer_sync();

            // Phase 2b: per group of 4 tile cells: the winner's group enters each
            // empty cell, cells whose agent won are vacated, pheromone evaporates
            // (Eq. 3) and the deposit lands in the mover's own plane (Eq. 4).
            // Agents at t+1 on the tile's border mark the neighbouring tiles
            // they touch: bit (dy + 1) * 3 + (dx + 1) for tile (tx + dx, ty + dy).
            uint32_t mark = 0;
            {
                const float q = d.q;
                const float dep0 = d.deposit;
                uint8_t *occ_dst = d.occ[p ^ 1];
                float *tA_dst = d.tau[0][p ^ 1];
                float *tB_dst = d.tau[1][p ^ 1];
                for (int gi = threadIdx.x; gi < TH * GW; gi += NT) {
                    const int iy = gi / GW, gx = gi - iy * GW;
                    const int x = x0 + 4 * gx, y = y0 + iy;
                    if (x >= W || y >= H) continue;
                    const int cxo = 16 + 4 * gx;
                    const uint32_t o4 = *reinterpret_cast<const uint32_t *>(O + (iy + 3) * OW + cxo);
                    const uint32_t w4 = *reinterpret_cast<const uint32_t *>(Cw + (iy + 1) * OW + cxo);
                    const uint64_t cell0 = (uint64_t)y * (uint64_t)W + (uint64_t)x;
                    float va[4], vb[4];
                    if (aco) {
                        const int ti = (iy + 3) * TWH + 4 * gx + 4;
                        const float4 a4 = *reinterpret_cast<const float4 *>(tA + ti);
                        const float4 b4 = *reinterpret_cast<const float4 *>(tB + ti);
                        va[0] = __fmul_rn(a4.x, q); va[1] = __fmul_rn(a4.y, q);
                        va[2] = __fmul_rn(a4.z, q); va[3] = __fmul_rn(a4.w, q);
                        vb[0] = __fmul_rn(b4.x, q); vb[1] = __fmul_rn(b4.y, q);
                        vb[2] = __fmul_rn(b4.z, q); vb[3] = __fmul_rn(b4.w, q);
                    }
                    uint32_t n4 = o4;
                    if (o4 | w4) {
                        const uint32_t p4 = *reinterpret_cast<const uint32_t *>(Pp + (iy + 2) * OW + cxo);
                        n4 = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int o = (o4 >> (8 * b)) & 255u;
                            int no = o;
                            if (o == 0) {
                                const int w = (w4 >> (8 * b)) & 255u;
                                if (w) {
                                    const int j = (w & 15) - 1;
                                    no = O[(iy + 3 + kCodeDY[j + 1]) * OW + cxo + b + kCodeDX[j + 1]];
                                    if (aco) {
                                        const float dep = const_deposit ? dep0 : depv[iy * TW + 4 * gx + b];
                                        if (no == 1) va[b] = __fadd_rn(va[b], dep);
                                        else vb[b] = __fadd_rn(vb[b], dep);
                                    }
                                }
                            } else {
                                const int code = (p4 >> (8 * b)) & 255u;
                                if (code) {
                                    const int wt = Cw[(iy + 1 + kCodeDY[code]) * OW + cxo + b + kCodeDX[code]];
                                    if ((wt & 15) == 9 - code) no = 0;  // this agent won its target
                                }
                            }
                            n4 |= (uint32_t)no << (8 * b);
                        }
                    }
                    if (n4) {
                        const bool top = iy == 0, bottom = iy == TH - 1;
                        uint32_t mk = 1u << 4;
                        if (top) mk |= 1u << 1;
                        if (bottom) mk |= 1u << 7;
                        if (gx == 0 && (n4 & 255u)) {
                            mk |= 1u << 3;
                            if (top) mk |= 1u << 0;
                            if (bottom) mk |= 1u << 6;
                        }
                        if (gx == GW - 1 && (n4 >> 24)) {
                            mk |= 1u << 5;
                            if (top) mk |= 1u << 2;
                            if (bottom) mk |= 1u << 8;
                        }
                        mark |= mk;
                    }
                    *reinterpret_cast<uint32_t *>(occ_dst + cell0) = n4;
                    if (aco) {
                        *reinterpret_cast<float4 *>(tA_dst + cell0) = make_float4(va[0], va[1], va[2], va[3]);
                        *reinterpret_cast<float4 *>(tB_dst + cell0) = make_float4(vb[0], vb[1], vb[2], vb[3]);
                    }
                }
            }
            mark = __reduce_or_sync(0xffffffffu, mark);
            if (lane == 0 && mark) atomicOr(&misc[4], mark);
            // Every consumer is done with the stage and the work area.
            consumer_sync();
            if (lane == 0) mbar_arrive(&empty[st]);
            mark = misc[4];

            // Marks for the next step: lanes 0-8 of warp 0 set the flags of the
            // marked tiles; the tiles whose flag they set first join the next
            // step's list.
            if (mark && warp == 0) {
                const int tiles_y = d.tiles_y;
                bool mine = false;
                uint32_t nb = 0;
                if (lane < 9 && ((mark >> lane) & 1u)) {
                    const int nx = tx + lane % 3 - 1, ny = ty + lane / 3 - 1;
                    if (nx >= 0 && nx < tiles_x && ny >= 0 && ny < tiles_y) {
                        nb = (item - local) + (uint32_t)ny * (uint32_t)tiles_x + (uint32_t)nx;
                        const uint32_t bit = 1u << (nb & 31u);
                        mine = (atomicOr(&F_next[nb >> 5], bit) & bit) == 0;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (m) {
                    uint32_t b0 = 0;
                    if (lane == 0) b0 = atomicAdd(n_next, (unsigned int)__popc(m));
                    b0 = __shfl_sync(0xffffffffu, b0, 0);
                    if (mine) L_next[b0 + (uint32_t)__popc(m & ((1u << lane) - 1u))] = nb;
                }
            }
            flush_counts(d, cnt, local);
            st = (st + 1) % kStages;
        }
        if (failed && threadIdx.x == 0) {
            // give a copy still in flight for the other stage a bounded chance
            // to land before the CTA leaves
            const int o = (st + 1) % kStages;
            (void)mbar_wait_bounded(&full[o], (fphase >> o) & 1u);
        }
    }
    // A wait that gave up is reported to every scenario of the work list.
    if (failed && (threadIdx.x == 0 || threadIdx.x == kFusedConsumers))
        for (int i = 0; i < n_scen; ++i) atomicExch(descs[i].error, kErrTimeout);

    // The last CTA to finish re-arms the work counters and rotates the
    // activity generations for the next launch.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(&act->ticket, 1u);
        if (ticket == gridDim.x - 1) {
            act->work = 0u;
            act->work_nat = 0u;
            act->n_act[(ph + 2u) % 3u] = 0u;
            act->reset = 0u;
            act->phase = (ph + 1u) % 3u;
            act->ticket = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled two-kernel step (the default variant)
//
// K1 propose_tile_kernel: one CTA per 128 x TH tile; TMA stages the tile's
// occupancy with a 1-cell halo (16 columns either side for the 16-byte rule);
// each thread owns 16 consecutive cells of a row and writes their proposal
// codes to the proposal plane with one 16-byte store.
// K2 resolve_tile_kernel: one CTA per tile; TMA stages the proposal plane with
// a 2-cell halo and the occupancy with a 1-cell halo while each thread's
// pheromone loads (4 x float4 per plane) are already in flight.  Pheromone
// evaporates (Eq. 3) and is stored at once; a 3 x 18 window test on the
// proposals sends every 16-cell segment with no nearby proposal down a fast
// path (occupancy unchanged); otherwise each empty cell gathers its winner
// (Sec. IV.d) and each agent checks whether it won its target.  A move
// overwrites the one pheromone value that receives a deposit (Eq. 4/5).
// ---------------------------------------------------------------------------
constexpr int kPipeTileW = 128;
constexpr int kPipeRowB = kPipeTileW + 32;  // staged row: 16-column halo either side

// Bit 8*b + 7 set for every nonzero byte b of v (bytes tested without carries
// between them).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t v)
{
    return (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
}

// One thread waits (bounded) for the TMA copies behind `bar`; the rest of the
// CTA blocks in the barrier instead of polling.  Returns false for every
// thread when the wait gave up.
__device__ __forceinline__ bool cta_wait_tma(uint64_t *bar, uint32_t parity,
                                             unsigned long long limit)
{
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait_bounded(bar, parity, limit ? (long long)limit : kWaitCycles);
    return __syncthreads_and(ok);
}

template <int TH>
__global__ void __launch_bounds__(8 * TH)
propose_tile_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                    int n_scen, int t_off)
{
    constexpr int NT = 8 * TH, RB = kPipeRowB, TW = kPipeTileW;
    __shared__ __align__(128) uint8_t occ_s[(TH + 2) * RB];
    __shared__ __align__(128) uint8_t code_s[TH * TW];
    __shared__ __align__(128) ScenarioDesc hdr_s;  // header part only
    __shared__ uint16_t blocked[TH * TW];
    __shared__ unsigned int n_blocked;
    __shared__ __align__(8) uint64_t bar;
    const uint32_t item = blockIdx.x;
    const int s = scenario_of(tile_prefix, n_scen, item);
    const ScenarioDesc *gd = descs + s;
    if (threadIdx.x == 32) {
        prefetch_tensormap(&gd->map_occ[0]);
        prefetch_tensormap(&gd->map_occ[1]);
    }
    // Everything below reads the previous kernel's results (the occupancy
    // of the previous resolution, the step index of an advance): wait for it,
    // then let the resolution kernel of this step start its prologue.
    pdl_wait();
    pdl_trigger();
    load_header(&hdr_s, gd);
    __syncthreads();
    const ScenarioDesc &d = hdr_s;
    const uint64_t t = d.step + (uint64_t)t_off;
    if (t >= d.end_step) return;
    const uint32_t local = item - __ldg(tile_prefix + s);
    const int ty = (int)(local / (uint32_t)d.tiles_x), tx = (int)(local % (uint32_t)d.tiles_x);
    const int x0 = tx * TW, y0 = ty * TH;
    const int p = (int)(t & 1);
    if (threadIdx.x == 0) {
        n_blocked = 0;
        mbar_init(&bar, 1);
        fence_mbarrier_init();
        mbar_arrive_expect_tx(&bar, (TH + 2) * RB);
        tma_load_2d(occ_s, &gd->map_occ[p], x0 - 16, y0 - 1, &bar);
    }
    __syncthreads();
    if (!cta_wait_tma(&bar, 0, d.wait_cycles)) {
        if (threadIdx.x == 0) atomicExch(d.error, kErrTimeout);
        return;
    }
    const int W = d.W, H = d.H;
    const int r = threadIdx.x >> 3, seg = threadIdx.x & 7;
    const int y = y0 + r, x = x0 + 16 * seg;
    const int c0 = (r + 1) * RB + 16 + 16 * seg;

    // Pass 1 (owner thread): forward-first codes; blocked agents are listed.
    uint32_t blocked_mask = 0;
    uint4 codes = make_uint4(0u, 0u, 0u, 0u);
    const uint4 o = *reinterpret_cast<const uint4 *>(occ_s + c0);  // zero outside the grid
    if (o.x | o.y | o.z | o.w) {
        uint64_t lo = 0, hi = 0;
#pragma unroll 4
        for (int b = 0; b < 16; ++b) {
            const int g = occ_s[c0 + b];
            if (!g) continue;
            const int code = forward_first(x + b, y, g, W, H,
                                           [&](int dx, int dy) { return (int)occ_s[c0 + b + dy * RB + dx]; });
            if (code < 0) { blocked_mask |= 1u << b; continue; }
            if (b < 8) lo |= (uint64_t)code << (8 * b);
            else hi |= (uint64_t)code << (8 * (b - 8));
        }
        codes = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
    }
    *reinterpret_cast<uint4 *>(code_s + r * TW + 16 * seg) = codes;
    int slot = warp_reserve(&n_blocked, __popc(blocked_mask));
    while (blocked_mask) {
        const int b = __ffs(blocked_mask) - 1;
        blocked_mask &= blocked_mask - 1;
        blocked[slot++] = (uint16_t)(r * TW + 16 * seg + b);
    }
    __syncthreads();

    // Pass 2: the full rule for blocked agents, one agent per thread.
    {
        const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
        const int nb = (int)n_blocked;
        for (int i = threadIdx.x; i < nb; i += NT) {
            const int li = blocked[i];
            const int ly = li / TW, lx = li - ly * TW;
            const int xc = x0 + lx, yc = y0 + ly;
            const int oi = (ly + 1) * RB + 16 + lx;
            const int g = occ_s[oi];
            const uint64_t cell = (uint64_t)yc * (uint64_t)W + (uint64_t)xc;
            const float *tp = d.tau[g == 2 ? 1 : 0][p];
            code_s[li] = (uint8_t)propose(
                xc, yc, g, W, H, cell, t, d.seed, rp,
                [&](int dx, int dy) { return (int)occ_s[oi + dy * RB + dx]; },
                tp ? tp + cell : nullptr, W);
        }
    }
    // Each thread stores its 16 codes (cells outside the grid are skipped).
    __syncthreads();
    if (y < H && x < W)
        *reinterpret_cast<uint4 *>(d.prop + (uint64_t)y * (uint64_t)W + x) =
            *reinterpret_cast<const uint4 *>(code_s + r * TW + 16 * seg);
}

template <int TH>
__global__ void __launch_bounds__(8 * TH)
resolve_tile_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                    int n_scen, int t_off)
{
    constexpr int NT = 8 * TH, RB = kPipeRowB, TW = kPipeTileW;
    __shared__ __align__(128) float tau_s[2][TH * TW];
    __shared__ __align__(128) uint8_t prop_s[(TH + 4) * RB];  // rows y0-2 .. y0+TH+1
    __shared__ __align__(128) uint8_t occ_s[(TH + 2) * RB];   // rows y0-1 .. y0+TH
    __shared__ __align__(128) uint8_t win_s[(TH + 2) * RB];   // claim masks, then winners
    __shared__ uint16_t moves[TH * TW];                        // tile cells receiving an agent
    __shared__ unsigned int n_moves;
    __shared__ __align__(128) ScenarioDesc hdr_s;  // header part only
    __shared__ __align__(8) uint64_t bar;
    const uint32_t item = blockIdx.x;
    const int s = scenario_of(tile_prefix, n_scen, item);
    const ScenarioDesc *gd = descs + s;
    if (threadIdx.x == 32) {  // maps are fetched while the header is read
        prefetch_tensormap(&gd->map_prop);
        prefetch_tensormap(&gd->map_occ[0]);
        prefetch_tensormap(&gd->map_occ[1]);
        prefetch_tensormap(&gd->map_tau[0][0]);
        prefetch_tensormap(&gd->map_tau[0][1]);
        prefetch_tensormap(&gd->map_tau[1][0]);
        prefetch_tensormap(&gd->map_tau[1][1]);
    }
    load_header(&hdr_s, gd);
    // claim masks and the move list start empty
    for (int i = threadIdx.x; i < (TH + 2) * RB / 16; i += NT)
        reinterpret_cast<uint4 *>(win_s)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) n_moves = 0;
    __syncthreads();
    const ScenarioDesc &d = hdr_s;
    const uint64_t t = d.step + (uint64_t)t_off;
    Counts cnt;
    if (t >= d.end_step) {
        pdl_wait();
        pdl_trigger();
    } else {
        const uint32_t local = item - __ldg(tile_prefix + s);
        const int ty = (int)(local / (uint32_t)d.tiles_x), tx = (int)(local % (uint32_t)d.tiles_x);
        const int x0 = tx * TW, y0 = ty * TH;
        const int p = (int)(t & 1);
        const bool aco = d.model == 1;
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbarrier_init();
            if (!(d.test_flags & kTestSkipResolveLoads)) {
                // The occupancy and pheromone at t come from the resolution of
                // the step before, complete before this step's proposal kernel
                // started: they are copied while the proposal kernel still runs.
                mbar_arrive_expect_tx(&bar, (TH + 4) * RB + (TH + 2) * RB +
                                                (aco ? 2 * TH * TW * 4 : 0));
                tma_load_2d(occ_s, &gd->map_occ[p], x0 - 16, y0 - 1, &bar);
                if (aco) {
                    tma_load_2d(tau_s[0], &gd->map_tau[0][p], x0, y0, &bar);
                    tma_load_2d(tau_s[1], &gd->map_tau[1][p], x0, y0, &bar);
                }
                // the proposals are the proposal kernel's output
                pdl_wait();
                tma_load_2d(prop_s, &gd->map_prop, x0 - 16, y0 - 2, &bar);
            }
            // (test hook: no load issued and no arrival, so the wait below
            // runs out and nothing is in flight when the CTA returns)
        }
        pdl_wait();
        pdl_trigger();
        const int W = d.W, H = d.H;
        __syncthreads();  // barrier initialised
        if (!cta_wait_tma(&bar, 0, d.wait_cycles)) {
            if (threadIdx.x == 0) atomicExch(d.error, kErrTimeout);
        } else {
            // Claim pass: every proposal of the tile and its 2-ring that targets
            // the tile or its 1-ring sets bit (8 - code) of the target's mask
            // (the claimant's scan offset seen from the target).  Cells outside
            // the grid hold no proposal (TMA zero fill).  16 bytes per load;
            // only nonzero bytes are visited.
            constexpr int NQ = RB / 16;  // 16-byte columns per staged row
            // Evaporation of both pheromone tiles (Eq. 3), contiguous float4 per
            // thread (conflict-free); deposits are added after the barrier.
            if (aco) {
                const float q = d.q;
#pragma unroll
                for (int g = 0; g < 2; ++g)
                    for (int i = threadIdx.x; i < TH * TW / 4; i += NT) {
                        float4 *v4 = reinterpret_cast<float4 *>(tau_s[g]) + i;
                        const float4 v = *v4;
                        *v4 = make_float4(__fmul_rn(v.x, q), __fmul_rn(v.y, q), __fmul_rn(v.z, q),
                                          __fmul_rn(v.w, q));
                    }
            }
            for (int i = threadIdx.x; i < (TH + 4) * NQ; i += NT) {
                const int r = i / NQ, q0 = 16 * (i % NQ);
                const uint4 v = *reinterpret_cast<const uint4 *>(prop_s + r * RB + q0);
                const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    uint32_t nz = nonzero_bytes(vw[w]);
                    while (nz) {
                        const int b = (__ffs(nz) - 1) >> 3;
                        nz &= nz - 1;
                        const int cx = q0 + 4 * w + b;
                        if (cx < 14 || cx > TW + 17) continue;
                        const int code = (vw[w] >> (8 * b)) & 255u;
                        const int tr = r - 1 + kCodeDY[code];  // target row in win_s
                        const int tc = cx + kCodeDX[code];
                        if (tr >= 0 && tr < TH + 2 && tc >= 15 && tc <= TW + 16) {
                            const int idx = tr * RB + tc;
                            atomicOr(reinterpret_cast<unsigned int *>(win_s + (idx & ~3)),
                                     (1u << (8 - code)) << (8 * (idx & 3)));
                        }
                    }
                }
            }
            __syncthreads();

            // Winner pass (Sec. IV.d): the only claimant, or claimant
            // floor(r * k / 2^32) in scan order from Philox stream 2 at the
            // target cell; the byte becomes (scan index + 1) | 0x10 if k >= 2.
            for (int i = threadIdx.x; i < (TH + 2) * NQ; i += NT) {
                const int r = i / NQ, q0 = 16 * (i % NQ);
                uint4 *wp = reinterpret_cast<uint4 *>(win_s + r * RB + q0);
                const uint4 mv = *wp;
                if (!(mv.x | mv.y | mv.z | mv.w)) continue;
                uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    uint32_t nz = nonzero_bytes(mw[w]);
                    uint32_t out = 0;
                    while (nz) {
                        const int b = (__ffs(nz) - 1) >> 3;
                        nz &= nz - 1;
                        const uint32_t m = (mw[w] >> (8 * b)) & 255u;
                        const uint32_t k = (uint32_t)__popc(m);
                        uint32_t j;
                        if (k == 1) {
                            j = (uint32_t)(__ffs(m) - 1);
                        } else {
                            const int xc = x0 - 16 + q0 + 4 * w + b, yc = y0 - 1 + r;
                            j = pick_claimant(m, k, (uint64_t)yc * (uint64_t)W + (uint64_t)xc, t,
                                              d.seed);
                        }
                        out |= ((j + 1u) | (k >= 2 ? 0x10u : 0u)) << (8 * b);
                    }
                    mw[w] = out;
                }
                *wp = make_uint4(mw[0], mw[1], mw[2], mw[3]);
            }
            __syncthreads();

            // Owner pass, 16 cells per thread: an empty cell takes its winner's
            // group, an agent whose target chose it leaves.  Only cells with a
            // winner byte (empty, claimed) or a proposal (agents) can change.
            // Cells that receive an agent go to the move list.
            const int r = threadIdx.x >> 3, seg = threadIdx.x & 7;
            const int y = y0 + r, x = x0 + 16 * seg;
            const int li0 = r * TW + 16 * seg;
            const int co = (r + 1) * RB + 16 + 16 * seg;  // this segment in occ_s / win_s
            const int cp = (r + 2) * RB + 16 + 16 * seg;  // this segment in prop_s
            const uint4 o = *reinterpret_cast<const uint4 *>(occ_s + co);
            const uint4 w = *reinterpret_cast<const uint4 *>(win_s + co);
            const uint4 pr = *reinterpret_cast<const uint4 *>(prop_s + cp);
            uint4 no = o;
            uint32_t arrivals = 0;  // bit b: cell b of the segment receives an agent
            if (y < H && x < W && (w.x | w.y | w.z | w.w | pr.x | pr.y | pr.z | pr.w)) {
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
                const uint32_t pw[4] = {pr.x, pr.y, pr.z, pr.w};
                uint32_t nw[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t nz = nonzero_bytes(ww[q] | pw[q]);
                    while (nz) {
                        const int bb = (__ffs(nz) - 1) >> 3;
                        nz &= nz - 1;
                        const int b = 4 * q + bb;
                        const int wb = (ww[q] >> (8 * bb)) & 255u;
                        if (wb) {  // empty cell with a winner
                            const int j = (wb & 15) - 1;
                            nw[q] |= (uint32_t)occ_s[co + b + kCodeDY[j + 1] * RB + kCodeDX[j + 1]]
                                     << (8 * bb);
                            arrivals |= 1u << b;
                        } else {  // an agent with a proposal
                            const int code = (pw[q] >> (8 * bb)) & 255u;
                            const int wt = win_s[co + b + kCodeDY[code] * RB + kCodeDX[code]];
                            if ((wt & 15) == 9 - code)  // this agent won its target: it leaves
                                nw[q] &= ~(255u << (8 * bb));
                        }
                    }
                }
                no = make_uint4(nw[0], nw[1], nw[2], nw[3]);
            }
            if (y < H && x < W)
                *reinterpret_cast<uint4 *>(d.occ[p ^ 1] + (uint64_t)y * (uint64_t)W + x) = no;
            int slot = warp_reserve(&n_moves, __popc(arrivals));
            while (arrivals) {
                const int b = __ffs(arrivals) - 1;
                arrivals &= arrivals - 1;
                moves[slot++] = (uint16_t)(li0 + b);
            }
            __syncthreads();

            // Move pass, one move per thread (their id / arrival / tour round
            // trips overlap): the agent's id follows it, Eq. 5 extends its tour,
            // its first entry into the opposite band is recorded (Sec. VI), and
            // its deposit (Eq. 4/5) lands on the evaporated pheromone.
            const int nm = (int)n_moves;
            for (int i = threadIdx.x; i < nm; i += NT) {
                const int li = moves[i];
                const int ly = li / TW, lx = li - ly * TW;
                const int wb = win_s[(ly + 1) * RB + 16 + lx];
                const int j = (wb & 15) - 1;
                const int dx = kCodeDX[j + 1], dy = kCodeDY[j + 1];
                const int inc = occ_s[(ly + 1 + dy) * RB + 16 + lx + dx];
                const uint64_t cell = (uint64_t)(y0 + ly) * (uint64_t)W + (uint64_t)(x0 + lx);
                const uint64_t rv = apply_move(d, cell, cell + (int64_t)dy * W + dx, inc, x0 + lx,
                                               dx != 0 && dy != 0, t);
                ++cnt.moved;
                if (wb & 0x10) ++cnt.conflicts;
                const unsigned crossed = (unsigned)(rv >> 32);
                if (inc == 1) cnt.crossed_a += crossed; else cnt.crossed_b += crossed;
                if (aco) {
                    float *v = &tau_s[inc == 1 ? 0 : 1][li];
                    *v = __fadd_rn(*v, __uint_as_float((uint32_t)rv));
                }
            }
            // Pheromone leaves by 16-byte stores (which, unlike a bulk copy's
            // read of shared memory, do not hold the CTA back) once every
            // deposit is in.
            if (aco) {
                __syncthreads();
#pragma unroll
                for (int g = 0; g < 2; ++g)
                    for (int i = threadIdx.x; i < TH * TW / 4; i += NT) {
                        const int ry = i / (TW / 4), cx4 = 4 * (i % (TW / 4));
                        if (y0 + ry < H && x0 + cx4 < W)
                            *reinterpret_cast<float4 *>(d.tau[g][p ^ 1] + (uint64_t)(y0 + ry) * W +
                                                        x0 + cx4) =
                                reinterpret_cast<const float4 *>(tau_s[g])[i];
                    }
            }
        }
    }
    flush_counts(d, cnt, item - __ldg(tile_prefix + s));
}

// ---------------------------------------------------------------------------
// Two-pass step (proposal plane in HBM)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
propose_plane_kernel(const ScenarioDesc *__restrict__ dp, uint8_t *__restrict__ prop, int t_off)
{
    const ScenarioDesc &d = *dp;
    const uint64_t t = d.step + (uint64_t)t_off;
    if (t >= d.end_step) return;
    const int W = d.W, H = d.H;
    const int p = (int)(t & 1);
    const uint8_t *occ = d.occ[p];
    const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};
    const size_t cells = (size_t)W * H;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x) {
        const int g = occ[c];
        int code = 0;
        if (g) {
            const int x = (int)(c % (size_t)W), y = (int)(c / (size_t)W);
            const float *tp = d.tau[g == 2 ? 1 : 0][p];
            code = propose(
                x, y, g, W, H, (uint64_t)c, t, d.seed, rp,
                [&](int dx, int dy) { return (int)occ[(int64_t)c + (int64_t)dy * W + dx]; },
                tp ? tp + c : nullptr, W);
        }
        prop[c] = (uint8_t)code;
    }
}

__global__ void __launch_bounds__(kThreads)
resolve_plane_kernel(const ScenarioDesc *__restrict__ dp, const uint8_t *__restrict__ prop,
                     int t_off)
{
    const ScenarioDesc &d = *dp;
    const uint64_t t = d.step + (uint64_t)t_off;
    if (t >= d.end_step) return;
    const int W = d.W, H = d.H;
    const int p = (int)(t & 1);
    const uint8_t *occ = d.occ[p];
    uint8_t *occ_dst = d.occ[p ^ 1];
    const size_t cells = (size_t)W * H;
    const float q = d.q;
    Counts cnt;
    // every thread runs the same number of iterations so that the warp-wide
    // counter reduction below sees all 32 lanes
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x; base < cells; base += stride) {
        const size_t c = base + threadIdx.x;
        if (c < cells) {
            const int x = (int)(c % (size_t)W), y = (int)(c / (size_t)W);
            int incoming;
            float dep;
            const int no = resolve_cell(
                d, x, y, (uint64_t)c, t, occ[c],
                [&](int dx, int dy) { return (int)occ[(int64_t)c + (int64_t)dy * W + dx]; },
                [&](int dx, int dy) { return (int)prop[(int64_t)c + (int64_t)dy * W + dx]; }, cnt,
                incoming, dep);
            occ_dst[c] = (uint8_t)no;
            if (d.model == 1) {
                float a = __fmul_rn(d.tau[0][p][c], q);
                float b = __fmul_rn(d.tau[1][p][c], q);
                if (incoming == 1) a = __fadd_rn(a, dep);
                else if (incoming == 2) b = __fadd_rn(b, dep);
                d.tau[0][p ^ 1][c] = a;
                d.tau[1][p ^ 1][c] = b;
            }
        }
        flush_counts(d, cnt, blockIdx.x);  // one counter slot per CTA
    }
}

__global__ void advance_kernel(const ScenarioDesc *__restrict__ descs, int n, int k)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ScenarioDesc *md = const_cast<ScenarioDesc *>(descs);
    unsigned long long v = md[i].step + (unsigned long long)k;
    if (v > md[i].end_step) v = md[i].end_step;
    md[i].step = v;
}

// Totals of one scenario's counter slots (integer sums: order-free).
__global__ void __launch_bounds__(256) sum_slots_kernel(const ScenarioDesc *__restrict__ dp,
                                                        unsigned long long *__restrict__ out)
{
    const ScenarioDesc &d = *dp;
    __shared__ unsigned long long red[kNumCounters][8];
    unsigned long long acc[kNumCounters] = {0, 0, 0, 0};
    for (uint32_t i = threadIdx.x; i < d.n_slots; i += blockDim.x)
        for (int k = 0; k < kNumCounters; ++k) acc[k] += d.part[(size_t)i * kNumCounters + k];
    for (int k = 0; k < kNumCounters; ++k) {
        unsigned long long v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumCounters) {
        unsigned long long v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        out[threadIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__global__ void grid_counts_kernel(const ScenarioDesc *__restrict__ dp, int parity,
                                   unsigned int *__restrict__ out)
{
    const ScenarioDesc &d = *dp;
    const int W = d.W;
    const size_t cells = (size_t)W * d.H;
    const uint8_t *occ = d.occ[parity];
    unsigned a = 0, b = 0, pa = 0, pb = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x; base < cells; base += stride) {
        const size_t c = base + threadIdx.x;
        if (c < cells) {
            const int g = occ[c];
            const int x = (int)(c % (size_t)W);
            a += g == 1;
            b += g == 2;
            pa += (g == 1) & (x == W - 1);
            pb += (g == 2) & (x == 0);
        }
    }
    a = __reduce_add_sync(0xffffffffu, a);
    b = __reduce_add_sync(0xffffffffu, b);
    pa = __reduce_add_sync(0xffffffffu, pa);
    pb = __reduce_add_sync(0xffffffffu, pb);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&out[0], a);
        if (b) atomicAdd(&out[1], b);
        if (pa) atomicAdd(&out[2], pa);
        if (pb) atomicAdd(&out[3], pb);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int grid_for(size_t work, int threads, int cap = 4096)
{
    size_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

cudaError_t launch_init(const ScenarioDesc *d_descs, int n, int max_cells, int max_agents,
                        cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const size_t work = (size_t)(max_cells > max_agents ? max_cells : max_agents);
    dim3 grid(grid_for(work, kThreads, 1024), (unsigned)n);
    init_kernel<<<grid, kThreads, 0, stream>>>(d_descs);
    return cudaGetLastError();
}

cudaError_t launch_place(const ScenarioDesc *d_descs, int n, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    place_kernel<<<2 * n, 1024, 0, stream>>>(d_descs);
    return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t ensure_fused_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<TW, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FusedLayout<TW, TH>::SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int TW, int TH>
static cudaError_t launch_fused_t(const ScenarioDesc *d_descs, const uint32_t *d_prefix, int n,
                                  uint32_t total, int t_off, ActivityCtl *act, int grid,
                                  cudaStream_t stream)
{
    cudaError_t e = ensure_fused_attr<TW, TH>();
    if (e != cudaSuccess) return e;
    fused_step_kernel<TW, TH><<<grid, kFusedThreads, FusedLayout<TW, TH>::SMEM, stream>>>(
        d_descs, d_prefix, n, total, t_off, act);
    return cudaGetLastError();
}

template <int TW, int TH>
static int blocks_per_sm_t()
{
    if (ensure_fused_attr<TW, TH>() != cudaSuccess) return 1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fused_step_kernel<TW, TH>, kFusedThreads,
                                                      FusedLayout<TW, TH>::SMEM) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

#define PEDSIM_TILES(X) X(32, 16) X(64, 8) X(64, 16) X(128, 8) X(128, 16)

bool tile_supported(int tile_w, int tile_h)
{
#define PEDSIM_TILE_OK(w, h) if (tile_w == w && tile_h == h) return true;
    PEDSIM_TILES(PEDSIM_TILE_OK)
#undef PEDSIM_TILE_OK
    return false;
}

cudaError_t launch_fused_step(const ScenarioDesc *d_descs, const uint32_t *d_tile_prefix, int n,
                              uint32_t total_tiles, int t_off, int tile_w, int tile_h, int grid,
                              ActivityCtl *act, cudaStream_t stream)
{
#define PEDSIM_TILE_LAUNCH(w, h)                                                               \
    if (tile_w == w && tile_h == h)                                                            \
        return launch_fused_t<w, h>(d_descs, d_tile_prefix, n, total_tiles, t_off, act, grid,   \
                                    stream);
    PEDSIM_TILES(PEDSIM_TILE_LAUNCH)
#undef PEDSIM_TILE_LAUNCH
    return cudaErrorInvalidValue;
}

int fused_blocks_per_sm(int tile_w, int tile_h)
{
#define PEDSIM_TILE_OCC(w, h) if (tile_w == w && tile_h == h) return blocks_per_sm_t<w, h>();
    PEDSIM_TILES(PEDSIM_TILE_OCC)
#undef PEDSIM_TILE_OCC
    return 1;
}

int fused_threads() { return kFusedThreads; }

bool pipeline_tile_supported(int tile_w, int tile_h)
{
    return tile_w == kPipeTileW && (tile_h == 8 || tile_h == 16);
}

cudaError_t launch_pipeline_step(const ScenarioDesc *d_descs, const uint32_t *d_tile_prefix, int n,
                                 uint32_t total_tiles, int t_off, int tile_h, cudaStream_t stream)
{
#define PEDSIM_PIPE(TH)                                                                        \
    if (tile_h == TH) {                                                                        \
        cudaError_t e = launch_pdl(propose_tile_kernel<TH>, total_tiles, 8 * TH, stream, d_descs, \
                                   d_tile_prefix, n, t_off);                                   \
        if (e != cudaSuccess) return e;                                                        \
        return launch_pdl(resolve_tile_kernel<TH>, total_tiles, 8 * TH, stream, d_descs,       \
                          d_tile_prefix, n, t_off);                                            \
    }
    PEDSIM_PIPE(8)
    PEDSIM_PIPE(16)
#undef PEDSIM_PIPE
    return cudaErrorInvalidValue;
}

int two_pass_grid(int W, int H) { return grid_for((size_t)W * H, kThreads, 152 * 16); }

cudaError_t launch_two_pass_step(const ScenarioDesc *d_desc, uint8_t *d_prop, int W, int H,
                                 int t_off, cudaStream_t stream)
{
    const int grid = two_pass_grid(W, H);
    propose_plane_kernel<<<grid, kThreads, 0, stream>>>(d_desc, d_prop, t_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resolve_plane_kernel<<<grid, kThreads, 0, stream>>>(d_desc, d_prop, t_off);
    return cudaGetLastError();
}

cudaError_t launch_advance(const ScenarioDesc *d_descs, int n, int k, cudaStream_t stream)
{
    if (n <= 0 || k == 0) return cudaSuccess;
    advance_kernel<<<(n + 255) / 256, 256, 0, stream>>>(d_descs, n, k);
    return cudaGetLastError();
}

cudaError_t launch_sum_slots(const ScenarioDesc *d_desc, unsigned long long *d_out,
                             cudaStream_t stream)
{
    sum_slots_kernel<<<1, 256, 0, stream>>>(d_desc, d_out);
    return cudaGetLastError();
}

cudaError_t launch_grid_counts(const ScenarioDesc *d_desc, int parity, int cells,
                               unsigned int *d_out, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_out, 0, kGridCounts * sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    grid_counts_kernel<<<grid_for((size_t)cells, kThreads, 1024), kThreads, 0, stream>>>(d_desc, parity,
                                                                                    d_out);
    return cudaGetLastError();
}

}  // namespace pedsim
