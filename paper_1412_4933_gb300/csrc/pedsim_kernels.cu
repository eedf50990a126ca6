// CUDA kernels of the GB300 pedestrian cellular automaton (sm_103a).
//
//   init_kernel        clear planes, fill pheromone with tau0, zero arrays
//   place_kernel       random placement in the edge bands (Sec. IV.a)
//   fused_step_kernel  one synchronous step (Sec. IV.b-d) in a single pass:
//                      persistent CTAs walk the (scenario, tile) work list;
//                      per tile a TMA copy stages the occupancy tile with a
//                      3-cell halo (16 columns either side, for the 16-byte
//                      TMA rule) and the two pheromone tiles in shared memory,
//                      double-buffered behind mbarriers; proposals of the tile
//                      plus a 2-cell ring are computed into shared memory, then
//                      every tile cell resolves (gather), evaporates (Eq. 3),
//                      deposits (Eq. 4/5) and counts
//   propose_plane_kernel + resolve_plane_kernel
//                      the same step in two passes through a proposal plane in
//                      HBM (baseline and cross-check of the fused pass)
//   advance_kernel     step index += k
//   grid_counts_kernel / mask_ids_kernel    read-back helpers
#include "pedsim_internal.h"
#include "pedsim_rules.cuh"

namespace pedsim {

constexpr int kThreads = 256;
constexpr int kErrTimeout = -110;
// A bounded wait gives up after this many SM clock cycles (about 2 s at the
// 2.07 GHz maximum clock).
constexpr long long kWaitCycles = 4000000000ll;

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and TMA (cp.async.bulk.tensor)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity; false after kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Shared per-cell resolution (Sec. IV.d), used by both step variants.
// occ_at(dx, dy): occupancy at t; prop_at(dx, dy): proposal code at t.
// Returns the occupancy byte at t+1 and reports the group of an agent that
// entered this cell (0 if none) plus the deposit it leaves.
// ---------------------------------------------------------------------------
struct Counts {
    unsigned moved = 0, conflicts = 0, crossed_a = 0, crossed_b = 0;
};

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

__device__ __forceinline__ void flush_counts(const ScenarioDesc &d, Counts &c)
{
    const unsigned m = __reduce_add_sync(0xffffffffu, c.moved);
    const unsigned k = __reduce_add_sync(0xffffffffu, c.conflicts);
    const unsigned a = __reduce_add_sync(0xffffffffu, c.crossed_a);
    const unsigned b = __reduce_add_sync(0xffffffffu, c.crossed_b);
    if ((threadIdx.x & 31) == 0) {
        if (m) atomicAdd(&d.counters[kMoved], (unsigned long long)m);
        if (k) atomicAdd(&d.counters[kConflicts], (unsigned long long)k);
        if (a) atomicAdd(&d.counters[kCrossedA], (unsigned long long)a);
        if (b) atomicAdd(&d.counters[kCrossedB], (unsigned long long)b);
    }
    c = Counts{};
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
        }
    }
    const size_t agents = 2 * (size_t)d.n_per_side + 1;
    for (size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x; a < agents; a += stride) {
        d.arrival[a] = 0;
        if (d.tour) d.tour[a] = 0.0f;
    }
    if (blockIdx.x == 0 && threadIdx.x < kNumCounters) d.counters[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d.step = 0;
        *d.error = 0;
    }
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

// ---------------------------------------------------------------------------
// Fused single-pass step
// ---------------------------------------------------------------------------
template <int TW, int TH>
struct FusedLayout {
    static constexpr int OW = TW + 32;        // occupancy tile row, 16-col halo each side
    static constexpr int OH = TH + 6;         // 3-row halo above and below
    static constexpr int PW = TW + 4;         // proposal region: tile + 2-cell ring
    static constexpr int PH = TH + 4;
    static constexpr int OCC_BYTES = ((OH * OW + 127) / 128) * 128;
    static constexpr int TAU_BYTES = TH * TW * 4;
    static constexpr int PROP_BYTES = ((PH * PW + 15) / 16) * 16;
    static constexpr int OFF_TAU = 2 * OCC_BYTES;                 // [stage][group]
    static constexpr int OFF_PROP = OFF_TAU + 4 * TAU_BYTES;
    static constexpr int OFF_BAR = OFF_PROP + PROP_BYTES;
    static constexpr int SMEM = OFF_BAR + 2 * 8 + 128;  // + slack to align the base
    static_assert(OW <= 256 && OH <= 256 && TW <= 256 && TH <= 256, "TMA box limit");
    static_assert((TAU_BYTES % 128) == 0, "tau tile alignment");
};

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

template <int TW, int TH>
__global__ void __launch_bounds__(kThreads)
fused_step_kernel(const ScenarioDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                  int n_scen, uint32_t total, int t_off)
{
    using Lay = FusedLayout<TW, TH>;
    constexpr int OW = Lay::OW, PW = Lay::PW, PH = Lay::PH;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // TMA destinations need 128-byte alignment: align the base explicitly
    uint8_t *const smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint8_t *const occ_s0 = smem;
    uint8_t *const prop_s = smem + Lay::OFF_PROP;
    uint64_t *const bar = reinterpret_cast<uint64_t *>(smem + Lay::OFF_BAR);
    auto occ_stage = [&](int st) { return smem + st * Lay::OCC_BYTES; };
    auto tau_stage = [&](int st, int g) {
        return reinterpret_cast<float *>(smem + Lay::OFF_TAU + (st * 2 + g) * Lay::TAU_BYTES);
    };
    (void)occ_s0;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbarrier_init();
    }
    __syncthreads();

    // Issues the TMA copies of one work item into a stage (thread 0 only).
    auto issue = [&](uint32_t item, int st) {
        const int s = scenario_of(tile_prefix, n_scen, item);
        const ScenarioDesc *d = descs + s;
        const uint64_t t = *d->step + (uint64_t)t_off;
        if (t >= d->end_step) return;
        const uint32_t local = item - __ldg(tile_prefix + s);
        const int ty = (int)(local / (uint32_t)d->tiles_x), tx = (int)(local % (uint32_t)d->tiles_x);
        const int p = (int)(t & 1);
        const bool aco = d->model == 1;
        mbar_arrive_expect_tx(&bar[st], Lay::OH * OW + (aco ? 2 * Lay::TAU_BYTES : 0));
        tma_load_2d(occ_stage(st), &d->map_occ[p], tx * TW - 16, ty * TH - 3, &bar[st]);
        if (aco) {
            tma_load_2d(tau_stage(st, 0), &d->map_tau[0][p], tx * TW, ty * TH, &bar[st]);
            tma_load_2d(tau_stage(st, 1), &d->map_tau[1][p], tx * TW, ty * TH, &bar[st]);
        }
    };

    uint32_t phase_bits = 0;
    uint32_t item = blockIdx.x;
    int st = 0;
    if (threadIdx.x == 0 && item < total) issue(item, 0);
    for (; item < total; item += gridDim.x, st ^= 1) {
        const uint32_t next = item + gridDim.x;
        if (threadIdx.x == 0 && next < total) {
            fence_proxy_async_smem();
            issue(next, st ^ 1);
        }
        const int s = scenario_of(tile_prefix, n_scen, item);
        const ScenarioDesc &d = descs[s];
        const uint64_t t = *d.step + (uint64_t)t_off;
        if (t >= d.end_step) continue;  // uniform: nothing was issued for it

        const bool ok = mbar_wait_bounded(&bar[st], (phase_bits >> st) & 1u);
        phase_bits ^= 1u << st;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicExch(d.error, kErrTimeout);
            // give the copy that may still be in flight for the next item a
            // bounded chance to land before the CTA exits
            if (next < total) (void)mbar_wait_bounded(&bar[st ^ 1], (phase_bits >> (st ^ 1)) & 1u);
            return;
        }

        const int W = d.W, H = d.H;
        const uint32_t local = item - __ldg(tile_prefix + s);
        const int ty = (int)(local / (uint32_t)d.tiles_x), tx = (int)(local % (uint32_t)d.tiles_x);
        const int x0 = tx * TW, y0 = ty * TH;
        const int p = (int)(t & 1);
        const uint8_t *O = occ_stage(st);
        const RuleParams rp{d.model, d.alpha, d.beta, d.lem_scale};

        // Phase 1: proposals of every agent in the tile and a 2-cell ring.
        for (int i = threadIdx.x; i < PH * PW; i += kThreads) {
            const int ry = i / PW, rx = i - ry * PW;
            const int x = x0 - 2 + rx, y = y0 - 2 + ry;
            int code = 0;
            if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H) {
                const int oi = (ry + 1) * OW + (rx + 14);
                const int g = O[oi];
                if (g) {
                    const uint64_t cell = (uint64_t)y * W + x;
                    const float *tp = d.tau[g - 1 < 2 ? g - 1 : 0][p];
                    code = propose(
                        x, y, g, W, H, cell, t, d.seed, rp,
                        [&](int dx, int dy) { return (int)O[oi + dy * OW + dx]; },
                        [&](int dx, int dy) { return __ldg(tp + (int64_t)cell + (int64_t)dy * W + dx); });
                }
            }
            prop_s[i] = (uint8_t)code;
        }
        __syncthreads();

        // Phase 2: gather, move, evaporate + deposit, count.
        Counts cnt;
        const float q = d.q;
        const bool aco = d.model == 1;
        const float *tA = tau_stage(st, 0);
        const float *tB = tau_stage(st, 1);
        uint8_t *occ_dst = d.occ[p ^ 1];
        float *tA_dst = d.tau[0][p ^ 1];
        float *tB_dst = d.tau[1][p ^ 1];
        for (int i = threadIdx.x; i < TH * TW; i += kThreads) {
            const int iy = i / TW, ix = i - iy * TW;
            const int x = x0 + ix, y = y0 + iy;
            if (x >= W || y >= H) continue;
            const int oi = (iy + 3) * OW + ix + 16;
            const int pi = (iy + 2) * PW + ix + 2;
            const uint64_t cell = (uint64_t)y * W + x;
            int incoming;
            float dep;
            const int no = resolve_cell(
                d, x, y, cell, t, O[oi], [&](int dx, int dy) { return (int)O[oi + dy * OW + dx]; },
                [&](int dx, int dy) { return (int)prop_s[pi + dy * PW + dx]; }, cnt, incoming, dep);
            occ_dst[cell] = (uint8_t)no;
            if (aco) {
                float a = __fmul_rn(tA[i], q);
                float b = __fmul_rn(tB[i], q);
                if (incoming == 1) a = __fadd_rn(a, dep);
                else if (incoming == 2) b = __fadd_rn(b, dep);
                tA_dst[cell] = a;
                tB_dst[cell] = b;
            }
        }
        flush_counts(d, cnt);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Two-pass step (proposal plane in HBM)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
propose_plane_kernel(const ScenarioDesc *__restrict__ dp, uint8_t *__restrict__ prop, int t_off)
{
    const ScenarioDesc &d = *dp;
    const uint64_t t = *d.step + (uint64_t)t_off;
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
            const float *tp = d.tau[g - 1 < 2 ? g - 1 : 0][p];
            code = propose(
                x, y, g, W, H, (uint64_t)c, t, d.seed, rp,
                [&](int dx, int dy) { return (int)occ[(int64_t)c + (int64_t)dy * W + dx]; },
                [&](int dx, int dy) { return tp[(int64_t)c + (int64_t)dy * W + dx]; });
        }
        prop[c] = (uint8_t)code;
    }
}

__global__ void __launch_bounds__(kThreads)
resolve_plane_kernel(const ScenarioDesc *__restrict__ dp, const uint8_t *__restrict__ prop,
                     int t_off)
{
    const ScenarioDesc &d = *dp;
    const uint64_t t = *d.step + (uint64_t)t_off;
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
        flush_counts(d, cnt);
    }
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__global__ void advance_kernel(const ScenarioDesc *__restrict__ descs, int n, int k)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long s = *descs[i].step + (unsigned long long)k;
    if (s > descs[i].end_step) s = descs[i].end_step;
    *descs[i].step = s;
}

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

__global__ void mask_ids_kernel(const ScenarioDesc *__restrict__ dp, int parity,
                                uint32_t *__restrict__ out)
{
    const ScenarioDesc &d = *dp;
    const size_t cells = (size_t)d.W * d.H;
    const uint8_t *occ = d.occ[parity];
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x)
        out[c] = occ[c] ? d.ids[c] : 0u;
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
                                  uint32_t total, int t_off, int grid, cudaStream_t stream)
{
    cudaError_t e = ensure_fused_attr<TW, TH>();
    if (e != cudaSuccess) return e;
    fused_step_kernel<TW, TH><<<grid, kThreads, FusedLayout<TW, TH>::SMEM, stream>>>(
        d_descs, d_prefix, n, total, t_off);
    return cudaGetLastError();
}

template <int TW, int TH>
static int blocks_per_sm_t()
{
    if (ensure_fused_attr<TW, TH>() != cudaSuccess) return 1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fused_step_kernel<TW, TH>, kThreads,
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
                              cudaStream_t stream)
{
#define PEDSIM_TILE_LAUNCH(w, h)                                                               \
    if (tile_w == w && tile_h == h)                                                            \
        return launch_fused_t<w, h>(d_descs, d_tile_prefix, n, total_tiles, t_off, grid, stream);
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

int fused_threads() { return kThreads; }

cudaError_t launch_two_pass_step(const ScenarioDesc *d_desc, uint8_t *d_prop, int W, int H,
                                 int t_off, cudaStream_t stream)
{
    const size_t cells = (size_t)W * H;
    const int grid = grid_for(cells, kThreads, 152 * 16);
    propose_plane_kernel<<<grid, kThreads, 0, stream>>>(d_desc, d_prop, t_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resolve_plane_kernel<<<grid, kThreads, 0, stream>>>(d_desc, d_prop, t_off);
    return cudaGetLastError();
}

cudaError_t launch_advance(const ScenarioDesc *d_descs, int n, int k, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    advance_kernel<<<(n + 255) / 256, 256, 0, stream>>>(d_descs, n, k);
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

cudaError_t launch_mask_ids(const ScenarioDesc *d_desc, int parity, int cells, uint32_t *d_out,
                            cudaStream_t stream)
{
    mask_ids_kernel<<<grid_for((size_t)cells, kThreads, 2048), kThreads, 0, stream>>>(d_desc, parity,
                                                                                 d_out);
    return cudaGetLastError();
}

}  // namespace pedsim
