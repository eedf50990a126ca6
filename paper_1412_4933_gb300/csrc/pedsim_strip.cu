// One synchronous step (Sec. IV.b-d) of a column strip of a larger grid:
// the building block of domain decomposition (one grid split into strips of
// columns, each strip on its own device or stream).
//
// A strip holds its interior columns plus a halo of up to kStripHalo columns
// on each side, copied from the neighbouring strips' interiors before every
// step.  The new state of a cell depends on cells at most three columns away
// (its claimants' proposals need their 3x3 neighbourhoods; an agent's
// departure needs its target's other claimants, two away, and their
// neighbourhoods, three away), so with a halo of three columns the strip's
// interior comes out exactly as in a step of the whole grid; the halo's own
// results are wrong near its outer edge and are replaced by the next
// exchange.  Everything that makes a step depend on where a cell lies in the
// whole grid uses global coordinates: the random numbers are keyed by the
// global cell index, and the goal edge and the crossing line are those of
// the whole grid; only the availability of neighbours beyond the strip's own
// columns is decided locally (as unavailable: wrong only in the halo).
// Counters count the events whose target cell lies in the interior, so the
// strips' counts add up to the whole grid's.
//
// The kernels are the cell-centric two-pass step: proposals into a scratch
// plane the caller provides, then one thread per cell resolves it.
#include "pedsim.h"
#include "pedsim_internal.h"
#include "pedsim_rules.cuh"

namespace pedsim {
namespace {

struct StripStep {
    int W, H;            // the strip's local width (interior + halos) and height
    int x0, Wg;          // global column of local column 0; width of the whole grid
    int lo, hi;          // interior: local columns lo .. hi-1 (counted)
    uint32_t model, alpha, beta, deposit_mode, band;
    float q, deposit, lem_scale;
    unsigned long long seed, step;
    const uint8_t *occ_in;
    uint8_t *occ_out;
    uint32_t *ids;
    const float *tau_in[2];
    float *tau_out[2];
    uint32_t *arrival;
    float *tour;
    unsigned long long *counters;
};

constexpr int kStripThreads = 256;

// Global cell index of local cell (x, y).
__device__ __forceinline__ uint64_t global_cell(const StripStep &a, int x, int y)
{
    return (uint64_t)y * (uint64_t)a.Wg + (uint64_t)(x + a.x0);
}

__global__ void __launch_bounds__(kStripThreads)
strip_propose_kernel(const __grid_constant__ StripStep a, uint8_t *__restrict__ prop)
{
    const int W = a.W, H = a.H;
    const RuleParams rp{a.model, a.alpha, a.beta, a.lem_scale};
    const size_t cells = (size_t)W * H;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (size_t)gridDim.x * blockDim.x) {
        const int g = a.occ_in[c];
        int code = 0;
        if (g) {
            const int x = (int)(c % (size_t)W), y = (int)(c / (size_t)W);
            const float *tp = a.model == 1 ? a.tau_in[g == 2 ? 1 : 0] + c : nullptr;
            // global coordinates for the rules; a neighbour outside the strip's
            // own columns counts as occupied (it is never read)
            const auto occ = [&](int dx, int dy) {
                return (unsigned)(x + dx) < (unsigned)W
                           ? (int)a.occ_in[(int64_t)c + (int64_t)dy * W + dx] : 1;
            };
            code = propose(x + a.x0, y, g, a.Wg, H, global_cell(a, x, y), a.step, a.seed, rp, occ,
                           tp, W);
        }
        prop[c] = (uint8_t)code;
    }
}

__global__ void __launch_bounds__(kStripThreads)
strip_resolve_kernel(const __grid_constant__ StripStep a, const uint8_t *__restrict__ prop)
{
    const int W = a.W, H = a.H;
    const size_t cells = (size_t)W * H;
    unsigned moved = 0, conflicts = 0, crossed_a = 0, crossed_b = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x; base < cells; base += stride) {
        const size_t c = base + threadIdx.x;
        if (c >= cells) continue;
        const int x = (int)(c % (size_t)W), y = (int)(c / (size_t)W);
        const bool interior = x >= a.lo && x < a.hi;
        auto prop_at = [&](int dx, int dy) { return (int)prop[(int64_t)c + (int64_t)dy * W + dx]; };
        const int o = a.occ_in[c];
        int no = o, incoming = 0;
        float dep = a.deposit;
        if (o == 0) {
            int k;
            const int w = resolve_winner(x, y, W, H, global_cell(a, x, y), a.step, a.seed, prop_at, &k);
            if (w >= 0) {
                const int dx = kCodeDX[w + 1], dy = kCodeDY[w + 1];
                const size_t src = (size_t)((int64_t)c + (int64_t)dy * W + dx);
                incoming = a.occ_in[src];
                no = incoming;
                const uint32_t id = a.ids[src];
                a.ids[c] = id;
                if (interior) {
                    ++moved;
                    if (k >= 2) ++conflicts;
                }
                if (a.model == 1 && a.deposit_mode == 1) {
                    const float L = __fadd_rn(a.tour[id], (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
                    a.tour[id] = L;
                    dep = __fdiv_rn(1.0f, L);
                }
                const int gx = x + a.x0;
                const bool in_band = incoming == 1 ? gx >= a.Wg - (int)a.band : gx < (int)a.band;
                if (in_band && a.arrival[id] == 0) {
                    a.arrival[id] = (uint32_t)(a.step + 1);
                    if (interior) {
                        if (incoming == 1) ++crossed_a; else ++crossed_b;
                    }
                }
            }
        } else {
            const int code = prop[c];
            if (code) {
                const int dx = kCodeDX[code], dy = kCodeDY[code];
                int k;
                const int w = resolve_winner(
                    x + dx, y + dy, W, H, global_cell(a, x + dx, y + dy), a.step, a.seed,
                    [&](int ex, int ey) { return prop_at(dx + ex, dy + ey); }, &k);
                if (w == 8 - code) no = 0;
            }
        }
        a.occ_out[c] = (uint8_t)no;
        if (a.model == 1) {
            float va = __fmul_rn(a.tau_in[0][c], a.q);
            float vb = __fmul_rn(a.tau_in[1][c], a.q);
            if (incoming == 1) va = __fadd_rn(va, dep);
            else if (incoming == 2) vb = __fadd_rn(vb, dep);
            a.tau_out[0][c] = va;
            a.tau_out[1][c] = vb;
        }
    }
    moved = __reduce_add_sync(0xffffffffu, moved);
    conflicts = __reduce_add_sync(0xffffffffu, conflicts);
    crossed_a = __reduce_add_sync(0xffffffffu, crossed_a);
    crossed_b = __reduce_add_sync(0xffffffffu, crossed_b);
    if ((threadIdx.x & 31) == 0 && a.counters) {
        if (moved) atomicAdd(&a.counters[kMoved], (unsigned long long)moved);
        if (conflicts) atomicAdd(&a.counters[kConflicts], (unsigned long long)conflicts);
        if (crossed_a) atomicAdd(&a.counters[kCrossedA], (unsigned long long)crossed_a);
        if (crossed_b) atomicAdd(&a.counters[kCrossedB], (unsigned long long)crossed_b);
    }
}

bool shares_bytes(const void *a, const void *b, size_t n)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + n && y < x + n;
}

// Halo copy between two strips: columns [src_col, src_col + ncols) of the
// source's local planes into [dst_col, ...) of the destination's, and the
// per-agent entries of the agents standing on the copied cells.
struct HaloCopy {
    int H, ncols, src_W, src_col, dst_W, dst_col;
    uint32_t n_agents;  // per-agent arrays hold n_agents + 1 entries
    const uint8_t *src_occ;
    const uint32_t *src_ids;
    const float *src_tau[2];
    const uint32_t *src_arrival;
    const float *src_tour;
    uint8_t *dst_occ;
    uint32_t *dst_ids;
    float *dst_tau[2];
    uint32_t *dst_arrival;
    float *dst_tour;
};

__global__ void __launch_bounds__(kStripThreads) strip_halo_kernel(const HaloCopy a)
{
    const size_t n = (size_t)a.H * (size_t)a.ncols;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const size_t y = i / (size_t)a.ncols, c = i - y * (size_t)a.ncols;
        const size_t s = y * (size_t)a.src_W + (size_t)a.src_col + c;
        const size_t d = y * (size_t)a.dst_W + (size_t)a.dst_col + c;
        const uint8_t o = a.src_occ[s];
        const uint32_t id = a.src_ids[s];
        a.dst_occ[d] = o;
        a.dst_ids[d] = id;
        if (a.src_tau[0]) {
            a.dst_tau[0][d] = a.src_tau[0][s];
            a.dst_tau[1][d] = a.src_tau[1][s];
        }
        if (o && id >= 1u && id <= a.n_agents) {
            a.dst_arrival[id] = a.src_arrival[id];
            if (a.src_tour) a.dst_tour[id] = a.src_tour[id];
        }
    }
}

}  // namespace
}  // namespace pedsim

using namespace pedsim;

extern "C" int sim_strip_halo(int H, int ncols, uint32_t n_agents, const uint8_t *src_occ,
                              const uint32_t *src_ids, const float *src_tauA,
                              const float *src_tauB, const uint32_t *src_arrival,
                              const float *src_tour, int src_W, int src_col, uint8_t *dst_occ,
                              uint32_t *dst_ids, float *dst_tauA, float *dst_tauB,
                              uint32_t *dst_arrival, float *dst_tour, int dst_W, int dst_col,
                              void *stream)
{
    if (H < 1 || ncols < 0 || src_W < 1 || dst_W < 1 || src_col < 0 || dst_col < 0 ||
        src_col + ncols > src_W || dst_col + ncols > dst_W)
        return PEDSIM_EINVAL;
    if (!src_occ || !src_ids || !src_arrival || !dst_occ || !dst_ids || !dst_arrival)
        return PEDSIM_EINVAL;
    if (!src_tauA != !src_tauB || !src_tauA != !dst_tauA || !dst_tauA != !dst_tauB)
        return PEDSIM_EINVAL;
    if (!src_tour != !dst_tour) return PEDSIM_EINVAL;
    if (ncols == 0) return PEDSIM_OK;
    HaloCopy a{};
    a.H = H;
    a.ncols = ncols;
    a.src_W = src_W;
    a.src_col = src_col;
    a.dst_W = dst_W;
    a.dst_col = dst_col;
    a.n_agents = n_agents;
    a.src_occ = src_occ;
    a.src_ids = src_ids;
    a.src_tau[0] = src_tauA;
    a.src_tau[1] = src_tauB;
    a.src_arrival = src_arrival;
    a.src_tour = src_tour;
    a.dst_occ = dst_occ;
    a.dst_ids = dst_ids;
    a.dst_tau[0] = dst_tauA;
    a.dst_tau[1] = dst_tauB;
    a.dst_arrival = dst_arrival;
    a.dst_tour = dst_tour;
    const size_t n = (size_t)H * (size_t)ncols;
    size_t blocks = (n + kStripThreads - 1) / kStripThreads;
    if (blocks > 1024) blocks = 1024;
    strip_halo_kernel<<<(unsigned)blocks, kStripThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? PEDSIM_OK : PEDSIM_ECUDA;
}

extern "C" int sim_step_strip(int W, int H, int x0, int W_global, int interior_lo,
                              int interior_hi, const sim_params *p, uint64_t seed, uint64_t step,
                              const uint8_t *occ_in, uint8_t *occ_out, uint32_t *ids,
                              const float *tauA_in, const float *tauB_in, float *tauA_out,
                              float *tauB_out, uint32_t *arrival, float *tour, uint8_t *scratch,
                              unsigned long long *counters, void *stream)
{
    if (sim_validate(W_global, H, p) != PEDSIM_OK) return PEDSIM_EINVAL;
    if (W < 1 || x0 < 0 || x0 + W > W_global || interior_lo < 0 || interior_lo > interior_hi ||
        interior_hi > W)
        return PEDSIM_EINVAL;
    const size_t cells = (size_t)W * (size_t)H;
    const bool aco = p->model == PEDSIM_ACO;
    if (!occ_in || !occ_out || !ids || !arrival || !scratch) return PEDSIM_EINVAL;
    if (shares_bytes(occ_in, occ_out, cells) || shares_bytes(scratch, occ_in, cells) ||
        shares_bytes(scratch, occ_out, cells))
        return PEDSIM_EINVAL;
    if (aco && (!tauA_in || !tauB_in || !tauA_out || !tauB_out)) return PEDSIM_EINVAL;
    if (aco && p->deposit_mode == 1 && !tour) return PEDSIM_EINVAL;

    StripStep a{};
    a.W = W;
    a.H = H;
    a.x0 = x0;
    a.Wg = W_global;
    a.lo = interior_lo;
    a.hi = interior_hi;
    a.model = p->model;
    a.alpha = p->alpha;
    a.beta = p->beta;
    a.deposit_mode = p->deposit_mode;
    a.band = p->band_cols;
    a.q = 1.0f - p->rho;
    a.deposit = p->deposit;
    a.lem_scale = 0x1p-16f / p->lem_sigma;
    a.seed = seed;
    a.step = step;
    a.occ_in = occ_in;
    a.occ_out = occ_out;
    a.ids = ids;
    a.tau_in[0] = tauA_in;
    a.tau_in[1] = tauB_in;
    a.tau_out[0] = tauA_out;
    a.tau_out[1] = tauB_out;
    a.arrival = arrival;
    a.tour = tour;
    a.counters = counters;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return PEDSIM_ECUDA;
    size_t blocks = (cells + kStripThreads - 1) / kStripThreads;
    if (blocks > 16u * (size_t)sms) blocks = 16u * (size_t)sms;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    strip_propose_kernel<<<(unsigned)blocks, kStripThreads, 0, st>>>(a, scratch);
    if (cudaGetLastError() != cudaSuccess) return PEDSIM_ECUDA;
    strip_resolve_kernel<<<(unsigned)blocks, kStripThreads, 0, st>>>(a, scratch);
    if (cudaGetLastError() != cudaSuccess) return PEDSIM_ECUDA;
    return PEDSIM_OK;
}
