// Host side of the C ABI declared in include/pedsim.h: device memory layout,
// TMA tensor-map encoding, CUDA-graph replay of the step loop, read-back,
// checkpoints, batched scenarios and the serving pool.
#include "pedsim.h"
#include "pedsim_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace pedsim;

namespace {

constexpr int kGraphSteps = 16;  // steps per captured graph

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Device memory layout of one scenario (one allocation)
// ---------------------------------------------------------------------------
struct Layout {
    size_t desc, occ[2], prop, codes, ids, tau[2][2], stamp, arrival, tour, pos, acode, part, error,
        prefix, counts, totals, act, act_bytes;
    size_t total;
    uint32_t n_slots;
    bool has_tau, has_tour;
};

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Counter slots: one per tile of the smallest tile shape of any variant, and
// at least one per CTA of the two-pass variant.
// Most work items any fused tile shape gives a W x H grid.
uint32_t fused_max_tiles(int W, int H)
{
    const uint32_t a = (uint32_t)ceil_div(W, 32) * (uint32_t)ceil_div(H, 16);
    const uint32_t b = (uint32_t)ceil_div(W, 64) * (uint32_t)ceil_div(H, 8);
    return std::max(a, b);
}

uint32_t counter_slots(int W, int H)
{
    int n = ceil_div(W, 32) * ceil_div(H, 16);
    n = std::max(n, ceil_div(W, 64) * ceil_div(H, 8));
    n = std::max(n, ceil_div(W, 128) * ceil_div(H, 8));
    n = std::max(n, two_pass_grid(W, H));
    return (uint32_t)n;
}

Layout make_layout(int W, int H, const sim_params &p)
{
    Layout L{};
    L.n_slots = counter_slots(W, H);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t cells = (size_t)W * (size_t)H;
    const size_t agents = 2 * (size_t)p.n_per_side + 1;
    L.has_tau = p.model == PEDSIM_ACO;
    L.has_tour = L.has_tau && p.deposit_mode == 1;
    L.desc = take(sizeof(ScenarioDesc));
    L.occ[0] = take(cells);
    L.occ[1] = take(cells);
    L.prop = take(cells);  // proposal plane of the two-kernel step variants
    L.codes = take(2 * cells);  // code planes of the agent-parallel variant
    L.ids = take(4 * cells);
    for (int g = 0; g < 2; ++g)
        for (int q = 0; q < 2; ++q) L.tau[g][q] = L.has_tau ? take(4 * cells) : 0;
    L.stamp = L.has_tau ? take(cells) : 0;  // deferred-evaporation stamps
    L.arrival = take(4 * agents);
    L.tour = L.has_tour ? take(4 * agents) : 0;
    L.pos = take(4 * agents);  // cell of each agent (agent-parallel variant)
    L.acode = take(agents);    // proposal code and group of each agent (same)
    L.part = take(8 * kNumCounters * (size_t)L.n_slots);
    L.error = take(4);
    L.prefix = take(4 * 8);  // tile, cell-block, agent-block and refresh-slice prefixes
    L.counts = take(4 * kGridCounts);
    L.totals = take(8 * kNumCounters);
    // tile-activity block of the fused step, sized for its smallest tiles
    L.act_bytes = activity_bytes(std::max(fused_max_tiles(W, H), 1u));
    L.act = take(L.act_bytes);
    L.total = off;
    return L;
}

// ---------------------------------------------------------------------------
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda).
// ---------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    });
    return fn;
}

bool encode_2d(CUtensorMap *map, CUtensorMapDataType type, size_t elem, void *base, int W, int H,
               int box_w, int box_h)
{
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)W * elem};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Marks a work list's activity block invalid: the next fused launch treats
// every tile as active and rebuilds flags and lists from scratch.
cudaError_t reset_activity(ActivityCtl *a, size_t bytes, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&a->reset, 1, sizeof(a->reset), st);
    return e;
}

int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scenario handle
// ---------------------------------------------------------------------------
struct sim_s {
    int W = 0, H = 0;
    sim_params p{};
    Layout L{};
    uint8_t *dmem = nullptr;
    ScenarioDesc hdesc{};
    ScenarioDesc *own_desc = nullptr;  // descriptor in this handle's allocation
    ScenarioDesc *d_desc = nullptr;    // where the live descriptor is (own or a work list)
    uint32_t *d_prefix = nullptr;
    ActivityCtl *d_act = nullptr;  // tile activity of the fused step
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used for graph capture
    unsigned long long step = 0; // host mirror of the device step index
    unsigned long long end_step = ~0ull;
    uint64_t seed = 0;
    int variant = kVariantAgent;
    int tile_w = 128, tile_h = 16, ctas_per_sm = 0;
    int sms = 1;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    unsigned long long wait_cycles = 0;  // bounded-wait limit of the tiled variant (0 = default)
    uint32_t test_flags = 0;             // failure-detection test hook
    std::string err;
};

namespace {

int fail(sim_t *s, int code, const std::string &msg)
{
    if (s) s->err = msg;
    return code;
}

int cuda_fail(sim_t *s, cudaError_t e, const char *what)
{
    return fail(s, PEDSIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SIM_CUDA(s, call)                                       \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
    } while (0)

void drop_graph(sim_t *s)
{
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
}

int tiles_of(int n, int t) { return (n + t - 1) / t; }

// Work blocks of the agent-parallel variant: pheromone stream blocks (none
// for LEM, which keeps no pheromone) and agent blocks.
uint32_t cell_blocks(int W, int H, const sim_params &p)
{
    if (p.model != PEDSIM_ACO) return 0;
    return (uint32_t)(((size_t)W * (size_t)H + kCellBlock - 1) / kCellBlock);
}
uint32_t agent_blocks(uint32_t n_per_side)
{
    return (uint32_t)((2ull * n_per_side + kAgentBlock - 1) / kAgentBlock);
}

// Fills hdesc (pointers, params, tensor maps for the current tiling) and
// uploads it with the tile prefix.
int upload_desc(sim_t *s)
{
    ScenarioDesc &d = s->hdesc;
    std::memset(&d, 0, sizeof(d));
    uint8_t *m = s->dmem;
    const Layout &L = s->L;
    d.occ[0] = m + L.occ[0];
    d.occ[1] = m + L.occ[1];
    d.prop = m + L.prop;
    d.codes[0] = m + L.codes;
    d.codes[1] = m + L.codes + (size_t)s->W * (size_t)s->H;
    d.ids = reinterpret_cast<uint32_t *>(m + L.ids);
    for (int g = 0; g < 2; ++g)
        for (int q = 0; q < 2; ++q)
            d.tau[g][q] = L.has_tau ? reinterpret_cast<float *>(m + L.tau[g][q]) : nullptr;
    d.stamp = L.has_tau ? m + L.stamp : nullptr;
    d.arrival = reinterpret_cast<uint32_t *>(m + L.arrival);
    d.tour = L.has_tour ? reinterpret_cast<float *>(m + L.tour) : nullptr;
    d.pos = reinterpret_cast<uint32_t *>(m + L.pos);
    d.acode = m + L.acode;
    d.part = reinterpret_cast<unsigned long long *>(m + L.part);
    d.n_slots = L.n_slots;
    d.step = s->step;
    d.error = reinterpret_cast<int *>(m + L.error);
    d.end_step = s->end_step;
    d.seed = s->seed;
    d.W = s->W;
    d.H = s->H;
    d.tile_w = s->tile_w;
    d.tile_h = s->tile_h;
    d.tiles_x = tiles_of(s->W, s->tile_w);
    d.tiles_y = tiles_of(s->H, s->tile_h);
    d.model = s->p.model;
    d.alpha = s->p.alpha;
    d.beta = s->p.beta;
    d.deposit_mode = s->p.deposit_mode;
    d.band = s->p.band_cols;
    d.n_per_side = s->p.n_per_side;
    d.q = 1.0f - s->p.rho;
    d.deposit = s->p.deposit;
    d.lem_scale = 0x1p-16f / s->p.lem_sigma;
    d.tau0 = s->p.tau0;
    division_by_width(s->W, &d.w_mul, &d.w_shr);
    d.wait_cycles = s->wait_cycles;
    d.test_flags = s->test_flags;
    const int TWd = s->tile_w, THd = s->tile_h;
    if (s->variant == kVariantFused) {
        for (int q = 0; q < 2; ++q)
            if (!encode_2d(&d.map_occ[q], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.occ[q], s->W, s->H,
                           s->tile_w + 32, s->tile_h + 6))
                return fail(s, PEDSIM_ECUDA, "cuTensorMapEncodeTiled failed (occupancy)");
        if (L.has_tau)
            for (int g = 0; g < 2; ++g)
                for (int q = 0; q < 2; ++q)
                    if (!encode_2d(&d.map_tau[g][q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d.tau[g][q],
                                   s->W, s->H, s->tile_w + 8, s->tile_h + 6) ||
                        !encode_2d(&d.map_tau_tile[g][q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                   d.tau[g][q], s->W, s->H, s->tile_w, s->tile_h))
                        return fail(s, PEDSIM_ECUDA, "cuTensorMapEncodeTiled failed (pheromone)");
    } else if (s->variant == kVariantPipeline) {
        bool ok = true;
        for (int q = 0; q < 2; ++q) {
            ok = ok && encode_2d(&d.map_occ[q], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.occ[q], s->W,
                                 s->H, TWd + 32, THd + 2);
            ok = ok && encode_2d(&d.map_occ_out[q], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.occ[q],
                                 s->W, s->H, TWd, THd);
        }
        ok = ok && encode_2d(&d.map_prop, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.prop, s->W, s->H,
                             TWd + 32, THd + 4);
        ok = ok && encode_2d(&d.map_prop_out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.prop, s->W,
                             s->H, TWd, THd);
        if (L.has_tau)
            for (int g = 0; g < 2; ++g)
                for (int q = 0; q < 2; ++q)
                    ok = ok && encode_2d(&d.map_tau[g][q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                         d.tau[g][q], s->W, s->H, TWd, THd);
        if (!ok) return fail(s, PEDSIM_ECUDA, "cuTensorMapEncodeTiled failed (tiled variant)");
    }
    const uint32_t cb = cell_blocks(s->W, s->H, s->p);
    const uint32_t prefix[8] = {0u, (uint32_t)(d.tiles_x * d.tiles_y), 0u, cb,
                                0u, agent_blocks(s->p.n_per_side), 0u, deferred_slices(cb)};
    // the handle's own descriptor becomes the live one again (a work list that
    // held it re-uploads its copy when it runs next)
    s->d_desc = s->own_desc;
    SIM_CUDA(s, cudaMemcpyAsync(s->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    // pageable host sources are staged before cudaMemcpyAsync returns
    SIM_CUDA(s, cudaMemcpyAsync(s->d_prefix, prefix, sizeof(prefix), cudaMemcpyHostToDevice,
                                s->stream));
    // tiling, state or step changed: the activity flags start over
    SIM_CUDA(s, reset_activity(s->d_act, s->L.act_bytes, s->stream));
    drop_graph(s);
    return PEDSIM_OK;
}

// The agent-parallel and deferred steps advance the device step index
// themselves (no launch_advance), keep their occupancy in plane 0 updated in
// place and need the per-agent positions.
bool self_advancing(int variant) { return variant == kVariantAgent || variant == kVariantDeferred; }

int fused_grid(const sim_t *s, uint32_t total)
{
    const int per_sm = s->ctas_per_sm > 0 ? s->ctas_per_sm : fused_blocks_per_sm(s->tile_w, s->tile_h);
    const uint32_t cap = (uint32_t)s->sms * (uint32_t)per_sm;
    return (int)std::max<uint32_t>(1, std::min(total, cap));
}

// Launches the kernels of step (step index + t_off) on stream st.
int launch_one_step(sim_t *s, int t_off, cudaStream_t st)
{
    const uint32_t total = (uint32_t)(s->hdesc.tiles_x * s->hdesc.tiles_y);
    if (s->variant == kVariantTwoPass) {
        SIM_CUDA(s, launch_two_pass_step(s->d_desc, s->hdesc.prop, s->W, s->H, t_off, st));
        return PEDSIM_OK;
    }
    if (s->variant == kVariantPipeline) {
        SIM_CUDA(s, launch_pipeline_step(s->d_desc, s->d_prefix, 1, total, t_off, s->tile_h, st));
        return PEDSIM_OK;
    }
    if (s->variant == kVariantAgent) {
        // the agent step reads and advances the step index itself
        SIM_CUDA(s, launch_agent_step(s->d_desc, s->d_prefix + 2, s->d_prefix + 4, 1,
                                      cell_blocks(s->W, s->H, s->p), agent_blocks(s->p.n_per_side),
                                      s->d_act, st));
        return PEDSIM_OK;
    }
    if (s->variant == kVariantDeferred) {
        SIM_CUDA(s, launch_deferred_step(s->d_desc, s->d_prefix + 2, s->d_prefix + 4,
                                         s->d_prefix + 6, 1,
                                         deferred_slices(cell_blocks(s->W, s->H, s->p)),
                                         agent_blocks(s->p.n_per_side), s->d_act, st));
        return PEDSIM_OK;
    }
    SIM_CUDA(s, launch_fused_step(s->d_desc, s->d_prefix, 1, total, t_off, s->tile_w, s->tile_h,
                                  fused_grid(s, total), s->d_act, st));
    return PEDSIM_OK;
}

int ensure_graph(sim_t *s)
{
    if (s->graph) return PEDSIM_OK;
    // make kernel attributes and occupancy queries happen outside the capture
    if (s->variant == kVariantFused) (void)fused_blocks_per_sm(s->tile_w, s->tile_h);
    SIM_CUDA(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    int rc = PEDSIM_OK;
    for (int k = 0; k < kGraphSteps && rc == PEDSIM_OK; ++k) rc = launch_one_step(s, k, s->cap);
    if (rc == PEDSIM_OK && !self_advancing(s->variant)) {
        cudaError_t ea = launch_advance(s->d_desc, 1, kGraphSteps, s->cap);
        if (ea != cudaSuccess) rc = cuda_fail(s, ea, "advance kernel capture");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    if (rc != PEDSIM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph = nullptr;
        return cuda_fail(s, e, "cudaGraphInstantiate");
    }
    return PEDSIM_OK;
}

bool params_ok(int W, int H, const sim_params *p)
{
    if (!p) return false;
    if (W < 16 || H < 16 || (W % 16) != 0 || (H % 16) != 0) return false;
    if ((int64_t)W * (int64_t)H > ((int64_t)1 << 31)) return false;
    if (p->model > 1 || p->deposit_mode > 1) return false;
    if (p->band_cols < 1 || 2ull * p->band_cols > (unsigned long long)W) return false;
    if ((uint64_t)p->n_per_side > (uint64_t)p->band_cols * (uint64_t)H) return false;
    if (!(p->lem_sigma > 0.0f) || !std::isfinite(p->lem_sigma)) return false;
    if (p->model == PEDSIM_ACO) {
        if (!(p->rho > 0.0f && p->rho <= 1.0f)) return false;
        if (p->alpha > 4 || p->beta > 4) return false;
        if (!(p->tau0 >= 0.0f) || !std::isfinite(p->tau0)) return false;
        if (!(p->deposit >= 0.0f) || !std::isfinite(p->deposit)) return false;
    }
    return true;
}

size_t agents_len(const sim_t *s) { return 2 * (size_t)s->p.n_per_side + 1; }

// Occupancy plane that holds the current state: the agent-parallel variant
// updates plane 0 in place, the others alternate by step parity.
int occ_plane(const sim_t *s, int variant, unsigned long long step)
{
    (void)s;
    return self_advancing(variant) ? 0 : (int)(step & 1);
}
// Pheromone plane that holds the current state: the deferred variant keeps
// one plane per group (plane 0, with per-cell stamps), the others alternate.
int tau_plane(int variant, unsigned long long step)
{
    return variant == kVariantDeferred ? 0 : (int)(step & 1);
}
int occ_plane(const sim_t *s) { return occ_plane(s, s->variant, s->step); }

// The step index the kernels use lives in the device descriptor; the host
// copy follows every sim_step call, but a caller that replays a CUDA graph it
// captured around sim_step advances only the device's.  Read-back calls take
// the device's value first (it selects the planes that hold the state).
int resync_step(sim_t *s)
{
    unsigned long long dstep = 0;
    SIM_CUDA(s, cudaMemcpyAsync(&dstep, &s->d_desc->step, 8, cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    s->step = dstep;
    return PEDSIM_OK;
}

// Changes the step variant and tiling of a scenario between steps: the
// occupancy moves to the plane the new variant keeps it in, and the agent
// positions are rebuilt when the new variant is the agent-parallel one (only
// that variant keeps them up to date).
int switch_variant(sim_t *s, int variant, int tw, int th, int cps)
{
    const size_t cells = (size_t)s->W * (size_t)s->H;
    const int from = occ_plane(s), to = occ_plane(s, variant, s->step);
    if (from != to)
        SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.occ[to], s->hdesc.occ[from], cells,
                                    cudaMemcpyDeviceToDevice, s->stream));
    const int old = s->variant;
    if (s->L.has_tau) {
        // pheromone: deferred planes are brought up to the step first, then
        // the state moves to the plane the new variant keeps it in
        if (old == kVariantDeferred) SIM_CUDA(s, launch_deferred_catch_up(s->d_desc, (int)cells, s->stream));
        const int tf = tau_plane(old, s->step), tt = tau_plane(variant, s->step);
        if (tf != tt)
            for (int g = 0; g < 2; ++g)
                SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.tau[g][tt], s->hdesc.tau[g][tf], 4 * cells,
                                            cudaMemcpyDeviceToDevice, s->stream));
        if (variant == kVariantDeferred && old != kVariantDeferred)
            SIM_CUDA(s, cudaMemsetAsync(s->hdesc.stamp, (int)(s->step & 255u), cells, s->stream));
    }
    s->variant = variant;
    s->tile_w = tw;
    s->tile_h = th;
    s->ctas_per_sm = cps;
    int rc = upload_desc(s);
    if (rc == PEDSIM_OK && self_advancing(variant) && !self_advancing(old))
        SIM_CUDA(s, launch_build_pos(s->d_desc, s->W * s->H, to, s->stream));
    return rc;
}

}  // namespace

// Creates a scenario whose allocation, initialisation and later work are
// ordered on `stream` (stream-ordered allocation: no device-wide sync).
// `mem`: the memory pool the allocation comes from (nullptr: the device's
// default pool).
static int pedsim_create_on_stream(int W, int H, const sim_params *p, cudaStream_t stream,
                                   sim_t **out, cudaMemPool_t mem = nullptr)
{
    if (!out) return PEDSIM_EINVAL;
    *out = nullptr;
    if (!params_ok(W, H, p)) return PEDSIM_EINVAL;
    sim_t *s = new (std::nothrow) sim_t();
    if (!s) return PEDSIM_ENOMEM;
    s->W = W;
    s->H = H;
    s->p = *p;
    s->stream = stream;
    s->L = make_layout(W, H, *p);
    s->sms = device_sms();
    cudaError_t e =
        mem ? cudaMallocFromPoolAsync(reinterpret_cast<void **>(&s->dmem), s->L.total, mem, stream)
            : cudaMallocAsync(reinterpret_cast<void **>(&s->dmem), s->L.total, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return e == cudaErrorMemoryAllocation ? PEDSIM_ENOMEM : PEDSIM_ECUDA;
    }
    s->own_desc = reinterpret_cast<ScenarioDesc *>(s->dmem + s->L.desc);
    s->d_desc = s->own_desc;
    s->d_prefix = reinterpret_cast<uint32_t *>(s->dmem + s->L.prefix);
    s->d_act = reinterpret_cast<ActivityCtl *>(s->dmem + s->L.act);
    if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFreeAsync(s->dmem, stream);
        delete s;
        return PEDSIM_ECUDA;
    }
    int rc = upload_desc(s);
    if (rc == PEDSIM_OK) {
        cudaError_t e2 = launch_init(s->d_desc, 1, W * H, (int)agents_len(s), s->stream);
        if (e2 != cudaSuccess) rc = cuda_fail(s, e2, "init kernel");
    }
    if (rc != PEDSIM_OK) {
        sim_destroy(s);
        return rc;
    }
    *out = s;
    return PEDSIM_OK;
}


extern "C" {

void sim_default_params(sim_params *p)
{
    if (!p) return;
    p->model = PEDSIM_LEM;
    p->n_per_side = 0;
    p->band_cols = 16;
    p->rho = 0.05f;
    p->tau0 = 1.0f;
    p->deposit = 1.0f;
    p->alpha = 1;
    p->beta = 1;
    p->deposit_mode = 0;
    p->lem_sigma = 1.0f;
}

int sim_validate(int W, int H, const sim_params *p)
{
    return params_ok(W, H, p) ? PEDSIM_OK : PEDSIM_EINVAL;
}

size_t sim_device_bytes(int W, int H, const sim_params *p)
{
    if (!params_ok(W, H, p)) return 0;
    return make_layout(W, H, *p).total;
}

int sim_create(int W, int H, const sim_params *p, sim_t **out)
{
    return pedsim_create_on_stream(W, H, p, nullptr, out);
}

int sim_set_stream(sim_t *s, void *stream)
{
    if (!s) return PEDSIM_EINVAL;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    return PEDSIM_OK;
}

int sim_place(sim_t *s, uint64_t seed)
{
    if (!s) return PEDSIM_EINVAL;
    s->seed = seed;
    s->step = 0;
    int rc = upload_desc(s);
    if (rc != PEDSIM_OK) return rc;
    SIM_CUDA(s, launch_init(s->d_desc, 1, s->W * s->H, (int)agents_len(s), s->stream));
    SIM_CUDA(s, launch_place(s->d_desc, 1, s->stream));
    SIM_CUDA(s, launch_build_pos(s->d_desc, s->W * s->H, 0, s->stream));
    return PEDSIM_OK;
}

int sim_step(sim_t *s, int n)
{
    if (!s || n < 0) return fail(s, PEDSIM_EINVAL, "negative step count");
    if (n == 0) return PEDSIM_OK;
    const int full = n / kGraphSteps, rem = n % kGraphSteps;
    if (full > 0) {
        int rc = ensure_graph(s);
        if (rc != PEDSIM_OK) return rc;
        for (int i = 0; i < full; ++i) SIM_CUDA(s, cudaGraphLaunch(s->graph, s->stream));
    }
    if (rem > 0) {
        if (s->variant == kVariantFused) (void)fused_blocks_per_sm(s->tile_w, s->tile_h);
        for (int k = 0; k < rem; ++k) {
            int rc = launch_one_step(s, k, s->stream);
            if (rc != PEDSIM_OK) return rc;
        }
        if (!self_advancing(s->variant))
            SIM_CUDA(s, launch_advance(s->d_desc, 1, rem, s->stream));
    }
    s->step += (unsigned long long)n;
    return PEDSIM_OK;
}

int sim_read_grid(sim_t *s, uint8_t *occ, uint32_t *ids, float *tauA, float *tauB)
{
    if (!s) return PEDSIM_EINVAL;
    if (int rc = resync_step(s)) return rc;
    const size_t cells = (size_t)s->W * s->H;
    const int par = (int)(s->step & 1);
    const int oplane = occ_plane(s);
    std::vector<uint8_t> occ_tmp;
    uint8_t *occ_h = occ;
    if (ids && !occ) {
        occ_tmp.resize(cells);
        occ_h = occ_tmp.data();
    }
    if (occ_h)
        SIM_CUDA(s, cudaMemcpyAsync(occ_h, s->hdesc.occ[oplane], cells, cudaMemcpyDeviceToHost,
                                    s->stream));
    if (ids)
        SIM_CUDA(s, cudaMemcpyAsync(ids, s->hdesc.ids, 4 * cells, cudaMemcpyDeviceToHost, s->stream));
    float *dst[2] = {tauA, tauB};
    const int tpl = s->variant == kVariantDeferred ? 0 : par;
    if (s->variant == kVariantDeferred && s->L.has_tau && (tauA || tauB))
        SIM_CUDA(s, launch_deferred_catch_up(s->d_desc, (int)cells, s->stream));
    for (int g = 0; g < 2; ++g) {
        if (!dst[g] || !s->L.has_tau) continue;
        SIM_CUDA(s, cudaMemcpyAsync(dst[g], s->hdesc.tau[g][tpl], 4 * cells, cudaMemcpyDeviceToHost,
                                    s->stream));
    }
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    if (ids)
        for (size_t c = 0; c < cells; ++c)
            if (!occ_h[c]) ids[c] = 0;
    // LEM keeps no pheromone: its planes read as tau0 everywhere
    for (int g = 0; g < 2; ++g)
        if (dst[g] && !s->L.has_tau) std::fill(dst[g], dst[g] + cells, s->p.tau0);
    return PEDSIM_OK;
}

int sim_read_agents(sim_t *s, uint32_t *arrival, float *tour)
{
    if (!s) return PEDSIM_EINVAL;
    const size_t n = agents_len(s);
    if (arrival)
        SIM_CUDA(s, cudaMemcpyAsync(arrival, s->hdesc.arrival, 4 * n, cudaMemcpyDeviceToHost, s->stream));
    if (tour && s->L.has_tour)
        SIM_CUDA(s, cudaMemcpyAsync(tour, s->hdesc.tour, 4 * n, cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    if (tour && !s->L.has_tour) std::fill(tour, tour + n, 0.0f);
    return PEDSIM_OK;
}

int sim_set_state(sim_t *s, uint64_t seed, uint64_t step, const uint8_t *occ, const uint32_t *ids,
                  const float *tauA, const float *tauB, const uint32_t *arrival, const float *tour)
{
    if (!s || !occ || !ids) return fail(s, PEDSIM_EINVAL, "occ and ids are required");
    const size_t cells = (size_t)s->W * s->H;
    const uint32_t n_agents = 2u * s->p.n_per_side;
    // validate: exactly 2N agents, groups 1/2, ids a permutation of 1..2N
    std::vector<uint8_t> seen(n_agents + 1, 0);
    uint32_t count = 0;
    for (size_t c = 0; c < cells; ++c) {
        if (!occ[c]) continue;
        if (occ[c] > 2 || ids[c] < 1 || ids[c] > n_agents || seen[ids[c]])
            return fail(s, PEDSIM_EINVAL, "occ/ids do not describe a valid agent set");
        seen[ids[c]] = 1;
        ++count;
    }
    if (count != n_agents) return fail(s, PEDSIM_EINVAL, "agent count differs from 2*n_per_side");
    s->seed = seed;
    s->step = step;
    int rc = upload_desc(s);
    if (rc != PEDSIM_OK) return rc;
    SIM_CUDA(s, launch_init(s->d_desc, 1, s->W * s->H, (int)agents_len(s), s->stream));
    const int par = (int)(step & 1);
    const int oplane = occ_plane(s);
    SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.occ[oplane], occ, cells, cudaMemcpyHostToDevice,
                                s->stream));
    SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.ids, ids, 4 * cells, cudaMemcpyHostToDevice, s->stream));
    if (s->L.has_tau) {
        // (init filled plane 0 with tau0 and the stamps with the step index)
        const int tpl = tau_plane(s->variant, step);
        const float *src[2] = {tauA, tauB};
        for (int g = 0; g < 2; ++g)
            if (src[g])
                SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.tau[g][tpl], src[g], 4 * cells,
                                            cudaMemcpyHostToDevice, s->stream));
            else if (tpl == 1)
                SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.tau[g][1], s->hdesc.tau[g][0], 4 * cells,
                                            cudaMemcpyDeviceToDevice, s->stream));
    }
    const size_t na = agents_len(s);
    if (arrival)
        SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.arrival, arrival, 4 * na, cudaMemcpyHostToDevice, s->stream));
    if (tour && s->L.has_tour)
        SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.tour, tour, 4 * na, cudaMemcpyHostToDevice, s->stream));
    SIM_CUDA(s, launch_build_pos(s->d_desc, s->W * s->H, oplane, s->stream));
    return PEDSIM_OK;
}

int sim_stats(sim_t *s, sim_stats_t *out)
{
    if (!s || !out) return PEDSIM_EINVAL;
    if (int rc = resync_step(s)) return rc;
    unsigned long long ctr[kNumCounters], dstep = 0;
    unsigned int counts[kGridCounts];
    const int par = occ_plane(s);
    unsigned int *d_counts = reinterpret_cast<unsigned int *>(s->dmem + s->L.counts);
    unsigned long long *d_tot = reinterpret_cast<unsigned long long *>(s->dmem + s->L.totals);
    SIM_CUDA(s, launch_grid_counts(s->d_desc, par, s->W * s->H, d_counts, s->stream));
    SIM_CUDA(s, launch_sum_slots(s->d_desc, d_tot, s->stream));
    SIM_CUDA(s, cudaMemcpyAsync(ctr, d_tot, sizeof(ctr), cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaMemcpyAsync(&dstep, &s->d_desc->step, 8, cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaMemcpyAsync(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    if (dstep != s->step) return fail(s, PEDSIM_ECUDA, "device step index out of sync");
    std::memset(out, 0, sizeof(*out));
    out->step = dstep;
    out->agents[0] = counts[0];
    out->agents[1] = counts[1];
    out->parked[0] = counts[2];
    out->parked[1] = counts[3];
    out->moved = ctr[kMoved];
    out->conflicts = ctr[kConflicts];
    out->crossed[0] = (uint32_t)ctr[kCrossedA];
    out->crossed[1] = (uint32_t)ctr[kCrossedB];
    return PEDSIM_OK;
}

// Checkpoint format: header, then occ, ids (0 at empty cells), tauA, tauB
// (ACO), arrival, tour (deposit_mode 1).
struct CkptHeader {
    char magic[8];
    uint32_t version, W, H, pad;
    sim_params p;
    uint64_t seed, step;
    unsigned long long counters[kNumCounters];
};

static size_t ckpt_size(const sim_t *s)
{
    const size_t cells = (size_t)s->W * s->H, na = agents_len(s);
    size_t n = sizeof(CkptHeader) + cells + 4 * cells + 4 * na;
    if (s->L.has_tau) n += 8 * cells;
    if (s->L.has_tour) n += 4 * na;
    return n;
}

int sim_save(sim_t *s, void *buf, size_t *len)
{
    if (!s || !len) return PEDSIM_EINVAL;
    const size_t need = ckpt_size(s);
    if (!buf) {
        *len = need;
        return PEDSIM_OK;
    }
    if (*len < need) return fail(s, PEDSIM_EINVAL, "checkpoint buffer too small");
    if (int rc = resync_step(s)) return rc;
    const size_t cells = (size_t)s->W * s->H, na = agents_len(s);
    CkptHeader h{};
    std::memcpy(h.magic, "PEDSIM01", 8);
    h.version = 1;
    h.W = (uint32_t)s->W;
    h.H = (uint32_t)s->H;
    h.p = s->p;
    h.seed = s->seed;
    h.step = s->step;
    uint8_t *b = static_cast<uint8_t *>(buf);
    uint8_t *occ = b + sizeof(h);
    uint32_t *ids = reinterpret_cast<uint32_t *>(occ + cells);
    float *tA = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(ids) + 4 * cells);
    float *tB = tA + (s->L.has_tau ? cells : 0);
    uint32_t *arr = reinterpret_cast<uint32_t *>(s->L.has_tau ? tB + cells : tA);
    float *tour = reinterpret_cast<float *>(arr + na);
    std::vector<uint32_t> ids_tmp(cells);
    std::vector<uint8_t> occ_tmp(cells);
    std::vector<float> ta, tb;
    if (s->L.has_tau) { ta.resize(cells); tb.resize(cells); }
    int rc = sim_read_grid(s, occ_tmp.data(), ids_tmp.data(), s->L.has_tau ? ta.data() : nullptr,
                           s->L.has_tau ? tb.data() : nullptr);
    if (rc) return rc;
    std::vector<uint32_t> arr_tmp(na);
    std::vector<float> tour_tmp(na);
    rc = sim_read_agents(s, arr_tmp.data(), tour_tmp.data());
    if (rc) return rc;
    unsigned long long *d_tot = reinterpret_cast<unsigned long long *>(s->dmem + s->L.totals);
    SIM_CUDA(s, launch_sum_slots(s->d_desc, d_tot, s->stream));
    SIM_CUDA(s, cudaMemcpyAsync(h.counters, d_tot, sizeof(h.counters), cudaMemcpyDeviceToHost,
                                s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    std::memcpy(b, &h, sizeof(h));
    std::memcpy(occ, occ_tmp.data(), cells);
    std::memcpy(ids, ids_tmp.data(), 4 * cells);
    if (s->L.has_tau) {
        std::memcpy(tA, ta.data(), 4 * cells);
        std::memcpy(tB, tb.data(), 4 * cells);
    }
    std::memcpy(arr, arr_tmp.data(), 4 * na);
    if (s->L.has_tour) std::memcpy(tour, tour_tmp.data(), 4 * na);
    *len = need;
    return PEDSIM_OK;
}

int sim_load(sim_t *s, const void *buf, size_t len)
{
    if (!s || !buf) return PEDSIM_EINVAL;
    if (len < sizeof(CkptHeader) || len < ckpt_size(s)) return fail(s, PEDSIM_EINVAL, "checkpoint too short");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "PEDSIM01", 8) != 0 || h.version != 1)
        return fail(s, PEDSIM_EINVAL, "not a checkpoint");
    if ((int)h.W != s->W || (int)h.H != s->H || std::memcmp(&h.p, &s->p, sizeof(sim_params)) != 0)
        return fail(s, PEDSIM_EINVAL, "checkpoint of a different scenario shape or parameters");
    const size_t cells = (size_t)s->W * s->H, na = agents_len(s);
    const uint8_t *b = static_cast<const uint8_t *>(buf);
    const uint8_t *occ = b + sizeof(h);
    const uint32_t *ids = reinterpret_cast<const uint32_t *>(occ + cells);
    const float *tA = reinterpret_cast<const float *>(reinterpret_cast<const uint8_t *>(ids) + 4 * cells);
    const float *tB = tA + (s->L.has_tau ? cells : 0);
    const uint32_t *arr = reinterpret_cast<const uint32_t *>(s->L.has_tau ? tB + cells : tA);
    const float *tour = reinterpret_cast<const float *>(arr + na);
    int rc = sim_set_state(s, h.seed, h.step, occ, ids, s->L.has_tau ? tA : nullptr,
                           s->L.has_tau ? tB : nullptr, arr, s->L.has_tour ? tour : nullptr);
    if (rc) return rc;
    // the saved totals go to slot 0 (sim_set_state cleared every slot)
    SIM_CUDA(s, cudaMemcpyAsync(s->hdesc.part, h.counters, sizeof(h.counters),
                                cudaMemcpyHostToDevice, s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    return PEDSIM_OK;
}

int sim_set_variant(sim_t *s, int variant)
{
    if (!s || (variant != kVariantPipeline && variant != kVariantTwoPass &&
               variant != kVariantFused && variant != kVariantAgent &&
               variant != kVariantDeferred))
        return fail(s, PEDSIM_EINVAL, "unknown variant");
    if (variant == s->variant) return PEDSIM_OK;
    // each variant starts from its own default tile shape
    return switch_variant(s, variant, variant == kVariantFused ? 64 : 128, 16, 0);
}

int sim_set_tiling(sim_t *s, int tile_w, int tile_h, int ctas_per_sm)
{
    const bool ok = s && !self_advancing(s->variant) && s->variant != kVariantTwoPass &&
                    (s->variant == kVariantFused ? tile_supported(tile_w, tile_h)
                                                 : pipeline_tile_supported(tile_w, tile_h));
    if (!ok || ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(s, PEDSIM_EINVAL, "unsupported tile shape");
    s->tile_w = tile_w;
    s->tile_h = tile_h;
    s->ctas_per_sm = ctas_per_sm;
    return upload_desc(s);
}

int sim_launches_per_step(sim_t *s, int *out)
{
    if (!s || !out) return fail(s, PEDSIM_EINVAL, "null argument");
    if (self_advancing(s->variant))
        *out = 2;  // proposals (and stream), then the resolution (it advances the step)
    else if (s->variant == kVariantFused)
        *out = 2;  // the step and the step-index advance
    else
        *out = 3;  // proposals, resolution and the step-index advance
    return PEDSIM_OK;
}

int sim_set_wait_test(sim_t *s, uint64_t wait_cycles, uint32_t test_flags)
{
    if (!s) return PEDSIM_EINVAL;
    if (test_flags & ~(uint32_t)PEDSIM_TEST_SKIP_RESOLVE_LOADS)
        return fail(s, PEDSIM_EINVAL, "unknown test flag");
    s->wait_cycles = (unsigned long long)wait_cycles;
    s->test_flags = test_flags;
    return upload_desc(s);
}

int sim_device_status(sim_t *s)
{
    if (!s) return PEDSIM_EINVAL;
    int v = 0;
    SIM_CUDA(s, cudaMemcpyAsync(&v, s->hdesc.error, 4, cudaMemcpyDeviceToHost, s->stream));
    SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    if (v) {
        SIM_CUDA(s, cudaMemsetAsync(s->hdesc.error, 0, 4, s->stream));
        SIM_CUDA(s, cudaStreamSynchronize(s->stream));
    }
    return v;
}

void sim_destroy(sim_t *s)
{
    if (!s) return;
    drop_graph(s);
    // stream-ordered frees: memory returns once the stream's prior work is done
    if (s->dmem) cudaFreeAsync(s->dmem, s->stream);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

const char *sim_last_error(const sim_t *s)
{
    return s ? s->err.c_str() : "null handle";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Work lists of several scenarios (batch and pool)
// ---------------------------------------------------------------------------
namespace {

// Device-side copy of several scenarios' descriptors plus the tile prefix of
// the (scenario, tile) work list, and the graph of kGraphSteps steps.
struct MultiRun {
    ScenarioDesc *d_descs = nullptr;
    uint32_t *d_prefix = nullptr;  // tile, cell-block, agent-block, slice prefixes (4 x capacity + 1)
    uint32_t cell_total = 0, agent_total = 0, slice_total = 0;
    ActivityCtl *d_act = nullptr;  // tile activity of the shared fused launches
    size_t act_capacity = 0;       // bytes
    int capacity = 0, count = 0, prefix_n = 0;
    uint32_t total = 0;
    int variant = kVariantAgent;
    int tile_w = 128, tile_h = 16, ctas_per_sm = 0, sms = 1;
    cudaStream_t stream = nullptr, cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::string err;

    int fail_(int code, const std::string &m) { err = m; return code; }
    int cuda_(cudaError_t e, const char *what)
    {
        return fail_(PEDSIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    void drop() { if (graph) cudaGraphExecDestroy(graph); graph = nullptr; }

    int reserve(int n)
    {
        if (n <= capacity) return PEDSIM_OK;
        int cap_new = std::max(n, 2 * capacity);
        if (d_descs) cudaFreeAsync(d_descs, stream);
        if (d_prefix) cudaFreeAsync(d_prefix, stream);
        d_descs = nullptr;
        d_prefix = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_descs),
                                        sizeof(ScenarioDesc) * (size_t)cap_new, stream);
        if (e == cudaSuccess)
            e = cudaMallocAsync(reinterpret_cast<void **>(&d_prefix),
                                4 * sizeof(uint32_t) * (size_t)(cap_new + 1), stream);
        if (e != cudaSuccess) return cuda_(e, "work list allocation");
        capacity = cap_new;
        return PEDSIM_OK;
    }

    // Uploads the descriptors of `sims` (in this order) and their tile prefix.
    int load(const std::vector<sim_t *> &sims)
    {
        int rc = reserve((int)sims.size());
        if (rc) return rc;
        const size_t n = sims.size();
        std::vector<ScenarioDesc> h(n);
        // tiles, cell blocks, agent blocks, refresh slices of the deferred step
        std::vector<uint32_t> pre(4 * (n + 1), 0);
        for (size_t i = 0; i < n; ++i) {
            h[i] = sims[i]->hdesc;
            const uint32_t cb = cell_blocks(sims[i]->W, sims[i]->H, sims[i]->p);
            pre[i + 1] = pre[i] + (uint32_t)(h[i].tiles_x * h[i].tiles_y);
            pre[n + 1 + i + 1] = pre[n + 1 + i] + cb;
            pre[2 * (n + 1) + i + 1] = pre[2 * (n + 1) + i] + agent_blocks(sims[i]->p.n_per_side);
            pre[3 * (n + 1) + i + 1] = pre[3 * (n + 1) + i] + deferred_slices(cb);
        }
        count = (int)n;
        total = pre[n];
        cell_total = pre[2 * n + 1];
        agent_total = pre[3 * n + 2];
        slice_total = pre[4 * n + 3];
        const size_t need = activity_bytes(std::max(total, 1u));
        if (need > act_capacity) {
            if (d_act) cudaFreeAsync(d_act, stream);
            d_act = nullptr;
            act_capacity = 0;
            cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_act), 2 * need, stream);
            if (e != cudaSuccess) return cuda_(e, "activity block allocation");
            act_capacity = 2 * need;
        }
        {
            cudaError_t e = reset_activity(d_act, need, stream);
            if (e != cudaSuccess) return cuda_(e, "activity block reset");
        }
        for (size_t i = 0; i < sims.size(); ++i) h[i].step = sims[i]->step;  // exact host mirror
        if (count) {
            cudaError_t e = cudaMemcpyAsync(d_descs, h.data(), sizeof(ScenarioDesc) * h.size(),
                                            cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_prefix, pre.data(), sizeof(uint32_t) * pre.size(),
                                    cudaMemcpyHostToDevice, stream);
            prefix_n = (int)n;
            if (e != cudaSuccess) return cuda_(e, "work list upload");
        }
        // the array now holds the live descriptors (and step indices) of these
        // scenarios: every per-scenario call reads them there
        for (size_t i = 0; i < sims.size(); ++i) sims[i]->d_desc = d_descs + i;
        drop();
        return PEDSIM_OK;
    }

    int grid() const
    {
        const int per_sm = ctas_per_sm > 0 ? ctas_per_sm : fused_blocks_per_sm(tile_w, tile_h);
        const uint32_t capn = (uint32_t)sms * (uint32_t)per_sm;
        return (int)std::max<uint32_t>(1, std::min(total, capn));
    }

    int launch_steps(int k, cudaStream_t st)
    {
        const int n = prefix_n;
        for (int i = 0; i < k; ++i) {
            cudaError_t e =
                variant == kVariantFused
                    ? launch_fused_step(d_descs, d_prefix, count, total, i, tile_w, tile_h, grid(),
                                        d_act, st)
                : variant == kVariantAgent
                    ? launch_agent_step(d_descs, d_prefix + (n + 1), d_prefix + 2 * (n + 1), count,
                                        cell_total, agent_total, d_act, st)
                : variant == kVariantDeferred
                    ? launch_deferred_step(d_descs, d_prefix + (n + 1), d_prefix + 2 * (n + 1),
                                           d_prefix + 3 * (n + 1), count, slice_total,
                                           agent_total, d_act, st)
                    : launch_pipeline_step(d_descs, d_prefix, count, total, i, tile_h, st);
            if (e != cudaSuccess) return cuda_(e, "batched step launch");
        }
        if (self_advancing(variant)) return PEDSIM_OK;  // the step advanced itself
        cudaError_t e = launch_advance(d_descs, count, k, st);
        if (e != cudaSuccess) return cuda_(e, "advance launch");
        return PEDSIM_OK;
    }

    int step(int n)
    {
        if (n < 0) return fail_(PEDSIM_EINVAL, "negative step count");
        if (n == 0 || count == 0) return PEDSIM_OK;
        if (variant == kVariantFused) (void)fused_blocks_per_sm(tile_w, tile_h);
        const int full = n / kGraphSteps, rem = n % kGraphSteps;
        if (full > 0 && !graph) {
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_(e, "cudaStreamBeginCapture");
            int rc = launch_steps(kGraphSteps, cap);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cap, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { graph = nullptr; return cuda_(e, "cudaGraphInstantiate"); }
        }
        for (int i = 0; i < full; ++i) {
            cudaError_t e = cudaGraphLaunch(graph, stream);
            if (e != cudaSuccess) return cuda_(e, "cudaGraphLaunch");
        }
        if (rem) return launch_steps(rem, stream);
        return PEDSIM_OK;
    }

    void release()
    {
        drop();
        if (d_descs) cudaFreeAsync(d_descs, stream);
        if (d_prefix) cudaFreeAsync(d_prefix, stream);
        if (d_act) cudaFreeAsync(d_act, stream);
        d_descs = nullptr;
        d_prefix = nullptr;
        d_act = nullptr;
        act_capacity = 0;
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
    }
};

int retile(sim_t *s, int variant, int tw, int th, int cps)
{
    return switch_variant(s, variant, tw, th, cps);
}

}  // namespace

struct batch_s {
    std::vector<sim_t *> sims;
    MultiRun run;
};

struct pool_s {
    size_t budget = 0, in_use = 0;
    int max_slots = 0;
    // The slots' memory pool: it keeps up to the budget reserved when slots
    // are released (the device's default pool returns freed memory to the
    // system at the next synchronisation, so each admission would map its
    // pages again).
    cudaMemPool_t mem = nullptr;
    std::vector<sim_t *> slots;        // nullptr = free
    std::vector<size_t> bytes;
    bool dirty = true;
    MultiRun run;
};

extern "C" {

int sim_batch_create(int n, const int *W, const int *H, const sim_params *params,
                     const uint64_t *seeds, batch_t **out)
{
    if (!out || n <= 0 || !W || !H || !params || !seeds) return PEDSIM_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!params_ok(W[i], H[i], &params[i])) return PEDSIM_EINVAL;
    batch_t *b = new (std::nothrow) batch_t();
    if (!b) return PEDSIM_ENOMEM;
    b->run.sms = device_sms();
    if (cudaStreamCreateWithFlags(&b->run.cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return PEDSIM_ECUDA;
    }
    int rc = PEDSIM_OK;
    for (int i = 0; i < n && rc == PEDSIM_OK; ++i) {
        sim_t *s = nullptr;
        rc = pedsim_create_on_stream(W[i], H[i], &params[i], b->run.stream, &s);
        if (rc) { b->run.err = "scenario " + std::to_string(i) + " creation failed"; break; }
        b->sims.push_back(s);
        rc = sim_place(s, seeds[i]);
        if (rc) b->run.err = s->err;
    }
    if (rc == PEDSIM_OK) rc = b->run.load(b->sims);
    if (rc != PEDSIM_OK) {
        sim_batch_destroy(b);
        return rc;
    }
    *out = b;
    return PEDSIM_OK;
}

int sim_batch_set_stream(batch_t *b, void *stream)
{
    if (!b) return PEDSIM_EINVAL;
    b->run.stream = reinterpret_cast<cudaStream_t>(stream);
    for (sim_t *s : b->sims) s->stream = b->run.stream;
    return PEDSIM_OK;
}

int sim_batch_step(batch_t *b, int n)
{
    if (!b) return PEDSIM_EINVAL;
    int rc = b->run.step(n);
    if (rc) return rc;
    for (sim_t *s : b->sims) s->step += (unsigned long long)n;
    return PEDSIM_OK;
}

int sim_batch_stats(batch_t *b, int i, sim_stats_t *out)
{
    if (!b || i < 0 || i >= (int)b->sims.size()) return PEDSIM_ENOENT;
    int rc = sim_stats(b->sims[i], out);
    if (rc) b->run.err = b->sims[i]->err;
    return rc;
}

int sim_batch_read_grid(batch_t *b, int i, uint8_t *occ, uint32_t *ids, float *tauA, float *tauB)
{
    if (!b || i < 0 || i >= (int)b->sims.size()) return PEDSIM_ENOENT;
    int rc = sim_read_grid(b->sims[i], occ, ids, tauA, tauB);
    if (rc) b->run.err = b->sims[i]->err;
    return rc;
}

int sim_batch_set_tiling(batch_t *b, int tile_w, int tile_h, int ctas_per_sm)
{
    if (!b) return PEDSIM_EINVAL;
    const bool ok = !self_advancing(b->run.variant) &&
                    (b->run.variant == kVariantFused ? tile_supported(tile_w, tile_h)
                                                     : pipeline_tile_supported(tile_w, tile_h));
    if (!ok || ctas_per_sm < 0 || ctas_per_sm > 32) return PEDSIM_EINVAL;
    for (sim_t *s : b->sims) {
        int rc = retile(s, b->run.variant, tile_w, tile_h, ctas_per_sm);
        if (rc) { b->run.err = s->err; return rc; }
    }
    b->run.tile_w = tile_w;
    b->run.tile_h = tile_h;
    b->run.ctas_per_sm = ctas_per_sm;
    return b->run.load(b->sims);
}

int sim_batch_set_variant(batch_t *b, int variant)
{
    if (!b || (variant != kVariantPipeline && variant != kVariantFused &&
               variant != kVariantAgent && variant != kVariantDeferred))
        return PEDSIM_EINVAL;
    b->run.variant = variant;
    const int tw = variant == kVariantFused ? 64 : 128;
    for (sim_t *s : b->sims) {
        int rc = retile(s, variant, tw, 16, 0);
        if (rc) { b->run.err = s->err; return rc; }
    }
    b->run.tile_w = tw;
    b->run.tile_h = 16;
    b->run.ctas_per_sm = 0;
    return b->run.load(b->sims);
}

int sim_batch_device_status(batch_t *b)
{
    if (!b) return PEDSIM_EINVAL;
    int worst = 0;
    for (sim_t *s : b->sims) {
        int v = sim_device_status(s);
        if (v) worst = v;
    }
    return worst;
}

void sim_batch_destroy(batch_t *b)
{
    if (!b) return;
    b->run.release();
    for (sim_t *s : b->sims) sim_destroy(s);
    delete b;
}

const char *sim_batch_last_error(const batch_t *b)
{
    return b ? b->run.err.c_str() : "null handle";
}

// ---- serving pool ---------------------------------------------------------
int sim_pool_create(size_t hbm_budget_bytes, int max_slots, pool_t **out)
{
    if (!out || max_slots <= 0 || hbm_budget_bytes == 0) return PEDSIM_EINVAL;
    pool_t *pl = new (std::nothrow) pool_t();
    if (!pl) return PEDSIM_ENOMEM;
    pl->budget = hbm_budget_bytes;
    pl->max_slots = max_slots;
    pl->slots.assign((size_t)max_slots, nullptr);
    pl->bytes.assign((size_t)max_slots, 0);
    pl->run.sms = device_sms();
    if (cudaStreamCreateWithFlags(&pl->run.cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete pl;
        return PEDSIM_ECUDA;
    }
    int dev = 0;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    const unsigned long long keep = hbm_budget_bytes;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        (props.location.id = dev, cudaMemPoolCreate(&pl->mem, &props)) != cudaSuccess ||
        cudaMemPoolSetAttribute(pl->mem, cudaMemPoolAttrReleaseThreshold,
                                const_cast<unsigned long long *>(&keep)) != cudaSuccess) {
        cudaGetLastError();
        if (pl->mem) cudaMemPoolDestroy(pl->mem);
        cudaStreamDestroy(pl->run.cap);
        delete pl;
        return PEDSIM_ECUDA;
    }
    *out = pl;
    return PEDSIM_OK;
}

int sim_pool_set_stream(pool_t *pl, void *stream)
{
    if (!pl) return PEDSIM_EINVAL;
    pl->run.stream = reinterpret_cast<cudaStream_t>(stream);
    for (sim_t *s : pl->slots)
        if (s) s->stream = pl->run.stream;
    return PEDSIM_OK;
}

int sim_pool_admit(pool_t *pl, int W, int H, const sim_params *p, uint64_t seed, uint64_t steps,
                   int *slot)
{
    if (!pl || !slot || !params_ok(W, H, p)) return PEDSIM_EINVAL;
    const size_t need = make_layout(W, H, *p).total;
    int free_slot = -1;
    for (int i = 0; i < pl->max_slots; ++i)
        if (!pl->slots[i]) { free_slot = i; break; }
    if (free_slot < 0 || pl->in_use + need > pl->budget) {
        pl->run.err = "HBM budget or slot count exceeded";
        return PEDSIM_ENOSPC;
    }
    sim_t *s = nullptr;
    int rc = pedsim_create_on_stream(W, H, p, pl->run.stream, &s, pl->mem);
    if (rc) { pl->run.err = "slot creation failed"; return rc; }
    s->end_step = steps;
    rc = retile(s, pl->run.variant, pl->run.tile_w, pl->run.tile_h, pl->run.ctas_per_sm);
    if (rc == PEDSIM_OK) rc = sim_place(s, seed);
    if (rc) {
        pl->run.err = s->err;
        sim_destroy(s);
        return rc;
    }
    pl->slots[free_slot] = s;
    pl->bytes[free_slot] = need;
    pl->in_use += need;
    pl->dirty = true;
    *slot = free_slot;
    return PEDSIM_OK;
}

int sim_pool_step(pool_t *pl, int n)
{
    if (!pl || n < 0) return PEDSIM_EINVAL;
    if (pl->dirty) {
        std::vector<sim_t *> live;
        for (sim_t *s : pl->slots) {
            if (!s) continue;
            if (s->step < s->end_step) {
                live.push_back(s);
            } else if (s->d_desc != s->own_desc) {
                // leaving the work list: its own descriptor becomes live again
                int rc = upload_desc(s);
                if (rc) { pl->run.err = s->err; return rc; }
            }
        }
        int rc = pl->run.load(live);
        if (rc) return rc;
        pl->dirty = false;
    }
    int rc = pl->run.step(n);
    if (rc) return rc;
    for (sim_t *s : pl->slots)
        if (s) {
            const unsigned long long left = s->end_step - s->step;
            const bool was_live = left > 0;
            s->step += std::min<unsigned long long>(left, (unsigned long long)n);
            // finished slots drop out of the work list at the next rebuild
            if (was_live && s->step == s->end_step) pl->dirty = true;
        }
    return PEDSIM_OK;
}

int sim_pool_finished(pool_t *pl, int *done, int max, int *n_done)
{
    if (!pl || !n_done || (max > 0 && !done)) return PEDSIM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(pl->run.stream);
    if (e != cudaSuccess) return pl->run.cuda_(e, "pool synchronise");
    int k = 0;
    for (int i = 0; i < pl->max_slots; ++i) {
        sim_t *s = pl->slots[i];
        if (s && s->step >= s->end_step) {
            if (k < max) done[k] = i;
            ++k;
        }
    }
    *n_done = std::min(k, std::max(max, 0));
    return PEDSIM_OK;
}

int sim_pool_stats(pool_t *pl, int slot, sim_stats_t *out)
{
    if (!pl || slot < 0 || slot >= pl->max_slots || !pl->slots[slot]) return PEDSIM_ENOENT;
    int rc = sim_stats(pl->slots[slot], out);
    if (rc) pl->run.err = pl->slots[slot]->err;
    return rc;
}

int sim_pool_read_grid(pool_t *pl, int slot, uint8_t *occ, uint32_t *ids, float *tauA, float *tauB)
{
    if (!pl || slot < 0 || slot >= pl->max_slots || !pl->slots[slot]) return PEDSIM_ENOENT;
    int rc = sim_read_grid(pl->slots[slot], occ, ids, tauA, tauB);
    if (rc) pl->run.err = pl->slots[slot]->err;
    return rc;
}

int sim_pool_release(pool_t *pl, int slot)
{
    if (!pl || slot < 0 || slot >= pl->max_slots || !pl->slots[slot]) return PEDSIM_ENOENT;
    sim_destroy(pl->slots[slot]);
    pl->slots[slot] = nullptr;
    pl->in_use -= pl->bytes[slot];
    pl->bytes[slot] = 0;
    pl->dirty = true;
    return PEDSIM_OK;
}

size_t sim_pool_bytes_in_use(const pool_t *pl) { return pl ? pl->in_use : 0; }

int sim_pool_live(const pool_t *pl)
{
    if (!pl) return 0;
    int k = 0;
    for (sim_t *s : pl->slots) k += s != nullptr;
    return k;
}

void sim_pool_destroy(pool_t *pl)
{
    if (!pl) return;
    pl->run.release();
    for (sim_t *s : pl->slots)
        if (s) sim_destroy(s);
    // (the pool's memory is given back once the slots' stream-ordered frees
    // have run)
    if (pl->mem) cudaMemPoolDestroy(pl->mem);
    delete pl;
}

const char *sim_pool_last_error(const pool_t *pl)
{
    return pl ? pl->run.err.c_str() : "null handle";
}

}  // extern "C"
