// Allocation-free single step (sim_step_noalloc in include/pedsim.h).
//
// Some callers cannot let a library allocate device memory while they run:
// applications that reserve all device memory up front under a fixed budget,
// frameworks whose caching allocator must account for every byte (a hidden
// cudaMalloc there fragments or exhausts its pool), and code that records
// work into a CUDA graph, where an allocation would become a graph memory
// node or fail.  sim_step_noalloc serves them: the caller owns every input and
// output buffer, the scenario parameters travel by value, and the only
// scratch the step needs -- the one-byte proposal plane between the proposal
// pass and the resolution pass -- lives in the file-scope device array below,
// which exists on every GPU that loads the library for as long as the library
// stays loaded.  The call never allocates or frees memory.
//
// The two kernels are the plain two-pass step (one thread per cell) with the
// scenario passed as a kernel argument instead of a device descriptor.
#include "pedsim.h"
#include "pedsim_internal.h"
#include "pedsim_rules.cuh"

#include <mutex>

namespace pedsim {
namespace {

// Largest grid the array serves: 2^24 cells (16 MiB), e.g. 4096 x 4096.
constexpr size_t kNoAllocMaxCells = size_t(1) << 24;

// The proposal plane of the allocation-free step.  Every call writes each of
// its W*H entries in the proposal pass before the resolution pass reads it,
// so nothing in it has to start at zero; calls share it, so two calls that
// overlap on the GPU race.
static __device__ __align__(256) uint8_t g_noalloc_prop[kNoAllocMaxCells];

struct NoAllocStep {
    int W, H;
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

constexpr int kNaThreads = 256;

__global__ void __launch_bounds__(kNaThreads)
noalloc_propose_kernel(const __grid_constant__ NoAllocStep a, uint8_t *__restrict__ prop)
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
            const float *tp = a.model == 1 ? a.tau_in[g == 2 ? 1 : 0] : nullptr;
            code = propose(
                x, y, g, W, H, (uint64_t)c, a.step, a.seed, rp,
                [&](int dx, int dy) { return (int)a.occ_in[(int64_t)c + (int64_t)dy * W + dx]; },
                tp ? tp + c : nullptr, W);
        }
        prop[c] = (uint8_t)code;
    }
}

__global__ void __launch_bounds__(kNaThreads)
noalloc_resolve_kernel(const __grid_constant__ NoAllocStep a, const uint8_t *__restrict__ prop)
{
    const int W = a.W, H = a.H;
    const size_t cells = (size_t)W * H;
    unsigned moved = 0, conflicts = 0, crossed_a = 0, crossed_b = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x; base < cells; base += stride) {
        const size_t c = base + threadIdx.x;
        if (c >= cells) continue;
        const int x = (int)(c % (size_t)W), y = (int)(c / (size_t)W);
        auto prop_at = [&](int dx, int dy) { return (int)prop[(int64_t)c + (int64_t)dy * W + dx]; };
        const int o = a.occ_in[c];
        int no = o, incoming = 0;
        float dep = a.deposit;
        if (o == 0) {
            int k;
            const int w = resolve_winner(x, y, W, H, (uint64_t)c, a.step, a.seed, prop_at, &k);
            if (w >= 0) {
                const int dx = kCodeDX[w + 1], dy = kCodeDY[w + 1];
                const size_t src = (size_t)((int64_t)c + (int64_t)dy * W + dx);
                incoming = a.occ_in[src];
                no = incoming;
                const uint32_t id = a.ids[src];
                a.ids[c] = id;
                ++moved;
                if (k >= 2) ++conflicts;
                if (a.model == 1 && a.deposit_mode == 1) {
                    const float L = __fadd_rn(a.tour[id], (dx != 0 && dy != 0) ? kSqrt2 : 1.0f);
                    a.tour[id] = L;
                    dep = __fdiv_rn(1.0f, L);
                }
                const bool in_band = incoming == 1 ? x >= W - (int)a.band : x < (int)a.band;
                if (in_band && a.arrival[id] == 0) {
                    a.arrival[id] = (uint32_t)(a.step + 1);
                    if (incoming == 1) ++crossed_a; else ++crossed_b;
                }
            }
        } else {
            const int code = prop[c];
            if (code) {
                const int dx = kCodeDX[code], dy = kCodeDY[code];
                int k;
                const int w = resolve_winner(
                    x + dx, y + dy, W, H, (uint64_t)((int64_t)c + (int64_t)dy * W + dx), a.step,
                    a.seed, [&](int ex, int ey) { return prop_at(dx + ex, dy + ey); }, &k);
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
    // warp totals into the caller's counters
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

// Device address of g_noalloc_prop, looked up once per device with that
// device current (host code cannot use the symbol itself: in host code its
// name stands for a host-side shadow, not device memory).
constexpr int kMaxDevices = 64;
// Per device, looked up once with that device current: the array's device
// address and the grid cap of the grid-stride kernels (16 CTAs per SM).  A
// cudaDeviceReset destroys the context these belong to; the library does not
// notice one, so the cached address must not be used after a reset.
std::mutex g_addr_mutex;
uint8_t *g_addr[kMaxDevices] = {};
unsigned g_max_blocks[kMaxDevices] = {};

int scratch_address(uint8_t **out, unsigned *max_blocks)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PEDSIM_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        int sms = 0;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_prop) != cudaSuccess || !ptr ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0) {
            cudaGetLastError();
            return PEDSIM_ECUDA;
        }
        g_max_blocks[dev] = 16u * (unsigned)sms;
        g_addr[dev] = static_cast<uint8_t *>(ptr);
    }
    *out = g_addr[dev];
    *max_blocks = g_max_blocks[dev];
    return PEDSIM_OK;
}

// [a, a + n) and [b, b + n) share a byte.
bool overlap(const void *a, const void *b, size_t n)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + n && y < x + n;
}

}  // namespace
}  // namespace pedsim

using namespace pedsim;

extern "C" int sim_step_noalloc(int W, int H, const sim_params *p, uint64_t seed, uint64_t step,
                                const uint8_t *occ_in, uint8_t *occ_out, uint32_t *ids,
                                const float *tauA_in, const float *tauB_in, float *tauA_out,
                                float *tauB_out, uint32_t *arrival, float *tour,
                                unsigned long long *counters, void *stream)
{
    if (sim_validate(W, H, p) != PEDSIM_OK) return PEDSIM_EINVAL;
    if ((size_t)W * (size_t)H > kNoAllocMaxCells) return PEDSIM_EINVAL;
    const bool aco = p->model == PEDSIM_ACO;
    const size_t cells = (size_t)W * H;
    if (!occ_in || !occ_out || !ids || !arrival) return PEDSIM_EINVAL;
    // the resolution pass reads occ_in around every cell while it writes
    // occ_out: the two may not share a byte
    if (overlap(occ_in, occ_out, cells)) return PEDSIM_EINVAL;
    if (aco && (!tauA_in || !tauB_in || !tauA_out || !tauB_out)) return PEDSIM_EINVAL;
    if (aco && p->deposit_mode == 1 && !tour) return PEDSIM_EINVAL;
    uint8_t *prop = nullptr;
    unsigned max_blocks = 0;
    const int rc = scratch_address(&prop, &max_blocks);
    if (rc != PEDSIM_OK) return rc;

    NoAllocStep a{};
    a.W = W;
    a.H = H;
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

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    size_t blocks = (cells + kNaThreads - 1) / kNaThreads;
    if (blocks > max_blocks) blocks = max_blocks;
    noalloc_propose_kernel<<<(unsigned)blocks, kNaThreads, 0, st>>>(a, prop);
    if (cudaGetLastError() != cudaSuccess) return PEDSIM_ECUDA;
    noalloc_resolve_kernel<<<(unsigned)blocks, kNaThreads, 0, st>>>(a, prop);
    if (cudaGetLastError() != cudaSuccess) return PEDSIM_ECUDA;
    return PEDSIM_OK;
}
