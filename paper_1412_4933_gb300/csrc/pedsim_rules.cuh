// Device-side rules of one synchronous step of the bi-directional pedestrian
// cellular automaton (Dutta, McLeod, Friesen, Sec. III-IV): the move proposal
// of one agent (forward first, else Eq. 1 for LEM or Eq. 2 for ACO) and the
// gather-side conflict resolution of one target cell (Sec. IV.d).
//
// Every float operation uses an explicitly rounded intrinsic (__fmul_rn,
// __fadd_rn, __fdiv_rn), which the compiler never fuses into an FMA; the
// library is additionally built with -fmad=false and without fast-math, so
// subnormals are kept.
#pragma once
#include <cstdint>

namespace pedsim {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64
// -> 128-bit products on words 0 and 2, half-swaps across the pairs, key xor,
// Weyl key bumps between rounds.
// ---------------------------------------------------------------------------
struct Rand4 { uint64_t r0, r1, r2, r3; };

__device__ __forceinline__ Rand4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                uint64_t c3, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ull, kMulB = 0xCA5A826395121157ull;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ull, kWeylB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hiA = __umul64hi(kMulA, c0), loA = kMulA * c0;
        const uint64_t hiB = __umul64hi(kMulB, c2), loB = kMulB * c2;
        const uint64_t n0 = hiB ^ c1 ^ k0;
        const uint64_t n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kWeylA; k1 += kWeylB;
    }
    return Rand4{c0, c1, c2, c3};
}

// Counter layout: (cell index, step, stream, 0); key: (seed, 0).
enum : uint64_t { kStreamPropose = 1, kStreamConflict = 2, kStreamPlace = 3 };

__device__ __forceinline__ Rand4 draw(uint64_t seed, uint64_t cell, uint64_t step,
                                      uint64_t stream)
{
    return philox4x64_10(cell, step, stream, 0, seed, 0);
}

// ---------------------------------------------------------------------------
// Direction codes.  A proposal is stored as an absolute code 0..8: 0 = stay,
// code j+1 = the j-th offset of the fixed row-major scan
// (dy,dx) = (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1).
// The offset of code 9-c is the negation of the offset of code c, so the
// neighbour at scan offset j of a cell T claims T iff its code is 8-j.
// ---------------------------------------------------------------------------
__constant__ const int8_t kCodeDX[9] = {0, -1, 0, 1, -1, 1, -1, 0, 1};
__constant__ const int8_t kCodeDY[9] = {0, -1, -1, -1, 0, 0, 1, 1, 1};

// Agent-frame neighbour i (1 forward, 2/3 forward-left/right, 4/5 left/right,
// 6 back, 7/8 back-left/right; "left" of the heading) -> absolute code, for a
// group A agent heading +x (row 0) and a group B agent heading -x (row 1).
__constant__ const uint8_t kFrameCode[2][9] = {
    {0, 5, 3, 8, 2, 7, 4, 1, 6},
    {0, 4, 6, 1, 7, 2, 5, 8, 3},
};

// eta_i = 1/D_i, D_i = distance from neighbour i to the point two cells
// ahead of the agent: 1, sqrt2, sqrt2, sqrt5, sqrt5, 3, sqrt10, sqrt10
// (correctly rounded binary32).
__constant__ const float kEta[9] = {
    0.0f, 0x1p+0f, 0x1.6a09e6p-1f, 0x1.6a09e6p-1f, 0x1.c9f25cp-2f, 0x1.c9f25cp-2f,
    0x1.555556p-2f, 0x1.43d136p-2f, 0x1.43d136p-2f};

constexpr float kSqrt2 = 0x1.6a09e6p+0f;  // fl(sqrt 2): diagonal tour length

struct RuleParams {
    uint32_t model;         // 0 LEM, 1 ACO
    uint32_t alpha, beta;   // Eq. 2 exponents
    float lem_scale;        // fl(2^-16 / sigma)
};

// Sum of the twelve 16-bit words of r0, r1, r2 (the normal draw's uniforms).
__device__ __forceinline__ int32_t twelve_word_sum(const Rand4 &r)
{
    constexpr uint64_t kLanes = 0x0000FFFF0000FFFFull;
    const uint64_t a = (r.r0 & kLanes) + ((r.r0 >> 16) & kLanes);
    const uint64_t b = (r.r1 & kLanes) + ((r.r1 >> 16) & kLanes);
    const uint64_t c = (r.r2 & kLanes) + ((r.r2 >> 16) & kLanes);
    const uint64_t t = a + b + c;  // two 32-bit lanes, each <= 393210
    return (int32_t)((t & 0xFFFFFFFFull) + (t >> 32));
}

// LEM rank: z = (sum - 393210) * 2^-16 / sigma; negative -> 0; rounded half
// up; clamped to the last rank m-1 (Sec. II.A).
__device__ __forceinline__ int lem_rank(int32_t sum12, int m, float scale)
{
    const float z = __fmul_rn(__int2float_rn(sum12 - 393210), scale);
    const int k = (int)floorf(__fadd_rn(fmaxf(z, 0.0f), 0.5f));
    return k < m - 1 ? k : m - 1;
}

__device__ __forceinline__ float int_pow(float v, uint32_t e)
{
    float p = 1.0f;
    if (e >= 1) p = v;
    for (uint32_t i = 1; i < e; ++i) p = __fmul_rn(p, v);
    return p;
}

// Own-group pheromone at offset (dx, dy) from an agent, read from a plane or
// a shared-memory tile: c points at the agent's own cell, stride is the row
// pitch in elements.  A reader has two phases so that every neighbour's load
// is issued before any value is used: fetch() loads (value, aux) and
// finish() turns the fetched entries of the available neighbours into the
// values at the current step (here they already are).
// fetch() takes the frame index i (1..8) of the neighbour and its absolute
// code.
struct PlaneTau {
    const float *c;
    int stride;
    __device__ __forceinline__ float fetch(int, int code, uint32_t &aux) const
    {
        aux = 0;
        return c[kCodeDY[code] * stride + kCodeDX[code]];
    }
    __device__ __forceinline__ void finish(float (&)[9], const uint32_t (&)[9], unsigned) const {}
};

// Choice of an agent whose forward cell is blocked (Sec. II.A, II.B, IV.c).
// avail: bit i set when frame neighbour i is in the grid and empty.  For ACO
// tau(dx, dy) returns the own-group pheromone at step t at offset (dx, dy)
// from the agent (read only at available neighbours).  Kept out of line: it
// is the rare, heavy path (one Philox block).
template <class TauFn>
static __device__ __noinline__ int choose_blocked(unsigned avail, int side, TauFn tau,
                                                  uint64_t cell, uint64_t step, uint64_t seed,
                                                  RuleParams rp)
{
    const Rand4 r = draw(seed, cell, step, kStreamPropose);

    if (rp.model == 1) {
        float tv[9], w[9];
        uint32_t aux[9];
#pragma unroll
        for (int i = 2; i <= 8; ++i) {
            tv[i] = 0.0f;
            aux[i] = 0;
            if (avail & (1u << i)) {
                tv[i] = tau.fetch(i, kFrameCode[side][i], aux[i]);
            }
        }
        tau.finish(tv, aux, avail);
        float S = 0.0f;
#pragma unroll
        for (int i = 2; i <= 8; ++i) {
            w[i] = 0.0f;
            if (avail & (1u << i)) w[i] = __fmul_rn(int_pow(tv[i], rp.alpha), int_pow(kEta[i], rp.beta));
            S = __fadd_rn(S, w[i]);
        }
        if (S > 0.0f) {
            const float u = __fmul_rn(__uint2float_rn((uint32_t)(r.r3 >> 40)), 0x1p-24f);
            const float target = __fmul_rn(u, S);
            float cum = 0.0f;
            int pick = 0;
            bool found = false;
#pragma unroll
            for (int i = 2; i <= 8; ++i) {
                cum = __fadd_rn(cum, w[i]);
                if (!found) {
                    if (w[i] > 0.0f) pick = i;
                    if (target < cum) found = true;
                }
            }
            return kFrameCode[side][pick];
        }
        // every weight zero: least-effort fallback
    }

    // LEM (Eq. 1): available cells by rank; equal pairs ordered by r3 bits
    int order[8] = {1, 2, 3, 4, 5, 6, 7, 8};
    if (r.r3 & 1u) { order[1] = 3; order[2] = 2; }
    if (r.r3 & 2u) { order[3] = 5; order[4] = 4; }
    if (r.r3 & 4u) { order[6] = 8; order[7] = 7; }
    int m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) m += (avail >> order[j]) & 1u;
    if (m == 0) return 0;
    const int k = lem_rank(twelve_word_sum(r), m, rp.lem_scale);
    int seen = 0, pick = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if ((avail >> order[j]) & 1u) {
            if (seen == k) pick = order[j];
            ++seen;
        }
    }
    return kFrameCode[side][pick];
}

// Proposal of an agent of group g (1 or 2) at (x, y) in a W x H grid at
// step t.  `occ(dx, dy)` returns the occupancy byte of the in-grid cell at
// that offset; `tau` reads the agent's own-group pheromone at t (ACO, see
// choose_blocked).  Returns the absolute direction code 0..8.
// An agent on its goal edge column stays there (Sec. III).
__device__ __forceinline__ bool parked(int x, int g, int W)
{
    return (g == 1 && x == W - 1) || (g == 2 && x == 0);
}

// Bit i (1..8) set when frame neighbour i of an agent of group g at (x, y)
// is in the grid and empty; occ(dx, dy) reads the in-grid neighbours.
template <class OccFn>
__device__ __forceinline__ unsigned frame_avail(int x, int y, int g, int W, int H, OccFn occ)
{
    const int side = g - 1;
    unsigned avail = 0;
#pragma unroll
    for (int i = 1; i <= 8; ++i) {
        const int code = kFrameCode[side][i];
        const int dx = kCodeDX[code], dy = kCodeDY[code];
        const int nx = x + dx, ny = y + dy;
        const bool inside = (unsigned)nx < (unsigned)W && (unsigned)ny < (unsigned)H;
        if (inside && occ(dx, dy) == 0) avail |= 1u << i;
    }
    return avail;
}

template <class OccFn, class TauFn>
__device__ __forceinline__ int propose_with(int x, int y, int g, int W, int H, uint64_t cell,
                                            uint64_t step, uint64_t seed, const RuleParams &rp,
                                            OccFn occ, TauFn tau)
{
    const int side = g - 1;
    if (parked(x, g, W)) return 0;
    const unsigned avail = frame_avail(x, y, g, W, H, occ);
    // forward first (Sec. III): no further calculation when #1 is free
    if (avail & 2u) return kFrameCode[side][1];
    return choose_blocked(avail, side, tau, cell, step, seed, rp);
}

// The same with the pheromone read from a plane or tile (tau_c points at the
// agent's own cell, tau_stride is the row pitch).
template <class OccFn>
__device__ __forceinline__ int propose(int x, int y, int g, int W, int H, uint64_t cell,
                                       uint64_t step, uint64_t seed, const RuleParams &rp,
                                       OccFn occ, const float *tau_c, int tau_stride)
{
    return propose_with(x, y, g, W, H, cell, step, seed, rp, occ, PlaneTau{tau_c, tau_stride});
}

// Scan index of the winning claimant of a cell with claim mask m (bit j set:
// the neighbour at scan offset j chose the cell) and k = popcount(m) >= 2:
// claimant floor(r * k / 2^32) in scan order, r from Philox stream 2 keyed by
// the target cell (Sec. IV.d).
static __device__ __noinline__ uint32_t pick_claimant(uint32_t m, uint32_t k, uint64_t cell,
                                                      uint64_t step, uint64_t seed)
{
    const Rand4 r = draw(seed, cell, step, kStreamConflict);
    const uint32_t idx = (uint32_t)(((uint64_t)(uint32_t)(r.r0 >> 32) * (uint64_t)k) >> 32);
    for (uint32_t u = 0; u < idx; ++u) m &= m - 1u;  // drop the idx lowest claimants
    return (uint32_t)(__ffs(m) - 1);
}

// Gather resolution of target cell (x, y) at step t (Sec. IV.d): the
// neighbours whose code points at it are the claimants, in scan order; one
// wins uniformly (Philox stream 2 keyed by the target cell) when k >= 2.
// `prop(dx, dy)` returns the code of the in-grid neighbour at that offset.
// Returns the scan index 0..7 of the winner, or -1; *k_out = claimant count.
template <class PropFn>
__device__ __forceinline__ int resolve_winner(int x, int y, int W, int H, uint64_t cell,
                                              uint64_t step, uint64_t seed, PropFn prop,
                                              int *k_out)
{
    uint32_t m = 0;  // bit j: the neighbour at scan offset j claims (x, y)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int dx = kCodeDX[j + 1], dy = kCodeDY[j + 1];
        const int nx = x + dx, ny = y + dy;
        const bool inside = (unsigned)nx < (unsigned)W && (unsigned)ny < (unsigned)H;
        if (inside && prop(dx, dy) == 8 - j) m |= 1u << j;
    }
    const int k = __popc(m);
    *k_out = k;
    if (k == 0) return -1;
    if (k == 1) return __ffs(m) - 1;
    return (int)pick_claimant(m, (uint32_t)k, cell, step, seed);
}

}  // namespace pedsim
