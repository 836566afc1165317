// Shared-memory staging of the gathered spinor field of an FP32 stencil kernel.
//
// A block computes the Wilson hopping term at a contiguous range of sites
// [s0, s0 + nb), nb <= kStageSites.  Before it starts, one thread copies into shared
// memory, with bulk asynchronous copies (cp.async.bulk, the TMA unit) completing on an
// mbarrier, the five site ranges from which the block gathers:
//   R0  [s0 - Lx, s0 + nb + Lx)  the sites themselves and every x-neighbour and
//                                non-wrapping y-neighbour,
//   R1  [s0 + P, s0 + nb + P)    the non-wrapping z+ neighbours (P = Lx Ly),
//   R2  [s0 - P, s0 + nb - P)    z-,
//   R3  [s0 + S, s0 + nb + S)    t+ (S = Lx Ly Lz),
//   R4  [s0 - S, s0 + nb - S)    t-,
// each clipped to [0, V), for each of the 6 float4 planes of the field.  The copies are
// issued together, so the block's gathers are in flight at once instead of one
// neighbour after another; a neighbour whose hop wraps around the lattice in y, z or t
// (a small fraction of the sites) is read from global memory.  The copy of a range
// starts and ends on 16-byte boundaries (one float4 per site and plane).
//
// Shared layout: plane c at c * stage_len(Lx) float4; within it R0 at 0 (site n at
// n - s0 + Lx), then R1..R4 at 2 Lx + kStageSites + (r - 1) kStageSites.
#pragma once

#include <cstdint>

#include "wilson_site.cuh"

namespace dlz {

constexpr int kStageSites = 128;

__host__ __device__ inline int stage_len(int Lx) { return 2 * Lx + 5 * kStageSites; }
__host__ __device__ inline int stage_bytes(int Lx) { return 6 * stage_len(Lx) * 16; }

struct StagedGather32 {
    const float4 *__restrict__ in;   // the field in global memory (wrapped neighbours)
    const float4 *sm;                // the staged planes
    int V, len;
    int b0, b1, b2, b3, b4;          // shared index of site n in range r: n + b_r
    template <int MU, int DIR>
    __device__ inline void get(int n, bool wrapped, float2 (&p)[12]) const {
        int idx;
        if (MU == 0 || DIR == 0) {
            idx = n + b0;                                  // x hops stay within R0
        } else if (wrapped) {
            Field<float>::load(in, V, n, p);
            return;
        } else if (MU == 1) {
            idx = n + b0;
        } else if (MU == 2) {
            idx = DIR > 0 ? n + b1 : n + b2;
        } else {
            idx = DIR > 0 ? n + b3 : n + b4;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 q = sm[c * len + idx];
            p[2 * c] = make_float2(q.x, q.y);
            p[2 * c + 1] = make_float2(q.z, q.w);
        }
    }
};

__device__ __forceinline__ uint32_t stage_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Issue the staging copies of the block's ranges (one thread): one arrival on `mbar`
// (initialised with an arrival count of 1) that expects every copied byte.
__device__ inline void stage_issue(const float4 *__restrict__ in, const Geom &g, int s0, int nb, float4 *sm,
                                   uint64_t *mbar) {
    const int Lx = g.L[0], P = g.L[0] * g.L[1], S = P * g.L[2], V = g.V, len = stage_len(Lx);
    int lo[5], hi[5], at[5];
    lo[0] = max(0, s0 - Lx);  hi[0] = min(V, s0 + nb + Lx);  at[0] = lo[0] - (s0 - Lx);
    lo[1] = s0 + P;           hi[1] = min(V, s0 + nb + P);   at[1] = 2 * Lx + kStageSites;
    lo[2] = max(0, s0 - P);   hi[2] = s0 + nb - P;           at[2] = 2 * Lx + 2 * kStageSites + (lo[2] - (s0 - P));
    lo[3] = s0 + S;           hi[3] = min(V, s0 + nb + S);   at[3] = 2 * Lx + 3 * kStageSites;
    lo[4] = max(0, s0 - S);   hi[4] = s0 + nb - S;           at[4] = 2 * Lx + 4 * kStageSites + (lo[4] - (s0 - S));
    uint32_t tx = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r)
        if (hi[r] > lo[r]) tx += 6u * (uint32_t)(hi[r] - lo[r]) * 16u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(stage_smem_u32(mbar)), "r"(tx)
                 : "memory");
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        if (hi[r] <= lo[r]) continue;
        const uint32_t bytes = (uint32_t)(hi[r] - lo[r]) * 16u;
        for (int c = 0; c < 6; ++c) {
            const float4 *src = in + (size_t)c * V + lo[r];
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    stage_smem_u32(sm + (size_t)c * len + at[r])),
                "l"(src), "r"(bytes), "r"(stage_smem_u32(mbar))
                : "memory");
        }
    }
}

__device__ inline StagedGather32 staged_gather(const float4 *__restrict__ in, const Geom &g, int s0, const float4 *sm) {
    const int Lx = g.L[0], P = g.L[0] * g.L[1], S = P * g.L[2];
    StagedGather32 ga;
    ga.in = in;
    ga.sm = sm;
    ga.V = g.V;
    ga.len = stage_len(Lx);
    ga.b0 = Lx - s0;
    ga.b1 = 2 * Lx + kStageSites - (s0 + P);
    ga.b2 = 2 * Lx + 2 * kStageSites - (s0 - P);
    ga.b3 = 2 * Lx + 3 * kStageSites - (s0 + S);
    ga.b4 = 2 * Lx + 4 * kStageSites - (s0 - S);
    return ga;
}

// Bounded wait for phase 0 of the staging mbarrier; false if it gave up.
__device__ inline bool stage_wait(uint64_t *mbar, long long polls) {
    uint32_t done = 0;
    for (long long it = 0; it < polls && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(stage_smem_u32(mbar))
                     : "memory");
    }
    return done != 0;
}

__device__ inline void stage_init(uint64_t *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(stage_smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Polls of a staging wait before it gives up (each poll may suspend the thread for a
// while; a completed copy of the block's ranges takes microseconds)
constexpr long long kStagePolls = 1LL << 24;

// Start of a staged kernel (all threads of the block call it): the copies of the ranges
// of `in` around [s0, s0 + nb) into sm, then the wait for them.  A block whose wait
// gives up sets *err, waits once more for its copies and returns false (the caller then
// leaves its outputs alone).  STAGED = false: nothing to do.
template <bool STAGED>
__device__ inline bool stage_begin(const float4 *__restrict__ in, const Geom &g, int s0, int nb, float4 *sm,
                                   uint64_t *mbar, int *err) {
    if (!STAGED || nb <= 0) return true;
    if (threadIdx.x == 0) stage_init(mbar);
    __syncthreads();
    if (threadIdx.x == 0) stage_issue(in, g, s0, nb, sm, mbar);
    if (stage_wait(mbar, kStagePolls)) return true;
    atomicExch(err, 1);
    stage_wait(mbar, kStagePolls);
    return false;
}

}  // namespace dlz
