// D-MinRes on many lattices of uneven size at once (arXiv:0901.3163, Sec. 2,
// applied lattice by lattice): every (lattice, right-hand side) pair is a slot
// with its own geometry, links, kappa and deflation set, and the fused FP32
// MinRes kernels of minres_fused.cu run over all slots in one launch per stage.
// Each launch walks a block table (block -> slot, first 128-site chunk), built on
// the host with each slot's chunks contiguous, so the per-slot sums of chunk
// partials are contiguous ranges read in a fixed order (deterministic, and the same
// for every block size).  The FP64 defect
// correction around it (true residuals, Galerkin projection over each lattice's
// deflation set, x updates) runs lattice by lattice with that lattice's operator.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "minres_state.cuh"
#include "prec.cuh"
#include "reduce.cuh"
#include "small_dense.h"
#include "solvers.h"
#include "wilson_site.cuh"

namespace dlz {

struct SlotDesc {
    Geom g;
    float kappa;
    int blk0, nb;                 // first chunk partial and number of 128-site chunks
    const float4 *links;          // FP32 two-row links of the slot's lattice
    size_t off;                   // float4 offset of the slot's vectors in the arenas
};

namespace {

constexpr int kMT = 128;

struct Scales16 {            // per-right-hand-side scale factors captured by value
    double v[16];
};

// Per-chunk partials: a block of TB = B * kMT threads covers B chunks of kMT sites of
// one slot; each chunk's partial (FP64 over its threads) goes to its own slot in the
// partials array, so the sums -- and the results -- do not depend on B.
template <int B>
__device__ inline void chunk_partials(float facc, double *__restrict__ out, int nvalid) {
    double acc = (double)facc;
    __shared__ double sm[B * kMT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if ((threadIdx.x % kMT) == 0) {
        const int ch = threadIdx.x / kMT;
        if (ch < nvalid) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kMT / 32; ++w) t += sm[ch * (kMT / 32) + w];
            out[ch] = t;
        }
    }
}

// sum of partials[blk0 .. blk0 + nb) in a fixed order (valid in thread 0)
__device__ inline double slot_sum(const double *__restrict__ partials, int blk0, int nb) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += partials[blk0 + b];
    __shared__ double sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    double a = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) a += sm[w];
    return a;
}

// table entry of a block: (slot, first chunk of the block within the slot)
template <int B>
__global__ void __launch_bounds__(B * kMT)
k_mm_norm(const float4 *__restrict__ R, const SlotDesc *__restrict__ sd, const int2 *__restrict__ table,
          double *__restrict__ partials) {
    const int2 t = table[blockIdx.x];
    const SlotDesc d = sd[t.x];
    const int s = t.y * kMT + threadIdx.x;
    float facc = 0.f;
    if (s < d.g.V) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 v = R[d.off + (size_t)c * d.g.V + s];
            facc += (v.x * v.x + v.y * v.y) + (v.z * v.z + v.w * v.w);
        }
    }
    chunk_partials<B>(facc, partials + d.blk0 + t.y, d.nb - t.y);
}

__global__ void __launch_bounds__(256)
k_mm_init(const double *__restrict__ partials, const SlotDesc *__restrict__ sd, FusedState *__restrict__ st) {
    const SlotDesc d = sd[blockIdx.x];
    const double r2 = slot_sum(partials, d.blk0, d.nb);
    if (threadIdx.x == 0) fused_init(st[blockIdx.x], sqrt(r2));
}

template <int B>
__global__ void __launch_bounds__(B * kMT)
k_mm_k1(const float4 *__restrict__ U, const float4 *__restrict__ Up, float4 *__restrict__ W,
        const float4 *__restrict__ D2, float4 *__restrict__ D3, float4 *__restrict__ E,
        const SlotDesc *__restrict__ sd, const int2 *__restrict__ table, const FusedState *__restrict__ st,
        const int *__restrict__ active, double *__restrict__ partials) {
    const int2 t = table[blockIdx.x];
    const SlotDesc d = sd[t.x];
    if (!active[t.x]) {                 // a finished slot: its blocks do no work (uniform per block)
        if (threadIdx.x % kMT == 0 && t.y + (int)(threadIdx.x / kMT) < d.nb)
            partials[d.blk0 + t.y + threadIdx.x / kMT] = 0.0;
        return;
    }
    const int s = t.y * kMT + threadIdx.x;
    float facc = 0.f;
    if (s < d.g.V)
        facc = minres_k1_site(s, d.g, d.kappa, U + d.off, Up + d.off, W + d.off, D2 + d.off, D3 + d.off,
                              E + d.off, d.links, st[t.x]);
    chunk_partials<B>(facc, partials + d.blk0 + t.y, d.nb - t.y);
}

__global__ void __launch_bounds__(256)
k_mm_alpha(const double *__restrict__ partials, const SlotDesc *__restrict__ sd, FusedState *__restrict__ st,
           const int *__restrict__ active) {
    if (!active[blockIdx.x]) return;
    const SlotDesc d = sd[blockIdx.x];
    const double a = slot_sum(partials, d.blk0, d.nb);
    if (threadIdx.x == 0) fused_alpha(st[blockIdx.x], a);
}

template <int B>
__global__ void __launch_bounds__(B * kMT)
k_mm_k2a(float4 *__restrict__ W, const float4 *__restrict__ U, const SlotDesc *__restrict__ sd,
         const int2 *__restrict__ table, const FusedState *__restrict__ st, const int *__restrict__ active,
         double *__restrict__ partials) {
    const int2 t = table[blockIdx.x];
    const SlotDesc d = sd[t.x];
    if (!active[t.x]) {
        if (threadIdx.x % kMT == 0 && t.y + (int)(threadIdx.x / kMT) < d.nb)
            partials[d.blk0 + t.y + threadIdx.x / kMT] = 0.0;
        return;
    }
    const int s = t.y * kMT + threadIdx.x;
    float facc = 0.f;
    if (s < d.g.V) facc = minres_k2a_site(s, d.g.V, W + d.off, U + d.off, st[t.x]);
    chunk_partials<B>(facc, partials + d.blk0 + t.y, d.nb - t.y);
}

__global__ void __launch_bounds__(256)
k_mm_k2b(const double *__restrict__ partials, const SlotDesc *__restrict__ sd, FusedState *__restrict__ st,
         const int *__restrict__ active) {
    if (!active[blockIdx.x]) return;
    const SlotDesc d = sd[blockIdx.x];
    const double r2 = slot_sum(partials, d.blk0, d.nb);
    if (threadIdx.x == 0) {
        FusedState s = st[blockIdx.x];
        fused_givens(s, r2);
        st[blockIdx.x] = s;
    }
}

template <int B>
__global__ void __launch_bounds__(B * kMT)
k_mm_last(const float4 *__restrict__ Uj, const float4 *__restrict__ D2, const float4 *__restrict__ D3,
          float4 *__restrict__ E, const SlotDesc *__restrict__ sd, const int2 *__restrict__ table,
          const FusedState *__restrict__ st) {
    const int2 t = table[blockIdx.x];
    const SlotDesc d = sd[t.x];
    const int s = t.y * kMT + threadIdx.x;
    if (s >= d.g.V) return;
    const FusedState q = st[t.x];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const size_t i = d.off + (size_t)c * d.g.V + s;
        float4 ev = E[i];
        minres_last_direction(Uj[i], D2[i], D3[i], ev, q);
        E[i] = ev;
    }
}

// ------------------------------------------------------------------ persistent form
// One cooperative launch runs every stage of every iteration for all slots, the stages
// separated by grid-wide barriers (all blocks are co-resident: the launch is
// cooperative and sized by the occupancy calculator).  Each barrier wait is bounded:
// a block that has waited `limit` polls sets the error word and returns, and so does
// every block that later finds the word set, so a lost block can never hang the
// kernel; the host turns the word into DLZ_ERR_DEVICE_TIMEOUT.
struct GridBar {
    unsigned count;      // blocks arrived at the current barrier
    unsigned gen;        // barrier generation
    int err;             // 1: a wait gave up
    int groups;          // 6-iteration groups completed (written by block 0)
};

__device__ inline bool grid_wait(GridBar *gb, long long limit) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *genp = &gb->gen;
        const unsigned g = *genp;
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            long long n = 0;
            while (*genp == g) {
                if (++n > limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (!ok) atomicExch(&gb->err, 1);
        if (*(volatile int *)&gb->err) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Up to `ngroups` groups of 6 fused MinRes iterations over all slots; at every
// iteration count that is a multiple of `check` (a multiple of 6), slots whose inner
// residual met their tolerance are frozen (as the host does between graph replays, so
// both forms give the same bits), and the kernel ends once every slot is frozen.
template <int B>
__global__ void __launch_bounds__(B * kMT)
k_mm_persistent(float4 *__restrict__ U0, float4 *__restrict__ Up0, float4 *__restrict__ W0, float4 *__restrict__ D20,
                float4 *__restrict__ D30, float4 *__restrict__ E, const SlotDesc *__restrict__ sd,
                const int2 *__restrict__ table, int ntab, int NS, FusedState *__restrict__ st, int *__restrict__ active,
                double *__restrict__ partials, double *__restrict__ partials2, const double *__restrict__ tol,
                int it0, int check, int ngroups, GridBar *gb, long long limit) {
    float4 *U = U0, *Up = Up0, *W = W0, *D2 = D20, *D3 = D30;
    for (int grp = 0; grp < ngroups; ++grp) {
        for (int sub = 0; sub < 6; ++sub) {
            for (int item = blockIdx.x; item < ntab; item += gridDim.x) {
                const int2 t = table[item];
                const SlotDesc d = sd[t.x];
                if (!active[t.x]) {
                    if (threadIdx.x % kMT == 0 && t.y + (int)(threadIdx.x / kMT) < d.nb)
                        partials[d.blk0 + t.y + threadIdx.x / kMT] = 0.0;
                    continue;
                }
                const int s = t.y * kMT + threadIdx.x;
                float facc = 0.f;
                if (s < d.g.V)
                    facc = minres_k1_site(s, d.g, d.kappa, U + d.off, Up + d.off, W + d.off, D2 + d.off, D3 + d.off,
                                          E + d.off, d.links, st[t.x]);
                chunk_partials<B>(facc, partials + d.blk0 + t.y, d.nb - t.y);
            }
            if (!grid_wait(gb, limit)) return;
            for (int q = blockIdx.x; q < NS; q += gridDim.x) {
                if (!active[q]) continue;
                const SlotDesc d = sd[q];
                const double a = slot_sum(partials, d.blk0, d.nb);
                if (threadIdx.x == 0) fused_alpha(st[q], a);
                __syncthreads();
            }
            if (!grid_wait(gb, limit)) return;
            for (int item = blockIdx.x; item < ntab; item += gridDim.x) {
                const int2 t = table[item];
                const SlotDesc d = sd[t.x];
                if (!active[t.x]) {
                    if (threadIdx.x % kMT == 0 && t.y + (int)(threadIdx.x / kMT) < d.nb)
                        partials2[d.blk0 + t.y + threadIdx.x / kMT] = 0.0;
                    continue;
                }
                const int s = t.y * kMT + threadIdx.x;
                float facc = 0.f;
                if (s < d.g.V) facc = minres_k2a_site(s, d.g.V, W + d.off, U + d.off, st[t.x]);
                chunk_partials<B>(facc, partials2 + d.blk0 + t.y, d.nb - t.y);
            }
            if (!grid_wait(gb, limit)) return;
            for (int q = blockIdx.x; q < NS; q += gridDim.x) {
                if (!active[q]) continue;
                const SlotDesc d = sd[q];
                const double r2 = slot_sum(partials2, d.blk0, d.nb);
                if (threadIdx.x == 0) {
                    FusedState v = st[q];
                    fused_givens(v, r2);
                    st[q] = v;
                }
                __syncthreads();
            }
            if (!grid_wait(gb, limit)) return;
            float4 *tUp = Up;
            Up = U; U = W; W = tUp;
            float4 *tD = D2; D2 = D3; D3 = tD;
        }
        const int it = it0 + 6 * (grp + 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) gb->groups = grp + 1;
        if (it % check != 0) continue;
        // freeze converged slots (the owner block of each slot decides), then all blocks
        // read the same flags after the barrier
        for (int q = blockIdx.x; q < NS; q += gridDim.x)
            if (threadIdx.x == 0 && active[q]) {
                const FusedState v = st[q];
                if (fabs(v.phibar) <= tol[q] * v.r0 || v.beta_next == 0.0) active[q] = 0;
            }
        if (!grid_wait(gb, limit)) return;
        __shared__ int any;
        if (threadIdx.x == 0) {
            int a = 0;
            for (int q = 0; q < NS && !a; ++q) a = ((volatile int *)active)[q];
            any = a;
        }
        __syncthreads();
        if (!any) return;
    }
}

}  // namespace

// One block-table layout: blocks of B chunks (B * 128 sites) of one slot.
struct Tile {
    int B;
    const int2 *table;
    int nblocks;
};

// The fused FP32 MinRes over all slots (r: normalised residuals in the arena; e:
// corrections, holding the start if e_init).  bufs: 5 arena-sized work vectors.
// A slot whose inner residual has met its tolerance at a check is frozen: its blocks
// return at once and its state stops changing (the buffer roles repeat every 6
// iterations and checks fall on multiples of 6, so the frozen slot's pending
// direction update is still found where k_mm_last looks for it).
// Tiles: the first three 6-iteration groups capture a graph per tile (128, 256 and
// 512 threads per block), the next three time one replay each (CUDA events), and the
// fastest serves the rest (DLZ_MULTI_TILE=1|2|4 forces one).  The partials are per
// 128-site chunk whatever the tile, so every tile gives bit-identical results.
// persistent launch of up to `ngroups` 6-iteration groups with B chunks per work item and
// `grid` blocks; returns the groups run (device count) or a DLZ error
static int launch_persistent(Op &op, int B, int grid, float4 *U0, float4 *Up0, float4 *W0, float4 *D20, float4 *D30,
                             float4 *e, const SlotDesc *sd, const Tile &t, int NS, FusedState *ms, int *active,
                             double *partials, double *partials2, const double *d_tol, int it0, int check, int ngroups,
                             GridBar *gb, long long limit, int &groups_run) {
    DLZ_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), op.stream));
    int ntab = t.nblocks;
    const int2 *table = t.table;
    void *args[] = {&U0, &Up0, &W0, &D20, &D30, &e, (void *)&sd, (void *)&table, &ntab, &NS, &ms, &active,
                    &partials, &partials2, (void *)&d_tol, &it0, &check, &ngroups, &gb, &limit};
    void *fn = B == 1 ? (void *)k_mm_persistent<1> : B == 2 ? (void *)k_mm_persistent<2> : (void *)k_mm_persistent<4>;
    DLZ_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(B * kMT), args, 0, op.stream));
    op.prof.launches += 1;
    GridBar h;
    DLZ_TRY(d2h_sync(op, &h, gb, sizeof(GridBar)));
    if (h.err) return fail(DLZ_ERR_DEVICE_TIMEOUT, "a grid barrier of the persistent multi-lattice kernel gave up");
    groups_run = h.groups;
    return DLZ_OK;
}

// blocks of the persistent kernel: `frac` of the co-resident maximum on every SM
static int persistent_grid(int B, int frac_half) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const void *fn = B == 1 ? (const void *)k_mm_persistent<1> : B == 2 ? (const void *)k_mm_persistent<2>
                                                                       : (const void *)k_mm_persistent<4>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, B * kMT, 0) != cudaSuccess) return 0;
    if (frac_half) per = std::max(1, per / 2);
    return per * nsm;
}

int minres_multi_batch(Op &op, int NS, const SlotDesc *sd, const Tile *tiles, int nchunks, size_t arena,
                       const float4 *r, float4 *e, float4 *const bufs[5], FusedState *ms, double *partials,
                       int *active, const double *d_tol, const dlz_params &p, int &iters, bool e_init,
                       GridBar *gb) {
    double *partials2 = partials + nchunks;
    k_mm_norm<1><<<tiles[0].nblocks, kMT, 0, op.stream>>>(r, sd, tiles[0].table, partials);
    k_mm_init<<<NS, 256, 0, op.stream>>>(partials, sd, ms);
    op.prof.launches += 2;
    DLZ_CUDA_TRY(cudaGetLastError());
    float4 *U0 = bufs[0], *Up0 = bufs[1], *W0 = bufs[2], *D20 = bufs[3], *D30 = bufs[4];
    DLZ_CUDA_TRY(cudaMemcpyAsync(U0, r, arena * sizeof(float4), cudaMemcpyDeviceToDevice, op.stream));
    for (float4 *z : {Up0, D20, D30}) DLZ_CUDA_TRY(cudaMemsetAsync(z, 0, arena * sizeof(float4), op.stream));
    if (!e_init) DLZ_CUDA_TRY(cudaMemsetAsync(e, 0, arena * sizeof(float4), op.stream));
    auto iteration = [&](const Tile &t, float4 *U, float4 *Up, float4 *W, float4 *D2, float4 *D3) -> int {
        switch (t.B) {
        case 1: k_mm_k1<1><<<t.nblocks, kMT, 0, op.stream>>>(U, Up, W, D2, D3, e, sd, t.table, ms, active, partials); break;
        case 2: k_mm_k1<2><<<t.nblocks, 2 * kMT, 0, op.stream>>>(U, Up, W, D2, D3, e, sd, t.table, ms, active, partials); break;
        default: k_mm_k1<4><<<t.nblocks, 4 * kMT, 0, op.stream>>>(U, Up, W, D2, D3, e, sd, t.table, ms, active, partials);
        }
        k_mm_alpha<<<NS, 256, 0, op.stream>>>(partials, sd, ms, active);
        switch (t.B) {
        case 1: k_mm_k2a<1><<<t.nblocks, kMT, 0, op.stream>>>(W, U, sd, t.table, ms, active, partials2); break;
        case 2: k_mm_k2a<2><<<t.nblocks, 2 * kMT, 0, op.stream>>>(W, U, sd, t.table, ms, active, partials2); break;
        default: k_mm_k2a<4><<<t.nblocks, 4 * kMT, 0, op.stream>>>(W, U, sd, t.table, ms, active, partials2);
        }
        k_mm_k2b<<<NS, 256, 0, op.stream>>>(partials2, sd, ms, active);
        op.prof.launches += 4;
        DLZ_CUDA_TRY(cudaGetLastError());
        return DLZ_OK;
    };
    GraphExec ge[3];
    int cur = 0;
    auto six = [&]() -> int {
        float4 *U = U0, *Up = Up0, *W = W0, *D2 = D20, *D3 = D30;
        for (int sub = 0; sub < 6; ++sub) {
            DLZ_TRY(iteration(tiles[cur], U, Up, W, D2, D3));
            float4 *tUp = Up;
            Up = U; U = W; W = tUp;
            std::swap(D2, D3);
        }
        return DLZ_OK;
    };
    // Autotuner over the launch forms: the graph form with 1, 2 or 4 chunks of 128 sites
    // per block (candidates 0-2; the first three groups capture their graphs, the next
    // three time one replay each), and the persistent form with 1, 2 or 4 chunks per
    // work item at the full or half co-resident grid (candidates 3-8, one timed group
    // each).  The fastest candidate runs the rest.  Chunk partials and slot freezing do
    // not depend on the candidate, so every choice gives the same bits.
    // DLZ_MULTI_TILE=1|2|4 fixes the chunks per block; DLZ_MULTI_FORM=graph|persistent
    // fixes the form (both: no search).
    int tile_forced = -1, form_forced = -1;
    if (const char *env = std::getenv("DLZ_MULTI_TILE")) {
        const int b = std::atoi(env);
        tile_forced = b == 1 ? 0 : b == 2 ? 1 : b == 4 ? 2 : -1;
    }
    if (const char *env = std::getenv("DLZ_MULTI_FORM")) {
        if (std::strcmp(env, "graph") == 0) form_forced = 0;
        else if (std::strcmp(env, "persistent") == 0) form_forced = 1;
    }
    long long limit = 1LL << 24;           // polls of a barrier wait (64 ns apart): about a second
    if (const char *env = std::getenv("DLZ_WAIT_LIMIT")) limit = std::atoll(env);
    const int check = std::max(6, (p.check_every / 6) * 6);
    struct Cand { int form, tile, half, grid; };
    std::vector<Cand> cands;
    for (int v = 0; v < 3; ++v)
        if ((tile_forced < 0 || tile_forced == v) && form_forced != 1) cands.push_back({0, v, 0, 0});
    for (int v = 0; v < 3; ++v)
        for (int half = 0; half < 2; ++half)
            if ((tile_forced < 0 || tile_forced == v) && form_forced != 0) {
                const int grid = persistent_grid(1 << v, half);
                if (grid > 0) cands.push_back({1, v, half, grid});
            }
    if (cands.empty()) return fail(DLZ_ERR_CUDA, "no launch form available for the multi-lattice kernel");
    std::vector<float> tms(cands.size(), 0.f);
    Event ev0, ev1;
    DLZ_CUDA_TRY(ev0.create());
    DLZ_CUDA_TRY(ev1.create());
    std::vector<FusedState> h(NS);
    std::vector<double> tol(NS);
    DLZ_TRY(d2h_sync(op, tol.data(), d_tol, NS * sizeof(double)));
    std::vector<int> act(NS, 1);
    DLZ_TRY(h2d(op, active, act.data(), NS * sizeof(int)));
    // the schedule: capture (graph candidates), then one timed group per candidate, then the best
    std::vector<int> sched;
    for (size_t c = 0; c < cands.size(); ++c)
        if (cands[c].form == 0 && cands.size() > 1) sched.push_back((int)c);      // capture groups (untimed)
    const size_t ncapture = sched.size();
    if (cands.size() > 1)
        for (size_t c = 0; c < cands.size(); ++c) sched.push_back((int)c);        // timed groups
    int it = 0, group = 0, best = 0;
    bool all_done = false;
    auto host_check = [&]() -> int {
        DLZ_TRY(d2h_sync(op, h.data(), ms, NS * sizeof(FusedState)));
        bool done = true, changed = false;
        for (int q = 0; q < NS; ++q) {
            if (!std::isfinite(h[q].phibar)) return fail(DLZ_ERR_NONFINITE, "MinRes residual not finite");
            const bool ok = std::fabs(h[q].phibar) <= tol[q] * h[q].r0 || h[q].beta_next == 0.0;
            if (!ok) done = false;
            else if (act[q]) { act[q] = 0; changed = true; }
        }
        all_done = done;
        if (!done && changed) DLZ_TRY(h2d(op, active, act.data(), NS * sizeof(int)));
        return DLZ_OK;
    };
    while (iters < p.max_iter && !all_done) {
        const bool tuning = (size_t)group < sched.size();
        const int ci = tuning ? sched[group] : best;
        const Cand &c = cands[ci];
        const bool timed = tuning && (size_t)group >= ncapture;
        if (c.form == 0) {
            cur = c.tile;
            if (timed) DLZ_CUDA_TRY(cudaEventRecord(ev0.e, op.stream));
            DLZ_TRY(run_graph(op, ge[cur], six));
            if (timed) DLZ_CUDA_TRY(cudaEventRecord(ev1.e, op.stream));
            iters += 6;
            it += 6;
            if (it % check == 0 || iters >= p.max_iter) DLZ_TRY(host_check());
        } else {
            // one group while tuning, else every remaining group in one launch
            const int ngroups = tuning ? 1 : std::max(1, (p.max_iter - iters + 5) / 6);
            int ran = 0;
            if (timed) DLZ_CUDA_TRY(cudaEventRecord(ev0.e, op.stream));
            DLZ_TRY(launch_persistent(op, 1 << c.tile, c.grid, U0, Up0, W0, D20, D30, e, sd, tiles[c.tile], NS, ms,
                                      active, partials, partials2, d_tol, it, check, ngroups, gb, limit, ran));
            if (timed) DLZ_CUDA_TRY(cudaEventRecord(ev1.e, op.stream));
            iters += 6 * ran;
            it += 6 * ran;
            // the kernel froze slots itself: bring the flags back, and see whether all are done
            DLZ_TRY(d2h_sync(op, act.data(), active, NS * sizeof(int)));
            bool any = false;
            for (int q = 0; q < NS; ++q) any = any || act[q];
            all_done = !any;
            if (!all_done && (it % check == 0 || iters >= p.max_iter)) DLZ_TRY(host_check());
        }
        if (timed) {
            DLZ_CUDA_TRY(cudaEventSynchronize(ev1.e));
            if (cudaEventElapsedTime(&tms[ci], ev0.e, ev1.e) != cudaSuccess) {
                cudaGetLastError();
                tms[ci] = 1e30f;
            }
            if ((size_t)group + 1 == sched.size())
                for (size_t v = 0; v < cands.size(); ++v)
                    if (tms[v] < tms[best]) best = (int)v;
        }
        ++group;
    }
    op.multi_choice = cands[best].form * 100 + (1 << cands[best].tile) * 10 + cands[best].half;
    k_mm_last<1><<<tiles[0].nblocks, kMT, 0, op.stream>>>(Up0, D20, D30, e, sd, tiles[0].table, ms);
    op.prof.launches += 1;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

// FP32 D-MinRes with FP64 defect correction on every lattice's right-hand sides
// at once.  B[l], X[l]: nrhs[l] internal FP64 vectors of lattice l.
int dminres_multi(int nlat, Op *const *ops, const dlz_defl_s *const *defls, const double2 *const *B,
                  double2 *const *X, const int *nrhs, const dlz_params &p, dlz_stats *st) {
    // slots (their 128-site chunks contiguous in the partials) and the block tables of
    // the three tiles (1, 2 or 4 chunks per block)
    std::vector<SlotDesc> hsd;
    std::vector<int2> tab[3];
    std::vector<int> slot_lat, slot_rhs, lat_slot0(nlat);
    size_t arena = 0;
    int nchunks = 0;
    for (int l = 0; l < nlat; ++l) {
        lat_slot0[l] = (int)hsd.size();
        const Op &o = *ops[l];
        for (int r = 0; r < nrhs[l]; ++r) {
            SlotDesc d;
            d.g = o.g;
            d.kappa = (float)o.kappa;
            d.links = o.gauge32.as<float4>();
            d.off = arena;
            d.blk0 = nchunks;
            d.nb = (o.g.V + kMT - 1) / kMT;
            for (int v = 0; v < 3; ++v)
                for (int c0 = 0; c0 < d.nb; c0 += (1 << v)) tab[v].push_back(make_int2((int)hsd.size(), c0));
            nchunks += d.nb;
            arena += 6L * o.g.V;
            hsd.push_back(d);
            slot_lat.push_back(l);
            slot_rhs.push_back(r);
        }
    }
    const int NS = (int)hsd.size();
    if (NS == 0) return DLZ_OK;
    Op &op = *ops[0];
    DevBuf dsd, dtab[3], f32, part, scal, gbar;
    DLZ_TRY(gbar.alloc(sizeof(GridBar)));
    DLZ_TRY(dsd.alloc(NS * sizeof(SlotDesc)));
    Tile tiles[3];
    for (int v = 0; v < 3; ++v) {
        DLZ_TRY(dtab[v].alloc(tab[v].size() * sizeof(int2)));
        DLZ_TRY(h2d(op, dtab[v].p, tab[v].data(), tab[v].size() * sizeof(int2)));
        tiles[v] = Tile{1 << v, dtab[v].as<int2>(), (int)tab[v].size()};
    }
    DLZ_TRY(f32.alloc(7 * arena * sizeof(float4)));
    DLZ_TRY(part.alloc(2 * (size_t)nchunks * sizeof(double)));
    DLZ_TRY(scal.alloc((size_t)NS * (sizeof(FusedState) + 2 * sizeof(double) + sizeof(int))));
    DLZ_TRY(h2d(op, dsd.p, hsd.data(), NS * sizeof(SlotDesc)));
    float4 *r32 = f32.as<float4>(), *e32 = r32 + arena;
    float4 *const bufs[5] = {r32 + 2 * arena, r32 + 3 * arena, r32 + 4 * arena, r32 + 5 * arena, r32 + 6 * arena};
    FusedState *ms = reinterpret_cast<FusedState *>(scal.p);
    double *d_tol = reinterpret_cast<double *>(ms + NS);
    int *d_active = reinterpret_cast<int *>(d_tol + 2 * NS);
    // per-lattice FP64 work: b' = gamma5 b, x, r, Q x
    struct Lat {
        DevBuf bp, x, r, t, dots, nrm;
        std::vector<double> bn, rn;
    };
    std::vector<Lat> L(nlat);
    for (int l = 0; l < nlat; ++l) {
        Op &o = *ops[l];
        const long n64 = 12L * o.g.V;
        const int N = nrhs[l];
        if (N > 16) return fail(DLZ_ERR_BADARG, "at most 16 right-hand sides per lattice");
        Lat &a = L[l];
        DLZ_TRY(a.bp.alloc((size_t)N * n64 * sizeof(double2)));
        DLZ_TRY(a.x.alloc((size_t)N * n64 * sizeof(double2)));
        DLZ_TRY(a.r.alloc((size_t)N * n64 * sizeof(double2)));
        DLZ_TRY(a.t.alloc((size_t)N * n64 * sizeof(double2)));
        DLZ_TRY(a.nrm.alloc(16 * sizeof(double)));
        if (defls[l] && defls[l]->k > 0) {
            DLZ_TRY(a.dots.alloc((size_t)N * defls[l]->k * sizeof(double2)));
            DLZ_TRY(reserve_multidot(o, defls[l]->k));
            DLZ_TRY(deflation_v32(o, const_cast<dlz_defl_s *>(defls[l])));
        }
        const long half = 6L * o.g.V;
        double2 *pbp = a.bp.as<double2>();
        const double2 *pb = B[l];
        DLZ_TRY(map(o, n64 * N, [=] __device__(long i) {
            double2 v = pb[i];
            if ((i % n64) >= half) { v.x = -v.x; v.y = -v.y; }
            pbp[i] = v;
        }));
        double *dn = a.nrm.as<double>();
        DLZ_TRY(reduce<16>(o, n64, [=] __device__(long i, double (&acc)[16]) {
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (q < N) { const double2 v = pbp[(size_t)q * n64 + i]; acc[q] += v.x * v.x + v.y * v.y; }
        }, [=] __device__(const double *res) { for (int q = 0; q < N; ++q) dn[q] = sqrt(res[q]); }));
        a.bn.resize(N);
        a.rn.resize(N);
        DLZ_TRY(d2h_sync(o, a.bn.data(), dn, N * sizeof(double)));
        DLZ_CUDA_TRY(cudaMemsetAsync(a.x.p, 0, (size_t)N * n64 * sizeof(double2), o.stream));
    }
    for (int q = 0; q < NS; ++q) std::memset(&st[q], 0, sizeof(dlz_stats));
    std::vector<char> done(NS, 0);
    std::vector<double> inv(NS), tl(NS);
    int iters = 0, outer = 0;
    while (true) {
        // FP64 residuals lattice by lattice
        bool all = true;
        for (int l = 0; l < nlat; ++l) {
            Op &o = *ops[l];
            Lat &a = L[l];
            const int N = nrhs[l];
            const long n64 = 12L * o.g.V;
            DLZ_TRY(wilson64_batch(o, a.t.as<double2>(), a.x.as<double2>(), DLZ_Q, N));
            const double2 *pbp = a.bp.as<double2>(), *pt = a.t.as<double2>();
            double2 *pr = a.r.as<double2>();
            double *dn = a.nrm.as<double>();
            DLZ_TRY(reduce<16>(o, n64, [=] __device__(long i, double (&acc)[16]) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (q < N) {
                        const size_t k = (size_t)q * n64 + i;
                        const double2 u = pbp[k], v = pt[k];
                        const double2 t = make_double2(u.x - v.x, u.y - v.y);
                        pr[k] = t;
                        acc[q] += t.x * t.x + t.y * t.y;
                    }
                }
            }, [=] __device__(const double *res) { for (int q = 0; q < N; ++q) dn[q] = sqrt(res[q]); }));
            DLZ_TRY(d2h_sync(o, a.rn.data(), dn, N * sizeof(double)));
            for (int r = 0; r < N; ++r) {
                const int q = lat_slot0[l] + r;
                if (!std::isfinite(a.rn[r])) return fail(DLZ_ERR_NONFINITE, "residual is not finite");
                if (!done[q] && (a.bn[r] == 0.0 || a.rn[r] <= p.tol * a.bn[r])) {
                    done[q] = 1;
                    st[q].iterations = iters;
                    st[q].cycles = outer;
                }
                all = all && done[q];
                const bool open = !done[q];
                inv[q] = open ? 1.0 / a.rn[r] : 0.0;
                tl[q] = open ? std::max(0.5 * p.tol * a.bn[r] / a.rn[r], p.reliable_delta) : 1.0;
            }
        }
        if (all || iters >= p.max_iter) break;
        // normalised FP32 residuals into the arena; Galerkin projection per lattice
        for (int l = 0; l < nlat; ++l) {
            Op &o = *ops[l];
            Lat &a = L[l];
            const int N = nrhs[l];
            const int V = o.g.V;
            const long n64 = 12L * V, n32 = 6L * V;
            float4 *rl = r32 + hsd[lat_slot0[l]].off, *el = e32 + hsd[lat_slot0[l]].off;
            const double2 *pr = a.r.as<double2>();
            Scales16 scv;
            for (int r = 0; r < N; ++r) scv.v[r] = inv[lat_slot0[l] + r];
            DLZ_TRY(map(o, n32 * N, [=] __device__(long i) {
                const int q = (int)(i / n32);
                const long j = i % n32;
                const int c = (int)(j / V), s = (int)(j % V);
                const double f = scv.v[q];
                const double2 *src = pr + (size_t)q * n64;
                const double2 u = src[(size_t)(2 * c) * V + s], w = src[(size_t)(2 * c + 1) * V + s];
                rl[i] = make_float4((float)(f * u.x), (float)(f * u.y), (float)(f * w.x), (float)(f * w.y));
            }));
            const dlz_defl_s *d = defls[l];
            if (d && d->k > 0) {
                const int k = d->k;
                const float4 *V32 = d->V32.as<float4>();
                double2 *pd = a.dots.as<double2>();
                for (int r = 0; r < N; ++r)
                    DLZ_TRY(multidot<P32>(o, V32, n32, k, rl + (size_t)r * n32, pd + (size_t)r * k, 1.0));
                std::vector<double2> hc((size_t)N * k);
                DLZ_TRY(d2h_sync(o, hc.data(), pd, hc.size() * sizeof(double2)));
                std::vector<std::complex<double>> z(k);
                for (int r = 0; r < N; ++r) {
                    for (int i = 0; i < k; ++i) z[i] = std::complex<double>(hc[(size_t)r * k + i].x, hc[(size_t)r * k + i].y);
                    lu_solve(k, d->Hlu.data(), d->piv.data(), z.data());
                    for (int i = 0; i < k; ++i) hc[(size_t)r * k + i] = make_double2(z[i].real(), z[i].imag());
                }
                DLZ_TRY(h2d(o, pd, hc.data(), hc.size() * sizeof(double2)));
                for (int r = 0; r < N; ++r)
                    DLZ_TRY(combine<P32>(o, el + (size_t)r * n32, n32, 1, V32, n32, k, pd + (size_t)r * k, 1, false, false));
                float4 *qe = bufs[0] + hsd[lat_slot0[l]].off;      // scratch: Q e0
                DLZ_TRY(wilson32_batch(o, qe, el, DLZ_Q, N));
                DLZ_TRY(map(o, n32 * N, [=] __device__(long i) {
                    const float4 u = rl[i], w = qe[i];
                    rl[i] = make_float4(u.x - w.x, u.y - w.y, u.z - w.z, u.w - w.w);
                }));
            } else {
                DLZ_CUDA_TRY(cudaMemsetAsync(el, 0, (size_t)N * n32 * sizeof(float4), o.stream));
            }
            DLZ_CUDA_TRY(cudaStreamSynchronize(o.stream));
        }
        DLZ_TRY(h2d(op, d_tol, tl.data(), NS * sizeof(double)));
        DLZ_TRY(minres_multi_batch(op, NS, dsd.as<SlotDesc>(), tiles, nchunks, arena, r32, e32, bufs, ms,
                                   part.as<double>(), d_active, d_tol, p, iters, true, gbar.as<GridBar>()));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        // x += ||r|| e, lattice by lattice
        for (int l = 0; l < nlat; ++l) {
            Op &o = *ops[l];
            Lat &a = L[l];
            const int N = nrhs[l];
            const int V = o.g.V;
            const long n64 = 12L * V, n32 = 6L * V;
            const float4 *el = e32 + hsd[lat_slot0[l]].off;
            Scales16 scv;
            for (int r = 0; r < N; ++r) {
                const double iv = inv[lat_slot0[l] + r];
                scv.v[r] = iv > 0.0 ? 1.0 / iv : 0.0;
            }
            double2 *px = a.x.as<double2>();
            DLZ_TRY(map(o, n32 * N, [=] __device__(long i) {
                const int q = (int)(i / n32);
                const double f = scv.v[q];
                const long j = i % n32;
                const int c = (int)(j / V), s = (int)(j % V);
                const float4 qv = el[i];
                double2 *xq = px + (size_t)q * n64;
                double2 &u = xq[(size_t)(2 * c) * V + s];
                double2 &w = xq[(size_t)(2 * c + 1) * V + s];
                u.x += f * qv.x; u.y += f * qv.y; w.x += f * qv.z; w.y += f * qv.w;
            }));
        }
        ++outer;
    }
    int rc = DLZ_OK;
    for (int l = 0; l < nlat; ++l) {
        Op &o = *ops[l];
        const long n64 = 12L * o.g.V;
        DLZ_CUDA_TRY(cudaMemcpyAsync(X[l], L[l].x.p, (size_t)nrhs[l] * n64 * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     o.stream));
        DLZ_CUDA_TRY(cudaStreamSynchronize(o.stream));
        for (int r = 0; r < nrhs[l]; ++r) {
            const int q = lat_slot0[l] + r;
            st[q].true_residual = L[l].bn[r] > 0 ? L[l].rn[r] / L[l].bn[r] : 0.0;
            st[q].converged = done[q] ? 1 : 0;
            if (!done[q]) { st[q].iterations = iters; st[q].cycles = outer; rc = DLZ_ERR_NOT_CONVERGED; }
            st[q].mvps = iters + outer;
        }
    }
    return rc;
}

}  // namespace dlz
