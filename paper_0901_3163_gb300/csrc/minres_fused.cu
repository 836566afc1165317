// Fused FP32 MinRes iteration for a batch of right-hand sides (the inner
// solve of the mixed-precision D-MinRes, arXiv:0901.3163 Sec. 2).
//
// Two full passes over the vectors per iteration:
//   K1 (stencil + epilogue, one block = 128 sites of one right-hand side):
//        v_j   = u_j / beta_j                      (u_j: unnormalised Lanczos vector; the
//                                                   v's are never stored, only the u's)
//        w     = Q v_j - beta_j v_{j-1}            (Q u_j / beta_j: Q is linear)
//        alpha_j partial = Re <v_j, w>
//        d_{j-1} = (v_{j-1} - delta d_{j-2} - eps d_{j-3}) / gamma,  e += tau d_{j-1}
//        (the direction update of the previous step: its Givens rotation needed
//         beta_j, known only now)
//   K2a: u_{j+1} = w - alpha_j v_j and the block partials of ||u_{j+1}||^2;
//   K1b: alpha_j = sum of K1's block partials (one block per right-hand side);
//   K2b: beta_{j+1}, and the Givens rotation of step j (one block per right-hand side);
// for a single right-hand side K1b and K2b are folded into the last block of K1 and
// K2a to finish.  The partials (block b belongs to right-hand side b mod N) are summed
// in a fixed order, so results are deterministic.  Buffers rotate with periods 3 and 2, so a group of 6 iterations is
// captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "solvers.h"
#include "minres_state.cuh"
#include "wilson_site.cuh"

namespace dlz {



namespace {

constexpr int kThreads = 128;


__global__ void __launch_bounds__(kThreads)
k_minres_k1(const float4 *__restrict__ Ub, const float4 *__restrict__ Up, float4 *__restrict__ W,
            const float4 *__restrict__ D2, float4 *__restrict__ D3, float4 *__restrict__ E,
            const float4 *__restrict__ links, Geom g, float kappa, int N,
            FusedState *__restrict__ st, double *__restrict__ partials, unsigned *__restrict__ counters) {
    const int q = blockIdx.x % N;
    const int s = (blockIdx.x / N) * blockDim.x + threadIdx.x;
    const long nel = 6L * g.V;
    const size_t base = (size_t)q * nel;
    float facc = 0.f;
    if (s < g.V) {
        facc = minres_k1_site(s, g, kappa, Ub + base, Up + base, W + base, D2 + base, D3 + base, E + base,
                              links, st[q]);
    }
    // block partials of alpha_q; with counters, the last block of q to finish forms
    // alpha_q (one right-hand side: saves a launch); without, k_minres_alpha does
    const int nbq = gridDim.x / N;
    if (!counters) {
        block_partial_store<kThreads>(facc, partials + (size_t)q * nbq + blockIdx.x / N);
        return;
    }
    double a;
    if (partial_then_last_sum<kThreads>(facc, partials + (size_t)q * nbq, blockIdx.x / N, nbq, counters + q, &a) &&
        threadIdx.x == 0)
        fused_alpha(st[q], a);
}

__global__ void __launch_bounds__(kThreads)
k_minres_k2a(float4 *__restrict__ W, const float4 *__restrict__ Vc, Geom g, int N,
             FusedState *__restrict__ st, double *__restrict__ partials, unsigned *__restrict__ counters) {
    // Vc: the unnormalised u_j; alpha_j v_j = (alpha_j / beta_j) u_j
    const int q = blockIdx.x % N;
    const int s = (blockIdx.x / N) * blockDim.x + threadIdx.x;
    const size_t base = (size_t)q * 6 * g.V;
    float facc = 0.f;
    if (s < g.V) {
        facc = minres_k2a_site(s, g.V, W + base, Vc + base, st[q]);
    }
    // the last block of q to finish: beta_{j+1} and the Givens rotation of step j
    // (with counters; without, k_minres_k2b does it)
    const int nbq = gridDim.x / N;
    if (!counters) {
        block_partial_store<kThreads>(facc, partials + (size_t)q * nbq + blockIdx.x / N);
        return;
    }
    double r2;
    if (partial_then_last_sum<kThreads>(facc, partials + (size_t)q * nbq, blockIdx.x / N, nbq, counters + q, &r2) &&
        threadIdx.x == 0) {
        FusedState t = st[q];
        fused_givens(t, r2);
        st[q] = t;
    }
}

// alpha_q = sum of the block partials of right-hand side q (block q of the grid),
// in a fixed order
__global__ void __launch_bounds__(256)
k_minres_alpha(const double *__restrict__ partials, int nbq, FusedState *__restrict__ st) {
    const int q = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nbq; b += blockDim.x) t += partials[(size_t)q * nbq + b];
    __shared__ double sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) a += sm[w];
        fused_alpha(st[q], a);
    }
}

// K2b: beta_{j+1} = sqrt(sum of K2a's partials) and the Givens rotation of step j,
// one block per right-hand side
__global__ void __launch_bounds__(256)
k_minres_k2b(const double *__restrict__ partials, int nbq, FusedState *__restrict__ st) {
    const int q = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nbq; b += blockDim.x) t += partials[(size_t)q * nbq + b];
    __shared__ double sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) r2 += sm[w];
        FusedState s = st[q];
        fused_givens(s, r2);
        st[q] = s;
    }
}


}  // namespace

int minres_fused_batch(Op &op, int N, const float4 *r, float4 *e, float4 *const bufs[6],
                       FusedState *ms, double *partials, const double *d_tol,
                       const dlz_params &p, int &iters, HostScratch &hs, bool e_init) {
    const long n = 6L * op.g.V;
    // beta_1 = ||r_q||, rotations reset, a no-op direction update for step 0
    DLZ_TRY(reduce32<16>(op, n, [=] __device__(long i, float (&acc)[16]) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q < N) { const float4 v = r[(size_t)q * n + i]; acc[q] += (v.x * v.x + v.y * v.y) + (v.z * v.z + v.w * v.w); }
    }, [=] __device__(const double *res) {
        for (int q = 0; q < N; ++q) {
            fused_init(ms[q], sqrt(res[q]));
        }
    }));
    // u_j, u_{j-1} (unnormalised Lanczos vectors), w, d_{j-2}, d_{j-3}
    float4 *U0 = bufs[0], *Up0 = bufs[1], *W0 = bufs[2], *D20 = bufs[3], *D30 = bufs[4];
    DLZ_CUDA_TRY(cudaMemcpyAsync(U0, r, (size_t)N * n * sizeof(float4), cudaMemcpyDeviceToDevice, op.stream));
    for (float4 *z : {Up0, D20, D30})
        DLZ_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)N * n * sizeof(float4), op.stream));
    if (!e_init) DLZ_CUDA_TRY(cudaMemsetAsync(e, 0, (size_t)N * n * sizeof(float4), op.stream));
    const Geom g = op.g;
    const float kappa = (float)op.kappa;
    const float4 *links = op.gauge32.as<float4>();
    const unsigned blocks = (unsigned)(((g.V + kThreads - 1) / kThreads) * N);
    double *partials2 = partials + blocks;    // K2a's partials after K1's
    DevBuf cnt;                               // per-RHS block counters (reset by their last block)
    DLZ_TRY(cnt.alloc((size_t)N * sizeof(unsigned)));
    DLZ_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, (size_t)N * sizeof(unsigned), op.stream));
    unsigned *counters = cnt.as<unsigned>();
    auto iteration = [&](float4 *U, float4 *Up, float4 *W, float4 *D2, float4 *D3) -> int {
        // K1 moves 192 reals per site and right-hand side: u_j, u_{j-1}, d_{j-2}, d_{j-3}, e
        // read; w, d_{j-1}, e written (24 each), plus the links once per site
        op.prof.stencil_start(op.stream, true, g.V, N, 192, 1);
        // one right-hand side: the sums are taken by the kernels' last blocks (latency);
        // several: by one-block-per-RHS kernels (cheaper than a tail in every block)
        unsigned *cn = N == 1 ? counters : nullptr;
        k_minres_k1<<<blocks, kThreads, 0, op.stream>>>(U, Up, W, D2, D3, e, links, g, kappa, N, ms, partials, cn);
        op.prof.stencil_stop(op.stream);
        if (!cn) k_minres_alpha<<<N, 256, 0, op.stream>>>(partials, (int)(blocks / N), ms);
        op.prof.launches += cn ? 1 : 2;
        DLZ_CUDA_TRY(cudaGetLastError());
        // u_{j+1} = w - alpha v_j ; beta_{j+1} ; Givens rotation of step j
        k_minres_k2a<<<blocks, kThreads, 0, op.stream>>>(W, U, g, N, ms, partials2, cn);
        if (!cn) k_minres_k2b<<<N, 256, 0, op.stream>>>(partials2, (int)(blocks / N), ms);
        op.prof.launches += cn ? 1 : 2;
        DLZ_CUDA_TRY(cudaGetLastError());
        return DLZ_OK;
    };
    GraphExec ge;
    auto six = [&]() -> int {
        float4 *U = U0, *Up = Up0, *W = W0, *D2 = D20, *D3 = D30;
        for (int sub = 0; sub < 6; ++sub) {
            DLZ_TRY(iteration(U, Up, W, D2, D3));
            float4 *tUp = Up;
            Up = U; U = W; W = tUp;               // (U, Up, W) -> (W, U, Up): period 3
            std::swap(D2, D3);                     // period 2
        }
        return DLZ_OK;
    };
    const int check = std::max(6, (p.check_every / 6) * 6);
    int it = 0;
    // DLZ_TRACE=1: time the replays of the 6-iteration group (diagnostics)
    const char *trace_env = std::getenv("DLZ_TRACE");
    const bool trace = trace_env && trace_env[0] == '1';
    Event te0, te1;
    double t_graph = 0.0;
    int n_timed = 0;
    if (trace) {
        DLZ_CUDA_TRY(te0.create());
        DLZ_CUDA_TRY(te1.create());
    }
    while (iters < p.max_iter) {
        const bool timed = trace && ge.exec;      // not the replay that captures the graph
        if (timed) DLZ_CUDA_TRY(cudaEventRecord(te0.e, op.stream));
        DLZ_TRY(run_graph(op, ge, six));
        if (timed) {
            DLZ_CUDA_TRY(cudaEventRecord(te1.e, op.stream));
            DLZ_CUDA_TRY(cudaEventSynchronize(te1.e));
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, te0.e, te1.e) == cudaSuccess) { t_graph += ms; ++n_timed; }
            else cudaGetLastError();
        }
        iters += 6;
        it += 6;
        if (it % check == 0 || iters >= p.max_iter) {
            DLZ_TRY(d2h_sync(op, hs.p, ms, N * sizeof(FusedState)));
            ge.sample(op.prof);
            const FusedState *h = reinterpret_cast<const FusedState *>(hs.p);
            bool done = true;
            for (int q = 0; q < N; ++q)
                if (!std::isfinite(h[q].phibar)) return fail(DLZ_ERR_NONFINITE, "MinRes residual not finite");
            DLZ_TRY(d2h_sync(op, hs.p + 512, d_tol, N * sizeof(double)));
            for (int q = 0; q < N; ++q) {
                const FusedState *hq = reinterpret_cast<const FusedState *>(hs.p) + q;
                if (!(std::fabs(hq->phibar) <= hs.p[512 + q] * hq->r0 || hq->beta_next == 0.0)) done = false;
            }
            if (done) break;
        }
    }
    if (trace) {
        std::fprintf(stderr, "[dlz] fused MinRes N=%d: %d iterations, graph replay %.4f ms per iteration (%d timed)\n",
                     N, iters, n_timed ? t_graph / (6.0 * n_timed) : 0.0, n_timed);
    }
    // the direction update of the last step (after 6k steps the buffers are back
    // in their starting roles: u_J in Up, d_{J-1} in D2, d_{J-2} in D3; v_J = u_J / beta_J)
    {
        const float4 *vj = Up0, *d2 = D20, *d3 = D30;
        float4 *ee = e;
        DLZ_TRY(map(op, n * N, [=] __device__(long i) {
            const int q = (int)(i / n);
            minres_last_direction(vj[i], d2[i], d3[i], ee[i], ms[q]);
        }));
    }
    return DLZ_OK;
}

}  // namespace dlz
