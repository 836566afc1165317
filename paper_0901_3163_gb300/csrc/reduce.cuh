// Deterministic fused vector kernels: element-wise bodies with up to kMaxDots
// double accumulators, reduced in a fixed order (the inner products and norms of
// the Lanczos, CG and MinRes recurrences, Sec. 1-2).
//
// Every reduction runs on a fixed grid of kRedBlocks blocks with a
// grid-stride loop, so each element always lands in the same thread and
// block; each block writes its partial sums, and the last block to finish
// (completion counter) adds the partials in block order and runs a small
// `finish` functor on the results (e.g. alpha_j, beta_j, a Givens rotation).
// The result is bit-identical from run to run, and nothing leaves the GPU:
// later kernels read the scalars from device memory.
#pragma once

#include "dlz_internal.cuh"

namespace dlz {

template <int ND>
__device__ inline void block_sum(double (&acc)[ND], double (*sm)[kRedThreads / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        double v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kRedThreads / 32; ++w) v += sm[threadIdx.x][w];
        sm[threadIdx.x][0] = v;
    }
    __syncthreads();
}

// body(i, acc): element update and contributions for element i.
// fin(res): run once by one thread with the ND reduced values.
// A: the per-thread accumulator type.  FP32 vectors accumulate their few
// elements per thread in float (GB300's FP64 pipe runs at 1/64 of the FP32
// rate, so a double add per element would bound the kernel); every sum
// across threads and blocks is FP64.
template <int ND, typename A, class Body, class Fin>
__global__ void __launch_bounds__(kRedThreads) k_reduce(Body body, Fin fin, long n, RedScratch red) {
    __shared__ double sm[ND > 0 ? ND : 1][kRedThreads / 32];
    __shared__ bool last;
    double acc[ND > 0 ? ND : 1];
    {
        A local[ND > 0 ? ND : 1];
#pragma unroll
        for (int j = 0; j < ND; ++j) local[j] = A(0);
        const long stride = (long)gridDim.x * blockDim.x;
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) body(i, local);
#pragma unroll
        for (int j = 0; j < ND; ++j) acc[j] = (double)local[j];
    }
    block_sum<ND>(acc, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < ND; ++j) red.partials[j * kRedBlocks + blockIdx.x] = sm[j][0];
        __threadfence();
        last = (atomicAdd(red.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < ND; ++j) acc[j] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < ND; ++j) acc[j] += __ldcg(&red.partials[j * kRedBlocks + b]);
    }
    __syncthreads();
    block_sum<ND>(acc, sm);
    if (threadIdx.x == 0) {
        double res[ND > 0 ? ND : 1];
#pragma unroll
        for (int j = 0; j < ND; ++j) {
            res[j] = sm[j][0];
            red.result[j] = res[j];
        }
        fin(res);
        *red.counter = 0u;
    }
}

template <int ND, class Body, class Fin>
inline int reduce(Op &op, long n, Body body, Fin fin) {
    static_assert(ND <= kMaxDots, "too many accumulators");
    k_reduce<ND, double><<<kRedBlocks, kRedThreads, 0, op.stream>>>(body, fin, n, op.red);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
// Same, with float per-thread accumulators (body gets float (&)[ND]).
template <int ND, class Body, class Fin>
inline int reduce32(Op &op, long n, Body body, Fin fin) {
    static_assert(ND <= kMaxDots, "too many accumulators");
    k_reduce<ND, float><<<kRedBlocks, kRedThreads, 0, op.stream>>>(body, fin, n, op.red);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

template <class Body>
__global__ void __launch_bounds__(256) k_map(Body body, long n) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) body(i);
}

template <class Body>
inline int map(Op &op, long n, Body body) {
    long blocks = (n + 255) / 256;
    if (blocks > 4L * 152 * 8) blocks = 4L * 152 * 8;
    if (blocks < 1) blocks = 1;
    k_map<<<(int)blocks, 256, 0, op.stream>>>(body, n);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

struct NoFin {
    __device__ void operator()(const double *) const {}
};

// ------------------------------------------------------------------ combine
// out_l = (acc ? out_l : 0) + sum_j C[j][l] in_j for l < nout (nout <= 16),
// with vectors of n double2 elements at in + j*ld_in and out + l*ld_out.
// REAL: C real (double [nin][nout]); else complex (double2 [nin][nout]).
// The coefficient block sits in shared memory; each thread keeps its nout
// accumulators in registers and streams the nin input vectors once.
template <bool REAL, int NOUT>
__global__ void __launch_bounds__(128)
k_combine64(double2 *__restrict__ out, long ld_out, int nout, const double2 *__restrict__ in,
            long ld_in, int nin, const void *__restrict__ coef, int ld_coef, int col0, bool acc_out,
            long n) {
    extern __shared__ double2 csm[];   // [nin][NOUT]
    for (int t = threadIdx.x; t < nin * NOUT; t += blockDim.x) {
        const int j = t / NOUT, l = t % NOUT;
        double2 c = make_double2(0.0, 0.0);
        if (l < nout) {
            if (REAL) c.x = ((const double *)coef)[(size_t)j * ld_coef + col0 + l];
            else c = ((const double2 *)coef)[(size_t)j * ld_coef + col0 + l];
        }
        csm[t] = c;
    }
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double2 a[NOUT];
#pragma unroll
        for (int l = 0; l < NOUT; ++l) a[l] = make_double2(0.0, 0.0);
        for (int j = 0; j < nin; ++j) {
            const double2 v = in[(size_t)j * ld_in + i];
            const double2 *c = csm + j * NOUT;
#pragma unroll
            for (int l = 0; l < NOUT; ++l) {
                if (REAL) {
                    a[l].x = fma(c[l].x, v.x, a[l].x);
                    a[l].y = fma(c[l].x, v.y, a[l].y);
                } else {
                    a[l] = cfma(c[l], v, a[l]);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < NOUT; ++l) {
            if (l < nout) {
                double2 *o = out + (size_t)l * ld_out + i;
                if (acc_out) { double2 p = *o; a[l].x += p.x; a[l].y += p.y; }
                *o = a[l];
            }
        }
    }
}

}  // namespace dlz
