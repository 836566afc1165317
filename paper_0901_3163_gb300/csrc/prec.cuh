// Precision traits of the Krylov vectors of the Lanczos, CG and MinRes
// recurrences (Sec. 1-2): FP64 (double2 elements, 12 per site)
// and FP32 (float4 elements, 6 per site).  Reductions sum across threads and
// blocks in FP64 (FP32 vectors accumulate each thread's few elements in float
// first); element updates run in the vector precision.
#pragma once

#include "dlz_internal.cuh"
#include "reduce.cuh"

namespace dlz {

struct P64 {
    typedef double2 E;
    typedef double2 C;   // coefficient of a complex combination
    typedef double Acc;  // per-thread reduction accumulator
    typedef double S;    // scalar type of element updates
    static constexpr bool kF32 = false;
    static long nel(const Op &op) { return 12L * op.g.V; }
    static int apply(Op &op, E *out, const E *in, int which, E *tmp) { return apply64(op, out, in, which, tmp); }
    __device__ static double rdot(E a, E b) { return a.x * b.x + a.y * b.y; }
    __device__ static void cdot(E a, E b, double &re, double &im) {
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    __device__ static double nrm(E a) { return a.x * a.x + a.y * a.y; }
    __device__ static E axpy(double s, E x, E y) { return make_double2(fma(s, x.x, y.x), fma(s, x.y, y.y)); }
    __device__ static E scal(double s, E x) { return make_double2(s * x.x, s * x.y); }
    __device__ static E zero() { return make_double2(0.0, 0.0); }
    // y += c x (real c / complex c)
    __device__ static void racc(double c, E x, E &y) { y.x = fma(c, x.x, y.x); y.y = fma(c, x.y, y.y); }
    __device__ static void cacc(double2 c, E x, E &y) { y = cfma(c, x, y); }
    __device__ static E add(E a, E b) { return make_double2(a.x + b.x, a.y + b.y); }
};

struct P32 {
    typedef float4 E;
    typedef float2 C;
    typedef float Acc;
    typedef float S;     // FP32 updates take FP32 scalars (no FP64 op per element)
    static constexpr bool kF32 = true;
    static long nel(const Op &op) { return 6L * op.g.V; }
    static int apply(Op &op, E *out, const E *in, int which, E *tmp) { return apply32(op, out, in, which, tmp); }
    __device__ static float rdot(E a, E b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }
    __device__ static void cdot(E a, E b, float &re, float &im) {
        re += (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w);
        im += (a.x * b.y - a.y * b.x) + (a.z * b.w - a.w * b.z);
    }
    __device__ static float nrm(E a) { return (a.x * a.x + a.y * a.y) + (a.z * a.z + a.w * a.w); }
    __device__ static E axpy(float f, E x, E y) {
        return make_float4(fmaf(f, x.x, y.x), fmaf(f, x.y, y.y), fmaf(f, x.z, y.z), fmaf(f, x.w, y.w));
    }
    __device__ static E scal(float f, E x) { return make_float4(f * x.x, f * x.y, f * x.z, f * x.w); }
    __device__ static E zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static void racc(float c, E x, E &y) {
        y.x = fmaf(c, x.x, y.x); y.y = fmaf(c, x.y, y.y); y.z = fmaf(c, x.z, y.z); y.w = fmaf(c, x.w, y.w);
    }
    __device__ static void cacc(float2 c, E x, E &y) {
        y.x = fmaf(c.x, x.x, y.x); y.x = fmaf(-c.y, x.y, y.x);
        y.y = fmaf(c.x, x.y, y.y); y.y = fmaf(c.y, x.x, y.y);
        y.z = fmaf(c.x, x.z, y.z); y.z = fmaf(-c.y, x.w, y.z);
        y.w = fmaf(c.x, x.w, y.w); y.w = fmaf(c.y, x.z, y.w);
    }
    __device__ static E add(E a, E b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
};

// reduce with the per-thread accumulator type of precision P
template <class P, int ND, class Body, class Fin>
inline int red(Op &op, long n, Body body, Fin fin) {
    if constexpr (P::kF32) return reduce32<ND>(op, n, body, fin);
    else return reduce<ND>(op, n, body, fin);
}

// out_l = (acc ? out_l : 0) + sum_j coef[j][col0 + l] in_j, l < nout <= NOUT.
// Coefficients are given in FP64 (double or double2) and rounded to the
// vector precision in shared memory.
template <class P, bool REAL, int NOUT>
__global__ void __launch_bounds__(128)
k_combine(typename P::E *__restrict__ out, long ld_out, int nout, const typename P::E *__restrict__ in,
          long ld_in, int nin, const void *__restrict__ coef, int ld_coef, int col0, bool acc_out, long n) {
    typedef typename P::E E;
    typedef typename P::C C;
    extern __shared__ unsigned char csm_raw[];
    C *csm = reinterpret_cast<C *>(csm_raw);   // [nin][NOUT]
    for (int t = threadIdx.x; t < nin * NOUT; t += blockDim.x) {
        const int j = t / NOUT, l = t % NOUT;
        double cr = 0.0, ci = 0.0;
        if (l < nout) {
            if (REAL) cr = ((const double *)coef)[(size_t)j * ld_coef + col0 + l];
            else {
                const double2 c = ((const double2 *)coef)[(size_t)j * ld_coef + col0 + l];
                cr = c.x; ci = c.y;
            }
        }
        C c;
        c.x = cr; c.y = ci;
        csm[t] = c;
    }
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        E a[NOUT];
#pragma unroll
        for (int l = 0; l < NOUT; ++l) a[l] = P::zero();
        for (int j = 0; j < nin; ++j) {
            const E v = in[(size_t)j * ld_in + i];
            const C *c = csm + j * NOUT;
#pragma unroll
            for (int l = 0; l < NOUT; ++l) {
                if (REAL) P::racc(c[l].x, v, a[l]);
                else P::cacc(c[l], v, a[l]);
            }
        }
#pragma unroll
        for (int l = 0; l < NOUT; ++l) {
            if (l < nout) {
                E *o = out + (size_t)l * ld_out + i;
                *o = acc_out ? P::add(*o, a[l]) : a[l];
            }
        }
    }
}

template <class P>
inline int combine(Op &op, typename P::E *out, long ld_out, int nout, const typename P::E *in, long ld_in,
                   int nin, const void *dev_coef, int ld_coef, bool real, bool acc) {
    const long n = P::nel(op);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_combine<P, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine<P, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine<P, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine<P, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    if (nin <= 0 || nout <= 0) return DLZ_OK;
    long blocks = (n + 127) / 128;
    blocks = blocks < 152L * 8 ? blocks : 152L * 8;
    for (int l0 = 0; l0 < nout; l0 += 16) {
        const int nb = (nout - l0) < 16 ? (nout - l0) : 16;
        typename P::E *o = out + (size_t)l0 * ld_out;
        if (nb == 1) {
            const size_t sm = (size_t)nin * sizeof(typename P::C);
            if (real) k_combine<P, true, 1><<<(int)blocks, 128, sm, op.stream>>>(o, ld_out, 1, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
            else k_combine<P, false, 1><<<(int)blocks, 128, sm, op.stream>>>(o, ld_out, 1, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
        } else {
            const size_t sm = (size_t)nin * 16 * sizeof(typename P::C);
            if (real) k_combine<P, true, 16><<<(int)blocks, 128, sm, op.stream>>>(o, ld_out, nb, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
            else k_combine<P, false, 16><<<(int)blocks, 128, sm, op.stream>>>(o, ld_out, nb, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
        }
        op.prof.launches++;
        DLZ_CUDA_TRY(cudaGetLastError());
    }
    return DLZ_OK;
}

// ---------------------------------------------------------------- FP32 multi-dot
// <V_l, w> for l < nv in one pass over the V_l: block (site chunk, group of 8
// vectors); each thread loads w at its site once and accumulates 8 complex dots
// over the 6 planes in float; warps and blocks are summed in FP64 (fixed order).
constexpr int kMdThreads = 128;
static __global__ void __launch_bounds__(kMdThreads)
k_multidot32(const float4 *__restrict__ V, long ld, int nv, const float4 *__restrict__ w, int sites,
             double *__restrict__ partials) {
    const int grp = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float re[8], im[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) { re[l] = 0.f; im[l] = 0.f; }
    if (s < sites) {
        float4 x[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) x[c] = w[(size_t)c * sites + s];
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            const int vi = grp * 8 + l;
            if (vi < nv) {
                const float4 *v = V + (size_t)vi * ld;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const float4 a = v[(size_t)c * sites + s];
                    re[l] += (a.x * x[c].x + a.y * x[c].y) + (a.z * x[c].z + a.w * x[c].w);
                    im[l] += (a.x * x[c].y - a.y * x[c].x) + (a.z * x[c].w - a.w * x[c].z);
                }
            }
        }
    }
    __shared__ double sm[16][kMdThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        double a = (double)re[l], b = (double)im[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { sm[2 * l][warp] = a; sm[2 * l + 1][warp] = b; }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kMdThreads / 32; ++k) t += sm[threadIdx.x][k];
        // partials[(grp*16 + j) * gridDim.x + blockIdx.x]
        partials[((size_t)grp * 16 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}

// out[l] = scale * (sum over blocks of the partials of vector l), one block per vector
static __global__ void __launch_bounds__(256)
k_multidot_fin(const double *__restrict__ partials, int nblk, int nv, double scale, double2 *__restrict__ out) {
    const int l = blockIdx.x;
    const int grp = l / 8, j = l % 8;
    const double *pre = partials + ((size_t)grp * 16 + 2 * j) * nblk;
    const double *pim = pre + nblk;
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) { a += pre[t]; b += pim[t]; }
    __shared__ double sa[8], sb[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) { x += sa[k]; y += sb[k]; }
        out[l] = make_double2(scale * x, scale * y);
    }
}

// Grow the FP32 multi-dot scratch for up to nv vectors (call outside graph capture).
inline int reserve_multidot(Op &op, int nv) {
    const int nblk = (op.g.V + kMdThreads - 1) / kMdThreads;
    const size_t need = (size_t)((nv + 7) / 8) * 16 * nblk * sizeof(double);
    if (op.md_scratch.bytes < need) {
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        DLZ_TRY(op.md_scratch.alloc(need));
    }
    return DLZ_OK;
}

// dev_out[l] = scale * <V_l, w> (complex), l < nv, V_l = V + l*ld
template <class P>
inline int multidot(Op &op, const typename P::E *V, long ld, int nv, const typename P::E *w, double2 *dev_out,
                    double scale) {
    if constexpr (P::kF32) {
        if (nv <= 0) return DLZ_OK;
        const int sites = op.g.V;
        const int nblk = (sites + kMdThreads - 1) / kMdThreads;
        const int ngrp = (nv + 7) / 8;
        const size_t need = (size_t)ngrp * 16 * nblk;
        if (op.md_scratch.bytes < need * sizeof(double))
            return fail(DLZ_ERR_BADARG, "multidot scratch not reserved (reserve_multidot)");
        k_multidot32<<<dim3(nblk, ngrp), kMdThreads, 0, op.stream>>>(V, ld, nv, w, sites, op.md_scratch.as<double>());
        k_multidot_fin<<<nv, 256, 0, op.stream>>>(op.md_scratch.as<double>(), nblk, nv, scale, dev_out);
        op.prof.launches += 2;
        DLZ_CUDA_TRY(cudaGetLastError());
        return DLZ_OK;
    }
    typedef typename P::E E;
    const long n = P::nel(op);
    for (int l0 = 0; l0 < nv; l0 += 8) {
        const int nb = (nv - l0) < 8 ? (nv - l0) : 8;
        const E *Vb = V + (size_t)l0 * ld;
        double2 *o = dev_out + l0;
        DLZ_TRY(red<P, 16>(op, n, [=] __device__(long i, typename P::Acc (&acc)[16]) {
            const E x = w[i];
#pragma unroll
            for (int l = 0; l < 8; ++l)
                if (l < nb) P::cdot(Vb[(size_t)l * ld + i], x, acc[2 * l], acc[2 * l + 1]);
        }, [=] __device__(const double *r) {
            for (int l = 0; l < nb; ++l) o[l] = make_double2(scale * r[2 * l], scale * r[2 * l + 1]);
        }));
    }
    return DLZ_OK;
}

}  // namespace dlz
