// Wilson-Dirac stencil kernels (Sec. 2 of arXiv:0901.3163: the Wilson matrix M,
// used as gamma5 M and M^dagger M) and the layout conversions around them.
//
// One thread per lattice site.  Spinor and link planes are component-major,
// so each load instruction of a warp reads consecutive 16-byte (FP64 double2,
// FP32 float4) or 8-byte (FP32 link float2) words; the eight neighbour
// spinors of a site are re-read from L1/L2 (the time neighbour of site s is
// Lx*Ly*Lz sites away: a window of a few MB that stays in the 129 MB L2), so
// DRAM sees each spinor and link about once per application.
#include "dlz_internal.cuh"
#include "slab_walk.cuh"
#include "wilson_site.cuh"

namespace dlz {

namespace {

constexpr int kStencilThreads64 = 128;
constexpr int kStencilThreads32 = 128;

template <typename T, bool G5IN, bool G5OUT>
__global__ void __launch_bounds__(128)
k_wilson(typename Field<T>::vec *__restrict__ out, const typename Field<T>::vec *__restrict__ in,
         const typename Link<T>::vec *__restrict__ U, Geom g, T kappa) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    cx<T> o[12];
    wilson_site<T, G5IN, G5OUT>(s, g, kappa, in, U, o);
    Field<T>::store(out, g.V, s, o);
}

// N right-hand sides stored one after another (each nel elements); consecutive
// blocks take the same sites of different right-hand sides, so the links they
// share are read from L2 (and DRAM) once.
template <typename T, bool G5IN, bool G5OUT>
__device__ inline void wilson_batch_body(typename Field<T>::vec *__restrict__ out,
                                         const typename Field<T>::vec *__restrict__ in,
                                         const typename Link<T>::vec *__restrict__ U, const Geom &g, T kappa,
                                         int nrhs, long nel) {
    const int r = blockIdx.x % nrhs;
    const int s = (blockIdx.x / nrhs) * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    cx<T> o[12];
    wilson_site<T, G5IN, G5OUT>(s, g, kappa, in + (size_t)r * nel, U, o);
    Field<T>::store(out + (size_t)r * nel, g.V, s, o);
}

template <typename T, bool G5IN, bool G5OUT>
__global__ void __launch_bounds__(128)
k_wilson_batch(typename Field<T>::vec *__restrict__ out, const typename Field<T>::vec *__restrict__ in,
               const typename Link<T>::vec *__restrict__ U, Geom g, T kappa, int nrhs, long nel) {
    wilson_batch_body<T, G5IN, G5OUT>(out, in, U, g, kappa, nrhs, nel);
}

// FP32: at most 80 registers (6 blocks per SM), measured 5% faster at 11-16
// right-hand sides than without the bound.  Blocks of 128 sites in the slab walk
// (slab_walk.cuh).
template <bool G5IN, bool G5OUT>
__global__ void __launch_bounds__(kSlabBlock, 6)
k_wilson_batch32(float4 *__restrict__ out, const float4 *__restrict__ in, const float4 *__restrict__ U, Geom g,
                 SlabWalk w, float kappa, int nrhs, long nel) {
    const int r = blockIdx.x % nrhs;
    int s0, nb;
    slab_block(w, blockIdx.x / nrhs, s0, nb);
    if (threadIdx.x == 0 && nb > 0) {
        prefetch_planes_l2(in + (size_t)r * nel, 6, g.V, s0, nb);
        if (r == 0) prefetch_planes_l2(U, 12, g.V, s0, nb);
    }
    if ((int)threadIdx.x >= nb) return;
    const int s = s0 + threadIdx.x;
    float2 o[12];
    wilson_site<float, G5IN, G5OUT>(s, g, kappa, in + (size_t)r * nel, U, o);
    Field<float>::store(out + (size_t)r * nel, g.V, s, o);
}

template <typename T, bool G5IN, bool G5OUT>
inline void launch_batch_kernel(unsigned blocks, int threads, cudaStream_t st, typename Field<T>::vec *out,
                                const typename Field<T>::vec *in, const typename Link<T>::vec *U, const Geom &g,
                                const SlabWalk &w, T kappa, int nrhs, long nel) {
    if constexpr (sizeof(T) == 4)
        k_wilson_batch32<G5IN, G5OUT><<<blocks, kSlabBlock, 0, st>>>(out, in, U, g, w, kappa, nrhs, nel);
    else
        k_wilson_batch<T, G5IN, G5OUT><<<blocks, threads, 0, st>>>(out, in, U, g, kappa, nrhs, nel);
}

template <typename T>
int launch_wilson_batch(Op &op, typename Field<T>::vec *out, const typename Field<T>::vec *in,
                        const typename Link<T>::vec *U, int which, int nrhs, long nel, int threads) {
    const Geom &g = op.g;
    // FP32: the slab walk for a stencil moving ~200 bytes per site and right-hand side
    const SlabWalk w = make_slab_walk(g.L[0] * g.L[1], g.L[2], g.L[3], nrhs, 200.0);
    const long blocks = sizeof(T) == 4 ? slab_blocks(w) * nrhs : (long)((g.V + threads - 1) / threads) * nrhs;
    const T kappa = (T)op.kappa;
    op.prof.stencil_start(op.stream, sizeof(T) == 4, g.V, nrhs);
    switch (which) {
    case DLZ_D: launch_batch_kernel<T, false, false>((unsigned)blocks, threads, op.stream, out, in, U, g, w, kappa, nrhs, nel); break;
    case DLZ_DDAG: launch_batch_kernel<T, true, true>((unsigned)blocks, threads, op.stream, out, in, U, g, w, kappa, nrhs, nel); break;
    case DLZ_Q: launch_batch_kernel<T, false, true>((unsigned)blocks, threads, op.stream, out, in, U, g, w, kappa, nrhs, nel); break;
    default: return fail(DLZ_ERR_BADARG, "stencil: which must be D, DDAG or Q");
    }
    op.prof.stencil_stop(op.stream);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

template <typename T>
int launch_wilson(Op &op, typename Field<T>::vec *out, const typename Field<T>::vec *in,
                  const typename Link<T>::vec *U, int which, int threads) {
    const Geom &g = op.g;
    const int blocks = (g.V + threads - 1) / threads;
    const T kappa = (T)op.kappa;
    op.prof.stencil_start(op.stream, sizeof(T) == 4, g.V, 1);
    switch (which) {
    case DLZ_D: k_wilson<T, false, false><<<blocks, threads, 0, op.stream>>>(out, in, U, g, kappa); break;
    case DLZ_DDAG: k_wilson<T, true, true><<<blocks, threads, 0, op.stream>>>(out, in, U, g, kappa); break;
    case DLZ_Q: k_wilson<T, false, true><<<blocks, threads, 0, op.stream>>>(out, in, U, g, kappa); break;
    default: return fail(DLZ_ERR_BADARG, "stencil: which must be D, DDAG or Q");
    }
    op.prof.stencil_stop(op.stream);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

// ------------------------------------------------------------------ layout kernels
__global__ void k_pack64(double2 *__restrict__ dst, const double2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // canonical index s*12 + a
    if (i >= 12L * V) return;
    const int s = (int)(i / 12), a = (int)(i % 12);
    dst[(size_t)a * V + s] = src[i];
}
__global__ void k_unpack64(double2 *__restrict__ dst, const double2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 12L * V) return;
    const int s = (int)(i / 12), a = (int)(i % 12);
    dst[i] = src[(size_t)a * V + s];
}
__global__ void k_pack32(float4 *__restrict__ dst, const float2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // s*6 + c
    if (i >= 6L * V) return;
    const int s = (int)(i / 6), c = (int)(i % 6);
    const float2 a = src[(size_t)s * 12 + 2 * c], b = src[(size_t)s * 12 + 2 * c + 1];
    dst[(size_t)c * V + s] = make_float4(a.x, a.y, b.x, b.y);
}
__global__ void k_unpack32(float2 *__restrict__ dst, const float4 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6L * V) return;
    const int s = (int)(i / 6), c = (int)(i % 6);
    const float4 q = src[(size_t)c * V + s];
    dst[(size_t)s * 12 + 2 * c] = make_float2(q.x, q.y);
    dst[(size_t)s * 12 + 2 * c + 1] = make_float2(q.z, q.w);
}
// internal FP64 planes <-> internal FP32 planes (plane c of FP32 = planes 2c, 2c+1)
__global__ void k_64to32(float4 *__restrict__ dst, const double2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // c*V + s
    if (i >= 6L * V) return;
    const int c = (int)(i / V), s = (int)(i % V);
    const double2 a = src[(size_t)(2 * c) * V + s], b = src[(size_t)(2 * c + 1) * V + s];
    dst[i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
__global__ void k_32to64(double2 *__restrict__ dst, const float4 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6L * V) return;
    const int c = (int)(i / V), s = (int)(i % V);
    const float4 q = src[i];
    dst[(size_t)(2 * c) * V + s] = make_double2(q.x, q.y);
    dst[(size_t)(2 * c + 1) * V + s] = make_double2(q.z, q.w);
}

inline int grid_for(long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

// An even-odd operator applies its Schur complement (wilson_eo.cu) wherever a solver
// asks for D, D^dag or Q: the solvers run unchanged on its even-site vectors.
int wilson64(Op &op, double2 *out, const double2 *in, int which) {
    if (op.eo) return eo_apply64(op, out, in, which, 1);
    return launch_wilson<double>(op, out, in, op.gauge64.as<double2>(), which, kStencilThreads64);
}
int wilson32(Op &op, float4 *out, const float4 *in, int which) {
    if (op.eo) return eo_apply32(op, out, in, which, 1);
    return launch_wilson<float>(op, out, in, op.gauge32.as<float4>(), which, kStencilThreads32);
}

int wilson32_batch(Op &op, float4 *out, const float4 *in, int which, int nrhs) {
    if (op.eo) return eo_apply32(op, out, in, which, nrhs);
    return launch_wilson_batch<float>(op, out, in, op.gauge32.as<float4>(), which, nrhs, 6L * op.g.V,
                                      kStencilThreads32);
}
int wilson64_batch(Op &op, double2 *out, const double2 *in, int which, int nrhs) {
    if (op.eo) return eo_apply64(op, out, in, which, nrhs);
    return launch_wilson_batch<double>(op, out, in, op.gauge64.as<double2>(), which, nrhs, 12L * op.g.V,
                                       kStencilThreads64);
}

int apply64(Op &op, double2 *out, const double2 *in, int which, double2 *tmp) {
    if (which == DLZ_DDAGD) {
        // D^dag D = Q Q (gamma5 D is hermitian, Q^2 = gamma5 D gamma5 D = D^dag D)
        DLZ_TRY(wilson64(op, tmp, in, DLZ_Q));
        return wilson64(op, out, tmp, DLZ_Q);
    }
    return wilson64(op, out, in, which);
}
int apply32(Op &op, float4 *out, const float4 *in, int which, float4 *tmp) {
    if (which == DLZ_DDAGD) {
        DLZ_TRY(wilson32(op, tmp, in, DLZ_Q));
        return wilson32(op, out, tmp, DLZ_Q);
    }
    return wilson32(op, out, in, which);
}

int pack64(Op &op, double2 *dst, const double2 *src) {
    const long n = 12L * op.g.V;
    k_pack64<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
int unpack64(Op &op, double2 *dst, const double2 *src) {
    const long n = 12L * op.g.V;
    k_unpack64<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
int pack32(Op &op, float4 *dst, const float2 *src) {
    const long n = 6L * op.g.V;
    k_pack32<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
int unpack32(Op &op, float2 *dst, const float4 *src) {
    const long n = 6L * op.g.V;
    k_unpack32<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
int convert64to32(Op &op, float4 *dst, const double2 *src) {
    const long n = 6L * op.g.V;
    k_64to32<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}
int convert32to64(Op &op, double2 *dst, const float4 *src) {
    const long n = 6L * op.g.V;
    k_32to64<<<grid_for(n, 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

}  // namespace dlz
