// Wilson stencil on bfloat16 spinors with FP32 arithmetic (the Wilson matrix M of
// arXiv:0901.3163, Sec. 2, in a storage format the paper does not use).
//
// Spinor storage: 6 planes of uint2 per right-hand side, each uint2 holding two
// complex components as four bfloat16 values (re, im, re, im) -- the FP32 plane
// layout with half the bytes.  Links stay in the FP32 two-row form.  Every
// product and sum is FP32; the result is rounded to bfloat16 (nearest even) once,
// at the store.
#include <cuda_bf16.h>

#include "dlz_internal.cuh"
#include "wilson_site.cuh"

namespace dlz {
namespace {

__device__ inline void bf_load(const uint2 *__restrict__ p, int V, int s, float2 (&v)[12]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const uint2 q = p[(size_t)c * V + s];
        __nv_bfloat162 a, b;
        memcpy(&a, &q.x, 4);
        memcpy(&b, &q.y, 4);
        v[2 * c] = __bfloat1622float2(a);
        v[2 * c + 1] = __bfloat1622float2(b);
    }
}

__device__ inline void bf_store(uint2 *__restrict__ p, int V, int s, const float2 (&v)[12]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v[2 * c].x, v[2 * c].y);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * c + 1].x, v[2 * c + 1].y);
        uint2 q;
        memcpy(&q.x, &a, 4);
        memcpy(&q.y, &b, 4);
        p[(size_t)c * V + s] = q;
    }
}

template <int MU, bool G5IN>
__device__ inline void hop_pair_bf(int s, const int (&c)[4], const Geom &g, int stride, const uint2 *__restrict__ in,
                                   const float4 *__restrict__ U, float2 (&acc)[12]) {
    const int L = g.L[MU];
    const int sf = (c[MU] == L - 1) ? s - (L - 1) * stride : s + stride;
    const float phf = (MU == 3 && c[3] == L - 1) ? (float)g.bc_t : 1.f;
    const int sb = (c[MU] == 0) ? s + (L - 1) * stride : s - stride;
    const float phb = (MU == 3 && c[3] == 0) ? (float)g.bc_t : 1.f;
    float2 p[12], u[9];
    bf_load(in, g.V, sf, p);
    maybe_g5<G5IN>(p);
    load_link<float>(U, g.V, MU, s, u);
    hop_fwd<float, MU>(p, u, phf, acc);
    bf_load(in, g.V, sb, p);
    maybe_g5<G5IN>(p);
    load_link<float>(U, g.V, MU, sb, u);
    hop_bwd<float, MU>(p, u, phb, acc);
}

template <bool G5IN, bool G5OUT>
__global__ void __launch_bounds__(128)
k_wilson_bf16_batch(uint2 *__restrict__ out, const uint2 *__restrict__ in, const float4 *__restrict__ U, Geom g,
                    float kappa, int nrhs, long nel) {
    const int r = blockIdx.x % nrhs;
    const int s = (blockIdx.x / nrhs) * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const uint2 *inr = in + (size_t)r * nel;
    int c[4];
    int t = s;
    c[0] = t % g.L[0]; t /= g.L[0];
    c[1] = t % g.L[1]; t /= g.L[1];
    c[2] = t % g.L[2];
    c[3] = t / g.L[2];
    const int st1 = g.L[0], st2 = g.L[0] * g.L[1], st3 = st2 * g.L[2];
    float2 acc[12], o[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = make_float2(0.f, 0.f);
    hop_pair_bf<0, G5IN>(s, c, g, 1, inr, U, acc);
    hop_pair_bf<1, G5IN>(s, c, g, st1, inr, U, acc);
    hop_pair_bf<2, G5IN>(s, c, g, st2, inr, U, acc);
    hop_pair_bf<3, G5IN>(s, c, g, st3, inr, U, acc);
    bf_load(inr, g.V, s, o);
    maybe_g5<G5IN>(o);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        o[a].x = o[a].x - kappa * acc[a].x;
        o[a].y = o[a].y - kappa * acc[a].y;
    }
    maybe_g5<G5OUT>(o);
    bf_store(out + (size_t)r * nel, g.V, s, o);
}

// canonical complex64 [V][12] <-> bfloat16 planes
__global__ void k_pack_bf16(uint2 *__restrict__ dst, const float2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // s*6 + c
    if (i >= 6L * V) return;
    const int s = (int)(i / 6), c = (int)(i % 6);
    const float2 a = src[(size_t)s * 12 + 2 * c], b = src[(size_t)s * 12 + 2 * c + 1];
    const __nv_bfloat162 x = __floats2bfloat162_rn(a.x, a.y), y = __floats2bfloat162_rn(b.x, b.y);
    uint2 q;
    memcpy(&q.x, &x, 4);
    memcpy(&q.y, &y, 4);
    dst[(size_t)c * V + s] = q;
}
__global__ void k_unpack_bf16(float2 *__restrict__ dst, const uint2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6L * V) return;
    const int s = (int)(i / 6), c = (int)(i % 6);
    const uint2 q = src[(size_t)c * V + s];
    __nv_bfloat162 x, y;
    memcpy(&x, &q.x, 4);
    memcpy(&y, &q.y, 4);
    dst[(size_t)s * 12 + 2 * c] = __bfloat1622float2(x);
    dst[(size_t)s * 12 + 2 * c + 1] = __bfloat1622float2(y);
}

}  // namespace

int wilson_bf16_batch(Op &op, uint2 *out, const uint2 *in, int which, int nrhs) {
    const Geom &g = op.g;
    const long nel = 6L * g.V;
    const long blocks = (long)((g.V + 127) / 128) * nrhs;
    const float kappa = (float)op.kappa;
    const float4 *U = op.gauge32.as<float4>();
    switch (which) {
    case DLZ_D: k_wilson_bf16_batch<false, false><<<(unsigned)blocks, 128, 0, op.stream>>>(out, in, U, g, kappa, nrhs, nel); break;
    case DLZ_DDAG: k_wilson_bf16_batch<true, true><<<(unsigned)blocks, 128, 0, op.stream>>>(out, in, U, g, kappa, nrhs, nel); break;
    case DLZ_Q: k_wilson_bf16_batch<false, true><<<(unsigned)blocks, 128, 0, op.stream>>>(out, in, U, g, kappa, nrhs, nel); break;
    default: return fail(DLZ_ERR_BADARG, "stencil: which must be D, DDAG or Q");
    }
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int pack_bf16(Op &op, uint2 *dst, const float2 *src) {
    const long n = 6L * op.g.V;
    k_pack_bf16<<<(unsigned)((n + 255) / 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int unpack_bf16(Op &op, float2 *dst, const uint2 *src) {
    const long n = 6L * op.g.V;
    k_unpack_bf16<<<(unsigned)((n + 255) / 256), 256, 0, op.stream>>>(dst, src, op.g.V);
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

}  // namespace dlz
