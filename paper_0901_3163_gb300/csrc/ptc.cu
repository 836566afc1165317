// Learned seed for the deflation space: a gauge-covariant parallel-transport
// convolution (PTC) network, its backward pass and an Adam step, the subspace
// loss against a deflation set, and the Rayleigh-Ritz seed built from network
// outputs.  arXiv:0901.3163 computes its deflation space with Lan-DR /
// MinRes-DR only (Sec. 2); this part has no counterpart in the paper.
//
// Layer (C_in -> C_out channels, each channel a Wilson spinor field):
//   out[c'](x) = sum_o sum_c W[o][c'][c] (T_o in[c])(x),
// nine offsets o = 0, +mu (1 + 2 mu), -mu (2 + 2 mu); T_0 = 1,
// (T_+mu psi)(x) = U_mu(x) psi(x + mu), (T_-mu psi)(x) = U_mu(x - mu)^dag psi(x - mu)
// (periodic in all four directions); W[o][c'][c] a complex 4x4 spin matrix, so
// colour moves only with the links and the layer commutes with gauge
// transformations.  Weights are used in bfloat16 (an FP32 master copy is what
// Adam updates); every product and sum is FP32.
//
// Gradients follow G(z) = dL/dRe z + i dL/dIm z: for out = W t,
// G(W) = sum_{x, colour} G(out) t^dag, and G(in) = L^dag G(out), L^dag being the
// layer with weights W[opp(o)]^H (conjugate transpose in spin, channels swapped).
//
// Layouts: a field of C channels for nvec vectors is float4 [nvec][C][6][V]
// (the FP32 spinor planes of the solvers); weights of a layer [9][C_out][C_in][16],
// entry 4 s' + s of the spin matrix.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "solvers.h"
#include "wilson_site.cuh"

namespace dlz {
constexpr int kMaxLayersNet = 8;
namespace {

constexpr int kMaxWidth = 16;      // channels per layer (weight-gradient tile limit)
constexpr int kFwdThreads = 128;
constexpr int kTS = 32;            // sites per weight-gradient tile
constexpr int kLD = 3 * kTS + 1;   // padded row of a staged tile (float2)
constexpr int kGradBlocks = 64;    // weight-gradient blocks per offset

__device__ inline int opposite(int o) { return o == 0 ? 0 : (((o - 1) & 1) == 0 ? o + 1 : o - 1); }

// neighbour site of offset o (> 0) and the link that transports from it
__device__ inline void neighbour(int s, const Geom &g, int o, int &sn, int &ls, int &mu, bool &fwd) {
    mu = (o - 1) >> 1;
    fwd = ((o - 1) & 1) == 0;
    int st = 1, r = s;
    int cmu = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int cd = r % g.L[d];
        r /= g.L[d];
        if (d == mu) cmu = cd;
        if (d < mu) st *= g.L[d];
    }
    const int L = g.L[mu];
    if (fwd) {
        sn = (cmu == L - 1) ? s - (L - 1) * st : s + st;
        ls = s;
    } else {
        sn = (cmu == 0) ? s + (L - 1) * st : s - st;
        ls = sn;
    }
}

// t = U p (fwd) or U^dag p (bwd), per spin
__device__ inline void transport(const float2 (&p)[12], const float2 (&u)[9], bool fwd, float2 (&t)[12]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                a = fwd ? cfma(u[3 * i + j], p[3 * sp + j], a) : cfmaConj(u[3 * j + i], p[3 * sp + j], a);
            t[3 * sp + i] = a;
        }
    }
}

__device__ inline void load_transported(const float4 *__restrict__ x, const float4 *__restrict__ U,
                                        const Geom &g, int s, int o, float2 (&t)[12]) {
    if (o == 0) {
        Field<float>::load(x, g.V, s, t);
        return;
    }
    int sn, ls, mu;
    bool fwd;
    neighbour(s, g, o, sn, ls, mu, fwd);
    float2 p[12], u[9];
    Field<float>::load(x, g.V, sn, p);
    Link<float>::load(U, g.V, mu, ls, u);
    transport(p, u, fwd, t);
}

// out[vec][g0 + q] for q < CG; grid (site blocks, C_out / CG, nvec)
template <int CG>
__global__ void __launch_bounds__(kFwdThreads)
k_ptc_fwd(float4 *__restrict__ out, const float4 *__restrict__ in, const __nv_bfloat162 *__restrict__ W,
          const float4 *__restrict__ U, Geom g, int cin, int cout) {
    extern __shared__ __nv_bfloat162 ws[];   // [9][CG][cin][16]
    const int g0 = blockIdx.y * CG;
    const int vec = blockIdx.z;
    const int nws = 9 * CG * cin * 16;
    for (int t = threadIdx.x; t < nws; t += blockDim.x) {
        const int e = t % 16;
        int r = t / 16;
        const int c = r % cin;
        r /= cin;
        const int q = r % CG, o = r / CG;
        ws[t] = W[(((size_t)o * cout + g0 + q) * cin + c) * 16 + e];
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    float2 acc[CG][12];
#pragma unroll
    for (int q = 0; q < CG; ++q)
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[q][a] = make_float2(0.f, 0.f);
    const size_t plane = (size_t)6 * g.V;
    const float4 *inv = in + (size_t)vec * cin * plane;
    for (int o = 0; o < 9; ++o) {
        int sn = s, ls = s, mu = 0;
        bool fwd = true;
        float2 u[9];
        if (o > 0) {
            neighbour(s, g, o, sn, ls, mu, fwd);
            Link<float>::load(U, g.V, mu, ls, u);
        }
        for (int ci = 0; ci < cin; ++ci) {
            float2 p[12], t[12];
            Field<float>::load(inv + (size_t)ci * plane, g.V, sn, p);
            if (o > 0) transport(p, u, fwd, t);
            else {
#pragma unroll
                for (int a = 0; a < 12; ++a) t[a] = p[a];
            }
            const __nv_bfloat162 *wp = ws + ((size_t)o * CG * cin + ci) * 16;
#pragma unroll
            for (int q = 0; q < CG; ++q) {
                const __nv_bfloat162 *wq = wp + (size_t)q * cin * 16;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
#pragma unroll
                    for (int sp = 0; sp < 4; ++sp) {
                        const float2 w = __bfloat1622float2(wq[r * 4 + sp]);
#pragma unroll
                        for (int col = 0; col < 3; ++col)
                            acc[q][3 * r + col] = cfma(w, t[3 * sp + col], acc[q][3 * r + col]);
                    }
                }
            }
        }
    }
    float4 *ov = out + (size_t)vec * cout * plane;
#pragma unroll
    for (int q = 0; q < CG; ++q) Field<float>::store(ov + (size_t)(g0 + q) * plane, g.V, s, acc[q]);
}

// Block partials of G(W)[o] = sum_{x, colour} G(out) (T_o in)^dag, as the GEMM
// (C_out*4) x (3 sites) times (3 sites) x (C_in*4) over tiles of kTS sites.
// grid (kGradBlocks, 9); partials [o][block][C_out*4][C_in*4]
__global__ void __launch_bounds__(256)
k_ptc_wgrad(float2 *__restrict__ partials, const float4 *__restrict__ gout, const float4 *__restrict__ x,
            const float4 *__restrict__ U, Geom g, int cin, int cout, int nvec) {
    extern __shared__ float2 sm[];
    const int rows = cout * 4, cols = cin * 4;
    float2 *Gs = sm;                   // [rows][kLD]
    float2 *Ts = sm + rows * kLD;      // [cols][kLD]
    const int o = blockIdx.y;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    const size_t plane = (size_t)6 * g.V;
    const int tiles_per_vec = (g.V + kTS - 1) / kTS;
    const long ntiles = (long)tiles_per_vec * nvec;
    const int ls = threadIdx.x % kTS, slot = threadIdx.x / kTS;   // 32 sites x 8 slots
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int vec = (int)(tile / tiles_per_vec);
        const int s = (int)(tile % tiles_per_vec) * kTS + ls;
        const bool ok = s < g.V;
        __syncthreads();
        for (int cp = slot; cp < cout; cp += 8) {
            float2 p[12];
            if (ok) Field<float>::load(gout + ((size_t)vec * cout + cp) * plane, g.V, s, p);
            else {
#pragma unroll
                for (int a = 0; a < 12; ++a) p[a] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int a = 0; a < 3; ++a) Gs[(cp * 4 + sp) * kLD + a * kTS + ls] = p[3 * sp + a];
        }
        for (int ci = slot; ci < cin; ci += 8) {
            float2 t[12];
            if (ok) load_transported(x + ((size_t)vec * cin + ci) * plane, U, g, s, o, t);
            else {
#pragma unroll
                for (int a = 0; a < 12; ++a) t[a] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int a = 0; a < 3; ++a) Ts[(ci * 4 + sp) * kLD + a * kTS + ls] = t[3 * sp + a];
        }
        __syncthreads();
        for (int k = 0; k < 3 * kTS; ++k) {
            float2 gv[4], tv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = ty + 16 * i;
                gv[i] = r < rows ? Gs[r * kLD + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = tx + 16 * j;
                tv[j] = c < cols ? Ts[c * kLD + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfmaConj(tv[j], gv[i], acc[i][j]);
        }
    }
    float2 *pb = partials + ((size_t)o * gridDim.x + blockIdx.x) * rows * cols;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            if (r < rows && c < cols) pb[(size_t)r * cols + c] = acc[i][j];
        }
}

// grad[o][c'][c][4 s' + s] += sum over blocks (fixed order) of the partials
__global__ void k_ptc_wgrad_sum(float2 *__restrict__ grad, const float2 *__restrict__ partials, int nblk,
                                int cin, int cout) {
    const int rows = cout * 4, cols = cin * 4;
    const long n = 9L * rows * cols;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = (int)(i / ((long)rows * cols));
    const int rc = (int)(i % ((long)rows * cols));
    const int r = rc / cols, c = rc % cols;
    float2 a = make_float2(0.f, 0.f);
    for (int b = 0; b < nblk; ++b) {
        const float2 v = partials[((size_t)o * nblk + b) * rows * cols + rc];
        a.x += v.x;
        a.y += v.y;
    }
    const int cp = r / 4, sp_ = r % 4, ci = c / 4, sp = c % 4;
    float2 &gr = grad[(((size_t)o * cout + cp) * cin + ci) * 16 + sp_ * 4 + sp];
    gr.x += a.x;
    gr.y += a.y;
}

// adjoint weights: wa[o][c][c'][4 s + s'] = conj(w[opp(o)][c'][c][4 s' + s])
__global__ void k_ptc_adjoint(__nv_bfloat162 *__restrict__ wa, const __nv_bfloat162 *__restrict__ w, int cin,
                              int cout) {
    const long n = 9L * cin * cout * 16;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = (int)(i % 16);
    long r = i / 16;
    const int cp = (int)(r % cout);       // wa's input channel = w's output channel
    r /= cout;
    const int c = (int)(r % cin);         // wa's output channel
    const int o = (int)(r / cin);
    const int s = e / 4, sp_ = e % 4;
    __nv_bfloat162 v = w[(((size_t)opposite(o) * cout + cp) * cin + c) * 16 + sp_ * 4 + s];
    v.y = __hneg(v.y);
    wa[i] = v;
}

__global__ void k_to_bf16(__nv_bfloat162 *__restrict__ wb, const float2 *__restrict__ w, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __floats2bfloat162_rn(w[i].x, w[i].y);
}

// Adam on the FP32 master weights (each real and imaginary part a parameter)
__global__ void k_ptc_adam(float2 *__restrict__ w, float2 *__restrict__ gr, float2 *__restrict__ m1,
                           float2 *__restrict__ m2, long n, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 gv = gr[i];
    float2 a = m1[i], b = m2[i], x = w[i];
    a.x = b1 * a.x + (1.f - b1) * gv.x;
    a.y = b1 * a.y + (1.f - b1) * gv.y;
    b.x = b2 * b.x + (1.f - b2) * gv.x * gv.x;
    b.y = b2 * b.y + (1.f - b2) * gv.y * gv.y;
    x.x -= lr * (a.x * c1) / (sqrtf(b.x * c2) + eps);
    x.y -= lr * (a.y * c1) / (sqrtf(b.y * c2) + eps);
    m1[i] = a;
    m2[i] = b;
    w[i] = x;
    gr[i] = make_float2(0.f, 0.f);
}

inline unsigned blocks_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace dlz

struct dlz_net_s {
    dlz::Op *op = nullptr;
    int nl = 0;
    std::vector<int> w;                 // widths, nl + 1
    std::vector<size_t> off;            // first complex weight of each layer
    size_t nw = 0;
    dlz::DevBuf master, grad, m1, m2, wb, wadj, partials;
    int adam_t = 0;
    dlz::DevBuf act[dlz::kMaxLayersNet + 1];   // input of every layer from the last forward
    int act_nvec = 0;
    dlz::DevBuf gbuf[2];
};

namespace dlz {
namespace {

int layer_forward(Op &op, float4 *out, const float4 *in, const __nv_bfloat162 *W, int cin, int cout, int nvec) {
    const Geom g = op.g;
    const float4 *U = op.gauge32.as<float4>();
    const unsigned gx = blocks_for(g.V, kFwdThreads);
    if (cout % 4 == 0) {
        const size_t sm = (size_t)9 * 4 * cin * 16 * sizeof(__nv_bfloat162);
        k_ptc_fwd<4><<<dim3(gx, cout / 4, nvec), kFwdThreads, sm, op.stream>>>(out, in, W, U, g, cin, cout);
    } else if (cout % 2 == 0) {
        const size_t sm = (size_t)9 * 2 * cin * 16 * sizeof(__nv_bfloat162);
        k_ptc_fwd<2><<<dim3(gx, cout / 2, nvec), kFwdThreads, sm, op.stream>>>(out, in, W, U, g, cin, cout);
    } else {
        const size_t sm = (size_t)9 * 1 * cin * 16 * sizeof(__nv_bfloat162);
        k_ptc_fwd<1><<<dim3(gx, cout, nvec), kFwdThreads, sm, op.stream>>>(out, in, W, U, g, cin, cout);
    }
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int refresh_bf16(dlz_net_s *net) {
    Op &op = *net->op;
    k_to_bf16<<<blocks_for((long)net->nw, 256), 256, 0, op.stream>>>(net->wb.as<__nv_bfloat162>(),
                                                                    net->master.as<float2>(), (long)net->nw);
    for (int l = 0; l < net->nl; ++l) {
        const long n = 9L * net->w[l] * net->w[l + 1] * 16;
        k_ptc_adjoint<<<blocks_for(n, 256), 256, 0, op.stream>>>(net->wadj.as<__nv_bfloat162>() + net->off[l],
                                                                net->wb.as<__nv_bfloat162>() + net->off[l],
                                                                net->w[l], net->w[l + 1]);
    }
    op.prof.launches += 1 + net->nl;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int set_attrs() {
    static bool done = false;
    if (done) return DLZ_OK;
    const int wg = (int)((size_t)(2 * kMaxWidth * 4) * kLD * sizeof(float2));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_ptc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, wg));
    const int fw = 9 * 4 * kMaxWidth * 16 * (int)sizeof(__nv_bfloat162);
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_ptc_fwd<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, fw));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_ptc_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, fw));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_ptc_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, fw));
    done = true;
    return DLZ_OK;
}

bool device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace dlz

using namespace dlz;

extern "C" {

int dlz_net_create(dlz_op_t h, int nlayers, const int *widths, const void *weights, dlz_net_t *out) {
    if (!h || !widths || !weights || !out) return fail(DLZ_ERR_BADARG, "null argument");
    if (h->op.eo) return fail(DLZ_ERR_BADARG, "the network runs on full-lattice operators");
    if (nlayers < 1 || nlayers > kMaxLayersNet) return fail(DLZ_ERR_BADARG, "nlayers must be in [1, 8]");
    if (widths[0] != 1 || widths[nlayers] != 1) return fail(DLZ_ERR_BADARG, "first and last width must be 1");
    for (int l = 0; l <= nlayers; ++l)
        if (widths[l] < 1 || widths[l] > kMaxWidth) return fail(DLZ_ERR_BADARG, "widths must be in [1, 16]");
    *out = nullptr;
    DLZ_TRY(set_attrs());
    dlz_net_s *net = new dlz_net_s();
    net->op = &h->op;
    net->nl = nlayers;
    net->w.assign(widths, widths + nlayers + 1);
    size_t o = 0;
    for (int l = 0; l < nlayers; ++l) {
        net->off.push_back(o);
        o += (size_t)9 * widths[l] * widths[l + 1] * 16;
    }
    net->nw = o;
    Op &op = h->op;
    int rc = [&]() -> int {
        DLZ_TRY(net->master.alloc(o * sizeof(float2)));
        DLZ_TRY(net->grad.alloc(o * sizeof(float2)));
        DLZ_TRY(net->m1.alloc(o * sizeof(float2)));
        DLZ_TRY(net->m2.alloc(o * sizeof(float2)));
        DLZ_TRY(net->wb.alloc(o * sizeof(__nv_bfloat162)));
        DLZ_TRY(net->wadj.alloc(o * sizeof(__nv_bfloat162)));
        int maxp = 0;
        for (int l = 0; l < nlayers; ++l) maxp = std::max(maxp, 16 * widths[l] * widths[l + 1]);
        DLZ_TRY(net->partials.alloc((size_t)9 * kGradBlocks * maxp * sizeof(float2)));
        const void *src = weights;
        std::vector<float2> hw;
        if (!device_ptr(weights)) {
            hw.resize(o);
            std::memcpy(hw.data(), weights, o * sizeof(float2));
            src = hw.data();
        }
        DLZ_CUDA_TRY(cudaMemcpyAsync(net->master.p, src, o * sizeof(float2), cudaMemcpyDefault, op.stream));
        DLZ_CUDA_TRY(cudaMemsetAsync(net->grad.p, 0, o * sizeof(float2), op.stream));
        DLZ_CUDA_TRY(cudaMemsetAsync(net->m1.p, 0, o * sizeof(float2), op.stream));
        DLZ_CUDA_TRY(cudaMemsetAsync(net->m2.p, 0, o * sizeof(float2), op.stream));
        DLZ_TRY(refresh_bf16(net));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        return DLZ_OK;
    }();
    if (rc != DLZ_OK) {
        delete net;
        return rc;
    }
    *out = net;
    return DLZ_OK;
}

int dlz_net_destroy(dlz_net_t net) {
    delete net;
    return DLZ_OK;
}

int dlz_net_forward(dlz_net_t net, const void *in, int nvec, void *out) {
    if (!net || !in || !out || nvec < 1) return fail(DLZ_ERR_BADARG, "net_forward arguments");
    if (!device_ptr(in) || !device_ptr(out)) return fail(DLZ_ERR_BADARG, "net_forward takes device pointers");
    Op &op = *net->op;
    op.prof.begin(false, false);
    const size_t plane = (size_t)6 * op.g.V;      // float4 per channel
    if (net->act_nvec != nvec) {
        for (int l = 0; l <= net->nl; ++l)
            DLZ_TRY(net->act[l].alloc((size_t)nvec * net->w[l] * plane * sizeof(float4)));
        net->act_nvec = nvec;
    }
    const long n = 12L * op.g.V;
    for (int v = 0; v < nvec; ++v)
        DLZ_TRY(pack32(op, net->act[0].as<float4>() + (size_t)v * plane, (const float2 *)in + (size_t)v * n));
    for (int l = 0; l < net->nl; ++l)
        DLZ_TRY(layer_forward(op, net->act[l + 1].as<float4>(), net->act[l].as<float4>(),
                              net->wb.as<__nv_bfloat162>() + net->off[l], net->w[l], net->w[l + 1], nvec));
    for (int v = 0; v < nvec; ++v)
        DLZ_TRY(unpack32(op, (float2 *)out + (size_t)v * n, net->act[net->nl].as<float4>() + (size_t)v * plane));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_backward(dlz_net_t net, const void *grad_out, int nvec, void *grad_in) {
    if (!net || !grad_out || nvec < 1) return fail(DLZ_ERR_BADARG, "net_backward arguments");
    if (nvec != net->act_nvec) return fail(DLZ_ERR_BADARG, "net_backward needs a forward with the same nvec");
    if (!device_ptr(grad_out) || (grad_in && !device_ptr(grad_in)))
        return fail(DLZ_ERR_BADARG, "net_backward takes device pointers");
    Op &op = *net->op;
    op.prof.begin(false, false);
    const size_t plane = (size_t)6 * op.g.V;
    const long n = 12L * op.g.V;
    int maxw = 1;
    for (int l = 0; l <= net->nl; ++l) maxw = std::max(maxw, net->w[l]);
    for (int b = 0; b < 2; ++b)
        if (net->gbuf[b].bytes < (size_t)nvec * maxw * plane * sizeof(float4))
            DLZ_TRY(net->gbuf[b].alloc((size_t)nvec * maxw * plane * sizeof(float4)));
    float4 *gc = net->gbuf[0].as<float4>(), *gn = net->gbuf[1].as<float4>();
    for (int v = 0; v < nvec; ++v) DLZ_TRY(pack32(op, gc + (size_t)v * plane, (const float2 *)grad_out + (size_t)v * n));
    for (int l = net->nl - 1; l >= 0; --l) {
        const int cin = net->w[l], cout = net->w[l + 1];
        const size_t sm = (size_t)(cout * 4 + cin * 4) * kLD * sizeof(float2);
        k_ptc_wgrad<<<dim3(kGradBlocks, 9), 256, sm, op.stream>>>(net->partials.as<float2>(), gc,
                                                                 net->act[l].as<float4>(), op.gauge32.as<float4>(),
                                                                 op.g, cin, cout, nvec);
        const long ne = 9L * cin * cout * 16;
        k_ptc_wgrad_sum<<<blocks_for(ne, 256), 256, 0, op.stream>>>(net->grad.as<float2>() + net->off[l],
                                                                    net->partials.as<float2>(), kGradBlocks, cin, cout);
        op.prof.launches += 2;
        DLZ_CUDA_TRY(cudaGetLastError());
        if (l > 0 || grad_in) {
            DLZ_TRY(layer_forward(op, gn, gc, net->wadj.as<__nv_bfloat162>() + net->off[l], cout, cin, nvec));
            std::swap(gc, gn);
        }
    }
    if (grad_in)
        for (int v = 0; v < nvec; ++v) DLZ_TRY(unpack32(op, (float2 *)grad_in + (size_t)v * n, gc + (size_t)v * plane));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_get(dlz_net_t net, int what, void *host_out) {
    if (!net || !host_out || what < 0 || what > 2) return fail(DLZ_ERR_BADARG, "net_get arguments");
    Op &op = *net->op;
    if (what == 2) {
        std::vector<__nv_bfloat162> b(net->nw);
        DLZ_CUDA_TRY(cudaMemcpyAsync(b.data(), net->wb.p, net->nw * sizeof(__nv_bfloat162), cudaMemcpyDeviceToHost, op.stream));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        float2 *o = (float2 *)host_out;
        for (size_t i = 0; i < net->nw; ++i) o[i] = __bfloat1622float2(b[i]);
        return DLZ_OK;
    }
    const DevBuf &src = what == 0 ? net->master : net->grad;
    DLZ_CUDA_TRY(cudaMemcpyAsync(host_out, src.p, net->nw * sizeof(float2), cudaMemcpyDeviceToHost, op.stream));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_set_weights(dlz_net_t net, const void *weights) {
    if (!net || !weights) return fail(DLZ_ERR_BADARG, "net_set_weights arguments");
    Op &op = *net->op;
    DLZ_CUDA_TRY(cudaMemcpyAsync(net->master.p, weights, net->nw * sizeof(float2), cudaMemcpyDefault, op.stream));
    DLZ_TRY(refresh_bf16(net));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_zero_grad(dlz_net_t net) {
    if (!net) return fail(DLZ_ERR_BADARG, "null network");
    Op &op = *net->op;
    DLZ_CUDA_TRY(cudaMemsetAsync(net->grad.p, 0, net->nw * sizeof(float2), op.stream));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_adam_step(dlz_net_t net, double lr, double beta1, double beta2, double eps) {
    if (!net || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return fail(DLZ_ERR_BADARG, "adam arguments");
    Op &op = *net->op;
    net->adam_t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(beta1, net->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(beta2, net->adam_t)));
    k_ptc_adam<<<blocks_for((long)net->nw, 256), 256, 0, op.stream>>>(
        net->master.as<float2>(), net->grad.as<float2>(), net->m1.as<float2>(), net->m2.as<float2>(),
        (long)net->nw, (float)lr, (float)beta1, (float)beta2, (float)eps, c1, c2);
    DLZ_CUDA_TRY(cudaGetLastError());
    DLZ_TRY(refresh_bf16(net));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_net_bind(dlz_net_t net, dlz_op_t h) {
    if (!net || !h) return fail(DLZ_ERR_BADARG, "null argument");
    const Geom &a = net->op->g, &b = h->op.g;
    for (int d = 0; d < 4; ++d)
        if (a.L[d] != b.L[d]) return fail(DLZ_ERR_BADARG, "net_bind needs an operator on the same lattice");
    DLZ_CUDA_TRY(cudaStreamSynchronize(net->op->stream));
    net->op = &h->op;
    return DLZ_OK;
}

int dlz_net_weight_count(dlz_net_t net, long long *count) {
    if (!net || !count) return fail(DLZ_ERR_BADARG, "null argument");
    *count = (long long)net->nw;
    return DLZ_OK;
}

int dlz_subspace_loss(dlz_defl_t d, const void *f, int nvec, double grad_scale, double *loss, void *grad) {
    if (!d || !f || !loss || nvec < 1) return fail(DLZ_ERR_BADARG, "subspace_loss arguments");
    if (!std::isfinite(grad_scale)) return fail(DLZ_ERR_BADARG, "grad_scale is not finite");
    if (!device_ptr(f) || (grad && !device_ptr(grad))) return fail(DLZ_ERR_BADARG, "subspace_loss takes device pointers");
    Op &op = *d->op;
    op.prof.begin(false, false);
    const long n = 12L * op.g.V;
    const int k = d->k;
    DevBuf f32, f64, perp, dots, nrm;
    DLZ_TRY(f32.alloc(n * sizeof(float2)));
    DLZ_TRY(f64.alloc(n * sizeof(double2)));
    DLZ_TRY(perp.alloc(n * sizeof(double2)));
    DLZ_TRY(dots.alloc((size_t)std::max(k, 1) * sizeof(double2)));
    DLZ_TRY(nrm.alloc(2 * sizeof(double)));
    double *dn = nrm.as<double>();
    for (int v = 0; v < nvec; ++v) {
        DLZ_TRY(pack32(op, f32.as<float4>(), (const float2 *)f + (size_t)v * n));
        DLZ_TRY(convert32to64(op, f64.as<double2>(), f32.as<float4>()));
        DLZ_TRY(v64::copy(op, perp.as<double2>(), f64.as<double2>()));
        if (k > 0) {
            // perp = f - V (V^dag f)
            DLZ_TRY(v64::multidot(op, d->V64.as<double2>(), n, k, f64.as<double2>(), dots.as<double2>(), -1.0));
            DLZ_TRY(combine64(op, perp.as<double2>(), n, 1, d->V64.as<double2>(), n, k, dots.p, 1, false, true));
        }
        DLZ_TRY(v64::norm2_diff(op, f64.as<double2>(), nullptr, dn));
        DLZ_TRY(v64::norm2_diff(op, perp.as<double2>(), nullptr, dn + 1));
        double h[2];
        DLZ_TRY(d2h_sync(op, h, dn, 2 * sizeof(double)));
        if (!(h[0] > 0)) return fail(DLZ_ERR_NONFINITE, "network output is zero or not finite");
        const double L = h[1] / h[0];
        loss[v] = L;
        if (grad) {
            // G(f) = grad_scale * 2 (perp - L f) / ||f||^2
            const double a = grad_scale * 2.0 / h[0], b = -grad_scale * 2.0 * L / h[0];
            double2 *pp = perp.as<double2>();
            const double2 *ff = f64.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double2 p = pp[i], q = ff[i];
                pp[i] = make_double2(a * p.x + b * q.x, a * p.y + b * q.y);
            }));
            DLZ_TRY(convert64to32(op, f32.as<float4>(), perp.as<double2>()));
            DLZ_TRY(unpack32(op, (float2 *)grad + (size_t)v * n, f32.as<float4>()));
        }
    }
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_seed_deflation(dlz_op_t h, int which, const void *vecs, int dtype, int k, dlz_defl_t *out) {
    if (!h || !vecs || !out || k < 1) return fail(DLZ_ERR_BADARG, "seed_deflation arguments");
    if (which != DLZ_Q && which != DLZ_DDAGD) return fail(DLZ_ERR_BADARG, "which must be DLZ_Q or DLZ_DDAGD");
    if (dtype != DLZ_F64 && dtype != DLZ_F32) return fail(DLZ_ERR_BADARG, "dtype");
    if (!device_ptr(vecs)) return fail(DLZ_ERR_BADARG, "seed_deflation takes device pointers");
    *out = nullptr;
    Op &op = h->op;
    op.prof.begin(false, false);
    const long n = 12L * op.g.V;
    DevBuf Q, t32, dots, nrm;
    DLZ_TRY(Q.alloc((size_t)k * n * sizeof(double2)));
    DLZ_TRY(t32.alloc(n * sizeof(float2)));
    DLZ_TRY(dots.alloc((size_t)k * sizeof(double2)));
    DLZ_TRY(nrm.alloc(sizeof(double)));
    double2 *Qp = Q.as<double2>();
    for (int j = 0; j < k; ++j) {
        double2 *qj = Qp + (size_t)j * n;
        if (dtype == DLZ_F64) DLZ_TRY(pack64(op, qj, (const double2 *)vecs + (size_t)j * n));
        else {
            DLZ_TRY(pack32(op, t32.as<float4>(), (const float2 *)vecs + (size_t)j * n));
            DLZ_TRY(convert32to64(op, qj, t32.as<float4>()));
        }
        // modified Gram-Schmidt against the accepted columns, twice, then normalise
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            DLZ_TRY(v64::multidot(op, Qp, n, j, qj, dots.as<double2>(), -1.0));
            DLZ_TRY(combine64(op, qj, n, 1, Qp, n, j, dots.p, 1, false, true));
        }
        DLZ_TRY(v64::norm2_diff(op, qj, nullptr, nrm.as<double>()));
        double nn;
        DLZ_TRY(d2h_sync(op, &nn, nrm.p, sizeof(double)));
        if (!(nn > 0) || !std::isfinite(nn)) return fail(DLZ_ERR_BREAKDOWN, "seed vectors are linearly dependent");
        const double sc = 1.0 / std::sqrt(nn);
        DLZ_TRY(map(op, n, [=] __device__(long i) { qj[i].x *= sc; qj[i].y *= sc; }));
    }
    dlz_defl_s *d = nullptr;
    DLZ_TRY(build_deflation(op, which, Qp, k, &d, nullptr));
    *out = d;
    return DLZ_OK;
}

}  // extern "C"
