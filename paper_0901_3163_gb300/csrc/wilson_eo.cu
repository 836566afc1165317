// Even-odd (Schur complement) Wilson operator on the even sites -- not in the
// paper: the standard reduction of D x = b (the Wilson matrix M of
// arXiv:0901.3163, Sec. 2) to Dhat x_e = b_e + kappa H_eo b_o with
// Dhat = 1 - kappa^2 H_eo H_oe, to which Lan-DR / MinRes-DR and D-CG / D-MinRes
// apply unchanged; x_o = b_o + kappa H_oe x_e afterwards.
//
// Fields of one parity use the plane layout of full fields with stride Vh = V / 2,
// indexed by the checkerboard index cb = s >> 1 (wilson_eo_site.cuh).  Each
// application of Dhat is two launches: the odd field t = H_oe [gamma5] x (one
// thread per odd site), then the Schur step at the even sites
// [gamma5] ([gamma5] x - kappa^2 H_eo t); Dhat^dag = gamma5 Dhat gamma5 and
// Qhat = gamma5 Dhat take the gamma5 variants of the same two kernels.
#include "dlz_internal.cuh"
#include "slab_walk.cuh"
#include "wilson_eo_site.cuh"

namespace dlz {

namespace {

constexpr int kEoThreads = kSlabBlock;

// The walk over one parity's sites for a kernel moving `bytes` per site and right-hand
// side: slab_walk.cuh in FP32, the plain order in FP64 (FP64-ALU-bound kernels)
SlabWalk eo_walk(const Geom &gf, int nrhs, double bytes, bool f32) {
    const int plane = gf.L[0] * gf.L[1] / 2;
    return f32 ? make_slab_walk(plane, gf.L[2], gf.L[3], nrhs, bytes) : slab_walk_of(plane, gf.L[2], gf.L[3], gf.L[2]);
}

// out (parity par) = H [gamma5]^G5IN in (parity 1 - par), nrhs fields; RHS fastest in
// blockIdx so that blocks of the same sites share their links in L2
template <typename T, bool G5IN>
__global__ void __launch_bounds__(kEoThreads)
k_eo_hop(typename Field<T>::vec *__restrict__ out, const typename Field<T>::vec *__restrict__ in,
         const typename Link<T>::vec *__restrict__ U, Geom gf, SlabWalk w, int par, int nrhs, long nel) {
    const int r = blockIdx.x % nrhs;
    int c0, nb;
    slab_block(w, blockIdx.x / nrhs, c0, nb);
    if ((int)threadIdx.x >= nb) return;
    const int cb = c0 + threadIdx.x;
    cx<T> acc[12];
    wilson_eo_hop_site<T, G5IN>(cb, par, gf, in + (size_t)r * nel, U, acc);
    Field<T>::store(out + (size_t)r * nel, gf.V >> 1, cb, acc);
}

// out = [gamma5]^G5OUT ([gamma5]^G5X x - kappa2 H_eo t) at the even sites
template <typename T, bool G5X, bool G5OUT>
__global__ void __launch_bounds__(kEoThreads)
k_eo_schur(typename Field<T>::vec *__restrict__ out, const typename Field<T>::vec *__restrict__ x,
           const typename Field<T>::vec *__restrict__ t, const typename Link<T>::vec *__restrict__ U, Geom gf,
           SlabWalk w, T kappa2, int nrhs, long nel) {
    const int r = blockIdx.x % nrhs;
    int c0, nb;
    slab_block(w, blockIdx.x / nrhs, c0, nb);
    if ((int)threadIdx.x >= nb) return;
    const int cb = c0 + threadIdx.x;
    cx<T> o[12];
    wilson_eo_schur_site<T, G5X, G5OUT>(cb, gf, kappa2, x + (size_t)r * nel, t + (size_t)r * nel, U, o);
    Field<T>::store(out + (size_t)r * nel, gf.V >> 1, cb, o);
}

// user layout complex128 [V][12] (full lattice) <-> even and odd internal planes [12][Vh]
__global__ void k_eo_split_user(double2 *__restrict__ ev, double2 *__restrict__ od, const double2 *__restrict__ full,
                                Geom gf) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;    // s * 12 + a
    if (i >= 12L * gf.V) return;
    const int s = (int)(i / 12), a = (int)(i % 12);
    int r = s;
    const int x = r % gf.L[0]; r /= gf.L[0];
    const int y = r % gf.L[1]; r /= gf.L[1];
    const int z = r % gf.L[2];
    const int t = r / gf.L[2];
    const size_t j = (size_t)a * (gf.V >> 1) + (s >> 1);
    if (((x + y + z + t) & 1) == 0) ev[j] = full[i];
    else od[j] = full[i];
}
__global__ void k_eo_join_user(double2 *__restrict__ full, const double2 *__restrict__ ev,
                               const double2 *__restrict__ od, Geom gf) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 12L * gf.V) return;
    const int s = (int)(i / 12), a = (int)(i % 12);
    int r = s;
    const int x = r % gf.L[0]; r /= gf.L[0];
    const int y = r % gf.L[1]; r /= gf.L[1];
    const int z = r % gf.L[2];
    const int t = r / gf.L[2];
    const size_t j = (size_t)a * (gf.V >> 1) + (s >> 1);
    full[i] = (((x + y + z + t) & 1) == 0) ? ev[j] : od[j];
}
// y = x + c h (one parity, internal planes)
__global__ void k_eo_axpy(double2 *__restrict__ y, const double2 *__restrict__ x, const double2 *__restrict__ h,
                          double c, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 a = x[i], b = h[i];
    y[i] = make_double2(a.x + c * b.x, a.y + c * b.y);
}

template <typename T>
int eo_apply_t(Op &op, typename Field<T>::vec *out, const typename Field<T>::vec *in, int which, int nrhs,
               typename Field<T>::vec *tmp, const typename Link<T>::vec *U) {
    if (!op.eo) return fail(DLZ_ERR_BADARG, "not an even-odd operator");
    const Geom gf = op.gf;
    const long nel = (long)Field<T>::vec_per_site * (gf.V >> 1);
    const T kappa2 = (T)(op.kappa * op.kappa);
    for (int r0 = 0; r0 < nrhs; r0 += kEoBatch) {
        const int nb = nrhs - r0 < kEoBatch ? nrhs - r0 : kEoBatch;
        const SlabWalk wh = eo_walk(gf, nb, 200.0, sizeof(T) == 4), ws = eo_walk(gf, nb, 300.0, sizeof(T) == 4);
        const unsigned bh = (unsigned)(slab_blocks(wh) * nb), bs = (unsigned)(slab_blocks(ws) * nb);
        const typename Field<T>::vec *x = in + (size_t)r0 * nel;
        typename Field<T>::vec *o = out + (size_t)r0 * nel;
        const bool g5 = which == DLZ_DDAG;
        // per even site and RHS: the hop reads 24 reals (x at the even neighbours, once
        // from DRAM) and writes 24; the Schur step reads 24 (t) + 24 (x) and writes 24.
        // Each of the two passes reads every link once: 2 x 4 links per full site, i.e.
        // 4 x 48 (FP32, two rows) or 4 x 72 (FP64) reals per even site
        op.prof.stencil_start(op.stream, sizeof(T) == 4, gf.V >> 1, nb, 120, 0, sizeof(T) == 4 ? 192 : 288);
        if (g5) k_eo_hop<T, true><<<bh, kEoThreads, 0, op.stream>>>(tmp, x, U, gf, wh, 1, nb, nel);
        else k_eo_hop<T, false><<<bh, kEoThreads, 0, op.stream>>>(tmp, x, U, gf, wh, 1, nb, nel);
        switch (which) {
        case DLZ_D: k_eo_schur<T, false, false><<<bs, kEoThreads, 0, op.stream>>>(o, x, tmp, U, gf, ws, kappa2, nb, nel); break;
        case DLZ_DDAG: k_eo_schur<T, true, true><<<bs, kEoThreads, 0, op.stream>>>(o, x, tmp, U, gf, ws, kappa2, nb, nel); break;
        case DLZ_Q: k_eo_schur<T, false, true><<<bs, kEoThreads, 0, op.stream>>>(o, x, tmp, U, gf, ws, kappa2, nb, nel); break;
        default: return fail(DLZ_ERR_BADARG, "even-odd stencil: which must be D, DDAG or Q");
        }
        op.prof.stencil_stop(op.stream);
        op.prof.launches += 2;
        DLZ_CUDA_TRY(cudaGetLastError());
    }
    return DLZ_OK;
}

}  // namespace

int eo_apply64(Op &op, double2 *out, const double2 *in, int which, int nrhs) {
    return eo_apply_t<double>(op, out, in, which, nrhs, op.eo_tmp64.as<double2>(), op.gauge64.as<double2>());
}
int eo_apply32(Op &op, float4 *out, const float4 *in, int which, int nrhs) {
    return eo_apply_t<float>(op, out, in, which, nrhs, op.eo_tmp32.as<float4>(), op.gauge32.as<float4>());
}

int eo_hop64(Op &op, double2 *out, const double2 *in, int par, bool g5in, int nrhs) {
    const Geom gf = op.gf;
    const long nel = 12L * (gf.V >> 1);
    const SlabWalk w = eo_walk(gf, nrhs, 200.0, false);
    const unsigned blocks = (unsigned)(slab_blocks(w) * nrhs);
    if (g5in) k_eo_hop<double, true><<<blocks, kEoThreads, 0, op.stream>>>(out, in, op.gauge64.as<double2>(), gf, w, par, nrhs, nel);
    else k_eo_hop<double, false><<<blocks, kEoThreads, 0, op.stream>>>(out, in, op.gauge64.as<double2>(), gf, w, par, nrhs, nel);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int eo_hop32(Op &op, float4 *out, const float4 *in, int par, bool g5in, int nrhs) {
    const Geom gf = op.gf;
    const long nel = 6L * (gf.V >> 1);
    const SlabWalk w = eo_walk(gf, nrhs, 200.0, true);
    const unsigned blocks = (unsigned)(slab_blocks(w) * nrhs);
    if (g5in) k_eo_hop<float, true><<<blocks, kEoThreads, 0, op.stream>>>(out, in, op.gauge32.as<float4>(), gf, w, par, nrhs, nel);
    else k_eo_hop<float, false><<<blocks, kEoThreads, 0, op.stream>>>(out, in, op.gauge32.as<float4>(), gf, w, par, nrhs, nel);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int eo_prepare64(Op &op, double2 *be, double2 *bo, const double2 *b_user) {
    // be = b_e + kappa H_eo b_o (bo receives b_o; the hop result goes through the work field)
    const Geom gf = op.gf;
    const long nf = 12L * gf.V, nh = 12L * (gf.V >> 1);
    k_eo_split_user<<<(int)((nf + 255) / 256), 256, 0, op.stream>>>(be, bo, b_user, gf);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    double2 *h = op.eo_tmp64.as<double2>();
    DLZ_TRY(eo_hop64(op, h, bo, 0, false, 1));
    k_eo_axpy<<<(int)((nh + 255) / 256), 256, 0, op.stream>>>(be, be, h, op.kappa, nh);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

int eo_reconstruct64(Op &op, double2 *x_user, const double2 *xe, double2 *bo_work, const double2 *b_user) {
    // x_o = b_o + kappa H_oe x_e; x = (x_e, x_o) in the user layout
    const Geom gf = op.gf;
    const long nf = 12L * gf.V, nh = 12L * (gf.V >> 1);
    double2 *h = op.eo_tmp64.as<double2>();
    // split b into (h: even part, unused) and bo_work (odd part)
    k_eo_split_user<<<(int)((nf + 255) / 256), 256, 0, op.stream>>>(h, bo_work, b_user, gf);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    DLZ_TRY(eo_hop64(op, h, xe, 1, false, 1));
    k_eo_axpy<<<(int)((nh + 255) / 256), 256, 0, op.stream>>>(bo_work, bo_work, h, op.kappa, nh);
    k_eo_join_user<<<(int)((nf + 255) / 256), 256, 0, op.stream>>>(x_user, xe, bo_work, gf);
    op.prof.launches += 2;
    DLZ_CUDA_TRY(cudaGetLastError());
    return DLZ_OK;
}

}  // namespace dlz
