// Shared helpers of the solver drivers of Sec. 1-2: FP64 vector kernels on
// internal planes, pinned host scratch and stream-ordered copies.
#pragma once

#include <algorithm>

#include "dlz_internal.cuh"
#include "reduce.cuh"

namespace dlz {

// ------------------------------------------------------------------ vector helpers (FP64)
namespace v64 {

inline long nel(const Op &op) { return 12L * op.g.V; }

inline int copy(Op &op, double2 *dst, const double2 *src) {
    DLZ_CUDA_TRY(cudaMemcpyAsync(dst, src, nel(op) * sizeof(double2), cudaMemcpyDeviceToDevice, op.stream));
    return DLZ_OK;
}
inline int zero(Op &op, double2 *dst) {
    DLZ_CUDA_TRY(cudaMemsetAsync(dst, 0, nel(op) * sizeof(double2), op.stream));
    return DLZ_OK;
}
// gamma5 on internal planes: components 6..11 (spins 2, 3) change sign
inline int gamma5(Op &op, double2 *dst, const double2 *src) {
    const long half = 6L * op.g.V;
    return map(op, nel(op), [=] __device__(long i) {
        double2 v = src[i];
        if (i >= half) { v.x = -v.x; v.y = -v.y; }
        dst[i] = v;
    });
}
// result[slot] = ||a - b||^2 (b may be null: ||a||^2), copied to *host_out after sync
inline int norm2_diff(Op &op, const double2 *a, const double2 *b, double *dev_out) {
    return reduce<1>(op, nel(op), [=] __device__(long i, double (&acc)[1]) {
        double2 v = a[i];
        if (b) { const double2 w = b[i]; v.x -= w.x; v.y -= w.y; }
        acc[0] += v.x * v.x + v.y * v.y;
    }, [=] __device__(const double *r) { if (dev_out) *dev_out = r[0]; });
}
// out[l] (complex) = <V_l, w>  for l < nv, V_l = V + l*ld ; dev_out gets scale * dots
inline int multidot(Op &op, const double2 *V, long ld, int nv, const double2 *w, double2 *dev_out, double scale) {
    const long n = nel(op);
    for (int l0 = 0; l0 < nv; l0 += 8) {
        const int nb = std::min(8, nv - l0);
        const double2 *Vb = V + (size_t)l0 * ld;
        double2 *o = dev_out + l0;
        DLZ_TRY(reduce<16>(op, n, [=] __device__(long i, double (&acc)[16]) {
            const double2 x = w[i];
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                if (l < nb) {
                    const double2 v = Vb[(size_t)l * ld + i];
                    acc[2 * l] += v.x * x.x + v.y * x.y;        // Re conj(v) x
                    acc[2 * l + 1] += v.x * x.y - v.y * x.x;    // Im conj(v) x
                }
            }
        }, [=] __device__(const double *r) {
            for (int l = 0; l < nb; ++l) o[l] = make_double2(scale * r[2 * l], scale * r[2 * l + 1]);
        }));
    }
    return DLZ_OK;
}

}  // namespace v64

// combine: out_l = (acc ? out_l : 0) + sum_j C[j][l] in_j   (nout any, in groups of 16)
inline int combine64(Op &op, double2 *out, long ld_out, int nout, const double2 *in, long ld_in, int nin,
              const void *dev_coef, int ld_coef, bool real, bool acc) {
    const long n = 12L * op.g.V;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_combine64<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine64<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine64<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_combine64<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    if (nin <= 0 || nout <= 0) return DLZ_OK;
    long blocks = (n + 127) / 128;
    blocks = std::min(blocks, 152L * 8);
    for (int l0 = 0; l0 < nout; l0 += 16) {
        const int nb = std::min(16, nout - l0);
        if (nb == 1) {
            const size_t sm = (size_t)nin * 1 * sizeof(double2);
            if (real) k_combine64<true, 1><<<(int)blocks, 128, sm, op.stream>>>(out + (size_t)l0 * ld_out, ld_out, 1, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
            else k_combine64<false, 1><<<(int)blocks, 128, sm, op.stream>>>(out + (size_t)l0 * ld_out, ld_out, 1, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
        } else {
            const size_t sm = (size_t)nin * 16 * sizeof(double2);
            if (real) k_combine64<true, 16><<<(int)blocks, 128, sm, op.stream>>>(out + (size_t)l0 * ld_out, ld_out, nb, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
            else k_combine64<false, 16><<<(int)blocks, 128, sm, op.stream>>>(out + (size_t)l0 * ld_out, ld_out, nb, in, ld_in, nin, dev_coef, ld_coef, l0, acc, n);
        }
        op.prof.launches++;
        DLZ_CUDA_TRY(cudaGetLastError());
    }
    return DLZ_OK;
}

// ------------------------------------------------------------------ small pinned scalar block
struct HostScratch {
    double *p = nullptr;
    size_t n = 0;
    int ensure(size_t count) {
        if (count <= n) return DLZ_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        DLZ_CUDA_TRY(cudaMallocHost(&p, count * sizeof(double)));
        n = count;
        return DLZ_OK;
    }
    ~HostScratch() { if (p) cudaFreeHost(p); }
};

inline int d2h_sync(Op &op, void *dst, const void *src, size_t bytes) {
    DLZ_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, op.stream));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}
inline int h2d(Op &op, void *dst, const void *src, size_t bytes) {
    DLZ_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, op.stream));
    return DLZ_OK;
}

int project64(Op &op, const struct dlz_defl_s *d, const double2 *b, double2 *x0, DevBuf &dots);

}  // namespace dlz
