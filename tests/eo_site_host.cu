// Host build of the even-odd site functions (paper_0901_3163_gb300/csrc/wilson_eo_site.cuh)
// for tests/test_eo_site_host.py: the same __host__ __device__ code the kernels will
// run, executed site by site on the CPU.  Fields in the library's plane layout.
#include "wilson_eo_site.cuh"

using namespace dlz;

namespace {

template <typename T>
void hop_all(int par, const int *dims, int bc_t, const typename Field<T>::vec *in,
             const typename Link<T>::vec *U, typename Field<T>::vec *out) {
    Geom g{{dims[0], dims[1], dims[2], dims[3]}, dims[0] * dims[1] * dims[2] * dims[3], bc_t};
    const int Vh = g.V >> 1;
    for (int cb = 0; cb < Vh; ++cb) {
        cx<T> acc[12];
        wilson_eo_hop_site<T, false>(cb, par, g, in, U, acc);
        Field<T>::store(out, Vh, cb, acc);
    }
}

// which: 0 Dhat, 1 Dhat^dagger, 2 Qhat
template <typename T>
void dhat_all(int which, const int *dims, int bc_t, T kappa, const typename Field<T>::vec *x,
              const typename Link<T>::vec *U, typename Field<T>::vec *t, typename Field<T>::vec *out) {
    Geom g{{dims[0], dims[1], dims[2], dims[3]}, dims[0] * dims[1] * dims[2] * dims[3], bc_t};
    const int Vh = g.V >> 1;
    const bool g5x = which == 1;
    for (int cb = 0; cb < Vh; ++cb) {
        cx<T> acc[12];
        if (g5x) wilson_eo_hop_site<T, true>(cb, 1, g, x, U, acc);
        else wilson_eo_hop_site<T, false>(cb, 1, g, x, U, acc);
        Field<T>::store(t, Vh, cb, acc);
    }
    for (int cb = 0; cb < Vh; ++cb) {
        cx<T> o[12];
        if (which == 0) wilson_eo_schur_site<T, false, false>(cb, g, kappa * kappa, x, t, U, o);
        else if (which == 1) wilson_eo_schur_site<T, true, true>(cb, g, kappa * kappa, x, t, U, o);
        else wilson_eo_schur_site<T, false, true>(cb, g, kappa * kappa, x, t, U, o);
        Field<T>::store(out, Vh, cb, o);
    }
}

}  // namespace

extern "C" {
void eo_hop_f64(int par, const int *dims, int bc_t, const double2 *in, const double2 *U, double2 *out) {
    hop_all<double>(par, dims, bc_t, in, U, out);
}
void eo_hop_f32(int par, const int *dims, int bc_t, const float4 *in, const float4 *U, float4 *out) {
    hop_all<float>(par, dims, bc_t, in, U, out);
}
void eo_dhat_f64(int which, const int *dims, int bc_t, double kappa, const double2 *x, const double2 *U,
                 double2 *t, double2 *out) {
    dhat_all<double>(which, dims, bc_t, kappa, x, U, t, out);
}
void eo_dhat_f32(int which, const int *dims, int bc_t, float kappa, const float4 *x, const float4 *U,
                 float4 *t, float4 *out) {
    dhat_all<float>(which, dims, bc_t, kappa, x, U, t, out);
}
}
