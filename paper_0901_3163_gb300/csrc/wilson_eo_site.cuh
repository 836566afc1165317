// Even-odd (checkerboard) form of the Wilson hopping term -- not in the paper: the
// Schur complement Dhat = 1 - kappa^2 H_eo H_oe of the Wilson matrix (M of
// arXiv:0901.3163, Sec. 2) on the even sites, to which the deflated solvers apply
// unchanged (x_o = b_o + kappa H_oe x_e afterwards).
//
// Parity of a site: (x + y + z + t) mod 2, every extent even.  With x fastest and Lx
// even, the sites 2j and 2j+1 of a row have opposite parity, so the checkerboard
// index of site s is cb = s >> 1 in either parity.  A one-parity field uses the FP64
// / FP32 plane layout of the full field with stride Vh = V / 2, indexed by cb; the
// links stay full-lattice.  The hop itself is the spin-projected one of
// wilson_site.cuh.
#pragma once

#include "wilson_site.cuh"

namespace dlz {

// Full coordinates c and index of the site with checkerboard index cb and parity par.
__host__ __device__ inline int eo_site(int cb, int par, const Geom &g, int (&c)[4]) {
    const int lxh = g.L[0] >> 1;
    int r = cb / lxh;
    const int xh = cb - r * lxh;
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
    return ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

// Forward and backward hops in direction MU from full site s (coordinates c), reading
// a field of the other parity at the neighbours' checkerboard indices.
template <typename T, int MU, bool G5IN>
__host__ __device__ inline void hop_pair_eo(int s, const int (&c)[4], const Geom &g, int stride,
                                            const typename Field<T>::vec *__restrict__ in,
                                            const typename Link<T>::vec *__restrict__ U, cx<T> (&acc)[12]) {
    const int L = g.L[MU];
    const int Vh = g.V >> 1;
    const int sf = (c[MU] == L - 1) ? s - (L - 1) * stride : s + stride;
    const T phf = (MU == 3 && c[3] == L - 1) ? (T)g.bc_t : (T)1;
    const int sb = (c[MU] == 0) ? s + (L - 1) * stride : s - stride;
    const T phb = (MU == 3 && c[3] == 0) ? (T)g.bc_t : (T)1;
    cx<T> p[12], u[9];
    Field<T>::load(in, Vh, sf >> 1, p);
    maybe_g5<G5IN>(p);
    load_link<T>(U, g.V, MU, s, u);
    hop_fwd<T, MU>(p, u, phf, acc);
    Field<T>::load(in, Vh, sb >> 1, p);
    maybe_g5<G5IN>(p);
    load_link<T>(U, g.V, MU, sb, u);
    hop_bwd<T, MU>(p, u, phb, acc);
}

// acc = (H [gamma5]^G5IN in) at the site (cb, par), `in` a field of parity 1 - par
// (the hopping term only): H_oe in for par = 1, H_eo in for par = 0.
template <typename T, bool G5IN>
__host__ __device__ inline void wilson_eo_hop_site(int cb, int par, const Geom &g,
                                                   const typename Field<T>::vec *__restrict__ in,
                                                   const typename Link<T>::vec *__restrict__ U,
                                                   cx<T> (&acc)[12]) {
    int c[4];
    const int s = eo_site(cb, par, g, c);
    const int st1 = g.L[0], st2 = g.L[0] * g.L[1], st3 = st2 * g.L[2];
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = mk<T>(0, 0);
    hop_pair_eo<T, 0, G5IN>(s, c, g, 1, in, U, acc);
    hop_pair_eo<T, 1, G5IN>(s, c, g, st1, in, U, acc);
    hop_pair_eo<T, 2, G5IN>(s, c, g, st2, in, U, acc);
    hop_pair_eo<T, 3, G5IN>(s, c, g, st3, in, U, acc);
}

// Second half of Dhat at even site cb: out = [gamma5]^G5OUT ([gamma5]^G5X x - kappa2 H_eo t),
// t = H_oe [gamma5]^G5X x from the first half (an odd field).  G5X = G5OUT = true gives
// Dhat^dagger = gamma5 Dhat gamma5; G5X = false, G5OUT = true gives Qhat = gamma5 Dhat.
template <typename T, bool G5X, bool G5OUT>
__host__ __device__ inline void wilson_eo_schur_site(int cb, const Geom &g, T kappa2,
                                                     const typename Field<T>::vec *__restrict__ x,
                                                     const typename Field<T>::vec *__restrict__ t,
                                                     const typename Link<T>::vec *__restrict__ U,
                                                     cx<T> (&out)[12]) {
    cx<T> acc[12];
    wilson_eo_hop_site<T, false>(cb, 0, g, t, U, acc);
    Field<T>::load(x, g.V >> 1, cb, out);
    maybe_g5<G5X>(out);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        out[a].x = out[a].x - kappa2 * acc[a].x;
        out[a].y = out[a].y - kappa2 * acc[a].y;
    }
    maybe_g5<G5OUT>(out);
}

}  // namespace dlz
