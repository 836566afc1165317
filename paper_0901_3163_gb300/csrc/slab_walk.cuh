// Block order of the batched stencil kernels: z-slabs along t.
//
// A stencil kernel over N right-hand sides runs one block per (site block, right-hand
// side), right-hand side fastest, so each block's neighbour gathers hit data that other
// blocks brought into L2.  In the plain site order (x fastest, t slowest) a t-neighbour
// lies one whole 3-D slice away.  With 16 right-hand sides on 24^3 x 48 the traffic of a
// slice (~13824 sites x 16 x ~900 bytes for the fused CGNR kernels) is larger than L2, so
// those gathers go to DRAM a second time.
//
// The walk here takes slabs of bz z-planes at one t, each a contiguous range of
// bz * plane sites: the slabs of z-slab 0 for t = 0 .. Lt-1, then those of z-slab 1, and so
// on.  A t-neighbour is then one slab behind or ahead of the block that gathers it.  The
// price is the z-neighbours across a slab edge (2 of bz planes), which come from DRAM
// again.  bz = Lz is the plain order.
//
// `plane` counts the sites of one (x, y) plane of the field: Lx Ly for a full lattice,
// Lx Ly / 2 for one parity of an even-odd field (its checkerboard index s >> 1 keeps the
// planes contiguous).
#pragma once

#include <algorithm>
#include <cstdlib>

namespace dlz {

constexpr int kSlabBlock = 128;     // sites per block

struct SlabWalk {
    int bz;          // z-planes per slab
    int bps;         // blocks per slab
    int plane;       // sites per plane
    int Lz, Lt;
};

// first site s0 and site count nb of site block sb (nb = 0 for the spare blocks of a
// short last z-slab)
__host__ __device__ inline void slab_block(const SlabWalk &w, int sb, int &s0, int &nb) {
    const int j = sb / w.bps, off = (sb % w.bps) * kSlabBlock;
    const int t = j % w.Lt, z0 = (j / w.Lt) * w.bz;
    const int planes = w.bz < w.Lz - z0 ? w.bz : w.Lz - z0;
    const int len = planes * w.plane;
    s0 = (t * w.Lz + z0) * w.plane + off;
    const int rest = len - off;
    nb = rest <= 0 ? 0 : (rest < kSlabBlock ? rest : kSlabBlock);
}

// The walk with slabs of bz planes
inline SlabWalk slab_walk_of(int plane, int Lz, int Lt, int bz) {
    SlabWalk w;
    w.plane = plane;
    w.Lz = Lz;
    w.Lt = Lt;
    w.bz = std::max(1, std::min(bz, Lz));
    w.bps = (w.bz * plane + kSlabBlock - 1) / kSlabBlock;
    return w;
}

// The walk for N right-hand sides moving about `bytes` per site and right-hand side: the
// plain order when a slab's traffic fits in 36 MB, else the largest divisor of Lz whose
// slab does (at least one plane).  On 24^3 x 48 with 16 right-hand sides that is 4 planes
// for the fused CGNR kernels, which took 1.54 / 1.05 ms (K23 / K1) per launch against
// 1.88 / 1.20 ms in the plain order (3: 1.54 / 1.07; 6: 1.70 / 1.06; 2: 1.64 / 1.18).
// DLZ_SLAB=n fixes n planes.
inline SlabWalk make_slab_walk(int plane, int Lz, int Lt, int N, double bytes) {
    const double per_plane = (double)plane * N * bytes;
    int bmax = per_plane > 0.0 ? (int)std::min((double)Lz, 36.0e6 / per_plane) : Lz;
    int bz = 1;
    for (int d = 1; d <= std::max(1, bmax); ++d)
        if (Lz % d == 0) bz = d;
    if (const char *env = std::getenv("DLZ_SLAB")) {
        const int v = std::atoi(env);
        if (v > 0) bz = v;
    }
    return slab_walk_of(plane, Lz, Lt, bz);
}

// blocks per right-hand side
inline long slab_blocks(const SlabWalk &w) { return (long)w.bps * w.Lt * ((w.Lz + w.bz - 1) / w.bz); }

}  // namespace dlz
