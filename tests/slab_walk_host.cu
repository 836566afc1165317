// Host build of the block walk of the batched FP32 stencils (csrc/slab_walk.cuh) for
// tests/test_slab_walk_host.py: the walk the library would choose, and the first site and
// site count of every block.
#include <cstdint>

#include "slab_walk.cuh"

extern "C" {

// the chosen walk: out[0] = z-planes per slab, out[1] = blocks per slab, out[2] = blocks
int slab_choice(int plane, int Lz, int Lt, int nrhs, double bytes, long long *out) {
    const dlz::SlabWalk w = dlz::make_slab_walk(plane, Lz, Lt, nrhs, bytes);
    out[0] = w.bz;
    out[1] = w.bps;
    out[2] = dlz::slab_blocks(w);
    return 0;
}

// s0 and nb of every block of the walk with slabs of bz planes
int slab_blocks_of(int plane, int Lz, int Lt, int bz, int *s0, int *nb) {
    const dlz::SlabWalk w = dlz::slab_walk_of(plane, Lz, Lt, bz);
    const long long n = dlz::slab_blocks(w);
    for (long long b = 0; b < n; ++b) dlz::slab_block(w, (int)b, s0[b], nb[b]);
    return (int)n;
}

}
