// Tensor-core (tcgen05) products of the Krylov basis, FP32 data with 3xTF32 splitting:
// the Rayleigh-Ritz restart V_{k+1} = V_{m+1} P of Lan-DR / MinRes-DR (arXiv:0901.3163,
// Sec. 1-2) and the Galerkin projection of D-CG / D-MinRes, C = V_k^dag R and
// E = V_k C' for a batch of right-hand sides (Sec. 2: projection at the start, repeated
// at every defect-correction restart).
//
// Both are dense contractions whose intensity (tens of flops per byte) is above the FP32
// CUDA-core ridge, so they run on the 5th-generation tensor cores: operands staged in
// shared memory, one thread issues tcgen05.mma (kind::tf32, M = 128), the accumulator
// lives in tensor memory and is read back with tcgen05.ld.  FP32 accuracy comes from
// splitting each operand x = hi + lo with hi = tf32(x) and lo = x - hi, and summing
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), all accumulated in FP32.
//
// Shared-memory operand layout (both operands K-major, no swizzle, 8-row x 16-byte
// core matrices): element (row, k) of a 32-wide K chunk at
//   (row / 8) * 1024 + (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4 bytes;
// descriptor: leading byte offset 128 (the next 4 k), stride byte offset 1024 (the next
// 8 rows); an MMA's K step of 8 advances the start address by 256 bytes.  The basis
// vectors are contiguous along the rows of the combine's A operand, so its staging
// transposes 4 x 4 blocks in registers.
// Every mbarrier wait is bounded: a wait that gives up sets an error word (reported as
// DLZ_ERR_DEVICE_TIMEOUT) and the kernel still frees its tensor memory.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"

namespace dlz {

namespace {

constexpr int kTcThreads = 256;     // 8 warps: staging, epilogue (two per TMEM lane quarter)
constexpr int kKC = 32;             // K chunk staged per pipeline stage
constexpr long long kWaitPolls = 1LL << 26;
constexpr int kTcMaxSmem = 2 * (2 * 128 * kKC * 4 + 2 * 256 * kKC * 4);   // 192 KB

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the sm_100 family; no swizzle
    return d;
}

// instruction descriptor: D FP32 (bits 4-5), A and B TF32 (7-9, 10-12), both K-major
// (bits 15, 16 zero), N / 8 (17-22), M / 16 (24-28) with M = 128
__device__ __forceinline__ uint32_t idesc_tf32(int n, uint32_t a_mn) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (a_mn << 15) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t taddr, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit_to(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar)));
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long long it = 0; it < kWaitPolls && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(su32(mbar)), "r"(parity));
    }
    return done != 0;
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void st_split(float *hi, float *lo, int off_floats, float4 v) {
    const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
    *reinterpret_cast<float4 *>(hi + off_floats) = h;
    *reinterpret_cast<float4 *>(lo + off_floats) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

// ------------------------------------------------------------------ combine
// Out[j][r] = sum_k A[r][k] Bt[j][k] for r in [0, rows), j in [0, nout), with
//   A[r][k] = V_k[r] (k < nin) and, for complex coefficients (cplx), A[r][nin + i] =
//   (i V_i)[r] (re <- -im, im <- re of each complex pair), so that Bt = [Re C'^T | Im C'^T]
//   gives Out = V C' for complex C'.  Bt (npad x kpad, K contiguous) comes split in hi, lo.
struct CombineArgs {
    const float *V;
    long ldv;          // floats between consecutive input vectors
    int nin;
    long rows;         // floats per vector (a multiple of 4)
    const float *Bhi, *Blo;
    int kpad, npad, nout, cplx;
    float *Out;
    long ldo;
    int *err;
};

// A pipeline stage is reused only after the MMAs that last read it are complete: every
// commit to a stage's mbarrier completes one phase, and `issued` / `seen` count, per stage,
// the commits made and the completions waited for (all threads keep the same counts).
struct StageSync {
    uint32_t issued[2] = {0u, 0u}, seen[2] = {0u, 0u};
    // wait until stage st has no MMA in flight; false if a wait gave up
    __device__ bool drain(uint64_t *mbar, int st) {
        while (seen[st] < issued[st]) {
            if (!mbar_wait(&mbar[st], seen[st] & 1u)) return false;
            ++seen[st];
        }
        return true;
    }
};

__device__ __forceinline__ void tc_setup(uint64_t *mbar, uint32_t *tbase, int ncols) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ void tc_teardown(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

// The combine's A operand for one thread: vectors 4 kq .. 4 kq + 3 of K chunk kc at rows
// r .. r + 3 (zero beyond the data; for complex coefficients the second half of K holds
// i times the vectors)
__device__ __forceinline__ void combine_load_a(const CombineArgs &a, int kc, int kq, long r, float4 (&v)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = kc * kKC + 4 * kq + j;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < a.rows) {
            if (k < a.nin) {
                v[j] = *reinterpret_cast<const float4 *>(a.V + (size_t)k * a.ldv + r);
            } else if (a.cplx && k < 2 * a.nin) {
                const float4 u = *reinterpret_cast<const float4 *>(a.V + (size_t)(k - a.nin) * a.ldv + r);
                v[j] = make_float4(-u.y, u.x, -u.w, u.z);        // i times the complex pairs
            }
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_combine(CombineArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int a_bytes = 128 * kKC * 4, b_bytes = a.npad * kKC * 4;
    const int stage_bytes = 2 * a_bytes + 2 * b_bytes;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    __shared__ int fail_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncols = tmem_cols(a.npad);
    if (tid == 0) fail_s = 0;
    tc_setup(mbar, &tbase, ncols);
    const uint32_t taddr = tbase;
    const long ntiles = (a.rows + 127) / 128;
    const int nkc = a.kpad / kKC;
    const uint32_t idesc = idesc_tf32(a.npad, 0u);
    StageSync ss;
    // A chunk: 128 rows x 32 k, K-major.  Thread (row quad rq, k quad kq) loads the four
    // vectors 4 kq .. 4 kq + 3 at rows 4 rq .. 4 rq + 3 (float4 each, 64 contiguous bytes
    // per vector across the 4 lanes of equal kq), transposes the 4 x 4 block and stores
    // one 16-byte k quad per row; lane l stores its rows in the order (c + l % 4) so that
    // the eight lanes of a store instruction with equal row parity hit different banks.
    // The loads of the next chunk (or of the next tile's first chunk) are issued right
    // after the current chunk's MMAs, so they are in flight during the MMAs, the next
    // stage's wait and the epilogue.
    const int kq = tid & 7, rq = tid >> 3;                                    // 8 k quads x 32 row quads
    float4 v[4];
    if ((long)blockIdx.x < ntiles) combine_load_a(a, 0, kq, (long)blockIdx.x * 128 + 4 * rq, v);
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long r0 = t * 128;
        for (int kc = 0; kc < nkc; ++kc) {
            const int st = kc & 1;
            unsigned char *sbase = smem + st * stage_bytes;
            float *Ahi = reinterpret_cast<float *>(sbase), *Alo = reinterpret_cast<float *>(sbase + a_bytes);
            float *Bhi = reinterpret_cast<float *>(sbase + 2 * a_bytes);
            float *Blo = reinterpret_cast<float *>(sbase + 2 * a_bytes + b_bytes);
            if (!ss.drain(mbar, st) && tid == 0) fail_s = 1;
            __syncthreads();
            if (fail_s) break;
            {
                const int rot = tid & 3;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int cc = (c + rot) & 3;                             // the row this lane stores now
                    float4 w4;
                    w4.x = cc == 0 ? v[0].x : cc == 1 ? v[0].y : cc == 2 ? v[0].z : v[0].w;
                    w4.y = cc == 0 ? v[1].x : cc == 1 ? v[1].y : cc == 2 ? v[1].z : v[1].w;
                    w4.z = cc == 0 ? v[2].x : cc == 1 ? v[2].y : cc == 2 ? v[2].z : v[2].w;
                    w4.w = cc == 0 ? v[3].x : cc == 1 ? v[3].y : cc == 2 ? v[3].z : v[3].w;
                    const int row = 4 * rq + cc;
                    st_split(Ahi, Alo, (row >> 3) * 256 + kq * 32 + (row & 7) * 4, w4);
                }
            }
            // B chunk: npad rows (outputs) x 32 k, K-major, from the pre-split global copies
            for (int w = tid; w < a.npad * (kKC / 4); w += kTcThreads) {
                const int j = w % a.npad, kq = w / a.npad;                   // k = 4 kq .. 4 kq + 3
                const size_t gi = (size_t)j * a.kpad + kc * kKC + 4 * kq;
                const int off = (j / 8) * 256 + kq * 32 + (j % 8) * 4;
                *reinterpret_cast<float4 *>(Bhi + off) = *reinterpret_cast<const float4 *>(a.Bhi + gi);
                *reinterpret_cast<float4 *>(Blo + off) = *reinterpret_cast<const float4 *>(a.Blo + gi);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint64_t ah = sdesc(su32(Ahi) + ks * 256, 128, 1024);
                    const uint64_t al = sdesc(su32(Alo) + ks * 256, 128, 1024);
                    const uint64_t bh = sdesc(su32(Bhi) + ks * 256, 128, 1024);
                    const uint64_t bl = sdesc(su32(Blo) + ks * 256, 128, 1024);
                    mma_tf32(taddr, ah, bh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                    mma_tf32(taddr, ah, bl, idesc, 1u);
                    mma_tf32(taddr, al, bh, idesc, 1u);
                }
                commit_to(&mbar[st]);
            }
            ++ss.issued[st];
            if (kc + 1 < nkc) combine_load_a(a, kc + 1, kq, r0 + 4 * rq, v);
            else if (t + gridDim.x < ntiles) combine_load_a(a, 0, kq, (t + gridDim.x) * 128 + 4 * rq, v);
        }
        // epilogue: every MMA of the tile complete, then each warp reads its lane quarter
        // and half of the columns
        bool okd = ss.drain(mbar, 0);
        okd = ss.drain(mbar, 1) && okd;
        if (!okd && tid == 0) fail_s = 1;
        __syncthreads();
        if (fail_s) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int lq = warp & 3, half = warp >> 2;
        const int c_lo = half * (a.npad / 2), c_hi = c_lo + a.npad / 2;
        const long r = r0 + 32 * lq + lane;
        for (int c0 = c_lo; c0 < c_hi; c0 += 8) {
            float v[8];
            tmem_ld8(taddr + ((uint32_t)(32 * lq) << 16) + (uint32_t)c0, v);
            if (r < a.rows) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j < a.nout) a.Out[(size_t)(c0 + j) * a.ldo + r] = v[j];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (fail_s && tid == 0) atomicExch(a.err, 1);
    tc_teardown(taddr, ncols);
}

// ------------------------------------------------------------------ dots
// Cpart[blk][i][c] (FP64) = sum over this block's segments of A[i][k] B[c][k], k running
// over the floats of the vectors: A rows = the nin basis vectors (rows >= nin are zero),
// B rows c < nq = R_c, nq <= c < 2 nq = rot(R_{c-nq}) with (re, im) -> (im, -re), so that
// for complex vectors sum_k A[i][k] B[c][k] = Re <v_i, r_c> and the rotated rows give
// Im <v_i, r_c>.  Each block takes segments of kSeg floats in turn; after each segment
// the FP32 accumulator is added into FP64 registers and the next segment starts afresh.
struct DotsArgs {
    const float *V;
    long ldv;
    int nin;
    const float *R;
    long ldr;
    int nq, npad;
    long len;          // floats per vector (a multiple of 32)
    double *Cpart;     // [gridDim.x][128][npad]
    int *err;
};
constexpr int kSegChunks = 64;      // 64 chunks of 32 floats per segment

// The dots' operands of one thread for chunk ch: A items w = tid + 256 i (i < 4; row
// 8 (w >> 6) + (w & 7), k quad (w >> 3) & 7) and at most one B item w = tid (npad <= 32)
__device__ __forceinline__ void dots_load(const DotsArgs &a, long ch, int tid, float4 (&va)[4], float4 &vb) {
    const long k0 = ch * kKC;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int w = tid + kTcThreads * q;
        const int i = 8 * (w >> 6) + (w & 7), kq = (w >> 3) & 7;
        va[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.nin) va[q] = *reinterpret_cast<const float4 *>(a.V + (size_t)i * a.ldv + k0 + 4 * kq);
    }
    vb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < a.npad * (kKC / 4)) {
        const int c = 8 * (tid >> 6) + (tid & 7), kq = (tid >> 3) & 7;
        if (c < a.nq) {
            vb = *reinterpret_cast<const float4 *>(a.R + (size_t)c * a.ldr + k0 + 4 * kq);
        } else if (c < 2 * a.nq) {
            const float4 u = *reinterpret_cast<const float4 *>(a.R + (size_t)(c - a.nq) * a.ldr + k0 + 4 * kq);
            vb = make_float4(u.y, -u.x, u.w, -u.z);
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_dots(DotsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int a_bytes = 128 * kKC * 4, b_bytes = a.npad * kKC * 4;
    const int stage_bytes = 2 * a_bytes + 2 * b_bytes;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    __shared__ int fail_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncols = tmem_cols(a.npad);
    if (tid == 0) fail_s = 0;
    tc_setup(mbar, &tbase, ncols);
    const uint32_t taddr = tbase;
    const uint32_t idesc = idesc_tf32(a.npad, 0u);
    const long nchunks = a.len / kKC;
    const long nseg = (nchunks + kSegChunks - 1) / kSegChunks;
    // per thread: its TMEM row (lane quarter warp & 3) and half of the columns, in FP64
    const int lq = warp & 3, half = warp >> 2;
    const int c_lo = half * (a.npad / 2);
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    StageSync ss;
    // operands of the next chunk are loaded into registers while the current MMAs run
    float4 va[4], vb;
    if ((long)blockIdx.x < nseg) dots_load(a, (long)blockIdx.x * kSegChunks, tid, va, vb);
    for (long sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const long ch0 = sg * kSegChunks, ch1 = min(nchunks, ch0 + kSegChunks);
        for (long ch = ch0; ch < ch1; ++ch) {
            const int st = (int)((ch - ch0) & 1);
            unsigned char *sbase = smem + st * stage_bytes;
            float *Ahi = reinterpret_cast<float *>(sbase), *Alo = reinterpret_cast<float *>(sbase + a_bytes);
            float *Bhi = reinterpret_cast<float *>(sbase + 2 * a_bytes);
            float *Blo = reinterpret_cast<float *>(sbase + 2 * a_bytes + b_bytes);
            if (!ss.drain(mbar, st) && tid == 0) fail_s = 1;
            __syncthreads();
            if (fail_s) break;
            // A chunk: 128 rows x 32 k, K-major; a warp instruction covers 8 rows x 4 k quads
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = tid + kTcThreads * q;
                st_split(Ahi, Alo, (w >> 6) * 256 + ((w >> 3) & 7) * 32 + (w & 7) * 4, va[q]);
            }
            if (tid < a.npad * (kKC / 4))
                st_split(Bhi, Blo, (tid >> 6) * 256 + ((tid >> 3) & 7) * 32 + (tid & 7) * 4, vb);
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint64_t ah = sdesc(su32(Ahi) + ks * 256, 128, 1024);
                    const uint64_t al = sdesc(su32(Alo) + ks * 256, 128, 1024);
                    const uint64_t bh = sdesc(su32(Bhi) + ks * 256, 128, 1024);
                    const uint64_t bl = sdesc(su32(Blo) + ks * 256, 128, 1024);
                    mma_tf32(taddr, ah, bh, idesc, (ch > ch0 || ks > 0) ? 1u : 0u);
                    mma_tf32(taddr, ah, bl, idesc, 1u);
                    mma_tf32(taddr, al, bh, idesc, 1u);
                }
                commit_to(&mbar[st]);
            }
            ++ss.issued[st];
            if (ch + 1 < ch1) dots_load(a, ch + 1, tid, va, vb);
            else if (sg + gridDim.x < nseg) dots_load(a, (sg + gridDim.x) * kSegChunks, tid, va, vb);
        }
        if (fail_s) break;
        bool okd = ss.drain(mbar, 0);
        okd = ss.drain(mbar, 1) && okd;
        if (!okd && tid == 0) fail_s = 1;
        __syncthreads();
        if (fail_s) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int c0 = 0; c0 < a.npad / 2; c0 += 8) {
            float v[8];
            tmem_ld8(taddr + ((uint32_t)(32 * lq) << 16) + (uint32_t)(c_lo + c0), v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[c0 + j] += (double)v[j];
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    const int row = 32 * lq + lane;
    double *out = a.Cpart + ((size_t)blockIdx.x * 128 + row) * a.npad + c_lo;
    for (int j = 0; j < a.npad / 2; ++j) out[j] = acc[j];
    if (fail_s && tid == 0) atomicExch(a.err, 1);
    tc_teardown(taddr, ncols);
}

// C[i][q] (complex) = sum over blocks of Cpart[blk][i][q] + i Cpart[blk][i][nq + q], in a
// fixed order (one thread per entry)
__global__ void k_tc_dots_sum(const double *__restrict__ Cpart, int nblk, int nin, int nq, int npad,
                              double2 *__restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nin * nq) return;
    const int i = e / nq, q = e % nq;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const double *p = Cpart + ((size_t)b * 128 + i) * npad;
        re += p[q];
        im += p[nq + q];
    }
    C[(size_t)q * nin + i] = make_double2(re, im);
}

// round to the 10-bit TF32 mantissa (nearest, ties away), as cvt.rna.tf32.f32 does
inline float tf32_round_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 148;
    }
    return n;
}

int check_err(TcScratch &sc, cudaStream_t st) {
    int h = 0;
    DLZ_CUDA_TRY(cudaMemcpyAsync(&h, sc.err.ptr(), sizeof(int), cudaMemcpyDeviceToHost, st));
    DLZ_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) return fail(DLZ_ERR_DEVICE_TIMEOUT, "a tensor-core kernel's mbarrier wait gave up");
    return DLZ_OK;
}

}  // namespace

int tc_prepare() {
    // dynamic shared memory beyond 48 KB (set once, outside any graph capture): at most
    // two stages of 2 x 16 KB (A) + 2 x 32 KB (B, npad = 256) = 192 KB; the opt-in limit
    // (227 KB) also covers the kernels' static shared memory
    static int done = 0;
    if (done) return DLZ_OK;
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_tc_combine, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_tc_dots, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem));
    done = 1;
    return DLZ_OK;
}

int tc_combine32(TcScratch &sc, cudaStream_t st, float *out, long ldo, const float *in, long ldv, int nin, long len,
                 const double *coef, int nout, bool cplx, long long *launches) {
    if (nin < 1 || nout < 1 || len < 1) return DLZ_OK;
    if (len % 4 || ldv % 4 || ldo % 4 || nout > 256) return fail(DLZ_ERR_BADARG, "tensor-core combine: shape");
    DLZ_TRY(tc_prepare());
    const int K = cplx ? 2 * nin : nin;
    const int kpad = round_up(K, kKC), npad = std::max(16, round_up(nout, 16));
    // Bt[j][k] (K contiguous): real coef[i][j] at k = i; complex: Re at k = i, Im at k = nin + i
    std::vector<float> hi((size_t)npad * kpad, 0.f), lo((size_t)npad * kpad, 0.f);
    for (int j = 0; j < nout; ++j)
        for (int i = 0; i < nin; ++i) {
            const float re = (float)(cplx ? coef[2 * ((size_t)i * nout + j)] : coef[(size_t)i * nout + j]);
            const float h = tf32_round_host(re);
            hi[(size_t)j * kpad + i] = h;
            lo[(size_t)j * kpad + i] = re - h;
            if (cplx) {
                const float im = (float)coef[2 * ((size_t)i * nout + j) + 1];
                const float hm = tf32_round_host(im);
                hi[(size_t)j * kpad + nin + i] = hm;
                lo[(size_t)j * kpad + nin + i] = im - hm;
            }
        }
    const size_t nb = hi.size() * sizeof(float);
    DLZ_TRY(sc.coef.reserve(2 * nb));
    float *dhi = sc.coef.as<float>(), *dlo = dhi + hi.size();
    DLZ_CUDA_TRY(cudaMemcpyAsync(dhi, hi.data(), nb, cudaMemcpyHostToDevice, st));
    DLZ_CUDA_TRY(cudaMemcpyAsync(dlo, lo.data(), nb, cudaMemcpyHostToDevice, st));
    DLZ_TRY(sc.err.reserve(sizeof(int)));
    DLZ_CUDA_TRY(cudaMemsetAsync(sc.err.ptr(), 0, sizeof(int), st));
    CombineArgs a;
    a.V = in; a.ldv = ldv; a.nin = nin; a.rows = len; a.Bhi = dhi; a.Blo = dlo;
    a.kpad = kpad; a.npad = npad; a.nout = nout; a.cplx = cplx ? 1 : 0; a.Out = out; a.ldo = ldo;
    a.err = sc.err.as<int>();
    const int smem = 2 * (2 * 128 * kKC * 4 + 2 * npad * kKC * 4);
    const long ntiles = (len + 127) / 128;
    const int per_sm = smem <= 100 * 1024 ? 2 : 1;
    const int grid = (int)std::min<long>(ntiles, (long)per_sm * num_sms());
    k_tc_combine<<<grid, kTcThreads, smem, st>>>(a);
    if (launches) *launches += 1;
    DLZ_CUDA_TRY(cudaGetLastError());
    return check_err(sc, st);
}

int tc_dots32(TcScratch &sc, cudaStream_t st, double2 *C_host, const float *V, long ldv, int nin, const float *R,
              long ldr, int nq, long len, long long *launches) {
    if (nin < 1 || nq < 1) return DLZ_OK;
    if (nin > 128 || nq > 16 || len % kKC || ldv % 4 || ldr % 4) return fail(DLZ_ERR_BADARG, "tensor-core dots: shape");
    DLZ_TRY(tc_prepare());
    const int npad = std::max(16, round_up(2 * nq, 16));
    const long nchunks = len / kKC, nseg = (nchunks + kSegChunks - 1) / kSegChunks;
    const int smem = 2 * (2 * 128 * kKC * 4 + 2 * npad * kKC * 4);
    const int per_sm = smem <= 100 * 1024 ? 2 : 1;
    const int grid = (int)std::max<long>(1, std::min<long>(nseg, (long)per_sm * num_sms()));
    DLZ_TRY(sc.part.reserve((size_t)grid * 128 * npad * sizeof(double) + (size_t)nin * nq * sizeof(double2)));
    double *part = sc.part.as<double>();
    double2 *Cd = reinterpret_cast<double2 *>(part + (size_t)grid * 128 * npad);
    DLZ_TRY(sc.err.reserve(sizeof(int)));
    DLZ_CUDA_TRY(cudaMemsetAsync(sc.err.ptr(), 0, sizeof(int), st));
    DotsArgs a;
    a.V = V; a.ldv = ldv; a.nin = nin; a.R = R; a.ldr = ldr; a.nq = nq; a.npad = npad; a.len = len;
    a.Cpart = part; a.err = sc.err.as<int>();
    k_tc_dots<<<grid, kTcThreads, smem, st>>>(a);
    const int ne = nin * nq;
    k_tc_dots_sum<<<(ne + 127) / 128, 128, 0, st>>>(part, grid, nin, nq, npad, Cd);
    if (launches) *launches += 2;
    DLZ_CUDA_TRY(cudaGetLastError());
    DLZ_TRY(check_err(sc, st));
    DLZ_CUDA_TRY(cudaMemcpyAsync(C_host, Cd, (size_t)ne * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DLZ_CUDA_TRY(cudaStreamSynchronize(st));
    return DLZ_OK;
}

}  // namespace dlz

// ------------------------------------------------------------------ C ABI (test and measurement)
extern "C" int dlz_basis_combine(const float *V, long long ldv, int nin, long long len, const double *coef, int nout,
                                 int cplx, float *out, long long ldo) {
    if (!V || !coef || !out || nin < 0 || nout < 0 || len < 0) return dlz::fail(DLZ_ERR_BADARG, "basis_combine arguments");
    dlz::TcScratch sc;
    return dlz::tc_combine32(sc, 0, out, (long)ldo, V, (long)ldv, nin, (long)len, coef, nout, cplx != 0, nullptr);
}

extern "C" int dlz_basis_dots(const float *V, long long ldv, int nin, const float *R, long long ldr, int nq,
                              long long len, double *C) {
    if (!V || !R || !C || nin < 0 || nq < 0 || len < 0) return dlz::fail(DLZ_ERR_BADARG, "basis_dots arguments");
    dlz::TcScratch sc;
    return dlz::tc_dots32(sc, 0, reinterpret_cast<double2 *>(C), V, (long)ldv, nin, R, (long)ldr, nq, (long)len, nullptr);
}
