// Internal declarations of the dlz library (not part of the C ABI): the
// Wilson operator of Sec. 2 and the state the solvers of Sec. 1-2 share.
//
// Device data layout ("field order"): a spinor of V sites is stored as
// component-major planes so that thread s of a warp touches consecutive
// 16-byte words:
//   FP64: double2 [12][V]   element (a, s) at a*V + s   (a = 3*spin + colour)
//   FP32: float4  [6][V]    plane c holds components 2c, 2c+1 of site s
// Gauge links (per direction mu, entry e = 3*row + col of the 3x3 matrix):
//   FP64: double2 [4][9][V] at (mu*9 + e)*V + s
//   FP32: float2  [4][9][V] at (mu*9 + e)*V + s
// The canonical user layout is complex [V][12] (see include/dlz.h); pack
// and unpack kernels convert at the API boundary.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dlz.h"

namespace dlz {

// ---------------------------------------------------------------- complex
template <typename T> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };
template <typename T> using cx = typename cplx_of<T>::type;

template <typename T> __host__ __device__ inline cx<T> mk(T re, T im) { cx<T> r; r.x = re; r.y = im; return r; }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// i * a
__host__ __device__ inline double2 timesI(double2 a) { return make_double2(-a.y, a.x); }
__host__ __device__ inline float2 timesI(float2 a) { return make_float2(-a.y, a.x); }
// a + i b, a - i b
__host__ __device__ inline double2 addI(double2 a, double2 b) { return make_double2(a.x - b.y, a.y + b.x); }
__host__ __device__ inline double2 subI(double2 a, double2 b) { return make_double2(a.x + b.y, a.y - b.x); }
__host__ __device__ inline float2 addI(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }
__host__ __device__ inline float2 subI(float2 a, float2 b) { return make_float2(a.x + b.y, a.y - b.x); }
// acc + u * v
__host__ __device__ inline double2 cfma(double2 u, double2 v, double2 acc) {
    acc.x = fma(u.x, v.x, acc.x); acc.x = fma(-u.y, v.y, acc.x);
    acc.y = fma(u.x, v.y, acc.y); acc.y = fma(u.y, v.x, acc.y);
    return acc;
}
__host__ __device__ inline float2 cfma(float2 u, float2 v, float2 acc) {
    acc.x = fmaf(u.x, v.x, acc.x); acc.x = fmaf(-u.y, v.y, acc.x);
    acc.y = fmaf(u.x, v.y, acc.y); acc.y = fmaf(u.y, v.x, acc.y);
    return acc;
}
// acc + conj(u) * v
__host__ __device__ inline double2 cfmaConj(double2 u, double2 v, double2 acc) {
    acc.x = fma(u.x, v.x, acc.x); acc.x = fma(u.y, v.y, acc.x);
    acc.y = fma(u.x, v.y, acc.y); acc.y = fma(-u.y, v.x, acc.y);
    return acc;
}
__host__ __device__ inline float2 cfmaConj(float2 u, float2 v, float2 acc) {
    acc.x = fmaf(u.x, v.x, acc.x); acc.x = fmaf(u.y, v.y, acc.x);
    acc.y = fmaf(u.x, v.y, acc.y); acc.y = fmaf(-u.y, v.x, acc.y);
    return acc;
}

// ---------------------------------------------------------------- geometry
struct Geom {
    int L[4];      // Lx, Ly, Lz, Lt
    int V;         // sites
    int bc_t;      // +1 periodic, -1 antiperiodic time
};

// ---------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};
void set_error(int code, const std::string &msg);
int fail(int code, const std::string &msg);
#define DLZ_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::dlz::fail(e_ == cudaErrorMemoryAllocation ? DLZ_ERR_OOM : DLZ_ERR_CUDA, \
                               std::string(#expr) + ": " + cudaGetErrorString(e_));    \
    } while (0)
#define DLZ_TRY(...)                 \
    do {                             \
        int r_ = (__VA_ARGS__);      \
        if (r_ != DLZ_OK) return r_; \
    } while (0)

// ---------------------------------------------------------------- device buffers
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t nbytes);
    void release();
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Reduction scratch: per-block partials, a completion counter and results.
// One instance per concurrently used reduction slot.
constexpr int kRedBlocks = 608;      // 4 x 152 SMs: fixed grid -> fixed summation order
constexpr int kRedThreads = 256;
constexpr int kMaxDots = 16;         // dots reduced by one fused kernel
struct RedScratch {
    double *partials;   // [kMaxDots][kRedBlocks]
    unsigned *counter;  // 1
    double *result;     // [kMaxDots]
};

struct Op;

// Launch accounting and optional stencil timing.  Only stencil launches in the
// precision of the solve's hot loop (`hot_f32`) are timed, so the reported
// average describes one kernel; each timed launch adds its algorithmic bytes:
// per site 24 reals read + 24 written per right-hand side, plus 4 links read
// once per site: 18 reals (FP64, 8 bytes each) or 12 reals (FP32, 4 bytes).
struct GraphExec;
struct Profiler {
    bool enabled = false;
    bool hot_f32 = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    bool armed = false;             // the current launch is being timed
    long long launches = 0;         // all kernels
    long long stencils = 0;         // timed stencil launches (direct)
    double stencil_bytes = 0.0;     // their algorithmic bytes
    // the same per kernel kind (tag): 0 plain stencil, 1 first fused stencil kernel of
    // an inner solver (k_cg_k1, k_minres_k1, k_lanczos_k1), 2 second one (k_cg_k23)
    static constexpr int kTags = 3;
    double tag_ms[kTags] = {0, 0, 0}, tag_bytes[kTags] = {0, 0, 0};
    long long tag_n[kTags] = {0, 0, 0};
    std::vector<int> pair_tag;      // tag of each direct event pair
    std::vector<double> pair_bytes; // bytes of each direct event pair
    int cur_tag = 0;
    // stencils inside captured graphs: timed by external event nodes of the graph,
    // read after a host synchronisation (one replay sampled per read)
    GraphExec *capture = nullptr;
    double sampled_ms = 0.0, sampled_bytes = 0.0;
    long long sampled = 0;
    void begin(bool on, bool f32);
    // reals_per_rhs: spinor reals moved per site and right-hand side (48 for a plain
    // stencil: read 24, write 24; more for a stencil with a fused epilogue)
    // link_reals: link reals read per site (< 0: 48 in FP32, two rows of 4 links; 72 in FP64)
    void stencil_start(cudaStream_t s, bool f32, long long sites, int nrhs, int reals_per_rhs = 48,
                       int tag = 0, int link_reals = -1);
    void stencil_stop(cudaStream_t s);
    double stencil_ms();            // synchronises the events; sums pairs
    ~Profiler();
};

// Grow-only device buffer (never shrinks; no allocation while large enough).
struct GrowBuf {
    DevBuf b;
    int reserve(size_t nbytes) {
        if (b.bytes >= nbytes) return 0;
        b.release();
        return b.alloc(nbytes);
    }
    void *ptr() const { return b.p; }
    template <typename T> T *as() const { return reinterpret_cast<T *>(b.p); }
};
// scratch of the tensor-core basis products (tc_gemm.cu)
struct TcScratch {
    GrowBuf coef, part, err;
};
// Tensor-core (tcgen05, 3xTF32) products of FP32 basis vectors on stream st:
//   tc_combine32: out[j] (len floats, stride ldo) = sum_i c_ij in[i] (stride ldv), i < nin,
//     j < nout <= 256; coef on the host, real [nin][nout] or complex interleaved
//     [nin][nout][2] (cplx: the vectors are complex, c_ij multiplies each complex entry);
//   tc_dots32: C_host[q][i] = <in_i, r_q> (complex; nin <= 128, nq <= 16, len % 32 == 0).
// launches (may be null) counts the kernels.  Set-up outside graphs: tc_prepare().
int tc_prepare();
int tc_combine32(TcScratch &sc, cudaStream_t st, float *out, long ldo, const float *in, long ldv, int nin, long len,
                 const double *coef, int nout, bool cplx, long long *launches);
int tc_dots32(TcScratch &sc, cudaStream_t st, double2 *C_host, const float *V, long ldv, int nin, const float *R,
              long ldr, int nq, long len, long long *launches);

// even-odd operators: right-hand sides per launch of the batched even-odd stencil
constexpr int kEoBatch = 16;

struct Op {
    Geom g;           // geometry of the operator's vectors (even-odd: g.V = V / 2 even sites)
    bool eo = false;  // even-odd (Schur complement) operator on the even sites
    Geom gf;          // full-lattice geometry (the stencil kernels of an even-odd operator)
    DevBuf eo_tmp64;  // odd-site work fields of the even-odd stencil, kEoBatch FP64 ...
    DevBuf eo_tmp32;  // ... and FP32 (allocated with the operator: no allocation inside graphs)
    double kappa;
    cudaStream_t stream;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture CUDA graphs
    bool use_graphs = true;
    DevBuf gauge64;   // double2 [4][9][V]
    DevBuf gauge32;   // float4  [4][3][V] (two rows)
    DevBuf red_mem;   // reduction scratch
    RedScratch red;
    Profiler prof;
    DevBuf md_scratch;   // block partials of the FP32 multi-dot (grown on demand, outside graphs)
    int multi_choice = 0;   // launch form the multi-lattice autotuner chose last (100 form + 10 chunks + half)
    TcScratch tc;           // scratch of the tensor-core basis products
    DevBuf stage_err;       // int: set by a stencil kernel whose staging wait gave up
};



// A CUDA event destroyed on every return path.
struct Event {
    cudaEvent_t e = nullptr;
    Event() = default;
    Event(const Event &) = delete;
    Event &operator=(const Event &) = delete;
    ~Event() {
        if (e) cudaEventDestroy(e);
    }
    cudaError_t create() { return e ? cudaSuccess : cudaEventCreate(&e); }
};

// ---------------------------------------------------------------- CUDA graphs
// A launch-bound sequence of kernels (a Lanczos cycle, a group of MinRes
// iterations on one right-hand side) is captured once on the private stream
// and replayed on op.stream.  Stencil timing is off while capturing; the
// launch count of the captured body is added on every replay.
struct GraphExec {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    std::vector<cudaEvent_t> ev;      // start/stop pairs of the timed stencils
    std::vector<double> bytes;        // algorithmic bytes of each timed stencil
    std::vector<int> tags;            // kernel kind of each timed stencil (Profiler tags)
    bool fresh = false;               // replayed since the last sample
    GraphExec() = default;
    GraphExec(const GraphExec &) = delete;
    GraphExec &operator=(const GraphExec &) = delete;
    ~GraphExec() {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    // add the stencil times of the last completed replay (call after a host sync)
    void sample(Profiler &pr) {
        if (!fresh) return;
        fresh = false;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) {
                pr.sampled_ms += ms;
                pr.sampled_bytes += bytes[i / 2];
                pr.sampled++;
                const int t = tags[i / 2];
                pr.tag_ms[t] += ms;
                pr.tag_bytes[t] += bytes[i / 2];
                pr.tag_n[t]++;
            } else {
                cudaGetLastError();   // a sample that cannot be read must not poison later checks
            }
        }
    }
};

template <class F>
int run_graph(Op &op, GraphExec &ge, F &&body) {
    if (!op.use_graphs || !op.cap_stream) return body();
    if (!ge.exec) {
        cudaStream_t saved = op.stream;
        const bool prof_saved = op.prof.enabled;
        const long long l0 = op.prof.launches;
        cudaError_t e = cudaStreamBeginCapture(op.cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return fail(DLZ_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        op.stream = op.cap_stream;
        op.prof.capture = prof_saved ? &ge : nullptr;
        const int rc = body();
        op.stream = saved;
        op.prof.capture = nullptr;
        op.prof.enabled = prof_saved;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(op.cap_stream, &graph);
        if (rc != DLZ_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return fail(DLZ_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { ge.exec = nullptr; return fail(DLZ_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
        ge.launches = op.prof.launches - l0;
        op.prof.launches = l0;
    }
    DLZ_CUDA_TRY(cudaGraphLaunch(ge.exec, op.stream));
    op.prof.launches += ge.launches;
    ge.fresh = true;
    return DLZ_OK;
}

// ---------------------------------------------------------------- kernels (launchers)
// Wilson stencil: out = [g5_out] (1 - kappa H) [g5_in] in, FP64 or FP32.
// which: DLZ_D (0,0), DLZ_DDAG (1,1), DLZ_Q (0,1).
int wilson64(Op &op, double2 *out, const double2 *in, int which);
int wilson32(Op &op, float4 *out, const float4 *in, int which);
// nrhs spinors stored one after another (FP32: 6V float4 each, FP64: 12V double2 each)
int wilson32_batch(Op &op, float4 *out, const float4 *in, int which, int nrhs);
// Even-odd operators (op.eo): out = A in on even-site fields for A = Dhat (DLZ_D),
// Dhat^dag (DLZ_DDAG), Qhat = gamma5 Dhat (DLZ_Q), nrhs fields one after another.
int eo_apply64(Op &op, double2 *out, const double2 *in, int which, int nrhs);
int eo_apply32(Op &op, float4 *out, const float4 *in, int which, int nrhs);
// out (parity par, nrhs fields) = H [gamma5]^g5in in (parity 1 - par), FP64
int eo_hop64(Op &op, double2 *out, const double2 *in, int par, bool g5in, int nrhs);
// FP32 hop for the fused even-odd CGNR (parity 1 - par input, parity par output)
int eo_hop32(Op &op, float4 *out, const float4 *in, int par, bool g5in, int nrhs);
// Full-lattice user vector (complex128 [V][12]) b -> be = b_e + kappa H_eo b_o (even
// internal planes) and bo = b_o (odd planes); and x_e (even planes) + b -> the full
// solution x = (x_e, b_o + kappa H_oe x_e) in the user layout (bo_work: odd planes).
int eo_prepare64(Op &op, double2 *be, double2 *bo, const double2 *b_user);
int eo_reconstruct64(Op &op, double2 *x_user, const double2 *xe, double2 *bo_work, const double2 *b_user);
int wilson64_batch(Op &op, double2 *out, const double2 *in, int which, int nrhs);
// A = D, D^dag, Q or D^dag D on internal FP64 vectors (tmp used for D^dag D).
int apply64(Op &op, double2 *out, const double2 *in, int which, double2 *tmp);
int apply32(Op &op, float4 *out, const float4 *in, int which, float4 *tmp);

// pack / unpack between canonical complex [V][12] and internal planes
int pack64(Op &op, double2 *dst, const double2 *src_canon);
int unpack64(Op &op, double2 *dst_canon, const double2 *src);
int pack32(Op &op, float4 *dst, const float2 *src_canon);
int unpack32(Op &op, float2 *dst_canon, const float4 *src);
// bfloat16 spinors (uint2 planes [6][V]) with FP32 arithmetic (wilson_bf16.cu)
int wilson_bf16_batch(Op &op, uint2 *out, const uint2 *in, int which, int nrhs);
int pack_bf16(Op &op, uint2 *dst, const float2 *src_canon);
int unpack_bf16(Op &op, float2 *dst_canon, const uint2 *src);
int convert64to32(Op &op, float4 *dst, const double2 *src);
int convert32to64(Op &op, double2 *dst, const float4 *src);

}  // namespace dlz
