// C ABI of the dlz library (include/dlz.h, where each entry point names the
// passage of the paper it implements): operator objects, host/device staging of
// user vectors, the solver and deflation-set entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "solvers.h"

namespace dlz {

namespace {
thread_local std::string g_last_error;
}

void set_error(int code, const std::string &msg) {
    g_last_error = std::string(dlz_strerror(code)) + ": " + msg;
}
int fail(int code, const std::string &msg) {
    set_error(code, msg);
    return code;
}

int DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) return DLZ_OK;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DLZ_ERR_OOM : DLZ_ERR_CUDA,
                    "cudaMalloc(" + std::to_string(nbytes) + "): " + cudaGetErrorString(e));
    }
    bytes = nbytes;
    return DLZ_OK;
}
void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

void Profiler::begin(bool on, bool f32) {
    enabled = on;
    hot_f32 = f32;
    used = 0;
    launches = 0;
    stencils = 0;
    stencil_bytes = 0.0;
    armed = false;
    capture = nullptr;
    sampled_ms = sampled_bytes = 0.0;
    sampled = 0;
    for (int t = 0; t < kTags; ++t) tag_ms[t] = tag_bytes[t] = 0.0, tag_n[t] = 0;
    pair_tag.clear();
    pair_bytes.clear();
}
void Profiler::stencil_start(cudaStream_t s, bool f32, long long sites, int nrhs, int reals_per_rhs,
                             int tag, int link_reals) {
    armed = enabled && f32 == hot_f32;
    if (!armed) return;
    cur_tag = (tag >= 0 && tag < kTags) ? tag : 0;
    const double lr = link_reals >= 0 ? (double)link_reals : (f32 ? 48.0 : 72.0);
    const double nbytes = f32 ? (double)sites * ((double)reals_per_rhs * nrhs + lr) * 4.0
                              : (double)sites * ((double)reals_per_rhs * nrhs + lr) * 8.0;
    if (capture) {
        // inside a graph capture: an external event node, owned by the graph
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        capture->ev.push_back(a);
        capture->ev.push_back(b);
        capture->bytes.push_back(nbytes);
        capture->tags.push_back(cur_tag);
        cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
        return;
    }
    if (used + 2 > pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
    }
    cudaEventRecord(pool[used], s);
    stencils++;
    stencil_bytes += nbytes;
    pair_tag.push_back(cur_tag);
    pair_bytes.push_back(nbytes);
}
void Profiler::stencil_stop(cudaStream_t s) {
    if (!armed) return;
    if (capture) {
        cudaEventRecordWithFlags(capture->ev.back(), s, cudaEventRecordExternal);
        armed = false;
        return;
    }
    cudaEventRecord(pool[used + 1], s);
    used += 2;
    armed = false;
}
double Profiler::stencil_ms() {
    double tot = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
        float ms = 0.f;
        cudaEventSynchronize(pool[i + 1]);
        if (cudaEventElapsedTime(&ms, pool[i], pool[i + 1]) == cudaSuccess) {
            tot += ms;
            const int t = pair_tag[i / 2];
            tag_ms[t] += ms;
            tag_bytes[t] += pair_bytes[i / 2];
            tag_n[t]++;
        } else {
            cudaGetLastError();
        }
    }
    return tot;
}
Profiler::~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

namespace {

bool on_device(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A user buffer that may live in host memory: `dev` is always a device pointer.
struct Staged {
    void *user = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    bool host = false;
    DevBuf buf;
    int in(Op &op, const void *p, size_t nbytes) {
        user = const_cast<void *>(p);
        bytes = nbytes;
        host = !on_device(p);
        if (!host) { dev = user; return DLZ_OK; }
        DLZ_TRY(buf.alloc(nbytes));
        dev = buf.p;
        DLZ_CUDA_TRY(cudaMemcpyAsync(dev, p, nbytes, cudaMemcpyHostToDevice, op.stream));
        return DLZ_OK;
    }
    int out(Op &, void *p, size_t nbytes) {
        user = p;
        bytes = nbytes;
        host = !on_device(p);
        if (!host) { dev = user; return DLZ_OK; }
        DLZ_TRY(buf.alloc(nbytes));
        dev = buf.p;
        return DLZ_OK;
    }
    int flush(Op &op) {
        if (host) DLZ_CUDA_TRY(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, op.stream));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        return DLZ_OK;
    }
};

// canonical gauge [4][V][9] complex128 -> FP64 planes [4][9][V] and FP32 planes; flags non-SU(3) links
// FP32 copy: first two rows only, float4 planes [4][3][V] (the stencil rebuilds row 3)
__global__ void k_gauge_pack(double2 *__restrict__ g64, float4 *__restrict__ g32,
                             const double2 *__restrict__ src, int V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // mu*V + s
    if (i >= 4L * V) return;
    const int mu = (int)(i / V), s = (int)(i % V);
    double2 u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        u[e] = src[i * 9 + e];
        g64[(size_t)(mu * 9 + e) * V + s] = u[e];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        g32[(size_t)(mu * 3 + q) * V + s] =
            make_float4((float)u[2 * q].x, (float)u[2 * q].y, (float)u[2 * q + 1].x, (float)u[2 * q + 1].y);
}

struct CountBadLinks {
    const double2 *src;
    __device__ void operator()(long i, double (&acc)[1]) const {
        double2 u[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = src[i * 9 + e];
        bool bad = false;
        // (U^dag U)_{ab} - delta_ab
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double re = 0.0, im = 0.0;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const double2 x = u[3 * r + a], y = u[3 * r + b];
                    re += x.x * y.x + x.y * y.y;
                    im += x.x * y.y - x.y * y.x;
                }
                if (a == b) re -= 1.0;
                if (!(fabs(re) <= 1e-10 && fabs(im) <= 1e-10)) bad = true;   // NaN fails too
            }
        // det U - 1
        auto cm = [](double2 p, double2 q) { return make_double2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x); };
        const double2 m0 = cm(u[4], u[8]), m1 = cm(u[5], u[7]);
        const double2 m2 = cm(u[3], u[8]), m3 = cm(u[5], u[6]);
        const double2 m4 = cm(u[3], u[7]), m5 = cm(u[4], u[6]);
        const double2 c0 = make_double2(m0.x - m1.x, m0.y - m1.y);
        const double2 c1 = make_double2(m2.x - m3.x, m2.y - m3.y);
        const double2 c2 = make_double2(m4.x - m5.x, m4.y - m5.y);
        const double2 t0 = cm(u[0], c0), t1 = cm(u[1], c1), t2 = cm(u[2], c2);
        const double dre = t0.x - t1.x + t2.x - 1.0, dim = t0.y - t1.y + t2.y;
        if (!(fabs(dre) <= 1e-10 && fabs(dim) <= 1e-10)) bad = true;
        if (bad) acc[0] += 1.0;
    }
};

int check_op(dlz_op_t op) {
    if (!op) return dlz::fail(DLZ_ERR_BADARG, "null operator");
    return DLZ_OK;
}

int check_params(const dlz_params *p) {
    if (!p) return fail(DLZ_ERR_BADARG, "null params");
    if (p->m < 2 || p->k < 0 || p->k >= p->m) return fail(DLZ_ERR_BADARG, "need m >= 2 and 0 <= k < m");
    if (p->m > 1000) return fail(DLZ_ERR_BADARG, "m > 1000");
    if (!(p->tol > 0.0)) return fail(DLZ_ERR_BADARG, "tol must be > 0");
    if (p->max_cycles < 1 || p->max_iter < 1 || p->check_every < 1)
        return fail(DLZ_ERR_BADARG, "max_cycles, max_iter, check_every must be >= 1");
    if (p->precision != DLZ_F64 && p->precision != DLZ_F32) return fail(DLZ_ERR_BADARG, "precision");
    if (!(p->reliable_delta > 0.0 && p->reliable_delta < 1.0)) return fail(DLZ_ERR_BADARG, "reliable_delta must be in (0, 1)");
    if (p->finish != 0 && p->finish != 1) return fail(DLZ_ERR_BADARG, "finish must be 0 or 1");
    if (p->eig_only != 0 && p->eig_only != 1) return fail(DLZ_ERR_BADARG, "eig_only must be 0 or 1");
    return DLZ_OK;
}

struct CallStats {
    Op &op;
    dlz_stats *out;
    std::chrono::steady_clock::time_point t0;
    CallStats(Op &o, dlz_stats *s, bool profile, bool f32) : op(o), out(s), t0(std::chrono::steady_clock::now()) {
        op.prof.begin(profile, f32);
    }
    void finish(dlz_stats &st) {
        st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st.gpu_launches = op.prof.launches;
        if (op.prof.enabled) {
            st.stencil_ms = op.prof.stencil_ms() + op.prof.sampled_ms;
            st.stencil_launches = op.prof.stencils + op.prof.sampled;
            st.stencil_bytes = op.prof.stencil_bytes + op.prof.sampled_bytes;
            for (int t = 0; t < Profiler::kTags; ++t) {
                st.kernel_ms[t] = op.prof.tag_ms[t];
                st.kernel_bytes[t] = op.prof.tag_bytes[t];
                st.kernel_launches[t] = op.prof.tag_n[t];
            }
        }
    }
};

}  // namespace
}  // namespace dlz

using namespace dlz;

// Static scratch of dlz_apply_noalloc (one per device; shared by all callers on it).
static __device__ __align__(256) unsigned char g_noalloc_scratch[DLZ_NOALLOC_SCRATCH_BYTES];

namespace dlz {
namespace {
// Device address of g_noalloc_scratch, looked up once per device.
int noalloc_scratch(void **out) {
    static std::mutex mu;
    static void *addr[128] = {};
    int dev = 0;
    DLZ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(DLZ_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(DLZ_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        addr[dev] = p;
    }
    *out = addr[dev];
    return DLZ_OK;
}
}  // namespace
}  // namespace dlz

extern "C" {

int dlz_params_default(dlz_params *p) {
    if (!p) return DLZ_ERR_BADARG;
    p->m = 40;
    p->k = 10;
    p->tol = 1e-10;
    p->tol_eig = 0.0;
    p->oversolve = 1.0;
    p->max_cycles = 1000;
    p->max_iter = 100000;
    p->reorth_period = 10;
    p->precision = DLZ_F64;
    p->reliable_delta = 1e-2;
    p->check_every = 16;
    p->profile = 0;
    p->finish = 0;
    p->eig_only = 0;
    return DLZ_OK;
}

const char *dlz_strerror(int code) {
    switch (code) {
    case DLZ_OK: return "DLZ_OK";
    case DLZ_ERR_BADARG: return "DLZ_ERR_BADARG";
    case DLZ_ERR_BAD_GAUGE: return "DLZ_ERR_BAD_GAUGE";
    case DLZ_ERR_NONFINITE: return "DLZ_ERR_NONFINITE";
    case DLZ_ERR_NOT_CONVERGED: return "DLZ_ERR_NOT_CONVERGED";
    case DLZ_ERR_BREAKDOWN: return "DLZ_ERR_BREAKDOWN";
    case DLZ_ERR_DEVICE_TIMEOUT: return "DLZ_ERR_DEVICE_TIMEOUT";
    case DLZ_ERR_CUDA: return "DLZ_ERR_CUDA";
    case DLZ_ERR_OOM: return "DLZ_ERR_OOM";
    case DLZ_ERR_IO: return "DLZ_ERR_IO";
    default: return "DLZ_ERR_UNKNOWN";
    }
}

const char *dlz_last_error(void) { return g_last_error.c_str(); }

int dlz_create_operator(const int dims[4], const void *gauge, double kappa, int bc_t, void *stream,
                        dlz_op_t *out) {
    if (!dims || !gauge || !out) return fail(DLZ_ERR_BADARG, "null argument");
    *out = nullptr;
    long long V = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 1) return fail(DLZ_ERR_BADARG, "lattice extents must be >= 1");
        V *= dims[i];
    }
    if (V * 12 > 0x7fffffffLL) return fail(DLZ_ERR_BADARG, "lattice too large (12 V must fit in int32)");
    if (bc_t != 1 && bc_t != -1) return fail(DLZ_ERR_BADARG, "bc_t must be +1 or -1");
    if (!std::isfinite(kappa)) return fail(DLZ_ERR_BADARG, "kappa not finite");
    dlz_op_s *h = new dlz_op_s();
    Op &op = h->op;
    for (int i = 0; i < 4; ++i) op.g.L[i] = dims[i];
    op.g.V = (int)V;
    op.g.bc_t = bc_t;
    op.kappa = kappa;
    op.stream = (cudaStream_t)stream;
    auto bail = [&](int rc) { delete h; return rc; };
    int rc = op.gauge64.alloc((size_t)36 * V * sizeof(double2));
    if (rc) return bail(rc);
    rc = op.gauge32.alloc((size_t)12 * V * sizeof(float4));
    if (rc) return bail(rc);
    rc = op.stage_err.alloc(sizeof(int));
    if (rc == DLZ_OK && cudaMemsetAsync(op.stage_err.p, 0, sizeof(int), op.stream) != cudaSuccess)
        rc = fail(DLZ_ERR_CUDA, "memset");
    if (rc == DLZ_OK) rc = op.red_mem.alloc((kMaxDots * kRedBlocks + kMaxDots + 8) * sizeof(double));
    if (rc) return bail(rc);
    op.red.partials = op.red_mem.as<double>();
    op.red.result = op.red.partials + kMaxDots * kRedBlocks;
    op.red.counter = reinterpret_cast<unsigned *>(op.red.result + kMaxDots);
    if (cudaMemsetAsync(op.red.counter, 0, sizeof(unsigned) * 2, op.stream) != cudaSuccess)
        return bail(fail(DLZ_ERR_CUDA, "memset"));
    if (cudaStreamCreateWithFlags(&op.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(DLZ_ERR_CUDA, "stream create"));
    {
        const char *env = std::getenv("DLZ_NO_GRAPHS");
        op.use_graphs = !(env && env[0] == '1');
    }
    rc = prepare_kernels(op);
    if (rc) return bail(rc);
    Staged g;
    rc = g.in(op, gauge, (size_t)36 * V * sizeof(double2));
    if (rc) return bail(rc);
    const double2 *src = (const double2 *)g.dev;
    k_gauge_pack<<<(int)((4 * V + 255) / 256), 256, 0, op.stream>>>(op.gauge64.as<double2>(),
                                                                      op.gauge32.as<float4>(), src, (int)V);
    if (cudaGetLastError() != cudaSuccess) return bail(fail(DLZ_ERR_CUDA, "gauge pack launch"));
    double *d_bad = op.red.result + kMaxDots - 1;
    rc = reduce<1>(op, 4L * V, CountBadLinks{src}, [=] __device__(const double *r) { *d_bad = r[0]; });
    if (rc) return bail(rc);
    double bad = 0.0;
    if (cudaMemcpyAsync(&bad, d_bad, sizeof(double), cudaMemcpyDeviceToHost, op.stream) != cudaSuccess ||
        cudaStreamSynchronize(op.stream) != cudaSuccess)
        return bail(fail(DLZ_ERR_CUDA, "gauge check"));
    if (bad != 0.0)
        return bail(fail(DLZ_ERR_BAD_GAUGE, std::to_string((long long)bad) + " links are not SU(3) to 1e-10"));
    *out = h;
    return DLZ_OK;
}

int dlz_destroy_operator(dlz_op_t h) {
    if (!h) return fail(DLZ_ERR_BADARG, "null operator");
    cudaStreamSynchronize(h->op.stream);
    delete h;
    return DLZ_OK;
}

int dlz_op_volume(dlz_op_t h, long long *V) {
    DLZ_TRY(check_op(h));
    if (!V) return fail(DLZ_ERR_BADARG, "null V");
    *V = h->op.g.V;
    return DLZ_OK;
}

int dlz_create_operator_eo(const int dims[4], const void *gauge, double kappa, int bc_t, void *stream,
                           dlz_op_t *out) {
    if (!dims || !out) return fail(DLZ_ERR_BADARG, "null argument");
    *out = nullptr;
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 2 || dims[i] % 2) return fail(DLZ_ERR_BADARG, "even-odd operator needs every lattice extent even");
    dlz_op_t h = nullptr;
    DLZ_TRY(dlz_create_operator(dims, gauge, kappa, bc_t, stream, &h));
    Op &op = h->op;
    op.gf = op.g;
    op.g.V = op.gf.V / 2;
    op.eo = true;
    const size_t vh = (size_t)op.g.V;
    int rc = op.eo_tmp64.alloc((size_t)kEoBatch * 12 * vh * sizeof(double2));
    if (rc == DLZ_OK) rc = op.eo_tmp32.alloc((size_t)kEoBatch * 6 * vh * sizeof(float4));
    if (rc != DLZ_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return DLZ_OK;
}

static int check_eo(dlz_op_t h) {
    DLZ_TRY(check_op(h));
    if (!h->op.eo) return fail(DLZ_ERR_BADARG, "not an even-odd operator (dlz_create_operator_eo)");
    return DLZ_OK;
}

int dlz_eo_prepare(dlz_op_t h, const void *b, void *b_e, int nrhs) {
    DLZ_TRY(check_eo(h));
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (nrhs == 0) return DLZ_OK;
    if (!b || !b_e) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    op.prof.begin(false, false);
    const long nf = 12L * op.gf.V, nh = 12L * op.g.V;
    Staged sb, so;
    DLZ_TRY(sb.in(op, b, (size_t)nf * nrhs * sizeof(double2)));
    DLZ_TRY(so.out(op, b_e, (size_t)nh * nrhs * sizeof(double2)));
    DevBuf be, bo;
    DLZ_TRY(be.alloc((size_t)nh * sizeof(double2)));
    DLZ_TRY(bo.alloc((size_t)nh * sizeof(double2)));
    for (int r = 0; r < nrhs; ++r) {
        DLZ_TRY(eo_prepare64(op, be.as<double2>(), bo.as<double2>(), (const double2 *)sb.dev + (size_t)r * nf));
        DLZ_TRY(unpack64(op, (double2 *)so.dev + (size_t)r * nh, be.as<double2>()));
    }
    return so.flush(op);
}

int dlz_eo_reconstruct(dlz_op_t h, const void *x_e, const void *b, void *x, int nrhs) {
    DLZ_TRY(check_eo(h));
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (nrhs == 0) return DLZ_OK;
    if (!x_e || !b || !x) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    op.prof.begin(false, false);
    const long nf = 12L * op.gf.V, nh = 12L * op.g.V;
    Staged sxe, sb, sx;
    DLZ_TRY(sxe.in(op, x_e, (size_t)nh * nrhs * sizeof(double2)));
    DLZ_TRY(sb.in(op, b, (size_t)nf * nrhs * sizeof(double2)));
    DLZ_TRY(sx.out(op, x, (size_t)nf * nrhs * sizeof(double2)));
    DevBuf xe, bo;
    DLZ_TRY(xe.alloc((size_t)nh * sizeof(double2)));
    DLZ_TRY(bo.alloc((size_t)nh * sizeof(double2)));
    for (int r = 0; r < nrhs; ++r) {
        DLZ_TRY(pack64(op, xe.as<double2>(), (const double2 *)sxe.dev + (size_t)r * nh));
        DLZ_TRY(eo_reconstruct64(op, (double2 *)sx.dev + (size_t)r * nf, xe.as<double2>(), bo.as<double2>(),
                                 (const double2 *)sb.dev + (size_t)r * nf));
    }
    return sx.flush(op);
}

int dlz_apply(dlz_op_t h, int which, const void *in, void *out, int dtype, int nrhs) {
    DLZ_TRY(check_op(h));
    Op &op = h->op;
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (which < DLZ_D || which > DLZ_DDAGD) return fail(DLZ_ERR_BADARG, "which");
    if (dtype != DLZ_F64 && dtype != DLZ_F32 && dtype != DLZ_BF16) return fail(DLZ_ERR_BADARG, "dtype");
    if (dtype == DLZ_BF16 && op.eo) return fail(DLZ_ERR_BADARG, "bfloat16 storage is not built for even-odd operators");
    if (nrhs == 0) return DLZ_OK;
    if (!in || !out) return fail(DLZ_ERR_BADARG, "null vector");
    op.prof.begin(false, false);
    const long n = 12L * op.g.V;
    const size_t esz = dtype == DLZ_F64 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = (size_t)n * esz * nrhs;
    const char *ip = (const char *)in, *op_ = (const char *)out;
    if (ip < op_ + bytes && op_ < ip + bytes) return fail(DLZ_ERR_BADARG, "in and out overlap");
    Staged si, so;
    DLZ_TRY(si.in(op, in, bytes));
    DLZ_TRY(so.out(op, out, bytes));
    DevBuf a, b, t;
    DLZ_TRY(a.alloc(n * esz));
    DLZ_TRY(b.alloc(n * esz));
    DLZ_TRY(t.alloc(n * esz));
    for (int r = 0; r < nrhs; ++r) {
        if (dtype == DLZ_F64) {
            const double2 *src = (const double2 *)si.dev + (size_t)r * n;
            double2 *dst = (double2 *)so.dev + (size_t)r * n;
            DLZ_TRY(pack64(op, a.as<double2>(), src));
            DLZ_TRY(apply64(op, b.as<double2>(), a.as<double2>(), which, t.as<double2>()));
            DLZ_TRY(unpack64(op, dst, b.as<double2>()));
        } else if (dtype == DLZ_F32) {
            const float2 *src = (const float2 *)si.dev + (size_t)r * n;
            float2 *dst = (float2 *)so.dev + (size_t)r * n;
            DLZ_TRY(pack32(op, a.as<float4>(), src));
            DLZ_TRY(apply32(op, b.as<float4>(), a.as<float4>(), which, t.as<float4>()));
            DLZ_TRY(unpack32(op, dst, b.as<float4>()));
        } else {
            // bfloat16 storage: D^dag D is Q applied twice, rounded to bfloat16 in between
            const float2 *src = (const float2 *)si.dev + (size_t)r * n;
            float2 *dst = (float2 *)so.dev + (size_t)r * n;
            DLZ_TRY(pack_bf16(op, a.as<uint2>(), src));
            if (which == DLZ_DDAGD) {
                DLZ_TRY(wilson_bf16_batch(op, t.as<uint2>(), a.as<uint2>(), DLZ_Q, 1));
                DLZ_TRY(wilson_bf16_batch(op, b.as<uint2>(), t.as<uint2>(), DLZ_Q, 1));
            } else {
                DLZ_TRY(wilson_bf16_batch(op, b.as<uint2>(), a.as<uint2>(), which, 1));
            }
            DLZ_TRY(unpack_bf16(op, dst, b.as<uint2>()));
        }
    }
    return so.flush(op);
}

int dlz_apply_noalloc(dlz_op_t h, int which, const void *in, void *out, int dtype, int nrhs) {
    DLZ_TRY(check_op(h));
    Op &op = h->op;
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (which < DLZ_D || which > DLZ_DDAGD) return fail(DLZ_ERR_BADARG, "which");
    if (dtype != DLZ_F64 && dtype != DLZ_F32) return fail(DLZ_ERR_BADARG, "dtype");
    const long n = 12L * op.g.V;
    const size_t esz = dtype == DLZ_F64 ? sizeof(double2) : sizeof(float2);
    const size_t vec = (size_t)n * esz;
    const size_t need = (which == DLZ_DDAGD ? 3 : 2) * vec;
    if (need > (size_t)DLZ_NOALLOC_SCRATCH_BYTES)
        return fail(DLZ_ERR_BADARG, "lattice too large for the static scratch of dlz_apply_noalloc");
    if (nrhs == 0) return DLZ_OK;
    if (!in || !out) return fail(DLZ_ERR_BADARG, "null vector");
    if (!on_device(in) || !on_device(out))
        return fail(DLZ_ERR_BADARG, "dlz_apply_noalloc takes device pointers only");
    const size_t bytes = vec * nrhs;
    const char *ip = (const char *)in, *op_ = (const char *)out;
    if (ip < op_ + bytes && op_ < ip + bytes) return fail(DLZ_ERR_BADARG, "in and out overlap");
    void *scratch = nullptr;
    DLZ_TRY(noalloc_scratch(&scratch));
    op.prof.begin(false, false);
    // packed input, packed output and (D^dag D only) the intermediate Q vector
    unsigned char *sa = (unsigned char *)scratch, *sb = sa + vec, *st = sb + vec;
    for (int r = 0; r < nrhs; ++r) {
        if (dtype == DLZ_F64) {
            const double2 *src = (const double2 *)in + (size_t)r * n;
            double2 *dst = (double2 *)out + (size_t)r * n;
            DLZ_TRY(pack64(op, (double2 *)sa, src));
            DLZ_TRY(apply64(op, (double2 *)sb, (const double2 *)sa, which, (double2 *)st));
            DLZ_TRY(unpack64(op, dst, (const double2 *)sb));
        } else {
            const float2 *src = (const float2 *)in + (size_t)r * n;
            float2 *dst = (float2 *)out + (size_t)r * n;
            DLZ_TRY(pack32(op, (float4 *)sa, src));
            DLZ_TRY(apply32(op, (float4 *)sb, (const float4 *)sa, which, (float4 *)st));
            DLZ_TRY(unpack32(op, dst, (const float4 *)sb));
        }
    }
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return DLZ_OK;
}

int dlz_batch_dminres(int nlat, dlz_op_t *ops, dlz_defl_t *defls, const void *const *B, void *const *X,
                      const int *nrhs, const dlz_params *p, dlz_stats *stats) {
    if (nlat < 1 || !ops || !B || !X || !nrhs) return fail(DLZ_ERR_BADARG, "batch_dminres arguments");
    DLZ_TRY(check_params(p));
    int total = 0;
    for (int l = 0; l < nlat; ++l) {
        if (!ops[l]) return fail(DLZ_ERR_BADARG, "null operator");
        if (ops[l]->op.eo) return fail(DLZ_ERR_BADARG, "dlz_batch_dminres takes full-lattice operators");
        if (nrhs[l] < 0 || nrhs[l] > 16) return fail(DLZ_ERR_BADARG, "nrhs per lattice must be in [0, 16]");
        if (nrhs[l] > 0 && (!B[l] || !X[l])) return fail(DLZ_ERR_BADARG, "null vector");
        if (defls && defls[l]) {
            if (defls[l]->op != &ops[l]->op) return fail(DLZ_ERR_BADARG, "deflation set of another operator");
            if (defls[l]->which != DLZ_Q) return fail(DLZ_ERR_BADARG, "D-MinRes needs a MinRes-DR (Q) deflation set");
        }
        total += nrhs[l];
    }
    if (p->precision == DLZ_F64) {
        // the plain form: one lattice after another
        int worst = DLZ_OK, q = 0;
        for (int l = 0; l < nlat; ++l) {
            if (nrhs[l] == 0) continue;
            const int rc = dlz_dminres(ops[l], defls ? defls[l] : nullptr, B[l], X[l], nrhs[l], p,
                                       stats ? stats + q : nullptr);
            if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) return rc;
            if (rc != DLZ_OK) worst = rc;
            q += nrhs[l];
        }
        return worst;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<Op *> opv(nlat);
    std::vector<const dlz_defl_s *> dv(nlat);
    std::vector<Staged> sb(nlat), sx(nlat);
    std::vector<DevBuf> bi(nlat), xi(nlat);
    std::vector<const double2 *> bptr(nlat);
    std::vector<double2 *> xptr(nlat);
    for (int l = 0; l < nlat; ++l) {
        Op &op = ops[l]->op;
        op.prof.begin(false, true);
        opv[l] = &op;
        dv[l] = defls ? defls[l] : nullptr;
        const long n = 12L * op.g.V;
        const size_t bytes = (size_t)n * std::max(nrhs[l], 1) * sizeof(double2);
        DLZ_TRY(bi[l].alloc(bytes));
        DLZ_TRY(xi[l].alloc(bytes));
        if (nrhs[l] > 0) {
            DLZ_TRY(sb[l].in(op, B[l], (size_t)n * nrhs[l] * sizeof(double2)));
            DLZ_TRY(sx[l].out(op, X[l], (size_t)n * nrhs[l] * sizeof(double2)));
            for (int r = 0; r < nrhs[l]; ++r)
                DLZ_TRY(pack64(op, bi[l].as<double2>() + (size_t)r * n, (const double2 *)sb[l].dev + (size_t)r * n));
        }
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        bptr[l] = bi[l].as<double2>();
        xptr[l] = xi[l].as<double2>();
    }
    std::vector<dlz_stats> st(std::max(total, 1));
    const int rc = dminres_multi(nlat, opv.data(), dv.data(), bptr.data(), xptr.data(), nrhs, *p, st.data());
    if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) return rc;
    for (int l = 0; l < nlat; ++l) {
        Op &op = ops[l]->op;
        const long n = 12L * op.g.V;
        for (int r = 0; r < nrhs[l]; ++r)
            DLZ_TRY(unpack64(op, (double2 *)sx[l].dev + (size_t)r * n, xi[l].as<double2>() + (size_t)r * n));
        if (nrhs[l] > 0) DLZ_TRY(sx[l].flush(op));
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int q = 0; q < total; ++q) {
            stats[q] = st[q];
            stats[q].seconds = secs / total;
        }
    return rc;
}

int dlz_batch_last_choice(dlz_op_t h, int *form, int *chunks_per_block, int *half_grid) {
    DLZ_TRY(check_op(h));
    const int c = h->op.multi_choice;
    if (form) *form = c / 100;
    if (chunks_per_block) *chunks_per_block = (c / 10) % 10;
    if (half_grid) *half_grid = c % 10;
    return DLZ_OK;
}

int dlz_stencil_bench(dlz_op_t h, int dtype, int which, int nrhs, int iters, const void *in,
                      double *ms_per_launch) {
    DLZ_TRY(check_op(h));
    Op &op = h->op;
    if (!in || !ms_per_launch || nrhs < 1 || nrhs > 64 || iters < 1) return fail(DLZ_ERR_BADARG, "stencil_bench arguments");
    if (which != DLZ_D && which != DLZ_DDAG && which != DLZ_Q) return fail(DLZ_ERR_BADARG, "which");
    if (dtype != DLZ_F64 && dtype != DLZ_F32 && dtype != DLZ_BF16) return fail(DLZ_ERR_BADARG, "dtype");
    if (dtype == DLZ_BF16 && op.eo) return fail(DLZ_ERR_BADARG, "bfloat16 storage is not built for even-odd operators");
    op.prof.begin(false, false);
    const long n = 12L * op.g.V;
    const size_t esz = dtype == DLZ_F64 ? sizeof(double2) : sizeof(float2);
    Staged si;
    DLZ_TRY(si.in(op, in, (size_t)n * nrhs * esz));
    DevBuf a, b;
    DLZ_TRY(a.alloc((size_t)n * nrhs * esz));
    DLZ_TRY(b.alloc((size_t)n * nrhs * esz));
    for (int r = 0; r < nrhs; ++r) {
        if (dtype == DLZ_F64) DLZ_TRY(pack64(op, a.as<double2>() + (size_t)r * n, (const double2 *)si.dev + (size_t)r * n));
        else if (dtype == DLZ_F32) DLZ_TRY(pack32(op, a.as<float4>() + (size_t)r * n / 2, (const float2 *)si.dev + (size_t)r * n));
        else DLZ_TRY(pack_bf16(op, a.as<uint2>() + (size_t)r * n / 2, (const float2 *)si.dev + (size_t)r * n));
    }
    auto launch = [&]() -> int {
        if (dtype == DLZ_F64) return wilson64_batch(op, b.as<double2>(), a.as<double2>(), which, nrhs);
        if (dtype == DLZ_BF16) return wilson_bf16_batch(op, b.as<uint2>(), a.as<uint2>(), which, nrhs);
        return wilson32_batch(op, b.as<float4>(), a.as<float4>(), which, nrhs);
    };
    for (int i = 0; i < 3; ++i) DLZ_TRY(launch());
    Event e0, e1;
    DLZ_CUDA_TRY(e0.create());
    DLZ_CUDA_TRY(e1.create());
    DLZ_CUDA_TRY(cudaEventRecord(e0.e, op.stream));
    for (int i = 0; i < iters; ++i) DLZ_TRY(launch());
    DLZ_CUDA_TRY(cudaEventRecord(e1.e, op.stream));
    DLZ_CUDA_TRY(cudaEventSynchronize(e1.e));
    float ms = 0.f;
    DLZ_CUDA_TRY(cudaEventElapsedTime(&ms, e0.e, e1.e));
    *ms_per_launch = ms / iters;
    return DLZ_OK;
}

static int dr_entry(dlz_op_t h, bool harmonic, const void *b, void *x, const dlz_params *p,
                    dlz_defl_t *defl_out, dlz_stats *stats) {
    DLZ_TRY(check_op(h));
    DLZ_TRY(check_params(p));
    if (!b || !x) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    if (defl_out) *defl_out = nullptr;
    dlz_stats st;
    std::memset(&st, 0, sizeof(st));
    CallStats cs(op, stats, p->profile != 0, p->precision == DLZ_F32);
    const long n = 12L * op.g.V;
    Staged sb, sx;
    DLZ_TRY(sb.in(op, b, n * sizeof(double2)));
    DLZ_TRY(sx.out(op, x, n * sizeof(double2)));
    DevBuf bi, xi;
    DLZ_TRY(bi.alloc(n * sizeof(double2)));
    DLZ_TRY(xi.alloc(n * sizeof(double2)));
    DLZ_TRY(pack64(op, bi.as<double2>(), (const double2 *)sb.dev));
    dlz_defl_s *d = nullptr;
    const int rc = dr_solve(op, harmonic, bi.as<double2>(), xi.as<double2>(), *p, defl_out ? &d : nullptr, st);
    if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) {
        delete d;
        return rc;
    }
    DLZ_TRY(unpack64(op, (double2 *)sx.dev, xi.as<double2>()));
    DLZ_TRY(sx.flush(op));
    if (defl_out) *defl_out = d;
    cs.finish(st);
    if (stats) *stats = st;
    if (rc == DLZ_ERR_NOT_CONVERGED) set_error(rc, "max_cycles reached");
    return rc;
}

int dlz_landr(dlz_op_t h, const void *b, void *x, const dlz_params *p, dlz_defl_t *defl_out,
              dlz_stats *stats) {
    return dr_entry(h, false, b, x, p, defl_out, stats);
}
int dlz_minresdr(dlz_op_t h, const void *b, void *x, const dlz_params *p, dlz_defl_t *defl_out,
                 dlz_stats *stats) {
    return dr_entry(h, true, b, x, p, defl_out, stats);
}

static int dsolve_entry(dlz_op_t h, dlz_defl_t d, const void *B, void *X, int nrhs,
                        const dlz_params *p, dlz_stats *stats, bool minres) {
    DLZ_TRY(check_op(h));
    DLZ_TRY(check_params(p));
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (nrhs == 0) return DLZ_OK;
    if (!B || !X) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    if (d) {
        if (d->op != &op) return fail(DLZ_ERR_BADARG, "deflation set belongs to another operator");
        if (d->which != (minres ? DLZ_Q : DLZ_DDAGD))
            return fail(DLZ_ERR_BADARG, minres ? "D-MinRes needs a MinRes-DR (Q) deflation set"
                                               : "D-CG needs a Lan-DR (D^dag D) deflation set");
    }
    const long n = 12L * op.g.V;
    Staged sb, sx;
    DLZ_TRY(sb.in(op, B, (size_t)n * nrhs * sizeof(double2)));
    DLZ_TRY(sx.out(op, X, (size_t)n * nrhs * sizeof(double2)));
    int worst = DLZ_OK;
    if (p->precision == DLZ_F32) {
        // batched mixed-precision D-MinRes / D-CG, up to 16 right-hand sides per pass
        const int chunk = std::min(nrhs, 16);
        DevBuf bi, xi;
        DLZ_TRY(bi.alloc((size_t)chunk * n * sizeof(double2)));
        DLZ_TRY(xi.alloc((size_t)chunk * n * sizeof(double2)));
        std::vector<dlz_stats> sts(chunk);
        for (int r0 = 0; r0 < nrhs; r0 += chunk) {
            const int nb = std::min(chunk, nrhs - r0);
            CallStats cs(op, nullptr, p->profile != 0, p->precision == DLZ_F32);
            for (int q = 0; q < nb; ++q)
                DLZ_TRY(pack64(op, bi.as<double2>() + (size_t)q * n, (const double2 *)sb.dev + (size_t)(r0 + q) * n));
            const int rc = dsolve_mixed_batch(op, d, minres, bi.as<double2>(), xi.as<double2>(), nb, *p, sts.data());
            if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) return rc;
            if (rc != DLZ_OK) worst = rc;
            for (int q = 0; q < nb; ++q)
                DLZ_TRY(unpack64(op, (double2 *)sx.dev + (size_t)(r0 + q) * n, xi.as<double2>() + (size_t)q * n));
            DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
            dlz_stats shared;
            std::memset(&shared, 0, sizeof(shared));
            cs.finish(shared);
            // the batch's totals shared out over its right-hand sides; counts are split
            // so that they add up to the batch's counts exactly
            auto share = [nb](long long total, int q) { return total / nb + (q < total % nb ? 1 : 0); };
            for (int q = 0; q < nb; ++q) {
                sts[q].seconds = shared.seconds / nb;
                sts[q].gpu_launches = share(shared.gpu_launches, q);
                sts[q].stencil_ms = shared.stencil_ms / nb;
                sts[q].stencil_launches = share(shared.stencil_launches, q);
                sts[q].stencil_bytes = shared.stencil_bytes / nb;
                for (int t = 0; t < 3; ++t) {
                    sts[q].kernel_ms[t] = shared.kernel_ms[t] / nb;
                    sts[q].kernel_bytes[t] = shared.kernel_bytes[t] / nb;
                    sts[q].kernel_launches[t] = share(shared.kernel_launches[t], q);
                }
                if (stats) stats[r0 + q] = sts[q];
            }
        }
        DLZ_TRY(sx.flush(op));
        if (worst != DLZ_OK) set_error(worst, "max_iter reached for at least one right-hand side");
        return worst;
    }
    DevBuf bi, xi;
    DLZ_TRY(bi.alloc(n * sizeof(double2)));
    DLZ_TRY(xi.alloc(n * sizeof(double2)));
    for (int r = 0; r < nrhs; ++r) {
        dlz_stats st;
        std::memset(&st, 0, sizeof(st));
        CallStats cs(op, nullptr, p->profile != 0, p->precision == DLZ_F32);
        DLZ_TRY(pack64(op, bi.as<double2>(), (const double2 *)sb.dev + (size_t)r * n));
        // the plain FP64 form, one right-hand side at a time
        const int rc = minres ? dminres64(op, d, bi.as<double2>(), xi.as<double2>(), *p, st)
                              : dcg64(op, d, bi.as<double2>(), xi.as<double2>(), *p, st);
        if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) return rc;
        if (rc != DLZ_OK) worst = rc;
        DLZ_TRY(unpack64(op, (double2 *)sx.dev + (size_t)r * n, xi.as<double2>()));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        cs.finish(st);
        if (stats) stats[r] = st;
    }
    DLZ_TRY(sx.flush(op));
    if (worst != DLZ_OK) set_error(worst, "max_iter reached for at least one right-hand side");
    return worst;
}

int dlz_dcg(dlz_op_t h, dlz_defl_t d, const void *B, void *X, int nrhs, const dlz_params *p,
            dlz_stats *stats) {
    return dsolve_entry(h, d, B, X, nrhs, p, stats, false);
}
int dlz_dminres(dlz_op_t h, dlz_defl_t d, const void *B, void *X, int nrhs, const dlz_params *p,
                dlz_stats *stats) {
    return dsolve_entry(h, d, B, X, nrhs, p, stats, true);
}

int dlz_gmresdr(dlz_op_t h, const void *b, void *x, const dlz_params *p, dlz_defl_t *defl_out, dlz_stats *stats) {
    DLZ_TRY(check_op(h));
    DLZ_TRY(check_params(p));
    if (p->precision != DLZ_F64) return fail(DLZ_ERR_BADARG, "GMRES-DR is built in FP64 (precision DLZ_F64)");
    if (!b || !x) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    if (defl_out) *defl_out = nullptr;
    dlz_stats st;
    std::memset(&st, 0, sizeof(st));
    CallStats cs(op, stats, p->profile != 0, false);
    const long n = 12L * op.g.V;
    Staged sb, sx;
    DLZ_TRY(sb.in(op, b, n * sizeof(double2)));
    DLZ_TRY(sx.out(op, x, n * sizeof(double2)));
    DevBuf bi, xi;
    DLZ_TRY(bi.alloc(n * sizeof(double2)));
    DLZ_TRY(xi.alloc(n * sizeof(double2)));
    DLZ_TRY(pack64(op, bi.as<double2>(), (const double2 *)sb.dev));
    dlz_defl_s *d = nullptr;
    const int rc = gmresdr64(op, bi.as<double2>(), xi.as<double2>(), *p, defl_out ? &d : nullptr, st);
    if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) {
        delete d;
        return rc;
    }
    DLZ_TRY(unpack64(op, (double2 *)sx.dev, xi.as<double2>()));
    DLZ_TRY(sx.flush(op));
    if (defl_out) *defl_out = d;
    cs.finish(st);
    if (stats) *stats = st;
    if (rc == DLZ_ERR_NOT_CONVERGED) set_error(rc, "max_cycles reached");
    return rc;
}

int dlz_dgmres(dlz_op_t h, dlz_defl_t d, const void *B, void *X, int nrhs, const dlz_params *p, dlz_stats *stats) {
    DLZ_TRY(check_op(h));
    DLZ_TRY(check_params(p));
    if (p->precision != DLZ_F64) return fail(DLZ_ERR_BADARG, "D-GMRES is built in FP64 (precision DLZ_F64)");
    if (nrhs < 0) return fail(DLZ_ERR_BADARG, "nrhs < 0");
    if (nrhs == 0) return DLZ_OK;
    if (!B || !X) return fail(DLZ_ERR_BADARG, "null vector");
    Op &op = h->op;
    if (d && (d->op != &op || d->which != DLZ_D))
        return fail(DLZ_ERR_BADARG, "D-GMRES needs a GMRES-DR deflation set of this operator");
    const long n = 12L * op.g.V;
    Staged sb, sx;
    DLZ_TRY(sb.in(op, B, (size_t)n * nrhs * sizeof(double2)));
    DLZ_TRY(sx.out(op, X, (size_t)n * nrhs * sizeof(double2)));
    DevBuf bi, xi;
    DLZ_TRY(bi.alloc(n * sizeof(double2)));
    DLZ_TRY(xi.alloc(n * sizeof(double2)));
    int worst = DLZ_OK;
    for (int r = 0; r < nrhs; ++r) {
        dlz_stats st;
        std::memset(&st, 0, sizeof(st));
        CallStats cs(op, nullptr, p->profile != 0, false);
        DLZ_TRY(pack64(op, bi.as<double2>(), (const double2 *)sb.dev + (size_t)r * n));
        const int rc = dgmres64(op, d, bi.as<double2>(), xi.as<double2>(), *p, st);
        if (rc != DLZ_OK && rc != DLZ_ERR_NOT_CONVERGED) return rc;
        if (rc != DLZ_OK) worst = rc;
        DLZ_TRY(unpack64(op, (double2 *)sx.dev + (size_t)r * n, xi.as<double2>()));
        DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
        cs.finish(st);
        if (stats) stats[r] = st;
    }
    DLZ_TRY(sx.flush(op));
    if (worst != DLZ_OK) set_error(worst, "max_iter reached for at least one right-hand side");
    return worst;
}

int dlz_defl_value_complex(dlz_defl_t d, int i, double *re, double *im) {
    if (!d) return fail(DLZ_ERR_BADARG, "null deflation set");
    if (i < 0 || i >= d->k) return fail(DLZ_ERR_BADARG, "index out of range");
    const std::complex<double> v = d->which == DLZ_D ? d->theta[i] : std::complex<double>(d->values[i], 0.0);
    if (re) *re = v.real();
    if (im) *im = v.imag();
    return DLZ_OK;
}

int dlz_defl_count(dlz_defl_t d, int *k, int *which) {
    if (!d) return fail(DLZ_ERR_BADARG, "null deflation set");
    if (k) *k = d->k;
    if (which) *which = d->which;
    return DLZ_OK;
}

int dlz_defl_get(dlz_defl_t d, int i, void *vec_out, double *value, double *residual) {
    if (!d) return fail(DLZ_ERR_BADARG, "null deflation set");
    if (i < 0 || i >= d->k) return fail(DLZ_ERR_BADARG, "index out of range");
    if (d->which == DLZ_D) {
        // GMRES-DR set: harmonic Ritz pair i (value: Re theta; dlz_defl_value_complex for theta)
        Op &op = *d->op;
        if (value) *value = d->theta[i].real();
        if (residual) {
            DLZ_TRY(gmres_deflation_residuals(op, d));
            *residual = d->residuals[i];
        }
        if (!vec_out) return DLZ_OK;
        const long n = 12L * op.g.V;
        const int k = d->k;
        DevBuf y, coef, nrm;
        DLZ_TRY(y.alloc(n * sizeof(double2)));
        DLZ_TRY(coef.alloc((size_t)(k + 1) * sizeof(double2)));
        DLZ_TRY(nrm.alloc(sizeof(double)));
        std::vector<double2> z(k + 1);
        for (int a = 0; a <= k; ++a) z[a] = make_double2(d->Z[(size_t)a * k + i].real(), d->Z[(size_t)a * k + i].imag());
        DLZ_CUDA_TRY(cudaMemcpyAsync(coef.p, z.data(), (k + 1) * sizeof(double2), cudaMemcpyHostToDevice, op.stream));
        DLZ_TRY(combine64(op, y.as<double2>(), n, 1, d->V64.as<double2>(), n, k + 1, coef.p, 1, false, false));
        DLZ_TRY(v64::norm2_diff(op, y.as<double2>(), nullptr, nrm.as<double>()));
        double2 *py = y.as<double2>();
        const double *pn = nrm.as<double>();
        DLZ_TRY(map(op, n, [=] __device__(long j) {
            const double s = 1.0 / sqrt(*pn);
            py[j] = make_double2(s * py[j].x, s * py[j].y);
        }));
        Staged so;
        DLZ_TRY(so.out(op, vec_out, n * sizeof(double2)));
        DLZ_TRY(unpack64(op, (double2 *)so.dev, y.as<double2>()));
        return so.flush(op);
    }
    if (value) *value = d->values[i];
    if (residual) {
        DLZ_TRY(deflation_residuals(*d->op, d));
        *residual = d->residuals[i];
    }
    if (!vec_out) return DLZ_OK;
    Op &op = *d->op;
    const long n = 12L * op.g.V;
    DevBuf y, coef;
    DLZ_TRY(y.alloc(n * sizeof(double2)));
    DLZ_TRY(coef.alloc((size_t)d->k * sizeof(double2)));
    std::vector<double2> z(d->k);
    for (int j = 0; j < d->k; ++j) z[j] = make_double2(d->Z[(size_t)j * d->k + i].real(), d->Z[(size_t)j * d->k + i].imag());
    DLZ_CUDA_TRY(cudaMemcpyAsync(coef.p, z.data(), d->k * sizeof(double2), cudaMemcpyHostToDevice, op.stream));
    DLZ_TRY(combine64(op, y.as<double2>(), n, 1, d->V64.as<double2>(), n, d->k, coef.p, 1, false, false));
    Staged so;
    DLZ_TRY(so.out(op, vec_out, n * sizeof(double2)));
    DLZ_TRY(unpack64(op, (double2 *)so.dev, y.as<double2>()));
    return so.flush(op);
}

namespace {
const char kMagic[8] = {'D', 'L', 'Z', 'D', 'E', 'F', 'L', '1'};
struct FileHeader {
    char magic[8];
    int dims[4];
    int bc_t;
    int k;
    int which;
    int reserved;
    double kappa;
};
}  // namespace

int dlz_defl_save(dlz_defl_t d, const char *path) {
    if (!d || !path) return fail(DLZ_ERR_BADARG, "null argument");
    if (d->which == DLZ_D) return fail(DLZ_ERR_BADARG, "GMRES-DR deflation sets are not saved to files");
    Op &op = *d->op;
    const long n = 12L * op.g.V;
    FileHeader hd;
    std::memcpy(hd.magic, kMagic, 8);
    for (int i = 0; i < 4; ++i) hd.dims[i] = op.g.L[i];
    hd.bc_t = op.g.bc_t;
    hd.k = d->k;
    hd.which = d->which;
    hd.reserved = op.eo ? 1 : 0;        // 1: even-site vectors of an even-odd operator
    hd.kappa = op.kappa;
    std::vector<double2> host((size_t)n);
    DevBuf tmp;
    DLZ_TRY(tmp.alloc(n * sizeof(double2)));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(DLZ_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    for (int j = 0; ok && j < d->k; ++j) {
        if (unpack64(op, tmp.as<double2>(), d->V64.as<double2>() + (size_t)j * n) != DLZ_OK) { ok = false; break; }
        if (cudaMemcpyAsync(host.data(), tmp.p, n * sizeof(double2), cudaMemcpyDeviceToHost, op.stream) != cudaSuccess ||
            cudaStreamSynchronize(op.stream) != cudaSuccess) { ok = false; break; }
        ok = std::fwrite(host.data(), sizeof(double2), n, f) == (size_t)n;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DLZ_OK : fail(DLZ_ERR_IO, std::string("write failed: ") + path);
}

int dlz_defl_load(dlz_op_t h, const char *path, dlz_defl_t *out) {
    DLZ_TRY(check_op(h));
    if (!path || !out) return fail(DLZ_ERR_BADARG, "null argument");
    *out = nullptr;
    Op &op = h->op;
    const long n = 12L * op.g.V;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(DLZ_ERR_IO, std::string("cannot open ") + path);
    FileHeader hd;
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0;
    for (int i = 0; ok && i < 4; ++i) ok = hd.dims[i] == op.g.L[i];
    ok = ok && hd.bc_t == op.g.bc_t && hd.kappa == op.kappa && hd.k >= 0 && hd.k <= 1000 &&
         hd.reserved == (op.eo ? 1 : 0) &&
         (hd.which == DLZ_Q || hd.which == DLZ_DDAGD);
    if (!ok) {
        std::fclose(f);
        return fail(DLZ_ERR_IO, "deflation file does not match this operator");
    }
    dlz_defl_s *d = new dlz_defl_s();
    d->op = &op;
    d->k = hd.k;
    d->which = hd.which;
    std::vector<double2> host((size_t)n);
    DevBuf tmp;
    int rc = d->V64.alloc((size_t)d->k * n * sizeof(double2));
    if (!rc) rc = tmp.alloc(n * sizeof(double2));
    for (int j = 0; !rc && j < d->k; ++j) {
        if (std::fread(host.data(), sizeof(double2), n, f) != (size_t)n) { rc = fail(DLZ_ERR_IO, "short read"); break; }
        if (cudaMemcpyAsync(tmp.p, host.data(), n * sizeof(double2), cudaMemcpyHostToDevice, op.stream) != cudaSuccess) { rc = fail(DLZ_ERR_CUDA, "upload"); break; }
        rc = pack64(op, d->V64.as<double2>() + (size_t)j * n, tmp.as<double2>());
        if (!rc && cudaStreamSynchronize(op.stream) != cudaSuccess) rc = fail(DLZ_ERR_CUDA, "sync");
    }
    std::fclose(f);
    if (!rc) rc = deflation_finish(op, d);
    if (rc) { delete d; return rc; }
    *out = d;
    return DLZ_OK;
}

int dlz_defl_destroy(dlz_defl_t d) {
    if (!d) return fail(DLZ_ERR_BADARG, "null deflation set");
    if (d->op) cudaStreamSynchronize(d->op->stream);
    delete d;
    return DLZ_OK;
}

}  // extern "C"
