// capi.cu -- the C ABI of libsap (declared in include/sap.h) and the engine
// behind it: device buffers of a handle, the launch sequence of one SAP
// iteration, CUDA-graph capture of the iteration loop, and kernel timing.
//
// One iteration (Algorithm 1 of Kvinge et al., arXiv:1807.03425):
//   plain form:         plain pass -> FP64 recheck -> update
//   restructured form:  Y = X U (tensor cores) -> restructured pass ->
//                       explicit-difference recheck -> FP64 recheck -> update
// Nothing returns to the host inside the loop; sap_run replays captured
// graphs of `chunk` iterations.
#include "sap_internal.cuh"
#include "restructured.cuh"
#include "softmin.cuh"
#include "sweep.cuh"
#include "tune.cuh"
#include "../../include/sap.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace sap;

namespace {

// NVTX range around a public call that launches work, so profiler timelines
// (ncu, Nsight Systems) show the library's stages by name; without a tool
// attached the calls cost next to nothing.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kClasses = 10;
// 6..9: soft-min forward pass, backward pass, near pairs, other (softmin.cu)
enum KClass { K_GEMM = 0, K_RESTR = 1, K_PLAIN = 2, K_EXPL = 3, K_FP64 = 4, K_UPDATE = 5 };

struct GraphEntry {
    cudaGraphExec_t exec;
    double alpha;
    int eval_only;
    int chunk;
    long long launches;   // kernels one replay launches (batch graphs)
};

double gamma_u(double m, double u) { return m * u / (1.0 - m * u); }

} // namespace

struct sap_ctx {
    int device = 0;
    int sms = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    bool sticky = false;

    int64_t N = 0;
    int n = 0;
    sap_dtype dt = SAP_F32;
    float *X32 = nullptr;
    double *X64 = nullptr;

    int k = 0, KP = 0;
    double *U64 = nullptr;
    float *U32 = nullptr;
    float *U32lo = nullptr;   // fl(U64 - U32), for the extended-precision recheck

    int2 *tiles = nullptr;   // plain-form point blocks
    int ntiles = 0;
    int2 *cand1 = nullptr, *cand2 = nullptr;
    long long cap = 0;
    Partial *partials = nullptr;
    double *work = nullptr;
    size_t work_elems = 0;
    ProbState *st = nullptr;
    double *hist = nullptr;
    int2 *am = nullptr;
    int hist_cap = 0;
    int last_iters = -1;

    sap_path path = SAP_PLAIN;
    sap_update_mode mode = SAP_UPDATE_LITERAL;
    sap_split split = SAP_SPLIT_FP16;
    double eps = 0.0;
    double eps2_f64 = 0.0;
    float eps2_lo = 0.f, eps2_hi = 0.f;
    int64_t n_excluded = 0;

    RestrState rs;           // restructured-form buffers (restructured.cuh)
    SoftState ss;            // soft-min buffers (softmin.cuh)
    SweepState *sw = nullptr; // dimension sweep (sweep.cuh)

    // uneven batch: one ordinary handle per dataset, run together
    bool is_batch = false;
    std::vector<sap_handle> kids;
    std::vector<cudaEvent_t> kid_done;
    cudaEvent_t fork = nullptr;

    cudaError_t inject = cudaSuccess;  // result forced on the next checked call (sap_inject_fault)

    long long launches = 0;
    std::vector<GraphEntry> graphs;
    long long graph_gen = 0;   // bumped whenever this handle's graphs are dropped
    long long kids_gen = -1;   // batch: sum of the datasets' graph_gen its graphs were made at

    // multi-GPU split: this handle is rank shard_rank of shard_world and
    // stores the tiles [shard_t0, shard_t1) of the row-major tile order
    int shard_world = 1, shard_rank = 0;
    long long shard_t0 = 0, shard_t1 = -1;
    Partial *shard_rec = nullptr;   // this rank's minimum (sap_shard_min)
    Partial *recs = nullptr;        // all ranks' records (sap_shard_step, host input)
    int shard_steps = 0;

    TuneParams tune;          // launch parameters (tune.cu)
    TuneKey tune_key;         // shape the parameters were last applied for
    bool tuning = false;      // the autotuner is timing this handle
    bool profiling = false;
    double ktime[kClasses] = {};
    long long kcount[kClasses] = {};
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

sap_status fail(sap_handle h, sap_status s, const std::string &msg)
{
    if (h) {
        h->err = msg;
        if (s == SAP_E_CUDA) h->sticky = true;
    }
    return s;
}

// A checked CUDA call of the engine; an error injected by sap_inject_fault
// replaces the next call's result.
#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (h->inject != cudaSuccess) {                                            \
            e_ = h->inject;                                                        \
            h->inject = cudaSuccess;                                               \
        }                                                                          \
        if (e_ != cudaSuccess)                                                     \
            return fail(h, e_ == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

#define CHECK_HANDLE(h)                                                            \
    do {                                                                           \
        if (!(h)) return SAP_E_ARG;                                                \
        if ((h)->sticky) return fail(h, SAP_E_CUDA, "handle has a sticky CUDA error: " + (h)->err); \
        (h)->err.clear();                                                          \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void **)p, count * sizeof(T));
}

template <typename T>
void dfree(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void drop_graphs(sap_handle h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    h->graph_gen++;
}

cudaEvent_t get_event(sap_handle h)
{
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Certified error models (see sap_internal.cuh and plain.cu).
Cert cert_plain_f32(int n, int k)
{
    const double u = std::ldexp(1.0, -24);
    Cert c;
    c.A = (float)(std::sqrt((double)k) * gamma_u(n + 3, u) * 1.05);
    c.rho = (float)((gamma_u(n + 2, u) + gamma_u(k, u) + 3 * u) * 1.05);
    return c;
}

Cert cert_plain_f64()
{
    Cert c;
    c.A = 1e-12f;
    c.rho = (float)(std::ldexp(1.0, -23) * 1.05);
    return c;
}

sap_status sync_and_status(sap_handle h)
{
    CK(cudaStreamSynchronize(h->stream));
    int status = 0;
    CK(cudaMemcpy(&status, &h->st->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        CK(cudaMemset(&h->st->status, 0, sizeof(int)));
        if (status & ST_BOUNDS) return fail(h, SAP_E_BOUNDS, "a device index was out of range (debug build)");
        if (status & ST_NO_SECANT) return fail(h, SAP_E_NO_SECANT, "every pair is excluded");
        if (status & ST_TIMEOUT) return fail(h, SAP_E_TIMEOUT, "a device-side wait gave up");
        if (status & ST_OVERFLOW)
            return fail(h, SAP_E_UNSUPPORTED, "candidate list overflow (too many near-ties)");
    }
    return SAP_OK;
}

// Launch bracket for kernel timing in profiling mode.
struct Timed {
    sap_handle h;
    int cls;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(sap_handle hh, int c) : h(hh), cls(c)
    {
        if (h->profiling) {
            a = get_event(h);
            b = get_event(h);
            cudaEventRecord(a, h->stream);
        }
        h->launches++;
    }
    ~Timed()
    {
        if (h->profiling) {
            cudaEventRecord(b, h->stream);
            h->pending.push_back({cls, a, b});
        }
    }
};

// Arguments of the FP64 recheck + update over candidate list `list`
// (count in st->cnt<which>), without the fused-tier fields.
SelectUpdateArgs su_args(sap_handle h, double alpha, int eval_only, const int2 *list, int which)
{
    const bool f64 = h->dt == SAP_F64;
    SelectUpdateArgs u;
    u.X = f64 ? (const void *)h->X64 : (const void *)h->X32;
    u.x_is_f64 = f64; u.N = (int)h->N; u.n = h->n;
    u.U64 = h->U64; u.U32 = h->U32; u.U32lo = h->U32lo; u.KP = h->KP;
    u.Uhi = h->rs.Uhi; u.Ulo = h->rs.Ulo; u.NP = h->rs.NP;
    u.split_bf16 = h->split == SAP_SPLIT_BF16; u.split_scale = h->split == SAP_SPLIT_BF16 ? 256.f : 2048.f;
    u.k = h->k; u.alpha = alpha; u.mode = (int)h->mode; u.eval_only = eval_only;
    u.eps2 = h->eps2_f64; u.list = list; u.cap = (unsigned int)h->cap; u.which = which;
    u.partials = h->partials;
    u.grid = std::min(h->tune.su_blocks > 0 ? h->tune.su_blocks : h->sms, kRecheckBlocks);
    u.work = h->work; u.st = h->st; u.hist = h->hist; u.argmin = h->am; u.seed_cert = cert_plain_f32(h->n, h->k);
    u.pdl = h->tune.pdl;
    u.fused = 0; u.near = nullptr; u.n_near = 0; u.cert2 = u.seed_cert;
    return u;
}

sap_status enqueue_iteration(sap_handle h, double alpha, int eval_only, Partial *shard_rec = nullptr)
{
    cudaStream_t s = h->stream;
    const Cert c32 = cert_plain_f32(h->n, h->k);
    const bool f64 = h->dt == SAP_F64;
    int which = 1;
    const int2 *list = h->cand1;
    if (h->path == SAP_PLAIN) {
        if (f64) {
            PlainArgsF64 a;
            a.X = h->X64; a.N = (int)h->N; a.n = h->n; a.U64 = h->U64; a.k = h->k;
            a.tiles = h->tiles; a.ntiles = h->ntiles;
            a.grid = std::min(h->ntiles, 2 * std::max(1, h->tune.plain_per_sm) * h->sms);
            a.eps2 = h->eps2_f64; a.cert = cert_plain_f64(); a.st = h->st;
            a.cand = h->cand1; a.cand_cap = h->cap;
            Timed t(h, K_PLAIN);
            CK(launch_plain_f64(a, s));
        } else {
            PlainArgsF32 a;
            a.X = h->X32; a.N = (int)h->N; a.n = h->n; a.U32 = h->U32; a.k = h->k; a.KP = h->KP;
            a.tiles = h->tiles; a.ntiles = h->ntiles;
            a.grid = std::min(h->ntiles, std::max(1, h->tune.plain_per_sm) * h->sms);
            a.eps2_lo = h->eps2_lo; a.eps2_hi = h->eps2_hi; a.cert = c32; a.st = h->st;
            a.cand = h->cand1; a.cand_cap = h->cap;
            Timed t(h, K_PLAIN);
            CK(launch_plain_f32(a, s));
        }
    } else {
        sap_status st = restructured_enqueue(h, alpha);
        if (st != SAP_OK) return st;
        which = 2;
        list = h->cand2;
    }
    {
        SelectUpdateArgs u = su_args(h, alpha, eval_only, list, which);
        u.shard_rec = shard_rec;
        if (h->path != SAP_PLAIN) {
            u.seeds_in_product = 1;  // the next iteration's product evaluates them
            BasisView bv;
            bv.k = h->k;
            bv.cand1 = h->cand1;
            bv.cand2 = h->cand2;
            restructured_fuse_args(h, bv, u);
        }
        Timed t(h, K_UPDATE);
        CK(launch_select_update(u, s));
    }
    return SAP_OK;
}

sap_status reset_state(sap_handle h)
{
    ProbState p;
    std::memset(&p, 0, sizeof(p));
    p.seed_ub = 0x7f800000u;
    p.run_ub1 = 0x7f800000u;
    p.run_ub2 = 0x7f800000u;
    p.hist_cap = h->hist_cap;
    p.last_r = INFINITY;
    p.last_i = p.last_j = -1;
    CK(cudaMemcpyAsync(h->st, &p, sizeof(p), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SAP_OK;
}

sap_status ensure_hist(sap_handle h, int need)
{
    if (h->hist_cap >= need) return SAP_OK;
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    dfree(h->hist);
    dfree(h->am);
    int cap = std::max(need, 1024);
    CK(dalloc(&h->hist, cap));
    CK(dalloc(&h->am, cap));
    h->hist_cap = cap;
    CK(cudaMemcpy(&h->st->hist_cap, &cap, sizeof(int), cudaMemcpyHostToDevice));
    return SAP_OK;
}

sap_status set_eps(sap_handle h, double eps)
{
    h->eps = eps;
    h->eps2_f64 = eps * eps;
    if (eps > 0.0) {
        const double m = 4.0 * gamma_u(h->n + 2, std::ldexp(1.0, -24)) + 1e-6;
        h->eps2_lo = std::nextafter((float)(h->eps2_f64 * (1.0 - m)), 0.f);
        h->eps2_hi = std::nextafter((float)(h->eps2_f64 * (1.0 + m)), INFINITY);
    } else {
        h->eps2_lo = h->eps2_hi = 0.f;
    }
    return SAP_OK;
}

__global__ void bf16_to_f32_kernel(const uint16_t *in, float *out, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = __uint_as_float(((unsigned int)in[i]) << 16);
}

sap_status build_tiles(sap_handle h, int edge)
{
    const int nb = (int)((h->N + edge - 1) / edge);
    std::vector<int2> t;
    t.reserve((size_t)nb * (nb + 1) / 2);
    for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J) t.push_back(make_int2(I, J));
    dfree(h->tiles);
    CK(dalloc(&h->tiles, t.size()));
    CK(cudaMemcpy(h->tiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice));
    h->ntiles = (int)t.size();
    return SAP_OK;
}

} // namespace

// Accessors used by restructured.cu (kept here so the handle layout stays
// private to this file).
namespace sap {
RestrState &restr_state(sap_handle h) { return h->rs; }
cudaStream_t handle_stream(sap_handle h) { return h->stream; }
int handle_sms(sap_handle h) { return h->sms; }
ProbState *handle_state(sap_handle h) { return h->st; }
const float *handle_x32(sap_handle h) { return h->X32; }
const double *handle_x64(sap_handle h) { return h->X64; }
sap_status secant_pca(sap_handle h, int k, double *U_out, double *sigma_out);  // pca.cu
const float *handle_u32(sap_handle h) { return h->U32; }
const float *handle_u32lo(sap_handle h) { return h->U32lo; }
int2 *handle_cand1(sap_handle h) { return h->cand1; }
int2 *handle_cand2(sap_handle h) { return h->cand2; }
long long handle_cap(sap_handle h) { return h->cap; }
int handle_k(sap_handle h) { return h->k; }
int handle_kp(sap_handle h) { return h->KP; }
int64_t handle_n_points(sap_handle h) { return h->N; }
int handle_n_dim(sap_handle h) { return h->n; }
int handle_split_bf16(sap_handle h) { return h->split == SAP_SPLIT_BF16; }
double handle_eps2(sap_handle h) { return h->eps2_f64; }
float handle_eps2_lo(sap_handle h) { return h->eps2_lo; }
float handle_eps2_hi(sap_handle h) { return h->eps2_hi; }
void handle_count_launch(sap_handle h, int cls, cudaEvent_t *a, cudaEvent_t *b)
{
    h->launches++;
    if (h->profiling) {
        *a = get_event(h);
        *b = get_event(h);
    } else {
        *a = *b = nullptr;
    }
    (void)cls;
}
void handle_push_timing(sap_handle h, int cls, cudaEvent_t a, cudaEvent_t b)
{
    if (a) h->pending.push_back({cls, a, b});
}
sap_status handle_fail(sap_handle h, sap_status s, const char *msg) { return fail(h, s, msg); }
SoftState &soft_state(sap_handle h) { return h->ss; }
double *handle_u64(sap_handle h) { return h->U64; }
Partial *handle_partials(sap_handle h) { return h->partials; }
float *handle_u32_mut(sap_handle h) { return h->U32; }
sap_status handle_reset_state(sap_handle h) { return reset_state(h); }
int handle_profiling(sap_handle h) { return h->profiling ? 1 : 0; }
long long handle_launches(sap_handle h) { return h->launches; }
SweepState *&sweep_state(sap_handle h) { return h->sw; }
long long handle_graph_gen(sap_handle h) { return h->graph_gen; }
TuneParams &handle_tune(sap_handle h) { return h->tune; }
TuneKey handle_tune_key(sap_handle h)
{
    TuneKey t;
    t.N = h->N;
    t.n = h->n;
    t.k = h->k;
    t.dt = (int)h->dt;
    t.path = (int)h->path;
    t.split = (int)h->split;
    std::memcpy(&t.eps_bits, &h->eps, sizeof(double));
    return t;
}
bool &handle_tuning_flag(sap_handle h) { return h->tuning; }
void handle_shard(sap_handle h, long long *t0, long long *t1)
{
    *t0 = h->shard_world > 1 ? h->shard_t0 : 0;
    *t1 = h->shard_world > 1 ? h->shard_t1 : -1;
}
TuneKey &handle_applied_key(sap_handle h) { return h->tune_key; }
void handle_drop_graphs(sap_handle h) { drop_graphs(h); }
bool handle_path_restructured(sap_handle h) { return h->path == SAP_RESTRUCTURED && h->dt != SAP_F64; }
int handle_mode(sap_handle h) { return (int)h->mode; }
Cert handle_seed_cert(int n, int k) { return cert_plain_f32(n, k); }
sap_status handle_check_status(sap_handle h, ProbState *st)
{
    int status = 0;
    CK(cudaMemcpy(&status, &st->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        CK(cudaMemset(&st->status, 0, sizeof(int)));
        if (status & ST_BOUNDS) return fail(h, SAP_E_BOUNDS, "a device index was out of range (debug build)");
        if (status & ST_NO_SECANT) return fail(h, SAP_E_NO_SECANT, "every pair is excluded");
        if (status & ST_TIMEOUT) return fail(h, SAP_E_TIMEOUT, "a device-side wait gave up");
        if (status & ST_OVERFLOW) return fail(h, SAP_E_UNSUPPORTED, "candidate list overflow (too many near-ties)");
    }
    return SAP_OK;
}
void handle_add_launches(sap_handle h, long long delta) { h->launches += delta; }
} // namespace sap

extern "C" {

const char *sap_version(void) { return "libsap 0.2 (sm_103a)"; }

sap_status sap_inject_fault(sap_handle h, int32_t kind)
{
    if (!h || (kind != 1 && kind != 2)) return SAP_E_ARG;
    h->inject = kind == 1 ? cudaErrorMemoryAllocation : cudaErrorLaunchFailure;
    return SAP_OK;
}

namespace {
// Waits on an mbarrier that nothing arrives on, with the library's bounded
// wait; records whether the wait gave up.
__global__ void selftest_wait_kernel(long long budget, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long t0 = clock64();
    bool done = false;
    while (!done) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(a) : "memory");
        if (ok) done = true;
        else if (clock64() - t0 > budget) break;
    }
    *status = done ? 0 : ST_TIMEOUT;
}
} // namespace

sap_status sap_selftest_wait(void *cuda_stream, int64_t budget_cycles)
{
    if (budget_cycles < 0 || budget_cycles > 4000000000ll) return SAP_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return SAP_E_NO_DEVICE;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return SAP_E_OOM;
    int status = -1;
    selftest_wait_kernel<<<1, 1, 0, s>>>((long long)budget_cycles, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return SAP_E_CUDA;
    return status == 0 ? SAP_OK : SAP_E_TIMEOUT;
}

const char *sap_status_str(sap_status s)
{
    switch (s) {
    case SAP_OK: return "SAP_OK";
    case SAP_E_ARG: return "SAP_E_ARG";
    case SAP_E_STATE: return "SAP_E_STATE";
    case SAP_E_NOT_ORTHONORMAL: return "SAP_E_NOT_ORTHONORMAL";
    case SAP_E_NO_SECANT: return "SAP_E_NO_SECANT";
    case SAP_E_OOM: return "SAP_E_OOM";
    case SAP_E_CUDA: return "SAP_E_CUDA";
    case SAP_E_TIMEOUT: return "SAP_E_TIMEOUT";
    case SAP_E_NO_DEVICE: return "SAP_E_NO_DEVICE";
    case SAP_E_UNSUPPORTED: return "SAP_E_UNSUPPORTED";
    case SAP_E_BOUNDS: return "SAP_E_BOUNDS";
    }
    return "SAP_E_UNKNOWN";
}

const char *sap_last_error(sap_handle h) { return h ? h->err.c_str() : "null handle"; }

sap_status sap_destroy(sap_handle h)
{
    if (!h) return SAP_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);  // before the datasets whose buffers the graphs name
    for (sap_handle k : h->kids) sap_destroy(k);
    h->kids.clear();
    for (cudaEvent_t e : h->kid_done) cudaEventDestroy(e);
    h->kid_done.clear();
    if (h->fork) cudaEventDestroy(h->fork);
    drop_graphs(h);
    for (auto &p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    restructured_free(h);
    softmin_free(h);
    sweep_free(h->sw);
    dfree(h->X32); dfree(h->X64); dfree(h->U64); dfree(h->U32); dfree(h->U32lo);
    dfree(h->shard_rec); dfree(h->recs);
    dfree(h->tiles); dfree(h->cand1); dfree(h->cand2); dfree(h->partials);
    dfree(h->work); dfree(h->st); dfree(h->hist); dfree(h->am);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return SAP_OK;
}

static sap_status create_impl(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device, int32_t world,
                              int32_t rank, sap_handle *out)
{
    TraceRange trace("sap_create");
    if (!out) return SAP_E_ARG;
    *out = nullptr;
    if (!X || N < 2 || N > 92681 || n < 1 || n > 16384) return SAP_E_ARG;
    if (dt != SAP_F32 && dt != SAP_BF16 && dt != SAP_F64) return SAP_E_ARG;
    long long t0 = 0, t1 = -1;
    if (world > 1) {
        if (dt == SAP_F64) return SAP_E_UNSUPPORTED;  // the split covers the restructured form
        int64_t a = 0, b = 0, pairs = 0;
        if (sap_shard_range(N, world, rank, &a, &b, &pairs) != SAP_OK || b <= a) return SAP_E_ARG;
        t0 = a;
        t1 = b;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return SAP_E_NO_DEVICE;
    }
    sap_handle h = new sap_ctx();
    h->N = N; h->n = n; h->dt = dt;
    if (world > 1) {
        h->shard_world = world;
        h->shard_rank = rank;
        h->shard_t0 = t0;
        h->shard_t1 = t1;
    }
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
    if (x_is_device) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, X) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
            pa.device != h->device) {
            cudaGetLastError();
            delete h;
            return SAP_E_ARG;
        }
    }
    auto cleanup_fail = [&](sap_status s) { sap_destroy(h); return s; };
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup_fail(SAP_E_CUDA);
    h->own_stream = true;

    const size_t cnt = (size_t)N * n;
    sap_status st = SAP_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && st == SAP_OK)
            st = e == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA;
    };
    const cudaMemcpyKind kind = x_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (dt == SAP_F64) {
        chk(dalloc(&h->X64, cnt));
        if (st == SAP_OK) chk(cudaMemcpy(h->X64, X, cnt * sizeof(double), kind));
        h->path = SAP_PLAIN;
    } else {
        chk(dalloc(&h->X32, cnt));
        if (st == SAP_OK && dt == SAP_F32) chk(cudaMemcpy(h->X32, X, cnt * sizeof(float), kind));
        if (st == SAP_OK && dt == SAP_BF16) {
            uint16_t *tmp = nullptr;
            chk(dalloc(&tmp, cnt));
            if (st == SAP_OK) chk(cudaMemcpy(tmp, X, cnt * sizeof(uint16_t), kind));
            if (st == SAP_OK) {
                bf16_to_f32_kernel<<<4 * h->sms, 256, 0, h->stream>>>(tmp, h->X32, cnt);
                chk(cudaGetLastError());
                chk(cudaStreamSynchronize(h->stream));
            }
            dfree(tmp);
        }
        h->path = SAP_RESTRUCTURED;
    }
    const long long P = (long long)N * (N - 1) / 2;
    h->cap = std::min<long long>(P + 64, 1ll << 26);
    chk(dalloc(&h->cand1, (size_t)h->cap));
    chk(dalloc(&h->partials, kRecheckBlocks));
    chk(dalloc(&h->st, 1));
    if (st != SAP_OK) return cleanup_fail(st);
    if (ensure_hist(h, 1024) != SAP_OK) return cleanup_fail(SAP_E_CUDA);
    if (build_tiles(h, dt == SAP_F64 ? 16 : 64) != SAP_OK) return cleanup_fail(SAP_E_CUDA);
    set_eps(h, 0.0);
    if (dt != SAP_F64) {
        chk(dalloc(&h->cand2, (size_t)h->cap));
        if (st != SAP_OK) return cleanup_fail(st);
        sap_status rs = restructured_prepare(h);
        if (rs != SAP_OK) return cleanup_fail(rs);
    }
    if (world > 1) {
        chk(dalloc(&h->shard_rec, 1));
        chk(dalloc(&h->recs, 4096));
        if (st != SAP_OK) return cleanup_fail(st);
    }
    if (reset_state(h) != SAP_OK) return cleanup_fail(SAP_E_CUDA);
    *out = h;
    return SAP_OK;
}

sap_status sap_create(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device, sap_handle *out)
{
    return create_impl(X, N, n, dt, x_is_device, 1, 0, out);
}

sap_status sap_create_shard(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device, int32_t world,
                            int32_t rank, sap_handle *out)
{
    if (world < 1 || world > 4096 || rank < 0 || rank >= world) return SAP_E_ARG;
    return create_impl(X, N, n, dt, x_is_device, world, rank, out);
}

// Batch handles forward the dataset-wide settings to every dataset; calls
// that act on one basis need the _b variants.
#define FORWARD_BATCH(h, call)                                        \
    do {                                                              \
        if ((h)->is_batch) {                                          \
            for (size_t b_ = 0; b_ < (h)->kids.size(); ++b_) {        \
                sap_handle kid = (h)->kids[b_];                       \
                const sap_status s_ = (call);                         \
                if (s_ != SAP_OK) {                                   \
                    (h)->err = "dataset " + std::to_string(b_) + ": " + kid->err; \
                    return s_;                                        \
                }                                                     \
            }                                                         \
            return SAP_OK;                                            \
        }                                                             \
    } while (0)

#define NOT_SHARD(h)                                                                 \
    do {                                                                             \
        if ((h)->shard_world > 1)                                                    \
            return fail(h, SAP_E_STATE, "shard handle: use sap_shard_min / sap_shard_step"); \
    } while (0)

#define NOT_BATCH(h)                                                                 \
    do {                                                                             \
        if ((h)->is_batch) return fail(h, SAP_E_STATE, "batch handle: use the _b calls"); \
    } while (0)

sap_status sap_set_stream(sap_handle h, void *cuda_stream)
{
    CHECK_HANDLE(h);
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
        h->own_stream = false;
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    return SAP_OK;
}

sap_status sap_set_path(sap_handle h, sap_path p)
{
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_path(kid, p));
    if (p != SAP_PLAIN && p != SAP_RESTRUCTURED) return fail(h, SAP_E_ARG, "unknown path");
    if (p == SAP_PLAIN && h->shard_world > 1)
        return fail(h, SAP_E_UNSUPPORTED, "the split covers the restructured form only");
    if (p == SAP_RESTRUCTURED && h->dt == SAP_F64)
        return fail(h, SAP_E_UNSUPPORTED, "the restructured form needs FP32 or BF16 data");
    if (p == SAP_PLAIN && h->dt != SAP_F64 && h->k > 8)
        return fail(h, SAP_E_UNSUPPORTED, "the FP32 plain form supports k <= 8");
    if (p != h->path) drop_graphs(h);
    h->path = p;
    return tune_lookup(h);
}

sap_status sap_set_update_mode(sap_handle h, sap_update_mode m)
{
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_update_mode(kid, m));
    if (m != SAP_UPDATE_LITERAL && m != SAP_UPDATE_ANGLE) return fail(h, SAP_E_ARG, "unknown mode");
    if (m != h->mode) drop_graphs(h);
    h->mode = m;
    return SAP_OK;
}

sap_status sap_set_split(sap_handle h, sap_split s)
{
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_split(kid, s));
    if (s != SAP_SPLIT_FP16 && s != SAP_SPLIT_BF16) return fail(h, SAP_E_ARG, "unknown split");
    if (h->dt == SAP_F64) return fail(h, SAP_E_UNSUPPORTED, "no tensor-core product for FP64 data");
    if (s == h->split) return SAP_OK;
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->split = s;
    sap_status st = restructured_prepare(h);
    if (st != SAP_OK || h->k == 0) return st;
    // re-split the current basis for the new operand type
    std::vector<double> Uh((size_t)h->n * h->k);
    CK(cudaMemcpy(Uh.data(), h->U64, Uh.size() * sizeof(double), cudaMemcpyDeviceToHost));
    st = restructured_upload_basis(h, Uh.data());
    if (st != SAP_OK) return st;
    return tune_lookup(h);
}

sap_status sap_set_min_secant_length(sap_handle h, double eps)
{
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_min_secant_length(kid, eps));
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(h, SAP_E_ARG, "eps must be finite and >= 0");
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    set_eps(h, eps);
    if (h->dt != SAP_F64) {
        sap_status s = restructured_prepare(h);
        if (s != SAP_OK) return s;
    }
    sap_status s = tune_lookup(h);
    if (s != SAP_OK) return s;
    return reset_state(h);
}

sap_status sap_secant_pca(sap_handle h, int32_t k, double *U_out, double *sigma_out)
{
    TraceRange trace("sap_secant_pca");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    std::vector<double> U((size_t)h->n * std::max(k, 1));
    sap_status s = secant_pca(h, k, U.data(), sigma_out);
    if (s != SAP_OK) return s;
    s = sap_set_basis(h, U.data(), k, 0);
    if (s != SAP_OK) return s;
    if (U_out) std::memcpy(U_out, U.data(), U.size() * sizeof(double));
    return SAP_OK;
}

sap_status sap_set_pass_bound(sap_handle h, double b_cap)
{
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_pass_bound(kid, b_cap));
    if (!(b_cap >= 1e-6 && b_cap <= 0.25)) return fail(h, SAP_E_ARG, "b_cap must be in [1e-6, 0.25]");
    if (h->dt == SAP_F64) return fail(h, SAP_E_UNSUPPORTED, "no restructured form for FP64 data");
    CK(cudaStreamSynchronize(h->stream));
    TuneParams p = h->tune;
    p.b_cap = b_cap;
    p.us_per_iter = 0;
    return tune_apply(h, p);
}

static void to_public(const TuneParams &p, sap_tuning *out)
{
    out->pass_bound = p.b_cap;
    out->pass_stages = p.pass_stages;
    out->explicit_blocks_per_sm = p.expl_per_sm;
    out->update_blocks = p.su_blocks;
    out->plain_blocks_per_sm = p.plain_per_sm;
    out->programmatic_launch = p.pdl;
    out->refine_tier = p.refine;
    out->us_per_iteration = p.us_per_iter;
}

sap_status sap_get_tuning(sap_handle h, sap_tuning *out)
{
    CHECK_HANDLE(h);
    if (!out) return fail(h, SAP_E_ARG, "null output");
    to_public(h->is_batch ? h->kids[0]->tune : h->tune, out);  // a batch: its first dataset's
    return SAP_OK;
}

sap_status sap_set_tuning(sap_handle h, const sap_tuning *in)
{
    CHECK_HANDLE(h);
    if (!in) return fail(h, SAP_E_ARG, "null input");
    FORWARD_BATCH(h, sap_set_tuning(kid, in));
    if (!(in->pass_bound >= 1e-6 && in->pass_bound <= 0.25) || in->pass_stages < 0 || in->pass_stages > 5 ||
        in->explicit_blocks_per_sm < 1 || in->explicit_blocks_per_sm > 8 || in->update_blocks < 0 ||
        in->update_blocks > kRecheckBlocks || in->plain_blocks_per_sm < 1 || in->plain_blocks_per_sm > 8 ||
        (in->programmatic_launch != 0 && in->programmatic_launch != 1) || in->refine_tier < -1 ||
        in->refine_tier > 5)
        return fail(h, SAP_E_ARG, "tuning parameter out of range");
    CK(cudaStreamSynchronize(h->stream));
    TuneParams p;
    p.b_cap = in->pass_bound;
    p.pass_stages = in->pass_stages;
    p.expl_per_sm = in->explicit_blocks_per_sm;
    p.su_blocks = in->update_blocks;
    p.plain_per_sm = in->plain_blocks_per_sm;
    p.pdl = in->programmatic_launch;
    p.refine = in->refine_tier;
    p.us_per_iter = 0;
    return tune_apply(h, p);
}

// Batch handles: one parameter set for every dataset, chosen by timing whole
// batch iterations (the datasets run concurrently, so what matters is the
// batch's time, not each dataset's alone): coordinate descent over the same
// parameters as the single-handle tuner, from the first dataset's current
// set.  The bases are restored afterwards (iteration counters restart).
static sap_status tune_batch(sap_handle h, double alpha, int iters)
{
    const size_t B = h->kids.size();
    std::vector<std::vector<double>> U(B);
    for (size_t b = 0; b < B; ++b) {
        sap_handle kid = h->kids[b];
        if (kid->k == 0) return fail(h, SAP_E_STATE, "dataset " + std::to_string(b) + " has no basis");
        U[b].resize((size_t)kid->n * kid->k);
        sap_status st = sap_get_basis_b(h, (int32_t)b, U[b].data(), 0);
        if (st != SAP_OK) return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(h, SAP_E_CUDA, "autotune: event creation failed");
    }
    for (sap_handle kid : h->kids) kid->tuning = true;
    sap_status st = SAP_OK;
    auto restore = [&]() -> sap_status {
        for (size_t b = 0; b < B; ++b) {
            sap_status r = sap_set_basis_b(h, (int32_t)b, U[b].data(), h->kids[b]->k, 0);
            if (r != SAP_OK) return r;
        }
        return SAP_OK;
    };
    auto timed = [&](const TuneParams &c, double *us) -> sap_status {
        for (sap_handle kid : h->kids) {
            sap_status r = tune_apply(kid, c);
            if (r != SAP_OK) return fail(h, r, kid->err);
        }
        double best = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            sap_status r = restore();
            if (r != SAP_OK) return r;
            if (rep > 0 && cudaEventRecord(e0, h->stream) != cudaSuccess) return fail(h, SAP_E_CUDA, "event");
            r = sap_run_batch(h, alpha, iters, nullptr, nullptr);
            if (r != SAP_OK) return r;
            if (rep > 0) {
                if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                    return fail(h, SAP_E_CUDA, "event");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::fmin(best, 1e3 * ms / iters);
            }
        }
        *us = best;
        return SAP_OK;
    };
    TuneParams best = h->kids[0]->tune;
    double best_us = INFINITY;
    st = timed(best, &best_us);
    auto consider = [&](TuneParams c) {
        if (st != SAP_OK || tune_same_launch(c, best)) return;
        double us = INFINITY;
        st = timed(c, &us);
        if (st == SAP_OK && us < best_us) {
            best = c;
            best_us = us;
        }
    };
    if (handle_path_restructured(h->kids[0])) {
        for (int rf : {0, 1, 5, 2, 3, 4}) { TuneParams c = best; c.refine = rf; consider(c); }
        for (int pdl : {0, 1}) { TuneParams c = best; c.pdl = pdl; consider(c); }
        for (double b : {5e-4, 1e-3, 2e-3, 4e-3, 8e-3}) { TuneParams c = best; c.b_cap = b; consider(c); }
        for (int stg : {0, 2, 3}) { TuneParams c = best; c.pass_stages = stg; consider(c); }
        for (int e : {1, 2, 4}) { TuneParams c = best; c.expl_per_sm = e; consider(c); }
    } else {
        for (int p : {1, 2, 4}) { TuneParams c = best; c.plain_per_sm = p; consider(c); }
    }
    for (int sb : {38, 76, 152}) { TuneParams c = best; c.su_blocks = sb; consider(c); }
    if (handle_path_restructured(h->kids[0])) {  // a second look (see tune_handle)
        for (int pdl : {0, 1}) { TuneParams c = best; c.pdl = pdl; consider(c); }
        for (int stg : {0, 2, 3}) { TuneParams c = best; c.pass_stages = stg; consider(c); }
    }
    if (st == SAP_OK) {
        best.us_per_iter = best_us;
        for (sap_handle kid : h->kids) {
            sap_status r = tune_apply(kid, best);
            if (r != SAP_OK && st == SAP_OK) st = fail(h, r, kid->err);
        }
    }
    const sap_status rs = restore();
    if (st == SAP_OK) st = rs;
    for (sap_handle kid : h->kids) kid->tuning = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

sap_status sap_autotune(sap_handle h, double alpha, int32_t iters, sap_tuning *out)
{
    TraceRange trace("sap_autotune");
    CHECK_HANDLE(h);
    NOT_SHARD(h);
    if (h->is_batch) {
        if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
        if (iters < 1 || iters > 4096) return fail(h, SAP_E_ARG, "iters must be in [1, 4096]");
        sap_status st = tune_batch(h, alpha, iters);
        if (st != SAP_OK) return st;
        if (out) to_public(h->kids[0]->tune, out);
        return SAP_OK;
    }
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
    if (iters < 1 || iters > 4096) return fail(h, SAP_E_ARG, "iters must be in [1, 4096]");
    sap_status st = tune_handle(h, alpha, iters);
    if (st != SAP_OK) return st;
    if (out) to_public(h->tune, out);
    return SAP_OK;
}

sap_status sap_set_basis(sap_handle h, const double *U, int32_t k, int u_is_device)
{
    TraceRange trace("sap_set_basis");
    CHECK_HANDLE(h);
    FORWARD_BATCH(h, sap_set_basis(kid, U, k, u_is_device));
    if (!U || k < 1 || k > kMaxK || k > h->n) return fail(h, SAP_E_ARG, "need 1 <= k <= min(n, 32)");
    if (h->path == SAP_PLAIN && h->dt != SAP_F64 && k > 8)
        return fail(h, SAP_E_UNSUPPORTED, "the FP32 plain form supports k <= 8");
    const int n = h->n;
    std::vector<double> Uh((size_t)n * k);
    if (u_is_device) {
        CK(cudaMemcpy(Uh.data(), U, Uh.size() * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(Uh.data(), U, Uh.size() * sizeof(double));
    }
    double dev = 0.0;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += Uh[(size_t)a * n + l] * Uh[(size_t)b * n + l];
            dev = std::max(dev, std::fabs(s - (a == b ? 1.0 : 0.0)));
        }
    if (!(dev <= 1e-10)) return fail(h, SAP_E_NOT_ORTHONORMAL, "max |U^T U - I| > 1e-10");
    CK(cudaStreamSynchronize(h->stream));
    if (k != h->k) {
        drop_graphs(h);
        dfree(h->U64); dfree(h->U32); dfree(h->U32lo); dfree(h->work);
        h->k = k;
        h->KP = padded_stride(k);  // pad columns stay zero
        CK(dalloc(&h->U64, (size_t)n * k));
        CK(dalloc(&h->U32, (size_t)n * h->KP));
        CK(dalloc(&h->U32lo, (size_t)n * h->KP));
        h->work_elems = (size_t)(kMaxK + 1) * n;
        CK(dalloc(&h->work, h->work_elems));
        if (h->dt != SAP_F64) {
            sap_status s = restructured_basis_alloc(h);
            if (s != SAP_OK) return s;
        }
    }
    CK(cudaMemcpy(h->U64, Uh.data(), Uh.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<float> u32((size_t)n * h->KP, 0.f), u32lo((size_t)n * h->KP, 0.f);
    for (int l = 0; l < n; ++l)
        for (int c = 0; c < k; ++c) {
            const double v = Uh[(size_t)c * n + l];
            const float f = (float)v;
            u32[(size_t)l * h->KP + c] = f;
            u32lo[(size_t)l * h->KP + c] = (float)(v - (double)f);
        }
    CK(cudaMemcpy(h->U32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->U32lo, u32lo.data(), u32lo.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (h->dt != SAP_F64) {
        sap_status s = restructured_upload_basis(h, Uh.data());
        if (s != SAP_OK) return s;
    }
    sap_status s = tune_lookup(h);
    if (s != SAP_OK) return s;
    h->shard_steps = 0;
    return reset_state(h);
}

sap_status sap_get_basis(sap_handle h, double *U_out, int out_is_device)
{
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    if (!U_out) return fail(h, SAP_E_ARG, "null output");
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    CK(cudaMemcpyAsync(U_out, h->U64, (size_t)h->n * h->k * sizeof(double),
                       out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SAP_OK;
}

static sap_status read_last(sap_handle h, int64_t *i, int64_t *j, double *ratio)
{
    sap_status s = sync_and_status(h);
    if (s != SAP_OK) return s;
    ProbState p;
    CK(cudaMemcpy(&p, h->st, sizeof(p), cudaMemcpyDeviceToHost));
    if (i) *i = p.last_i;
    if (j) *j = p.last_j;
    if (ratio) *ratio = p.last_r;
    return SAP_OK;
}

sap_status sap_min_secant(sap_handle h, int64_t *i, int64_t *j, double *ratio)
{
    TraceRange trace("sap_min_secant");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    sap_status s = enqueue_iteration(h, 0.0, 1);
    if (s != SAP_OK) return s;
    return read_last(h, i, j, ratio);
}

sap_status sap_step(sap_handle h, double alpha, int64_t *i, int64_t *j, double *ratio)
{
    TraceRange trace("sap_step");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
    sap_status s = enqueue_iteration(h, alpha, 0);
    if (s != SAP_OK) return s;
    if (i || j || ratio) return read_last(h, i, j, ratio);
    return SAP_OK;
}

// ---------------------------------------------------------------- shards --

static_assert(sizeof(sap_record) == sizeof(Partial), "a record is the recheck's (q, i, j)");

// The ranks' records to the candidate list of the FP64 recheck (its count in
// st->cnt1); records without a pair are skipped.
__global__ void records_to_list_kernel(const Partial *recs, int count, int2 *list, ProbState *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int c = 0;
        for (int e = 0; e < count; ++e)
            if (recs[e].i >= 0) list[c++] = make_int2(recs[e].i, recs[e].j);
        st->cnt1 = c;
    }
}

sap_status sap_shard_min(sap_handle h, sap_record *rec_out, int out_is_device)
{
    TraceRange trace("sap_shard_min");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    if (h->shard_world <= 1) return fail(h, SAP_E_STATE, "not a shard handle (sap_create_shard)");
    if (!rec_out) return fail(h, SAP_E_ARG, "rec_out is NULL");
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    sap_status s = enqueue_iteration(h, 0.0, 1, h->shard_rec);
    if (s != SAP_OK) return s;
    if (out_is_device) {
        CK(cudaMemcpyAsync(rec_out, h->shard_rec, sizeof(sap_record), cudaMemcpyDeviceToDevice, h->stream));
        return SAP_OK;
    }
    CK(cudaMemcpyAsync(rec_out, h->shard_rec, sizeof(sap_record), cudaMemcpyDeviceToHost, h->stream));
    return sync_and_status(h);
}

sap_status sap_shard_step(sap_handle h, double alpha, const sap_record *recs, int32_t count, int recs_is_device)
{
    TraceRange trace("sap_shard_step");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    if (h->shard_world <= 1) return fail(h, SAP_E_STATE, "not a shard handle (sap_create_shard)");
    if (!recs || count < 1 || count > 4096 || count > h->cap) return fail(h, SAP_E_ARG, "1 <= count <= 4096 records");
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
    // the history grows by one entry per step, keeping what it holds
    if (h->shard_steps + 1 > h->hist_cap) {
        const int cap = 2 * h->hist_cap;
        double *nh = nullptr;
        int2 *na = nullptr;
        CK(dalloc(&nh, cap));
        CK(dalloc(&na, cap));
        CK(cudaMemcpyAsync(nh, h->hist, (size_t)h->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(na, h->am, (size_t)h->hist_cap * sizeof(int2), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(&h->st->hist_cap, &cap, sizeof(int), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        dfree(h->hist);
        dfree(h->am);
        h->hist = nh;
        h->am = na;
        h->hist_cap = cap;
    }
    const Partial *src = reinterpret_cast<const Partial *>(recs);
    if (!recs_is_device) {
        CK(cudaMemcpyAsync(h->recs, recs, (size_t)count * sizeof(sap_record), cudaMemcpyHostToDevice, h->stream));
        src = h->recs;
    }
    records_to_list_kernel<<<1, 32, 0, h->stream>>>(src, count, h->cand1, h->st);
    CK(cudaGetLastError());
    h->launches++;
    SelectUpdateArgs u = su_args(h, alpha, 0, h->cand1, 1);
    u.grid = 1;  // a few pairs: one block rechecks them and updates
    u.pdl = 0;
    u.seeds_in_product = 1;  // a split handle is restructured: its product evaluates them
    {
        Timed t(h, K_UPDATE);
        CK(launch_select_update(u, h->stream));
    }
    h->shard_steps++;
    h->last_iters = h->shard_steps - 1;
    if (!recs_is_device) return sync_and_status(h);
    return SAP_OK;
}

static sap_status graph_for(sap_handle h, double alpha, int eval_only, int chunk, cudaGraphExec_t *out)
{
    for (auto &g : h->graphs)
        if (g.alpha == alpha && g.eval_only == eval_only && g.chunk == chunk) {
            *out = g.exec;
            return SAP_OK;
        }
    cudaGraph_t graph = nullptr;
    const long long before = h->launches;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    sap_status s = SAP_OK;
    for (int c = 0; c < chunk && s == SAP_OK; ++c) s = enqueue_iteration(h, alpha, eval_only);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->launches = before;  // capture only records; replays are counted
    if (s != SAP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    CK(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    h->graphs.push_back({exec, alpha, eval_only, chunk, 0});
    *out = exec;
    return SAP_OK;
}

static int kernels_per_iteration(sap_handle h)
{
    return h->path == SAP_PLAIN ? 2 : restructured_kernels_per_iteration(h) + 1;
}

sap_status sap_run(sap_handle h, double alpha, int32_t iters, double *hist, int64_t *argmins)
{
    TraceRange trace("sap_run");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (iters < 0) return fail(h, SAP_E_ARG, "iters must be >= 0");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
    sap_status s = ensure_hist(h, iters + 1);
    if (s != SAP_OK) return s;
    CK(cudaMemsetAsync(&h->st->iter, 0, sizeof(int), h->stream));
    if (h->profiling) {
        for (int it = 0; it < iters && s == SAP_OK; ++it) s = enqueue_iteration(h, alpha, 0);
        if (s == SAP_OK) s = enqueue_iteration(h, alpha, 1);
        if (s != SAP_OK) return s;
    } else {
        const int chunk = std::min(iters, 32);
        const int kpi = kernels_per_iteration(h);
        if (chunk > 0) {
            cudaGraphExec_t g;
            s = graph_for(h, alpha, 0, chunk, &g);
            if (s != SAP_OK) return s;
            for (int r = 0; r < iters / chunk; ++r) {
                CK(cudaGraphLaunch(g, h->stream));
                h->launches += (long long)kpi * chunk;
            }
            const int rem = iters % chunk;
            if (rem) {
                s = graph_for(h, alpha, 0, rem, &g);
                if (s != SAP_OK) return s;
                CK(cudaGraphLaunch(g, h->stream));
                h->launches += (long long)kpi * rem;
            }
        }
        cudaGraphExec_t ge;
        s = graph_for(h, 0.0, 1, 1, &ge);
        if (s != SAP_OK) return s;
        CK(cudaGraphLaunch(ge, h->stream));
        h->launches += kpi;
    }
    h->last_iters = iters;
    if (hist || argmins) return sap_get_history(h, hist, argmins, iters + 1);
    return SAP_OK;
}

sap_status sap_get_history(sap_handle h, double *hist, int64_t *argmins, int32_t capacity)
{
    CHECK_HANDLE(h);
    if (h->last_iters < 0) return fail(h, SAP_E_STATE, "no sap_run yet");
    const int cnt = std::min(capacity, h->last_iters + 1);
    if (cnt < 0) return fail(h, SAP_E_ARG, "negative capacity");
    sap_status s = sync_and_status(h);
    if (s != SAP_OK) return s;
    if (hist) CK(cudaMemcpy(hist, h->hist, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost));
    if (argmins) {
        std::vector<int2> tmp(cnt);
        CK(cudaMemcpy(tmp.data(), h->am, (size_t)cnt * sizeof(int2), cudaMemcpyDeviceToHost));
        for (int q = 0; q < cnt; ++q) {
            argmins[2 * q] = tmp[q].x;
            argmins[2 * q + 1] = tmp[q].y;
        }
    }
    return SAP_OK;
}

sap_status sap_project(sap_handle h, float *Y_out, int out_is_device)
{
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    if (!Y_out) return fail(h, SAP_E_ARG, "null output");
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (h->dt == SAP_F64) return fail(h, SAP_E_UNSUPPORTED, "no tensor-core product for FP64 data");
    sap_status s = restructured_project(h, Y_out, out_is_device);
    if (s != SAP_OK) return s;
    return sync_and_status(h);
}

sap_status sap_project_df(sap_handle h, float *Yh_out, float *Yl_out, int out_is_device)
{
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    if (!Yh_out || !Yl_out) return fail(h, SAP_E_ARG, "null output");
    if (h->k == 0) return fail(h, SAP_E_STATE, "no basis set");
    if (h->dt == SAP_F64) return fail(h, SAP_E_UNSUPPORTED, "FP32 or BF16 data only");
    sap_status s = restructured_project_df(h, Yh_out, Yl_out, out_is_device);
    if (s != SAP_OK) return s;
    return sync_and_status(h);
}

sap_status sap_get_stats(sap_handle h, sap_stats *out)
{
    if (!h || !out) return SAP_E_ARG;
    std::memset(out, 0, sizeof(*out));
    if (h->is_batch) {
        // sums over the datasets (k and the tier counts of the last one)
        out->kernel_launches = h->launches;
        out->n_dim = h->n;
        for (sap_handle kid : h->kids) {
            sap_stats ks;
            const sap_status st = sap_get_stats(kid, &ks);
            if (st != SAP_OK) return st;
            out->n_points += ks.n_points;
            out->n_pairs += ks.n_pairs;
            out->n_excluded += ks.n_excluded;
            out->n_near += ks.n_near;
            out->kernel_launches += ks.kernel_launches;
            out->k = ks.k;
            out->last_tier1 = ks.last_tier1;
            out->last_tier2 = ks.last_tier2;
            out->cert_bound = ks.cert_bound;
            out->y_error_unit = std::max(out->y_error_unit, ks.y_error_unit);
            out->ydf_error_unit = std::max(out->ydf_error_unit, ks.ydf_error_unit);
        }
        return SAP_OK;
    }
    out->n_points = h->N;
    out->n_dim = h->n;
    out->k = h->k;
    out->n_pairs = h->N * (h->N - 1) / 2;
    out->kernel_launches = h->launches;
    restructured_stats(h, out);
    if (h->sticky) return SAP_E_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SAP_E_CUDA, "sync failed");
    ProbState p;
    if (cudaMemcpy(&p, h->st, sizeof(p), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(h, SAP_E_CUDA, "copy failed");
    out->last_tier1 = p.last_cnt1;
    out->last_tier2 = p.last_cnt2;
    return SAP_OK;
}

sap_status sap_set_profiling(sap_handle h, int enable)
{
    CHECK_HANDLE(h);
    CK(cudaStreamSynchronize(h->stream));
    for (auto &p : h->pending) {
        h->event_pool.push_back(p.a);
        h->event_pool.push_back(p.b);
    }
    h->pending.clear();
    for (int c = 0; c < kClasses; ++c) { h->ktime[c] = 0.0; h->kcount[c] = 0; }
    h->profiling = enable != 0;
    return SAP_OK;
}

sap_status sap_get_kernel_time(sap_handle h, int32_t kernel_class, double *total_ms, int64_t *launches)
{
    CHECK_HANDLE(h);
    if (kernel_class < 0 || kernel_class >= kClasses) return fail(h, SAP_E_ARG, "unknown kernel class");
    CK(cudaStreamSynchronize(h->stream));
    for (auto &p : h->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        h->ktime[p.cls] += ms;
        h->kcount[p.cls] += 1;
        h->event_pool.push_back(p.a);
        h->event_pool.push_back(p.b);
    }
    h->pending.clear();
    if (total_ms) *total_ms = h->ktime[kernel_class];
    if (launches) *launches = h->kcount[kernel_class];
    return SAP_OK;
}

sap_status sap_softmin_forward(sap_handle h, double tau, double *L_out)
{
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    if (!L_out) return fail(h, SAP_E_ARG, "null output");
    return softmin_forward(h, tau, L_out);
}

sap_status sap_softmin_backward(sap_handle h, double tau, double L, double *G_out, int out_is_device)
{
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    return softmin_backward(h, tau, L, G_out, out_is_device);
}

sap_status sap_softmin_ascent(sap_handle h, double tau, double eta, int32_t steps, double *hist)
{
    TraceRange trace("sap_softmin_ascent");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    return softmin_ascent(h, tau, eta, steps, hist);
}

sap_status sap_estimate_dim(sap_handle h, const double *U0, int32_t k_max, int32_t iters,
                            double alpha, double threshold, int32_t *k_out, double *ratios_out)
{
    TraceRange trace("sap_estimate_dim");
    CHECK_HANDLE(h);
    NOT_BATCH(h);
    NOT_SHARD(h);
    if (!k_out && !ratios_out) return fail(h, SAP_E_ARG, "no output");
    const sap_status s = sweep_run(h, U0, k_max, iters, alpha, threshold, k_out, ratios_out);
    if (s != SAP_OK) return s;
    return reset_state(h);  // the handle's own watch list and bounds start afresh
}

sap_status sap_get_sweep_history(sap_handle h, int32_t k, double *hist, int64_t *argmins, int32_t capacity)
{
    CHECK_HANDLE(h);
    return sweep_history(h, k, hist, argmins, capacity);
}

sap_status sap_get_sweep_basis(sap_handle h, int32_t k, double *U_out, int out_is_device)
{
    CHECK_HANDLE(h);
    return sweep_basis(h, k, U_out, out_is_device);
}

sap_status sap_create_batch(const void *const *Xs, const int64_t *Ns, int32_t B, int32_t n, sap_dtype dt,
                            int x_is_device, sap_handle *out)
{
    if (!out) return SAP_E_ARG;
    *out = nullptr;
    if (!Xs || !Ns || B < 1 || B > 4096 || n < 1 || n > 16384) return SAP_E_ARG;
    if (dt != SAP_F32 && dt != SAP_BF16 && dt != SAP_F64) return SAP_E_ARG;
    for (int b = 0; b < B; ++b)
        if (!Xs[b] || Ns[b] < 2 || Ns[b] > 92681) return SAP_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return SAP_E_NO_DEVICE;
    }
    sap_handle h = new sap_ctx();
    h->is_batch = true;
    h->n = n;
    h->dt = dt;
    auto cleanup_fail = [&](sap_status s) { sap_destroy(h); return s; };
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup_fail(SAP_E_CUDA);
    h->own_stream = true;
    if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) return cleanup_fail(SAP_E_CUDA);
    for (int b = 0; b < B; ++b) {
        sap_handle kid = nullptr;
        const sap_status st = sap_create(Xs[b], Ns[b], n, dt, x_is_device, &kid);
        if (st != SAP_OK) return cleanup_fail(st);
        h->kids.push_back(kid);
        h->N += Ns[b];
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cleanup_fail(SAP_E_CUDA);
        h->kid_done.push_back(e);
    }
    *out = h;
    return SAP_OK;
}

sap_status sap_create_subsamples(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device,
                                 const int64_t *idx, int32_t R, int32_t m, sap_handle *out)
{
    if (!out) return SAP_E_ARG;
    *out = nullptr;
    if (!X || !idx || N < 2 || n < 1 || n > 16384 || R < 1 || R > 4096 || m < 2 || m > N || m > 92681)
        return SAP_E_ARG;
    if (dt != SAP_F32 && dt != SAP_BF16 && dt != SAP_F64) return SAP_E_ARG;
    for (long long q = 0; q < (long long)R * m; ++q)
        if (idx[q] < 0 || idx[q] >= N) return SAP_E_ARG;
    const size_t es = dt == SAP_F64 ? 8 : dt == SAP_BF16 ? 2 : 4;
    const size_t row = (size_t)n * es;
    // gather each subset's rows into one staging buffer on the side X lives on
    std::vector<unsigned char> host;
    unsigned char *dev = nullptr;
    if (x_is_device) {
        if (cudaMalloc(&dev, (size_t)R * m * row) != cudaSuccess) {
            cudaGetLastError();
            return SAP_E_OOM;
        }
        for (long long q = 0; q < (long long)R * m; ++q)
            if (cudaMemcpy(dev + q * row, static_cast<const unsigned char *>(X) + idx[q] * row, row,
                           cudaMemcpyDeviceToDevice) != cudaSuccess) {
                cudaFree(dev);
                return SAP_E_CUDA;
            }
    } else {
        host.resize((size_t)R * m * row);
        for (long long q = 0; q < (long long)R * m; ++q)
            std::memcpy(host.data() + q * row, static_cast<const unsigned char *>(X) + idx[q] * row, row);
    }
    const unsigned char *base = x_is_device ? dev : host.data();
    std::vector<const void *> Xs(R);
    std::vector<int64_t> Ns(R, m);
    for (int b = 0; b < R; ++b) Xs[b] = base + (size_t)b * m * row;
    const sap_status st = sap_create_batch(Xs.data(), Ns.data(), R, n, dt, x_is_device, out);
    if (dev) cudaFree(dev);  // each dataset copied its rows
    return st;
}

sap_status sap_batch_count(sap_handle h, int32_t *B)
{
    CHECK_HANDLE(h);
    if (!B) return fail(h, SAP_E_ARG, "null output");
    *B = h->is_batch ? (int32_t)h->kids.size() : 1;
    return SAP_OK;
}

static sap_status kid_of(sap_handle h, int32_t b, sap_handle *kid)
{
    if (!h->is_batch) return fail(h, SAP_E_STATE, "not a batch handle");
    if (b < 0 || b >= (int32_t)h->kids.size()) return fail(h, SAP_E_ARG, "dataset index out of range");
    *kid = h->kids[b];
    return SAP_OK;
}

static sap_status kid_result(sap_handle h, int32_t b, sap_handle kid, sap_status st)
{
    if (st != SAP_OK) h->err = "dataset " + std::to_string(b) + ": " + kid->err;
    return st;
}

sap_status sap_estimate_dim_b(sap_handle h, int32_t b, const double *U0, int32_t k_max, int32_t iters,
                              double alpha, double threshold, int32_t *k_out, double *ratios_out)
{
    CHECK_HANDLE(h);
    sap_handle kid;
    sap_status st = kid_of(h, b, &kid);
    if (st != SAP_OK) return st;
    return kid_result(h, b, kid, sap_estimate_dim(kid, U0, k_max, iters, alpha, threshold, k_out, ratios_out));
}

sap_status sap_set_basis_b(sap_handle h, int32_t b, const double *U, int32_t k, int u_is_device)
{
    CHECK_HANDLE(h);
    sap_handle kid;
    sap_status st = kid_of(h, b, &kid);
    if (st != SAP_OK) return st;
    return kid_result(h, b, kid, sap_set_basis(kid, U, k, u_is_device));
}

sap_status sap_get_basis_b(sap_handle h, int32_t b, double *U_out, int out_is_device)
{
    CHECK_HANDLE(h);
    sap_handle kid;
    sap_status st = kid_of(h, b, &kid);
    if (st != SAP_OK) return st;
    return kid_result(h, b, kid, sap_get_basis(kid, U_out, out_is_device));
}

sap_status sap_min_secant_b(sap_handle h, int32_t b, int64_t *i, int64_t *j, double *ratio)
{
    CHECK_HANDLE(h);
    sap_handle kid;
    sap_status st = kid_of(h, b, &kid);
    if (st != SAP_OK) return st;
    return kid_result(h, b, kid, sap_min_secant(kid, i, j, ratio));
}

// One graph: fork to every dataset's stream, `chunk` iterations of each
// dataset's own chain (they are independent), join.
static sap_status batch_graph(sap_handle h, double alpha, int eval_only, int chunk, cudaGraphExec_t *out,
                              long long *launches)
{
    cudaGraph_t graph = nullptr;
    std::vector<long long> before;
    for (sap_handle kid : h->kids) before.push_back(kid->launches);
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    sap_status s = SAP_OK;
    cudaError_t e = cudaEventRecord(h->fork, h->stream);
    for (size_t b = 0; b < h->kids.size() && s == SAP_OK && e == cudaSuccess; ++b) {
        sap_handle kid = h->kids[b];
        e = cudaStreamWaitEvent(kid->stream, h->fork, 0);
        for (int c = 0; c < chunk && s == SAP_OK && e == cudaSuccess; ++c) s = enqueue_iteration(kid, alpha, eval_only);
        if (s == SAP_OK && e == cudaSuccess) e = cudaEventRecord(h->kid_done[b], kid->stream);
        if (s == SAP_OK && e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->kid_done[b], 0);
        if (s != SAP_OK) h->err = "dataset " + std::to_string(b) + ": " + kid->err;
    }
    const cudaError_t ee = cudaStreamEndCapture(h->stream, &graph);
    *launches = 0;
    for (size_t b = 0; b < h->kids.size(); ++b) {
        *launches += h->kids[b]->launches - before[b];
        h->kids[b]->launches = before[b];  // capture only records; replays are counted
    }
    if (s != SAP_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (s != SAP_OK) return s;
        CK(e != cudaSuccess ? e : ee);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    *out = exec;
    return SAP_OK;
}

sap_status sap_run_batch(sap_handle h, double alpha, int32_t iters, double *hist, int64_t *argmins)
{
    TraceRange trace("sap_run_batch");
    CHECK_HANDLE(h);
    if (!h->is_batch) return fail(h, SAP_E_STATE, "not a batch handle");
    if (iters < 0) return fail(h, SAP_E_ARG, "iters must be >= 0");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(h, SAP_E_ARG, "alpha must be in [0, 1]");
    for (size_t b = 0; b < h->kids.size(); ++b) {
        sap_handle kid = h->kids[b];
        if (kid->k == 0) return fail(h, SAP_E_STATE, "dataset " + std::to_string(b) + " has no basis");
        sap_status st = ensure_hist(kid, iters + 1);
        if (st != SAP_OK) return kid_result(h, (int32_t)b, kid, st);
        if (cudaMemsetAsync(&kid->st->iter, 0, sizeof(int), kid->stream) != cudaSuccess ||
            cudaStreamSynchronize(kid->stream) != cudaSuccess)
            return fail(h, SAP_E_CUDA, "dataset stream");
    }
    // the batch's graphs replay the datasets' buffers: rebuild them once any
    // dataset dropped its own graphs (new basis, lengths, history buffers ...)
    long long gen = 0;
    for (sap_handle kid : h->kids) gen += kid->graph_gen;
    if (gen != h->kids_gen) {
        drop_graphs(h);
        h->kids_gen = gen;
    }
    auto run = [&](int chunk, int eval_only, int reps) -> sap_status {
        if (reps <= 0) return SAP_OK;
        const double a = eval_only ? 0.0 : alpha;
        const GraphEntry *ge = nullptr;
        for (const auto &g : h->graphs)
            if (g.alpha == a && g.eval_only == eval_only && g.chunk == chunk) ge = &g;
        if (!ge) {
            cudaGraphExec_t exec = nullptr;
            long long per = 0;
            sap_status st = batch_graph(h, a, eval_only, chunk, &exec, &per);
            if (st != SAP_OK) return st;
            h->graphs.push_back({exec, a, eval_only, chunk, per});
            ge = &h->graphs.back();
        }
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = cudaGraphLaunch(ge->exec, h->stream);
            h->launches += ge->launches;
        }
        CK(e);
        return SAP_OK;
    };
    const int chunk = std::min(iters, 16);
    sap_status st = SAP_OK;
    if (chunk > 0) {
        st = run(chunk, 0, iters / chunk);
        if (st == SAP_OK && iters % chunk) st = run(iters % chunk, 0, 1);
    }
    if (st == SAP_OK) st = run(1, 1, 1);
    if (st != SAP_OK) return st;
    CK(cudaStreamSynchronize(h->stream));
    for (size_t b = 0; b < h->kids.size(); ++b) {
        sap_handle kid = h->kids[b];
        kid->last_iters = iters;
        const size_t off = b * (size_t)(iters + 1);
        st = sap_get_history(kid, hist ? hist + off : nullptr, argmins ? argmins + 2 * off : nullptr, iters + 1);
        if (st != SAP_OK) return kid_result(h, (int32_t)b, kid, st);
    }
    return SAP_OK;
}

} // extern "C"
