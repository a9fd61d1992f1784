// noalloc.cu -- sap_min_secant_noalloc: the argmin step of SAP for callers
// that cannot allocate GPU memory.
//
// Some callers must not call cudaMalloc: code whose device memory is owned
// by another allocator (a framework's pool) and must not be fragmented or
// grown behind its back, and latency-critical loops that cannot afford an
// allocation's implicit device-wide synchronisation or its failure at run
// time.  This entry point serves them: it allocates nothing.  Its working
// memory is one file-scope __device__ array of fixed size (about 4.2 MB),
// which every GPU that loads the library holds until the process exits.
//
// It runs the same kernels as sap_min_secant on a handle in the plain form:
// the FP32 all-pairs pass (secants formed on the fly, certified candidate
// emission) followed by the FP64 recheck and argmin, so it returns the same
// pair and ratio.  It copies the result to the host and synchronises the
// caller's stream before returning.
//
// Limits: 2 <= N <= 1024 points, 1 <= n <= 1024, 1 <= k <= min(n, 8); larger
// problems are rejected with SAP_E_ARG.  The scratch holds every pair of the
// largest problem, so the candidate list cannot overflow.
//
// Host code cannot use the array's name as a device address (it names a
// host-side stand-in), so the first call on each device looks the address
// up with cudaGetSymbolAddress while that device is current; make that first
// call outside any stream capture.  All calls share the array and each one
// re-initialises what must start from zero, so calls that overlap on the
// GPU (different streams or threads at the same time) race and must be
// serialised by the caller.
#include "sap_internal.cuh"
#include "../../include/sap.h"

#include <cmath>
#include <mutex>

using namespace sap;

namespace {

constexpr int kNaMaxN = 1024;
constexpr int kNaMaxDim = 1024;
constexpr int kNaMaxK = 8;
constexpr int kNaBlocks = (kNaMaxN + 63) / 64;
constexpr int kNaTiles = kNaBlocks * (kNaBlocks + 1) / 2;
constexpr unsigned int kNaCandCap = (unsigned int)kNaMaxN * (kNaMaxN - 1) / 2;
constexpr int kNaParts = 64;
constexpr int kNaMaxDevices = 64;

struct NoAllocScratch {
    ProbState st;
    Partial partials[kNaParts];
    double hist[1];
    int2 argmin[1];
    int2 tiles[kNaTiles];
    float U32[kNaMaxDim * kNaMaxK];
    int2 cand[kNaCandCap];
};

static __device__ __align__(256) NoAllocScratch g_scratch;

std::mutex g_mutex;
NoAllocScratch *g_addr[kNaMaxDevices] = {};
int g_sms[kNaMaxDevices] = {};

// Resets the shared state, lists the 64-point blocks (I, J), I <= J, and
// writes the FP32 copy of U (n x KP row-major, zero pad columns).
__global__ void na_init_kernel(NoAllocScratch *g, const double *U, int n, int k, int KP, int nb)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    if (tid == 0) {
        ProbState &s = g->st;
        s.seed_ub = 0x7f800000u;
        s.run_ub1 = 0x7f800000u;
        s.run_ub2 = 0x7f800000u;
        s.cnt1 = 0;
        s.cnt2 = 0;
        s.iter = 0;
        s.status = 0;
        s.watch_n = 0;
        s.watch_pos = 0;
        s.last_cnt1 = 0;
        s.last_cnt2 = 0;
        s.hist_cap = 1;
        s.ticket = 0;
        s.last_r = INFINITY;
        s.last_i = -1;
        s.last_j = -1;
    }
    for (int t = tid; t < nb * nb; t += nthreads) {
        const int I = t / nb, J = t % nb;
        if (J < I) continue;
        // row-major index of (I, J) in the upper triangle of an nb x nb grid
        const int idx = I * nb - I * (I - 1) / 2 + (J - I);
        g->tiles[idx] = make_int2(I, J);
    }
    for (int e = tid; e < n * KP; e += nthreads) {
        const int l = e / KP, c = e % KP;
        g->U32[e] = c < k ? (float)U[(size_t)c * n + l] : 0.f;
    }
}

double gam(double m)
{
    const double u = std::ldexp(1.0, -24);
    return m * u / (1.0 - m * u);
}

} // namespace

extern "C" sap_status sap_min_secant_noalloc(const float *X, int64_t N, int32_t n, const double *U, int32_t k,
                                             double eps, void *cuda_stream, int64_t *i_out, int64_t *j_out,
                                             double *ratio_out)
{
    if (!X || !U) return SAP_E_ARG;
    if (N < 2 || N > kNaMaxN || n < 1 || n > kNaMaxDim || k < 1 || k > kNaMaxK || k > n) return SAP_E_ARG;
    if (!(eps >= 0.0) || !std::isfinite(eps)) return SAP_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SAP_E_NO_DEVICE;
    }
    if (dev < 0 || dev >= kNaMaxDevices) return SAP_E_UNSUPPORTED;
    NoAllocScratch *g;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SAP_E_CUDA;
            }
            int s = 0;
            if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SAP_E_CUDA;
            g_addr[dev] = static_cast<NoAllocScratch *>(p);
            g_sms[dev] = s;
        }
        g = g_addr[dev];
        sms = g_sms[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int KP = padded_stride(k);
    const int nb = (int)((N + 63) / 64);
    const int ntiles = nb * (nb + 1) / 2;

    na_init_kernel<<<8, 256, 0, s>>>(g, U, n, k, KP, nb);
    if (cudaGetLastError() != cudaSuccess) return SAP_E_CUDA;

    // the FP32 all-pairs pass (error model of the plain form)
    const double u = std::ldexp(1.0, -24);
    PlainArgsF32 a;
    a.X = X;
    a.N = (int)N;
    a.n = n;
    a.U32 = g->U32;
    a.k = k;
    a.KP = KP;
    a.tiles = g->tiles;
    a.ntiles = ntiles;
    a.grid = ntiles < 2 * sms ? ntiles : 2 * sms;
    const double eps2 = eps * eps;
    if (eps > 0.0) {
        const double m = 4.0 * gam(n + 2) + 1e-6;
        a.eps2_lo = std::nextafter((float)(eps2 * (1.0 - m)), 0.f);
        a.eps2_hi = std::nextafter((float)(eps2 * (1.0 + m)), INFINITY);
    } else {
        a.eps2_lo = a.eps2_hi = 0.f;
    }
    a.cert.A = (float)(std::sqrt((double)k) * gam(n + 3) * 1.05);
    a.cert.rho = (float)((gam(n + 2) + gam(k) + 3 * u) * 1.05);
    a.st = &g->st;
    a.cand = g->cand;
    a.cand_cap = kNaCandCap;
    if (launch_plain_f32(a, s) != cudaSuccess) return SAP_E_CUDA;

    // FP64 recheck and argmin (evaluation only: U is not touched)
    SelectUpdateArgs q;
    q.X = X;
    q.x_is_f64 = 0;
    q.N = (int)N;
    q.n = n;
    q.U64 = const_cast<double *>(U);
    q.U32 = g->U32;
    q.U32lo = nullptr;
    q.KP = KP;
    q.Uhi = nullptr;
    q.Ulo = nullptr;
    q.NP = 0;
    q.split_bf16 = 0;
    q.split_scale = 1.f;
    q.k = k;
    q.alpha = 0.0;
    q.mode = 0;
    q.eval_only = 1;
    q.eps2 = eps2;
    q.list = g->cand;
    q.cap = kNaCandCap;
    q.which = 1;
    q.partials = g->partials;
    q.grid = kNaParts < sms ? kNaParts : sms;
    q.work = nullptr;
    q.st = &g->st;
    q.hist = g->hist;
    q.argmin = g->argmin;
    q.seed_cert = a.cert;
    q.pdl = 0;
    q.fused = 0;
    q.near = nullptr;
    q.n_near = 0;
    q.cert2 = a.cert;
    if (launch_select_update(q, s) != cudaSuccess) return SAP_E_CUDA;

    ProbState st;
    if (cudaMemcpyAsync(&st, &g->st, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SAP_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SAP_E_CUDA;
    if (st.status & ST_BOUNDS) return SAP_E_BOUNDS;
    if (st.status & ST_NO_SECANT) return SAP_E_NO_SECANT;
    if (st.status & ST_TIMEOUT) return SAP_E_TIMEOUT;
    if (st.status & ST_OVERFLOW) return SAP_E_UNSUPPORTED;
    if (i_out) *i_out = st.last_i;
    if (j_out) *j_out = st.last_j;
    if (ratio_out) *ratio_out = st.last_r;
    return SAP_OK;
}
