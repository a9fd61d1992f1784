// sweep.cu -- the dimension-estimation sweep (Sec. VI-A) over k = 1..k_max.
//
// Every basis is an independent SAP problem (Algorithm 1) over the same
// dataset, so the bases share the handle's point copy, stored lengths and
// near-pair list (classified for k_max: the pass bound grows like sqrt(k),
// so that list is a superset of each smaller k's).  One iteration is one
// tensor-core product Y = X [U_1 .. U_kmax] for all bases at once (their
// padded widths sum to 256 at k_max = 20: a single MMA N), then, per basis
// and on its own stream, the all-pairs pass, the explicit-difference tier
// and the FP64 recheck fused with the update.  A chunk of iterations is
// captured once as a CUDA graph with one branch per basis and replayed;
// the bases' chains overlap on the GPU.
#include "sweep.cuh"
#include "restructured.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace sap {

// (declared in softmin.cuh as well)
int handle_profiling(sap_handle h);
long long handle_launches(sap_handle h);
void handle_add_launches(sap_handle h, long long delta);

namespace {

constexpr int kSweepMaxKY = 256;          // padded widths of all bases: one MMA N
constexpr long long kSweepCap = 1ll << 22;  // candidate list entries per basis
constexpr int kSweepChunk = 8;            // iterations per captured graph

#define WCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return handle_fail(h, e_ == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA, \
                               cudaGetErrorString(e_));                                     \
    } while (0)

template <typename T_>
void wfree(T_ *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

int total_width(int kmax)
{
    int t = 0;
    for (int k = 1; k <= kmax; ++k) t += padded_stride(k);
    return t;
}

sap_status alloc_impl(sap_handle h, SweepState *&swp, int kmax, int hist_need);

sap_status alloc(sap_handle h, SweepState *&swp, int kmax, int hist_need)
{
    if (swp && swp->kmax == kmax && swp->hist_cap >= hist_need) return SAP_OK;
    sweep_free(swp);
    const sap_status st = alloc_impl(h, swp, kmax, hist_need);
    if (st != SAP_OK) sweep_free(swp);
    return st;
}

sap_status alloc_impl(sap_handle h, SweepState *&swp, int kmax, int hist_need)
{
    swp = new SweepState();
    SweepState &sw = *swp;
    RestrState &r = restr_state(h);
    const int n = handle_n_dim(h);
    const long long N = handle_n_points(h);
    sw.kmax = kmax;
    sw.hist_cap = std::max(hist_need, 64);
    sw.cap = std::min<long long>(N * (N - 1) / 2 + 64, kSweepCap);
    sw.KY = total_width(kmax);
    sw.KPG = (sw.KY + 15) / 16 * 16;
    sw.ksplit = r.ksplit;
    WCK(cudaMalloc(&sw.Uhi, (size_t)sw.KPG * r.NP * 2));
    WCK(cudaMalloc(&sw.Ulo, (size_t)sw.KPG * r.NP * 2));
    WCK(cudaMalloc(&sw.Y, (size_t)sw.KY * r.Npad * sizeof(float)));
    WCK(cudaMalloc(&sw.Yd, (size_t)sw.KY * r.Npad * 2 * sizeof(float)));
    if (sw.ksplit > 1) WCK(cudaMalloc(&sw.Ypart, (size_t)sw.ksplit * sw.KY * r.Npad * sizeof(float)));
    WCK(cudaMalloc(&sw.gst, sizeof(ProbState)));
    WCK(cudaMemset(sw.gst, 0, sizeof(ProbState)));
    WCK(cudaEventCreateWithFlags(&sw.fork, cudaEventDisableTiming));
    if (!restructured_u_maps(h, sw.Uhi, sw.Ulo, sw.KPG, &sw.mhi, &sw.mlo))
        return handle_fail(h, SAP_E_CUDA, "cuTensorMapEncodeTiled failed for the sweep's bases");
    sw.b.resize(kmax);
    // Stream priorities, copied into the captured kernel nodes: the wider a
    // basis, the longer its chain (its one-block FP64 update grows like n k^2
    // and bounds the iteration), so its kernels are dispatched first when
    // the chains of all bases compete for SMs.
    int prio_least = 0, prio_greatest = 0;
    WCK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    int off = 0;
    for (int q = 0; q < kmax; ++q) {
        SweepBasis &b = sw.b[q];
        b.k = q + 1;
        b.KP = padded_stride(b.k);
        b.KY = padded_stride(b.k);
        b.off = off;
        off += b.KY;
        WCK(cudaMalloc(&b.U64, (size_t)n * b.k * sizeof(double)));
        WCK(cudaMalloc(&b.Ydh, (size_t)b.KY * r.Npad * sizeof(float)));
        WCK(cudaMalloc(&b.Ydl, (size_t)b.KY * r.Npad * sizeof(float)));
        WCK(cudaMemset(b.Ydh, 0, (size_t)b.KY * r.Npad * sizeof(float)));
        WCK(cudaMemset(b.Ydl, 0, (size_t)b.KY * r.Npad * sizeof(float)));
        WCK(cudaMalloc(&b.U32, (size_t)n * b.KP * sizeof(float)));
        WCK(cudaMalloc(&b.U32lo, (size_t)n * b.KP * sizeof(float)));
        WCK(cudaMalloc(&b.work, (size_t)(kMaxK + 1) * n * sizeof(double)));
        WCK(cudaMalloc(&b.st, sizeof(ProbState)));
        WCK(cudaMalloc(&b.cand1, (size_t)sw.cap * sizeof(int2)));
        WCK(cudaMalloc(&b.cand2, (size_t)sw.cap * sizeof(int2)));
        WCK(cudaMalloc(&b.partials, (size_t)kRecheckBlocks * sizeof(Partial)));
        WCK(cudaMalloc(&b.hist, (size_t)sw.hist_cap * sizeof(double)));
        WCK(cudaMalloc(&b.am, (size_t)sw.hist_cap * sizeof(int2)));
        const int prio = prio_least + (int)std::lround((double)(prio_greatest - prio_least) * q / std::max(1, kmax - 1));
        WCK(cudaStreamCreateWithPriority(&b.stream, cudaStreamNonBlocking, prio));
        WCK(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
    }
    return SAP_OK;
}

// Initial bases: basis k is the first k columns of U0 (n x kmax).
sap_status upload(sap_handle h, SweepState &sw, const double *U0)
{
    RestrState &r = restr_state(h);
    const int n = handle_n_dim(h);
    std::vector<uint16_t> hi((size_t)sw.KPG * r.NP, 0), lo((size_t)sw.KPG * r.NP, 0);
    for (SweepBasis &b : sw.b) {
        WCK(cudaMemcpy(b.U64, U0, (size_t)n * b.k * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<float> u32((size_t)n * b.KP, 0.f), u32lo((size_t)n * b.KP, 0.f);
        for (int l = 0; l < n; ++l)
            for (int c = 0; c < b.k; ++c) {
                const double v = U0[(size_t)c * n + l];
                const float f = (float)v;
                u32[(size_t)l * b.KP + c] = f;
                u32lo[(size_t)l * b.KP + c] = (float)(v - (double)f);
            }
        WCK(cudaMemcpy(b.U32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice));
        WCK(cudaMemcpy(b.U32lo, u32lo.data(), u32lo.size() * sizeof(float), cudaMemcpyHostToDevice));
        restructured_split_host(h, U0, b.k, hi.data() + (size_t)b.off * r.NP, lo.data() + (size_t)b.off * r.NP);
        ProbState p;
        std::memset(&p, 0, sizeof(p));
        p.seed_ub = p.run_ub1 = p.run_ub2 = 0x7f800000u;
        p.hist_cap = sw.hist_cap;
        p.last_r = INFINITY;
        p.last_i = p.last_j = -1;
        WCK(cudaMemcpy(b.st, &p, sizeof(p), cudaMemcpyHostToDevice));
    }
    WCK(cudaMemcpy(sw.Uhi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice));
    WCK(cudaMemcpy(sw.Ulo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice));
    WCK(cudaMemset(sw.Y, 0, (size_t)sw.KY * r.Npad * sizeof(float)));
    WCK(cudaMemset(sw.Yd, 0, (size_t)sw.KY * r.Npad * 2 * sizeof(float)));
    return SAP_OK;
}

SelectUpdateArgs update_args(sap_handle h, SweepState &sw, SweepBasis &b, double alpha, int eval_only)
{
    RestrState &r = restr_state(h);
    SelectUpdateArgs u;
    std::memset(&u, 0, sizeof(u));
    const bool bf16 = handle_split_bf16(h) != 0;
    u.X = handle_x32(h);
    u.x_is_f64 = 0;
    u.N = (int)handle_n_points(h);
    u.n = handle_n_dim(h);
    u.U64 = b.U64;
    u.U32 = b.U32;
    u.U32lo = b.U32lo;
    u.KP = b.KP;
    u.Uhi = static_cast<uint16_t *>(sw.Uhi) + (size_t)b.off * r.NP;
    u.Ulo = static_cast<uint16_t *>(sw.Ulo) + (size_t)b.off * r.NP;
    u.NP = r.NP;
    u.split_bf16 = bf16;
    u.split_scale = bf16 ? 256.f : 2048.f;
    u.k = b.k;
    u.alpha = alpha;
    u.mode = handle_mode(h);
    u.eval_only = eval_only;
    u.eps2 = handle_eps2(h);
    u.list = b.cand2;
    u.cap = (unsigned int)sw.cap;
    u.which = 2;
    u.partials = b.partials;
    u.grid = std::min(handle_tune(h).su_blocks > 0 ? handle_tune(h).su_blocks : handle_sms(h), kRecheckBlocks);
    u.work = b.work;
    u.st = b.st;
    u.hist = b.hist;
    u.argmin = b.am;
    u.seed_cert = handle_seed_cert(u.n, b.k);
    u.pdl = handle_tune(h).pdl;
    BasisView v;
    v.k = b.k;
    v.cand1 = b.cand1;
    v.cand2 = b.cand2;
    restructured_fuse_args(h, v, u);
    return u;
}

// One iteration of every basis (evaluation only when eval_only).
sap_status enqueue_iteration(sap_handle h, SweepState &sw, double alpha, int eval_only)
{
    RestrState &r = restr_state(h);
    cudaStream_t s0 = handle_stream(h);
    sap_status st = restructured_enqueue_product(h, &sw.mhi, &sw.mlo, sw.KPG, sw.Y, sw.Yd, sw.KY, sw.Ypart, sw.gst, s0);
    if (st != SAP_OK) return st;
    WCK(cudaEventRecord(sw.fork, s0));
    for (SweepBasis &b : sw.b) {
        WCK(cudaStreamWaitEvent(b.stream, sw.fork, 0));
        BasisView v;
        v.k = b.k;
        v.KP = b.KP;
        v.KY = b.KY;
        v.U32 = b.U32;
        v.U32lo = b.U32lo;
        v.Y = sw.Y + (size_t)b.off * 128;  // block-major: the basis's components within each block
        v.Yd = sw.Yd + (size_t)b.off * 256;
        v.Ykt = sw.KY;
        v.Ydh = b.Ydh;
        v.Ydl = b.Ydl;
        v.st = b.st;
        v.cand1 = b.cand1;
        v.cand2 = b.cand2;
        v.cap = sw.cap;
        v.U64 = b.U64;
        v.partials = b.partials;
        st = restructured_enqueue_basis(h, v, b.stream);
        if (st != SAP_OK) return st;
        const SelectUpdateArgs u = update_args(h, sw, b, alpha, eval_only);
        cudaEvent_t ea, eb;
        handle_count_launch(h, 5, &ea, &eb);
        if (ea) cudaEventRecord(ea, b.stream);
        WCK(launch_select_update(u, b.stream));
        if (eb) cudaEventRecord(eb, b.stream);
        handle_push_timing(h, 5, ea, eb);
        WCK(cudaEventRecord(b.done, b.stream));
        WCK(cudaStreamWaitEvent(s0, b.done, 0));
    }
    return SAP_OK;
}

sap_status run_graph(sap_handle h, SweepState &sw, double alpha, int eval_only, int iters)
{
    cudaStream_t s0 = handle_stream(h);
    if (handle_profiling(h)) {
        for (int q = 0; q < iters; ++q) {
            sap_status st = enqueue_iteration(h, sw, alpha, eval_only);
            if (st != SAP_OK) return st;
        }
        return SAP_OK;
    }
    // a captured chunk names the handle's buffers and the near-list length:
    // reuse it while neither changed (the handle bumps its generation
    // whenever it drops its own graphs)
    const long long gen = handle_graph_gen(h);
    const int n_near = restr_state(h).n_near;
    for (size_t q = 0; q < sw.graphs.size();) {
        if (sw.graphs[q].gen != gen || sw.graphs[q].n_near != n_near) {
            cudaGraphExecDestroy(sw.graphs[q].exec);
            sw.graphs.erase(sw.graphs.begin() + q);
        } else {
            ++q;
        }
    }
    int done = 0;
    while (done < iters) {
        const int chunk = std::min(kSweepChunk, iters - done);
        const SweepState::Graph *g = nullptr;
        for (const auto &c : sw.graphs)
            if (c.alpha == alpha && c.eval_only == eval_only && c.chunk == chunk) g = &c;
        if (!g) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            const long long before = handle_launches(h);
            WCK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
            sap_status st = SAP_OK;
            for (int q = 0; q < chunk && st == SAP_OK; ++q) st = enqueue_iteration(h, sw, alpha, eval_only);
            cudaError_t e = cudaStreamEndCapture(s0, &graph);
            const long long per_chunk = handle_launches(h) - before;
            handle_add_launches(h, -per_chunk);
            if (st != SAP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            WCK(e);
            e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(graph);
            WCK(e);
            sw.graphs.push_back({exec, alpha, eval_only, chunk, n_near, gen, per_chunk});
            g = &sw.graphs.back();
        }
        const int reps = (iters - done) / chunk;
        cudaError_t e = cudaSuccess;
        for (int q = 0; q < reps && e == cudaSuccess; ++q) {
            e = cudaGraphLaunch(g->exec, s0);
            handle_add_launches(h, g->launches);
        }
        WCK(e);
        done += reps * chunk;
    }
    return SAP_OK;
}

} // namespace

sap_status sweep_run(sap_handle h, const double *U0, int kmax, int iters, double alpha, double threshold,
                     int *k_out, double *ratios_out)
{
    const int n = handle_n_dim(h);
    if (!U0 || kmax < 1 || kmax > n || iters < 0 || !(alpha >= 0.0 && alpha <= 1.0) || !std::isfinite(threshold))
        return handle_fail(h, SAP_E_ARG, "need U0, 1 <= k_max <= n, iters >= 0, alpha in [0, 1]");
    if (!handle_x32(h)) return handle_fail(h, SAP_E_UNSUPPORTED, "the sweep needs FP32 or BF16 data");
    if (total_width(kmax) > kSweepMaxKY) return handle_fail(h, SAP_E_UNSUPPORTED, "the sweep supports k_max <= 20");
    // U0 must have orthonormal columns (then every prefix does)
    double dev = 0.0;
    for (int a = 0; a < kmax; ++a)
        for (int c = 0; c <= a; ++c) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += U0[(size_t)a * n + l] * U0[(size_t)c * n + l];
            dev = std::max(dev, std::fabs(s - (a == c ? 1.0 : 0.0)));
        }
    if (!(dev <= 1e-10)) return handle_fail(h, SAP_E_NOT_ORTHONORMAL, "max |U0^T U0 - I| > 1e-10");
    cudaStream_t s0 = handle_stream(h);
    WCK(cudaStreamSynchronize(s0));
    SweepState *&swp = sweep_state(h);
    sap_status st = alloc(h, swp, kmax, iters + 1);
    if (st != SAP_OK) return st;
    SweepState &sw = *swp;
    st = restructured_classify(h, kmax);
    if (st != SAP_OK) return st;
    st = upload(h, sw, U0);
    if (st != SAP_OK) return st;
    st = run_graph(h, sw, alpha, 0, iters);
    if (st == SAP_OK) st = run_graph(h, sw, 0.0, 1, 1);
    if (st != SAP_OK) return st;
    WCK(cudaStreamSynchronize(s0));
    st = handle_check_status(h, sw.gst);
    for (SweepBasis &b : sw.b)
        if (st == SAP_OK) st = handle_check_status(h, b.st);
    if (st != SAP_OK) return st;
    sw.last_iters = iters;
    int kk = -1;
    for (SweepBasis &b : sw.b) {
        double r = 0.0;
        WCK(cudaMemcpy(&r, b.hist + iters, sizeof(double), cudaMemcpyDeviceToHost));
        if (ratios_out) ratios_out[b.k - 1] = r;
        if (kk < 0 && r > threshold) kk = b.k;
    }
    if (k_out) *k_out = kk;
    // the handle's own basis goes back to its own near classification
    const int k = handle_k(h);
    if (k > 0 && k != kmax) return restructured_classify(h, k);
    return SAP_OK;
}

sap_status sweep_history(sap_handle h, int k, double *hist, int64_t *argmins, int capacity)
{
    SweepState *sw = sweep_state(h);
    if (!sw || sw->last_iters < 0) return handle_fail(h, SAP_E_STATE, "no sweep yet");
    if (k < 1 || k > sw->kmax || capacity < 0) return handle_fail(h, SAP_E_ARG, "k out of range");
    const int cnt = std::min(capacity, sw->last_iters + 1);
    SweepBasis &b = sw->b[k - 1];
    if (hist) WCK(cudaMemcpy(hist, b.hist, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost));
    if (argmins) {
        std::vector<int2> tmp(cnt);
        WCK(cudaMemcpy(tmp.data(), b.am, (size_t)cnt * sizeof(int2), cudaMemcpyDeviceToHost));
        for (int q = 0; q < cnt; ++q) {
            argmins[2 * q] = tmp[q].x;
            argmins[2 * q + 1] = tmp[q].y;
        }
    }
    return SAP_OK;
}

sap_status sweep_basis(sap_handle h, int k, double *U_out, int out_is_device)
{
    SweepState *sw = sweep_state(h);
    if (!sw || sw->last_iters < 0) return handle_fail(h, SAP_E_STATE, "no sweep yet");
    if (k < 1 || k > sw->kmax || !U_out) return handle_fail(h, SAP_E_ARG, "k out of range or null output");
    WCK(cudaMemcpy(U_out, sw->b[k - 1].U64, (size_t)handle_n_dim(h) * k * sizeof(double),
                   out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return SAP_OK;
}

void sweep_free(SweepState *&s)
{
    if (!s) return;
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
    s->graphs.clear();
    for (SweepBasis &b : s->b) {
        wfree(b.U64); wfree(b.U32); wfree(b.U32lo); wfree(b.work); wfree(b.st); wfree(b.Ydh); wfree(b.Ydl);
        wfree(b.cand1); wfree(b.cand2); wfree(b.partials); wfree(b.hist); wfree(b.am);
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.done) cudaEventDestroy(b.done);
    }
    wfree(s->Uhi); wfree(s->Ulo); wfree(s->Y); wfree(s->Yd); wfree(s->Ypart); wfree(s->gst);
    if (s->fork) cudaEventDestroy(s->fork);
    delete s;
    s = nullptr;
}

} // namespace sap
