// select_update.cu -- the FP64 argmin over the certified candidate list and
// the basis update of one SAP iteration (Algorithm 1 and Sec. IV of Kvinge
// et al., arXiv:1807.03425), fused into one launch.
//
// Phase 1 (all blocks): one warp per candidate forms the explicit FP64
// difference D = x_i - x_j, d^2 = |D|^2 and z = U^T D, applies the exclusion
// rules exactly (d^2 == 0: not distinct, Sec. II; d^2 < eps^2: shorter than
// the threshold, Sec. VII) and keeps the best squared ratio q = |z|^2/d^2
// (the square root is monotone, so the argmin is the same; ties go to the
// smallest pair index).  Candidates are dealt to blocks first and to warps
// second, so each SM's FP64 pipe serves as few warps as possible (FP64
// throughput per SM, not latency, is what limits this phase on this part).
// Each block publishes its best; the last block to finish (ticket counter)
// continues with phase 2.
//
// Phase 2 (last block):
//   1. argmin over the block results; record r = sqrt(q) in the history;
//   2. s = D/|D|, c = U^T s (one multi-value block reduction);
//   3. pivot t = argmax_l |c_l| (first on ties; the first column if all are
//      zero), then modified Gram-Schmidt on [c, e_l (l != t)] in the
//      k-dimensional coefficient space: since U has orthonormal columns,
//      MGS of [U c, u_l (l != t)] in R^n is U times MGS of [c, e_l] in R^k;
//   4. new first column along (1-a) v + a (s - v) (literal reading) or
//      (1-a) v/|v| + a e/|e| (angle reading), v = U c, e = s - v;
//   5. re-orthonormalisation in FP64, as a Cholesky QR of the new basis U':
//      G = U'^T U' = (I + R)^T (I + R), U'' = U' (I + R)^-1, the QR factor one
//      MGS re-pass gives in exact arithmetic.  When max|G - I| <= 1e-6 (the
//      usual case: U' is orthonormal to working precision) R and (I + R)^-1
//      are taken from their series in E = G - I to second order, whose
//      truncation error (order |E|^3) is below FP64 rounding; otherwise the
//      Cholesky factor is computed directly;
//   6. U'' written in FP64, FP32 and as the split 16-bit operands of the
//      tensor-core product; the recent argmin pairs are re-evaluated under
//      U'' (FP32 explicit differences) to seed the next evaluation's bound.
// Steps 2-4 run in the data's precision (FP32 for FP32 data, FP64 for FP64
// data); the recheck and the re-orthonormalisation are FP64.
#include "sap_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sap {
namespace {

constexpr int SB = 256;          // threads per block
constexpr int NW = SB / 32;
constexpr size_t kDynSmem = 40 * 1024;  // dynamic part of phase 2 (static part < 8 KB: total within 48 KB)
constexpr int kSeedRegs = 4;     // watch-pair coordinates prefetched per lane (n <= 128)

template <typename TX>
__device__ __forceinline__ TX ld_x(const void *X, size_t idx)
{
    return static_cast<const TX *>(X)[idx];
}

// Warp sums of M values at once (levels outer, values inner, so the M
// dependency chains overlap).
template <typename V, int M>
__device__ __forceinline__ void warp_sum_multi(V (&v)[M])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < M; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
}

// Block sums of M values; result in out[0..M-1] (shared), visible to all.
template <typename V, int M>
__device__ __forceinline__ void block_sum_multi(V (&v)[M], V *scratch /* NW*M */, V *out)
{
    warp_sum_multi<V, M>(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int q = 0; q < M; ++q) scratch[w * M + q] = v[q];
    __syncthreads();
    if (threadIdx.x < M) {
        V s = 0;
#pragma unroll
        for (int p = 0; p < NW; ++p) s += scratch[p * M + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// d2 = |D|^2 and zz = |U^T D|^2 from per-lane partial sums v[0..K-1] (U^T D)
// and v[K] (|D|^2), delivered to every lane.
template <int K>
__device__ __forceinline__ void warp_ratio_parts(double (&v)[K + 1], int lane, double &zz, double &d2)
{
    constexpr int M = K + 1;
    if constexpr (M <= 32) {
        constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
        constexpr int dup = 32 / S;  // lanes holding the same entry
        double r[S];
#pragma unroll
        for (int q = 0; q < S; ++q) r[q] = q < M ? v[q < M ? q : 0] : 0.0;
        const double t = warp_reduce_scatter<S>(r, lane);
        const int idx = rs_index<S>(lane);
        double sq = (idx < K && lane % dup == 0) ? t * t : 0.0;
#pragma unroll
        for (int o = 16; o >= dup; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        zz = __shfl_sync(0xffffffffu, sq, 0);
        d2 = __shfl_sync(0xffffffffu, t, K * dup);
    } else {
        warp_sum_multi<double, K + 1>(v);
        d2 = v[K];
        zz = 0.0;
#pragma unroll
        for (int c = 0; c < K; ++c) zz = fma(v[c], v[c], zz);
    }
}

// (q, i, j) ordering for q >= 0 (no NaN): the bit patterns of non-negative
// doubles order like their values, so the compare stays off the FP64 pipe.
__device__ __forceinline__ bool better_q(double q, int i, int j, double qb, int ib, int jb)
{
    const unsigned long long a = (unsigned long long)__double_as_longlong(q);
    const unsigned long long b = (unsigned long long)__double_as_longlong(qb);
    if (a != b) return a < b;
    if (i != ib) return i < ib;
    return j < jb;
}

// Dynamic shared memory of phase 2 when the basis fits: U' (FP64), D (data
// precision, padded to 8 bytes) and the FP32 final basis.
template <typename TX>
__host__ __device__ inline size_t su_dyn_bytes(int n, int K)
{
    return (size_t)n * K * 8 + ((size_t)n * sizeof(TX) + 7) / 8 * 8 + (size_t)n * K * 4;
}

template <typename WT, int K>
struct Shared {
    double red_d[NW * (K + 1)];
    float red_f[NW * (K + 1)];
    Partial wb[NW];
    int last, alive0, series;
    // problem state prefetched at the start of phase 2
    int iter, hist_cap, cnt1, cnt2, watch_n, watch_pos;
    int2 watch[kWatch];
    double cvec[K + 1];            // U^T D and |D|^2 (data precision, widened)
    WT cw[K];                      // c = U^T s
    WT Bw[K][K];                   // coefficient MGS result, column m = q_m
    WT av, asd, dnorm, nd2;        // direction coefficients, |D|, |dir|^2
    double G[K][K];                // Gram matrix (upper), then R (upper)
    double T1[K][K], T2[K][K];     // series terms (K > 8) 
    static constexpr int KS = K <= 8 ? K : 1;
    static constexpr int GW = K * (K + 1) / 2 <= 32 ? NW : 1;
    float S1f[KS][KS];             // first-order term in FP32 (series, K <= 8)
    double gred[GW][32];           // per-warp Gram partials (reduce-scatter, K <= 7)
    float emaxw;
    double Ri[K][K];               // (I + R)^-1 (upper)
    double Rd[K];                  // 1 / R_jj (direct path)
    float seed[NW];
};

template <typename TX, int K>
__global__ void __launch_bounds__(SB) select_update_kernel(SelectUpdateArgs a)
{
    extern __shared__ double dyn[];
    __shared__ Shared<TX, K> sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = a.n;
    const int kk = a.k;            // actual k (<= K)
    ProbState *st = a.st;

    // Programmatic launch: the next iteration's product may start its
    // prologue (it waits for this kernel before reading the basis); this
    // kernel's inputs are the explicit tier's list, so wait for it.
    grid_dep_launch();
    grid_dep_wait();

    // ---------------- phase 1: FP64 recheck of the candidate list ----------
    {
        Partial best = {INFINITY, 0x7fffffff, 0x7fffffff};
        // the FP64 evaluation of one pair by the warp; keeps the best
        auto eval64 = [&](int2 ij) {
            double v[K + 1];
#pragma unroll
            for (int q = 0; q <= K; ++q) v[q] = 0.0;
#pragma unroll 4
            for (int l = lane; l < n; l += 32) {
                const double D = (double)ld_x<TX>(a.X, (size_t)ij.x * n + l) -
                                 (double)ld_x<TX>(a.X, (size_t)ij.y * n + l);
                v[K] = fma(D, D, v[K]);
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (c < kk) v[c] = fma(a.U64[(size_t)c * n + l], D, v[c]);
            }
            double zz, d2;
            warp_ratio_parts<K>(v, lane, zz, d2);
            if (d2 == 0.0 || d2 < a.eps2) return;
            const double q = zz / d2;  // squared ratio
            if (better_q(q, ij.x, ij.y, best.r, best.i, best.j)) best = Partial{q, ij.x, ij.y};
        };
        bool fused = false;
        if constexpr (sizeof(TX) == 4) fused = a.fused != 0;  // FP32 data only
        if (fused) {
            // Fused second tier: the near pairs and the pass's candidates,
            // each first from explicit FP32 differences (the explicit tier's
            // arithmetic and error model), then, if it can still be the
            // argmin against the running bound, in FP64 by the same warp.
            // The bound is valid whenever it is read, so no list of
            // survivors and no second launch are needed.
            constexpr int EPW = 4;                 // pairs per warp per round
            constexpr int KU = (K + 3) / 4 * 4;    // U32 row stride covers KU
            constexpr int M = EPW * (K + 1);
            unsigned int c1 = *(volatile const unsigned int *)&st->cnt1;
            if (c1 > a.cap) c1 = a.cap;
            const long long nn = a.n_near, total = nn + c1;
            const float seed = load_pos_float(&st->seed_ub);
            const float *X32 = static_cast<const float *>(a.X);
            for (long long base = ((long long)blockIdx.x * NW + w) * EPW; base < total;
                 base += (long long)gridDim.x * NW * EPW) {
                int2 pr[EPW];
                bool valid[EPW];
#pragma unroll
                for (int e = 0; e < EPW; ++e) {
                    const long long idx = base + e;
                    valid[e] = idx < total;
                    pr[e] = valid[e] ? (idx < nn ? __ldcg(a.near + idx) : __ldcg(a.list + (idx - nn))) : make_int2(0, 0);
                }
                const float ub2 = load_pos_float(&st->run_ub2);
                float acc[M];
#pragma unroll
                for (int q = 0; q < M; ++q) acc[q] = 0.f;
#pragma unroll 2
                for (int l = lane; l < n; l += 32) {
                    float u[KU];
#pragma unroll
                    for (int c = 0; c < KU; c += 4) {
                        const float4 t = __ldcg(reinterpret_cast<const float4 *>(a.U32 + (size_t)l * a.KP + c));
                        u[c] = t.x; u[c + 1] = t.y; u[c + 2] = t.z; u[c + 3] = t.w;
                    }
#pragma unroll
                    for (int e = 0; e < EPW; ++e) {
                        const float D = X32[(size_t)pr[e].x * n + l] - X32[(size_t)pr[e].y * n + l];
                        acc[e * (K + 1) + K] = fmaf(D, D, acc[e * (K + 1) + K]);
#pragma unroll
                        for (int c = 0; c < K; ++c) acc[e * (K + 1) + c] = fmaf(u[c], D, acc[e * (K + 1) + c]);
                    }
                }
                // lane e < EPW finishes pair e
                float z[K + 1];
                if constexpr (M <= 32) {
                    constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
                    constexpr int dup = 32 / S;
                    float r[S];
#pragma unroll
                    for (int q = 0; q < S; ++q) r[q] = q < M ? acc[q < M ? q : 0] : 0.f;
                    const float t = warp_reduce_scatter<S>(r, lane);
                    const int e = lane < EPW ? lane : 0;
#pragma unroll
                    for (int c = 0; c <= K; ++c) z[c] = __shfl_sync(0xffffffffu, t, (e * (K + 1) + c) * dup);
                } else {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int q = 0; q < M; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
#pragma unroll
                    for (int c = 0; c <= K; ++c) z[c] = acc[c];
#pragma unroll
                    for (int e = 1; e < EPW; ++e)
                        if (lane == e)
#pragma unroll
                            for (int c = 0; c <= K; ++c) z[c] = acc[e * (K + 1) + c];
                }
                int2 mypr = pr[0];
                bool myvalid = valid[0];
#pragma unroll
                for (int e = 1; e < EPW; ++e)
                    if (lane == e) { mypr = pr[e]; myvalid = valid[e]; }
                const float dd = z[K];
                float zz = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) zz = fmaf(z[c], z[c], zz);
                const int code = (lane >= EPW || !myvalid) ? 0 : (dd < 1e-30f ? 2 : 1);  // 2: too short for FP32
                const float rr = code == 1 ? sqrtf(zz / dd) : INFINITY;
                const float wmin = warp_min(rr);
                float U = fminf(seed, ub2);
                if (wmin < INFINITY) {
                    const float ub = cert_upper(wmin, a.cert2);
                    if (lane == 0) atomic_min_pos_float(&st->run_ub2, ub);
                    U = fminf(U, ub);
                }
                const float th = cert_emit_threshold(U, a.cert2);
                unsigned int m = __ballot_sync(0xffffffffu, code == 2 || (code == 1 && rr <= th));
                if (m && lane == 0) atomicAdd((unsigned int *)&st->cnt2, (unsigned int)__popc(m));
                while (m) {
                    const int e = __ffs(m) - 1;
                    m &= m - 1;
                    int2 ij;
                    ij.x = __shfl_sync(0xffffffffu, mypr.x, e);
                    ij.y = __shfl_sync(0xffffffffu, mypr.y, e);
                    eval64(ij);
                }
            }
        } else {
            unsigned int cnt = a.which == 1 ? (unsigned int)st->cnt1 : (unsigned int)st->cnt2;
            if (cnt > a.cap) cnt = a.cap;
            // the pair is read (within the list's storage) before the count
            // is needed, so the two loads overlap
            for (unsigned int e = blockIdx.x + gridDim.x * w; e < a.cap; e += gridDim.x * NW) {
                const int2 ij = a.list[e];
                if (e >= cnt) break;  // uniform over the warp
                eval64(ij);
            }
        }
        if (lane == 0) sh.wb[w] = best;
        __syncthreads();
        if (tid == 0) {
            Partial b = sh.wb[0];
            for (int q = 1; q < NW; ++q)
                if (better_q(sh.wb[q].r, sh.wb[q].i, sh.wb[q].j, b.r, b.i, b.j)) b = sh.wb[q];
            a.partials[blockIdx.x] = b;
            __threadfence();
            const unsigned int t = atomicAdd(&st->ticket, 1u);
            sh.last = (t == gridDim.x - 1) ? 1 : 0;
        }
        __syncthreads();
        if (!sh.last) return;
        __threadfence();
    }

    // ---------------- phase 2: argmin, record, update ----------------------
    using WT = TX;  // working precision of the pivot, MGS and rotation
    // this thread's row of the current basis (n <= SB, k <= 8), loaded now so
    // that the loads overlap the argmin over the blocks' results
    constexpr int KR = K <= 8 ? K : 1;
    WT urow[KR];
    const bool have_row = K <= 8 && n <= SB && tid < n;
    if (have_row) {
#pragma unroll
        for (int c = 0; c < KR; ++c)
            urow[c] = c < kk ? (sizeof(WT) == 8 ? (WT)a.U64[(size_t)c * n + tid] : (WT)a.U32[(size_t)tid * a.KP + c])
                             : (WT)0;
    }
    // the basis entry (l, c) as the working precision reads it
    auto ucol = [&](int l, int c) -> WT {
        if (K <= 8 && have_row && l == tid) return urow[c < KR ? c : 0];
        return sizeof(WT) == 8 ? (WT)a.U64[(size_t)c * n + l] : (WT)a.U32[(size_t)l * a.KP + c];
    };
    if (w == 0) {
        Partial b = {INFINITY, 0x7fffffff, 0x7fffffff};
        for (int p = lane; p < (int)gridDim.x; p += 32) {
            const volatile Partial *vp = &a.partials[p];
            const Partial q = {vp->r, vp->i, vp->j};
            if (better_q(q.r, q.i, q.j, b.r, b.i, b.j)) b = q;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Partial q;
            q.r = __shfl_xor_sync(0xffffffffu, b.r, o);
            q.i = __shfl_xor_sync(0xffffffffu, b.i, o);
            q.j = __shfl_xor_sync(0xffffffffu, b.j, o);
            if (better_q(q.r, q.i, q.j, b.r, b.i, b.j)) b = q;
        }
        if (lane == 0) sh.wb[0] = b;
    } else if (w == 1) {
        // prefetch the problem state while warp 0 reduces
        if (lane == 0) {
            sh.iter = st->iter;
            sh.hist_cap = st->hist_cap;
            sh.cnt1 = st->cnt1;
            sh.cnt2 = st->cnt2;
            sh.watch_n = st->watch_n;
            sh.watch_pos = st->watch_pos;
        }
        if (lane < kWatch) sh.watch[lane] = st->watch[lane];
    }
    __syncthreads();
    if (tid == 0) {
        Partial b = sh.wb[0];
        const bool none = !(b.r < INFINITY);
        const double r = none ? b.r : sqrt(b.r);
        const int it = sh.iter;
        if (none) atomicOr(&st->status, ST_NO_SECANT);
        if (it < sh.hist_cap) {
            a.hist[it] = none ? __longlong_as_double(0x7ff8000000000000ll) : r;
            a.argmin[it] = none ? make_int2(-1, -1) : make_int2(b.i, b.j);
        }
        st->iter = it + 1;
        st->last_r = r;
        st->last_i = none ? -1 : b.i;
        st->last_j = none ? -1 : b.j;
        st->last_cnt1 = sh.cnt1;
        st->last_cnt2 = sh.cnt2;
        st->cnt1 = 0;
        st->tile_next = 0;
        st->cnt2 = 0;
        st->ticket = 0;
        st->run_ub1 = 0x7f800000u;
        st->run_ub2 = 0x7f800000u;
        if (!none) {
            bool present = false;
            for (int q = 0; q < sh.watch_n; ++q) present |= (sh.watch[q].x == b.i && sh.watch[q].y == b.j);
            if (!present) {
                sh.watch[sh.watch_pos] = make_int2(b.i, b.j);
                st->watch[sh.watch_pos] = make_int2(b.i, b.j);
                sh.watch_pos = (sh.watch_pos + 1) % kWatch;
                if (sh.watch_n < kWatch) ++sh.watch_n;
                st->watch_pos = sh.watch_pos;
                st->watch_n = sh.watch_n;
            }
            if (a.eval_only)  // the basis stays: the exact minimum bounds the next one
                st->seed_ub = __float_as_uint(__double2float_ru(r) * 1.000001f);
        }
        sh.wb[0].r = r;
    }
    __syncthreads();
    const Partial b = sh.wb[0];
    if (!(b.r < INFINITY) || a.eval_only) return;

    // the watch pairs' coordinates, loaded now and used at the very end
    const int nwatch = sh.watch_n;
    const bool prefetch = n <= 32 * kSeedRegs;
    float wxi[kSeedRegs], wxj[kSeedRegs];
    if (prefetch && w < nwatch) {
        const int2 pr = sh.watch[w];
#pragma unroll
        for (int q = 0; q < kSeedRegs; ++q) {
            const int l = lane + 32 * q;
            wxi[q] = l < n ? (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) : 0.f;
            wxj[q] = l < n ? (float)ld_x<TX>(a.X, (size_t)pr.y * n + l) : 0.f;
        }
    }

    const bool in_smem = K <= 8 && su_dyn_bytes<TX>(n, K) <= kDynSmem;
    double *Up = in_smem ? dyn : a.work;           // n x K: the new basis before QR
    WT *Ds = reinterpret_cast<WT *>(Up + (size_t)n * K);  // n
    // FP32 copy of the final basis (n x K) for the seeds, when in shared memory
    float *Uf = in_smem ? reinterpret_cast<float *>(dyn + (size_t)n * K + ((size_t)n * sizeof(WT) + 7) / 8) : nullptr;

    // 2. D = x_i - x_j, |D|^2 and U^T D in one multi-value reduction
    {
        WT v[K + 1];
#pragma unroll
        for (int q = 0; q <= K; ++q) v[q] = 0;
#pragma unroll 1
        for (int l = tid; l < n; l += SB) {
            const WT D = ld_x<TX>(a.X, (size_t)b.i * n + l) - ld_x<TX>(a.X, (size_t)b.j * n + l);
            Ds[l] = D;
            v[K] += D * D;
#pragma unroll
            for (int c = 0; c < K; ++c)
                if (c < kk) v[c] += ucol(l, c) * D;
        }
        WT *scr = sizeof(WT) == 8 ? (WT *)sh.red_d : (WT *)sh.red_f;
        warp_sum_multi<WT, K + 1>(v);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q <= K; ++q) scr[w * (K + 1) + q] = v[q];
        __syncthreads();
        if (tid <= K) {
            WT s = 0;
            for (int p = 0; p < NW; ++p) s += scr[p * (K + 1) + tid];
            sh.cvec[tid] = (double)s;
        }
        __syncthreads();
    }

    // 3-4. pivot, coefficient MGS on [c, e_l (l != t)] and the rotation
    //      coefficients, in one thread (k x k work, unrolled for small k)
    if (tid == 0) {
        const WT d = sqrt((WT)sh.cvec[K]);
        WT c[K];
        WT r2 = 0;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            c[q] = q < kk ? (WT)sh.cvec[q] / d : (WT)0;
            r2 += c[q] * c[q];
        }
        int t = 0;
        WT cmax = fabs(c[0]);
#pragma unroll
        for (int q = 1; q < K; ++q)
            if (q < kk && fabs(c[q]) > cmax) { cmax = fabs(c[q]); t = q; }
        WT Q[K][K];
        bool alive[K];
#pragma unroll
        for (int m = 0; m < K; ++m) {
            WT x[K];
            const int l = (m - 1) < t ? (m - 1) : m;  // list entry m >= 1 is column l
#pragma unroll
            for (int q = 0; q < K; ++q) x[q] = m == 0 ? c[q] : (q == l ? (WT)1 : (WT)0);
#pragma unroll
            for (int p = 0; p < K; ++p) {
                if (p >= m || !alive[p]) continue;
                WT h = 0;
#pragma unroll
                for (int q = 0; q < K; ++q) h += Q[p][q] * x[q];
#pragma unroll
                for (int q = 0; q < K; ++q) x[q] -= h * Q[p][q];
            }
            WT nn = 0;
#pragma unroll
            for (int q = 0; q < K; ++q) nn += x[q] * x[q];
            alive[m] = m < kk && nn > (WT)0;
            const WT inv = alive[m] ? (WT)1 / sqrt(nn) : (WT)0;
#pragma unroll
            for (int q = 0; q < K; ++q) Q[m][q] = x[q] * inv;
        }
#pragma unroll
        for (int m = 0; m < K; ++m)
#pragma unroll
            for (int q = 0; q < K; ++q) sh.Bw[q][m] = Q[m][q];
#pragma unroll
        for (int q = 0; q < K; ++q) sh.cw[q] = c[q];
        sh.alive0 = alive[0];
        const WT al = (WT)a.alpha;
        WT av, as;
        if (a.mode == 1) {  // angle reading
            const WT nv = sqrt(r2);
            const WT ne = sqrt(r2 < (WT)1 ? (WT)1 - r2 : (WT)0);
            av = (nv > 0 ? (1 - al) / nv : (WT)0) - (ne > 0 ? al / ne : (WT)0);
            as = ne > 0 ? al / ne : (WT)0;
        } else {            // literal reading: (1-a) v + a (s - v)
            av = 1 - 2 * al;
            as = al;
        }
        sh.av = av;
        sh.asd = as / d;  // applied to D = d s
        sh.dnorm = d;
    }
    __syncthreads();

    // new basis before QR: column 0 = av U c + as s, column m >= 1 = U q_m
    {
        const WT av = sh.av, asd = sh.asd;
        WT p0 = 0;
#pragma unroll 1
        for (int l = tid; l < n; l += SB) {
            WT u[K];
#pragma unroll
            for (int c = 0; c < K; ++c)
                u[c] = c < kk ? ucol(l, c) : (WT)0;
            WT v0 = 0;
#pragma unroll
            for (int c = 0; c < K; ++c) v0 += u[c] * sh.cw[c];
            const WT d0 = av * v0 + asd * Ds[l];
            p0 += d0 * d0;
            WT col[K];
            col[0] = d0;
#pragma unroll
            for (int m = 1; m < K; ++m) {
                WT s = 0;
#pragma unroll
                for (int c = 0; c < K; ++c) s += u[c] * sh.Bw[c][m];
                col[m] = s;
            }
            // q1 in place of column 0 when the direction vanishes (alpha = 1
            // with s in the span); s itself when P P^T s = 0
            WT q1 = 0;
#pragma unroll
            for (int c = 0; c < K; ++c) q1 += u[c] * sh.Bw[c][0];
            Ds[l] = sh.alive0 ? q1 : Ds[l] / sh.dnorm;
#pragma unroll
            for (int m = 0; m < K; ++m) Up[(size_t)l * K + m] = (double)col[m];
        }
        WT pv[1] = {p0};
        WT *scr = sizeof(WT) == 8 ? (WT *)sh.red_d : (WT *)sh.red_f;
        block_sum_multi<WT, 1>(pv, scr, &sh.nd2);
        const double nd = sqrt((double)sh.nd2);
#pragma unroll 1
        for (int l = tid; l < n; l += SB)
            Up[(size_t)l * K] = nd > 0.0 ? Up[(size_t)l * K] / nd : (double)Ds[l];
        __syncthreads();
    }

    // 5. FP64 Gram matrix of U' (upper triangle)
    if constexpr (K * (K + 1) / 2 <= 32) {
        // every thread sums the products of its rows; one reduce-scatter per
        // warp; the warps' partials are added in shared memory
        constexpr int M = K * (K + 1) / 2;
        constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
        constexpr int dup = 32 / S;
        const int nrw = (min(n, SB) + 31) >> 5;  // warps holding rows
        if (w < nrw) {
            double g[S];
#pragma unroll
            for (int e = 0; e < S; ++e) g[e] = 0.0;
#pragma unroll 1
            for (int l = tid; l < n; l += SB) {
                double row[K];
#pragma unroll
                for (int m = 0; m < K; ++m) row[m] = m < kk ? Up[(size_t)l * K + m] : 0.0;
                int e = 0;
#pragma unroll
                for (int p = 0; p < K; ++p)
#pragma unroll
                    for (int q = p; q < K; ++q) {
                        g[e] = fma(row[p], row[q], g[e]);
                        ++e;
                    }
            }
            const double t = warp_reduce_scatter<S>(g, lane);
            if (lane % dup == 0) sh.gred[w][rs_index<S>(lane)] = t;
        }
        __syncthreads();
        if (tid < M) {
            int p = 0, e = tid;
            while (e >= K - p) { e -= K - p; ++p; }
            double sum = 0.0;
            for (int q = 0; q < nrw; ++q) sum += sh.gred[q][tid];
            sh.G[p][p + e] = sum;
        }
    } else {
        // entries spread over the warps
#pragma unroll 1
        for (int e = w; e < kk * kk; e += NW) {
            const int p = e / kk, q = e % kk;
            if (q < p) continue;
            double s = 0.0;
            for (int l = lane; l < n; l += 32) s = fma(Up[(size_t)l * K + p], Up[(size_t)l * K + q], s);
            s = warp_sum(s);
            if (lane == 0) sh.G[p][q] = s;
        }
    }
    __syncthreads();
    if (w == 0) {
        // E = G - I; the series needs max|E| <= 1e-6 (a vote, not an FP64
        // max-reduction; NaN entries are ignored as fmax would ignore them)
        bool small = true;
        for (int e = lane; e < kk * kk; e += 32) {
            const int p = e / kk, q = e % kk;
            if (q >= p && fabs(sh.G[p][q] - (p == q ? 1.0 : 0.0)) > 1e-6) small = false;
        }
        small = __all_sync(0xffffffffu, small);
        if (Shared<TX, K>::KS == K && small) {
            // S1 = triu(E) with the diagonal halved (FP64), S2 = the same of
            // -S1^T S1, R = S1 + S2, and (I + R)^-1 = I - S1 + [S1^2 - S2] +
            // O(|E|^3).  The bracket is second order (<= k^2 1e-12): its FP32
            // evaluation from FP32(S1) errs by ~1e-19, below FP64 rounding of
            // the unit diagonal, so each lane forms its entries independently.
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                const double v = q > p ? sh.G[p][q] : (q == p ? 0.5 * (sh.G[p][p] - 1.0) : 0.0);
                sh.T1[p][q] = v;
                sh.S1f[p][q] = (float)v;
            }
            __syncwarp();
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                if (q < p) {
                    sh.Ri[p][q] = 0.0;
                    continue;
                }
                float sq = 0.f, tt = 0.f;
                for (int m = p; m <= q; ++m) sq = fmaf(sh.S1f[p][m], sh.S1f[m][q], sq);  // (S1^2)_pq
                for (int m = 0; m <= p; ++m) tt = fmaf(sh.S1f[m][p], sh.S1f[m][q], tt);  // (S1^T S1)_pq
                const float second = sq + (q > p ? tt : 0.5f * tt);                      // S1^2 - S2
                sh.Ri[p][q] = (p == q ? 1.0 : 0.0) - sh.T1[p][q] + (double)second;
            }
        } else if (small) {
            // R1 = triu(E) with the diagonal halved; R2 from -R1^T R1 the same
            // way; R = R1 + R2; (I + R)^-1 = I - R + R^2 (error O(|E|^3))
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                sh.T1[p][q] = q > p ? sh.G[p][q] : (q == p ? 0.5 * (sh.G[p][p] - 1.0) : 0.0);
            }
            __syncwarp();
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                double s = 0.0;
                for (int m = 0; m <= (p < q ? p : q); ++m) s = fma(sh.T1[m][p], sh.T1[m][q], s);
                sh.T2[p][q] = s;  // (R1^T R1)_pq
            }
            __syncwarp();
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                const double r2v = q > p ? -sh.T2[p][q] : (q == p ? -0.5 * sh.T2[p][p] : 0.0);
                sh.G[p][q] = sh.T1[p][q] + r2v;  // R (upper; lower entries zero)
            }
            __syncwarp();
            for (int e = lane; e < kk * kk; e += 32) {
                const int p = e / kk, q = e % kk;
                double s = 0.0;
                for (int m = p; m <= q; ++m) s = fma(sh.G[p][m], sh.G[m][q], s);  // (R^2)_pq
                sh.Ri[p][q] = (p == q ? 1.0 : 0.0) - (q >= p ? sh.G[p][q] : 0.0) + (q >= p ? s : 0.0);
            }
        } else {
            // direct right-looking Cholesky on the upper triangle (lane m owns
            // column m), then (R)^-1 by back substitution
            double rinv_own = 0.0;
#pragma unroll 1
            for (int j = 0; j < kk; ++j) {
                const double gjj = sh.G[j][j];
                const double rinv = rsqrt(gjj);
                if (lane == j) { sh.G[j][j] = gjj * rinv; rinv_own = rinv; }
                if (lane > j && lane < kk) sh.G[j][lane] *= rinv;
                __syncwarp();
                if (lane > j && lane < kk)
                    for (int p = j + 1; p <= lane; ++p) sh.G[p][lane] = fma(-sh.G[j][p], sh.G[j][lane], sh.G[p][lane]);
                __syncwarp();
            }
            if (lane < kk) sh.Rd[lane] = rinv_own;
            __syncwarp();
            if (lane < kk) {
                for (int i = 0; i < kk; ++i) sh.Ri[i][lane] = 0.0;
#pragma unroll 1
                for (int i = lane; i >= 0; --i) {
                    double s = (i == lane) ? 1.0 : 0.0;
                    for (int p = i + 1; p <= lane; ++p) s = fma(-sh.G[i][p], sh.Ri[p][lane], s);
                    sh.Ri[i][lane] = s * sh.Rd[i];
                }
            }
        }
    }
    __syncthreads();

    // 6. U'' = U' (I + R)^-1, written in every form the kernels read
#pragma unroll 1
    for (int l = tid; l < n; l += SB) {
        double row[K];
#pragma unroll
        for (int m = 0; m < K; ++m) row[m] = m < kk ? Up[(size_t)l * K + m] : 0.0;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            if (m >= kk) break;
            double s = 0.0;
#pragma unroll
            for (int p = 0; p < K; ++p)
                if (p <= m) s = fma(row[p], sh.Ri[p][m], s);
            a.U64[(size_t)m * n + l] = s;
            const float sf = (float)s;
            a.U32[(size_t)l * a.KP + m] = sf;
            if (Uf) Uf[(size_t)l * K + m] = sf;
            if (a.U32lo) a.U32lo[(size_t)l * a.KP + m] = (float)(s - (double)sf);
            if (a.Uhi) {
                // hi + lo * 2^-s of the FP32 value (the FP32 rounding adds 2^-24
                // relative to the split residual)
                const size_t idx = (size_t)m * a.NP + l;
                if (a.split_bf16) {
                    const __nv_bfloat16 h = __float2bfloat16_rn(sf);
                    static_cast<__nv_bfloat16 *>(a.Uhi)[idx] = h;
                    static_cast<__nv_bfloat16 *>(a.Ulo)[idx] =
                        __float2bfloat16_rn((sf - __bfloat162float(h)) * a.split_scale);
                } else {
                    const __half h = __float2half_rn(sf);
                    static_cast<__half *>(a.Uhi)[idx] = h;
                    static_cast<__half *>(a.Ulo)[idx] = __float2half_rn((sf - __half2float(h)) * a.split_scale);
                }
            }
        }
    }
    __syncthreads();

    // seeds: the recent argmin pairs under the new basis
    if (w < nwatch) {
        const int2 pr = sh.watch[w];
        float seed = INFINITY;
        if (sizeof(TX) == 8) {
            double v[K + 1];
#pragma unroll
            for (int q = 0; q <= K; ++q) v[q] = 0.0;
            for (int l = lane; l < n; l += 32) {
                const double D = (double)ld_x<TX>(a.X, (size_t)pr.x * n + l) - (double)ld_x<TX>(a.X, (size_t)pr.y * n + l);
                v[K] = fma(D, D, v[K]);
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (c < kk) v[c] = fma(a.U64[(size_t)c * n + l], D, v[c]);
            }
            warp_sum_multi<double, K + 1>(v);
            double zz = 0.0;
#pragma unroll
            for (int c = 0; c < K; ++c) zz = fma(v[c], v[c], zz);
            if (v[K] > 0.0) seed = __double2float_ru(sqrt(zz / v[K])) * 1.000001f;
        } else {
            float v[K + 1];
#pragma unroll
            for (int q = 0; q <= K; ++q) v[q] = 0.f;
            if (prefetch) {
#pragma unroll
                for (int q = 0; q < kSeedRegs; ++q) {
                    const int l = lane + 32 * q;
                    if (l < n) {
                        const float D = wxi[q] - wxj[q];
                        v[K] = fmaf(D, D, v[K]);
                        const float *ur = Uf ? Uf + (size_t)l * K : a.U32 + (size_t)l * a.KP;
#pragma unroll
                        for (int c = 0; c < K; ++c)
                            if (c < kk) v[c] = fmaf(ur[c], D, v[c]);
                    }
                }
            } else {
                for (int l = lane; l < n; l += 32) {
                    const float D = (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) - (float)ld_x<TX>(a.X, (size_t)pr.y * n + l);
                    v[K] = fmaf(D, D, v[K]);
                    const float *ur = Uf ? Uf + (size_t)l * K : a.U32 + (size_t)l * a.KP;
#pragma unroll
                    for (int c = 0; c < K; ++c)
                        if (c < kk) v[c] = fmaf(ur[c], D, v[c]);
                }
            }
            warp_sum_multi<float, K + 1>(v);
            float zz = 0.f;
#pragma unroll
            for (int c = 0; c < K; ++c) zz = fmaf(v[c], v[c], zz);
            if (v[K] > 1e-30f) seed = cert_upper(sqrtf(zz / v[K]), a.seed_cert);
        }
        if (lane == 0) sh.seed[w] = seed;
    }
    __syncthreads();
    if (tid == 0) {
        float m = INFINITY;
        for (int q = 0; q < nwatch; ++q) m = fminf(m, sh.seed[q]);
        st->seed_ub = __float_as_uint(m);
    }
}

template <typename TX, int K>
cudaError_t launch_su(const SelectUpdateArgs &a, cudaStream_t s)
{
    const size_t need = su_dyn_bytes<TX>(a.n, K);
    const size_t shm = (K <= 8 && need <= kDynSmem) ? need : 0;
    return launch_pdl(a.pdl != 0, select_update_kernel<TX, K>, dim3(a.grid), dim3(SB), shm, s, a);
}

template <typename TX>
cudaError_t launch_su_t(const SelectUpdateArgs &a, cudaStream_t s)
{
    switch (a.k) {
    case 1: return launch_su<TX, 1>(a, s);
    case 2: return launch_su<TX, 2>(a, s);
    case 3: return launch_su<TX, 3>(a, s);
    case 4: return launch_su<TX, 4>(a, s);
    case 5: return launch_su<TX, 5>(a, s);
    case 6: return launch_su<TX, 6>(a, s);
    case 7: return launch_su<TX, 7>(a, s);
    case 8: return launch_su<TX, 8>(a, s);
    default: break;
    }
    if (a.k <= 12) return launch_su<TX, 12>(a, s);
    if (a.k <= 16) return launch_su<TX, 16>(a, s);
    if (a.k <= 24) return launch_su<TX, 24>(a, s);
    return launch_su<TX, 32>(a, s);
}

} // namespace

cudaError_t launch_select_update(const SelectUpdateArgs &a, cudaStream_t s)
{
    return a.x_is_f64 ? launch_su_t<double>(a, s) : launch_su_t<float>(a, s);
}

} // namespace sap
