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
constexpr int kQW = 4;           // warps of the small-basis update (one row per thread, n <= 128)

// Named barriers of phase 2: warps 0..kQW-1 (the small-basis update) and
// warps kQW..NW-1 (recording and seed prefetch); barrier 0 is __syncthreads.
__device__ __forceinline__ void quad_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kQW * 32) : "memory"); }
__device__ __forceinline__ void seed_bar() { asm volatile("bar.sync 2, %0;" ::"n"(SB - kQW * 32) : "memory"); }

// 1/sqrt(x) in the working precision (FP32: the hardware approximation)
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

// An approximate 1/sqrt(x) for x > 0 used as a column scale: the FP32
// hardware estimate (relative error ~2^-23), widened.  A scale s applied to
// column 0 of the Gram matrix (G' = S G S, S = diag(s, 1, ...)) and to row 0
// of the Cholesky factor's inverse gives the same orthonormal basis for any
// s; it only has to bring G'_00 within the series' 1e-5 of one, and this
// estimate leaves it within ~5e-7.  (Each dependent FP64 operation costs
// about 0.12 us here, so Newton steps toward full precision are not taken.)
__device__ __forceinline__ double rsqrt_scale(double x)
{
    const float xf = (float)x;
    if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / sqrt(x);
    return (double)rsqrtf(xf);
}

template <typename TX>
__device__ __forceinline__ TX ld_x(const void *X, size_t idx)
{
    return static_cast<const TX *>(X)[idx];
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
    static constexpr int GQ = K == 8 ? 36 : 1;
    double gq[K == 8 ? kQW : 1][GQ];  // per-warp Gram sums of the small-basis update (k = 8)
    float R2f[KS][KS], Sqf[KS][KS];  // second-order terms of the series (K <= 8)
    int degen;                     // the rotated direction vanished (small-basis update)
    int scan[33];
};

// FP64 evaluation of one pair by a warp: D = x_i - x_j, d^2 = |D|^2 and
// z = U^T D from explicit FP64 differences, the exclusion rules applied
// exactly (d^2 == 0: not distinct, Sec. II; d^2 < eps^2: shorter than the
// threshold, Sec. VII); keeps the best squared ratio q = |z|^2 / d^2 (ties
// to the smallest pair index).
template <typename TX, int K>
__device__ __forceinline__ void fp64_eval(const SelectUpdateArgs &a, int2 ij, int lane, Partial &best)
{
    if (!SAP_PAIR_OK(a.st, ij, a.N)) return;
    const int n = a.n, kk = a.k;
    double v[K + 1];
#pragma unroll
    for (int q = 0; q <= K; ++q) v[q] = 0.0;
#pragma unroll 4
    for (int l = lane; l < n; l += 32) {
        const double D = (double)ld_x<TX>(a.X, (size_t)ij.x * n + l) - (double)ld_x<TX>(a.X, (size_t)ij.y * n + l);
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
}

// The same evaluation from coordinates prefetched in registers (rows
// l = lane + 32 r, r < R) and the basis's hi and lo FP32 parts in shared
// memory (row-major, stride K).
template <int K, int E, int R>
__device__ __forceinline__ void df_eval_pref(const float (&xi)[E][R], const float (&xj)[E][R], const float *Uh,
                                             const float *Ul, int n, const bool (&valid)[E], int lane, float &rr,
                                             int &code)
{
    float zh[E][K + 1], zl[E][K + 1];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int q = 0; q <= K; ++q) zh[e][q] = zl[e][q] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = lane + 32 * r;
        if (l >= n) break;
        float uh[K], ul[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            uh[c] = Uh[l * K + c];
            ul[c] = Ul[l * K + c];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float D = xi[e][r] - xj[e][r];
            xs_fma(zh[e][K], zl[e][K], D, D, 0.f);
#pragma unroll
            for (int c = 0; c < K; ++c) xs_fma(zh[e][c], zl[e][c], D, uh[c], ul[c]);
        }
    }
    df_finish<K, E>(zh, zl, valid, lane, rr, code);
}


// (I + R)^-1 of the Cholesky factor I + R of the Gram matrix in sh.G (upper
// triangle), by warp 0: the second-order series in E = G - I when
// max|E| <= 1e-6, else a direct Cholesky factorisation and back substitution.
template <typename TX, int K>
__device__ __forceinline__ void chol_inverse(Shared<TX, K> &sh, int kk, int lane)
{
    // E = G - I; the series needs max|E| <= 1e-5 (third order, k <= 8) or
    // 1e-6 (second order) (a vote, not an FP64 max-reduction; NaN entries
    // are ignored as fmax would ignore them)
    constexpr int KS = Shared<TX, K>::KS;
    const double lim = KS == K ? 1e-5 : 1e-6;
    bool small = true;
    // k = K: compile-time bounds, loops unrolled with predicated iterations
    // (straight-line code: it runs once per launch, so its instruction
    // fetch is part of the critical path)
    constexpr int NREP = (K * K + 31) / 32;
    if (KS == K) {
#pragma unroll
        for (int rep = 0; rep < NREP; ++rep) {
            const int e = lane + 32 * rep;
            const int p = e / K, q = e % K;
            if (e < K * K && q >= p && fabs(sh.G[p % K][q % K] - (p == q ? 1.0 : 0.0)) > lim) small = false;
        }
    } else {
        for (int e = lane; e < kk * kk; e += 32) {
            const int p = e / kk, q = e % kk;
            if (q >= p && fabs(sh.G[p][q] - (p == q ? 1.0 : 0.0)) > lim) small = false;
        }
    }
    small = __all_sync(0xffffffffu, small);
    if (KS == K && small) {
        // G = (I + R)^T (I + R) with R = R1 + R2 + R3 + O(|E|^4) by orders:
        // R1 = S1 = triu(E) with the diagonal halved (FP64), R2 = split of
        // -R1^T R1, R3 = split of -(R1^T R2 + R2^T R1) (split: upper
        // triangle, diagonal halved), and (I + R)^-1 = I - R1 - R2 - R3 +
        // R1^2 + R1 R2 + R2 R1 - R1^3 + O(|E|^4).  Every term past R1 is at
        // most k^2 1e-10: its FP32 evaluation from FP32(R1) errs by ~1e-17,
        // below FP64 rounding of the unit diagonal, and the truncation by
        // ~1e-20; each lane forms its entries independently.
#pragma unroll
        for (int rep = 0; rep < NREP; ++rep) {
            const int e = lane + 32 * rep;
            const int p = (e / K) % K, q = e % K;
            if (e < K * K) {
                const double v = q > p ? sh.G[p][q] : (q == p ? 0.5 * (sh.G[p][p] - 1.0) : 0.0);
                sh.T1[p][q] = v;
                sh.S1f[p % KS][q % KS] = (float)v;
            }
        }
        __syncwarp();
#pragma unroll
        for (int rep = 0; rep < NREP; ++rep) {
            const int e = lane + 32 * rep;
            const int p = (e / K) % K, q = e % K;
            if (e < K * K) {
                float tt = 0.f, sq = 0.f;
                if (q >= p) {
#pragma unroll
                    for (int m = 0; m < K; ++m)
                        if (m <= p) tt = fmaf(sh.S1f[m % KS][p % KS], sh.S1f[m % KS][q % KS], tt);  // (R1^T R1)_pq
#pragma unroll
                    for (int m = 0; m < K; ++m)
                        if (m >= p && m <= q) sq = fmaf(sh.S1f[p % KS][m % KS], sh.S1f[m % KS][q % KS], sq);  // (R1^2)_pq
                }
                sh.R2f[p % KS][q % KS] = q > p ? -tt : (q == p ? -0.5f * tt : 0.f);
                sh.Sqf[p % KS][q % KS] = q >= p ? sq : 0.f;
            }
        }
        __syncwarp();
#pragma unroll
        for (int rep = 0; rep < NREP; ++rep) {
            const int e = lane + 32 * rep;
            const int p = (e / K) % K, q = e % K;
            if (e < K * K) {
                if (q < p) {
                    sh.Ri[p][q] = 0.0;
                } else {
                    float m3 = 0.f, r12 = 0.f, r21 = 0.f, r13 = 0.f;
#pragma unroll
                    for (int m = 0; m < K; ++m)
                        if (m <= p) {
                            m3 = fmaf(sh.S1f[m % KS][p % KS], sh.R2f[m % KS][q % KS], m3);
                            m3 = fmaf(sh.R2f[m % KS][p % KS], sh.S1f[m % KS][q % KS], m3);
                        }
#pragma unroll
                    for (int m = 0; m < K; ++m)
                        if (m >= p && m <= q) {
                            r12 = fmaf(sh.S1f[p % KS][m % KS], sh.R2f[m % KS][q % KS], r12);  // (R1 R2)_pq
                            r21 = fmaf(sh.R2f[p % KS][m % KS], sh.S1f[m % KS][q % KS], r21);  // (R2 R1)_pq
                            r13 = fmaf(sh.Sqf[p % KS][m % KS], sh.S1f[m % KS][q % KS], r13);  // (R1^3)_pq
                        }
                    const float r3 = q > p ? -m3 : -0.5f * m3;
                    const float hi = -sh.R2f[p % KS][q % KS] - r3 + sh.Sqf[p % KS][q % KS] + r12 + r21 - r13;
                    sh.Ri[p][q] = (p == q ? 1.0 : 0.0) - sh.T1[p][q] + (double)hi;
                }
            }
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
    __syncwarp();
}

// One basis row l of U'' = U' (I + R)^-1 (row[] = U' row l), written in every
// form the kernels read: FP64 column-major, FP32 row-major (and its FP32
// residual), the split 16-bit operands of the tensor-core product, and (Uf,
// optional) an FP32 copy in shared memory for the seeds.
template <typename TX, int K>
__device__ __forceinline__ void write_row(const SelectUpdateArgs &a, const Shared<TX, K> &sh, int kk, int l,
                                          const double (&row)[K], float *Uf, float *Ulf = nullptr)
{
    const int n = a.n;
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
        if (a.U32lo || Ulf) {
            const float lo = (float)(s - (double)sf);
            if (a.U32lo) a.U32lo[(size_t)l * a.KP + m] = lo;
            if (Ulf) Ulf[(size_t)l * K + m] = lo;
        }
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

template <typename TX, int K>
__global__ void __launch_bounds__(SB) select_update_kernel(SelectUpdateArgs a)
{
    extern __shared__ double dyn[];
    __shared__ Shared<TX, K> sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = a.n;
    const int kk = a.k;            // actual k (<= K)
    ProbState *st = a.st;
    bool fused3 = false;
    if constexpr (sizeof(TX) == 4 && K <= 8) fused3 = a.fused == 3;

    constexpr int KW = K <= 8 ? K : 1;

    // Programmatic launch: the next iteration's product may start its
    // prologue (it waits for this kernel before reading the basis).  The
    // fused extended tier reads the near list (fixed) and the previous
    // iteration's basis and seed bound before it waits for the pass, so its
    // near pairs are evaluated while the pass may still run.
    if (!fused3) {
        grid_dep_launch();
        grid_dep_wait();
    }
    Partial best = {INFINITY, 0x7fffffff, 0x7fffffff};
    if (a.pass_parts > 0) {
        // the pass evaluated every candidate: its blocks' best pairs wait in
        // partials[], and this single block goes straight to phase 2
    } else if (fused3) {
        // ---------------- phase 1 (fused == 3): extended-precision tier ----
        // Each warp evaluates E0 listed pairs from explicit differences in
        // extended precision, tightens the running bound from their minimum
        // and evaluates in FP64 at once every pair that can still be the
        // argmin under the bound it holds (valid whenever it is read).  The
        // seed bound comes from the previous update's extended-precision
        // evaluation of the recent argmin pairs, so it is within ~1e-7 of
        // the minimum whenever that pair recurs.
        const float seed = load_pos_float(&st->seed_ub);
        const float *X32 = reinterpret_cast<const float *>(a.X);
        for (int seg = 0; seg < (a.pdl ? 2 : 1); ++seg) {
            long long nn = a.n_near, total = a.n_near;
            if (seg == 1 || !a.pdl) {
                grid_dep_wait();
                grid_dep_launch();
                unsigned int c1 = *(volatile const unsigned int *)&st->cnt1;
                if (c1 > a.cap) c1 = a.cap;
                nn = a.pdl ? 0 : a.n_near;
                total = nn + c1;
            }
            constexpr int E0 = (KW + 1) <= 8 ? 4 : 2;  // pairs per warp per round
            for (long long base = ((long long)blockIdx.x * NW + w) * E0; base < total;
                 base += (long long)gridDim.x * NW * E0) {
                int2 pr[E0];
                bool valid[E0];
#pragma unroll
                for (int e = 0; e < E0; ++e) {
                    const long long idx = base + e;
                    valid[e] = idx < total;
                    pr[e] = valid[e] ? (idx < nn ? __ldcg(a.near + idx) : __ldcg(a.list + (idx - nn)))
                                     : make_int2(0, 0);
                }
                // any earlier value of the running bound is a valid (looser)
                // bound: read it now, so its latency overlaps the evaluation
                const float ub2 = load_pos_float(&st->run_ub2);
                float rr;
                int code;
                df_eval<KW, E0>(X32, n, a.U32, a.U32lo, a.KP, pr, valid, lane, rr, code);
                const float wmin = warp_min(rr);
                float U = fminf(seed, ub2);
                if (wmin < INFINITY) {
                    const float ub = cert_upper(wmin, a.cert2);
                    if (lane == 0 && ub < ub2) atomic_min_pos_float(&st->run_ub2, ub);
                    U = fminf(U, ub);
                }
                const float th = cert_emit_threshold(U, a.cert2);
                unsigned int m = __ballot_sync(0xffffffffu, code == 2 || (code == 1 && rr <= th));
                if (m && lane == 0) atomicAdd((unsigned int *)&st->cnt2, (unsigned int)__popc(m));
                int2 mp = pr[0];
#pragma unroll
                for (int e = 1; e < E0; ++e)
                    if (lane == e) mp = pr[e];
                while (m) {
                    const int e = __ffs(m) - 1;
                    m &= m - 1;
                    int2 ij;
                    ij.x = __shfl_sync(0xffffffffu, mp.x, e);
                    ij.y = __shfl_sync(0xffffffffu, mp.y, e);
                    fp64_eval<TX, K>(a, ij, lane, best);
                }
            }
        }
    } else {
        // ---------------- phase 1: FP64 recheck of the candidate list ------
        bool fused = false;
        if constexpr (sizeof(TX) == 4) fused = a.fused == 2;  // FP32 data only
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
                    fp64_eval<TX, K>(a, ij, lane, best);
                }
            }
        } else if (sizeof(TX) == 4 && a.fused == 4) {
            // the extended-precision tier's list with its ratios: every pair
            // that can still be the argmin under the final running bound is
            // evaluated in FP64 (the tier emitted against earlier, looser
            // values of the bound)
            unsigned int cnt = *(volatile const unsigned int *)&st->cnt2;
            if (cnt > a.cap) cnt = a.cap;
            const float U = fminf(load_pos_float(&st->seed_ub), load_pos_float(&st->run_ub2));
            const float th = cert_emit_threshold(U, a.cert2);
            const unsigned long long *lst = reinterpret_cast<const unsigned long long *>(a.list);
            for (unsigned int e = blockIdx.x + gridDim.x * w; e < cnt; e += gridDim.x * NW) {
                const unsigned long long v = __ldcg(lst + e);
                if (packed_ratio(v) <= th) fp64_eval<TX, K>(a, packed_pair(v), lane, best);  // uniform
            }
        } else {
            unsigned int cnt = a.which == 1 ? (unsigned int)st->cnt1 : (unsigned int)st->cnt2;
            if (cnt > a.cap) cnt = a.cap;
            // the pair is read (within the list's storage) before the count
            // is needed, so the two loads overlap
            for (unsigned int e = blockIdx.x + gridDim.x * w; e < a.cap; e += gridDim.x * NW) {
                const int2 ij = a.list[e];
                if (e >= cnt) break;  // uniform over the warp
                fp64_eval<TX, K>(a, ij, lane, best);
            }
        }
    }
    // each block publishes its best; the last block to finish continues
    if (lane == 0) sh.wb[w] = best;
    __syncthreads();
    if (a.pass_parts > 0) {
        if (tid == 0) sh.last = 1;
    } else if (tid == 0) {
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

    // ---------------- phase 2: argmin, record, update ----------------------
    using WT = TX;  // working precision of the pivot, MGS and rotation
    // Small bases (k <= 8, n <= 128) are updated by warps 0-3 with one basis
    // row per thread (qpath): the FP64 steps then spread over the SM's four
    // sub-partitions, the k x k steps (pivot, coefficient MGS, rotation) run
    // redundantly in every thread on identical sums, and the four warps meet
    // at named barriers only; warps 4-7 meanwhile record the result and
    // fetch the seed pairs.  Larger bases are updated by the whole block.
    const bool qpath = K <= 8 && n <= 32 * kQW;  // block-uniform
    // this thread's row of the current basis (n <= SB, k <= 8), loaded now
    // so that the loads overlap the argmin over the blocks' results
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
        const int nparts = a.pass_parts > 0 ? a.pass_parts : (int)gridDim.x;
        // eight results per lane and round, their loads issued together
        // (L2 only: the writers were other blocks)
        for (int p0 = 0; p0 < nparts; p0 += 256) {
            long long rq[8], ij[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int p = p0 + lane + 32 * u;
                const long long *src = reinterpret_cast<const long long *>(a.partials + (p < nparts ? p : 0));
                rq[u] = __ldcg(src);
                ij[u] = __ldcg(src + 1);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (p0 + lane + 32 * u >= nparts) break;
                const Partial q = {__longlong_as_double(rq[u]), (int)(ij[u] & 0xffffffff), (int)(ij[u] >> 32)};
                if (better_q(q.r, q.i, q.j, b.r, b.i, b.j)) b = q;
            }
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

    // record the result (history, state, watch list); the best pair's
    // squared ratio is in sh.wb[0] and is not modified here
    auto record = [&](const Partial &b) {
        const bool none = !(b.r < INFINITY);
        if (a.shard_rec) {  // one rank's shard: its minimum, then a clean state
            *a.shard_rec = none ? Partial{INFINITY, -1, -1} : b;
            st->last_cnt1 = sh.cnt1;
            st->last_cnt2 = sh.cnt2;
            st->cnt1 = 0;
            st->tile_next = 0;
            st->cnt2 = 0;
            st->ticket = 0;
            st->run_ub1 = 0x7f800000u;
            st->run_ub2 = 0x7f800000u;
            return;
        }
        const double r = none ? b.r : sqrt(b.r);
        const int it = sh.iter;
        if (!none) {
            // whether the seed bound this evaluation started from was tight
            const float sd = __uint_as_float(st->seed_ub);
            st->seed_miss = sd <= (float)r * 1.01f ? 0 : min(st->seed_miss + 1, 1 << 20);
        }
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
    };

    if (qpath) {
        const Partial b = sh.wb[0];
        const bool go = b.r < INFINITY && !a.eval_only;  // block-uniform
        // the new basis's FP32 hi and lo parts for the seeds (FP32 data)
        float *Ufs = sizeof(TX) == 4 ? reinterpret_cast<float *>(dyn) : nullptr;
        float *Uls = sizeof(TX) == 4 ? Ufs + n * K : nullptr;
        float wxi[2][kQW], wxj[2][kQW];  // seed pairs' coordinates (warps 4-7)
        if (w < kQW) {
            if (go) {
                // rows l = tid; threads beyond n carry zero rows
                const int l = tid;
                const bool ok = l < n;
                WT u[KW];
#pragma unroll
                for (int c = 0; c < KW; ++c) u[c] = (ok && c < kk) ? urow[c < KR ? c : 0] : (WT)0;
                // 2. D = x_i - x_j, |D|^2 and U^T D
                const WT D = ok ? (WT)ld_x<TX>(a.X, (size_t)b.i * n + l) - (WT)ld_x<TX>(a.X, (size_t)b.j * n + l)
                                : (WT)0;
                WT v[KW + 1];
#pragma unroll
                for (int c = 0; c < KW; ++c) v[c] = u[c] * D;
                v[KW] = D * D;
                warp_sum_multi<WT, KW + 1>(v);
                WT *scr = sizeof(WT) == 8 ? (WT *)sh.red_d : (WT *)sh.red_f;
                if (lane == 0)
#pragma unroll
                    for (int q = 0; q <= KW; ++q) scr[w * (KW + 1) + q] = v[q];
                quad_bar();
                // every thread adds the warps' sums in the same order
#pragma unroll
                for (int q = 0; q <= KW; ++q) {
                    WT s = 0;
#pragma unroll
                    for (int p = 0; p < kQW; ++p) s += scr[p * (KW + 1) + q];
                    v[q] = s;
                }
                // 3-4. pivot, coefficient MGS on [c, e_l (l != t)], rotation;
                // reciprocals and reciprocal square roots instead of divisions
                // (this precision only shapes U', which the FP64 step makes
                // orthonormal)
                const WT d = sqrt(v[KW]);
                const WT id = (WT)1 / d;
                WT c[KW];
                WT r2 = 0;
#pragma unroll
                for (int q = 0; q < KW; ++q) {
                    c[q] = q < kk ? v[q] * id : (WT)0;
                    r2 += c[q] * c[q];
                }
                int t = 0;
                WT cmax = fabs(c[0]);
#pragma unroll
                for (int q = 1; q < KW; ++q)
                    if (q < kk && fabs(c[q]) > cmax) { cmax = fabs(c[q]); t = q; }
                WT Q[KW][KW];
                bool alive[KW];
#pragma unroll
                for (int m = 0; m < KW; ++m) {
                    WT x[KW];
                    const int lm = (m - 1) < t ? (m - 1) : m;  // list entry m >= 1 is column lm
#pragma unroll
                    for (int q = 0; q < KW; ++q) x[q] = m == 0 ? c[q] : (q == lm ? (WT)1 : (WT)0);
#pragma unroll
                    for (int p = 0; p < KW; ++p) {
                        if (p >= m || !alive[p]) continue;
                        WT h = 0;
#pragma unroll
                        for (int q = 0; q < KW; ++q) h += Q[p][q] * x[q];
#pragma unroll
                        for (int q = 0; q < KW; ++q) x[q] -= h * Q[p][q];
                    }
                    WT nn = 0;
#pragma unroll
                    for (int q = 0; q < KW; ++q) nn += x[q] * x[q];
                    alive[m] = m < kk && nn > (WT)0;
                    const WT inv = alive[m] ? rsq(nn) : (WT)0;
#pragma unroll
                    for (int q = 0; q < KW; ++q) Q[m][q] = x[q] * inv;
                }
                const WT al = (WT)a.alpha;
                WT av, as;
                if (a.mode == 1) {  // angle reading: (1-a) v/|v| + a e/|e|
                    const WT e2 = r2 < (WT)1 ? (WT)1 - r2 : (WT)0;
                    const WT inv_e = e2 > 0 ? rsq(e2) : (WT)0;
                    av = (r2 > 0 ? (1 - al) * rsq(r2) : (WT)0) - al * inv_e;
                    as = al * inv_e;
                } else {            // literal reading: (1-a) v + a (s - v)
                    av = 1 - 2 * al;
                    as = al;
                }
                const WT asd = as * id;  // applied to D = d s
                // new row before QR: column 0 = av U c + as s (its length is
                // taken out of the k x k Gram matrix below: the Q factor does
                // not depend on it), column m >= 1 = U q_m; q_1 in place of
                // column 0 when the direction vanishes (alpha = 1 with s in
                // the span), s itself when P P^T s = 0
                WT v0 = 0, q1 = 0;
#pragma unroll
                for (int cc = 0; cc < KW; ++cc) {
                    v0 += u[cc] * c[cc];
                    q1 += u[cc] * Q[0][cc];
                }
                double row[K];
                row[0] = (double)(av * v0 + asd * D);
#pragma unroll
                for (int m = 1; m < KW; ++m) {
                    WT s = 0;
#pragma unroll
                    for (int cc = 0; cc < KW; ++cc) s += u[cc] * Q[m][cc];
                    row[m] = (double)s;
                }
                const WT alt = alive[0] ? q1 : D * id;
                if (tid == 0) sh.degen = 0;
                // 5. FP64 Gram matrix G' of U' (upper triangle): this row's
                // products, one reduce-scatter per warp, the four warps'
                // partials added by warp 0, which then normalises column 0
                // (G = S G' S, S = diag(1/|u'_0|, 1, ...)) and forms
                // (I + R)^-1 with R the Cholesky factor of G minus I; the
                // scale 1/|u'_0| goes into row 0 of that inverse.  A
                // vanishing direction (G'_00 = 0) repeats this with column 0
                // replaced as above.
                constexpr int M = KW * (KW + 1) / 2;
#pragma unroll 1
                for (int pass = 0; pass < 2; ++pass) {
                    if constexpr (M <= 32) {
                        constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
                        constexpr int dup = 32 / S;
                        double g[S];
                        {
                            int e = 0;
#pragma unroll
                            for (int p = 0; p < KW; ++p)
#pragma unroll
                                for (int q = p; q < KW; ++q) g[e++] = row[p] * row[q];
#pragma unroll
                            for (int e2 = M; e2 < S; ++e2) g[e2] = 0.0;
                        }
                        const double tsum = warp_reduce_scatter<S>(g, lane);
                        if (lane % dup == 0) sh.gred[w][rs_index<S>(lane)] = tsum;
                        quad_bar();
                        if (w == 0 && lane < M) {
                            int p = 0, e = lane;
                            while (e >= KW - p) { e -= KW - p; ++p; }
                            // the four warps' sums as a tree: two dependent FP64 additions
                            static_assert(kQW == 4, "four update warps");
                            sh.G[p][p + e] = (sh.gred[0][lane] + sh.gred[1][lane]) + (sh.gred[2][lane] + sh.gred[3][lane]);
                        }
                    } else {
                        // k = 8: the 36 products of the row by warp sums
                        double g[M];
                        {
                            int e = 0;
#pragma unroll
                            for (int p = 0; p < KW; ++p)
#pragma unroll
                                for (int q = p; q < KW; ++q) g[e++] = row[p] * row[q];
                        }
                        warp_sum_multi<double, M>(g);
                        if (lane == 0)
#pragma unroll
                            for (int e = 0; e < M; ++e) sh.gq[w][e] = g[e];
                        quad_bar();
                        if (w == 0)
                            for (int e = lane; e < M; e += 32) {
                                int p = 0, e2 = e;
                                while (e2 >= KW - p) { e2 -= KW - p; ++p; }
                                sh.G[p][p + e2] = (sh.gq[0][e] + sh.gq[1][e]) + (sh.gq[2][e] + sh.gq[3][e]);
                            }
                    }
                    if (w == 0) {
                        __syncwarp();
                        const double g00 = sh.G[0][0];
                        if (g00 > 0.0) {
                            const double inv = rsqrt_scale(g00);
                            if (lane < KW) {
                                if (lane == 0) sh.G[0][0] = g00 * inv * inv;
                                else sh.G[0][lane] *= inv;
                            }
                            __syncwarp();
                            chol_inverse<TX, K>(sh, kk, lane);
                            if (lane < KW) sh.Ri[0][lane] *= inv;
                        } else if (lane == 0) {
                            sh.degen = 1;
                        }
                    }
                    quad_bar();
                    if (!sh.degen) break;  // uniform over the four warps
                    row[0] = (double)alt;
                }
                // 6. U'' = U' (I + R)^-1, written in every form the kernels read
                if (ok) write_row<TX, K>(a, sh, kk, l, row, Ufs, Uls);
            }
        } else {
            // warp 4 records the result meanwhile; warps 4-7 then fetch the
            // coordinates of the seed pairs (two per warp)
            if (w == kQW && lane == 0) record(b);
            if (go && sizeof(TX) == 4 && !a.seeds_in_product) {
                seed_bar();
                const int nw = sh.watch_n;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = (w - kQW) + h * (NW - kQW);
                    const int2 pr = sh.watch[q < nw ? q : 0];
                    const bool okq = q < nw && SAP_PAIR_OK(st, pr, a.N);
#pragma unroll
                    for (int r = 0; r < kQW; ++r) {
                        const int l = lane + 32 * r;
                        wxi[h][r] = (okq && l < n) ? (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) : 0.f;
                        wxj[h][r] = (okq && l < n) ? (float)ld_x<TX>(a.X, (size_t)pr.y * n + l) : 0.f;
                    }
                }
            }
        }
        // with the seeds in the next product, the bound it merges into starts at +inf
        if (go && a.seeds_in_product && tid == 0) st->seed_ub = 0x7f800000u;
        if (!go || a.seeds_in_product) return;
        __syncthreads();  // the new basis is written
        // seeds: the recent argmin pairs under the new basis, two per warp of
        // warps 4-7; FP32 data in extended precision from the basis's hi +
        // lo FP32 parts (a tight bound for every tier of the next
        // evaluation), FP64 data in FP64
        const int nwatch = sh.watch_n;
        if (w >= kQW) {
            const int q0 = w - kQW, q1 = q0 + (NW - kQW);
            if (sizeof(TX) == 4) {
                if (q0 < nwatch) {
                    bool valid[2] = {true, q1 < nwatch};
                    float rr;
                    int code;
                    df_eval_pref<KW, 2, kQW>(wxi, wxj, Ufs, Uls, n, valid, lane, rr, code);
                    const float sd = code == 1 ? cert_upper(rr, cert_explicit_df_dev(n, kk)) : INFINITY;
                    const float s0 = __shfl_sync(0xffffffffu, sd, 0), s1 = __shfl_sync(0xffffffffu, sd, 1);
                    if (lane == 0) {
                        sh.seed[q0] = s0;
                        if (q1 < nwatch) sh.seed[q1] = s1;
                    }
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = h == 0 ? q0 : q1;
                    if (q >= nwatch || !SAP_PAIR_OK(st, sh.watch[q], a.N)) continue;  // uniform over the warp
                    const int2 pr = sh.watch[q];
                    double v[K + 1];
#pragma unroll
                    for (int e = 0; e <= K; ++e) v[e] = 0.0;
                    for (int l = lane; l < n; l += 32) {
                        const double D = (double)ld_x<TX>(a.X, (size_t)pr.x * n + l) -
                                         (double)ld_x<TX>(a.X, (size_t)pr.y * n + l);
                        v[K] = fma(D, D, v[K]);
#pragma unroll
                        for (int c = 0; c < K; ++c)
                            if (c < kk) v[c] = fma(a.U64[(size_t)c * n + l], D, v[c]);
                    }
                    warp_sum_multi<double, K + 1>(v);
                    double zz = 0.0;
#pragma unroll
                    for (int c = 0; c < K; ++c) zz = fma(v[c], v[c], zz);
                    if (lane == 0) sh.seed[q] = v[K] > 0.0 ? __double2float_ru(sqrt(zz / v[K])) * 1.000001f : INFINITY;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            float m = INFINITY;
            for (int q = 0; q < nwatch; ++q) m = fminf(m, sh.seed[q]);
            st->seed_ub = __float_as_uint(m);
        }
        return;
    }

    // ---- the whole block records the result and updates (larger bases)
    if (tid == 0) {
        record(sh.wb[0]);
        const Partial b0 = sh.wb[0];
        sh.wb[0].r = !(b0.r < INFINITY) ? b0.r : sqrt(b0.r);
    }
    __syncthreads();
    const Partial b = sh.wb[0];
    if (!(b.r < INFINITY) || a.eval_only) return;

    // the watch pairs' coordinates, loaded now and used at the very end
    const int nwatch = sh.watch_n;
    const bool prefetch = n <= 32 * kSeedRegs;
    float wxi[kSeedRegs], wxj[kSeedRegs];
    if (prefetch && w < nwatch && !a.seeds_in_product && SAP_PAIR_OK(st, sh.watch[w], a.N)) {
        const int2 pr = sh.watch[w];
#pragma unroll
        for (int q = 0; q < kSeedRegs; ++q) {
            const int l = lane + 32 * q;
            wxi[q] = l < n ? (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) : 0.f;
            wxj[q] = l < n ? (float)ld_x<TX>(a.X, (size_t)pr.y * n + l) : 0.f;
        }
    }

    float *Uf = nullptr;  // FP32 copy of the final basis (n x K) for the seeds
    {
        const bool in_smem = K <= 8 && su_dyn_bytes<TX>(n, K) <= kDynSmem;
        double *Up = in_smem ? dyn : a.work;           // n x K: the new basis before QR
        WT *Ds = reinterpret_cast<WT *>(Up + (size_t)n * K);  // n
        if (in_smem) Uf = reinterpret_cast<float *>(dyn + (size_t)n * K + ((size_t)n * sizeof(WT) + 7) / 8);

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
        if (w == 0) chol_inverse<TX, K>(sh, kk, lane);
        __syncthreads();

        // 6. U'' = U' (I + R)^-1, written in every form the kernels read
#pragma unroll 1
        for (int l = tid; l < n; l += SB) {
            double row[K];
#pragma unroll
            for (int m = 0; m < K; ++m) row[m] = m < kk ? Up[(size_t)l * K + m] : 0.0;
            write_row<TX, K>(a, sh, kk, l, row, Uf);
        }
        __syncthreads();
    }

    if (a.seeds_in_product) {
        if (tid == 0) st->seed_ub = 0x7f800000u;  // the next product merges its seeds into +inf
        return;
    }

    // seeds: the recent argmin pairs under the new basis
    if (w < nwatch && SAP_PAIR_OK(st, sh.watch[w], a.N)) {
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
                        const float *ur_ = Uf ? Uf + (size_t)l * K : a.U32 + (size_t)l * a.KP;
#pragma unroll
                        for (int c = 0; c < K; ++c)
                            if (c < kk) v[c] = fmaf(ur_[c], D, v[c]);
                    }
                }
            } else {
                for (int l = lane; l < n; l += 32) {
                    const float D = (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) - (float)ld_x<TX>(a.X, (size_t)pr.y * n + l);
                    v[K] = fmaf(D, D, v[K]);
                    const float *ur_ = Uf ? Uf + (size_t)l * K : a.U32 + (size_t)l * a.KP;
#pragma unroll
                    for (int c = 0; c < K; ++c)
                        if (c < kk) v[c] = fmaf(ur_[c], D, v[c]);
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
    size_t shm = 0;
    if (K <= 8 && a.n <= 32 * kQW) {
        // the small-basis update keeps its rows in registers; the new basis's
        // FP32 hi and lo parts go to shared memory for the seeds
        shm = sizeof(TX) == 4 ? (size_t)a.n * K * 8 : 0;
    } else {
        const size_t need = su_dyn_bytes<TX>(a.n, K);
        shm = (K <= 8 && need <= kDynSmem) ? need : 0;
    }
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
