// select_update.cu -- the FP64 argmin over the certified candidate list and
// the basis update of one SAP iteration (Algorithm 1 and Sec. IV of Kvinge
// et al., arXiv:1807.03425), fused into one launch.
//
// Phase 1 (all blocks): one warp per candidate forms the explicit FP64
// difference D = x_i - x_j, d^2 = |D|^2 and z = U^T D, r = sqrt(|z|^2/d^2),
// applies the exclusion rules exactly (d^2 == 0: not distinct, Sec. II;
// d^2 < eps^2: shorter than the threshold, Sec. VII) and keeps the best
// (r, i, j), ties to the smallest pair index.  Each block publishes its best;
// the last block to finish (ticket counter) continues with phase 2.
//
// Phase 2 (last block):
//   1. argmin over the block results; record it in the history;
//   2. s = D/|D|, c = U^T s (one multi-value block reduction);
//   3. pivot t = argmax_l |c_l| (first on ties; the first column if all are
//      zero), then modified Gram-Schmidt on [c, e_l (l != t)] in the
//      k-dimensional coefficient space: since U has orthonormal columns,
//      MGS of [U c, u_l (l != t)] in R^n is U times MGS of [c, e_l] in R^k;
//   4. new first column along (1-a) v + a (s - v) (literal reading) or
//      (1-a) v/|v| + a e/|e| (angle reading), v = U c, e = s - v;
//   5. re-orthonormalisation in FP64: Cholesky QR of the new basis
//      (G = U'^T U', G = R^T R, U'' = U' R^-1), the QR factor that one MGS
//      re-pass produces in exact arithmetic;
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
constexpr size_t kDynSmem = 24 * 1024;  // vectors kept in shared memory up to this size

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

template <typename WT, int K>
struct Shared {
    double red_d[NW * (K + 1)];
    float red_f[NW * (K + 1)];
    Partial wb[NW];
    int last;
    int alive0;
    double cvec[K + 1];            // U^T D and |D|^2 (data precision, widened)
    WT cw[K];                      // c = U^T s
    WT Bw[K][K];                   // coefficient MGS result, column m = q_m
    WT av, asd, dnorm, nd2;        // direction coefficients, |D|, |dir|^2
    double G[K][K];                // Gram matrix, then R (upper)
    double Rd[K];                  // 1 / R_jj
    double Ri[K][K];               // R^-1 (upper)
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

    // ---------------- phase 1: FP64 recheck of the candidate list ----------
    {
        unsigned int cnt = a.which == 1 ? (unsigned int)st->cnt1 : (unsigned int)st->cnt2;
        if (cnt > a.cap) cnt = a.cap;
        Partial best = {INFINITY, 0x7fffffff, 0x7fffffff};
        for (unsigned int e = blockIdx.x * NW + w; e < cnt; e += gridDim.x * NW) {
            const int2 ij = a.list[e];
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
            warp_sum_multi<double, K + 1>(v);
            const double d2 = v[K];
            if (d2 == 0.0 || d2 < a.eps2) continue;
            double zz = 0.0;
#pragma unroll
            for (int c = 0; c < K; ++c) zz = fma(v[c], v[c], zz);
            const double r = sqrt(zz / d2);
            if (better(r, ij.x, ij.y, best.r, best.i, best.j)) best = Partial{r, ij.x, ij.y};
        }
        if (lane == 0) sh.wb[w] = best;
        __syncthreads();
        if (tid == 0) {
            Partial b = sh.wb[0];
            for (int q = 1; q < NW; ++q)
                if (better(sh.wb[q].r, sh.wb[q].i, sh.wb[q].j, b.r, b.i, b.j)) b = sh.wb[q];
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
    if (w == 0) {
        Partial b = {INFINITY, 0x7fffffff, 0x7fffffff};
        for (int p = lane; p < (int)gridDim.x; p += 32) {
            const volatile Partial *vp = &a.partials[p];
            const Partial q = {vp->r, vp->i, vp->j};
            if (better(q.r, q.i, q.j, b.r, b.i, b.j)) b = q;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Partial q;
            q.r = __shfl_xor_sync(0xffffffffu, b.r, o);
            q.i = __shfl_xor_sync(0xffffffffu, b.i, o);
            q.j = __shfl_xor_sync(0xffffffffu, b.j, o);
            if (better(q.r, q.i, q.j, b.r, b.i, b.j)) b = q;
        }
        if (lane == 0) {
            sh.wb[0] = b;
            const int it = st->iter;
            const bool none = !(b.r < INFINITY);
            if (none) atomicOr(&st->status, ST_NO_SECANT);
            if (it < st->hist_cap) {
                a.hist[it] = none ? __longlong_as_double(0x7ff8000000000000ll) : b.r;
                a.argmin[it] = none ? make_int2(-1, -1) : make_int2(b.i, b.j);
            }
            st->iter = it + 1;
            st->last_r = b.r;
            st->last_i = none ? -1 : b.i;
            st->last_j = none ? -1 : b.j;
            st->last_cnt1 = st->cnt1;
            st->last_cnt2 = st->cnt2;
            st->cnt1 = 0;
            st->cnt2 = 0;
            st->ticket = 0;
            st->run_ub1 = 0x7f800000u;
            st->run_ub2 = 0x7f800000u;
            if (!none) {
                bool present = false;
                for (int q = 0; q < st->watch_n; ++q)
                    present |= (st->watch[q].x == b.i && st->watch[q].y == b.j);
                if (!present) {
                    st->watch[st->watch_pos] = make_int2(b.i, b.j);
                    st->watch_pos = (st->watch_pos + 1) % kWatch;
                    if (st->watch_n < kWatch) ++st->watch_n;
                }
                if (a.eval_only)  // the basis stays: the exact minimum bounds the next one
                    st->seed_ub = __float_as_uint(__double2float_ru(b.r) * 1.000001f);
            }
        }
    }
    __syncthreads();
    const Partial b = sh.wb[0];
    if (!(b.r < INFINITY) || a.eval_only) return;

    const bool in_smem = (size_t)n * (K + 1) * sizeof(WT) <= kDynSmem;
    WT *Up = in_smem ? reinterpret_cast<WT *>(dyn) : reinterpret_cast<WT *>(a.work);  // n x K
    WT *Ds = Up + (size_t)n * K;                                                       // n

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
                if (c < kk) v[c] += (sizeof(WT) == 8 ? (WT)a.U64[(size_t)c * n + l] : (WT)a.U32[(size_t)l * a.KP + c]) * D;
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
    //      coefficients, in one thread (k x k work)
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
        for (int q = 1; q < kk; ++q)
            if (fabs(c[q]) > cmax) { cmax = fabs(c[q]); t = q; }
        WT Q[K][K];
        int alive[K];
#pragma unroll 1
        for (int m = 0; m < kk; ++m) {
            WT x[K];
            const int l = (m - 1) < t ? (m - 1) : m;  // list entry m >= 1 is column l
#pragma unroll
            for (int q = 0; q < K; ++q) x[q] = m == 0 ? c[q] : (q == l ? (WT)1 : (WT)0);
#pragma unroll 1
            for (int p = 0; p < m; ++p) {
                if (!alive[p]) continue;
                WT h = 0;
#pragma unroll
                for (int q = 0; q < K; ++q) h += Q[p][q] * x[q];
#pragma unroll
                for (int q = 0; q < K; ++q) x[q] -= h * Q[p][q];
            }
            WT nn = 0;
#pragma unroll
            for (int q = 0; q < K; ++q) nn += x[q] * x[q];
            alive[m] = nn > (WT)0;
            const WT inv = alive[m] ? (WT)1 / sqrt(nn) : (WT)0;
#pragma unroll
            for (int q = 0; q < K; ++q) Q[m][q] = x[q] * inv;
        }
        for (int m = 0; m < kk; ++m)
            for (int q = 0; q < K; ++q) sh.Bw[q][m] = Q[m][q];
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
                u[c] = c < kk ? (sizeof(WT) == 8 ? (WT)a.U64[(size_t)c * n + l] : (WT)a.U32[(size_t)l * a.KP + c]) : (WT)0;
            WT v0 = 0;
#pragma unroll
            for (int c = 0; c < K; ++c) v0 += u[c] * sh.cw[c];
            const WT d0 = av * v0 + asd * Ds[l];
            Up[(size_t)l * K] = d0;
            p0 += d0 * d0;
#pragma unroll
            for (int m = 1; m < K; ++m) {
                WT s = 0;
#pragma unroll
                for (int c = 0; c < K; ++c) s += u[c] * sh.Bw[c][m];
                Up[(size_t)l * K + m] = s;
            }
        }
        WT pv[1] = {p0};
        WT *scr = sizeof(WT) == 8 ? (WT *)sh.red_d : (WT *)sh.red_f;
        block_sum_multi<WT, 1>(pv, scr, &sh.nd2);
        const WT nd = sqrt(sh.nd2);
        const bool keep_q1 = sh.alive0 != 0;
#pragma unroll 1
        for (int l = tid; l < n; l += SB) {
            if (nd > 0) {
                Up[(size_t)l * K] /= nd;
            } else if (keep_q1) {  // alpha = 1 with s in the span: keep q1
                WT s = 0;
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (c < kk)
                        s += (sizeof(WT) == 8 ? (WT)a.U64[(size_t)c * n + l] : (WT)a.U32[(size_t)l * a.KP + c]) *
                             sh.Bw[c][0];
                Up[(size_t)l * K] = s;
            } else {               // P P^T s = 0: the new column is s
                Up[(size_t)l * K] = Ds[l] / sh.dnorm;
            }
        }
        __syncthreads();
    }

    // 5. FP64 Cholesky QR of Up: Gram entries spread over the warps
#pragma unroll 1
    for (int e = w; e < kk * kk; e += NW) {
        const int p = e / kk, q = e % kk;
        if (q < p) continue;
        double s = 0.0;
        for (int l = lane; l < n; l += 32) s = fma((double)Up[(size_t)l * K + p], (double)Up[(size_t)l * K + q], s);
        s = warp_sum(s);
        if (lane == 0) sh.G[p][q] = s;
    }
    __syncthreads();
    if (w == 0) {
        // right-looking Cholesky G = R^T R on the upper triangle, lane m owns
        // column m; 1/R_jj from one reciprocal square root per step
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
        // R^-1 (upper): lane m solves R x = e_m by back substitution
        if (lane < kk) {
            double x[K];
#pragma unroll
            for (int q = 0; q < K; ++q) x[q] = 0.0;
#pragma unroll 1
            for (int i = lane; i >= 0; --i) {
                double s = (i == lane) ? 1.0 : 0.0;
                for (int p = i + 1; p <= lane; ++p) s = fma(-sh.G[i][p], x[p], s);
                x[i] = s * sh.Rd[i];
            }
            for (int i = 0; i <= lane; ++i) sh.Ri[i][lane] = x[i];
        }
    }
    __syncthreads();

    // 6. U'' = Up R^-1, written in every form the kernels read
#pragma unroll 1
    for (int l = tid; l < n; l += SB) {
        double row[K];
#pragma unroll
        for (int m = 0; m < K; ++m) row[m] = m < kk ? (double)Up[(size_t)l * K + m] : 0.0;
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
    const int nwatch = st->watch_n;
    if (w < nwatch) {
        const int2 pr = st->watch[w];
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
            for (int l = lane; l < n; l += 32) {
                const float D = (float)ld_x<TX>(a.X, (size_t)pr.x * n + l) - (float)ld_x<TX>(a.X, (size_t)pr.y * n + l);
                v[K] = fmaf(D, D, v[K]);
                const float *ur = a.U32 + (size_t)l * a.KP;
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (c < kk) v[c] = fmaf(ur[c], D, v[c]);
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
    const size_t need = (size_t)a.n * (K + 1) * sizeof(double);
    const size_t shm = need <= kDynSmem ? need : 0;
    select_update_kernel<TX, K><<<a.grid, SB, shm, s>>>(a);
    return cudaGetLastError();
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
