// softmin.cu -- the soft-min objective, its gradient, and Riemannian ascent.
//
// Objective (a smooth surrogate of the SAP minimum min r_ij; the paper has no
// counterpart):
//     L(U) = -tau log sum_{i<j kept} exp(-r_ij / tau),   r_ij = ||U^T (x_i - x_j)|| / d_ij,
// evaluated as L = M - tau log sum exp((M - r_ij)/tau) for a shift M near the
// minimum.  With p_ij = exp((L - r_ij)/tau) (the weights sum to 1) and
//     dr_ij/dU = (x_i - x_j)(y_i - y_j)^T / (d_ij^2 r_ij),   y = U^T x,
// the gradient is dL/dU = sum_ij c_ij (x_i - x_j)(y_i - y_j)^T with
// c_ij = p_ij w_ij / r_ij, w_ij = 1/d_ij^2.  Written per point,
//     dL/dU = sum_i (x_i - xbar) z_i^T,   z_i = sum_{j != i} c_ij (y_i - y_j),
// X^T times a weighted graph Laplacian times Y (sum_i z_i = 0, so xbar is
// free; the column mean keeps the factors small).  The backward pass
// recomputes every pair from the stored lengths rather than keeping the
// N^2/2 weights of the forward pass.
//
// Precision.  Y is held as an unevaluated sum hi + lo of two FP32 numbers per
// entry, formed from the exact FP32 data and the FP64 basis with error-free
// products and sums, so y_i - y_j is accurate to a few units in the last
// place of its own size, whatever d_ij: each r_ij is then as accurate as its
// FP32 length.  (A single FP32 Y, or the split 16-bit product of the SAP
// pass, loses y_i - y_j to cancellation for short secants, and dp/p = dr/tau
// is large at small tau.)  The Laplacian form multiplies partial sums of
// c_ij (y_i - y_j), of size p_ij/d_ij, by points of size ||x - xbar||, so its
// rounding error grows like ||x - xbar||/d_ij.  The near pairs of the
// restructured form (the short secants the SAP pass skips) therefore
// contribute c_ij (x_i - x_j)(y_i - y_j)^T from explicit differences.
// Pairs with r_ij^2 below the smallest normal FP32 number (r < 1.1e-19) count
// in L but not in the gradient (dr/dU is undefined at r = 0).
#include "softmin.cuh"
#include "restructured.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace sap {
namespace {

constexpr int T = kTile;                 // 128
constexpr unsigned FULL = 0xffffffffu;
constexpr int kSoftStagesMax = 3;
constexpr int kFwdWarps = 16;            // consumer warps of the forward pass
constexpr int kBwdWarps = 8;             // consumer warps of the backward pass
constexpr int kNearWarps = 8;            // warps per block of the near-pair kernels
constexpr int kNearChunk = 16;           // near pairs per warp
constexpr int kSoftMaxN = 512;           // ambient dimension limit of this objective
constexpr float kFltMin = 1.17549435e-38f;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void named_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- double-float (hi + lo) arithmetic; the _rn intrinsics are never fused
// into FMAs, which would break the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_add(float &hi, float &lo, float v)
{
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}
// (hi, lo) += x * (yh + yl): exact product x*yh (FMA residual) plus x*yl.
__device__ __forceinline__ void df_fma(float &hi, float &lo, float x, float yh, float yl)
{
    const float p = __fmul_rn(x, yh);
    const float pe = fmaf(x, yh, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, fmaf(x, yl, pe)));
}
__device__ __forceinline__ void df_merge(float &hi, float &lo, float h2, float l2)
{
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, e));
}
// Renormalise so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ void df_norm(float &hi, float &lo)
{
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}

// Merge two shifted sums (M1, S1), (M2, S2): S = sum exp((M - r)/tau).
__device__ __forceinline__ void lse_merge(float &M, double &S, float M2, double S2, float K2)
{
    const float Mn = fminf(M, M2);
    const double f1 = (double)ex2_approx(fmaxf((Mn - M) * K2, -200.f));
    const double f2 = (double)ex2_approx(fmaxf((Mn - M2) * K2, -200.f));
    S = S * f1 + S2 * f2;
    M = Mn;
}

__device__ __forceinline__ int tile_index(int I, int J, int nb)
{
    return I * nb - I * (I - 1) / 2 + (J - I);
}

// ---------------------------------------------------------------- Y = X U ---

// Y = X U as hi + lo pairs, component-major (Yh[c * Npad + i]); rows >= N are
// zero.  Eight lanes per row, four rows per warp.  U is split once per block
// into FP32 hi + lo parts in shared memory.
template <int K>
__global__ void __launch_bounds__(256) ydf_kernel(const float *X, int N, int n, const double *U64, int Npad,
                                                  float *Yh, float *Yl)
{
    extern __shared__ float su[];  // su[l * 2K + c] = hi, su[l * 2K + K + c] = lo
    for (int idx = threadIdx.x; idx < n * K; idx += blockDim.x) {
        const int l = idx / K, c = idx % K;
        const double u = U64[(size_t)c * n + l];
        const float uh = (float)u;
        su[l * 2 * K + c] = uh;
        su[l * 2 * K + K + c] = (float)(u - (double)uh);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane >> 3, sl = lane & 7;
    for (int base = (blockIdx.x * 8 + warp) * 4; base < Npad; base += gridDim.x * 32) {
        const int row = base + sub;
        float hi[K], lo[K];
#pragma unroll
        for (int c = 0; c < K; ++c) hi[c] = lo[c] = 0.f;
        if (row < N)
#pragma unroll 4
            for (int l = sl; l < n; l += 8) {
                const float x = X[(size_t)row * n + l];
#pragma unroll
                for (int c = 0; c < K; ++c) df_fma(hi[c], lo[c], x, su[l * 2 * K + c], su[l * 2 * K + K + c]);
            }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float h2 = __shfl_xor_sync(FULL, hi[c], o), l2 = __shfl_xor_sync(FULL, lo[c], o);
                df_merge(hi[c], lo[c], h2, l2);
            }
        if (sl == 0)
#pragma unroll
            for (int c = 0; c < K; ++c) {
                float h = hi[c], l = lo[c];
                df_norm(h, l);
                Yh[(size_t)c * Npad + row] = h;
                Yl[(size_t)c * Npad + row] = l;
            }
    }
}

// ------------------------------------------------------- all-pairs passes ---

struct SoftPassArgs {
    const float *w;
    const int2 *wtiles;
    int ntiles;
    const float *Yh, *Yl;  // K x Npad
    int Npad;
    int stages;
    float K2;              // log2(e) / tau
    double tau;
    SoftDev *dev;
    SoftPart *part;        // forward: this pass's blocks, then the near blocks
    int nparts;            // partials merged by the forward's last block
    double *hist;          // forward: L is also stored at hist[dev->step] (or null)
    float *P;              // backward: tile partials, ntiles x 2 x K x 128
};

__host__ __device__ inline uint32_t soft_stage_bytes(int K) { return (uint32_t)T * T * 4 + 4u * K * T * 4; }

// Persistent, warp-specialised pass over the stored lengths (layout of
// restructured.cu): a producer warp fills a ring of shared-memory stages by
// 1-D bulk copies (the 64 KB w tile and, per component, the hi and lo parts
// of both point blocks' Y); NW consumer warps evaluate the tiles.  Consumer
// thread: four adjacent columns j of the rows warp, warp + NW, ...; the
// squared projected lengths are formed with packed FP32 pairs from the
// hi + lo differences.
//
// Forward: each thread keeps a shift M (its first ratio, lowered only when a
// ratio falls 60/K2 below it, so terms stay below 2^60) and the sum of
// exp((M - r)/tau) (per tile in FP32, across tiles in FP64); threads, warps,
// blocks and finally the last block to finish merge (M, S) pairs in a fixed
// order, so L is reproducible bit for bit.
//
// Backward: c_ij = p_ij w_ij / r_ij and t_ij = c_ij (y_i - y_j).  A thread
// accumulates t over its rows for its four columns (registers) and over its
// four columns for each row; row sums of a warp are finished by a shuffle
// reduce-scatter (16 slots: G = 16/K rows x K components), column sums across
// warps in shared memory.  Each tile writes its row sums (z contributions
// of block I) and negated column sums (of block J) to P; no atomics, so the
// gradient is reproducible too.
template <int K, int NW, bool BWD>
__global__ void __launch_bounds__((NW + 1) * 32, 1) soft_pass_kernel(SoftPassArgs a)
{
    constexpr int RPW = T / NW;
    constexpr int G = 16 / K;                   // rows per reduce-scatter group
    constexpr int NG = (RPW + G - 1) / G;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[kSoftStagesMax], empty[kSoftStagesMax];
    __shared__ int sT[kSoftStagesMax];
    __shared__ float redM[NW];
    __shared__ double redS[NW];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = a.stages;
    const uint32_t wbytes = T * T * 4, seg = T * 4, sbytes = soft_stage_bytes(K);
    const int nmine = blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long budget = 4000000000ll;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], NW);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();

    if (warp == NW) {
        if (lane == 0) {
            int issued = 0;
            for (int it = 0; it < nmine; ++it) {
                const int s = it % S;
                if (it >= S && !tc::mbar_wait_bounded(&empty[s], ((it / S) - 1) & 1, budget)) {
                    atomicOr(&a.dev->status, ST_TIMEOUT);
                    break;
                }
                const int t = blockIdx.x + it * gridDim.x;
                const int2 IJ = a.wtiles[t];
                sT[s] = t;  // published by the mbarrier completion below
                unsigned char *base = sm + (size_t)s * sbytes;
                tc::mbar_expect_tx(&full[s], sbytes);
                tc::bulk_g2s(base, a.w + (size_t)t * T * T, wbytes, &full[s]);
                const size_t oI = (size_t)IJ.x * T, oJ = (size_t)IJ.y * T;
                for (int c = 0; c < K; ++c) {
                    const size_t oc = (size_t)c * a.Npad;
                    tc::bulk_g2s(base + wbytes + (0 * K + c) * seg, a.Yh + oc + oI, seg, &full[s]);
                    tc::bulk_g2s(base + wbytes + (1 * K + c) * seg, a.Yl + oc + oI, seg, &full[s]);
                    tc::bulk_g2s(base + wbytes + (2 * K + c) * seg, a.Yh + oc + oJ, seg, &full[s]);
                    tc::bulk_g2s(base + wbytes + (3 * K + c) * seg, a.Yl + oc + oJ, seg, &full[s]);
                }
                ++issued;
            }
            for (int it = issued > S ? issued - S : 0; it < issued; ++it)
                tc::mbar_wait_bounded(&full[it % S], (it / S) & 1, budget);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const int col0 = lane * 4;
    const float K2 = a.K2;
    float M = INFINITY, MK2 = INFINITY;  // forward shift and M * K2
    double S64 = 0.0;
    const float LK2 = BWD ? (float)(a.dev->L * (double)K2) : 0.f;
    float *rowbuf = reinterpret_cast<float *>(sm + (size_t)S * sbytes);  // K x T (backward)
    float *colbuf = rowbuf + K * T;                                       // NW x K x T
    bool ok = true;

    for (int it = 0; it < nmine; ++it) {
        const int s = it % S;
        // After a timed-out wait the warp stops waiting but (backward) still
        // walks its tiles, so every consumer warp reaches the named barriers;
        // the status word tells the host to discard the result.
        if (ok && !tc::mbar_wait_bounded(&full[s], (it / S) & 1, budget)) {
            if (lane == 0) atomicOr(&a.dev->status, ST_TIMEOUT);
            ok = false;
        }
        ok = __all_sync(FULL, ok);
        if (!BWD && !ok) break;
        const int t = sT[s];
        (void)t;
        const float *ws = reinterpret_cast<const float *>(sm + (size_t)s * sbytes);
        const float *yIh = ws + T * T, *yIl = yIh + K * T, *yJh = yIl + K * T, *yJl = yJh + K * T;

        uint64_t jh[2][K], jl[2][K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float4 h4 = *reinterpret_cast<const float4 *>(yJh + c * T + col0);
            const float4 l4 = *reinterpret_cast<const float4 *>(yJl + c * T + col0);
            jh[0][c] = tc::pk2(h4.x, h4.y);
            jh[1][c] = tc::pk2(h4.z, h4.w);
            jl[0][c] = tc::pk2(l4.x, l4.y);
            jl[1][c] = tc::pk2(l4.z, l4.w);
        }

        if (!BWD) {
            float St = 0.f;
#pragma unroll 4
            for (int r = 0; r < RPW; ++r) {
                const int row = warp + NW * r;
                uint64_t s2[2] = {0ull, 0ull};
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float yh = yIh[c * T + row], yl = yIl[c * T + row];
                    const uint64_t hh = tc::pk2(yh, yh), ll = tc::pk2(yl, yl);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const uint64_t e = tc::add2(tc::sub2(hh, jh[p][c]), tc::sub2(ll, jl[p][c]));
                        s2[p] = tc::fma2(e, e, s2[p]);
                    }
                }
                const float4 w4 = *reinterpret_cast<const float4 *>(ws + row * T + col0);
                const float2 qa = tc::upk2(tc::mul2(s2[0], tc::pk2(w4.x, w4.y)));
                const float2 qb = tc::upk2(tc::mul2(s2[1], tc::pk2(w4.z, w4.w)));
                const float rr[4] = {sqrt_approx(qa.x), sqrt_approx(qa.y), sqrt_approx(qb.x), sqrt_approx(qb.y)};
                float ag[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) ag[m] = fmaf(rr[m], -K2, MK2);
                const float amax = fmaxf(fmaxf(ag[0], ag[1]), fmaxf(ag[2], ag[3]));
                if (amax > 60.f) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float am = fmaf(rr[m], -K2, MK2);
                        if (am > 0.f) {
                            S64 = (S64 + (double)St) * (double)ex2_approx(-am) + 1.0;
                            St = 0.f;
                            M = rr[m];
                            MK2 = M * K2;
                        } else {
                            St += ex2_approx(fmaxf(am, -200.f));
                        }
                    }
                } else {
                    St += (ex2_approx(fmaxf(ag[0], -200.f)) + ex2_approx(fmaxf(ag[1], -200.f))) +
                          (ex2_approx(fmaxf(ag[2], -200.f)) + ex2_approx(fmaxf(ag[3], -200.f)));
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
            S64 += (double)St;
        } else {
            uint64_t zc[2][K];
#pragma unroll
            for (int c = 0; c < K; ++c) zc[0][c] = zc[1][c] = 0ull;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                uint64_t zr[G][K];
#pragma unroll
                for (int q = 0; q < G; ++q)
#pragma unroll
                    for (int c = 0; c < K; ++c) zr[q][c] = 0ull;
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (g * G + q >= RPW) break;
                    const int row = warp + NW * (g * G + q);
                    uint64_t e[2][K];
                    uint64_t s2[2] = {0ull, 0ull};
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float yh = yIh[c * T + row], yl = yIl[c * T + row];
                        const uint64_t hh = tc::pk2(yh, yh), ll = tc::pk2(yl, yl);
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            e[p][c] = tc::add2(tc::sub2(hh, jh[p][c]), tc::sub2(ll, jl[p][c]));
                            s2[p] = tc::fma2(e[p][c], e[p][c], s2[p]);
                        }
                    }
                    const float4 w4 = *reinterpret_cast<const float4 *>(ws + row * T + col0);
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
                    const float2 qa = tc::upk2(tc::mul2(s2[0], tc::pk2(w4.x, w4.y)));
                    const float2 qb = tc::upk2(tc::mul2(s2[1], tc::pk2(w4.z, w4.w)));
                    const float q4[4] = {qa.x, qa.y, qb.x, qb.y};
                    float cc[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float rs = rsqrt_approx(q4[m]);
                        const float rv = q4[m] * rs;
                        const float pw = ex2_approx(fmaxf(fmaf(rv, -K2, LK2), -200.f));
                        cc[m] = q4[m] >= kFltMin ? pw * (wv[m] * rs) : 0.f;  // NaN (skipped) fails too
                    }
                    const uint64_t c2[2] = {tc::pk2(cc[0], cc[1]), tc::pk2(cc[2], cc[3])};
#pragma unroll
                    for (int c = 0; c < K; ++c)
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            zc[p][c] = tc::fma2(c2[p], e[p][c], zc[p][c]);
                            zr[q][c] = tc::fma2(c2[p], e[p][c], zr[q][c]);
                        }
                }
                // reduce-scatter the group's row sums over the 32 lanes
                float v[16];
#pragma unroll
                for (int sl = 0; sl < 16; ++sl) v[sl] = 0.f;
#pragma unroll
                for (int q = 0; q < G; ++q)
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float2 t2 = tc::upk2(zr[q][c]);
                        v[q * K + c] = t2.x + t2.y;
                    }
#pragma unroll
                for (int lev = 0; lev < 4; ++lev) {
                    const int half = 8 >> lev, o = 16 >> lev;
                    const bool upper = (lane & o) != 0;
#pragma unroll
                    for (int sl = 0; sl < half; ++sl) {
                        const float send = upper ? v[sl] : v[sl + half];
                        const float keep = upper ? v[sl + half] : v[sl];
                        v[sl] = keep + __shfl_xor_sync(FULL, send, o);
                    }
                }
                v[0] += __shfl_xor_sync(FULL, v[0], 1);
                const int slot = lane >> 1;
                if (!(lane & 1) && slot < G * K) {
                    const int q = slot / K, c = slot % K;
                    if (g * G + q < RPW) rowbuf[c * T + warp + NW * (g * G + q)] = v[0];
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float2 u0 = tc::upk2(zc[0][c]), u1 = tc::upk2(zc[1][c]);
                *reinterpret_cast<float4 *>(colbuf + (warp * K + c) * T + col0) = make_float4(u0.x, u0.y, u1.x, u1.y);
            }
            named_bar(1, NW * 32);
            float *Pt = a.P + (size_t)t * 2 * K * T;
            for (int e = tid; e < 2 * K * T; e += NW * 32) {
                if (e < K * T) {
                    Pt[e] = rowbuf[e];
                } else {
                    const int f = e - K * T;
                    float acc = 0.f;
#pragma unroll
                    for (int wv = 0; wv < NW; ++wv) acc += colbuf[wv * K * T + f];
                    Pt[e] = -acc;
                }
            }
            named_bar(1, NW * 32);
        }
    }

    if constexpr (!BWD) {
        // ---- forward: merge (M, S) over the block, then over all blocks
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float M2 = __shfl_xor_sync(FULL, M, o);
            const double S2 = __shfl_xor_sync(FULL, S64, o);
            lse_merge(M, S64, M2, S2, K2);
        }
        if (lane == 0) {
            redM[warp] = M;
            redS[warp] = S64;
        }
        named_bar(1, NW * 32);
        if (warp != 0) return;
        M = lane < NW ? redM[lane] : INFINITY;
        S64 = lane < NW ? redS[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float M2 = __shfl_xor_sync(FULL, M, o);
            const double S2 = __shfl_xor_sync(FULL, S64, o);
            lse_merge(M, S64, M2, S2, K2);
        }
        unsigned int ticket = 0;
        if (lane == 0) {
            SoftPart pt;
            pt.S = S64;
            pt.M = M;
            pt.pad = 0;
            a.part[blockIdx.x] = pt;
            __threadfence();
            ticket = atomicAdd(&a.dev->ticket, 1u);
        }
        ticket = __shfl_sync(FULL, ticket, 0);
        if (ticket != gridDim.x - 1) return;
        __threadfence();
        M = INFINITY;
        S64 = 0.0;
        for (int q = lane; q < a.nparts; q += 32) {
            const double Sq = __ldcg(&a.part[q].S);
            const float Mq = __ldcg(&a.part[q].M);
            lse_merge(M, S64, Mq, Sq, K2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float M2 = __shfl_xor_sync(FULL, M, o);
            const double S2 = __shfl_xor_sync(FULL, S64, o);
            lse_merge(M, S64, M2, S2, K2);
        }
        if (lane == 0) {
            if (S64 > 0.0 && M < INFINITY) {
                const double L = (double)M - a.tau * log(S64);
                a.dev->L = L;
                if (a.hist && a.dev->step < a.dev->hist_cap) a.hist[a.dev->step] = L;
            } else {
                atomicOr(&a.dev->status, ST_NO_SECANT);
            }
            a.dev->ticket = 0;
        }
    }
}

// ------------------------------------------------------------ near pairs ---

struct SoftNearArgs {
    const float *X;
    int N, n;
    const float *Yh, *Yl;
    int Npad;
    const double *U64;     // d^2 below the FP32 range: FP64 from the data
    const int2 *near;
    int n_near;
    float K2;
    SoftDev *dev;
    SoftPart *part;        // forward: slot base for these blocks
    float2 *GP;            // backward: slot base for these blocks (K x n each)
};

// The near pairs from explicit differences, one warp per pair, kNearChunk
// consecutive pairs per warp taken kNearIlp at a time with their loads
// interleaved (the kernel is latency-bound: a pair is a few hundred flops).
// Lane l holds coordinates l, l + 32, ... (NM of them, n <= 32 NM) of the
// differences in registers.  r from the explicit FP32 length and the hi+lo
// differences of Y.  Forward: (M, S) per block.  Backward: per-lane FP32
// accumulation of c_ij (x_i - x_j)(y_i - y_j)^T for its coordinates, summed
// over the block's warps as hi + lo pairs.
constexpr int kNearIlp = 4;

template <int K, int NM, bool BWD>
__global__ void __launch_bounds__(kNearWarps * 32) soft_near_kernel(SoftNearArgs a)
{
    extern __shared__ float gw[];  // backward: kNearWarps x n x K
    __shared__ float redM[kNearWarps];
    __shared__ double redS[kNearWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n;
    const float K2 = a.K2;
    const float LK2 = BWD ? (float)(a.dev->L * (double)K2) : 0.f;
    float gacc[BWD ? NM : 1][K];
#pragma unroll
    for (int m = 0; m < (BWD ? NM : 1); ++m)
#pragma unroll
        for (int c = 0; c < K; ++c) gacc[m][c] = 0.f;
    float M = INFINITY;
    double S64 = 0.0;
    const long long p0 = ((long long)blockIdx.x * kNearWarps + warp) * kNearChunk;
    const long long p1 = min((long long)a.n_near, p0 + kNearChunk);
    for (long long pb = p0; pb < p1; pb += kNearIlp) {
        int ii[kNearIlp], jj[kNearIlp];
        bool valid[kNearIlp];
#pragma unroll
        for (int e = 0; e < kNearIlp; ++e) {
            valid[e] = pb + e < p1;
            const int2 pr = valid[e] ? a.near[pb + e] : a.near[p0];
            ii[e] = pr.x;
            jj[e] = pr.y;
        }
        float D[kNearIlp][NM], dd[kNearIlp], dyl[kNearIlp];
#pragma unroll
        for (int e = 0; e < kNearIlp; ++e) {
            dd[e] = 0.f;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const int l = lane + 32 * m;
                D[e][m] = l < n ? a.X[(size_t)ii[e] * n + l] - a.X[(size_t)jj[e] * n + l] : 0.f;
                dd[e] = fmaf(D[e][m], D[e][m], dd[e]);
            }
            dyl[e] = 0.f;
            if (lane < K) {
                const size_t o = (size_t)lane * a.Npad;
                dyl[e] = (a.Yh[o + ii[e]] - a.Yh[o + jj[e]]) + (a.Yl[o + ii[e]] - a.Yl[o + jj[e]]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int e = 0; e < kNearIlp; ++e) dd[e] += __shfl_xor_sync(FULL, dd[e], o);
#pragma unroll
        for (int e = 0; e < kNearIlp; ++e) {
            if (!valid[e]) continue;
            float dy[K];
#pragma unroll
            for (int c = 0; c < K; ++c) dy[c] = __shfl_sync(FULL, dyl[e], c);
            float r, inv_d2;  // ratio; 1/d^2
            if (dd[e] >= 1e-30f) {
                float zz = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) zz = fmaf(dy[c], dy[c], zz);
                r = sqrtf(zz / dd[e]);
                inv_d2 = 1.0f / dd[e];
            } else {
                // too short for FP32 squares: projection and length in FP64,
                // D and dy rescaled by 1/d so the FP32 products stay in range
                const int i = ii[e], j = jj[e];
                double d2 = 0.0, z[K];
#pragma unroll
                for (int c = 0; c < K; ++c) z[c] = 0.0;
                for (int l = lane; l < n; l += 32) {
                    const double Dl = (double)a.X[(size_t)i * n + l] - (double)a.X[(size_t)j * n + l];
                    d2 = fma(Dl, Dl, d2);
#pragma unroll
                    for (int c = 0; c < K; ++c) z[c] = fma(a.U64[(size_t)c * n + l], Dl, z[c]);
                }
                d2 = warp_sum(d2);
                double zz = 0.0;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    z[c] = warp_sum(z[c]);
                    zz = fma(z[c], z[c], zz);
                }
                const double sc = d2 > 0.0 ? 1.0 / sqrt(d2) : 0.0;
#pragma unroll
                for (int c = 0; c < K; ++c) dy[c] = (float)(z[c] * sc);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const int l = lane + 32 * m;
                    D[e][m] = l < n ? (float)(((double)a.X[(size_t)i * n + l] - (double)a.X[(size_t)j * n + l]) * sc)
                                    : 0.f;
                }
                r = d2 > 0.0 ? (float)sqrt(zz / d2) : NAN;
                inv_d2 = 1.0f;
            }
            if (!BWD) {
                if (r == r) {
                    const float am = (M - r) * K2;
                    if (am > 0.f) {
                        S64 = S64 * (double)ex2_approx(-am) + 1.0;
                        M = r;
                    } else {
                        S64 += (double)ex2_approx(fmaxf(am, -200.f));
                    }
                }
            } else {
                const float pw = ex2_approx(fmaxf(fmaf(r, -K2, LK2), -200.f));
                const float coef = (r * r >= kFltMin) ? pw * inv_d2 / r : 0.f;
#pragma unroll
                for (int m = 0; m < (BWD ? NM : 1); ++m) {
                    const float cD = coef * D[e][m];
#pragma unroll
                    for (int c = 0; c < K; ++c) gacc[m][c] = fmaf(cD, dy[c], gacc[m][c]);
                }
            }
        }
    }
    if (!BWD) {
        if (lane == 0) {
            redM[warp] = M;
            redS[warp] = S64;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kNearWarps; ++w) lse_merge(M, S64, redM[w], redS[w], K2);
            SoftPart pt;
            pt.S = S64;
            pt.M = M;
            pt.pad = 0;
            a.part[blockIdx.x] = pt;
        }
    } else {
        float *g = gw + (size_t)warp * n * K;
#pragma unroll
        for (int m = 0; m < (BWD ? NM : 1); ++m) {
            const int l = lane + 32 * m;
            if (l < n)
#pragma unroll
                for (int c = 0; c < K; ++c) g[l * K + c] = gacc[m][c];
        }
        __syncthreads();
        float2 *out = a.GP + (size_t)blockIdx.x * K * n;
        for (int o = threadIdx.x; o < n * K; o += blockDim.x) {
            const int c = o / n, l = o % n;
            float hi = 0.f, lo = 0.f;
            for (int w = 0; w < kNearWarps; ++w) df_add(hi, lo, gw[(size_t)w * n * K + l * K + c]);
            df_norm(hi, lo);
            out[o] = make_float2(hi, lo);
        }
    }
}

// ------------------------------------------------------- gradient blocks ---

// Gradient of the far pairs for point block B = blockIdx.x (one wave of
// nb blocks), in two phases.
// (1) z_i, i in block B: the rows of tiles (B, J), J >= B, plus the (negated)
//     columns of tiles (I, B), I <= B.  The nb + 1 terms of each entry are
//     dealt to 8 thread groups, accumulated in hi + lo and merged in a fixed
//     order, so the sum is reproducible and (near) exact.
// (2) g_cl = sum_i (x_il - xbar_l) z_ic with error-free products: thread
//     (group q, coordinate l) takes the rows q, q + 8, ... (loads issued
//     together) for all K components; the groups merge in a fixed order;
//     GP[B][c * n + l] = (hi, lo).
constexpr int kZGroups = 8;

template <int K>
__global__ void __launch_bounds__(kZGroups * T, 1) soft_grad_kernel(const float *P, int nb, const float *X,
                                                                    const float *center, int N, int n, float2 *GP)
{
    extern __shared__ float2 part_[];  // kZGroups x K x T (40 KB at K = 5)
    auto part = reinterpret_cast<float2 (*)[K][T]>(part_);
    __shared__ float zh[K][T], zl[K][T];
    const int B = blockIdx.x;
    const int a = threadIdx.x % T, q = threadIdx.x / T;
    {
        float hi[K], lo[K];
#pragma unroll
        for (int c = 0; c < K; ++c) hi[c] = lo[c] = 0.f;
        const int nterms = nb + 1;  // J = B..nb-1 (rows), then I = 0..B (columns)
#pragma unroll 2
        for (int t = q; t < nterms; t += kZGroups) {
            const int J = B + t;
            const float *src = J < nb ? P + (size_t)tile_index(B, J, nb) * 2 * K * T + a
                                      : P + (size_t)tile_index(t - (nb - B), B, nb) * 2 * K * T + (size_t)K * T + a;
            float v[K];
#pragma unroll
            for (int c = 0; c < K; ++c) v[c] = src[c * T];
#pragma unroll
            for (int c = 0; c < K; ++c) df_add(hi[c], lo[c], v[c]);
        }
#pragma unroll
        for (int c = 0; c < K; ++c) part[q][c][a] = make_float2(hi[c], lo[c]);
        __syncthreads();
        if (q < K) {
            const int c = q;  // group q finishes component c = q
            float h = part[0][c][a].x, l = part[0][c][a].y;
            for (int g2 = 1; g2 < kZGroups; ++g2) df_merge(h, l, part[g2][c][a].x, part[g2][c][a].y);
            df_norm(h, l);
            zh[c][a] = h;
            zl[c][a] = l;
        }
        __syncthreads();
    }
    constexpr int RPG = T / kZGroups;  // rows per group
    const int rows = min(T, N - B * T);
    for (int l0 = 0; l0 < n; l0 += T) {
        const int l = l0 + a;
        float hi[K], lo[K];
#pragma unroll
        for (int c = 0; c < K; ++c) hi[c] = lo[c] = 0.f;
        if (l < n) {
            const float cl = center[l];
            float xv[RPG];
#pragma unroll
            for (int t = 0; t < RPG; ++t) {
                const int row = q + kZGroups * t;
                xv[t] = row < rows ? X[(size_t)(B * T + row) * n + l] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < RPG; ++t) {
                const int row = q + kZGroups * t;
                if (row < rows) {
                    const float x = __fsub_rn(xv[t], cl);
#pragma unroll
                    for (int c = 0; c < K; ++c) df_fma(hi[c], lo[c], x, zh[c][row], zl[c][row]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < K; ++c) part[q][c][a] = make_float2(hi[c], lo[c]);
        __syncthreads();
        if (q < K && l < n) {
            const int c = q;
            float h = part[0][c][a].x, lw = part[0][c][a].y;
            for (int g2 = 1; g2 < kZGroups; ++g2) df_merge(h, lw, part[g2][c][a].x, part[g2][c][a].y);
            df_norm(h, lw);
            GP[(size_t)B * K * n + (size_t)c * n + l] = make_float2(h, lw);
        }
        __syncthreads();
    }
}

// G[o] = sum of the partials GP[p][o], one warp per output entry.
__global__ void __launch_bounds__(256) soft_gsum_kernel(const float2 *GP, int nparts, int nK, double *G)
{
    const int o = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= nK) return;
    float hi = 0.f, lo = 0.f;
#pragma unroll 4
    for (int p = lane; p < nparts; p += 32) {
        const float2 v = GP[(size_t)p * nK + o];
        df_merge(hi, lo, v.x, v.y);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const float h2 = __shfl_xor_sync(FULL, hi, s), l2 = __shfl_xor_sync(FULL, lo, s);
        df_merge(hi, lo, h2, l2);
    }
    if (lane == 0) G[o] = (double)hi + (double)lo;
}

// ------------------------------------------------------- Riemannian step ---

struct SoftStepArgs {
    const double *G;     // n x K column-major (dL/dU)
    double *U64;         // n x K column-major, updated in place
    float *U32;          // n x KP row-major
    float *U32lo;        // n x KP, fl(U64 - U32)
    int KP;
    void *Uhi, *Ulo;     // tensor-core operands of the SAP pass (KPG x NP 16-bit) or null
    int NP;
    int split_bf16;
    float split_scale;
    int n;
    double eta;
    SoftDev *dev;
};

// One block: G_R = G - U (U^T G) (projection onto the tangent space of the
// Grassmannian at U), V = U + eta G_R / ||G_R||_F, U <- Q factor of V (two
// Cholesky-QR passes in FP64; positive diagonal of R, as a Householder QR
// with signs fixed), and the FP32 / 16-bit copies the other kernels read.
template <int K>
__global__ void __launch_bounds__(256) soft_step_kernel(SoftStepArgs a)
{
    extern __shared__ double sd[];
    double *sU = sd, *sV = sd + (size_t)K * a.n;
    __shared__ double sA[K][K], sR[K][K], sRi[K][K];
    __shared__ double red[8];
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int idx = tid; idx < K * n; idx += blockDim.x) {
        sU[idx] = a.U64[idx];
        sV[idx] = a.G[idx];
    }
    __syncthreads();
    // A = U^T G (A[c][m] = <u_c, g_m>)
    for (int d = warp; d < K * K; d += 8) {
        const int c = d / K, m = d % K;
        double s = 0.0;
        for (int l = lane; l < n; l += 32) s = fma(sU[c * n + l], sV[m * n + l], s);
        s = warp_sum(s);
        if (lane == 0) sA[c][m] = s;
    }
    __syncthreads();
    double nr2 = 0.0;
    for (int idx = tid; idx < K * n; idx += blockDim.x) {
        const int m = idx / n, l = idx % n;
        double g = sV[idx];
#pragma unroll
        for (int c = 0; c < K; ++c) g = fma(-sU[c * n + l], sA[c][m], g);
        sV[idx] = g;
        nr2 = fma(g, g, nr2);
    }
    nr2 = warp_sum(nr2);
    if (lane == 0) red[warp] = nr2;
    __syncthreads();
    nr2 = 0.0;
    for (int w = 0; w < 8; ++w) nr2 += red[w];
    const double gn = sqrt(nr2);
    if (tid == 0) {
        a.dev->gnorm = gn;
        a.dev->step += 1;
    }
    if (!(gn > 0.0)) return;  // stationary: U unchanged
    const double f = a.eta / gn;
    for (int idx = tid; idx < K * n; idx += blockDim.x) sV[idx] = fma(f, sV[idx], sU[idx]);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int d = warp; d < K * K; d += 8) {
            const int c = d / K, m = d % K;
            if (m < c) continue;
            double s = 0.0;
            for (int l = lane; l < n; l += 32) s = fma(sV[c * n + l], sV[m * n + l], s);
            s = warp_sum(s);
            if (lane == 0) sA[c][m] = s;
        }
        __syncthreads();
        if (tid == 0) {
            // H = R^T R, R upper triangular with positive diagonal
            for (int c = 0; c < K; ++c) {
                double dgn = sA[c][c];
                for (int q = 0; q < c; ++q) dgn -= sR[q][c] * sR[q][c];
                const double rc = sqrt(dgn > 0.0 ? dgn : 0.0);
                sR[c][c] = rc;
                for (int m = c + 1; m < K; ++m) {
                    double v = sA[c][m];
                    for (int q = 0; q < c; ++q) v -= sR[q][c] * sR[q][m];
                    sR[c][m] = rc > 0.0 ? v / rc : 0.0;
                }
                for (int m = 0; m < c; ++m) sR[c][m] = 0.0;
            }
            // Ri = R^-1 (upper), column by column
            for (int m = 0; m < K; ++m) {
                for (int c = K - 1; c >= 0; --c) {
                    double v = (c == m) ? 1.0 : 0.0;
                    for (int q = c + 1; q < K; ++q) v -= sR[c][q] * sRi[q][m];
                    sRi[c][m] = (c <= m && sR[c][c] > 0.0) ? v / sR[c][c] : 0.0;
                }
            }
        }
        __syncthreads();
        for (int l = tid; l < n; l += blockDim.x) {
            double row[K];
#pragma unroll
            for (int c = 0; c < K; ++c) row[c] = sV[c * n + l];
#pragma unroll
            for (int m = 0; m < K; ++m) {
                double s = 0.0;
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (c <= m) s = fma(row[c], sRi[c][m], s);
                sV[m * n + l] = s;
            }
        }
        __syncthreads();
    }
    for (int l = tid; l < n; l += blockDim.x)
#pragma unroll
        for (int m = 0; m < K; ++m) {
            const double s = sV[m * n + l];
            a.U64[(size_t)m * n + l] = s;
            const float sf = (float)s;
            a.U32[(size_t)l * a.KP + m] = sf;
            a.U32lo[(size_t)l * a.KP + m] = (float)(s - (double)sf);
            if (a.Uhi) {
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

// ------------------------------------------------------------ host side ---

#define SCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return handle_fail(h, e_ == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA, \
                               cudaGetErrorString(e_));                                     \
    } while (0)

template <typename T_>
void sfree(T_ *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

size_t fwd_smem(int K, int S) { return (size_t)S * soft_stage_bytes(K); }
size_t bwd_smem(int K, int S) { return (size_t)S * soft_stage_bytes(K) + (size_t)(K * T + kBwdWarps * K * T) * 4; }
// dynamic shared memory per block: the 227 KB opt-in limit less 1 KB for
// the kernels' static barriers and reduction slots
constexpr size_t kSmemLimit = 226 * 1024;

int fwd_stages(int K)
{
    int s = kSoftStagesMax;
    while (s > 2 && fwd_smem(K, s) > kSmemLimit) --s;
    return s;
}
int bwd_stages(int K)
{
    int s = kSoftStagesMax;
    while (s > 2 && bwd_smem(K, s) > kSmemLimit) --s;
    return s;
}

template <int K>
struct SoftKernels {
    static cudaError_t configure()
    {
        cudaError_t e = cudaFuncSetAttribute(soft_pass_kernel<K, kFwdWarps, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(soft_pass_kernel<K, kBwdWarps, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemLimit);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(soft_near_kernel<K, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kNearWarps * kSoftMaxN * K * 4);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(soft_step_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     2 * K * kSoftMaxN * 8);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ydf_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     2 * K * kSoftMaxN * 4);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(soft_grad_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kZGroups * K * T * sizeof(float2)));
        return e;
    }
    static cudaError_t ydf(const float *X, int N, int n, const double *U64, int Npad, float *Yh, float *Yl, int grid,
                           cudaStream_t s)
    {
        ydf_kernel<K><<<grid, 256, 2 * K * n * 4, s>>>(X, N, n, U64, Npad, Yh, Yl);
        return cudaGetLastError();
    }
    static cudaError_t pass(const SoftPassArgs &a, bool bwd, int grid, cudaStream_t s)
    {
        if (bwd)
            soft_pass_kernel<K, kBwdWarps, true><<<grid, (kBwdWarps + 1) * 32, bwd_smem(K, a.stages), s>>>(a);
        else
            soft_pass_kernel<K, kFwdWarps, false><<<grid, (kFwdWarps + 1) * 32, fwd_smem(K, a.stages), s>>>(a);
        return cudaGetLastError();
    }
    template <int NM>
    static void near_nm(const SoftNearArgs &a, bool bwd, int grid, cudaStream_t s)
    {
        if (bwd)
            soft_near_kernel<K, NM, true><<<grid, kNearWarps * 32, kNearWarps * a.n * K * 4, s>>>(a);
        else
            soft_near_kernel<K, NM, false><<<grid, kNearWarps * 32, 0, s>>>(a);
    }
    static cudaError_t near(const SoftNearArgs &a, bool bwd, int grid, cudaStream_t s)
    {
        if (a.n <= 128)
            near_nm<4>(a, bwd, grid, s);
        else
            near_nm<16>(a, bwd, grid, s);
        return cudaGetLastError();
    }
    static cudaError_t grad(const float *P, int nb, const float *X, const float *center, int N, int n, float2 *GP,
                            cudaStream_t s)
    {
        soft_grad_kernel<K><<<nb, kZGroups * T, kZGroups * K * T * sizeof(float2), s>>>(P, nb, X, center, N, n, GP);
        return cudaGetLastError();
    }
    static cudaError_t step(const SoftStepArgs &a, cudaStream_t s)
    {
        soft_step_kernel<K><<<1, 256, 2 * K * a.n * 8, s>>>(a);
        return cudaGetLastError();
    }
};

template <typename F>
cudaError_t dispatch_k(int k, F &&f)
{
    switch (k) {
    case 1: return f(SoftKernels<1>());
    case 2: return f(SoftKernels<2>());
    case 3: return f(SoftKernels<3>());
    case 4: return f(SoftKernels<4>());
    case 5: return f(SoftKernels<5>());
    case 6: return f(SoftKernels<6>());
    case 7: return f(SoftKernels<7>());
    case 8: return f(SoftKernels<8>());
    default: return cudaErrorInvalidValue;
    }
}

// Kernel classes of the profiling accessors (capi.cu numbers them).
constexpr int kClsFwd = 6, kClsBwd = 7, kClsNear = 8, kClsAux = 9;

struct Bracket {
    sap_handle h;
    int cls;
    cudaEvent_t a = nullptr, b = nullptr;
    Bracket(sap_handle hh, int c) : h(hh), cls(c)
    {
        handle_count_launch(h, cls, &a, &b);
        if (a) cudaEventRecord(a, handle_stream(h));
    }
    ~Bracket()
    {
        if (b) cudaEventRecord(b, handle_stream(h));
        handle_push_timing(h, cls, a, b);
    }
};

sap_status check_ready(sap_handle h)
{
    const int k = handle_k(h);
    if (k == 0) return handle_fail(h, SAP_E_STATE, "no basis set");
    if (!handle_x32(h)) return handle_fail(h, SAP_E_UNSUPPORTED, "the soft-min objective needs FP32 or BF16 data");
    if (k > 8) return handle_fail(h, SAP_E_UNSUPPORTED, "the soft-min objective supports k <= 8");
    if (handle_n_dim(h) > kSoftMaxN) return handle_fail(h, SAP_E_UNSUPPORTED, "the soft-min objective supports n <= 512");
    return SAP_OK;
}

sap_status ensure_buffers(sap_handle h, bool need_bwd)
{
    SoftState &ss = soft_state(h);
    RestrState &r = restr_state(h);
    const int k = handle_k(h), n = handle_n_dim(h);
    const int sms = handle_sms(h);
    if (ss.k != k) {
        softmin_free(h);
        SCK(dispatch_k(k, [](auto kk) { return decltype(kk)::configure(); }));
        SCK(cudaMalloc(&ss.Yh, (size_t)k * r.Npad * sizeof(float)));
        SCK(cudaMalloc(&ss.Yl, (size_t)k * r.Npad * sizeof(float)));
        SCK(cudaMalloc(&ss.G, (size_t)k * n * sizeof(double)));
        SCK(cudaMalloc(&ss.dev, sizeof(SoftDev)));
        SoftDev d;
        std::memset(&d, 0, sizeof(d));
        SCK(cudaMemcpy(ss.dev, &d, sizeof(d), cudaMemcpyHostToDevice));
        ss.k = k;
        ss.grid_far = std::min(r.nwtiles, sms);
        ss.n_near = -1;
    }
    if (ss.n_near != r.n_near) {
        ss.n_near = r.n_near;
        ss.near_blocks = (r.n_near + kNearWarps * kNearChunk - 1) / (kNearWarps * kNearChunk);
        const int parts = ss.grid_far + ss.near_blocks;
        if (parts > ss.part_cap) {
            sfree(ss.part);
            SCK(cudaMalloc(&ss.part, (size_t)parts * sizeof(SoftPart)));
            ss.part_cap = parts;
        }
        const int nb = r.Npad / T;
        const int gparts = nb + ss.near_blocks;
        if (gparts > ss.gp_cap) {
            sfree(ss.GP);
            SCK(cudaMalloc(&ss.GP, (size_t)gparts * k * n * sizeof(float2)));
            ss.gp_cap = gparts;
        }
    }
    if (need_bwd && !ss.P) SCK(cudaMalloc(&ss.P, (size_t)r.nwtiles * 2 * k * T * sizeof(float)));
    return SAP_OK;
}

sap_status enqueue_forward(sap_handle h, double tau, bool with_hist)
{
    SoftState &ss = soft_state(h);
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int k = handle_k(h), n = handle_n_dim(h), N = (int)handle_n_points(h);
    const float K2 = (float)(1.4426950408889634 / tau);
    {
        Bracket b(h, kClsAux);
        const float *X = handle_x32(h);
        const double *U64 = handle_u64(h);
        const int grid = std::min(r.Npad / 32, 4 * handle_sms(h));
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::ydf(X, N, n, U64, r.Npad, ss.Yh, ss.Yl, grid, s); }));
    }
    if (ss.near_blocks > 0) {
        SoftNearArgs na;
        na.X = handle_x32(h); na.N = N; na.n = n;
        na.Yh = ss.Yh; na.Yl = ss.Yl; na.Npad = r.Npad;
        na.U64 = handle_u64(h);
        na.near = r.near; na.n_near = r.n_near;
        na.K2 = K2; na.dev = ss.dev;
        na.part = ss.part + ss.grid_far;
        na.GP = nullptr;
        Bracket b(h, kClsNear);
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::near(na, false, ss.near_blocks, s); }));
    }
    SoftPassArgs pa;
    pa.w = r.w; pa.wtiles = r.wtiles; pa.ntiles = r.nwtiles;
    pa.Yh = ss.Yh; pa.Yl = ss.Yl; pa.Npad = r.Npad;
    pa.stages = fwd_stages(k);
    pa.K2 = K2; pa.tau = tau; pa.dev = ss.dev;
    pa.part = ss.part; pa.nparts = ss.grid_far + ss.near_blocks;
    pa.hist = with_hist ? ss.hist : nullptr;
    pa.P = nullptr;
    Bracket b(h, kClsFwd);
    SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::pass(pa, false, ss.grid_far, s); }));
    return SAP_OK;
}

// Backward pass; Y must hold the current basis's product (the forward makes
// it) and dev->L the forward value.
sap_status enqueue_backward(sap_handle h, double tau)
{
    SoftState &ss = soft_state(h);
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int k = handle_k(h), n = handle_n_dim(h), N = (int)handle_n_points(h);
    const float K2 = (float)(1.4426950408889634 / tau);
    const int nb = r.Npad / T;
    if (ss.near_blocks > 0) {
        SoftNearArgs na;
        na.X = handle_x32(h); na.N = N; na.n = n;
        na.Yh = ss.Yh; na.Yl = ss.Yl; na.Npad = r.Npad;
        na.U64 = handle_u64(h);
        na.near = r.near; na.n_near = r.n_near;
        na.K2 = K2; na.dev = ss.dev;
        na.part = nullptr;
        na.GP = ss.GP + (size_t)nb * k * n;
        Bracket b(h, kClsNear);
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::near(na, true, ss.near_blocks, s); }));
    }
    {
        SoftPassArgs pa;
        pa.w = r.w; pa.wtiles = r.wtiles; pa.ntiles = r.nwtiles;
        pa.Yh = ss.Yh; pa.Yl = ss.Yl; pa.Npad = r.Npad;
        pa.stages = bwd_stages(k);
        pa.K2 = K2; pa.tau = tau; pa.dev = ss.dev;
        pa.part = nullptr; pa.nparts = 0; pa.hist = nullptr;
        pa.P = ss.P;
        Bracket b(h, kClsBwd);
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::pass(pa, true, ss.grid_far, s); }));
    }
    {
        Bracket b(h, kClsAux);
        const float *X = handle_x32(h);
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::grad(ss.P, nb, X, r.center, N, n, ss.GP, s); }));
    }
    {
        Bracket b(h, kClsAux);
        const int nK = n * k;
        soft_gsum_kernel<<<(nK + 7) / 8, 256, 0, s>>>(ss.GP, nb + ss.near_blocks, nK, ss.G);
        SCK(cudaGetLastError());
    }
    return SAP_OK;
}

sap_status enqueue_step(sap_handle h, double eta)
{
    SoftState &ss = soft_state(h);
    RestrState &r = restr_state(h);
    SoftStepArgs sa;
    sa.G = ss.G;
    sa.U64 = handle_u64(h);
    sa.U32 = handle_u32_mut(h);
    sa.U32lo = const_cast<float *>(handle_u32lo(h));
    sa.KP = handle_kp(h);
    sa.Uhi = r.Uhi; sa.Ulo = r.Ulo; sa.NP = r.NP;
    sa.split_bf16 = handle_split_bf16(h);
    sa.split_scale = sa.split_bf16 ? 256.f : 2048.f;
    sa.n = handle_n_dim(h);
    sa.eta = eta;
    sa.dev = ss.dev;
    Bracket b(h, kClsAux);
    SCK(dispatch_k(handle_k(h), [&](auto kk) { return decltype(kk)::step(sa, handle_stream(h)); }));
    return SAP_OK;
}

sap_status read_dev(sap_handle h, SoftDev *out)
{
    SoftState &ss = soft_state(h);
    cudaStream_t s = handle_stream(h);
    SCK(cudaMemcpyAsync(out, ss.dev, sizeof(SoftDev), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (out->status) {
        const int st = out->status;
        SCK(cudaMemsetAsync(&ss.dev->status, 0, sizeof(int), s));
        SCK(cudaStreamSynchronize(s));
        if (st & ST_BOUNDS) return handle_fail(h, SAP_E_BOUNDS, "a device index was out of range (debug build)");
        if (st & ST_NO_SECANT) return handle_fail(h, SAP_E_NO_SECANT, "every pair is excluded");
        if (st & ST_TIMEOUT) return handle_fail(h, SAP_E_TIMEOUT, "a device-side wait gave up");
        return handle_fail(h, SAP_E_CUDA, "soft-min kernel status");
    }
    return SAP_OK;
}

bool tau_ok(double tau) { return tau > 0.0 && std::isfinite(tau) && 1.4426950408889634 / tau < 3.0e38; }

} // namespace

sap_status softmin_forward(sap_handle h, double tau, double *L_out)
{
    if (!tau_ok(tau)) return handle_fail(h, SAP_E_ARG, "tau must be positive and finite");
    sap_status st = check_ready(h);
    if (st != SAP_OK) return st;
    st = ensure_buffers(h, false);
    if (st != SAP_OK) return st;
    st = enqueue_forward(h, tau, false);
    if (st != SAP_OK) return st;
    SoftDev d;
    st = read_dev(h, &d);
    if (st != SAP_OK) return st;
    if (L_out) *L_out = d.L;
    return SAP_OK;
}

sap_status softmin_backward(sap_handle h, double tau, double L, double *G_out, int out_is_device)
{
    if (!tau_ok(tau)) return handle_fail(h, SAP_E_ARG, "tau must be positive and finite");
    if (!std::isfinite(L)) return handle_fail(h, SAP_E_ARG, "L must be finite");
    if (!G_out) return handle_fail(h, SAP_E_ARG, "null output");
    sap_status st = check_ready(h);
    if (st != SAP_OK) return st;
    st = ensure_buffers(h, true);
    if (st != SAP_OK) return st;
    SoftState &ss = soft_state(h);
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int k = handle_k(h), n = handle_n_dim(h), N = (int)handle_n_points(h);
    {
        // Y for the current basis (the backward does not rely on a previous forward)
        Bracket b(h, kClsAux);
        const float *X = handle_x32(h);
        const double *U64 = handle_u64(h);
        const int grid = std::min(r.Npad / 32, 4 * handle_sms(h));
        SCK(dispatch_k(k, [&](auto kk) { return decltype(kk)::ydf(X, N, n, U64, r.Npad, ss.Yh, ss.Yl, grid, s); }));
    }
    SCK(cudaMemcpyAsync(&ss.dev->L, &L, sizeof(double), cudaMemcpyHostToDevice, s));
    st = enqueue_backward(h, tau);
    if (st != SAP_OK) return st;
    SCK(cudaMemcpyAsync(G_out, ss.G, (size_t)k * n * sizeof(double),
                        out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SoftDev d;
    return read_dev(h, &d);
}

sap_status softmin_ascent(sap_handle h, double tau, double eta, int steps, double *hist)
{
    if (!tau_ok(tau)) return handle_fail(h, SAP_E_ARG, "tau must be positive and finite");
    if (!(eta >= 0.0) || !std::isfinite(eta)) return handle_fail(h, SAP_E_ARG, "eta must be finite and >= 0");
    if (steps < 0) return handle_fail(h, SAP_E_ARG, "steps must be >= 0");
    sap_status st = check_ready(h);
    if (st != SAP_OK) return st;
    st = ensure_buffers(h, true);
    if (st != SAP_OK) return st;
    SoftState &ss = soft_state(h);
    cudaStream_t s = handle_stream(h);
    SCK(cudaStreamSynchronize(s));
    if (steps + 1 > ss.hist_cap) {
        sfree(ss.hist);
        const int cap = std::max(steps + 1, 256);
        SCK(cudaMalloc(&ss.hist, (size_t)cap * sizeof(double)));
        ss.hist_cap = cap;
    }
    SoftDev d;
    std::memset(&d, 0, sizeof(d));
    d.hist_cap = ss.hist_cap;
    SCK(cudaMemcpy(ss.dev, &d, sizeof(d), cudaMemcpyHostToDevice));
    // one step = forward (records L), backward, update; captured once and
    // replayed `steps` times
    if (steps > 0 && handle_profiling(h)) {
        // timed launch by launch
        for (int q = 0; q < steps && st == SAP_OK; ++q) {
            st = enqueue_forward(h, tau, true);
            if (st == SAP_OK) st = enqueue_backward(h, tau);
            if (st == SAP_OK) st = enqueue_step(h, eta);
        }
        if (st != SAP_OK) return st;
    } else if (steps > 0) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long before = handle_launches(h);
        SCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = enqueue_forward(h, tau, true);
        if (st == SAP_OK) st = enqueue_backward(h, tau);
        if (st == SAP_OK) st = enqueue_step(h, eta);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        const long long per_step = handle_launches(h) - before;
        handle_add_launches(h, -per_step);  // capture records; replays count
        if (st != SAP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        SCK(e);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        SCK(e);
        for (int q = 0; q < steps; ++q) {
            e = cudaGraphLaunch(exec, s);
            if (e != cudaSuccess) break;
            handle_add_launches(h, per_step);
        }
        cudaGraphExecDestroy(exec);
        SCK(e);
    }
    // the value at the final basis
    st = enqueue_forward(h, tau, true);
    if (st != SAP_OK) return st;
    st = read_dev(h, &d);
    if (st != SAP_OK) return st;
    if (hist) SCK(cudaMemcpy(hist, ss.hist, (size_t)(steps + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    // the SAP watch list and bounds refer to the old basis
    return handle_reset_state(h);
}

void softmin_free(sap_handle h)
{
    SoftState &ss = soft_state(h);
    sfree(ss.Yh); sfree(ss.Yl); sfree(ss.part); sfree(ss.P); sfree(ss.GP); sfree(ss.G); sfree(ss.dev);
    sfree(ss.hist);
    ss.k = 0;
    ss.part_cap = ss.gp_cap = ss.hist_cap = 0;
    ss.n_near = -1;
}

} // namespace sap
