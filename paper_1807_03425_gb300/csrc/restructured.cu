// restructured.cu -- the restructured form of the SAP argmin step.
//
// For a basis U and Y = X U, U^T (x_i - x_j) = y_i - y_j, so
//     r_ij^2 = ||y_i - y_j||^2 * w_ij,   w_ij = 1 / ||x_i - x_j||^2.
// The lengths are computed once per dataset (and threshold eps, Sec. VII)
// from explicit FP32 differences; each iteration then costs one tensor-core
// product and one pass over the stored w (4 bytes per pair).
//
// Precision.  The rows of Y carry absolute errors of order eps_Y ||x - mean||
// (split-operand product, FP32 accumulation), so y_i - y_j cancels for close
// pairs.  Per pair the pass's error is bounded by
//     beta_ij = sqrt(k) eps_Y (nu_i + nu_j) / d_ij  (+ a relative FP32 term),
// with nu_i = ||x_i - mean||.  Pairs with beta_ij above a cap are "near": the
// pass skips them (w = NaN) and every iteration re-evaluates them from
// explicit differences instead.  All other pairs are certified to within the
// cap, so the pass emits every pair that can still be the argmin (selection
// scheme of sap_internal.cuh); the explicit-difference tier narrows the list
// and the FP64 tier decides.
//
// Layout.  w is stored tile-major over the upper triangle: tile t = (I, J),
// I <= J, holds the 128 x 128 pairs (I*128 + a, J*128 + b) row-major at
// w + t*128*128; entries with i >= j, with an index beyond N, excluded pairs
// and near pairs hold NaN.
#include "restructured.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace sap {
namespace {

constexpr int T = kTile;       // 128
constexpr int WLC = 16;        // coordinates per chunk in the length prep

// ------------------------------------------------------------------ prep ---

__global__ void colmean_kernel(const float *X, int N, int n, float *center)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += (double)X[(size_t)i * n + l];
    center[l] = (float)(acc / N);
}

__global__ void absmax_kernel(const float *X, size_t count, int n, const float *center,
                              unsigned int *out)
{
    float m = 0.f;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count;
         idx += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(X[idx] - center[idx % n]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <typename H>
__device__ __forceinline__ H to16(float v);
template <>
__device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }

// hi = 16-bit(xs), lo = 16-bit((xs - hi) * lo_mul), xs = (x - mean) * scale;
// zero outside N x n.  The difference xs - hi is exact in FP32 and the
// scalings are powers of two.
template <typename H>
__global__ void split_kernel(const float *X, int N, int n, const float *center, float scale,
                             float lo_mul, H *hi, H *lo, int Npad, int NP)
{
    const size_t count = (size_t)Npad * NP;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / NP), l = (int)(idx % NP);
        const float x = (r < N && l < n) ? X[(size_t)r * n + l] - center[l] : 0.f;
        const float xs = x * scale;
        const H h = to16<H>(xs);
        hi[idx] = h;
        lo[idx] = to16<H>((xs - from16(h)) * lo_mul);
    }
}

// nu_i = ||fl(x_i - mean)||_2, rounded up (one warp per row; 0 for pad rows).
__global__ void rownorm_kernel(const float *X, int N, int n, const float *center, float *nu, int Npad)
{
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= Npad) return;
    double acc = 0.0;
    if (row < N)
        for (int l = lane; l < n; l += 32) {
            const double v = (double)(X[(size_t)row * n + l] - center[l]);
            acc = fma(v, v, acc);
        }
    acc = warp_sum(acc);
    if (lane == 0) nu[row] = row < N ? __double2float_ru(sqrt(acc)) * (1.0f + 1e-6f) : 0.f;
}

// ||x_i|| of the points as given (not centred), rounded up; 0 for pad rows.
__global__ void xnorm_kernel(const float *X, int N, int n, float *xn, int Npad)
{
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= Npad) return;
    double acc = 0.0;
    if (row < N)
        for (int l = lane; l < n; l += 32) {
            const double v = (double)X[(size_t)row * n + l];
            acc = fma(v, v, acc);
        }
    acc = warp_sum(acc);
    if (lane == 0) xn[row] = row < N ? __double2float_ru(sqrt(acc)) * (1.0f + 1e-6f) : 0.f;
}

struct WPrepArgs {
    const float *X;
    int N, n;
    const float *nu;
    const int2 *wtiles;
    float *w;
    __nv_bfloat16 *wb;       // BF16 1/d^2 of the stored pairs (NaN elsewhere)
    float eps2_lo, eps2_hi;  // FP32 window around eps^2 (0,0: no threshold)
    double eps2;
    float beta_coef;         // sqrt(k) * eps_Y, rounded up
    float b_cap;
    int2 *near;
    float *near_w;           // 1/d^2 of each near pair (+inf below FP32 range)
    unsigned int near_cap;
    unsigned int *counters;  // [0] near count, [1] excluded count (low), [2] status
};

// Exact decision in FP64 for pairs too close to call in FP32.
__device__ bool excluded_fp64(const float *X, int n, int i, int j, double eps2)
{
    double d2 = 0.0;
    for (int l = 0; l < n; ++l) {
        const double D = (double)X[(size_t)i * n + l] - (double)X[(size_t)j * n + l];
        d2 = fma(D, D, d2);
    }
    return d2 == 0.0 || d2 < eps2;
}

// One 128 x 128 tile of lengths per block: 256 threads, 8 x 8 pairs each.
__global__ void __launch_bounds__(256) wprep_kernel(WPrepArgs a)
{
    __shared__ __align__(16) float xsI[WLC][T + 4];
    __shared__ __align__(16) float xsJ[WLC][T + 4];
    __shared__ int scan[33];
    __shared__ int base_sh;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int2 IJ = a.wtiles[blockIdx.x];
    const int i0 = IJ.x * T, j0 = IJ.y * T;
    float d2[8][8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) d2[p][q] = 0.f;
    for (int l0 = 0; l0 < a.n; l0 += WLC) {
        __syncthreads();
        for (int idx = tid; idx < T * WLC; idx += 256) {
            const int r = idx / WLC, l = idx % WLC, gl = l0 + l;
            xsI[l][r] = (i0 + r < a.N && gl < a.n) ? a.X[(size_t)(i0 + r) * a.n + gl] : 0.f;
            xsJ[l][r] = (j0 + r < a.N && gl < a.n) ? a.X[(size_t)(j0 + r) * a.n + gl] : 0.f;
        }
        __syncthreads();
        const int lc = min(WLC, a.n - l0);
        for (int l = 0; l < lc; ++l) {
            const float4 i4a = *reinterpret_cast<const float4 *>(&xsI[l][ty * 8]);
            const float4 i4b = *reinterpret_cast<const float4 *>(&xsI[l][ty * 8 + 4]);
            const float4 j4a = *reinterpret_cast<const float4 *>(&xsJ[l][tx * 8]);
            const float4 j4b = *reinterpret_cast<const float4 *>(&xsJ[l][tx * 8 + 4]);
            const float xi[8] = {i4a.x, i4a.y, i4a.z, i4a.w, i4b.x, i4b.y, i4b.z, i4b.w};
            const float xj[8] = {j4a.x, j4a.y, j4a.z, j4a.w, j4b.x, j4b.y, j4b.z, j4b.w};
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float D = xi[p] - xj[q];
                    d2[p][q] = fmaf(D, D, d2[p][q]);
                }
        }
    }
    const bool epson = a.eps2_hi > 0.f;
    int nnear = 0, nexcl = 0;
    unsigned long long near_bits = 0ull;  // bit p*8+q marks a near pair
    float *wt = a.w + (size_t)blockIdx.x * T * T;
    __nv_bfloat16 *ht = a.wb + (size_t)blockIdx.x * T * T;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int i = i0 + ty * 8 + p;
        float out[8];
        __nv_bfloat16 hout[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + tx * 8 + q;
            const float dd = d2[p][q];
            float wv = __int_as_float(0x7fc00000);  // NaN: skipped by the pass
            __nv_bfloat16 hv = __ushort_as_bfloat16((unsigned short)0x7fc0);
            if (i < j && j < a.N) {
                int cls;  // 0 excluded, 1 near, 2 stored
                if (epson && dd < a.eps2_lo) cls = 0;
                else if ((epson && dd < a.eps2_hi) || dd < 1e-30f)
                    cls = excluded_fp64(a.X, a.n, i, j, a.eps2) ? 0 : 1;
                else {
                    const float inv = 1.0f / dd;
                    const float id = 1.0f / sqrtf(dd);
                    const float beta = a.beta_coef * (a.nu[i] + a.nu[j]) * id;
                    // near: the bound exceeds the cap
                    if (beta > a.b_cap) cls = 1;
                    else { cls = 2; wv = inv; hv = __float2bfloat16_rn(inv); }
                }
                if (cls == 0) ++nexcl;
                if (cls == 1) { ++nnear; near_bits |= 1ull << (p * 8 + q); }
            }
            out[q] = wv;
            hout[q] = hv;
        }
        float4 *dst = reinterpret_cast<float4 *>(wt + (size_t)(ty * 8 + p) * T + tx * 8);
        dst[0] = make_float4(out[0], out[1], out[2], out[3]);
        dst[1] = make_float4(out[4], out[5], out[6], out[7]);
        uint4 hp;
        hp.x = (unsigned)__bfloat16_as_ushort(hout[0]) | ((unsigned)__bfloat16_as_ushort(hout[1]) << 16);
        hp.y = (unsigned)__bfloat16_as_ushort(hout[2]) | ((unsigned)__bfloat16_as_ushort(hout[3]) << 16);
        hp.z = (unsigned)__bfloat16_as_ushort(hout[4]) | ((unsigned)__bfloat16_as_ushort(hout[5]) << 16);
        hp.w = (unsigned)__bfloat16_as_ushort(hout[6]) | ((unsigned)__bfloat16_as_ushort(hout[7]) << 16);
        *reinterpret_cast<uint4 *>(ht + (size_t)(ty * 8 + p) * T + tx * 8) = hp;
    }
    int total;
    const int off = block_exclusive_scan(nnear, scan, &total);
    if (tid == 0 && total > 0) base_sh = (int)atomicAdd(&a.counters[0], (unsigned int)total);
    __syncthreads();
    if (total > 0) {
        unsigned int pos = (unsigned int)base_sh + off;
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (near_bits >> (p * 8 + q) & 1ull) {
                    if (pos < a.near_cap) {
                        a.near[pos] = make_int2(i0 + ty * 8 + p, j0 + tx * 8 + q);
                        a.near_w[pos] = d2[p][q] < 1e-30f ? INFINITY : 1.0f / d2[p][q];
                    } else {
                        atomicOr(&a.counters[2], 1u);
                    }
                    ++pos;
                }
    }
    int ex_total;
    block_exclusive_scan(nexcl, scan, &ex_total);
    if (tid == 0 && ex_total > 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.counters[4]), (unsigned long long)ex_total);
}

// ------------------------------------------------------- all-pairs pass ---

constexpr int kPassStagesMax = 5;

struct PassArgs {
    const uint16_t *wb;  // BF16 1/d^2 tiles (tile-major upper triangle; NaN: skipped)
    const int2 *wtiles;
    int ntiles;
    const float *Y;   // this basis's first component in block 0 of the block-major Y
    const float *Yd;  // the same in the doubled row-side copy (block stride Ykt * 256 floats)
    int KY;           // components of this basis
    int Ykt;          // components per block of the Y buffer (block stride / 128)
    int Npad;
    const float *nu;  // ||fl(x_i - mean)||, rounded up (Npad)
    float beta;       // sqrt(k) eps_Y, rounded up: per-pair bound beta (nu_i + nu_j) / d_ij
    int stages;
    Cert cert;        // A = the cap of every stored pair's bound (b_cap), rho
    ProbState *st;
    int2 *cand;
    long long cap;
    int pdl;
    // second and third tiers inside the pass (non-null X; k <= 16): the
    // near pairs (before the tiles) and every emitted pair are evaluated at
    // once by the warp that holds them, from explicit FP32 differences (the
    // explicit tier's arithmetic and error model, cert32), which tightens
    // the bounds; the survivors wait in the warp's list and, once its tiles
    // are done, those that can still be the argmin under the bound as it is
    // then are evaluated in FP64 (the FP64 recheck's arithmetic).  Every
    // block leaves its best (q = r^2, i, j) in partials[blockIdx.x] for the
    // update.  No list is written; st->cnt1 counts the emitted pairs,
    // st->cnt2 the FP64 evaluations.
    const float *X = nullptr;  // N x n FP32 points
    int N = 0, n = 0;
    const float *U32 = nullptr;  // n x KP FP32 basis (pad columns zero)
    int KP = 0;
    const double *U64 = nullptr;  // n x k FP64 basis, column-major
    int k = 0;
    double eps2 = 0.0;            // squared minimum secant length
    const int2 *near = nullptr;
    int n_near = 0;
    Partial *partials = nullptr;
    Cert cert32;
};

// One ring stage: the BF16 1/d^2 tile (32 KB), then the row side's point
// block -- for k <= 8 the k used components of the doubled copy ({y, y}
// pairs, 1 KB each), else the KY components of Y -- and the column side's
// (k, else KY, components of Y; one copy each, block-major), then the 128
// point norms nu of each side.
// kd: the compute width of a pass class with four columns per thread
// (k <= 16), which stages kd components per side (the row side from the
// doubled copy); 0: the other classes, which stage all KY components.
__host__ __device__ inline uint32_t pass_row_bytes(int kd, int KY) { return kd ? (uint32_t)kd * T * 8 : (uint32_t)T * KY * 4; }
__host__ __device__ inline uint32_t pass_col_bytes(int kd, int KY) { return kd ? (uint32_t)kd * T * 4 : (uint32_t)T * KY * 4; }
__host__ __device__ inline uint32_t pass_stage_bytes(int kd, int KY)
{
    return (uint32_t)T * T * 2 + pass_row_bytes(kd, KY) + pass_col_bytes(kd, KY) + 2u * T * 4;
}
inline int pass_kd(int k) { return k <= 8 ? k : k <= 10 ? 10 : k <= 12 ? 12 : k <= 16 ? 16 : 0; }

// Certified error of one stored pair's ratio from the tensor-core Y:
// |r~ - r| <= beta (nu_i + nu_j) / d_ij + rho r.  1/d_ij is taken as the
// square root of the stored BF16 w = 1/d^2 (relative error of w <= 2^-8, so
// of its root <= 2^-9 + 2^-23 with the FP32 root: inflated by 3 10^-3).  The
// same product the length preparation compares with b_cap.
__device__ __forceinline__ float pair_bound(float beta, float nui, float nuj, float w)
{
    return beta * (nui + nuj) * sqrtf(w) * 1.003f;
}

// Two BF16 values packed in a 32-bit word, widened exactly to FP32 (a BF16
// value is the upper half of the FP32 value): integer-pipe operations only.
__device__ __forceinline__ float bf16_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t x) { return __uint_as_float(x & 0xffff0000u); }
__device__ __forceinline__ float bf16_at(const uint16_t *p) { return __uint_as_float((uint32_t)*p << 16); }

// Persistent, warp-specialised pass: one block per SM.  Each block's first
// `stages` tiles are blockIdx.x + it * gridDim.x (their constant parts are
// fetched before the previous kernel has finished); the remaining tiles
// are handed out from a counter, so a block that starts late (its SM still
// busy with the previous kernels) takes fewer.  A producer warp keeps a ring of
// `stages` shared-memory buffers filled by 1-D TMA bulk copies (the 32 KB
// BF16 w tile, for each side the basis's components of the point block and
// the point norms); 16
// consumer warps evaluate the tiles.  Full/empty mbarriers hand the buffers
// over, so the loop has no block-wide barrier.  Each consumer thread owns CPT
// adjacent columns (j) of rows spaced 16/(4/CPT) apart (32 pairs per tile);
// K = compute width (k, or k rounded up for large k: Y's pad components are
// zero).  q = ||y_i - y_j||^2 w is formed with packed FP32 pairs; w is
// widened from BF16 by integer operations, off the FP32 pipe.  Every warp
// bounds the minimum from its own pairs (a valid upper bound like any other),
// tightens the global running bound with a fire-and-forget atomic, and
// emits its candidates with one atomic per warp when it has any.
//
// Bounds.  Every stored pair's error is at most b_p = beta (nu_i + nu_j) /
// d_ij <= A (= b_cap; pairs above it are on the near list).  The fast path
// tests each pair against the uniform A; a warp whose tile could tighten the
// upper bound takes the bound of its minimum from that pair's own b_p, and a
// pair that passes the uniform test is emitted only if it passes its own:
// r~_p <= U (1 + rho) + b_p.  Both refinements touch only the rare slow path.
constexpr int kConsumerWarps = 16;
constexpr int kPassThreads = (kConsumerWarps + 1) * 32;

// A second-tier survivor of the pass waiting for the FP64 tier (r: its FP32
// explicit ratio, -1 when too short for FP32).
struct DeferredPair {
    int i, j;
    float r;
};
constexpr int kDefer = 32;     // deferred survivors per consumer warp
constexpr int kDrainTile = 6;  // tiles before the first check of the deferred survivors
// dynamic shared memory of the pass: the 227 KB a block may hold, less the
// static part (barriers, tile coordinates, the deferred survivors)
constexpr int kPassDynSmem = 216 * 1024;

// Explicit FP32 differences of E pairs by one warp (lanes over the
// coordinates, the E (K + 1) sums reduced together), as in the explicit
// tier: lane e < E receives pair e's ratio rr and code (1: rr valid, 2:
// |x_i - x_j|^2 too small for FP32, a later tier decides; 0: none).
// expl32_finish reduces the per-lane sums acc[e (K + 1) + c].
template <int K, int E>
__device__ __forceinline__ void expl32_finish(float (&acc)[E * (K + 1)], const bool (&valid)[E], int lane, float &rr,
                                              int &code)
{
    constexpr int M = E * (K + 1);
    static_assert(M <= 32, "pairs per warp times components");
    constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
    constexpr int dup = 32 / S;
    float r[S];
#pragma unroll
    for (int q = 0; q < S; ++q) r[q] = q < M ? acc[q < M ? q : 0] : 0.f;
    const float t = warp_reduce_scatter<S>(r, lane);
    const int me = lane < E ? lane : 0;
    float z[K + 1];
#pragma unroll
    for (int c = 0; c <= K; ++c) z[c] = __shfl_sync(0xffffffffu, t, (me * (K + 1) + c) * dup);
    bool myvalid = valid[0];
#pragma unroll
    for (int e = 1; e < E; ++e)
        if (lane == e) myvalid = valid[e];
    const float dd = z[K];
    float zz = 0.f;
#pragma unroll
    for (int c = 0; c < K; ++c) zz = fmaf(z[c], z[c], zz);
    code = (lane >= E || !myvalid) ? 0 : (dd < 1e-30f ? 2 : 1);
    rr = code == 1 ? sqrtf(zz / dd) : INFINITY;
}

// One coordinate l of the sums: |D|^2 and U^T D for each pair's D[e]
template <int K, int E>
__device__ __forceinline__ void expl32_step(float (&acc)[E * (K + 1)], const float *U32, int KP, int l,
                                            const float (&D)[E])
{
    constexpr int KU = (K + 3) / 4 * 4;
    float u[KU];
#pragma unroll
    for (int c = 0; c < KU; c += 4) {
        // L2 only, like the point rows below: the pass leaves little L1
        // beside its shared memory (read-only loads through the L1 measured
        // 0.6-0.9 us slower per iteration)
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(U32 + (size_t)l * KP + c));
        u[c] = t.x; u[c + 1] = t.y; u[c + 2] = t.z; u[c + 3] = t.w;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        acc[e * (K + 1) + K] = fmaf(D[e], D[e], acc[e * (K + 1) + K]);
#pragma unroll
        for (int c = 0; c < K; ++c) acc[e * (K + 1) + c] = fmaf(u[c], D[e], acc[e * (K + 1) + c]);
    }
}

template <int K, int E>
__device__ __forceinline__ void expl32_eval(const float *X, int n, const float *U32, int KP, const int2 (&pr)[E],
                                            const bool (&valid)[E], int lane, float &rr, int &code)
{
    float acc[E * (K + 1)];
#pragma unroll
    for (int q = 0; q < E * (K + 1); ++q) acc[q] = 0.f;
#pragma unroll 2
    for (int l = lane; l < n; l += 32) {
        float D[E];
#pragma unroll
        for (int e = 0; e < E; ++e) D[e] = __ldcg(X + (size_t)pr[e].x * n + l) - __ldcg(X + (size_t)pr[e].y * n + l);
        expl32_step<K, E>(acc, U32, KP, l, D);
    }
    expl32_finish<K, E>(acc, valid, lane, rr, code);
}

template <int K, int CPT, bool EXPL>
__global__ void __launch_bounds__(kPassThreads, 1) restr_pass_kernel(PassArgs a)
{
    constexpr int SR = 4 / CPT;                  // warps sharing one row
    constexpr int RSTEP = kConsumerWarps / SR;   // row step of one warp
    constexpr int RPW = T / RSTEP;               // rows per warp
    constexpr int NPR = CPT / 2;                 // column pairs per thread
    static_assert(RPW * CPT == 32, "one bit per pair of a thread in the emission mask");
    // indexed directly (no integer round trip) so reads stay shared-memory loads
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[kPassStagesMax], empty[kPassStagesMax];
    __shared__ int2 sIJ[kPassStagesMax];
    __shared__ Partial pbest[kConsumerWarps];  // tiers inside: the warps' best pairs
    __shared__ unsigned int pdone;             // consumer warps finished
    __shared__ DeferredPair defer[EXPL ? kConsumerWarps : 1][EXPL ? kDefer : 1];

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int KY = a.KY, S = a.stages;
    constexpr bool DBL = CPT == 4;  // row side from the doubled copy (K <= 16)
    const uint32_t wbytes = T * T * 2, ibytes = pass_row_bytes(DBL ? K : 0, KY),
                   jbytes = pass_col_bytes(DBL ? K : 0, KY), sbytes = wbytes + ibytes + jbytes + 2 * T * 4;
    // tiles below gridDim.x * S are static (it < S); the rest are dynamic
    const int nall = blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int nstatic = nall < S ? nall : S;
    const long long budget = 4000000000ll;

    if (tid == 0) {
        pdone = 0;
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kConsumerWarps);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ---------------- producer warp ----------------
        if (lane == 0) {
            // The stored lengths and point norms are constant: the first
            // stages' copies start before the product of this iteration has
            // finished (programmatic launch); Y follows after the wait.
            const int pre = nstatic;
            for (int it = 0; it < pre; ++it) {
                const int t = blockIdx.x + it * gridDim.x;
                int2 IJ = a.wtiles[t];
                if (!SAP_BOUNDS_OK(a.st, IJ.x >= 0 && IJ.x <= IJ.y && IJ.y < a.Npad / T)) IJ = make_int2(0, 0);
                sIJ[it] = IJ;  // published by the mbarrier completion
                unsigned char *base = sm + (size_t)it * sbytes;
                tc::mbar_expect_tx(&full[it], sbytes);
                tc::bulk_g2s(base, a.wb + (size_t)t * T * T, wbytes, &full[it]);
                tc::bulk_g2s(base + wbytes + ibytes + jbytes, a.nu + (size_t)IJ.x * T, T * 4, &full[it]);
                tc::bulk_g2s(base + wbytes + ibytes + jbytes + T * 4, a.nu + (size_t)IJ.y * T, T * 4, &full[it]);
            }
            grid_dep_wait();
            grid_dep_launch();
            for (int it = 0; it < pre; ++it) {
                const int2 IJ = sIJ[it];
                unsigned char *base = sm + (size_t)it * sbytes;
                if (DBL) tc::bulk_g2s(base + wbytes, a.Yd + (size_t)IJ.x * a.Ykt * 2 * T, ibytes, &full[it]);
                else tc::bulk_g2s(base + wbytes, a.Y + (size_t)IJ.x * a.Ykt * T, ibytes, &full[it]);
                tc::bulk_g2s(base + wbytes + ibytes, a.Y + (size_t)IJ.y * a.Ykt * T, jbytes, &full[it]);
            }
            int issued = pre;
            bool marked = false;
            // Tiles after the first `stages`: with programmatic launch they
            // are claimed from a counter (some blocks start late); otherwise
            // block b takes b + it * gridDim.x.  Either way the next tile and
            // its coordinates are fetched one step ahead of their use.
            const int t0 = gridDim.x * S;
            auto next_tile = [&](int it) -> int {
                if (a.pdl) return t0 < a.ntiles ? t0 + (int)atomicAdd(&a.st->tile_next, 1u) : a.ntiles;
                return (int)blockIdx.x + it * (int)gridDim.x;
            };
            int tnext = next_tile(pre);
            int2 IJnext = tnext < a.ntiles ? a.wtiles[tnext] : make_int2(-1, -1);
            if (tnext < a.ntiles && !SAP_BOUNDS_OK(a.st, IJnext.x >= 0 && IJnext.x <= IJnext.y && IJnext.y < a.Npad / T))
                IJnext = make_int2(0, 0);
            for (int it = pre;; ++it) {
                const int s = it % S;
                const int t = tnext;
                const int2 IJ = IJnext;
                if (t < a.ntiles) {
                    tnext = next_tile(it + 1);
                    IJnext = tnext < a.ntiles ? a.wtiles[tnext] : make_int2(-1, -1);
                    if (tnext < a.ntiles &&
                        !SAP_BOUNDS_OK(a.st, IJnext.x >= 0 && IJnext.x <= IJnext.y && IJnext.y < a.Npad / T))
                        IJnext = make_int2(0, 0);
                }
                if (it >= S && !tc::mbar_wait_bounded(&empty[s], ((it / S) - 1) & 1, budget)) {
                    atomicOr(&a.st->status, ST_TIMEOUT);
                    break;
                }
                if (t >= a.ntiles) {
                    // no tile left: an arrival without bytes tells the consumers
                    sIJ[s] = make_int2(-1, -1);
                    tc::mbar_arrive(&full[s]);
                    marked = true;
                    break;
                }
                sIJ[s] = IJ;  // published by the mbarrier completion below
                unsigned char *base = sm + (size_t)s * sbytes;
                tc::mbar_expect_tx(&full[s], sbytes);
                tc::bulk_g2s(base, a.wb + (size_t)t * T * T, wbytes, &full[s]);
                // one copy per side: the basis's components of the point block
                if (DBL) tc::bulk_g2s(base + wbytes, a.Yd + (size_t)IJ.x * a.Ykt * 2 * T, ibytes, &full[s]);
                else tc::bulk_g2s(base + wbytes, a.Y + (size_t)IJ.x * a.Ykt * T, ibytes, &full[s]);
                tc::bulk_g2s(base + wbytes + ibytes, a.Y + (size_t)IJ.y * a.Ykt * T, jbytes, &full[s]);
                tc::bulk_g2s(base + wbytes + ibytes + jbytes, a.nu + (size_t)IJ.x * T, T * 4, &full[s]);
                tc::bulk_g2s(base + wbytes + ibytes + jbytes + T * 4, a.nu + (size_t)IJ.y * T, T * 4, &full[s]);
                ++issued;
            }
            // no copy of ours may still be in flight when the block exits
            // (the stage the end marker reused was consumed, so its copies
            // have landed; its barrier is past that phase)
            for (int it = issued > S ? issued - S : 0; it < issued; ++it)
                if (!(marked && it % S == issued % S)) tc::mbar_wait_bounded(&full[it % S], (it / S) & 1, budget);
        } else {
            grid_dep_wait();
            grid_dep_launch();
        }
        return;
    }

    // ---------------- consumer warps ----------------
    grid_dep_wait();  // Y, the bounds and the lists of this iteration
    grid_dep_launch();
    const int seg = warp % SR, row0 = warp / SR;
    const int col0 = seg * 32 * CPT + lane * CPT;
    const float seed = load_pos_float(&a.st->seed_ub);
    float uwarp = INFINITY;  // best upper bound this warp has produced
    // second tier inside the pass: EX pairs per warp and round; the pairs
    // that survive it are evaluated in FP64 later (this warp's best)
    constexpr int EX = (K + 1) * 2 <= 32 ? 2 : 1;
    Partial best = {INFINITY, 0x7fffffff, 0x7fffffff};
    int nd = 0;  // deferred survivors of this warp (warp-uniform)
    auto fp64_pair = [&](int2 ij) {
        if constexpr (EXPL) {
            if (!SAP_PAIR_OK(a.st, ij, a.N)) return;
            if (lane == 0) atomicAdd((unsigned int *)&a.st->cnt2, 1u);
            // FP64: |D|^2 and U^T D with D = x_i - x_j (the FP64 recheck's sums)
            // (the FP64 recheck's compute width for this k, so its sums
            // are the same in the same order: the same q = r^2 bits)
            constexpr int KS = K <= 8 ? K : K <= 12 ? 12 : K <= 16 ? 16 : K <= 24 ? 24 : 32;
            double v[KS + 1];
#pragma unroll
            for (int q = 0; q <= KS; ++q) v[q] = 0.0;
#pragma unroll 4
            for (int l = lane; l < a.n; l += 32) {
                const double D = (double)__ldg(a.X + (size_t)ij.x * a.n + l) - (double)__ldg(a.X + (size_t)ij.y * a.n + l);
                v[KS] = fma(D, D, v[KS]);
#pragma unroll
                for (int c = 0; c < KS; ++c)
                    if (c < a.k) v[c] = fma(__ldg(a.U64 + (size_t)c * a.n + l), D, v[c]);
            }
            double zz, d2;
            warp_ratio_parts<KS>(v, lane, zz, d2);
            if (d2 == 0.0 || d2 < a.eps2) return;
            const double q = zz / d2;
            if (better_q(q, ij.x, ij.y, best.r, best.i, best.j)) best = Partial{q, ij.x, ij.y};
        }
    };
    // the bounds from a round's FP32 ratios (lane e < EX: pair e), then its
    // survivors to the warp's deferred list
    auto expl_after = [&](const int2 (&pr)[EX], float rr, int code) {
        if constexpr (EXPL) {
            const float wmin = warp_min(rr);
            // any earlier value of the running bound is a valid (looser) bound
            float U2 = fminf(fminf(seed, uwarp), load_pos_float(&a.st->run_ub2));
            auto tighten = [&](float ub) {
                if (lane == 0 && ub < U2) {
                    atomic_min_pos_float(&a.st->run_ub2, ub);
                    atomic_min_pos_float(&a.st->run_ub1, ub);  // bounds the pass's own emission too
                }
                U2 = fminf(U2, ub);
                uwarp = fminf(uwarp, ub);
            };
            if (wmin < INFINITY) tighten(cert_upper(wmin, a.cert32));
            unsigned int m = __ballot_sync(0xffffffffu, code == 2 || (code == 1 && rr <= cert_emit_threshold(U2, a.cert32)));
            // survivors wait in the warp's list until its tiles are done (the
            // bound is far tighter by then); a full list evaluates at once
            while (m) {
                const int e = __ffs(m) - 1;
                m &= m - 1u;
                const float re = __shfl_sync(0xffffffffu, code == 2 ? -1.f : rr, e);
                if (nd < kDefer) {
                    if (lane == 0) defer[warp][nd] = DeferredPair{pr[e].x, pr[e].y, re};
                    ++nd;
                } else {
                    fp64_pair(pr[e]);
                }
            }
        }
    };
    // the deferred survivors against the bound as it is now
    auto drain = [&]() {
        if constexpr (EXPL) {
            __syncwarp();
            const float U2 = fminf(fminf(seed, uwarp), load_pos_float(&a.st->run_ub2));
            const float th = cert_emit_threshold(U2, a.cert32);
            for (int q = 0; q < nd; ++q) {
                const DeferredPair d = defer[warp][q];
                if (d.r <= th) fp64_pair(make_int2(d.i, d.j));  // r < 0: too short for FP32
            }
            nd = 0;
        }
    };
    auto expl_round = [&](const int2 (&pr)[EX], const bool (&valid)[EX]) {
        if constexpr (EXPL) {
            float rr;
            int code;
            expl32_eval<K, EX>(a.X, a.n, a.U32, a.KP, pr, valid, lane, rr, code);
            expl_after(pr, rr, code);
        }
    };
    if constexpr (EXPL) {
        // the near pairs first, while the first stages' copies land: their
        // bounds tighten the pass's early (survivors wait, see above)
        const long long G = (long long)gridDim.x * kConsumerWarps * EX;
        for (long long base = ((long long)blockIdx.x * kConsumerWarps + warp) * EX; base < a.n_near; base += G) {
            int2 pr[EX];
            bool valid[EX];
#pragma unroll
            for (int e = 0; e < EX; ++e) {
                valid[e] = base + e < a.n_near;
                pr[e] = valid[e] ? __ldcg(a.near + base + e) : make_int2(0, 0);
                if (valid[e] && !SAP_PAIR_OK(a.st, pr[e], a.N)) {
                    valid[e] = false;
                    pr[e] = make_int2(0, 0);
                }
            }
            expl_round(pr, valid);
        }
    }
    // ring position and barrier phase, advanced without integer division
    int s = 0;
    uint32_t phase = 0;
    int tcount = 0;  // tiles this warp has consumed
    for (;; s = (s + 1 == S) ? 0 : s + 1, phase ^= (s == 0) ? 1u : 0u) {
        // a checkpoint part-way: the survivors so far against the bound as it
        // is by then (tight once the minimum's tile has been seen), so their
        // FP64 evaluations overlap the other warps' tiles instead of the tail
        if constexpr (EXPL) {
            if (tcount == kDrainTile && nd) drain();
            ++tcount;
        }
        if (!tc::mbar_wait_bounded(&full[s], phase, budget)) {
            if (lane == 0) atomicOr(&a.st->status, ST_TIMEOUT);
            break;
        }
        const int2 IJ = sIJ[s];
        if (IJ.x < 0) break;  // the producer has no more tiles
        const float gnow = load_pos_float(&a.st->run_ub1);  // consumed after the tile
        const uint16_t *hs = reinterpret_cast<const uint16_t *>(sm + (size_t)s * sbytes);
        // row side: yI[c * T + a], or (DBL) the doubled copy yI[c * 2T + yd_offset(a)]
        const float *yI = reinterpret_cast<const float *>(sm + (size_t)s * sbytes + wbytes);
        const float *yJ = reinterpret_cast<const float *>(sm + (size_t)s * sbytes + wbytes + ibytes);  // yJ[c * T + b]

        float v[RPW][CPT];
        float mymin = INFINITY;
        if (NPR > 0) {
            uint64_t yj2[NPR > 0 ? NPR : 1][K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                if (CPT == 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(yJ + c * T + col0);
                    yj2[0][c] = tc::pk2(t.x, t.y);
                    yj2[NPR > 1 ? 1 : 0][c] = tc::pk2(t.z, t.w);
                } else {
                    const float2 t = *reinterpret_cast<const float2 *>(yJ + c * T + col0);
                    yj2[0][c] = tc::pk2(t.x, t.y);
                }
            }
#pragma unroll
            for (int r0 = 0; r0 < RPW; r0 += 2) {
                uint64_t s2[2][NPR > 0 ? NPR : 1];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int p = 0; p < NPR; ++p) s2[h][p] = 0ull;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    // rows row0 + r0 RSTEP and the next, each as a {y, y} pair (broadcast)
                    uint64_t yya, yyb;
                    if constexpr (DBL) {
                        const ulonglong2 yy = *reinterpret_cast<const ulonglong2 *>(yI + c * 2 * T + row0 * 16 + (r0 >> 1) * 4);
                        yya = yy.x;
                        yyb = yy.y;
                    } else {
                        const float yca = yI[c * T + row0 + r0 * RSTEP];
                        const float ycb = yI[c * T + row0 + (r0 + 1) * RSTEP];
                        yya = tc::pk2(yca, yca);
                        yyb = tc::pk2(ycb, ycb);
                    }
#pragma unroll
                    for (int p = 0; p < NPR; ++p) {
                        const uint64_t ea = tc::sub2(yya, yj2[p][c]);
                        const uint64_t eb = tc::sub2(yyb, yj2[p][c]);
                        s2[0][p] = tc::fma2(ea, ea, s2[0][p]);
                        s2[1][p] = tc::fma2(eb, eb, s2[1][p]);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = r0 + h;
                    const uint16_t *hr = hs + (row0 + r * RSTEP) * T + col0;
                    float wv[CPT];  // 1/d^2 of the thread's columns
                    if (CPT == 4) {
                        const uint2 raw = *reinterpret_cast<const uint2 *>(hr);
                        wv[0] = bf16_lo(raw.x); wv[1 % CPT] = bf16_hi(raw.x);
                        wv[2 % CPT] = bf16_lo(raw.y); wv[3 % CPT] = bf16_hi(raw.y);
                    } else {
                        const uint32_t raw = *reinterpret_cast<const uint32_t *>(hr);
                        wv[0] = bf16_lo(raw); wv[1 % CPT] = bf16_hi(raw);
                    }
#pragma unroll
                    for (int p = 0; p < NPR; ++p) {
                        const uint64_t ww = tc::pk2(wv[2 * p], wv[(2 * p + 1) % CPT]);
                        const float2 q = tc::upk2(tc::mul2(s2[h][p], ww));
                        v[r][(2 * p) % CPT] = q.x;
                        v[r][(2 * p + 1) % CPT] = q.y;
                        mymin = fminf(mymin, fminf(q.x, q.y));
                    }
                }
            }
        } else {
            float yj[K];
#pragma unroll
            for (int c = 0; c < K; ++c) yj[c] = yJ[c * T + col0];
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
                const int row = row0 + r * RSTEP;
                float sacc = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float e = yI[c * T + row] - yj[c];
                    sacc = fmaf(e, e, sacc);
                }
                v[r][0] = sacc * bf16_at(hs + row * T + col0);
                mymin = fminf(mymin, v[r][0]);
            }
        }
        float U = fminf(fminf(seed, gnow), uwarp);
        float thc = cert_emit_threshold(U, a.cert);
        float thc2 = thc * thc * 1.000001f;
        // thc >= U, so a tile that could tighten the bound (minimum below
        // U^2) also fails this test: the fast path needs no warp minimum
        if (!__any_sync(0xffffffffu, mymin <= thc2)) {
            // fast path: nothing in this tile can bound or be the minimum
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
            continue;
        }
        const float wmin = warp_min(mymin);
        const bool refine = wmin < INFINITY && sqrtf(wmin) < U;  // warp-uniform
        const float *nuI = reinterpret_cast<const float *>(sm + (size_t)s * sbytes + wbytes + ibytes + jbytes);
        const float *nuJ = nuI + T;
        if (refine) {
            // the bound of the tile's minimum from that pair's own error
            const int src = __ffs(__ballot_sync(0xffffffffu, mymin == wmin)) - 1;
            float ub = 0.f;
            if (lane == src) {
                int prow = row0, pcol = col0;
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int q = 0; q < CPT; ++q)
                        if (v[r][q] == wmin) { prow = row0 + r * RSTEP; pcol = col0 + q; }
                const float b = pair_bound(a.beta, nuI[prow], nuJ[pcol], bf16_at(hs + prow * T + pcol));
                ub = (sqrtf(wmin) + b) / (1.0f - a.cert.rho) * 1.000001f;
            }
            ub = __shfl_sync(0xffffffffu, ub, src);
            if (lane == 0 && ub < gnow) atomic_min_pos_float(&a.st->run_ub1, ub);
            U = fminf(U, ub);
            uwarp = fminf(uwarp, ub);
            thc = cert_emit_threshold(U, a.cert);
            thc2 = thc * thc * 1.000001f;
        }
        // emission: the uniform test, then each survivor against its own bound
        const float ut = U * (1.0f + a.cert.rho);
        uint32_t emit = 0u;
        int cnt = 0;
        if (mymin <= thc2)
#pragma unroll
            for (int r = 0; r < RPW; ++r)
#pragma unroll
                for (int q = 0; q < CPT; ++q)
                    if (v[r][q] <= thc2) {
                        const int prow = row0 + r * RSTEP, pcol = col0 + q;
                        const float th = (ut + pair_bound(a.beta, nuI[prow], nuJ[pcol], bf16_at(hs + prow * T + pcol))) *
                                         1.000001f;
                        if (v[r][q] <= th * th * 1.000001f) {
                            emit |= 1u << (r * CPT + q);
                            ++cnt;
                        }
                    }
        // the warp's reads of stage s are done
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[s]);
        if constexpr (EXPL) {
            const int total = __reduce_add_sync(0xffffffffu, cnt);
            if (total == 0) continue;
            if (lane == 0) atomicAdd((unsigned int *)&a.st->cnt1, (unsigned int)total);
            // the emitted pairs, EX per round: each round takes the lowest
            // pending pair of each of the first EX lanes that have one
            const int i0 = IJ.x * T, j0 = IJ.y * T;
            uint32_t rem = emit;
            for (;;) {
                unsigned int has = __ballot_sync(0xffffffffu, rem != 0u);
                if (!has) break;
                const int bit = rem ? __ffs(rem) - 1 : 0;
                const int pi = i0 + row0 + (bit / CPT) * RSTEP, pj = j0 + col0 + bit % CPT;
                int2 pr[EX];
                bool valid[EX];
#pragma unroll
                for (int e = 0; e < EX; ++e) {
                    const int src = has ? __ffs(has) - 1 : 0;
                    valid[e] = has != 0u;
                    pr[e].x = __shfl_sync(0xffffffffu, pi, src);
                    pr[e].y = __shfl_sync(0xffffffffu, pj, src);
                    if (!valid[e]) pr[e] = make_int2(0, 0);
                    if (has && lane == src) rem &= rem - 1u;
                    has &= has - 1u;
                }
                expl_round(pr, valid);
            }
            continue;
        }
        if (__any_sync(0xffffffffu, cnt > 0)) {
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            unsigned int base = 0;
            if (lane == 31) base = atomicAdd((unsigned int *)&a.st->cnt1, (unsigned int)total);
            base = __shfl_sync(0xffffffffu, base, 31);
            if (cnt) {
                long long pos = (long long)base + incl - cnt;
                const int i0 = IJ.x * T, j0 = IJ.y * T;
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int q = 0; q < CPT; ++q)
                        if (emit >> (r * CPT + q) & 1u) {
                            if (pos < a.cap) a.cand[pos] = make_int2(i0 + row0 + r * RSTEP, j0 + col0 + q);
                            else atomicOr(&a.st->status, ST_OVERFLOW);
                            ++pos;
                        }
            }
        }
    }
    if constexpr (EXPL) {
        drain();
        // the block's best pair: the last consumer warp to finish merges
        if (lane == 0) {
            pbest[warp] = best;
            __threadfence_block();
            if (atomicAdd(&pdone, 1u) == kConsumerWarps - 1) {
                __threadfence_block();
                const volatile Partial *vb = pbest;
                Partial b = {vb[0].r, vb[0].i, vb[0].j};
                for (int w2 = 1; w2 < kConsumerWarps; ++w2)
                    if (better_q(vb[w2].r, vb[w2].i, vb[w2].j, b.r, b.i, b.j)) b = Partial{vb[w2].r, vb[w2].i, vb[w2].j};
                a.partials[blockIdx.x] = b;
            }
        }
    }
}

// ------------------------------------------- explicit-difference recheck ---

struct ExplArgs {
    const float *X;
    int N, n;
    const float *U32;  // n x KP
    const float *U32lo;  // n x KP, fl(U64 - U32) (extended-precision variant)
    int k, KP;
    const int2 *cand1;
    unsigned int cap1;
    const int2 *near;
    int n_near;
    Cert cert;
    ProbState *st;
    int2 *cand2;
    long long cap2;
    int pdl;
    int pack;          // extended-precision kernel: write cand2 as packed (i, j, ratio) entries
};

constexpr int EPW = 4;  // entries per warp per round

// Re-evaluates the pass's candidates and the near pairs from explicit FP32
// differences (error model of plain.cu), one warp per pair, and emits the
// pairs that can still be the argmin for the FP64 tier.  A warp handles EPW
// pairs per round with their loads interleaved, so a round costs one memory
// latency; the EPW*(K+1) warp sums are reduced together.  K is the compute
// width (k, or k rounded up; U32's pad columns are zero).
template <int K>
__global__ void __launch_bounds__(256) explicit_recheck_kernel(ExplArgs a)
{
    constexpr int KU = (K + 3) / 4 * 4;
    __shared__ float red[32];
    __shared__ int scan[33];
    __shared__ int base_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // The near list is fixed and the basis and bounds are the previous
    // iteration's (complete once this kernel runs): it is evaluated while the
    // pass may still be running.  The pass's candidates follow its end.
    // With programmatic launch the lists are two segments (the near list
    // first, while the pass may still run; then, after the wait, the pass's
    // candidates); otherwise one segment covering both.
    const float seed = load_pos_float(&a.st->seed_ub);
    for (int seg = 0; seg < (a.pdl ? 2 : 1); ++seg) {
    long long nn = a.n_near, total = a.n_near, lim = a.n_near;
    if (seg == 1 || !a.pdl) {
        grid_dep_wait();
        grid_dep_launch();
        unsigned int c1 = *(volatile const unsigned int *)&a.st->cnt1;
        if (c1 > a.cap1) c1 = a.cap1;
        nn = a.pdl ? 0 : a.n_near;
        total = nn + c1;
        lim = nn + a.cap1;  // bound of the lists' storage
    }
    // A round's pairs are read up to the lists' storage bound before the
    // count is needed (entries past the count are read but not used), so the
    // count's load and the pairs' loads overlap.
    for (long long base = (long long)blockIdx.x * 8 * EPW; base < lim;
         base += (long long)gridDim.x * 8 * EPW) {
        int2 pr[EPW];
        bool valid[EPW];
#pragma unroll
        for (int e = 0; e < EPW; ++e) {
            const long long idx = base + warp * EPW + e;
            pr[e] = idx < lim ? (idx < nn ? __ldcg(a.near + idx) : __ldcg(a.cand1 + (idx - nn))) : make_int2(0, 0);
        }
        if (base >= total) break;  // uniform over the block
#pragma unroll
        for (int e = 0; e < EPW; ++e) {
            valid[e] = base + warp * EPW + e < total && SAP_PAIR_OK(a.st, pr[e], a.N);
            if (!valid[e]) pr[e] = make_int2(0, 0);
        }
        // any earlier value of the running bound is a valid (looser) bound:
        // read it now, so its latency overlaps the loads below
        const float ub2 = load_pos_float(&a.st->run_ub2);
        float acc[EPW * (K + 1)];
#pragma unroll
        for (int q = 0; q < EPW * (K + 1); ++q) acc[q] = 0.f;
#pragma unroll 2
        for (int l = lane; l < a.n; l += 32) {
            float u[KU];
#pragma unroll
            for (int c = 0; c < KU; c += 4) {
                const float4 t = __ldcg(reinterpret_cast<const float4 *>(a.U32 + (size_t)l * a.KP + c));
                u[c] = t.x; u[c + 1] = t.y; u[c + 2] = t.z; u[c + 3] = t.w;
            }
#pragma unroll
            for (int e = 0; e < EPW; ++e) {
                const float D = a.X[(size_t)pr[e].x * a.n + l] - a.X[(size_t)pr[e].y * a.n + l];
                acc[e * (K + 1) + K] = fmaf(D, D, acc[e * (K + 1) + K]);
#pragma unroll
                for (int c = 0; c < K; ++c) acc[e * (K + 1) + c] = fmaf(u[c], D, acc[e * (K + 1) + c]);
            }
        }
        // lane e < EPW finishes entry e: |D|^2 in z[K], U^T D in z[0..K-1]
        float z[K + 1];
        constexpr int M = EPW * (K + 1);
        if constexpr (M <= 32) {
            // reduce-scatter (M - 1 + a few shuffles instead of 5 M), then
            // each finishing lane gathers its entry's K + 1 totals
            constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
            constexpr int dup = 32 / S;  // lanes holding the same total
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
        const float bmin = block_min(rr, red);
        float U = fminf(seed, ub2);
        if (bmin < INFINITY) {
            const float ub = cert_upper(bmin, a.cert);
            if (threadIdx.x == 0) atomic_min_pos_float(&a.st->run_ub2, ub);
            U = fminf(U, ub);
        }
        const float th = cert_emit_threshold(U, a.cert);
        const int cnt = (code == 2 || (code == 1 && rr <= th)) ? 1 : 0;
        int tot;
        const int off = block_exclusive_scan(cnt, scan, &tot);
        if (tot == 0) continue;
        if (threadIdx.x == 0) base_sh = (int)atomicAdd((unsigned int *)&a.st->cnt2, (unsigned int)tot);
        __syncthreads();
        if (cnt) {
            const long long pos = (long long)(unsigned int)base_sh + off;
            if (pos < a.cap2) a.cand2[pos] = mypr;
            else atomicOr(&a.st->status, ST_OVERFLOW);
        }
        __syncthreads();
    }
    }
}

// ---- extended-precision explicit recheck (large n; helpers in sap_internal.cuh)

// The same tier for large n, where the FP32 dot products' certified error
// (gamma_{n+3}) would pass too many pairs on: D = fl(x_i - x_j) in FP32, then
// |D|^2 and U^T D accumulated as hi + lo FP32 pairs with error-free products
// against the hi + lo FP32 basis.  Since U is orthonormal, the rounding of D
// moves U^T D by at most 2^-24 d and d by 2^-24 d, so |r~ - r| <= 2^-24 +
// 2 * 2^-24 r plus the final FP32 roundings (cert_explicit_df).  One warp per
// pair, K + 1 extended accumulators per lane.
template <int K>
__global__ void __launch_bounds__(256) explicit_df_kernel(ExplArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // pairs per warp and round: as many as the reduce-scatter holds
    constexpr int E = (K + 1) <= 8 ? 4 : (K + 1) <= 16 ? 2 : 1;
    // near list first (while the pass may still run), then the pass's candidates
    const float seed = load_pos_float(&a.st->seed_ub);
    for (int seg = 0; seg < (a.pdl ? 2 : 1); ++seg) {
    long long nn = a.n_near, total = a.n_near;
    if (seg == 1 || !a.pdl) {
        grid_dep_wait();
        grid_dep_launch();
        unsigned int c1 = *(volatile const unsigned int *)&a.st->cnt1;
        if (c1 > a.cap1) c1 = a.cap1;
        nn = a.pdl ? 0 : a.n_near;
        total = nn + c1;
    }
    for (long long base = ((long long)blockIdx.x * 8 + warp) * E; base < total; base += (long long)gridDim.x * 8 * E) {
        int2 pr[E];
        bool valid[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long idx = base + e;
            valid[e] = idx < total;
            pr[e] = valid[e] ? (idx < nn ? __ldcg(a.near + idx) : __ldcg(a.cand1 + (idx - nn))) : make_int2(0, 0);
            if (valid[e] && !SAP_PAIR_OK(a.st, pr[e], a.N)) {
                valid[e] = false;
                pr[e] = make_int2(0, 0);
            }
        }
        // any earlier value of the running bound is a valid (looser) bound
        const float ub2 = load_pos_float(&a.st->run_ub2);
        float rr;
        int code;
        if constexpr ((K + 1) * E <= 32) {
            df_eval<K, E>(a.X, a.n, a.U32, a.U32lo, a.KP, pr, valid, lane, rr, code);
        } else {
            // k = 32: K + 1 sums per pair, one pair per warp, butterfly sums
            float zh[K + 1], zl[K + 1];
#pragma unroll
            for (int q = 0; q <= K; ++q) zh[q] = zl[q] = 0.f;
            if (valid[0]) {
#pragma unroll 2
                for (int l = lane; l < a.n; l += 32) {
                    const float D = a.X[(size_t)pr[0].x * a.n + l] - a.X[(size_t)pr[0].y * a.n + l];
                    xs_fma(zh[K], zl[K], D, D, 0.f);
                    const float *uh = a.U32 + (size_t)l * a.KP, *ul = a.U32lo + (size_t)l * a.KP;
#pragma unroll
                    for (int c = 0; c < K; ++c) xs_fma(zh[c], zl[c], D, __ldcg(uh + c), __ldcg(ul + c));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q <= K; ++q) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, zh[q], o);
                    const float l2 = __shfl_xor_sync(0xffffffffu, zl[q], o);
                    float s, e;
                    xs_two_sum(zh[q], h2, s, e);
                    zh[q] = s;
                    zl[q] = __fadd_rn(zl[q], __fadd_rn(l2, e));
                }
            const float dd = zh[K] + zl[K];
            float zz = 0.f;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float z = zh[c] + zl[c];
                zz = fmaf(z, z, zz);
            }
            code = (lane != 0 || !valid[0]) ? 0 : (dd < 1e-30f ? 2 : 1);  // 2: too short for FP32
            rr = code == 1 ? sqrtf(zz / dd) : INFINITY;
        }
        const float wmin = warp_min(rr);
        float U = fminf(seed, ub2);
        if (wmin < INFINITY) {
            const float ub = cert_upper(wmin, a.cert);
            if (lane == 0 && ub < ub2) atomic_min_pos_float(&a.st->run_ub2, ub);
            U = fminf(U, ub);
        }
        const float th = cert_emit_threshold(U, a.cert);
        const bool emit = code == 2 || (code == 1 && rr <= th);
        const unsigned int m = __ballot_sync(0xffffffffu, emit);
        if (!m) continue;
        unsigned int b0 = 0;
        if (lane == 0) b0 = atomicAdd((unsigned int *)&a.st->cnt2, (unsigned int)__popc(m));
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        int2 mp = pr[0];
#pragma unroll
        for (int e = 1; e < E; ++e)
            if (lane == e) mp = pr[e];
        if (emit) {
            const long long pos = (long long)b0 + __popc(m & ((1u << lane) - 1u));
            if (pos < a.cap2) {
                if (a.pack) reinterpret_cast<unsigned long long *>(a.cand2)[pos] = pack_cand(mp.x, mp.y, rr, code == 2);
                else a.cand2[pos] = mp;
            } else {
                atomicOr(&a.st->status, ST_OVERFLOW);
            }
        }
    }
    }
}

template <int K>
cudaError_t launch_expl_k(const ExplArgs &x, bool df, int grid, cudaStream_t s)
{
    if (df) return launch_pdl(x.pdl != 0, explicit_df_kernel<K>, dim3(grid), dim3(256), 0, s, x);
    return launch_pdl(x.pdl != 0, explicit_recheck_kernel<K>, dim3(grid), dim3(256), 0, s, x);
}

cudaError_t launch_explicit(const ExplArgs &x, bool df, int grid, cudaStream_t s)
{
    switch (x.k) {
    case 1: return launch_expl_k<1>(x, df, grid, s);
    case 2: return launch_expl_k<2>(x, df, grid, s);
    case 3: return launch_expl_k<3>(x, df, grid, s);
    case 4: return launch_expl_k<4>(x, df, grid, s);
    case 5: return launch_expl_k<5>(x, df, grid, s);
    case 6: return launch_expl_k<6>(x, df, grid, s);
    case 7: return launch_expl_k<7>(x, df, grid, s);
    case 8: return launch_expl_k<8>(x, df, grid, s);
    default: break;
    }
    if (x.k <= 12) return launch_expl_k<12>(x, df, grid, s);
    if (x.k <= 16) return launch_expl_k<16>(x, df, grid, s);
    if (x.k <= 24) return launch_expl_k<24>(x, df, grid, s);
    return launch_expl_k<32>(x, df, grid, s);
}

// ------------------------------------------ the double-float refine tier ---
//
// Y is formed a second time per iteration in double-float arithmetic: every
// entry an unevaluated sum hi + lo of two FP32 numbers, from the exact FP32
// points (not centred: centring in FP32 would round the differences this
// tier exists to resolve) and the basis split as U32 + U32lo.  Each step is
// an error-free product x * uh (FMA residual), an error-free sum into hi, the
// small terms added to lo, and a renormalisation (|lo| <= ulp(hi)/2), so a
// step adds at most 9 * 2^-48 * S to the error, S = sum_l |x_l||u_l| <=
// ||x|| (u a unit vector); the split residual of u adds 2^-48 S and the five
// five lane merges 20 * 2^-48 S.  Hence |y~_c - y_c| <= eps_df ||x_i|| with
// eps_df = 1.25 (9n + 60) 2^-48 (about 4e-12 at n = 100).
//
// The refine tier evaluates every candidate of the pass and every near pair
// from these rows, one thread per pair, O(k) work: z_c = (yh_i - yh_j) +
// (yl_i - yl_j) (relative FP32 roundings only), r~ = |z| sqrt(w_ij) with the
// stored 1/d^2 (near pairs keep theirs in near_w).  Certified error
// |r~ - r| <= A_p + rho r, A_p = sqrt(k) (eps_df + 2^-46)(||x_i|| + ||x_j||)
// sqrt(w_ij): at least a thousand times below the pass's bound, and below the
// FP32 rounding of explicit differences x_i - x_j.  Emission as in every
// tier: r~_p <= U (1 + rho) + A_p against the running upper bound U.

double df_error_unit(int n)
{
    return 1.25 * (9.0 * n + 60.0) * std::ldexp(1.0, -48);
}

__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x * (uh + ul), then renormalised.  The _rn intrinsics keep the
// compiler from fusing the error-free steps into FMAs.
__device__ __forceinline__ void df_step(float &hi, float &lo, float x, float uh, float ul)
{
    const float p = __fmul_rn(x, uh);
    const float pe = fmaf(x, uh, -p);
    float s, e;
    df_two_sum(hi, p, s, e);
    const float l = __fadd_rn(lo, __fadd_rn(e, fmaf(x, ul, pe)));
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}
struct YdfArgs {
    const float *X;          // N x n row-major FP32
    int N, n;
    const float *U32, *U32lo;  // n x KP: hi and lo parts of the basis
    int KP;
    int Npad;
    float *Yh, *Yl;          // KY x Npad each, component-major; rows >= N zero
    int KY;
};

__device__ __forceinline__ void df_merge_norm(float &hi, float &lo, float h2, float l2)
{
    float s, e;
    df_two_sum(hi, h2, s, e);
    const float l = __fadd_rn(lo, __fadd_rn(l2, e));
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// A block of 16 warps computes 32 rows at a time, two per warp; the lanes of
// a warp split the coordinates (l = lane, lane + 32, ...), and their partial
// sums are merged by a 5-level shuffle tree at the end (within the error
// allowance above).  The basis goes through shared memory in chunks of CH
// coordinates, component-major (lanes read consecutive words), each chunk
// serving all 32 rows.  K = compute width (U32's pad columns are zero).
constexpr int kYdfWarps = 16;
constexpr int kYdfRpw = 2;

template <int K>
struct YdfShape {
    static constexpr int CH = K <= 8 ? 256 : 128;
};

template <int K>
__global__ void __launch_bounds__(kYdfWarps * 32) ydf_warp_kernel(YdfArgs a)
{
    constexpr int CH = YdfShape<K>::CH;
    __shared__ float us[2 * K][CH];  // [c][l] hi, [K + c][l] lo
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunks = (a.n + CH - 1) / CH;
    for (int rbase = blockIdx.x * (kYdfWarps * kYdfRpw); rbase < a.Npad;
         rbase += gridDim.x * (kYdfWarps * kYdfRpw)) {
        float hi[kYdfRpw][K], lo[kYdfRpw][K];
#pragma unroll
        for (int q = 0; q < kYdfRpw; ++q)
#pragma unroll
            for (int c = 0; c < K; ++c) hi[q][c] = lo[q][c] = 0.f;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int c0 = ch * CH, nc = min(CH, a.n - c0);
            if (nchunks > 1 || rbase == blockIdx.x * (kYdfWarps * kYdfRpw)) {
                __syncthreads();
                for (int idx = threadIdx.x; idx < K * CH; idx += kYdfWarps * 32) {
                    const int c = idx / CH, l = idx % CH;
                    const bool in = l < nc;
                    us[c][l] = in ? a.U32[(size_t)(c0 + l) * a.KP + c] : 0.f;
                    us[K + c][l] = in ? a.U32lo[(size_t)(c0 + l) * a.KP + c] : 0.f;
                }
                __syncthreads();
            }
#pragma unroll
            for (int q = 0; q < kYdfRpw; ++q) {
                const int row = rbase + warp * kYdfRpw + q;
                if (row >= a.N) continue;
                const float *xr = a.X + (size_t)row * a.n + c0;
#pragma unroll 2
                for (int l = lane; l < nc; l += 32) {
                    const float x = xr[l];
#pragma unroll
                    for (int c = 0; c < K; ++c) df_step(hi[q][c], lo[q][c], x, us[c][l], us[K + c][l]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kYdfRpw; ++q) {
            const int row = rbase + warp * kYdfRpw + q;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, hi[q][c], o);
                    const float l2 = __shfl_xor_sync(0xffffffffu, lo[q][c], o);
                    df_merge_norm(hi[q][c], lo[q][c], h2, l2);
                }
            if (row < a.Npad)
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (lane == c % 32 && c < a.KY) {
                        a.Yh[(size_t)c * a.Npad + row] = hi[q][c];
                        a.Yl[(size_t)c * a.Npad + row] = lo[q][c];
                    }
        }
    }
}

struct RefineArgs {
    const float *Yh, *Yl;    // double-float Y, KY x Npad each
    int Npad;
    const float *w;          // stored 1/d^2, tile-major upper triangle
    int nb;                  // point blocks per side (Npad / 128)
    long long tile0;         // global index of the first stored tile
    long long nwt;           // stored tiles (index checks of the debug build)
    const float *xn;         // ||x_i||, rounded up
    float beta;              // sqrt(k) (eps_df + 2^-46), rounded up
    const int2 *cand1;
    unsigned int cap1;
    const int2 *near;
    const float *near_w;     // 1/d^2 of the near pairs (+inf: too short for FP32)
    int n_near;
    Cert cert;               // rho (A unused: each pair has its own bound)
    ProbState *st;
    int2 *cand2;
    long long cap2;
    int pdl;
};

// One thread per pair; K = compute width (Y's pad components are zero).
// Warps aggregate their bound and their emissions (one atomic each).
template <int K>
__global__ void __launch_bounds__(256) refine_kernel(RefineArgs a)
{
    const int lane = threadIdx.x & 31;
    const float seed = load_pos_float(&a.st->seed_ub);
    const float rho = a.cert.rho;
    // With programmatic launch the near list is evaluated first (it needs
    // only the previous iteration's results), the pass's candidates after
    // the wait; otherwise one range covers both.
    for (int seg = 0; seg < (a.pdl ? 2 : 1); ++seg) {
        long long nn = a.n_near, total = a.n_near;
        if (seg == 1 || !a.pdl) {
            grid_dep_wait();
            grid_dep_launch();
            unsigned int c1 = *(volatile const unsigned int *)&a.st->cnt1;
            if (c1 > a.cap1) c1 = a.cap1;
            nn = a.pdl ? 0 : a.n_near;
            total = nn + c1;
        }
        const long long stride = (long long)gridDim.x * blockDim.x;
        // rounds are warp-uniform: every lane of a warp runs the same count
        for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
             base += stride) {
            const long long idx = base + lane;
            const float Uround = fminf(seed, load_pos_float(&a.st->run_ub2));  // issued early
            int code = 0;  // 0 none, 1 evaluated, 2 too short for FP32 (always emitted)
            int2 pr = make_int2(0, 0);
            float r = INFINITY, bnd = 0.f;
            if (idx < total) {
                float wv = INFINITY;
                bool ok;
                if (idx < nn) {
                    pr = __ldcg(a.near + idx);
                    ok = SAP_BOUNDS_OK(a.st, pr.x >= 0 && pr.x < pr.y && pr.y < a.Npad);
                    wv = __ldcg(a.near_w + idx);
                } else {
                    pr = __ldcg(a.cand1 + (idx - nn));
                    const int I = pr.x >> 7, J = pr.y >> 7;
                    const long long t = (long long)I * a.nb - (long long)I * (I - 1) / 2 + (J - I) - a.tile0;
                    ok = SAP_BOUNDS_OK(a.st, pr.x >= 0 && pr.x < pr.y && pr.y < a.Npad && t >= 0 && t < a.nwt);
                    if (ok) wv = __ldg(a.w + t * (T * T) + (pr.x & (T - 1)) * T + (pr.y & (T - 1)));
                }
                if (!ok) {
                    pr = make_int2(0, 0);  // skipped (code 0)
                } else if (!(wv < INFINITY)) {
                    code = 2;
                } else {
                    float zz = 0.f;
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const size_t oi = (size_t)c * a.Npad + pr.x, oj = (size_t)c * a.Npad + pr.y;
                        const float z = __fadd_rn(__fsub_rn(__ldcg(a.Yh + oi), __ldcg(a.Yh + oj)),
                                                  __fsub_rn(__ldcg(a.Yl + oi), __ldcg(a.Yl + oj)));
                        zz = fmaf(z, z, zz);
                    }
                    const float sw = sqrtf(wv);
                    r = sqrtf(zz * wv);
                    bnd = a.beta * (__ldg(a.xn + pr.x) + __ldg(a.xn + pr.y)) * sw * 1.000002f;
                    code = 1;
                }
            }
            // the warp's best upper bound tightens the running bound
            const float ub = code == 1 ? (r + bnd) / (1.0f - rho) * 1.000001f : INFINITY;
            const float wub = warp_min(ub);
            float U = Uround;
            if (wub < U) {
                if (lane == 0) atomic_min_pos_float(&a.st->run_ub2, wub);
                U = wub;
            }
            const bool emit = code == 2 || (code == 1 && r <= (U * (1.0f + rho) + bnd) * 1.000001f);
            const unsigned m = __ballot_sync(0xffffffffu, emit);
            if (m) {
                unsigned int b = 0;
                if (lane == 0) b = atomicAdd((unsigned int *)&a.st->cnt2, (unsigned int)__popc(m));
                b = __shfl_sync(0xffffffffu, b, 0);
                if (emit) {
                    const long long pos = (long long)b + __popc(m & ((1u << lane) - 1u));
                    if (pos < a.cap2) a.cand2[pos] = pr;
                    else atomicOr(&a.st->status, ST_OVERFLOW);
                }
            }
        }
    }
}

template <int K>
cudaError_t launch_ydf_refine_k(const YdfArgs &y, const RefineArgs &x, int ygrid, int rgrid, bool ydf,
                                cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (ydf) {
        const int need = (y.Npad + kYdfWarps * kYdfRpw - 1) / (kYdfWarps * kYdfRpw);
        ydf_warp_kernel<K><<<std::min(need, ygrid), kYdfWarps * 32, 0, s>>>(y);
        e = cudaGetLastError();
    } else {
        e = launch_pdl(x.pdl != 0, refine_kernel<K>, dim3(rgrid), dim3(256), 0, s, x);
    }
    return e;
}

// The double-float product (ydf = true) or the refine tier, for width k.
cudaError_t launch_ydf_refine(const YdfArgs &y, const RefineArgs &x, int k, int ygrid, int rgrid, bool ydf,
                              cudaStream_t s)
{
    switch (k) {
    case 1: return launch_ydf_refine_k<1>(y, x, ygrid, rgrid, ydf, s);
    case 2: return launch_ydf_refine_k<2>(y, x, ygrid, rgrid, ydf, s);
    case 3: return launch_ydf_refine_k<3>(y, x, ygrid, rgrid, ydf, s);
    case 4: return launch_ydf_refine_k<4>(y, x, ygrid, rgrid, ydf, s);
    case 5: return launch_ydf_refine_k<5>(y, x, ygrid, rgrid, ydf, s);
    case 6: return launch_ydf_refine_k<6>(y, x, ygrid, rgrid, ydf, s);
    case 7: return launch_ydf_refine_k<7>(y, x, ygrid, rgrid, ydf, s);
    case 8: return launch_ydf_refine_k<8>(y, x, ygrid, rgrid, ydf, s);
    default: break;
    }
    if (k <= 12) return launch_ydf_refine_k<12>(y, x, ygrid, rgrid, ydf, s);
    if (k <= 16) return launch_ydf_refine_k<16>(y, x, ygrid, rgrid, ydf, s);
    if (k <= 24) return launch_ydf_refine_k<24>(y, x, ygrid, rgrid, ydf, s);
    return launch_ydf_refine_k<32>(y, x, ygrid, rgrid, ydf, s);
}

// -------------------------------------------------------------- host side --

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D map of a row-major [outer x inner] 16-bit matrix, box [box_outer x 64]
// with 128-byte swizzling (the K-major operand layout of the product).
bool make_map(CUtensorMap *m, void *base, bool bf16, uint64_t inner, uint64_t outer, uint32_t box_outer)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {64, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// block-major Y ([Npad/128][KY][128]) -> N x k row-major
__global__ void transpose_y_kernel(const float *Yb, int KY, int N, int k, float *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * k) return;
    const int i = e / k, c = e % k;
    out[e] = Yb[(size_t)(i >> 7) * KY * 128 + (size_t)c * 128 + (i & 127)];
}

template <typename T_>
void dfree(T_ *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

#define RCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return handle_fail(h, e_ == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA,  \
                               cudaGetErrorString(e_));                                      \
    } while (0)

// Bound on |y~_c - y_c| per unit ||fl(x - mean)|| (see gemm_tc.cu):
// centring and epilogue roundings, the split residuals and dropped low
// product, the FP32 accumulation chain of the high product within a K slice
// (ceil(NP/(16 ksplit)) MMAs, plus slack for the in-instruction adder
// tree), each accumulation step bounded by 2^-23 (truncation) of twice the
// running magnitude, and the FP32 sum of the slices.  Times 1.25 for margin.
double y_error_unit(int NP, bool bf16, int ksplit)
{
    const double u = std::ldexp(1.0, -24);
    const double split = bf16 ? 3.0 * std::ldexp(1.0, -16) : 3.0 * std::ldexp(1.0, -22);
    const double acc = (std::ceil(NP / (16.0 * ksplit)) + 4.0) * 2.0 * std::ldexp(1.0, -23);
    const double slices = (ksplit - 1) * 2.0 * u;  // FP32 sum of the K slices
    return (3.0 * u + split + acc + slices) * 1.25;
}

// K slices of the product: each slice at least 8 blocks of 64, at most 8
// slices (shorter FP32 accumulation chains for large n).
int pick_ksplit(int nkb) { return std::max(1, std::min(8, nkb / 8)); }

Cert cert_pass(int n, int k, double b_cap)
{
    const double u = std::ldexp(1.0, -24);
    auto g = [&](double m) { return m * u / (1.0 - m * u); };
    Cert c;
    c.A = (float)(b_cap * 1.002);  // >= every stored pair's own bound (FP32 rounding)
    // 2^-9: the BF16 rounding of w = 1/d^2 (halved by the square root); the
    // rest as for explicit differences
    c.rho = (float)((std::ldexp(1.0, -9) + g(n + 2) + g(k) + 8 * u) * 1.05);
    return c;
}

// Extended-precision tier: 2^-24 absolute from the rounding of D (U
// orthonormal), n^1.5 2^-46 from the hi + lo accumulation; relative: the
// rounding of d, the FP32 squares and sum of the k components, the division
// and the square root.

// Explicit tier in extended precision for large n (the FP32 tier's
// gamma_{n+3} bound grows with n).
bool explicit_uses_df(int n) { return n > 256; }

Cert cert_explicit(int n, int k)
{
    const double u = std::ldexp(1.0, -24);
    auto g = [&](double m) { return m * u / (1.0 - m * u); };
    Cert c;
    c.A = (float)(std::sqrt((double)k) * g(n + 3) * 1.05);
    c.rho = (float)((g(n + 2) + g(k) + 3 * u) * 1.05);
    return c;
}

// Refine tier: relative errors only besides each pair's own bound (the
// rounding of the stored length, the FP32 differences, squares and sum of
// the k components, the product with w and the square root).
Cert cert_refine(int n, int k)
{
    const double u = std::ldexp(1.0, -24);
    auto g = [&](double m) { return m * u / (1.0 - m * u); };
    Cert c;
    c.A = 0.f;
    c.rho = (float)((g(n + 2) + g(k + 2) + 8 * u) * 1.05);
    return c;
}

sap_status classify(sap_handle h, int k)
{
    RestrState &r = restr_state(h);
    r.b_cap = handle_tune(h).b_cap;
    cudaStream_t s = handle_stream(h);
    RCK(cudaMemsetAsync(r.counters, 0, 8 * sizeof(unsigned int), s));
    WPrepArgs a;
    a.X = handle_x32(h);
    a.N = (int)handle_n_points(h);
    a.n = handle_n_dim(h);
    a.nu = r.nu;
    a.wtiles = r.wtiles;
    a.w = r.w;
    a.wb = reinterpret_cast<__nv_bfloat16 *>(r.wb);
    a.eps2_lo = handle_eps2_lo(h);
    a.eps2_hi = handle_eps2_hi(h);
    a.eps2 = handle_eps2(h);
    a.beta_coef = (float)(std::sqrt((double)k) * r.y_eps * 1.02);
    a.b_cap = (float)r.b_cap;
    a.near = r.near;
    a.near_w = r.near_w;
    a.near_cap = r.near_cap;
    a.counters = r.counters;
    wprep_kernel<<<r.nwtiles, 256, 0, s>>>(a);
    RCK(cudaGetLastError());
    unsigned int cnt[8];
    RCK(cudaMemcpyAsync(cnt, r.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    if (cnt[2]) return handle_fail(h, SAP_E_UNSUPPORTED, "near-pair list overflow; raise the pass bound");
    r.n_near = (int)cnt[0];
    unsigned long long ex;
    std::memcpy(&ex, &cnt[4], sizeof(ex));
    r.n_excluded = (long long)ex;
    r.k_cls = k;
    return SAP_OK;
}

size_t pass_smem_bytes(int kd, int KY, int stages) { return (size_t)stages * pass_stage_bytes(kd, KY); }

int pass_pick_stages(int k, int KY)
{
    int s = kPassStagesMax;
    while (s > 2 && pass_smem_bytes(pass_kd(k), KY, s) > (size_t)kPassDynSmem) --s;
    return s;
}

// the form with the second tier inside exists for k <= 16
template <int K, int CPT>
cudaError_t launch_pass_k(const PassArgs &a, int grid, cudaStream_t s)
{
    const size_t shm = pass_smem_bytes(CPT == 4 ? K : 0, a.KY, a.stages);
    if constexpr (K <= 16) {
        if (a.X) return launch_pdl(a.pdl != 0, restr_pass_kernel<K, CPT, true>, dim3(grid), dim3(kPassThreads), shm, s, a);
    } else {
        if (a.X) return cudaErrorNotSupported;
    }
    return launch_pdl(a.pdl != 0, restr_pass_kernel<K, CPT, false>, dim3(grid), dim3(kPassThreads), shm, s, a);
}

template <int K, int CPT>
cudaError_t config_pass_k()
{
    cudaError_t e = cudaFuncSetAttribute(restr_pass_kernel<K, CPT, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPassDynSmem);
    if constexpr (K <= 16)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(restr_pass_kernel<K, CPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kPassDynSmem);
    return e;
}

cudaError_t configure_pass_kernels()
{
    cudaError_t e = cudaSuccess;
    auto f = [&](cudaError_t x) { if (x != cudaSuccess) e = x; };
    f(config_pass_k<1, 4>()); f(config_pass_k<2, 4>()); f(config_pass_k<3, 4>()); f(config_pass_k<4, 4>());
    f(config_pass_k<5, 4>()); f(config_pass_k<6, 4>()); f(config_pass_k<7, 4>()); f(config_pass_k<8, 4>());
    f(config_pass_k<10, 4>()); f(config_pass_k<12, 4>()); f(config_pass_k<16, 4>()); f(config_pass_k<24, 1>()); f(config_pass_k<32, 1>());
    return e;
}

cudaError_t launch_pass(const PassArgs &a, int k, int grid, cudaStream_t s)
{
    switch (k) {
    case 1: return launch_pass_k<1, 4>(a, grid, s);
    case 2: return launch_pass_k<2, 4>(a, grid, s);
    case 3: return launch_pass_k<3, 4>(a, grid, s);
    case 4: return launch_pass_k<4, 4>(a, grid, s);
    case 5: return launch_pass_k<5, 4>(a, grid, s);
    case 6: return launch_pass_k<6, 4>(a, grid, s);
    case 7: return launch_pass_k<7, 4>(a, grid, s);
    case 8: return launch_pass_k<8, 4>(a, grid, s);
    default: break;
    }
    if (k <= 10) return launch_pass_k<10, 4>(a, grid, s);
    if (k <= 12) return launch_pass_k<12, 4>(a, grid, s);
    if (k <= 16) return launch_pass_k<16, 4>(a, grid, s);
    if (k <= 24) return launch_pass_k<24, 1>(a, grid, s);
    return launch_pass_k<32, 1>(a, grid, s);
}

} // namespace

sap_status restructured_prepare(sap_handle h)
{
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int N = (int)handle_n_points(h), n = handle_n_dim(h);
    const bool bf16 = handle_split_bf16(h) != 0;
    const float *X = handle_x32(h);
    RCK(cudaStreamSynchronize(s));
    if (!r.center) {
        r.Npad = (N + T - 1) / T * T;
        r.NP = (n + 63) / 64 * 64;
        RCK(cudaMalloc(&r.center, n * sizeof(float)));
        RCK(cudaMalloc(&r.nu, r.Npad * sizeof(float)));
        RCK(cudaMalloc(&r.Xhi, (size_t)r.Npad * r.NP * 2));
        RCK(cudaMalloc(&r.Xlo, (size_t)r.Npad * r.NP * 2));
        RCK(cudaMalloc(&r.counters, 8 * sizeof(unsigned int)));
        const int nb = r.Npad / T;
        long long t0 = 0, t1 = -1;  // a shard stores the tiles [t0, t1) of the row-major order only
        handle_shard(h, &t0, &t1);
        std::vector<int2> t;
        long long g = 0;
        for (int I = 0; I < nb; ++I)
            for (int J = I; J < nb; ++J, ++g)
                if (g >= t0 && (t1 < 0 || g < t1)) t.push_back(make_int2(I, J));
        r.tile0 = t0;
        r.nwtiles = (int)t.size();
        RCK(cudaMalloc(&r.wtiles, t.size() * sizeof(int2)));
        RCK(cudaMemcpy(r.wtiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice));
        RCK(cudaMalloc(&r.w, (size_t)r.nwtiles * T * T * sizeof(float)));
        RCK(cudaMalloc(&r.wb, (size_t)r.nwtiles * T * T * sizeof(uint16_t)));
        const long long P = (long long)N * (N - 1) / 2;
        r.near_cap = (unsigned int)std::min<long long>(P + 64, 1ll << 24);
        RCK(cudaMalloc(&r.near, (size_t)r.near_cap * sizeof(int2)));
        RCK(cudaMalloc(&r.near_w, (size_t)r.near_cap * sizeof(float)));
        RCK(cudaMalloc(&r.xn, r.Npad * sizeof(float)));
        RCK(gemm_configure());
        RCK(configure_pass_kernels());
    }
    const int sms = handle_sms(h);
    colmean_kernel<<<(n + 127) / 128, 128, 0, s>>>(X, N, n, r.center);
    RCK(cudaGetLastError());
    RCK(cudaMemsetAsync(r.counters, 0, 8 * sizeof(unsigned int), s));
    absmax_kernel<<<4 * sms, 256, 0, s>>>(X, (size_t)N * n, n, r.center, r.counters);
    RCK(cudaGetLastError());
    unsigned int mbits = 0;
    RCK(cudaMemcpyAsync(&mbits, r.counters, sizeof(mbits), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    float mx;
    std::memcpy(&mx, &mbits, sizeof(mx));
    int e = 0;
    if (mx > 0.f) e = (int)std::ceil(std::log2((double)mx));
    r.xscale = (float)std::ldexp(1.0, -e);
    const float lo_mul = bf16 ? 256.f : 2048.f;
    if (bf16)
        split_kernel<__nv_bfloat16><<<4 * sms, 256, 0, s>>>(X, N, n, r.center, r.xscale, lo_mul,
                                                          (__nv_bfloat16 *)r.Xhi, (__nv_bfloat16 *)r.Xlo,
                                                          r.Npad, r.NP);
    else
        split_kernel<__half><<<4 * sms, 256, 0, s>>>(X, N, n, r.center, r.xscale, lo_mul, (__half *)r.Xhi,
                                                     (__half *)r.Xlo, r.Npad, r.NP);
    RCK(cudaGetLastError());
    rownorm_kernel<<<(r.Npad + 7) / 8, 256, 0, s>>>(X, N, n, r.center, r.nu, r.Npad);
    RCK(cudaGetLastError());
    xnorm_kernel<<<(r.Npad + 7) / 8, 256, 0, s>>>(X, N, n, r.xn, r.Npad);
    RCK(cudaGetLastError());
    r.ksplit = pick_ksplit(r.NP / 64);
    r.y_eps = y_error_unit(r.NP, bf16, r.ksplit);
    if (!make_map(&r.gemm.ta_hi, r.Xhi, bf16, r.NP, r.Npad, 128) ||
        !make_map(&r.gemm.ta_lo, r.Xlo, bf16, r.NP, r.Npad, 128))
        return handle_fail(h, SAP_E_CUDA, "cuTensorMapEncodeTiled failed for X");
    r.maps_x = true;
    if (r.Uhi) {
        if (!make_map(&r.gemm.tb_hi, r.Uhi, bf16, r.NP, r.KPG, r.KPG) ||
            !make_map(&r.gemm.tb_lo, r.Ulo, bf16, r.NP, r.KPG, r.KPG))
            return handle_fail(h, SAP_E_CUDA, "cuTensorMapEncodeTiled failed for U");
    }
    r.k_cls = 0;
    const int k = handle_k(h);
    if (k > 0) return classify(h, k);
    RCK(cudaStreamSynchronize(s));
    return SAP_OK;
}

sap_status restructured_basis_alloc(sap_handle h)
{
    RestrState &r = restr_state(h);
    const int k = handle_k(h);
    const bool bf16 = handle_split_bf16(h) != 0;
    dfree(r.Uhi);
    dfree(r.Ulo);
    dfree(r.Y);
    dfree(r.Yd);
    dfree(r.Ypart);
    r.KPG = (k + 15) / 16 * 16;
    r.KY = padded_stride(k);   // <= KPG; columns >= k are zero
    RCK(cudaMalloc(&r.Uhi, (size_t)r.KPG * r.NP * 2));
    RCK(cudaMalloc(&r.Ulo, (size_t)r.KPG * r.NP * 2));
    RCK(cudaMalloc(&r.Y, (size_t)r.Npad * r.KY * sizeof(float)));
    RCK(cudaMemset(r.Y, 0, (size_t)r.Npad * r.KY * sizeof(float)));
    RCK(cudaMalloc(&r.Yd, (size_t)r.Npad * r.KY * 2 * sizeof(float)));
    RCK(cudaMemset(r.Yd, 0, (size_t)r.Npad * r.KY * 2 * sizeof(float)));
    dfree(r.Ydh);
    dfree(r.Ydl);
    RCK(cudaMalloc(&r.Ydh, (size_t)r.Npad * r.KY * sizeof(float)));
    RCK(cudaMalloc(&r.Ydl, (size_t)r.Npad * r.KY * sizeof(float)));
    RCK(cudaMemset(r.Ydh, 0, (size_t)r.Npad * r.KY * sizeof(float)));
    RCK(cudaMemset(r.Ydl, 0, (size_t)r.Npad * r.KY * sizeof(float)));
    dfree(r.Ypart);
    if (r.ksplit > 1) RCK(cudaMalloc(&r.Ypart, (size_t)r.ksplit * r.Npad * r.KY * sizeof(float)));
    if (!make_map(&r.gemm.tb_hi, r.Uhi, bf16, r.NP, r.KPG, r.KPG) ||
        !make_map(&r.gemm.tb_lo, r.Ulo, bf16, r.NP, r.KPG, r.KPG))
        return handle_fail(h, SAP_E_CUDA, "cuTensorMapEncodeTiled failed for U");
    r.maps_u = true;
    return SAP_OK;
}

sap_status restructured_upload_basis(sap_handle h, const double *U)
{
    RestrState &r = restr_state(h);
    const int k = handle_k(h);
    std::vector<uint16_t> hi((size_t)r.KPG * r.NP, 0), lo((size_t)r.KPG * r.NP, 0);
    restructured_split_host(h, U, k, hi.data(), lo.data());
    RCK(cudaMemcpy(r.Uhi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice));
    RCK(cudaMemcpy(r.Ulo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice));
    if (r.k_cls != k) return classify(h, k);
    return SAP_OK;
}

sap_status restructured_set_bound(sap_handle h, double b_cap)
{
    handle_tune(h).b_cap = b_cap;
    const int k = handle_k(h);
    if (k > 0) return classify(h, k);
    return SAP_OK;
}

GemmArgs product_args(sap_handle h, const RestrState &r)
{
    GemmArgs g = r.gemm;
    g.Yd = nullptr;
    g.seed_st = nullptr;
    g.Npad = r.Npad;
    g.nkb = r.NP / 64;
    g.ab_bf16 = handle_split_bf16(h);
    g.lo_scale = g.ab_bf16 ? 1.0f / 256.f : 1.0f / 2048.f;
    g.out_scale = 1.0f / r.xscale;
    g.ksplit = r.ksplit;
    g.pdl = handle_tune(h).pdl;
    return g;
}

sap_status restructured_enqueue_product(sap_handle h, const CUtensorMap *mhi, const CUtensorMap *mlo, int KPG,
                                        float *Y, float *Yd, int KY, float *Ypart, ProbState *st, cudaStream_t s,
                                        bool seeds)
{
    RestrState &r = restr_state(h);
    GemmArgs g = product_args(h, r);
    if (seeds) {
        g.seed_X = handle_x32(h);
        g.seed_U = handle_u32(h);
        g.seed_Ulo = handle_u32lo(h);
        g.seed_st = st;
        g.seed_N = (int)handle_n_points(h);
        g.seed_n = handle_n_dim(h);
        g.seed_k = handle_k(h);
        g.seed_KP = handle_kp(h);
    }
    g.tb_hi = *mhi;
    g.tb_lo = *mlo;
    g.Y = Y;
    g.Yd = Yd;
    g.KY = KY;
    g.KPG = KPG;
    g.stages = gemm_pick_stages(KPG, g.nkb);
    g.st = st;
    g.Ypart = Ypart;
    cudaEvent_t ea, eb;
    handle_count_launch(h, 0, &ea, &eb);
    if (ea) cudaEventRecord(ea, s);
    RCK(launch_gemm_y(g, s));
    if (eb) cudaEventRecord(eb, s);
    handle_push_timing(h, 0, ea, eb);
    return SAP_OK;
}

sap_status restructured_enqueue_basis(sap_handle h, const BasisView &b, cudaStream_t s)
{
    RestrState &r = restr_state(h);
    const int n = handle_n_dim(h);
    cudaEvent_t ea, eb;
    const int tier = restructured_tier_for(h, b.k);
    {
        PassArgs p;
        p.wb = r.wb;
        p.wtiles = r.wtiles;
        p.ntiles = r.nwtiles;
        p.Y = b.Y;
        p.Yd = b.Yd;
        p.KY = b.KY;
        p.Ykt = b.Ykt;
        p.Npad = r.Npad;
        p.nu = r.nu;
        p.beta = (float)(std::sqrt((double)b.k) * r.y_eps * 1.02);
        p.stages = pass_pick_stages(b.k, b.KY);
        if (handle_tune(h).pass_stages >= 2) p.stages = std::min(p.stages, handle_tune(h).pass_stages);
        p.cert = cert_pass(n, b.k, r.b_cap);
        p.st = b.st;
        p.cand = b.cand1;
        p.cap = b.cap;
        p.pdl = handle_tune(h).pdl;
        if (tier == 5) {
            p.X = handle_x32(h);
            p.N = (int)handle_n_points(h);
            p.n = n;
            p.U32 = b.U32;
            p.KP = b.KP;
            p.U64 = b.U64;
            p.k = b.k;
            p.eps2 = handle_eps2(h);
            p.near = r.near;
            p.n_near = r.n_near;
            p.partials = b.partials;
            p.cert32 = cert_explicit(n, b.k);
        }
        handle_count_launch(h, 1, &ea, &eb);
        if (ea) cudaEventRecord(ea, s);
        RCK(launch_pass(p, b.k, restructured_pass_grid(h), s));
        if (eb) cudaEventRecord(eb, s);
        handle_push_timing(h, 1, ea, eb);
    }
    if (tier == 2 || tier == 3 || tier == 5) {
        // the explicit tier runs inside the FP64 recheck (restructured_fuse_args)
        // or (5) inside the pass
    } else if (tier == 0 || tier == 4) {
        ExplArgs x;
        x.X = handle_x32(h);
        x.N = (int)handle_n_points(h);
        x.n = n;
        x.U32 = b.U32;
        x.U32lo = b.U32lo;
        x.k = b.k;
        x.KP = b.KP;
        x.cand1 = b.cand1;
        x.cap1 = (unsigned int)b.cap;
        x.near = r.near;
        x.n_near = r.n_near;
        const bool df = tier == 4 || explicit_uses_df(n);
        x.cert = df ? cert_explicit_df(n, b.k) : cert_explicit(n, b.k);
        x.pack = tier == 4;
        x.st = b.st;
        x.cand2 = b.cand2;
        x.cap2 = b.cap;
        x.pdl = handle_tune(h).pdl;
        handle_count_launch(h, 3, &ea, &eb);
        if (ea) cudaEventRecord(ea, s);
        RCK(launch_explicit(x, df, std::max(1, handle_tune(h).expl_per_sm) * handle_sms(h), s));
        if (eb) cudaEventRecord(eb, s);
        handle_push_timing(h, 3, ea, eb);
    } else {
        // double-float Y of this basis, then the refine tier
        YdfArgs y;
        y.X = handle_x32(h);
        y.N = (int)handle_n_points(h);
        y.n = n;
        y.U32 = b.U32;
        y.U32lo = b.U32lo;
        y.KP = b.KP;
        y.Npad = r.Npad;
        y.Yh = b.Ydh;
        y.Yl = b.Ydl;
        y.KY = b.KY;
        RefineArgs x;
        x.Yh = b.Ydh;
        x.Yl = b.Ydl;
        x.Npad = r.Npad;
        x.w = r.w;
        x.nb = r.Npad / T;
        x.tile0 = r.tile0;
        x.nwt = r.nwtiles;
        x.xn = r.xn;
        x.beta = (float)(std::sqrt((double)b.k) * (df_error_unit(n) + std::ldexp(1.0, -46)) * 1.02);
        x.cand1 = b.cand1;
        x.cap1 = (unsigned int)b.cap;
        x.near = r.near;
        x.near_w = r.near_w;
        x.n_near = r.n_near;
        x.cert = cert_refine(n, b.k);
        x.st = b.st;
        x.cand2 = b.cand2;
        x.cap2 = b.cap;
        x.pdl = handle_tune(h).pdl;
        const int sms = handle_sms(h);
        handle_count_launch(h, 4, &ea, &eb);
        if (ea) cudaEventRecord(ea, s);
        RCK(launch_ydf_refine(y, x, b.k, 2 * sms, 0, true, s));
        if (eb) cudaEventRecord(eb, s);
        handle_push_timing(h, 4, ea, eb);
        handle_count_launch(h, 3, &ea, &eb);
        if (ea) cudaEventRecord(ea, s);
        RCK(launch_ydf_refine(y, x, b.k, 0, std::max(1, handle_tune(h).expl_per_sm) * sms, false, s));
        if (eb) cudaEventRecord(eb, s);
        handle_push_timing(h, 3, ea, eb);
    }
    return SAP_OK;
}

sap_status restructured_enqueue(sap_handle h, double alpha)
{
    (void)alpha;
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    sap_status st = restructured_enqueue_product(h, &r.gemm.tb_hi, &r.gemm.tb_lo, r.KPG, r.Y, r.Yd, r.KY, r.Ypart,
                                                 handle_state(h), s, true);
    if (st != SAP_OK) return st;
    BasisView b;
    b.k = handle_k(h);
    b.KP = handle_kp(h);
    b.KY = r.KY;
    b.U32 = handle_u32(h);
    b.U32lo = handle_u32lo(h);
    b.Y = r.Y;
    b.Yd = r.Yd;
    b.Ykt = r.KY;
    b.Ydh = r.Ydh;
    b.Ydl = r.Ydl;
    b.st = handle_state(h);
    b.cand1 = handle_cand1(h);
    b.cand2 = handle_cand2(h);
    b.cap = handle_cap(h);
    b.U64 = handle_u64(h);
    b.partials = handle_partials(h);
    return restructured_enqueue_basis(h, b, s);
}

bool restructured_u_maps(sap_handle h, void *Uhi, void *Ulo, int KPG, CUtensorMap *mhi, CUtensorMap *mlo)
{
    RestrState &r = restr_state(h);
    const bool bf16 = handle_split_bf16(h) != 0;
    return make_map(mhi, Uhi, bf16, r.NP, KPG, KPG) && make_map(mlo, Ulo, bf16, r.NP, KPG, KPG);
}

void restructured_split_host(sap_handle h, const double *U, int k, uint16_t *hi, uint16_t *lo)
{
    RestrState &r = restr_state(h);
    const int n = handle_n_dim(h);
    const bool bf16 = handle_split_bf16(h) != 0;
    const double lo_mul = bf16 ? 256.0 : 2048.0;
    for (int c = 0; c < k; ++c)
        for (int l = 0; l < n; ++l) {
            const double v = U[(size_t)c * n + l];
            const size_t idx = (size_t)c * r.NP + l;
            if (bf16) {
                const __nv_bfloat16 hv = __double2bfloat16(v);
                const __nv_bfloat16 lv = __double2bfloat16((v - (double)__bfloat162float(hv)) * lo_mul);
                std::memcpy(&hi[idx], &hv, 2);
                std::memcpy(&lo[idx], &lv, 2);
            } else {
                const __half hv = __double2half(v);
                const __half lv = __double2half((v - (double)__half2float(hv)) * lo_mul);
                std::memcpy(&hi[idx], &hv, 2);
                std::memcpy(&lo[idx], &lv, 2);
            }
        }
}

sap_status restructured_classify(sap_handle h, int k)
{
    const RestrState &r = restr_state(h);
    if (r.k_cls == k && r.b_cap == handle_tune(h).b_cap) return SAP_OK;
    return classify(h, k);
}

sap_status restructured_project(sap_handle h, float *Y_out, int out_is_device)
{
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int k = handle_k(h);
    const int N = (int)handle_n_points(h);
    GemmArgs g = product_args(h, r);
    g.Y = r.Y;
    g.KY = r.KY;
    g.KPG = r.KPG;
    g.stages = gemm_pick_stages(r.KPG, g.nkb);
    g.st = handle_state(h);
    g.Ypart = r.Ypart;
    cudaEvent_t ea, eb;
    handle_count_launch(h, 0, &ea, &eb);
    if (ea) cudaEventRecord(ea, s);
    RCK(launch_gemm_y(g, s));
    if (eb) cudaEventRecord(eb, s);
    handle_push_timing(h, 0, ea, eb);
    // Y^T (component-major) -> N x k row-major
    if (out_is_device) {
        transpose_y_kernel<<<(N * k + 255) / 256, 256, 0, s>>>(r.Y, r.KY, N, k, Y_out);
        RCK(cudaGetLastError());
        RCK(cudaStreamSynchronize(s));
    } else {
        std::vector<float> yt((size_t)r.KY * r.Npad);  // the whole block-major buffer
        RCK(cudaMemcpyAsync(yt.data(), r.Y, yt.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
        RCK(cudaStreamSynchronize(s));
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < k; ++c)
                Y_out[(size_t)i * k + c] = yt[(size_t)(i >> 7) * r.KY * 128 + (size_t)c * 128 + (i & 127)];
    }
    return SAP_OK;
}

sap_status restructured_project_df(sap_handle h, float *Yh_out, float *Yl_out, int out_is_device)
{
    RestrState &r = restr_state(h);
    cudaStream_t s = handle_stream(h);
    const int k = handle_k(h);
    const int N = (int)handle_n_points(h);
    YdfArgs y;
    y.X = handle_x32(h);
    y.N = N;
    y.n = handle_n_dim(h);
    y.U32 = handle_u32(h);
    y.U32lo = handle_u32lo(h);
    y.KP = handle_kp(h);
    y.Npad = r.Npad;
    y.Yh = r.Ydh;
    y.Yl = r.Ydl;
    y.KY = r.KY;
    RefineArgs unused;
    std::memset(&unused, 0, sizeof(unused));
    RCK(launch_ydf_refine(y, unused, k, 2 * handle_sms(h), 0, true, s));
    std::vector<float> th((size_t)k * r.Npad), tl((size_t)k * r.Npad);
    RCK(cudaMemcpyAsync(th.data(), r.Ydh, th.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    RCK(cudaMemcpyAsync(tl.data(), r.Ydl, tl.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    std::vector<float> oh((size_t)N * k), ol((size_t)N * k);
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < k; ++c) {
            oh[(size_t)i * k + c] = th[(size_t)c * r.Npad + i];
            ol[(size_t)i * k + c] = tl[(size_t)c * r.Npad + i];
        }
    const cudaMemcpyKind kind = out_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    RCK(cudaMemcpy(Yh_out, oh.data(), oh.size() * sizeof(float), kind));
    RCK(cudaMemcpy(Yl_out, ol.data(), ol.size() * sizeof(float), kind));
    return SAP_OK;
}

int restructured_tier_for(sap_handle h, int k)
{
    const int t = handle_tune(h).refine;
    const int n = handle_n_dim(h);
    if (t == 5) return k > 16 ? 0 : 5;
    if (t == 4) return 4;
    if (t == 3) return k <= 8 ? 3 : 0;
    if (t == 2) return explicit_uses_df(n) ? 0 : 2;
    if (t < 0) return n > 256 ? 1 : k <= 16 ? 5 : 0;
    return t != 0 ? 1 : 0;
}

int restructured_tier(sap_handle h) { return restructured_tier_for(h, handle_k(h)); }

int restructured_pass_grid(sap_handle h) { return std::min(restr_state(h).nwtiles, handle_sms(h)); }

bool restructured_uses_refine(sap_handle h) { return restructured_tier(h) == 1; }

void restructured_fuse_args(sap_handle h, const BasisView &b, SelectUpdateArgs &u)
{
    u.fused = 0;
    u.near = nullptr;
    u.n_near = 0;
    u.cert2 = cert_explicit(handle_n_dim(h), b.k);
    const int tier = restructured_tier_for(h, b.k);
    if (tier == 5) {
        // the pass left its blocks' best pairs: one block takes the argmin
        u.pass_parts = restructured_pass_grid(h);
        u.grid = 1;
        return;
    }
    if (tier == 4) {
        // the extended tier's packed list, filtered by the final bound
        u.fused = 4;
        u.list = b.cand2;
        u.which = 2;
        u.cert2 = cert_explicit_df(handle_n_dim(h), b.k);
        return;
    }
    if (tier != 2 && tier != 3) return;
    RestrState &r = restr_state(h);
    u.fused = tier;
    u.near = r.near;
    u.n_near = r.n_near;
    u.list = b.cand1;
    u.which = 1;
    if (tier == 3) {
        u.cert2 = cert_explicit_df(handle_n_dim(h), b.k);
        u.grid = std::min(std::max(1, handle_tune(h).expl_per_sm) * handle_sms(h), kRecheckBlocks);
    }
}

int restructured_kernels_per_iteration(sap_handle h)
{
    // product (+ slice sum), pass, and the explicit tier, or the double-float
    // product + refine tier, or nothing (fused into the FP64 recheck or, 5,
    // into the pass)
    const int tier = restructured_tier(h);
    return 2 + (tier == 1 ? 2 : (tier == 0 || tier == 4) ? 1 : 0) + (restr_state(h).ksplit > 1 ? 1 : 0);  // 2, 3: fused
}

void restructured_free(sap_handle h)
{
    RestrState &r = restr_state(h);
    dfree(r.Xhi); dfree(r.Xlo); dfree(r.center); dfree(r.nu); dfree(r.w); dfree(r.wtiles);
    dfree(r.near); dfree(r.counters); dfree(r.Uhi); dfree(r.Ulo); dfree(r.Y); dfree(r.Yd); dfree(r.Ypart);
    dfree(r.near_w); dfree(r.xn); dfree(r.Ydh); dfree(r.Ydl); dfree(r.wb);
}

void restructured_stats(sap_handle h, sap_stats *out)
{
    RestrState &r = restr_state(h);
    out->n_near = r.n_near;
    out->n_excluded = r.n_excluded;
    out->cert_bound = r.b_cap;
    out->y_error_unit = r.y_eps;
    out->ydf_error_unit = df_error_unit(handle_n_dim(h));
}

} // namespace sap
