// sap_internal.cuh -- device-side state, constants and helpers shared by the
// library's translation units (not part of the public C ABI).
//
// Method: Secant-Avoidance Projection (SAP), Kvinge et al., arXiv:1807.03425,
// Sec. IV and Algorithm 1.  Notation: N points x_i in R^n (row-major X), an
// orthonormal basis U (n x k), unit secants s_ij = (x_i - x_j)/d_ij and ratios
// r_ij = ||U^T s_ij||.
//
// Selection scheme used by every all-pairs pass.  A pass evaluates r~ for all
// pairs in some fast arithmetic whose error is certified:
//     |r~ - r| <= A + rho * r          (A absolute, rho relative)
// so  r >= lower(r~) = (r~ - A)/(1 + rho)  and  r <= upper(r~) = (r~ + A)/(1 - rho).
// Any upper(r~_g) of an evaluated pair, and any exact ratio, bounds the true
// minimum R* from above.  A pair can be the argmin only if lower(r~_p) <= R*,
// i.e. r~_p <= U (1 + rho) + A for every valid upper bound U, so the pass
// emits exactly those pairs against the tightest U it knows.  The next tier
// re-evaluates the emitted list more precisely; the last tier is FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace sap {

// Programmatic dependent launch.  A kernel launched with launch_pdl may start
// while the kernel before it in the stream is still running; it must call
// grid_dep_wait() before it touches anything that kernel (or an earlier
// one) writes, and everything it reads before that point must be constant
// over the run (the points, the stored lengths, the near list).  A kernel
// calls grid_dep_launch() once its dependents may start: every kernel of an
// iteration calls it only after its own grid_dep_wait(), except where noted,
// so that a kernel running past its wait implies that the whole previous
// iteration has completed.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with programmatic stream serialization when `pdl` is set (else an
// ordinary launch: the griddepcontrol instructions are then no-ops).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

constexpr int kMaxK = 32;          // largest target dimension
constexpr int kWatch = 8;          // recent argmin pairs re-evaluated as seeds
constexpr int kTile = 128;         // edge of a w tile (restructured form)
constexpr int kRecheckBlocks = 304; // FP64 recheck grid (2 x 152 SMs)

// Compute width of the kernels templated on k: k itself up to 8, else k
// rounded up to 12, 16, 24 or 32.  Row strides of Y and of the FP32 basis
// are this width rounded up to 4, with zero pad columns.
__host__ __device__ inline int padded_k(int k)
{
    return k <= 8 ? k : k <= 12 ? 12 : k <= 16 ? 16 : k <= 24 ? 24 : 32;
}
__host__ __device__ inline int padded_stride(int k) { return (padded_k(k) + 3) / 4 * 4; }

enum StatusBits : int {
    ST_NO_SECANT = 1,
    ST_TIMEOUT = 2,
    ST_OVERFLOW = 4,
    ST_BOUNDS = 8,  // debug build: a data-dependent index was out of range (the access was skipped)
};

// Debug build (compiled with SAP_DEBUG_BOUNDS): every index a kernel reads
// from data -- a pair from a list, a tile's block coordinates, the argmin --
// is checked before it addresses memory; an index out of range sets
// ST_BOUNDS in the problem's status word (reported as SAP_E_BOUNDS) and the
// access is skipped, so nothing traps.  Otherwise the check is `true`.
#ifdef SAP_DEBUG_BOUNDS
__device__ __forceinline__ bool sap_bounds_ok(int *status, bool cond)
{
    if (!cond) atomicOr(status, (int)ST_BOUNDS);
    return cond;
}
#define SAP_BOUNDS_OK(st, cond) sap_bounds_ok(&(st)->status, (cond))
#else
#define SAP_BOUNDS_OK(st, cond) true
#endif
#define SAP_PAIR_OK(st, ij, N) SAP_BOUNDS_OK(st, (ij).x >= 0 && (ij).x < (N) && (ij).y >= 0 && (ij).y < (N))

// Launch parameters of one handle, chosen by the autotuner (tune.cu) or set
// explicitly.  Results never depend on them: every choice evaluates the same
// certified candidate sets and takes the same FP64 decisions.
struct TuneParams {
    double b_cap = 5e-4;     // cap of the restructured pass's per-pair error bound
    int pass_stages = 0;     // ring depth of the restructured pass (0: as many as fit)
    int expl_per_sm = 2;     // explicit-difference tier: blocks per SM
    int su_blocks = 0;       // FP64 recheck + update: blocks (0: one per SM)
    int plain_per_sm = 2;    // plain pass: blocks per SM (FP64 data: twice as many)
    int pdl = 0;             // programmatic dependent launch between the kernels of an iteration
    int refine = -1;         // second tier: 1 double-float refine, 0 explicit differences, 2 / 3 explicit
                             // (FP32 / extended precision) fused into the FP64 recheck, 4 extended precision
                             // with ratios for a final filter, 5 extended precision and FP64 inside the
                             // pass, -1 by n and k (n > 256: refine, else k <= 16: 5, else 0)
    double us_per_iter = 0;  // measured by the tuner (0: not tuned)
};

// Per-problem device state (one basis over one dataset).
struct ProbState {
    unsigned int seed_ub;   // float bits: upper bound on R* from the watch list
    unsigned int run_ub1;   // float bits: running upper bound, all-pairs pass
    unsigned int run_ub2;   // float bits: running upper bound, explicit recheck
    int cnt1;               // entries emitted by the all-pairs pass
    int cnt2;               // entries emitted by the explicit recheck
    int iter;               // evaluations recorded in the history
    int status;             // StatusBits
    int watch_n;            // filled entries of watch[]
    int watch_pos;          // next ring slot
    int last_cnt1, last_cnt2;
    int hist_cap;           // capacity of the history arrays
    unsigned int ticket;    // blocks of the select/update launch that finished
    int2 watch[kWatch];
    int seed_miss;          // evaluations since the seed bound was last within 1% of the minimum
    double last_r;          // result of the latest evaluation
    int last_i, last_j;
    // dynamic tiles handed out by the restructured pass; on a cache line of
    // its own, away from the bounds every warp of the pass polls
    alignas(128) unsigned int tile_next;
};

// Certified error model of one tier (see the header comment).
struct Cert {
    float A;
    float rho;
};

// Best pair of one recheck block (FP64).
struct Partial {
    double r;
    int i, j;
};


// Error model of the explicit-difference tier in extended precision: D =
// fl(x_i - x_j) moves U^T D and d by at most 2^-24 d (U orthonormal), so
// |r~ - r| <= 2^-24 (+ n^1.5 2^-46 for the hi + lo accumulation) absolute,
// plus the final FP32 roundings of the k + 2 terms relative.
__host__ __device__ inline Cert cert_explicit_df(int n, int k)
{
    const double u = 5.9604644775390625e-8;  // 2^-24
    const double g = (k + 2) * u / (1.0 - (k + 2) * u);
    Cert c;
    c.A = (float)((u + (double)n * sqrt((double)n) * 1.4210854715202004e-14) * 1.1);  // 2^-46
    c.rho = (float)((g + 6 * u) * 1.1);
    return c;
}

// The same model evaluated in FP32 on the device (the 1.1 margin covers
// the rounding of this arithmetic; FP64 scalar operations are slow here).
__device__ __forceinline__ Cert cert_explicit_df_dev(int n, int k)
{
    const float u = 5.9604644775390625e-8f;
    const float g = (k + 2) * u / (1.0f - (k + 2) * u);
    Cert c;
    c.A = (u + (float)n * sqrtf((float)n) * 1.4210854715202004e-14f) * 1.1f;
    c.rho = (g + 6 * u) * 1.1f;
    return c;
}

__device__ __forceinline__ float cert_upper(float rt, Cert c)
{
    // rounded outward by a relative 1e-6 so the fp32 evaluation stays an
    // upper bound
    return (rt + c.A) / (1.0f - c.rho) * 1.000001f;
}

__device__ __forceinline__ float cert_emit_threshold(float U, Cert c)
{
    return (U * (1.0f + c.rho) + c.A) * 1.000001f;
}

// Non-negative floats order like their bit patterns.
__device__ __forceinline__ void atomic_min_pos_float(unsigned int *addr, float v)
{
    atomicMin(addr, __float_as_uint(v));
}

__device__ __forceinline__ float load_pos_float(const unsigned int *addr)
{
    return __uint_as_float(*(volatile const unsigned int *)addr);
}

__device__ __forceinline__ bool better(double r, int i, int j, double rb, int ib, int jb)
{
    // lexicographic (ratio, i, j): ties go to the smallest pair index
    if (r < rb) return true;
    if (r > rb) return false;
    if (i != ib) return i < ib;
    return j < jb;
}

// Reduce-scatter of S per-lane values (S a power of two, 8..32) over a warp:
// halving exchanges (each level adds half of the remaining values), then
// butterfly adds; S - 1 + log2(32/S) additions instead of 5 per value.  On
// return v[0] of lane L holds the warp total of entry rs_index<S>(L).
template <int S>
__device__ __forceinline__ int rs_index(int lane)
{
    constexpr int b = S == 8 ? 3 : S == 16 ? 4 : 5;
    return (lane >> (5 - b)) & (S - 1);
}

template <int S, typename V>
__device__ __forceinline__ V warp_reduce_scatter(V (&v)[S], int lane)
{
    static_assert(S == 8 || S == 16 || S == 32, "reduce-scatter width");
#pragma unroll
    for (int lvl = 0; (S >> lvl) > 1; ++lvl) {
        const int half = (S >> lvl) / 2, o = 16 >> lvl;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const V send = up ? v[i] : v[i + half];
            const V keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / S; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
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

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide minimum of a float; all threads get the result.  scratch holds
// at least blockDim.x/32 floats.
__device__ __forceinline__ float block_min(float v, float *scratch)
{
    v = warp_min(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    float r = (l < nw) ? scratch[l] : INFINITY;
    r = warp_min(r);
    return r;
}

// Exclusive prefix of per-thread counts over the block; returns the block
// total through *total.  scratch holds at least 33 ints.
__device__ __forceinline__ int block_exclusive_scan(int v, int *scratch, int *total)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
    }
    __syncthreads();
    if (l == 31) scratch[w] = x;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        int s = (l < nw) ? scratch[l] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (l >= o) s += y;
        }
        if (l < nw) scratch[l] = s;          // inclusive prefix of warp sums
        if (l == nw - 1) scratch[32] = s;    // block total
    }
    __syncthreads();
    *total = scratch[32];
    return (w > 0 ? scratch[w - 1] : 0) + x - v;
}

// Extended-precision FP32 arithmetic for the explicit-difference tiers:
// s + e = a + b exactly (Knuth's two-sum; the _rn intrinsics keep the
// compiler from contracting the steps into FMAs).
__device__ __forceinline__ void xs_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x * (yh + yl), the product x * yh error-free
__device__ __forceinline__ void xs_fma(float &hi, float &lo, float x, float yh, float yl)
{
    const float p = __fmul_rn(x, yh);
    const float pe = fmaf(x, yh, -p);
    float s, e;
    xs_two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, fmaf(x, yl, pe)));
}

// Reduce-scatter of the extended-precision sums of E pairs, then lane e < E
// forms pair e's ratio (rr, code as in df_eval below).
template <int K, int E>
__device__ __forceinline__ void df_finish(float (&zh)[E][K + 1], float (&zl)[E][K + 1], const bool (&valid)[E],
                                          int lane, float &rr, int &code)
{
    // Reduce-scatter of the E (K + 1) double-float sums (halving exchanges,
    // each addition an exact two-sum of the high parts with the low parts
    // added), then lane e < E gathers its pair's K + 1 totals.
    constexpr int M = E * (K + 1);
    static_assert(M <= 32, "pairs per warp times components");
    constexpr int S = M <= 8 ? 8 : M <= 16 ? 16 : 32;
    constexpr int dup = 32 / S;
    float h[S], lo[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
        h[q] = q < M ? zh[q < M ? q / (K + 1) : 0][q < M ? q % (K + 1) : 0] : 0.f;
        lo[q] = q < M ? zl[q < M ? q / (K + 1) : 0][q < M ? q % (K + 1) : 0] : 0.f;
    }
#pragma unroll
    for (int lvl = 0; (S >> lvl) > 1; ++lvl) {
        const int half = (S >> lvl) / 2, o = 16 >> lvl;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float sh_ = up ? h[i] : h[i + half], sl = up ? lo[i] : lo[i + half];
            const float kh = up ? h[i + half] : h[i], kl = up ? lo[i + half] : lo[i];
            const float rh = __shfl_xor_sync(0xffffffffu, sh_, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
            float sum, er;
            xs_two_sum(kh, rh, sum, er);
            h[i] = sum;
            lo[i] = __fadd_rn(kl, __fadd_rn(rl, er));
        }
    }
#pragma unroll
    for (int o = 16 / S; o > 0; o >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, h[0], o), rl = __shfl_xor_sync(0xffffffffu, lo[0], o);
        float sum, er;
        xs_two_sum(h[0], rh, sum, er);
        h[0] = sum;
        lo[0] = __fadd_rn(lo[0], __fadd_rn(rl, er));
    }
    const float tot = h[0] + lo[0];
    const int me = lane < E ? lane : 0;
    float z[K + 1];
#pragma unroll
    for (int q = 0; q <= K; ++q) z[q] = __shfl_sync(0xffffffffu, tot, (me * (K + 1) + q) * dup);
    const float dd = z[K];
    float zz = 0.f;
#pragma unroll
    for (int c = 0; c < K; ++c) zz = fmaf(z[c], z[c], zz);
    bool v = false;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (lane == e) v = valid[e];
    code = (lane >= E || !v) ? 0 : (dd < 1e-30f ? 2 : 1);
    rr = code == 1 ? sqrtf(zz / dd) : INFINITY;
}

// Extended-precision explicit evaluation of E pairs by one warp (the
// extended-precision second tiers): D = fl(x_i - x_j) in FP32, then |D|^2 and U^T D as
// hi + lo FP32 sums with error-free products against the hi + lo FP32 basis.
// Since U is orthonormal, the rounding of D moves U^T D and d by at most
// 2^-24 d, so the ratio's error is 2^-24 absolute plus small relative terms
// (the error model of the explicit extended-precision tier).  On return lane
// e < E holds pair e's ratio in rr with code 1, or code 2 when |D|^2 is too
// small for FP32 (decided in FP64 downstream); other lanes get code 0.
template <int K, int E>
__device__ __forceinline__ void df_eval(const float *X, int n, const float *U32, const float *U32lo, int KP,
                                        const int2 (&pr)[E], const bool (&valid)[E], int lane, float &rr,
                                        int &code)
{
    float zh[E][K + 1], zl[E][K + 1];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int q = 0; q <= K; ++q) zh[e][q] = zl[e][q] = 0.f;
#pragma unroll 2
    for (int l = lane; l < n; l += 32) {
        float uh[K], ul[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            uh[c] = __ldcg(U32 + (size_t)l * KP + c);
            ul[c] = __ldcg(U32lo + (size_t)l * KP + c);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float D = X[(size_t)pr[e].x * n + l] - X[(size_t)pr[e].y * n + l];
            xs_fma(zh[e][K], zl[e][K], D, D, 0.f);
#pragma unroll
            for (int c = 0; c < K; ++c) xs_fma(zh[e][c], zl[e][c], D, uh[c], ul[c]);
        }
    }
    df_finish<K, E>(zh, zl, valid, lane, rr, code);
}

// A candidate with its extended-precision ratio packed in 64 bits: i and j
// take 17 bits each (N <= 92681), the ratio's FP32 bits without the lowest
// (truncation rounds down, so a filter on it keeps a superset); a pair too
// short for FP32 carries ratio 0 (always kept).
__device__ __forceinline__ unsigned long long pack_cand(int i, int j, float r, bool short_pair)
{
    const unsigned long long rb = short_pair ? 0ull : (unsigned long long)(__float_as_uint(r) >> 1);
    return ((unsigned long long)i << 47) | ((unsigned long long)j << 30) | rb;
}
__device__ __forceinline__ float packed_ratio(unsigned long long v)
{
    return __uint_as_float((unsigned int)(v & 0x3fffffffull) << 1);
}
__device__ __forceinline__ int2 packed_pair(unsigned long long v)
{
    return make_int2((int)(v >> 47), (int)((v >> 30) & 0x1ffffull));
}

// Offset of row a (0..127) of a block in the doubled row-side copy of Y
// (per component 256 floats): the all-pairs pass's consumer warp g (0..15)
// takes rows g, g + 16, ..., g + 112, two at a time, so row a = 16 r + g
// sits at g * 16 + (r / 2) * 4 + (r % 2) * 2 as the pair {y_a, y_a}.
__host__ __device__ __forceinline__ int yd_offset(int a)
{
    const int g = a & 15, r = a >> 4;
    return g * 16 + (r >> 1) * 4 + (r & 1) * 2;
}

// ---------------------------------------------------------------------------
// Host-side launchers (implemented in the .cu files, called by the engine).

struct PlainArgsF32 {
    const float *X;        // N x n row-major
    int N, n;
    const float *U32;      // n x KP row-major (l, c)
    int k, KP;
    const int2 *tiles;     // (I, J) 64-point blocks, I <= J
    int ntiles;
    int grid;              // persistent grid size
    float eps2_lo, eps2_hi; // d^2 window decided in FP64 downstream (0,0: none)
    Cert cert;
    ProbState *st;
    int2 *cand;            // output list
    long long cand_cap;
};

struct PlainArgsF64 {
    const double *X;
    int N, n;
    const double *U64;     // n x k column-major
    int k;
    const int2 *tiles;     // (I, J) 16-point blocks, I <= J
    int ntiles;
    int grid;
    double eps2;
    Cert cert;
    ProbState *st;
    int2 *cand;
    long long cand_cap;
};

cudaError_t launch_plain_f32(const PlainArgsF32 &a, cudaStream_t s);
cudaError_t launch_plain_f64(const PlainArgsF64 &a, cudaStream_t s);

// FP64 recheck of a candidate list (count read from st->cnt1 when which == 1,
// st->cnt2 when which == 2) fused with the basis update, which the last
// block to finish performs (select_update.cu).
struct SelectUpdateArgs {
    const void *X;         // float or double, N x n
    int x_is_f64;
    int N, n;
    double *U64;           // n x k column-major, updated in place
    float *U32;            // n x KP row-major, written
    float *U32lo;          // n x KP: fl(U64 - U32), written when non-null
    int KP;
    void *Uhi, *Ulo;       // tensor-core operands (KPG x NP, 16-bit), or null
    int NP;
    int split_bf16;        // 0: FP16 split, 1: BF16 split
    float split_scale;     // multiplier of the low part (2^11 FP16, 2^8 BF16)
    int k;
    double alpha;
    int mode;              // 0 literal, 1 angle
    int eval_only;
    double eps2;
    const int2 *list;
    unsigned int cap;
    int which;
    Partial *partials;     // grid entries
    int grid;
    double *work;          // (kMaxK + 1) * n doubles of scratch
    ProbState *st;
    double *hist;          // hist_cap entries
    int2 *argmin;          // hist_cap entries
    Cert seed_cert;        // error model of the seed evaluation
    int pdl;               // launch with programmatic stream serialization
    // fused second tier (restructured form, FP32 data only):
    //  fused == 2: phase 1 takes the near pairs and the pass's candidates
    //    (list, count in st->cnt1), filters each by explicit FP32
    //    differences under cert2 and evaluates the survivors in FP64 at once;
    //  fused == 3: the same pairs from explicit differences in extended
    //    precision (cert2), each survivor evaluated in FP64 at once by the
    //    same warp (k <= 8; the grid is the tier's);
    //  fused == 4: the list (count in st->cnt2) holds the extended-precision
    //    tier's packed (i, j, ratio) entries; those within the final bound
    //    (cert2) are evaluated in FP64
    int fused;
    const int2 *near;
    int n_near;
    Cert cert2;
    // shard evaluation (eval_only): the best pair (q = r^2, i, j; i = -1 if
    // none) goes here instead of the history, and no status bit is set
    Partial *shard_rec = nullptr;
    // 1: the next iteration's product evaluates the seeds (FP32 and BF16
    // data); an update that changes the basis then only resets the seed
    // bound to +inf
    int seeds_in_product = 0;
    // > 0: the all-pairs pass evaluated every candidate in FP64 and left its
    // blocks' best pairs in partials[0 .. pass_parts - 1]; one block takes
    // the argmin and updates (no list is read)
    int pass_parts = 0;
};
cudaError_t launch_select_update(const SelectUpdateArgs &a, cudaStream_t s);

} // namespace sap
