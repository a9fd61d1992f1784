// gemm_tc.cu -- Y = X U on the 5th-generation tensor cores (tcgen05), the
// once-per-iteration product of the restructured form: since
// U^T (x_i - x_j) = y_i - y_j, every projected secant is a difference of two
// rows of Y.
//
// Precision: X (centred and scaled by a power of two) and U are each split
// into a 16-bit high part and a low part scaled by 2^s (s = 11 for FP16,
// 8 for BF16).  Two FP32 accumulators in TMEM collect
//     D1 = Xhi Uhi^T   and   D2 = Xhi Ulo^T + Xlo Uhi^T,
// and the epilogue forms Y = (D1 + 2^-s D2) / scale.  The dropped term
// Xlo Ulo^T and the split residuals are below 3 * 2^-2s relative to
// sum_l |x_l||u_l|; the engine adds the accumulation bound and certifies the
// all-pairs pass with the total.
//
// Kernel shape: one CTA of 128 threads per 128 rows of X.  Warp 0 lane 0
// issues TMA loads of 64-wide K blocks (128-byte swizzle) into a ring of
// shared-memory stages; warp 1 lane 0 issues the MMAs (M = 128, N = KPG,
// K = 16 per instruction) and releases each stage with tcgen05.commit; after
// the last commit all four warps read their 32 TMEM lanes and write Y.
#include "sap_internal.cuh"
#include "tc_ptx.cuh"
#include "gemm_tc.cuh"

#include <algorithm>

namespace sap {
namespace {

constexpr int GM = 128;   // rows per CTA (MMA M)
constexpr int GK = 64;    // K elements per stage (128 bytes of 16-bit)
constexpr long long kWaitBudget = 4000000000ll;  // ~2 s of clock

__host__ __device__ inline uint32_t tmem_cols_for(int n)
{
    uint32_t c = 32;
    while (c < (uint32_t)n) c <<= 1;
    return c;
}

// Butterfly sums of M hi + lo FP32 pairs over the warp, interleaved (each
// addition an exact two-sum of the high parts, the low parts added): entries
// below `live`, and the last one if `last`.  Every lane ends with a total
// (the lanes may differ in the last bits: the low parts add in lane order).
template <int M>
__device__ __forceinline__ void warp_df_totals(float (&h)[M], float (&l)[M], int live, bool last)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            if (!(c < live || (last && c == M - 1))) continue;
            const float h2 = __shfl_xor_sync(0xffffffffu, h[c], o), l2 = __shfl_xor_sync(0xffffffffu, l[c], o);
            float s, e;
            xs_two_sum(h[c], h2, s, e);
            h[c] = s;
            l[c] = __fadd_rn(l[c], __fadd_rn(l2, e));
        }
    }
}

// The seed bound of the next pass (see GemmArgs): one warp evaluates watch
// pairs q0, q0 + step, ... in extended precision (explicit FP32
// differences, error-free products with the hi + lo FP32 basis; the error
// model of the explicit extended-precision tier) and returns the smallest
// certified upper bound (lane 0's value is the one used).
__device__ float product_seeds(const GemmArgs &a, int q0, int step, int lane)
{
    const ProbState *st = a.seed_st;
    const int n = a.seed_n, k = a.seed_k, KP = a.seed_KP;
    const int nw = st->watch_n;
    const Cert cert = cert_explicit_df_dev(n, k);
    float best = INFINITY;
    for (int q = q0; q < nw; q += step) {
        const int2 pr = st->watch[q];
        if (!SAP_PAIR_OK(a.seed_st, pr, a.seed_N)) continue;
        const float *xi = a.seed_X + (size_t)pr.x * n, *xj = a.seed_X + (size_t)pr.y * n;
        float dd = 0.f, zz = 0.f;
        // components c0 .. c0 + 7, and (first chunk) |x_i - x_j|^2 in slot 8
        for (int c0 = 0; c0 < k; c0 += 8) {
            float zh[9], zl[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) zh[c] = zl[c] = 0.f;
            const int live = k - c0 < 8 ? k - c0 : 8;
            for (int l = lane; l < n; l += 32) {
                const float D = xi[l] - xj[l];
                if (c0 == 0) xs_fma(zh[8], zl[8], D, D, 0.f);
                const float *uh = a.seed_U + (size_t)l * KP + c0, *ul = a.seed_Ulo + (size_t)l * KP + c0;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < live) xs_fma(zh[c], zl[c], D, uh[c], ul[c]);
            }
            warp_df_totals<9>(zh, zl, live, c0 == 0);
            if (c0 == 0) dd = zh[8] + zl[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < live) {
                    const float z = zh[c] + zl[c];
                    zz = fmaf(z, z, zz);
                }
        }
        if (dd > 1e-30f) best = fminf(best, cert_upper(sqrtf(zz / dd), cert));
    }
    return best;
}

// 128 threads (TMA producer, MMA issuer, four epilogue warps over the TMEM
// lane quadrants), or 192 where warps 4 and 5 evaluate the seeds meanwhile.
__global__ void __launch_bounds__(192, 1) gemm_y_kernel(const __grid_constant__ GemmArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int KPG = a.KPG, S = a.stages;
    const uint32_t a_bytes = GM * GK * 2;
    const uint32_t b_bytes = (uint32_t)KPG * GK * 2;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * stage_bytes);
    uint64_t *empty = full + S;
    uint64_t *done = empty + S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_cols_for(2 * KPG);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        abort_sh = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tslot;
    // Programmatic launch: the next kernel (the pass) may start now and
    // prefetch its constant tiles; this product's operands and output belong
    // to the previous kernel's iteration, so wait for it before touching them.
    grid_dep_launch();
    grid_dep_wait();
    const int m0 = blockIdx.x * GM;
    // the next pass's seed bound, by warps 4 and 5 of every CTA (beside the
    // product): a pair per warp, merged by an atomic minimum
    // (skipped while the seeds keep missing the minimum -- the minimum pair
    // rarely recurs on some data -- and tried again every 32nd evaluation)
    if (a.seed_st && warp >= 4 && (a.seed_st->seed_miss < 2 || (a.seed_st->iter & 31) == 0)) {
        const int sw = 2 * (blockIdx.y * gridDim.x + blockIdx.x) + warp - 4;
        const int nsw = 2 * gridDim.x * gridDim.y;
        if (sw < a.seed_st->watch_n) {
            const float sb = product_seeds(a, sw, nsw, lane);
            if (lane == 0 && sb < INFINITY) atomicMin(&a.seed_st->seed_ub, __float_as_uint(sb));
        }
    }
    // this CTA's K slice
    const int kb0 = (int)(((long long)blockIdx.y * a.nkb) / a.ksplit);
    const int nkb = (int)(((long long)(blockIdx.y + 1) * a.nkb) / a.ksplit) - kb0;

    auto stage_a_hi = [&](int s) { return smem + (size_t)s * stage_bytes; };
    auto stage_a_lo = [&](int s) { return smem + (size_t)s * stage_bytes + a_bytes; };
    auto stage_b_hi = [&](int s) { return smem + (size_t)s * stage_bytes + 2 * a_bytes; };
    auto stage_b_lo = [&](int s) { return smem + (size_t)s * stage_bytes + 2 * a_bytes + b_bytes; };

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % S;
            if (kb >= S && !tc::mbar_wait_bounded(&empty[s], ((kb / S) & 1) ^ 1, kWaitBudget)) {
                atomicExch(&abort_sh, 1);
                break;
            }
            const int kx = (kb0 + kb) * GK;
            tc::mbar_expect_tx(&full[s], stage_bytes);
            tc::tma_load_2d(stage_a_hi(s), &a.ta_hi, kx, m0, &full[s]);
            tc::tma_load_2d(stage_a_lo(s), &a.ta_lo, kx, m0, &full[s]);
            tc::tma_load_2d(stage_b_hi(s), &a.tb_hi, kx, 0, &full[s]);
            tc::tma_load_2d(stage_b_lo(s), &a.tb_lo, kx, 0, &full[s]);
            ++issued;
        }
        // make sure no copy of ours is still in flight before the CTA exits
        for (int kb = issued > S ? issued - S : 0; kb < issued; ++kb)
            tc::mbar_wait_bounded(&full[kb % S], (kb / S) & 1, kWaitBudget);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_f16(GM, KPG, a.ab_bf16);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % S;
            if (!tc::mbar_wait_bounded(&full[s], (kb / S) & 1, kWaitBudget)) {
                atomicExch(&abort_sh, 1);
                break;
            }
            tc::tc_fence_after();
            const uint32_t ah = tc::smem_u32(stage_a_hi(s)), al = tc::smem_u32(stage_a_lo(s));
            const uint32_t bh = tc::smem_u32(stage_b_hi(s)), bl = tc::smem_u32(stage_b_lo(s));
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk) {
                const uint32_t off = kk * 32;
                const uint32_t acc = (kb | kk) != 0;
                tc::mma_f16(tbase, tc::desc_k_sw128(ah + off), tc::desc_k_sw128(bh + off), idesc, acc);
                tc::mma_f16(tbase + KPG, tc::desc_k_sw128(ah + off), tc::desc_k_sw128(bl + off), idesc, acc);
                tc::mma_f16(tbase + KPG, tc::desc_k_sw128(al + off), tc::desc_k_sw128(bh + off), idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();

    const bool ok = tc::mbar_wait_bounded(done, 0, kWaitBudget);
    tc::tc_fence_after();
    // the TMEM loads below are warp-collective: decide for the whole block
    const int good = __syncthreads_and(ok ? 1 : 0) && !abort_sh;
    if (good && warp < 4) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < a.KY; c0 += 8) {
            float d1[8], d2[8];
            tc::tmem_ld8(lane_base + c0, d1);
            tc::tmem_ld8(lane_base + KPG + c0, d2);
            if (row < a.Npad) {
                // component-major (Y^T): consecutive lanes write consecutive rows
                if (a.ksplit == 1) {
                    // block-major: the KY components of each 128-row block are contiguous
                    float *yb = a.Y + (size_t)(row >> 7) * ((size_t)a.KY * 128) + (row & 127);
                    float *yd = a.Yd ? a.Yd + (size_t)(row >> 7) * ((size_t)a.KY * 256) + yd_offset(row & 127)
                                     : nullptr;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < a.KY) {
                            const float y = fmaf(d2[q], a.lo_scale, d1[q]) * a.out_scale;
                            yb[(size_t)(c0 + q) * 128] = y;
                            if (yd) *reinterpret_cast<float2 *>(yd + (size_t)(c0 + q) * 256) = make_float2(y, y);
                        }
                } else {
                    float *dst = a.Ypart + (size_t)blockIdx.y * a.KY * a.Npad;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < a.KY) dst[(size_t)(c0 + q) * a.Npad + row] = fmaf(d2[q], a.lo_scale, d1[q]);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(&a.st->status, ST_TIMEOUT);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// Y = (sum of the K slices, in slice order) * out_scale; the slices are
// component-major (c * Npad + row), Y (and Yd) block-major like the
// product's output.
__global__ void ksum_kernel(const float *Ypart, int ksplit, int KY, int Npad, float out_scale, float *Y, float *Yd)
{
    const size_t count = (size_t)KY * Npad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        float s = Ypart[e];
        for (int q = 1; q < ksplit; ++q) s += Ypart[(size_t)q * count + e];
        const size_t c = e / Npad, row = e % Npad;
        const float y = s * out_scale;
        Y[(row >> 7) * ((size_t)KY * 128) + c * 128 + (row & 127)] = y;
        if (Yd)
            *reinterpret_cast<float2 *>(Yd + (row >> 7) * ((size_t)KY * 256) + c * 256 + yd_offset((int)(row & 127))) =
                make_float2(y, y);
    }
}

} // namespace

size_t gemm_smem_bytes(int KPG, int stages)
{
    const size_t stage = 2 * (size_t)GM * GK * 2 + 2 * (size_t)KPG * GK * 2;
    return 1024 + stages * stage + (2 * stages + 1) * 8 + 16;
}

int gemm_pick_stages(int KPG, int nkb)
{
    int s = 4;
    while (s > 1 && gemm_smem_bytes(KPG, s) > 200 * 1024) --s;
    return s < nkb ? s : (nkb > 0 ? nkb : 1);
}

cudaError_t gemm_configure()
{
    return cudaFuncSetAttribute(gemm_y_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

cudaError_t launch_gemm_y(const GemmArgs &a, cudaStream_t s)
{
    const size_t shm = gemm_smem_bytes(a.KPG, a.stages);
    const int ksplit = a.ksplit < 1 ? 1 : a.ksplit;
    if (ksplit > a.nkb) return cudaErrorInvalidValue;
    GemmArgs b = a;
    b.ksplit = ksplit;
    cudaError_t e = launch_pdl(a.pdl != 0, gemm_y_kernel, dim3(a.Npad / GM, ksplit), dim3(a.seed_st ? 192 : 128), shm,
                               s, b);
    if (e != cudaSuccess || ksplit == 1) return e;
    const size_t count = (size_t)a.KY * a.Npad;
    ksum_kernel<<<(unsigned)std::min<size_t>((count + 255) / 256, 2048), 256, 0, s>>>(a.Ypart, ksplit, a.KY, a.Npad,
                                                                                    a.out_scale, a.Y, a.Yd);
    return cudaGetLastError();
}

} // namespace sap
