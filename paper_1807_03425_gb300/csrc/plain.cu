// plain.cu -- the plain all-pairs pass: every unit secant is formed on the
// fly from tiles of X and projected with U (Sec. IV; the paper stores the
// secant matrix S, this form never materialises it).
//
// FP32 kernel: a block owns a 64 x 64 block of pairs (points i in block I,
// j in block J, I <= J; diagonal blocks keep i < j).  X rows of both blocks
// are staged in shared memory in chunks of 32 coordinates, transposed so a
// thread reads its 4 i's and 4 j's with one 16-byte load each; U's chunk is
// broadcast from shared memory.  Each thread accumulates, for its 4 x 4 pairs,
//     d^2 = sum_l (x_il - x_jl)^2  and  z_c = sum_l u_lc (x_il - x_jl)
// with explicit FP32 differences and FMA chains, then r~ = sqrt(|z|^2 / d^2).
// Error model (u = 2^-24, gamma_m = m u/(1 - m u)):
//     |r~ - r| <= sqrt(k) gamma_{n+3} + (gamma_{n+2} + gamma_k + 3u) r,
// from |z~_c - z_c| <= gamma_{n+2} sum_l |u_lc||D_l| <= gamma_{n+2} ||D||.
// The block emits every pair that can still be the argmin under that model
// (see the selection scheme in sap_internal.cuh); pairs whose exclusion
// (d == 0, or d < eps of Sec. VII) is too close to call in FP32 are emitted
// for the FP64 tier to decide.
#include "sap_internal.cuh"

namespace sap {
namespace {

constexpr int PB = 64;   // points per block edge
constexpr int LC = 32;   // coordinates per shared-memory chunk
constexpr int PAD = 4;

template <int K>
__global__ void __launch_bounds__(256) plain_f32_kernel(PlainArgsF32 a)
{
    __shared__ __align__(16) float xsI[LC][PB + PAD];
    __shared__ __align__(16) float xsJ[LC][PB + PAD];
    __shared__ float us[LC][K];
    __shared__ float red[32];
    __shared__ int scan[33];
    __shared__ int base_sh;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int2 IJ = a.tiles[t];
        const int i0 = IJ.x * PB, j0 = IJ.y * PB;
        float d2[4][4];
        float z[4][4][K];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d2[p][q] = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) z[p][q][c] = 0.f;
            }

        for (int l0 = 0; l0 < a.n; l0 += LC) {
            __syncthreads();
            for (int idx = tid; idx < PB * LC; idx += 256) {
                const int r = idx / LC, l = idx % LC;
                const int gl = l0 + l;
                const int gi = i0 + r, gj = j0 + r;
                xsI[l][r] = (gi < a.N && gl < a.n) ? a.X[(size_t)gi * a.n + gl] : 0.f;
                xsJ[l][r] = (gj < a.N && gl < a.n) ? a.X[(size_t)gj * a.n + gl] : 0.f;
            }
            for (int idx = tid; idx < LC * K; idx += 256) {
                const int l = idx / K, c = idx % K;
                const int gl = l0 + l;
                us[l][c] = (gl < a.n) ? a.U32[(size_t)gl * a.KP + c] : 0.f;
            }
            __syncthreads();
            const int lc = min(LC, a.n - l0);
            for (int l = 0; l < lc; ++l) {
                const float4 xi = *reinterpret_cast<const float4 *>(&xsI[l][ty * 4]);
                const float4 xj = *reinterpret_cast<const float4 *>(&xsJ[l][tx * 4]);
                const float ai[4] = {xi.x, xi.y, xi.z, xi.w};
                const float bj[4] = {xj.x, xj.y, xj.z, xj.w};
                float u[K];
#pragma unroll
                for (int c = 0; c < K; ++c) u[c] = us[l][c];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float D = ai[p] - bj[q];
                        d2[p][q] = fmaf(D, D, d2[p][q]);
#pragma unroll
                        for (int c = 0; c < K; ++c) z[p][q][c] = fmaf(u[c], D, z[p][q][c]);
                    }
            }
        }

        // classify and evaluate the 16 pairs: 0 excluded, 1 normal, 2 decide in FP64
        float rt[4][4];
        int code[4][4];
        float mymin = INFINITY;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
                const float dd = d2[p][q];
                int cd = 1;
                if (!(i < j && j < a.N)) cd = 0;
                else if (dd < 1e-30f) cd = 2;  // duplicate, or too short for FP32
                else if (a.eps2_hi > 0.f) {
                    if (dd < a.eps2_lo) cd = 0;
                    else if (dd < a.eps2_hi) cd = 2;
                }
                float zz = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) zz = fmaf(z[p][q][c], z[p][q][c], zz);
                const float r = sqrtf(zz / dd);
                rt[p][q] = r;
                code[p][q] = cd;
                if (cd == 1) mymin = fminf(mymin, r);
            }

        const float bmin = block_min(mymin, red);
        float U = load_pos_float(&a.st->seed_ub);
        if (bmin < INFINITY) {
            const float ub = cert_upper(bmin, a.cert);
            if (tid == 0) atomic_min_pos_float(&a.st->run_ub1, ub);
            U = fminf(U, ub);
        }
        U = fminf(U, load_pos_float(&a.st->run_ub1));
        const float th = cert_emit_threshold(U, a.cert);

        int cnt = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cnt += (code[p][q] == 2 || (code[p][q] == 1 && rt[p][q] <= th)) ? 1 : 0;
        int total;
        int off = block_exclusive_scan(cnt, scan, &total);
        if (total == 0) continue;
        if (tid == 0) base_sh = (int)atomicAdd((unsigned int *)&a.st->cnt1, (unsigned int)total);
        __syncthreads();
        long long pos = (long long)(unsigned int)base_sh + off;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (code[p][q] == 2 || (code[p][q] == 1 && rt[p][q] <= th)) {
                    if (pos < a.cand_cap)
                        a.cand[pos] = make_int2(i0 + ty * 4 + p, j0 + tx * 4 + q);
                    else
                        atomicOr(&a.st->status, ST_OVERFLOW);
                    ++pos;
                }
    }
}

// FP64 form (FP64 datasets): one thread per pair of a 16 x 16 block, X rows
// read through the cache.  The ratio is exact up to FP64 rounding; it is
// rounded to FP32 for the selection, hence the error model {0, 2^-23}.
// K is the basis width for k <= 8 (exactly k FP64 FMAs per coordinate:
// FP64 issue, not latency, is what a block of this kernel waits on), else
// kMaxK with the columns past k skipped.
template <int K>
__global__ void __launch_bounds__(256) plain_f64_kernel(PlainArgsF64 a)
{
    __shared__ float red[32];
    __shared__ int scan[33];
    __shared__ int base_sh;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int2 IJ = a.tiles[t];
        const int i = IJ.x * 16 + ty, j = IJ.y * 16 + tx;
        int cd = (i < j && j < a.N) ? 1 : 0;
        float rt = INFINITY;
        if (cd) {
            double d2 = 0.0;
            double z[K];
#pragma unroll
            for (int c = 0; c < K; ++c) z[c] = 0.0;
            const double *xi = a.X + (size_t)i * a.n;
            const double *xj = a.X + (size_t)j * a.n;
            for (int l = 0; l < a.n; ++l) {
                const double D = xi[l] - xj[l];
                d2 = fma(D, D, d2);
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (K <= 8 || c < a.k) z[c] = fma(a.U64[(size_t)c * a.n + l], D, z[c]);
            }
            if (d2 == 0.0 || d2 < a.eps2) {
                cd = 0;
            } else {
                double zz = 0.0;
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (K <= 8 || c < a.k) zz = fma(z[c], z[c], zz);
                rt = (float)sqrt(zz / d2);
            }
        }
        const float bmin = block_min(cd ? rt : INFINITY, red);
        float U = load_pos_float(&a.st->seed_ub);
        if (bmin < INFINITY) {
            const float ub = cert_upper(bmin, a.cert);
            if (tid == 0) atomic_min_pos_float(&a.st->run_ub1, ub);
            U = fminf(U, ub);
        }
        U = fminf(U, load_pos_float(&a.st->run_ub1));
        const float th = cert_emit_threshold(U, a.cert);
        const int emit = (cd && rt <= th) ? 1 : 0;
        int total;
        const int off = block_exclusive_scan(emit, scan, &total);
        if (total == 0) continue;
        if (tid == 0) base_sh = (int)atomicAdd((unsigned int *)&a.st->cnt1, (unsigned int)total);
        __syncthreads();
        if (emit) {
            const long long pos = (long long)(unsigned int)base_sh + off;
            if (pos < a.cand_cap) a.cand[pos] = make_int2(i, j);
            else atomicOr(&a.st->status, ST_OVERFLOW);
        }
    }
}

template <int K>
cudaError_t launch_k(const PlainArgsF32 &a, int grid, cudaStream_t s)
{
    plain_f32_kernel<K><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_plain_f32(const PlainArgsF32 &a, cudaStream_t s)
{
    const int grid = a.grid;
    switch (a.k) {
#define SAP_CASE(KK) case KK: return launch_k<KK>(a, grid, s);
        SAP_CASE(1) SAP_CASE(2) SAP_CASE(3) SAP_CASE(4)
        SAP_CASE(5) SAP_CASE(6) SAP_CASE(7) SAP_CASE(8)
#undef SAP_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_plain_f64(const PlainArgsF64 &a, cudaStream_t s)
{
    switch (a.k) {
#define SAP_CASE(KK) case KK: plain_f64_kernel<KK><<<a.grid, 256, 0, s>>>(a); break;
        SAP_CASE(1) SAP_CASE(2) SAP_CASE(3) SAP_CASE(4)
        SAP_CASE(5) SAP_CASE(6) SAP_CASE(7) SAP_CASE(8)
#undef SAP_CASE
    default: plain_f64_kernel<kMaxK><<<a.grid, 256, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

} // namespace sap
