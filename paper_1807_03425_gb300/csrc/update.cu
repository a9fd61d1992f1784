// update.cu -- the FP64 basis update of one SAP iteration (Algorithm 1 and
// the prose of Sec. IV), run by one thread block per problem:
//   1. reduce the FP64 recheck partials to the argmin pair (ties: smallest
//      pair index) and record it in the history;
//   2. s = (x_i - x_j)/||x_i - x_j||, c = U^T s, v = U c (= P P^T s);
//   3. pivot t = argmax_l |c_l| (first on ties; t = 1 if all are zero);
//   4. modified Gram-Schmidt on [v, u_1..u_{t-1}, u_{t+1}..u_k] (a zero v is
//      skipped, so the other columns are orthonormalised among themselves);
//   5. u_1' = unit((1-alpha) v + alpha (s - v))  (literal reading), or
//      unit((1-alpha) v/|v| + alpha e/|e|) with e = s - v (angle reading);
//   6. one more MGS pass over [u_1', q_2..q_k] (re-orthonormalisation);
//   7. write U in FP64 (master), FP32 (plain pass, explicit recheck) and as
//      the split 16-bit operands of the tensor-core product;
//   8. re-evaluate the recent argmin pairs under the new basis (FP32 explicit
//      differences) to seed the next evaluation's upper bound on the minimum;
//   9. reset the per-iteration counters.
// Vectors live in shared memory when (k+2) n doubles fit, else in the global
// scratch the engine provides.
#include "sap_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sap {
namespace {

constexpr int UB = 256; // threads per update block

__device__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = (l < UB / 32) ? red[l] : 0.0;
    r = warp_sum(r);
    return r;
}

// Sums of m per-thread partials (m <= kMaxK); results in out[0..m-1]
// (shared memory), visible to all threads on return.
__device__ void block_sum_multi(const double *part, int m, double *red, double *out)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    for (int c = 0; c < m; ++c) {
        double v = warp_sum(part[c]);
        if (l == 0) red[w * kMaxK + c] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double s = 0.0;
        for (int q = 0; q < UB / 32; ++q) s += red[q * kMaxK + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <typename TX>
__device__ __forceinline__ double xval(const void *X, size_t idx)
{
    return (double)static_cast<const TX *>(X)[idx];
}

// MGS over m vectors of length n stored at V + a*n; alive[a] = 0 marks a
// vector whose norm is exactly zero (it is skipped by later projections).
__device__ void mgs_block(double *V, int m, int n, int *alive, double *red)
{
    for (int a = 0; a < m; ++a) {
        double *w = V + (size_t)a * n;
        for (int b = 0; b < a; ++b) {
            if (!alive[b]) continue;
            const double *q = V + (size_t)b * n;
            double p = 0.0;
            for (int l = threadIdx.x; l < n; l += UB) p = fma(q[l], w[l], p);
            const double h = block_sum(p, red);
            for (int l = threadIdx.x; l < n; l += UB) w[l] = fma(-h, q[l], w[l]);
        }
        double p = 0.0;
        for (int l = threadIdx.x; l < n; l += UB) p = fma(w[l], w[l], p);
        const double nrm = sqrt(block_sum(p, red));
        if (nrm == 0.0) {
            if (threadIdx.x == 0) alive[a] = 0;
        } else {
            if (threadIdx.x == 0) alive[a] = 1;
            for (int l = threadIdx.x; l < n; l += UB) w[l] = w[l] / nrm;
        }
        __syncthreads();
    }
}

template <typename TX>
__global__ void __launch_bounds__(UB) update_kernel(UpdateArgs a)
{
    extern __shared__ double dyn[];
    __shared__ double red[(UB / 32) * kMaxK];
    __shared__ double cvec[kMaxK];
    __shared__ Partial wbest[UB / 32];
    __shared__ int list_sh[kMaxK];
    __shared__ int alive[kMaxK];
    __shared__ float seed_sh[kWatch];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = a.n, k = a.k;
    ProbState *st = a.st;

    // 1. argmin over the recheck partials
    Partial b = {INFINITY, 0x7fffffff, 0x7fffffff};
    for (int p = tid; p < a.nparts; p += UB) {
        const Partial q = a.partials[p];
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
    if (lane == 0) wbest[w] = b;
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < UB / 32; ++q)
            if (better(wbest[q].r, wbest[q].i, wbest[q].j, b.r, b.i, b.j)) b = wbest[q];
        wbest[0] = b;
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
        st->run_ub1 = 0x7f800000u;
        st->run_ub2 = 0x7f800000u;
        if (!none) {
            // remember the pair as a seed for later evaluations
            bool present = false;
            for (int q = 0; q < st->watch_n; ++q)
                present |= (st->watch[q].x == b.i && st->watch[q].y == b.j);
            if (!present) {
                st->watch[st->watch_pos] = make_int2(b.i, b.j);
                st->watch_pos = (st->watch_pos + 1) % kWatch;
                if (st->watch_n < kWatch) ++st->watch_n;
            }
        }
    }
    __syncthreads();
    b = wbest[0];
    if (!(b.r < INFINITY)) return;
    if (a.eval_only) {
        // the basis is unchanged, so the exact minimum bounds the next one
        if (tid == 0) st->seed_ub = __float_as_uint(__double2float_ru(b.r) * 1.000001f);
        return;
    }

    double *W = ((size_t)(k + 2) * n * sizeof(double) <= 48 * 1024) ? dyn : a.work;
    double *s = W;              // n
    double *v = W + n;          // n: P P^T s
    double *V = W + 2 * (size_t)n; // k vectors: MGS list, then the new basis

    // 2. unit secant
    double p = 0.0;
    for (int l = tid; l < n; l += UB) {
        const double D = xval<TX>(a.X, (size_t)b.i * n + l) - xval<TX>(a.X, (size_t)b.j * n + l);
        s[l] = D;
        p = fma(D, D, p);
    }
    const double d = sqrt(block_sum(p, red));
    double cp[kMaxK];
#pragma unroll
    for (int c = 0; c < kMaxK; ++c) cp[c] = 0.0;
    for (int l = tid; l < n; l += UB) {
        const double sl = s[l] / d;
        s[l] = sl;
#pragma unroll
        for (int c = 0; c < kMaxK; ++c)
            if (c < k) cp[c] = fma(a.U64[(size_t)c * n + l], sl, cp[c]);
    }
    block_sum_multi(cp, k, red, cvec);

    // 3. pivot and the MGS list order
    if (tid == 0) {
        int t = 0;
        double cmax = fabs(cvec[0]);
        for (int c = 1; c < k; ++c)
            if (fabs(cvec[c]) > cmax) { cmax = fabs(cvec[c]); t = c; }
        list_sh[0] = -1;
        int q = 1;
        for (int c = 0; c < k; ++c)
            if (c != t) list_sh[q++] = c;
    }
    __syncthreads();
    for (int l = tid; l < n; l += UB) {
        double vl = 0.0;
        for (int c = 0; c < k; ++c) vl = fma(cvec[c], a.U64[(size_t)c * n + l], vl);
        v[l] = vl;
        V[l] = vl;
        for (int q = 1; q < k; ++q) V[(size_t)q * n + l] = a.U64[(size_t)list_sh[q] * n + l];
    }
    __syncthreads();

    // 4. MGS on [v, remaining columns]
    mgs_block(V, k, n, alive, red);

    // 5. rotation of the first column
    double nv = 1.0, ne = 1.0;
    if (a.mode == 1) {
        double pv = 0.0, pe = 0.0;
        for (int l = tid; l < n; l += UB) {
            pv = fma(v[l], v[l], pv);
            const double e = s[l] - v[l];
            pe = fma(e, e, pe);
        }
        nv = sqrt(block_sum(pv, red));
        ne = sqrt(block_sum(pe, red));
    }
    const double al = a.alpha;
    double pd = 0.0;
    for (int l = tid; l < n; l += UB) {
        const double e = s[l] - v[l];
        double dl;
        if (a.mode == 1)
            dl = (1.0 - al) * (nv > 0.0 ? v[l] / nv : 0.0) + al * (ne > 0.0 ? e / ne : 0.0);
        else
            dl = (1.0 - al) * v[l] + al * e;
        v[l] = dl;  // v is no longer needed: hold the direction
        pd = fma(dl, dl, pd);
    }
    const double nd = sqrt(block_sum(pd, red));
    const bool keep_q1 = alive[0] != 0;
    for (int l = tid; l < n; l += UB) {
        if (nd > 0.0) V[l] = v[l] / nd;
        else if (!keep_q1) V[l] = s[l];
        // else: alpha = 1 with s in the span, keep q1
    }
    __syncthreads();

    // 6. re-orthonormalisation
    mgs_block(V, k, n, alive, red);

    // 7. outputs
    for (int l = tid; l < n; l += UB)
        for (int c = 0; c < k; ++c) a.U64[(size_t)c * n + l] = V[(size_t)c * n + l];
    for (int idx = tid; idx < n * a.KP; idx += UB) {
        const int l = idx / a.KP, c = idx % a.KP;
        a.U32[idx] = c < k ? (float)V[(size_t)c * n + l] : 0.f;
    }
    if (a.Uhi) {
        for (int idx = tid; idx < a.KPG * a.NP; idx += UB) {
            const int c = idx / a.NP, l = idx % a.NP;
            const double val = (c < k && l < n) ? V[(size_t)c * n + l] : 0.0;
            if (a.split_bf16) {
                const __nv_bfloat16 h = __double2bfloat16(val);
                const double rest = (val - (double)__bfloat162float(h)) * (double)a.split_scale;
                static_cast<__nv_bfloat16 *>(a.Uhi)[idx] = h;
                static_cast<__nv_bfloat16 *>(a.Ulo)[idx] = __double2bfloat16(rest);
            } else {
                const __half h = __double2half(val);
                const double rest = (val - (double)__half2float(h)) * (double)a.split_scale;
                static_cast<__half *>(a.Uhi)[idx] = h;
                static_cast<__half *>(a.Ulo)[idx] = __double2half(rest);
            }
        }
    }
    __syncthreads();

    // 8. seed: the recent argmin pairs under the new basis
    const int nwatch = st->watch_n;
    if (w < nwatch) {
        const int2 pr = st->watch[w];
        float seed = INFINITY;
        if (sizeof(TX) == 8) {
            double dd = 0.0, z[kMaxK];
#pragma unroll
            for (int c = 0; c < kMaxK; ++c) z[c] = 0.0;
            for (int l = lane; l < n; l += 32) {
                const double D = xval<TX>(a.X, (size_t)pr.x * n + l) - xval<TX>(a.X, (size_t)pr.y * n + l);
                dd = fma(D, D, dd);
#pragma unroll
                for (int c = 0; c < kMaxK; ++c)
                    if (c < k) z[c] = fma(a.U64[(size_t)c * n + l], D, z[c]);
            }
            dd = warp_sum(dd);
            double zz = 0.0;
#pragma unroll
            for (int c = 0; c < kMaxK; ++c)
                if (c < k) { const double zc = warp_sum(z[c]); zz = fma(zc, zc, zz); }
            if (dd > 0.0) seed = __double2float_ru(sqrt(zz / dd)) * 1.000001f;
        } else {
            const float *X = static_cast<const float *>(a.X);
            float dd = 0.f, z[kMaxK];
#pragma unroll
            for (int c = 0; c < kMaxK; ++c) z[c] = 0.f;
            for (int l = lane; l < n; l += 32) {
                const float D = X[(size_t)pr.x * n + l] - X[(size_t)pr.y * n + l];
                dd = fmaf(D, D, dd);
#pragma unroll
                for (int c = 0; c < kMaxK; ++c)
                    if (c < k) z[c] = fmaf(a.U32[(size_t)l * a.KP + c], D, z[c]);
            }
            dd = warp_sumf(dd);
            float zz = 0.f;
#pragma unroll
            for (int c = 0; c < kMaxK; ++c)
                if (c < k) { const float zc = warp_sumf(z[c]); zz = fmaf(zc, zc, zz); }
            if (dd > 1e-30f) seed = cert_upper(sqrtf(zz / dd), a.seed_cert);
        }
        if (lane == 0) seed_sh[w] = seed;
    }
    __syncthreads();
    if (tid == 0) {
        float m = INFINITY;
        for (int q = 0; q < nwatch; ++q) m = fminf(m, seed_sh[q]);
        st->seed_ub = __float_as_uint(m);
    }
}

} // namespace

cudaError_t launch_update(const UpdateArgs &a, cudaStream_t s)
{
    const size_t need = (size_t)(a.k + 2) * a.n * sizeof(double);
    const size_t shm = need <= 48 * 1024 ? need : 0;
    if (a.x_is_f64)
        update_kernel<double><<<1, UB, shm, s>>>(a);
    else
        update_kernel<float><<<1, UB, shm, s>>>(a);
    return cudaGetLastError();
}

} // namespace sap
