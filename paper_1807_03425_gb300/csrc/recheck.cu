// recheck.cu -- FP64 re-evaluation of the candidate pairs selected by the
// faster tiers, and the exact argmin among them (Algorithm 1, argmin step;
// ties go to the smallest pair index).
//
// One warp per candidate: lanes stride over the n coordinates, forming the
// explicit FP64 difference D = x_i - x_j, d^2 = |D|^2 and z = U^T D, then
// r = sqrt(|z|^2 / d^2).  The exclusion rules are applied here exactly: a
// pair is dropped if d^2 == 0 (not distinct, Sec. II) or d^2 < eps^2
// (shorter than the threshold of Sec. VII).  Each block writes its best
// (r, i, j) to partials[blockIdx.x]; the update kernel reduces them.
#include "sap_internal.cuh"

namespace sap {
namespace {

template <typename TX>
__global__ void __launch_bounds__(256) recheck_fp64_kernel(RecheckArgs a)
{
    __shared__ Partial wb[8];
    const TX *X = static_cast<const TX *>(a.X);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned int cnt = a.which == 1 ? (unsigned int)a.st->cnt1 : (unsigned int)a.st->cnt2;
    if (cnt > a.cap) cnt = a.cap;
    Partial best = {INFINITY, 0x7fffffff, 0x7fffffff};
    const unsigned int gw = blockIdx.x * 8 + w, nw = gridDim.x * 8;
    for (unsigned int e = gw; e < cnt; e += nw) {
        const int2 ij = a.list[e];
        const TX *xi = X + (size_t)ij.x * a.n;
        const TX *xj = X + (size_t)ij.y * a.n;
        double d2 = 0.0;
        double z[kMaxK];
#pragma unroll
        for (int c = 0; c < kMaxK; ++c) z[c] = 0.0;
        for (int l = lane; l < a.n; l += 32) {
            const double D = (double)xi[l] - (double)xj[l];
            d2 = fma(D, D, d2);
#pragma unroll
            for (int c = 0; c < kMaxK; ++c)
                if (c < a.k) z[c] = fma(a.U64[(size_t)c * a.n + l], D, z[c]);
        }
        d2 = warp_sum(d2);
        double zz = 0.0;
#pragma unroll
        for (int c = 0; c < kMaxK; ++c)
            if (c < a.k) {
                const double zc = warp_sum(z[c]);
                zz = fma(zc, zc, zz);
            }
        if (d2 == 0.0 || d2 < a.eps2) continue;
        const double r = sqrt(zz / d2);
        if (better(r, ij.x, ij.y, best.r, best.i, best.j)) best = Partial{r, ij.x, ij.y};
    }
    // all lanes of a warp hold the same best; reduce the 8 warps
    if (lane == 0) wb[w] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial b = wb[0];
        for (int q = 1; q < 8; ++q)
            if (better(wb[q].r, wb[q].i, wb[q].j, b.r, b.i, b.j)) b = wb[q];
        a.partials[blockIdx.x] = b;
    }
}

} // namespace

cudaError_t launch_recheck_fp64(const RecheckArgs &a, cudaStream_t s)
{
    if (a.x_is_f64)
        recheck_fp64_kernel<double><<<kRecheckBlocks, 256, 0, s>>>(a);
    else
        recheck_fp64_kernel<float><<<kRecheckBlocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace sap
