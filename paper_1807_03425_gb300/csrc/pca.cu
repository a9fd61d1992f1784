// pca.cu -- the PCA start of Algorithm 1 (Sec. IV of Kvinge et al.,
// arXiv:1807.03425): the first basis is made of the top k left singular
// vectors of the n x p matrix S whose columns are the unit secants, i.e. the
// eigenvectors of C = S S^T with the k largest eigenvalues.
//
// S is never formed (p = N(N-1)/2 columns).  C is built in FP64 through the
// weighted graph Laplacian of the pairs:
//     C = sum_{i<j kept} (x_i - x_j)(x_i - x_j)^T / d_ij^2 = Xc^T R,
//     R_i = sum_{j kept} w_ij (x_i - x_j),  w_ij = 1/d_ij^2,  Xc = X - mean,
// (sum_i R_i = 0, so centring X is free and keeps the terms small).  Three
// kernels: FP64 inverse squared lengths from explicit differences (upper
// triangle, 64 x 64 tiles, 0 for excluded pairs: d = 0, Sec. II, or d < eps,
// Sec. VII); the rows R_i (every block owns one block of rows and walks all
// column blocks, reading the stored upper triangle transposed where needed,
// so no atomics and a fixed summation order); and C = Xc^T R.
//
// The n x n symmetric eigenproblem (the paper calls cuSolver's SVD for this
// step, Sec. V) is solved here by the cyclic Jacobi method in FP64 (Golub
// and Van Loan, Matrix Computations, Sec. 8.5): sweeps of plane rotations,
// each zeroing one off-diagonal entry (p, q) with the rotation of the 2 x 2
// symmetric Schur decomposition, in the round-robin ("tournament") order of
// the parallel variant: n' - 1 rounds of n'/2 disjoint pairs per sweep (n'
// = n rounded up to even; an odd n's extra index pairs with nobody), so
// one round is one independent rotation per pair, applied to A from both
// sides and to the accumulated vectors V.  Sweeps stop when the
// off-diagonal Frobenius norm is below 4 n 2^-53 of the whole (quadratic
// convergence: typically 6 to 10 sweeps), or after 40.
#include "sap_internal.cuh"
#include "../../include/sap.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace sap {

// engine accessors (capi.cu)
cudaStream_t handle_stream(sap_handle h);
int64_t handle_n_points(sap_handle h);
int handle_n_dim(sap_handle h);
const float *handle_x32(sap_handle h);
const double *handle_x64(sap_handle h);
double handle_eps2(sap_handle h);
sap_status handle_fail(sap_handle h, sap_status s, const char *msg);

namespace {

constexpr int PT = 64;   // points per block side
constexpr int PC = 32;   // coordinates per chunk

template <typename TX>
__device__ __forceinline__ double ldx(const TX *X, size_t i)
{
    return (double)X[i];
}

// Inverse squared lengths of the pairs of one upper-triangle tile (I <= J).
template <typename TX>
__global__ void __launch_bounds__(256) w64_kernel(const TX *X, int N, int n, const int2 *tiles, double eps2,
                                                  double *w)
{
    __shared__ double xi[PC][PT + 1], xj[PC][PT + 1];
    const int2 IJ = tiles[blockIdx.x];
    const int i0 = IJ.x * PT, j0 = IJ.y * PT;
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;  // 4 x 4 pairs each
    double d2[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) d2[p][q] = 0.0;
    for (int c0 = 0; c0 < n; c0 += PC) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < PT * PC; idx += 256) {
            const int r = idx / PC, l = idx % PC;
            const bool inl = c0 + l < n;
            xi[l][r] = (i0 + r < N && inl) ? ldx(X, (size_t)(i0 + r) * n + c0 + l) : 0.0;
            xj[l][r] = (j0 + r < N && inl) ? ldx(X, (size_t)(j0 + r) * n + c0 + l) : 0.0;
        }
        __syncthreads();
        const int lc = min(PC, n - c0);
        for (int l = 0; l < lc; ++l)
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double D = xi[l][tr * 4 + p] - xj[l][tc * 4 + q];
                    d2[p][q] = fma(D, D, d2[p][q]);
                }
    }
    double *out = w + (size_t)blockIdx.x * PT * PT;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tr * 4 + p, j = j0 + tc * 4 + q;
            const double d = d2[p][q];
            const bool kept = i < j && j < N && d != 0.0 && !(d < eps2);
            out[(tr * 4 + p) * PT + tc * 4 + q] = kept ? 1.0 / d : 0.0;
        }
}

__device__ __forceinline__ long long tile_of(int I, int J, int nb)
{
    return (long long)I * nb - (long long)I * (I - 1) / 2 + (J - I);
}

// R_i = sum_j w_ij (x_i - x_j) for the 64 rows of block I and the
// coordinates c0 .. c0 + 31 (blockIdx.y); thread: one row, 8 coordinates.
template <typename TX>
__global__ void __launch_bounds__(256) lap_rows_kernel(const TX *X, int N, int n, const double *w, int nb,
                                                       double *R)
{
    __shared__ double wt[PT][PT + 1];
    __shared__ double xs[PT][PC + 1];
    const int I = blockIdx.x, c0 = blockIdx.y * PC;
    const int r = threadIdx.x & (PT - 1), g = threadIdx.x >> 6;  // 4 groups of 8 coordinates
    const int i = I * PT + r;
    double xi[8], acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int l = c0 + g * 8 + q;
        xi[q] = (i < N && l < n) ? ldx(X, (size_t)i * n + l) : 0.0;
        acc[q] = 0.0;
    }
    for (int J = 0; J < nb; ++J) {
        __syncthreads();
        const double *tw = w + tile_of(min(I, J), max(I, J), nb) * (PT * PT);
        for (int idx = threadIdx.x; idx < PT * PT; idx += 256) {
            const int a = idx / PT, b = idx % PT;  // a: row of this block, b: row of block J
            double v;
            if (I < J) v = tw[a * PT + b];
            else if (I > J) v = tw[b * PT + a];
            else v = a < b ? tw[a * PT + b] : (a > b ? tw[b * PT + a] : 0.0);
            wt[a][b] = v;
        }
        for (int idx = threadIdx.x; idx < PT * PC; idx += 256) {
            const int b = idx / PC, l = idx % PC;
            const int j = J * PT + b;
            xs[b][l] = (j < N && c0 + l < n) ? ldx(X, (size_t)j * n + c0 + l) : 0.0;
        }
        __syncthreads();
        for (int b = 0; b < PT; ++b) {
            const double wv = wt[r][b];
            if (wv == 0.0) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = fma(wv, xi[q] - xs[b][g * 8 + q], acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int l = c0 + g * 8 + q;
        if (i < N && l < n) R[(size_t)i * n + l] = acc[q];
    }
}

template <typename TX>
__global__ void colmean64_kernel(const TX *X, int N, int n, double *mean)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += ldx(X, (size_t)i * n + l);
    mean[l] = s / N;
}

// C[a][b] = sum_i (x_ia - mean_a) R_ib over a 16 x 16 block of (a, b).
template <typename TX>
__global__ void __launch_bounds__(256) gram_kernel(const TX *X, const double *mean, const double *R, int N, int n,
                                                   double *C)
{
    __shared__ double xa[32][17], rb[32][17];
    const int a0 = blockIdx.x * 16, b0 = blockIdx.y * 16;
    const int ta = threadIdx.x >> 4, tb = threadIdx.x & 15;
    double acc = 0.0;
    for (int i0 = 0; i0 < N; i0 += 32) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * 16; idx += 256) {
            const int q = idx / 16, c = idx % 16;
            const int i = i0 + q;
            xa[q][c] = (i < N && a0 + c < n) ? ldx(X, (size_t)i * n + a0 + c) - mean[a0 + c] : 0.0;
            rb[q][c] = (i < N && b0 + c < n) ? R[(size_t)i * n + b0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; ++q) acc = fma(xa[q][ta], rb[q][tb], acc);
    }
    if (a0 + ta < n && b0 + tb < n) C[(size_t)(a0 + ta) * n + b0 + tb] = acc;
}

// C <- (C + C^T) / 2 (the two halves differ only by rounding).
__global__ void symmetrize_kernel(double *C, int n)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int a = (int)(idx / n), b = (int)(idx % n);
    if (a < b) {
        const double v = 0.5 * (C[(size_t)a * n + b] + C[(size_t)b * n + a]);
        C[(size_t)a * n + b] = v;
        C[(size_t)b * n + a] = v;
    }
}

// ---- cyclic Jacobi eigensolver (FP64)

// Round r (0 <= r < m - 1) of the round-robin pairing of m (even) indices:
// index m - 1 meets r, and every other x meets (2r - x) mod (m - 1).
__device__ __forceinline__ int rr_partner(int x, int r, int m)
{
    if (x == m - 1) return r;
    if (x == r) return m - 1;
    int y = (2 * r - x) % (m - 1);
    return y < 0 ? y + (m - 1) : y;
}

// The rotation of every pair of round r: for pair (p, q), p < q, with
// a_pq != 0, tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c; J = [[c, s], [-s, c]] in
// the (p, q) plane makes (J^T A J)_pq = 0.  Each index x stores the column
// combination col'_x = f_x col_x + g_x col_partner: (c, -s) for p, (s, c)
// read as (c, s) for q.  Unpaired indices (the extra one of an odd n, or
// a pair with a_pq = 0) keep f = 1, g = 0.
__global__ void jacobi_angles_kernel(const double *A, int n, int m, int r, double2 *fg, int *partner)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int y = rr_partner(x, r, m);
    double f = 1.0, g = 0.0;
    int pt = x;
    if (y < n) {
        const int p = x < y ? x : y, q = x < y ? y : x;
        const double apq = A[(size_t)p * n + q];
        if (apq != 0.0) {
            const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
            f = c;
            g = x == p ? -sn : sn;
            pt = y;
        }
    }
    fg[x] = make_double2(f, g);
    partner[x] = pt;
}

// A' = J^T A J entry by entry (each entry reads at most four of A) and
// V' = V J (each entry reads two of V); one thread per entry.
__global__ void jacobi_apply_kernel(const double *A, const double *V, int n, const double2 *fg, const int *partner,
                                    double *A2, double *V2)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    const double2 ci = fg[i], cj = fg[j];
    const int pi = partner[i], pj = partner[j];
    const double a = A[(size_t)i * n + j], b = A[(size_t)i * n + pj];
    const double c = A[(size_t)pi * n + j], d = A[(size_t)pi * n + pj];
    // rows combine with (f_i, g_i), columns with (f_j, g_j)
    A2[(size_t)i * n + j] = ci.x * (cj.x * a + cj.y * b) + ci.y * (cj.x * c + cj.y * d);
    V2[(size_t)i * n + j] = cj.x * V[(size_t)i * n + j] + cj.y * V[(size_t)i * n + pj];
}

__global__ void jacobi_init_kernel(double *V, int n)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < (long long)n * n) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// off = sum of squared off-diagonal entries, all = sum of all squares (one
// block; fixed summation order).
__global__ void jacobi_norms_kernel(const double *A, int n, double *out)
{
    __shared__ double so[32], sa[32];
    double off = 0.0, all = 0.0;
    for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
        const double v = A[idx];
        all = fma(v, v, all);
        if (idx / n != idx % n) off = fma(v, v, off);
    }
    off = warp_sum(off);
    all = warp_sum(all);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { so[w] = off; sa[w] = all; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double o = 0.0, a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { o += so[q]; a += sa[q]; }
        out[0] = o;
        out[1] = a;
    }
}

struct Scratch {
    double *w = nullptr, *R = nullptr, *mean = nullptr, *C = nullptr, *C2 = nullptr, *V = nullptr, *V2 = nullptr,
           *norms = nullptr;
    double2 *fg = nullptr;
    int2 *tiles = nullptr;
    int *partner = nullptr;
    ~Scratch()
    {
        for (void *p : {(void *)w, (void *)R, (void *)mean, (void *)C, (void *)C2, (void *)V, (void *)V2,
                        (void *)norms, (void *)fg, (void *)tiles, (void *)partner})
            if (p) cudaFree(p);
    }
};

} // namespace

sap_status secant_pca(sap_handle h, int k, double *U_out, double *sigma_out)
{
    const int N = (int)handle_n_points(h), n = handle_n_dim(h);
    if (k < 1 || k > n || k > kMaxK) return handle_fail(h, SAP_E_ARG, "need 1 <= k <= min(n, 32)");
    cudaStream_t s = handle_stream(h);
    const float *X32 = handle_x32(h);
    const double *X64 = handle_x64(h);
    const int nb = (N + PT - 1) / PT;
    const long long ntiles = (long long)nb * (nb + 1) / 2;
    Scratch sc;
#define PCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return handle_fail(h, e_ == cudaErrorMemoryAllocation ? SAP_E_OOM : SAP_E_CUDA,        \
                               cudaGetErrorString(e_));                                            \
    } while (0)
    std::vector<int2> t;
    t.reserve(ntiles);
    for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J) t.push_back(make_int2(I, J));
    PCK(cudaMalloc(&sc.tiles, t.size() * sizeof(int2)));
    PCK(cudaMemcpyAsync(sc.tiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    PCK(cudaMalloc(&sc.w, (size_t)ntiles * PT * PT * sizeof(double)));
    PCK(cudaMalloc(&sc.R, (size_t)N * n * sizeof(double)));
    PCK(cudaMalloc(&sc.mean, (size_t)n * sizeof(double)));
    PCK(cudaMalloc(&sc.C, (size_t)n * n * sizeof(double)));
    PCK(cudaMalloc(&sc.C2, (size_t)n * n * sizeof(double)));
    PCK(cudaMalloc(&sc.V, (size_t)n * n * sizeof(double)));
    PCK(cudaMalloc(&sc.V2, (size_t)n * n * sizeof(double)));
    PCK(cudaMalloc(&sc.norms, 2 * sizeof(double)));
    PCK(cudaMalloc(&sc.fg, (size_t)n * sizeof(double2)));
    PCK(cudaMalloc(&sc.partner, (size_t)n * sizeof(int)));
    const double eps2 = handle_eps2(h);
    const dim3 lgrid(nb, (n + PC - 1) / PC), ggrid((n + 15) / 16, (n + 15) / 16);
    if (X64) {
        w64_kernel<double><<<(unsigned)ntiles, 256, 0, s>>>(X64, N, n, sc.tiles, eps2, sc.w);
        lap_rows_kernel<double><<<lgrid, 256, 0, s>>>(X64, N, n, sc.w, nb, sc.R);
        colmean64_kernel<double><<<(n + 127) / 128, 128, 0, s>>>(X64, N, n, sc.mean);
        gram_kernel<double><<<ggrid, 256, 0, s>>>(X64, sc.mean, sc.R, N, n, sc.C);
    } else {
        w64_kernel<float><<<(unsigned)ntiles, 256, 0, s>>>(X32, N, n, sc.tiles, eps2, sc.w);
        lap_rows_kernel<float><<<lgrid, 256, 0, s>>>(X32, N, n, sc.w, nb, sc.R);
        colmean64_kernel<float><<<(n + 127) / 128, 128, 0, s>>>(X32, N, n, sc.mean);
        gram_kernel<float><<<ggrid, 256, 0, s>>>(X32, sc.mean, sc.R, N, n, sc.C);
    }
    PCK(cudaGetLastError());
    symmetrize_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(sc.C, n);
    PCK(cudaGetLastError());
    // cyclic Jacobi sweeps: A (= C) towards diag(lambda), V accumulating the
    // rotations (its columns become the eigenvectors)
    const unsigned nn_blocks = (unsigned)(((long long)n * n + 255) / 256);
    jacobi_init_kernel<<<nn_blocks, 256, 0, s>>>(sc.V, n);
    PCK(cudaGetLastError());
    const int m = n + (n & 1);
    double *A = sc.C, *A2 = sc.C2, *V = sc.V, *V2 = sc.V2;
    const double u = std::ldexp(1.0, -53);
    bool converged = n == 1;
    for (int sweep = 0; sweep < 40 && !converged; ++sweep) {
        for (int r = 0; r < m - 1; ++r) {
            jacobi_angles_kernel<<<(n + 127) / 128, 128, 0, s>>>(A, n, m, r, sc.fg, sc.partner);
            jacobi_apply_kernel<<<nn_blocks, 256, 0, s>>>(A, V, n, sc.fg, sc.partner, A2, V2);
            std::swap(A, A2);
            std::swap(V, V2);
        }
        PCK(cudaGetLastError());
        jacobi_norms_kernel<<<1, 1024, 0, s>>>(A, n, sc.norms);
        double nrm[2] = {0.0, 0.0};
        PCK(cudaMemcpyAsync(nrm, sc.norms, sizeof(nrm), cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        const double tol = 4.0 * n * u;
        converged = !(nrm[0] > tol * tol * nrm[1]);
    }
    if (!converged) return handle_fail(h, SAP_E_CUDA, "Jacobi eigensolver did not converge in 40 sweeps");
    PCK(cudaStreamSynchronize(s));  // the copies below run on the legacy stream
    // the k largest eigenvalues (diagonal of A) and their columns of V,
    // largest first; each vector signed so that its entry of largest
    // magnitude is positive
    std::vector<double> Ah((size_t)n * n), Vh((size_t)n * n);
    PCK(cudaMemcpy(Ah.data(), A, Ah.size() * sizeof(double), cudaMemcpyDeviceToHost));
    PCK(cudaMemcpy(Vh.data(), V, Vh.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<int> order(n);
    for (int c = 0; c < n; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return Ah[(size_t)a * n + a] > Ah[(size_t)b * n + b]; });
    for (int c = 0; c < k; ++c) {
        const int col = order[c];
        int am = 0;
        for (int l = 1; l < n; ++l)
            if (std::fabs(Vh[(size_t)l * n + col]) > std::fabs(Vh[(size_t)am * n + col])) am = l;
        const double sg = Vh[(size_t)am * n + col] < 0 ? -1.0 : 1.0;
        for (int l = 0; l < n; ++l) U_out[(size_t)c * n + l] = sg * Vh[(size_t)l * n + col];
        if (sigma_out) sigma_out[c] = std::sqrt(std::max(Ah[(size_t)col * n + col], 0.0));
    }
    return SAP_OK;
#undef PCK
}

} // namespace sap
