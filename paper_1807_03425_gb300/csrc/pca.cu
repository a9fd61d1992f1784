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
// so no atomics and a fixed summation order); and C = Xc^T R.  The n x n
// symmetric eigenproblem goes to cuSOLVER's FP64 divide-and-conquer solver
// (the paper's own choice of library for this step, Sec. V), loaded at the
// first call so that the library does not depend on it otherwise.
#include "sap_internal.cuh"
#include "../../include/sap.h"

#include <cusolverDn.h>
#include <dlfcn.h>

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

// ---- cuSOLVER, loaded on first use
struct Solver {
    bool tried = false, ok = false;
    cusolverStatus_t (*create)(cusolverDnHandle_t *) = nullptr;
    cusolverStatus_t (*destroy)(cusolverDnHandle_t) = nullptr;
    cusolverStatus_t (*set_stream)(cusolverDnHandle_t, cudaStream_t) = nullptr;
    cusolverStatus_t (*bufsize)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, const double *, int,
                                const double *, int *) = nullptr;
    cusolverStatus_t (*syevd)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, double *, int, double *,
                              double *, int, int *) = nullptr;
};

Solver &solver()
{
    static Solver s;
    if (s.tried) return s;
    s.tried = true;
    std::vector<std::string> names = {"libcusolver.so.12", "libcusolver.so"};
    const char *home = std::getenv("CUDA_HOME");
    names.push_back(std::string(home ? home : "/usr/local/cuda") + "/lib64/libcusolver.so.12");
    void *lib = nullptr;
    for (const auto &nm : names)
        if ((lib = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) return s;
    s.create = (decltype(s.create))dlsym(lib, "cusolverDnCreate");
    s.destroy = (decltype(s.destroy))dlsym(lib, "cusolverDnDestroy");
    s.set_stream = (decltype(s.set_stream))dlsym(lib, "cusolverDnSetStream");
    s.bufsize = (decltype(s.bufsize))dlsym(lib, "cusolverDnDsyevd_bufferSize");
    s.syevd = (decltype(s.syevd))dlsym(lib, "cusolverDnDsyevd");
    s.ok = s.create && s.destroy && s.set_stream && s.bufsize && s.syevd;
    return s;
}

struct Scratch {
    double *w = nullptr, *R = nullptr, *mean = nullptr, *C = nullptr, *lam = nullptr, *work = nullptr;
    int2 *tiles = nullptr;
    int *info = nullptr;
    ~Scratch()
    {
        for (void *p : {(void *)w, (void *)R, (void *)mean, (void *)C, (void *)lam, (void *)work, (void *)tiles,
                        (void *)info})
            if (p) cudaFree(p);
    }
};

} // namespace

sap_status secant_pca(sap_handle h, int k, double *U_out, double *sigma_out)
{
    const int N = (int)handle_n_points(h), n = handle_n_dim(h);
    if (k < 1 || k > n || k > kMaxK) return handle_fail(h, SAP_E_ARG, "need 1 <= k <= min(n, 32)");
    Solver &sv = solver();
    if (!sv.ok) return handle_fail(h, SAP_E_UNSUPPORTED, "cuSOLVER (libcusolver.so.12) could not be loaded");
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
    PCK(cudaMalloc(&sc.lam, (size_t)n * sizeof(double)));
    PCK(cudaMalloc(&sc.info, sizeof(int)));
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
    // eigenvalues ascending, eigenvectors in the columns of C (column-major:
    // C is symmetric, so its row-major storage is the same matrix)
    cusolverDnHandle_t dn = nullptr;
    if (sv.create(&dn) != CUSOLVER_STATUS_SUCCESS) return handle_fail(h, SAP_E_CUDA, "cusolverDnCreate failed");
    int lwork = 0;
    cusolverStatus_t cs = sv.set_stream(dn, s);
    if (cs == CUSOLVER_STATUS_SUCCESS)
        cs = sv.bufsize(dn, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, sc.C, n, sc.lam, &lwork);
    if (cs == CUSOLVER_STATUS_SUCCESS && cudaMalloc(&sc.work, (size_t)std::max(lwork, 1) * sizeof(double)) != cudaSuccess)
        cs = CUSOLVER_STATUS_ALLOC_FAILED;
    if (cs == CUSOLVER_STATUS_SUCCESS)
        cs = sv.syevd(dn, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, sc.C, n, sc.lam, sc.work, lwork,
                      sc.info);
    int info = 0;
    if (cs == CUSOLVER_STATUS_SUCCESS &&
        (cudaMemcpyAsync(&info, sc.info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        cs = CUSOLVER_STATUS_EXECUTION_FAILED;
    sv.destroy(dn);
    if (cs != CUSOLVER_STATUS_SUCCESS || info != 0)
        return handle_fail(h, SAP_E_CUDA, "symmetric eigensolver failed");
    // the k largest: the last k columns, largest first; each signed so that
    // its entry of largest magnitude is positive
    std::vector<double> V((size_t)n * k), lam(n);
    PCK(cudaMemcpy(V.data(), sc.C + (size_t)(n - k) * n, V.size() * sizeof(double), cudaMemcpyDeviceToHost));
    PCK(cudaMemcpy(lam.data(), sc.lam, n * sizeof(double), cudaMemcpyDeviceToHost));
    for (int c = 0; c < k; ++c) {
        const double *src = V.data() + (size_t)(k - 1 - c) * n;
        int am = 0;
        for (int l = 1; l < n; ++l)
            if (std::fabs(src[l]) > std::fabs(src[am])) am = l;
        const double sg = src[am] < 0 ? -1.0 : 1.0;
        for (int l = 0; l < n; ++l) U_out[(size_t)c * n + l] = sg * src[l];
        if (sigma_out) sigma_out[c] = std::sqrt(std::max(lam[n - 1 - c], 0.0));
    }
    return SAP_OK;
#undef PCK
}

} // namespace sap
