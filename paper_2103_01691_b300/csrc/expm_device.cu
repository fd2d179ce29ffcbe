// FP64 matrix exponential on the device.
//
// The HKMP scheme (section 4.4) takes one order-two Magnus step per time
// step: u_{n+1} = exp(tau A(t_n + tau/2)) u_n (eq. (mag2)), so the d small
// exponentials change every step and, as the paper notes for its GPU code,
// must be computed on the GPU as well.  This file computes
//   E = exp(z (A + f B)),  A, B real n x n (B optional), z complex,
// by scaling and squaring a truncated Taylor series:
//   X = z (A + f B) / 2^s  with ||X||_1 <= 1 (s from a bound on ||z(A + fB)||_1),
//   T = sum_{k=0}^{18} X^k / k!,   E = T^(2^s).
// With ||X||_1 <= 1 the truncation error is at most sum_{k>18} 1/k! < 1e-17
// in the 1-norm, below FP64 rounding.  T is evaluated by the
// Paterson-Stockmeyer scheme with X^4 as the Horner variable:
//   T = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + X^4 B_4))),
//   B_j = sum_{i<4} X^i / (4j+i)!  (j < 4),  B_4 = I/16! + X/17! + X^2/18!,
// which takes 3 products for X^2, X^3, X^4 and 4 Horner products, plus s
// squarings.  The products are plain complex FP64 GEMMs (cuBLAS ZGEMM); the
// combinations are element-wise kernels.  Matrices are row-major.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

#include "internal.h"

namespace mm {

namespace {

__global__ void form_x(int64_t nn, const double *A, const double *B, double f, double zr, double zi,
                       double2 *X)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nn; q += int64_t(gridDim.x) * blockDim.x) {
        const double a = A[q] + (B ? f * B[q] : 0.0);
        X[q] = make_double2(zr * a, zi * a);
    }
}

// out = c0 I + c1 X + c2 X2 + c3 X3 (X2, X3 may be null when their c is 0)
__global__ void combo(int n, double c0, double c1, double c2, double c3, const double2 *X, const double2 *X2,
                      const double2 *X3, double2 *out)
{
    const int64_t nn = int64_t(n) * n;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nn; q += int64_t(gridDim.x) * blockDim.x) {
        double2 v = make_double2(c1 * X[q].x, c1 * X[q].y);
        if (X2) {
            v.x += c2 * X2[q].x;
            v.y += c2 * X2[q].y;
        }
        if (X3) {
            v.x += c3 * X3[q].x;
            v.y += c3 * X3[q].y;
        }
        if (q / n == q % n) v.x += c0;
        out[q] = v;
    }
}

// column sums of |A + f B| (row-major: column j sums over rows i)
__global__ void col_abs_sums(int n, const double *A, const double *B, double f, double *out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(A[int64_t(i) * n + j] + (B ? f * B[int64_t(i) * n + j] : 0.0));
        out[j] = s;
    }
}

int blocks_for(int64_t work) { return int(std::min<int64_t>((work + 255) / 256, 1184)); }

// C = P Q for row-major n x n matrices, as the column-major product Q^T-view times P^T-view
cublasStatus_t gemm(cublasHandle_t h, int n, const double2 *P, const double2 *Q, double2 *C, bool accumulate)
{
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
    const cuDoubleComplex beta = make_cuDoubleComplex(accumulate ? 1.0 : 0.0, 0.0);
    return cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, reinterpret_cast<const cuDoubleComplex *>(Q), n,
                       reinterpret_cast<const cuDoubleComplex *>(P), n, &beta, reinterpret_cast<cuDoubleComplex *>(C),
                       n);
}

}  // namespace

void expm_workspace_destroy(ExpmWorkspace *w)
{
    if (!w) return;
    for (auto &b : w->buf)
        if (b) {
            cudaFree(b);
            b = nullptr;
        }
    if (w->sums) cudaFree(w->sums);
    w->sums = nullptr;
    if (w->blas) cublasDestroy(static_cast<cublasHandle_t>(w->blas));
    w->blas = nullptr;
    w->n = 0;
}

cudaError_t expm_workspace_init(ExpmWorkspace *w, int n)
{
    if (w->n >= n && w->blas) return cudaSuccess;
    expm_workspace_destroy(w);
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    w->blas = h;
    for (auto &b : w->buf) {
        cudaError_t e = cudaMalloc(&b, sizeof(double2) * size_t(n) * n);
        if (e != cudaSuccess) {
            b = nullptr;
            expm_workspace_destroy(w);
            return e;
        }
    }
    cudaError_t e = cudaMalloc(&w->sums, sizeof(double) * size_t(n));
    if (e != cudaSuccess) {
        w->sums = nullptr;
        expm_workspace_destroy(w);
        return e;
    }
    w->n = n;
    return cudaSuccess;
}

cudaError_t expm_norm1_device(ExpmWorkspace *w, int n, const double *A, const double *B, double f, double *norm,
                              cudaStream_t s)
{
    col_abs_sums<<<blocks_for(n), 256, 0, s>>>(n, A, B, f, w->sums);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<double> h(size_t(n), 0.0);
    e = cudaMemcpyAsync(h.data(), w->sums, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    double m = 0.0;
    for (double v : h) m = std::max(m, v);
    *norm = m;
    return cudaSuccess;
}

cudaError_t expm_device(ExpmWorkspace *w, int n, const double *A, const double *B, double f, double zr, double zi,
                        double norm_bound, double2 *E, cudaStream_t s)
{
    if (w->n < n || !w->blas) return cudaErrorInvalidValue;
    cublasHandle_t h = static_cast<cublasHandle_t>(w->blas);
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const double za = std::hypot(zr, zi) * norm_bound;
    int sq = 0;
    if (za > 1.0) sq = int(std::ceil(std::log2(za)));
    while (std::ldexp(za, -sq) > 1.0) ++sq;  // guard the rounding of log2
    const double scale = std::ldexp(1.0, -sq);
    double2 *X = w->buf[0], *X2 = w->buf[1], *X3 = w->buf[2], *X4 = w->buf[3], *T0 = w->buf[4], *T1 = w->buf[5];
    const int64_t nn = int64_t(n) * n;
    const int g = blocks_for(nn);
    form_x<<<g, 256, 0, s>>>(nn, A, B, f, zr * scale, zi * scale, X);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (gemm(h, n, X, X, X2, false) != CUBLAS_STATUS_SUCCESS || gemm(h, n, X2, X, X3, false) != CUBLAS_STATUS_SUCCESS ||
        gemm(h, n, X2, X2, X4, false) != CUBLAS_STATUS_SUCCESS)
        return cudaErrorUnknown;
    double c[19];
    c[0] = 1.0;
    for (int k = 1; k <= 18; ++k) c[k] = c[k - 1] / double(k);
    // T = B_4, then T <- B_j + X^4 T for j = 3, 2, 1, 0
    combo<<<g, 256, 0, s>>>(n, c[16], c[17], c[18], 0.0, X, X2, nullptr, T0);
    count_launch();
    double2 *cur = T0, *nxt = T1;
    for (int j = 3; j >= 0; --j) {
        combo<<<g, 256, 0, s>>>(n, c[4 * j], c[4 * j + 1], c[4 * j + 2], c[4 * j + 3], X, X2, X3, nxt);
        count_launch();
        if (gemm(h, n, X4, cur, nxt, true) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        std::swap(cur, nxt);
    }
    for (int k = 0; k < sq; ++k) {
        double2 *dst = (k + 1 == sq) ? E : nxt;
        if (gemm(h, n, cur, cur, dst, false) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        nxt = cur;
        cur = dst;
    }
    if (cur != E) {
        e = cudaMemcpyAsync(E, cur, sizeof(double2) * size_t(nn), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace mm
