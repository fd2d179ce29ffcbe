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

// ---- imaginary z: cos / sin in real arithmetic, batched over several f ----------
//
// For real M and z = i w, exp(z M) = cos(w M) + i sin(w M).  With
// X = w M / 2^s (||X||_1 <= theta, theta = 1 or 2) and Y = X^2:
//   cos X = sum_{j<=9} (-1)^j Y^j / (2j)!,   sin X = X sum_{j<=9} (-1)^j Y^j / (2j+1)!,
// whose truncation errors are below theta^20/20! and theta^21/21! (below
// 1e-18 for theta = 1, 5e-13 for theta = 2).  Each degree-9
// polynomial in Y is evaluated by Paterson-Stockmeyer with Y^3 as the
// Horner variable (2 products each, given Y, Y^2, Y^3), and the angle is
// doubled s times by cos 2a = cos^2 a - sin^2 a, sin 2a = 2 sin a cos a (3
// products each; errors then grow as in a complex squaring).  All products
// are real FP64 GEMMs batched over the f values (gemm_batch below: the FP64
// tensor cores through warp MMA):
// 8 + 3 s real products, against 10 + s complex ones (40 + 4 s real) for
// the general series.

namespace {

// X_k = w (A + f_k B - mu I); f: count device values, or null for the single value f0
__global__ void form_x_batch(int64_t nn, int n, int count, const double *A, const double *B, const double *f,
                             double f0, double mu, double w, double *X)
{
    const int64_t total = nn * count;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = q / nn, e = q % nn;
        X[q] = w * (A[e] + (B ? (f ? f[k] : f0) * B[e] : 0.0) - (e / n == e % n ? mu : 0.0));
    }
}

// out = a0 I + a1 Y + a2 Y2 + a3 Y3 (batched; Y3 may be null when a3 = 0)
__global__ void combo_batch(int n, int count, double a0, double a1, double a2, double a3, const double *Y,
                            const double *Y2, const double *Y3, double *out)
{
    const int64_t nn = int64_t(n) * n, total = nn * count;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t e = q % nn;
        double v = a1 * Y[q] + a2 * Y2[q];
        if (Y3) v += a3 * Y3[q];
        if (e / n == e % n) v += a0;
        out[q] = v;
    }
}

// C <- cos^2 - sin^2, S <- 2 sin cos (from the three products)
__global__ void double_angle(int64_t total, const double *CC, const double *SS, const double *SC, double *C, double *S)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        C[q] = CC[q] - SS[q];
        S[q] = 2.0 * SC[q];
    }
}

// E = (pr + i pi) (C + i S) (S null: real C)
__global__ void interleave(int64_t total, const double *C, const double *S, double pr, double pi, double2 *E)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const double c = C[q], s = S ? S[q] : 0.0;
        E[q] = make_double2(pr * c - pi * s, pr * s + pi * c);
    }
}

// C_k = P_k Q_k (+ C_k when accumulating) for row-major n x n FP64 matrices, k < count, on the
// FP64 tensor cores (warp MMA m8n8k4; tcgen05 has no FP64 kind).  B300 runs FP64 MMAs at a low
// rate per SM, so the grid is what matters: block (x, y, k) computes the BT x BT tile (y, x) of
// C_k with one warp per 16 x 16 outputs, and BT (32, or 16 when 32 would leave SMs idle) is
// chosen so that the launch covers the GPU.  The k-dimension runs in chunks of 32 staged in
// shared memory; each thread loads its part of the next chunk into registers while the MMAs of
// the current one run.
constexpr int kGemmK = 32;

__device__ __forceinline__ void dmma_884(double (&d)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

template <int BT>
__global__ void __launch_bounds__(BT * BT / 8) dgemm_batched_kernel(int n, const double *__restrict__ P,
                                                                      const double *__restrict__ Q,
                                                                      double *__restrict__ C, int accumulate)
{
    constexpr int NT = BT * BT / 8;             // one warp per 16 x 16 outputs
    constexpr int LP = BT * kGemmK / NT;         // elements of each operand a thread stages per chunk
    __shared__ double sP[BT][kGemmK + 1];
    __shared__ double sQ[kGemmK][BT + 1];
    const int64_t off = int64_t(blockIdx.z) * n * n;
    P += off;
    Q += off;
    C += off;
    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    const int g = lane / 4, q = lane % 4;  // fragment row / column group of this lane
    const int wi = (warp % (BT / 16)) * 16, wc = (warp / (BT / 16)) * 16;
    const int i0 = int(blockIdx.y) * BT, j0 = int(blockIdx.x) * BT;
    double acc[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
    double rp[LP], rq[LP];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LP; ++r) {
            const int e = t + NT * r;
            const int pk = e % kGemmK, pi = e / kGemmK;  // P: a row's consecutive k
            const int qc = e % BT, qk = e / BT;          // Q: a k-row's consecutive columns
            const int i = i0 + pi, kp = k0 + pk, kq = k0 + qk, j = j0 + qc;
            rp[r] = (i < n && kp < n) ? P[int64_t(i) * n + kp] : 0.0;
            rq[r] = (kq < n && j < n) ? Q[int64_t(kq) * n + j] : 0.0;
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < n; k0 += kGemmK) {
#pragma unroll
        for (int r = 0; r < LP; ++r) {
            const int e = t + NT * r;
            sP[e / kGemmK][e % kGemmK] = rp[r];
            sQ[e / BT][e % BT] = rq[r];
        }
        __syncthreads();
        if (k0 + kGemmK < n) fetch(k0 + kGemmK);
#pragma unroll
        for (int kk = 0; kk < kGemmK; kk += 4) {
            double a[2], b[2];
#pragma unroll
            for (int ti = 0; ti < 2; ++ti) a[ti] = sP[wi + 8 * ti + g][kk + q];
#pragma unroll
            for (int tj = 0; tj < 2; ++tj) b[tj] = sQ[kk + q][wc + 8 * tj + g];
#pragma unroll
            for (int ti = 0; ti < 2; ++ti)
#pragma unroll
                for (int tj = 0; tj < 2; ++tj) dmma_884(acc[ti][tj], a[ti], b[tj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int ti = 0; ti < 2; ++ti) {
        const int i = i0 + wi + 8 * ti + g;
        if (i >= n) continue;
#pragma unroll
        for (int tj = 0; tj < 2; ++tj)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + wc + 8 * tj + 2 * q + h;
                if (j >= n) continue;
                double *c = C + int64_t(i) * n + j;
                *c = accumulate ? *c + acc[ti][tj][h] : acc[ti][tj][h];
            }
    }
}

cudaError_t gemm_batch(cudaStream_t s, int n, int count, const double *P, const double *Q, double *C,
                       bool accumulate)
{
    if (count < 1 || count > 65535 || n < 1) return cudaErrorInvalidValue;
    int sms = 148;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t t32 = (n + 31) / 32;
    if (int64_t(count) * t32 * t32 >= 2 * int64_t(sms)) {
        dgemm_batched_kernel<32><<<dim3(unsigned(t32), unsigned(t32), unsigned(count)), 128, 0, s>>>(
            n, P, Q, C, accumulate ? 1 : 0);
    } else {
        const unsigned t16 = unsigned((n + 15) / 16);
        dgemm_batched_kernel<16><<<dim3(t16, t16, unsigned(count)), 32, 0, s>>>(n, P, Q, C, accumulate ? 1 : 0);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace

void expm_batch_destroy(ExpmBatch *w)
{
    if (!w) return;
    for (auto &b : w->buf)
        if (b) {
            cudaFree(b);
            b = nullptr;
        }
    if (w->f) cudaFree(w->f);
    w->f = nullptr;
    w->n = w->cap = 0;
}

cudaError_t expm_batch_init(ExpmBatch *w, int n, int cap)
{
    if (w->n >= n && w->cap >= cap) return cudaSuccess;
    expm_batch_destroy(w);
    const size_t bytes = sizeof(double) * size_t(n) * n * size_t(cap);
    for (auto &b : w->buf) {
        cudaError_t e = cudaMalloc(&b, bytes);
        if (e != cudaSuccess) {
            b = nullptr;
            expm_batch_destroy(w);
            return e;
        }
    }
    cudaError_t e = cudaMalloc(&w->f, sizeof(double) * size_t(cap));
    if (e != cudaSuccess) {
        w->f = nullptr;
        expm_batch_destroy(w);
        return e;
    }
    w->n = n;
    w->cap = cap;
    return cudaSuccess;
}

// E_k = sum_j W[k][j] N_j (complex n x n matrices N_j, real weights): each thread holds one
// entry of the `nodes` node matrices and writes that entry of the cnt combinations.
__global__ void combine_nodes(int64_t nn, int cnt, int K, const double *__restrict__ W, const double2 *__restrict__ N,
                              double2 *__restrict__ E)
{
    constexpr int kMax = kInterpNodes;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nn; e += int64_t(gridDim.x) * blockDim.x) {
        double2 v[kMax];
#pragma unroll
        for (int j = 0; j < kMax; ++j) v[j] = j < K ? N[int64_t(j) * nn + e] : make_double2(0.0, 0.0);
        for (int k = 0; k < cnt; ++k) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int j = 0; j < kMax; ++j) {
                if (j >= K) break;
                const double w = __ldg(W + k * K + j);
                re += w * v[j].x;
                im += w * v[j].y;
            }
            E[int64_t(k) * nn + e] = make_double2(re, im);
        }
    }
}

cudaError_t combine_interp_nodes(int n, int cnt, int K, const double *W_dev, const double2 *nodes, double2 *E,
                                 cudaStream_t s)
{
    if (K < 1 || K > kInterpNodes) return cudaErrorInvalidValue;
    const int64_t nn = int64_t(n) * n;
    combine_nodes<<<blocks_for(nn), 256, 0, s>>>(nn, cnt, K, W_dev, nodes, E);
    count_launch();
    return cudaGetLastError();
}

int expm_batch_capacity(int n)
{
    const double per = 8.0 * 8.0 * double(n) * double(n);  // eight real n x n buffers per batch entry
    return int(std::max(1.0, std::min(64.0, 1.0e9 / per)));
}

cudaError_t expm_imag_batched(ExpmBatch *w, int n, const double *A, const double *B, const double *f_host, int count,
                              double wim, double norm_bound, double2 *E, cudaStream_t s, double mu, double theta)
{
    // exp(i w M) = exp(i w mu) exp(i w (M - mu I)): norm_bound bounds ||M - mu I||_1
    if (w->n < n || w->cap < count || count < 1) return cudaErrorInvalidValue;
    if (!(theta >= 1.0 && theta <= 2.0)) return cudaErrorInvalidValue;
    const double za = std::fabs(wim) * norm_bound;
    int sq = 0;
    if (za > theta) sq = int(std::ceil(std::log2(za / theta)));
    while (std::ldexp(za, -sq) > theta) ++sq;
    cudaError_t e = cudaSuccess;
    if (count > 1 && (e = cudaMemcpyAsync(w->f, f_host, sizeof(double) * size_t(count), cudaMemcpyHostToDevice, s)) !=
                         cudaSuccess)
        return e;
    double *X = w->buf[0], *Y = w->buf[1], *Y2 = w->buf[2], *Y3 = w->buf[3], *T0 = w->buf[4], *T1 = w->buf[5],
           *C = w->buf[6], *S = w->buf[7];
    const int64_t nn = int64_t(n) * n, total = nn * count;
    const int g = blocks_for(total);
    form_x_batch<<<g, 256, 0, s>>>(nn, n, count, A, B, count > 1 ? w->f : nullptr, f_host[0], mu, std::ldexp(wim, -sq),
                                   X);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (gemm_batch(s, n, count, X, X, Y, false) != cudaSuccess ||
        gemm_batch(s, n, count, Y, Y, Y2, false) != cudaSuccess ||
        gemm_batch(s, n, count, Y2, Y, Y3, false) != cudaSuccess)
        return cudaErrorUnknown;
    // a[j] = (-1)^j / (2j)! (cos) and (-1)^j / (2j+1)! (sin), j <= 9
    double ac[10], as[10];
    double fact = 1.0;  // k!
    for (int k = 0; k <= 19; ++k) {
        if (k > 0) fact *= double(k);
        const double sgn = ((k / 2) % 2) ? -1.0 : 1.0;
        if (k % 2 == 0) ac[k / 2] = sgn / fact;
        else as[k / 2] = sgn / fact;
    }
    // p(Y) = Q0 + Y3 (Q1 + Y3 (Q2 + a9 Y3)), Q_i = a_{3i} I + a_{3i+1} Y + a_{3i+2} Y2
    auto poly = [&](const double *a, double *out) -> cudaError_t {
        combo_batch<<<g, 256, 0, s>>>(n, count, a[6], a[7], a[8], a[9], Y, Y2, Y3, T0);
        count_launch();
        combo_batch<<<g, 256, 0, s>>>(n, count, a[3], a[4], a[5], 0.0, Y, Y2, nullptr, T1);
        count_launch();
        if (gemm_batch(s, n, count, Y3, T0, T1, true) != cudaSuccess) return cudaErrorUnknown;
        combo_batch<<<g, 256, 0, s>>>(n, count, a[0], a[1], a[2], 0.0, Y, Y2, nullptr, out);
        count_launch();
        if (gemm_batch(s, n, count, Y3, T1, out, true) != cudaSuccess) return cudaErrorUnknown;
        return cudaGetLastError();
    };
    if ((e = poly(ac, C)) != cudaSuccess) return e;
    // the sin polynomial goes into Y2: its last combination reads Y2 element by element in place,
    // and Y2 is not needed after it
    if ((e = poly(as, Y2)) != cudaSuccess) return e;
    if (gemm_batch(s, n, count, X, Y2, S, false) != cudaSuccess) return cudaErrorUnknown;
    // X, Y and Y3 are free now: products of the doublings
    double *CC = X, *SS = Y, *SC = Y3;
    for (int k = 0; k < sq; ++k) {
        // C' = C C - S S, S' = 2 S C (errors grow as in a complex squaring; the shorter
        // C' = 2 C C - I assumes C C + S S = I and lets them grow twice as fast)
        if (gemm_batch(s, n, count, C, C, CC, false) != cudaSuccess ||
            gemm_batch(s, n, count, S, S, SS, false) != cudaSuccess ||
            gemm_batch(s, n, count, S, C, SC, false) != cudaSuccess)
            return cudaErrorUnknown;
        double_angle<<<g, 256, 0, s>>>(total, CC, SS, SC, C, S);
        count_launch();
    }
    interleave<<<g, 256, 0, s>>>(total, C, S, std::cos(wim * mu), std::sin(wim * mu), E);
    count_launch();
    return cudaGetLastError();
}

// ---- HKP propagators on the device (section 4.3) --------------------------------------
//
// M = Psi exp(-i tau H) Phi^W for one direction: H = diag(k + 1/2) + P^T diag(g) P
// with P[l][k] = phi_k(x_l) and g_l = W_l (V_l - x_l^2/2) (host-computed values),
// the exponential by the cos / sin series, then two complex products.
__global__ void add_half_diag(int n, double *H)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        H[int64_t(k) * n + k] += k + 0.5;
}
__global__ void real_to_complex(int64_t total, const double *A, double2 *B)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x)
        B[q] = make_double2(A[q], 0.0);
}

cudaError_t hkp_propagator_device(ExpmWorkspace *wz, ExpmBatch *wb, int m, const double *P_host, const double *GP_host,
                                  const double *fwd_host, double tau, double2 *M, cudaStream_t s)
{
    if (wz->n < m || wb->n < m || wb->cap < 1) return cudaErrorInvalidValue;
    cublasHandle_t h = static_cast<cublasHandle_t>(wz->blas);
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const size_t nn = size_t(m) * m;
    // staging in the batch workspace (real); Psi and Phi^W go to the complex workspace before the
    // exponential, which reuses every real buffer of the batch workspace
    double *P = wb->buf[0], *GP = wb->buf[1], *H = wb->buf[2], *F = wb->buf[3];
    double2 *Bc = wz->buf[0], *Fc = wz->buf[1], *E = wz->buf[4], *T = wz->buf[5];
    cudaError_t e = cudaMemcpyAsync(P, P_host, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && GP_host) e = cudaMemcpyAsync(GP, GP_host, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, fwd_host, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // H = P^T (G P) (symmetric, so the column-major view of the product needs no transpose)
    const double one = 1.0, zero = 0.0;
    if (GP_host) {
        if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, m, m, m, &one, GP, m, P, m, &zero, H, m) != CUBLAS_STATUS_SUCCESS)
            return cudaErrorUnknown;
    } else if ((e = cudaMemsetAsync(H, 0, sizeof(double) * nn, s)) != cudaSuccess) {
        return e;
    }
    add_half_diag<<<blocks_for(m), 256, 0, s>>>(m, H);
    count_launch();
    real_to_complex<<<blocks_for(int64_t(nn)), 256, 0, s>>>(int64_t(nn), P, Bc);
    count_launch();
    real_to_complex<<<blocks_for(int64_t(nn)), 256, 0, s>>>(int64_t(nn), F, Fc);
    count_launch();
    double nrm = 0.0;  // ||H||_1, read back once
    if ((e = expm_norm1_device(wz, m, H, nullptr, 0.0, &nrm, s)) != cudaSuccess) return e;
    if ((e = expm_imag_batched(wb, m, H, nullptr, &zero, 1, -tau, nrm, E, s)) != cudaSuccess) return e;
    // M = Psi (E Phi^W), Psi = P
    if (gemm(h, m, E, Fc, T, false) != CUBLAS_STATUS_SUCCESS || gemm(h, m, Bc, T, M, false) != CUBLAS_STATUS_SUCCESS)
        return cudaErrorUnknown;
    return cudaGetLastError();
}

// ---- real z: the Taylor series in real arithmetic ----------------------------------
//
// For real M and real z the series of expm_device runs on real matrices
// (gemm_batch): X = z M / 2^s, T = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + X^4 B_4))),
// E = T^(2^s).  Squaring keeps the small entries of decaying flows (a
// cosh / sinh split would cancel them).
cudaError_t expm_real_device(ExpmBatch *w, int n, const double *A, const double *B, double f, double z,
                             double norm_bound, double2 *E, cudaStream_t s)
{
    if (w->n < n || w->cap < 1) return cudaErrorInvalidValue;
    const double za = std::fabs(z) * norm_bound;
    int sq = 0;
    if (za > 1.0) sq = int(std::ceil(std::log2(za)));
    while (std::ldexp(za, -sq) > 1.0) ++sq;
    double *X = w->buf[0], *X2 = w->buf[1], *X3 = w->buf[2], *X4 = w->buf[3], *cur = w->buf[4], *nxt = w->buf[5];
    const int64_t nn = int64_t(n) * n;
    const int g = blocks_for(nn);
    form_x_batch<<<g, 256, 0, s>>>(nn, n, 1, A, B, nullptr, f, 0.0, std::ldexp(z, -sq), X);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (gemm_batch(s, n, 1, X, X, X2, false) != cudaSuccess ||
        gemm_batch(s, n, 1, X2, X, X3, false) != cudaSuccess ||
        gemm_batch(s, n, 1, X2, X2, X4, false) != cudaSuccess)
        return cudaErrorUnknown;
    double c[19];
    c[0] = 1.0;
    for (int k = 1; k <= 18; ++k) c[k] = c[k - 1] / double(k);
    combo_batch<<<g, 256, 0, s>>>(n, 1, c[16], c[17], c[18], 0.0, X, X2, nullptr, cur);
    count_launch();
    for (int j = 3; j >= 0; --j) {
        combo_batch<<<g, 256, 0, s>>>(n, 1, c[4 * j], c[4 * j + 1], c[4 * j + 2], c[4 * j + 3], X, X2, X3, nxt);
        count_launch();
        if (gemm_batch(s, n, 1, X4, cur, nxt, true) != cudaSuccess) return cudaErrorUnknown;
        std::swap(cur, nxt);
    }
    for (int k = 0; k < sq; ++k) {
        if (gemm_batch(s, n, 1, cur, cur, nxt, false) != cudaSuccess) return cudaErrorUnknown;
        std::swap(cur, nxt);
    }
    interleave<<<g, 256, 0, s>>>(nn, cur, nullptr, 1.0, 0.0, E);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mm
