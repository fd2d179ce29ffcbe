// CUDA-core (SIMT) mu-mode product in FP64 or FP32: the "plain FP64 GPU
// form" against which the split-precision tensor-core form is compared, and
// the path for the real FP64 heat problem.
//
// Definition 2.1: with left = n_1..n_{mu-1} and right = n_{mu+1}..n_d the
// input is X[r][j][l] and the output Y[r][i][l] = sum_j L[i][j] X[r][j][l].
// Every direction is one strided GEMM on the tensor in place, with no
// permutation between directions (section 5: the direct approach the paper
// prefers over permute + GEMM): rows of the GEMM are the output index i,
// columns the flattened (r, l) pairs.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace mm {
namespace {

template <typename R, bool C>
struct Elem;
template <typename R>
struct Elem<R, false> {
    R v;
    __device__ static Elem zero() { return {R(0)}; }
    __device__ void fma(const Elem &a, const Elem &b) { v += a.v * b.v; }
};
template <typename R>
struct Elem<R, true> {
    R re, im;
    __device__ static Elem zero() { return {R(0), R(0)}; }
    __device__ void fma(const Elem &a, const Elem &b)
    {
        re += a.re * b.re - a.im * b.im;
        im += a.re * b.im + a.im * b.re;
    }
};

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// One CTA computes a BM x BN tile of Y for rows i0.. and columns c0..;
// thread (tx, ty) owns rows ty + 16 a and columns tx + 16 b, a, b < 4.
template <typename R, bool C>
__global__ void __launch_bounds__(NT) simt_mode_kernel(int64_t left, int64_t n, int64_t right, int64_t m,
                                                       const Elem<R, C> *__restrict__ L,
                                                       const Elem<R, C> *__restrict__ X,
                                                       Elem<R, C> *__restrict__ Y)
{
    using E = Elem<R, C>;
    __shared__ E sL[BK][BM + 1];
    __shared__ E sX[BK][BN + 1];
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int64_t i0 = int64_t(blockIdx.y) * BM;
    const int64_t c0 = int64_t(blockIdx.x) * BN;
    const int64_t ncols = left * right;
    const bool fiber_contig = (left == 1);
    E acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = E::zero();

    for (int64_t k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
        for (int q = 0; q < (BK * BM) / NT; ++q) {
            const int e = t + NT * q;
            const int kk = e % BK, ii = e / BK;  // consecutive threads walk j (row-major L)
            const int64_t i = i0 + ii, j = k0 + kk;
            sL[kk][ii] = (i < m && j < n) ? L[i * n + j] : E::zero();
        }
#pragma unroll
        for (int q = 0; q < (BK * BN) / NT; ++q) {
            const int e = t + NT * q;
            int kk, cc;
            if (fiber_contig) { kk = e % BK; cc = e / BK; }  // j contiguous in memory
            else { cc = e % BN; kk = e / BN; }               // l contiguous in memory
            const int64_t c = c0 + cc, j = k0 + kk;
            E v = E::zero();
            if (c < ncols && j < n) {
                const int64_t r = c / left, l = c - r * left;
                v = X[(r * n + j) * left + l];
            }
            sX[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            E a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = sL[kk][ty + 16 * q];
                b[q] = sX[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q].fma(a[p], b[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t i = i0 + ty + 16 * p;
        if (i >= m) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t c = c0 + tx + 16 * q;
            if (c >= ncols) continue;
            const int64_t r = c / left, l = c - r * left;
            Y[(r * m + i) * left + l] = acc[p][q];
        }
    }
}

// Small products (fewer 64 x 64 tiles than two per SM): 16 x 16 tiles, one output per thread,
// so that more SMs share the work (B300's FP64 rate per SM is low).  Each output accumulates
// over j in the same order as in simt_mode_kernel.
constexpr int SB = 16;
template <typename R, bool C>
__global__ void __launch_bounds__(SB * SB) simt_mode_kernel_small(int64_t left, int64_t n, int64_t right, int64_t m,
                                                                  const Elem<R, C> *__restrict__ L,
                                                                  const Elem<R, C> *__restrict__ X,
                                                                  Elem<R, C> *__restrict__ Y)
{
    using E = Elem<R, C>;
    __shared__ E sL[SB][SB + 1];  // [k][row]
    __shared__ E sX[SB][SB + 1];  // [k][column]
    const int t = threadIdx.x, tx = t % SB, ty = t / SB;
    const int64_t i0 = int64_t(blockIdx.y) * SB, c0 = int64_t(blockIdx.x) * SB;
    const int64_t ncols = left * right;
    const bool fiber_contig = (left == 1);
    E acc = E::zero();
    for (int64_t k0 = 0; k0 < n; k0 += SB) {
        {
            const int64_t i = i0 + ty, j = k0 + tx;  // consecutive threads walk j (row-major L)
            sL[tx][ty] = (i < m && j < n) ? L[i * n + j] : E::zero();
        }
        {
            int kk, cc;
            if (fiber_contig) { kk = tx; cc = ty; }  // j contiguous in memory
            else { cc = tx; kk = ty; }               // l contiguous in memory
            const int64_t c = c0 + cc, j = k0 + kk;
            E v = E::zero();
            if (c < ncols && j < n) {
                const int64_t r = c / left, l = c - r * left;
                v = X[(r * n + j) * left + l];
            }
            sX[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SB; ++kk) acc.fma(sL[kk][ty], sX[kk][tx]);
        __syncthreads();
    }
    const int64_t i = i0 + ty, c = c0 + tx;
    if (i < m && c < ncols) {
        const int64_t r = c / left, l = c - r * left;
        Y[(r * m + i) * left + l] = acc;
    }
}

// ---- FP64 on the tensor cores (legacy warp MMA m8n8k4, the only FP64 MMA form) -------
//
// D (8 x 8) += A (8 x 4) B (4 x 8) per instruction: lane t holds A[t/4][t%4], B[t%4][t/4] and
// D[t/4][2 (t%4)], D[t/4][2 (t%4) + 1].  One CTA of 8 warps computes a 64 x 64 tile of Y (rows i,
// columns c = (r, l)); warp w covers rows 16 (w % 4) .. + 15 and columns 32 (w / 4) .. + 31, as
// 2 x 4 MMA tiles.  Complex data take four real products per tile and k-step.
__device__ __forceinline__ void dmma_8x8x4(double (&d)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

template <bool C>
__global__ void __launch_bounds__(NT) dmma_mode_kernel(int64_t left, int64_t n, int64_t right, int64_t m,
                                                       const double *__restrict__ L, const double *__restrict__ X,
                                                       double *__restrict__ Y)
{
    constexpr int NC = C ? 2 : 1;  // real and imaginary planes
    __shared__ double sL[NC][BM][BK + 1];
    __shared__ double sX[NC][BK][BN + 1];
    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    const int g = lane / 4, q = lane % 4;
    const int wi = (warp % 4) * 16, wc = (warp / 4) * 32;
    const int64_t i0 = int64_t(blockIdx.y) * BM;
    const int64_t c0 = int64_t(blockIdx.x) * BN;
    const int64_t ncols = left * right;
    const bool fiber_contig = (left == 1);
    double acc[NC][2][4][2];  // [plane][row tile][column tile][2 values]
#pragma unroll
    for (int p = 0; p < NC; ++p)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[p][a][b][0] = acc[p][a][b][1] = 0.0;

    for (int64_t k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
        for (int s = 0; s < (BK * BM) / NT; ++s) {
            const int e = t + NT * s;
            const int kk = e % BK, ii = e / BK;
            const int64_t i = i0 + ii, j = k0 + kk;
            const bool ok = i < m && j < n;
#pragma unroll
            for (int p = 0; p < NC; ++p) sL[p][ii][kk] = ok ? L[(i * n + j) * NC + p] : 0.0;
        }
#pragma unroll
        for (int s = 0; s < (BK * BN) / NT; ++s) {
            const int e = t + NT * s;
            int kk, cc;
            if (fiber_contig) { kk = e % BK; cc = e / BK; }
            else { cc = e % BN; kk = e / BN; }
            const int64_t c = c0 + cc, j = k0 + kk;
            const bool ok = c < ncols && j < n;
            int64_t src = 0;
            if (ok) {
                const int64_t r = c / left, l = c - r * left;
                src = (r * n + j) * left + l;
            }
#pragma unroll
            for (int p = 0; p < NC; ++p) sX[p][kk][cc] = ok ? X[src * NC + p] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double a[NC][2], b[NC][4];
#pragma unroll
            for (int p = 0; p < NC; ++p) {
#pragma unroll
                for (int ti = 0; ti < 2; ++ti) a[p][ti] = sL[p][wi + 8 * ti + g][kk + q];
#pragma unroll
                for (int tj = 0; tj < 4; ++tj) b[p][tj] = sX[p][kk + q][wc + 8 * tj + g];
            }
#pragma unroll
            for (int ti = 0; ti < 2; ++ti)
#pragma unroll
                for (int tj = 0; tj < 4; ++tj) {
                    if (C) {
                        // re += Lr Xr - Li Xi ; im += Lr Xi + Li Xr
                        dmma_8x8x4(acc[0][ti][tj], a[0][ti], b[0][tj]);
                        dmma_8x8x4(acc[0][ti][tj], -a[NC - 1][ti], b[NC - 1][tj]);
                        dmma_8x8x4(acc[NC - 1][ti][tj], a[0][ti], b[NC - 1][tj]);
                        dmma_8x8x4(acc[NC - 1][ti][tj], a[NC - 1][ti], b[0][tj]);
                    } else {
                        dmma_8x8x4(acc[0][ti][tj], a[0][ti], b[0][tj]);
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int ti = 0; ti < 2; ++ti) {
        const int64_t i = i0 + wi + 8 * ti + g;
        if (i >= m) continue;
#pragma unroll
        for (int tj = 0; tj < 4; ++tj)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t c = c0 + wc + 8 * tj + 2 * q + h;
                if (c >= ncols) continue;
                const int64_t r = c / left, l = c - r * left;
                const int64_t dst = (r * m + i) * left + l;
#pragma unroll
                for (int p = 0; p < NC; ++p) Y[dst * NC + p] = acc[p][ti][tj][h];
            }
    }
}

__device__ __forceinline__ void sincos_of(float x, float &s, float &c) { sincosf(x, &s, &c); }
__device__ __forceinline__ void sincos_of(double x, double &s, double &c) { sincos(x, &s, &c); }

template <typename R>
__global__ void nonlinear_phase_kernel(int64_t count, double tb, Elem<R, true> *psi)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < count;
         q += int64_t(gridDim.x) * blockDim.x) {
        Elem<R, true> v = psi[q];
        // in the state's precision (FP32 for complex64, as in the tensor-core epilogue)
        const R th = R(tb) * (v.re * v.re + v.im * v.im);
        R s, c;
        sincos_of(th, s, c);
        // v * exp(-i th)
        psi[q] = {R(v.re * c + v.im * s), R(v.im * c - v.re * s)};
    }
}

// Adjoint of psi' = psi exp(-i theta), theta = tb |psi|^2, for a real loss
// with gradients g = dJ/dRe + i dJ/dIm:  g = e^{i theta} g' + 2 tb Im(conj(g') psi') psi.
template <typename R>
__global__ void nonlinear_adjoint_kernel(int64_t count, double tb, const Elem<R, true> *psi, Elem<R, true> *g)
{
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < count;
         q += int64_t(gridDim.x) * blockDim.x) {
        const Elem<R, true> p = psi[q], gp = g[q];
        // in the state's precision (FP32 for complex64)
        const R t = R(tb), th = t * (p.re * p.re + p.im * p.im);
        R sn, cs;
        sincos_of(th, sn, cs);
        // psi' = p (cs - i sn)
        const R pr = p.re * cs + p.im * sn, pi = p.im * cs - p.re * sn;
        // Im(conj(g') psi') = g'.re psi'.im - g'.im psi'.re
        const R im = gp.re * pi - gp.im * pr;
        // e^{i th} g' = (cs + i sn) g'
        const R gr = gp.re * cs - gp.im * sn + R(2) * t * im * p.re;
        const R gi = gp.re * sn + gp.im * cs + R(2) * t * im * p.im;
        g[q] = {gr, gi};
    }
}

template <typename T>
__device__ double abs2(const T &v);
template <>
__device__ double abs2<double>(const double &v) { return v * v; }
template <>
__device__ double abs2<float>(const float &v) { return double(v) * v; }
template <>
__device__ double abs2<double2>(const double2 &v) { return v.x * v.x + v.y * v.y; }
template <>
__device__ double abs2<float2>(const float2 &v) { return double(v.x) * v.x + double(v.y) * v.y; }

// |v|^2 with the weight: FP32 data squared in FP32 (its rounding is unbiased), so that a point
// costs one FP64 operation, the fused multiply-add with its weight; FP64 data in FP64.
template <typename T>
__device__ __forceinline__ double abs2_weighted(const T &v, double w)
{
    return abs2(v) * w;
}
template <>
__device__ __forceinline__ double abs2_weighted<float2>(const float2 &v, double w)
{
    return double(v.x * v.x + v.y * v.y) * w;
}
template <>
__device__ __forceinline__ double abs2_weighted<float>(const float &v, double w)
{
    return double(v * v) * w;
}

template <typename T>
__global__ void norm2_kernel(int64_t n1, int64_t n2, int64_t n3, const T *u, const double *w1,
                             const double *w2, const double *w3, double *out)
{
    const int64_t N = n1 * n2 * n3;
    double s = 0.0;
    if (!w1) {
        for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < N; q += int64_t(gridDim.x) * blockDim.x)
            s += abs2(u[q]);
    } else {
        // one warp per row (i2, i3) at a time: the row's weight w2 w3 once, then the row's points
        // (no index division per point)
        const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32), rows = n2 * n3;
        const int lane = threadIdx.x & 31;
        for (int64_t r = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32; r < rows; r += warps) {
            const int64_t i2 = r % n2, i3 = r / n2;
            const T *row = u + r * n1;
            double sr = 0.0;
            for (int64_t i1 = lane; i1 < n1; i1 += 32) sr += abs2_weighted(row[i1], w1[i1]);
            s += sr * (w2[i2] * w3[i3]);
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

}  // namespace

cudaError_t simt_mode_product(bool fp64, bool cplx, int64_t left, int64_t n, int64_t right, int64_t m,
                              const void *L, const void *X, void *Y, cudaStream_t s)
{
    const int64_t ncols = left * right;
    dim3 grid(unsigned((ncols + BN - 1) / BN), unsigned((m + BM - 1) / BM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    static int sms = 0;  // SM count of the device, queried once
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const bool small = int64_t(grid.x) * grid.y < 2 * int64_t(sms) && (m + SB - 1) / SB <= 65535;
    const dim3 grid_s(unsigned((ncols + SB - 1) / SB), unsigned((m + SB - 1) / SB));
#define MM_LAUNCH(R, C)                                                                                  \
    do {                                                                                                 \
        if (small)                                                                                       \
            simt_mode_kernel_small<R, C><<<grid_s, SB * SB, 0, s>>>(                                     \
                left, n, right, m, (const Elem<R, C> *)L, (const Elem<R, C> *)X, (Elem<R, C> *)Y);       \
        else                                                                                             \
            simt_mode_kernel<R, C><<<grid, NT, 0, s>>>(left, n, right, m, (const Elem<R, C> *)L,         \
                                                       (const Elem<R, C> *)X, (Elem<R, C> *)Y);          \
    } while (0)
    if (fp64 && cplx) MM_LAUNCH(double, true);
    else if (fp64) MM_LAUNCH(double, false);
    else if (cplx) MM_LAUNCH(float, true);
    else MM_LAUNCH(float, false);
#undef MM_LAUNCH
    count_launch();
    return cudaGetLastError();
}

cudaError_t dmma_mode_product(bool cplx, int64_t left, int64_t n, int64_t right, int64_t m, const void *L,
                              const void *X, void *Y, cudaStream_t s)
{
    const int64_t ncols = left * right;
    dim3 grid(unsigned((ncols + BN - 1) / BN), unsigned((m + BM - 1) / BM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    if (cplx)
        dmma_mode_kernel<true><<<grid, NT, 0, s>>>(left, n, right, m, (const double *)L, (const double *)X,
                                                  (double *)Y);
    else
        dmma_mode_kernel<false><<<grid, NT, 0, s>>>(left, n, right, m, (const double *)L, (const double *)X,
                                                   (double *)Y);
    count_launch();
    return cudaGetLastError();
}

cudaError_t simt_nonlinear_phase(bool fp64, int64_t count, double tb, void *psi, cudaStream_t s)
{
    const int blocks = int((count + 255) / 256 < 148 * 16 ? (count + 255) / 256 : 148 * 16);
    if (fp64) nonlinear_phase_kernel<double><<<blocks, 256, 0, s>>>(count, tb, (Elem<double, true> *)psi);
    else nonlinear_phase_kernel<float><<<blocks, 256, 0, s>>>(count, tb, (Elem<float, true> *)psi);
    count_launch();
    return cudaGetLastError();
}

cudaError_t simt_nonlinear_adjoint(bool fp64, int64_t count, double tb, const void *psi, void *g, cudaStream_t s)
{
    const int blocks = int((count + 255) / 256 < 148 * 16 ? (count + 255) / 256 : 148 * 16);
    if (fp64)
        nonlinear_adjoint_kernel<double><<<blocks, 256, 0, s>>>(count, tb, (const Elem<double, true> *)psi,
                                                                 (Elem<double, true> *)g);
    else
        nonlinear_adjoint_kernel<float><<<blocks, 256, 0, s>>>(count, tb, (const Elem<float, true> *)psi,
                                                                (Elem<float, true> *)g);
    count_launch();
    return cudaGetLastError();
}

// Even/odd folding of a complex64 tensor in the directions of `mask` (bit v: direction v + 1).
// In a folded direction of length n (c = ceil(n/2), h = floor(n/2)), index k < h of the folded
// tensor holds x_k + x_(n-1-k), index c + k holds x_k - x_(n-1-k), and for odd n index h holds
// x_h.  A centrosymmetric matrix E (E_ij = E_(n-1-i, n-1-j)) acts on the folded vector as a
// block-diagonal matrix, so the mu-mode products of a Tucker step run on half-size blocks.
// Each thread takes one orbit of the mirror maps: up to 2^d points read, butterflies in
// registers, 2^d points written.  inverse: the unfold, with the factors 1/2.
constexpr int kMaxFold = 5;  // folded directions at most (orbits of up to 32 points)
struct FoldDims {
    int d;
    int64_t n[kMaxDims], c[kMaxDims], h[kMaxDims], stride[kMaxDims], rep[kMaxDims];
    unsigned mask;
    // the unfold can also add sum |out|^2 w[0][i_1] w[1][i_2] ... over its outputs to *norm2 (FP64;
    // null table: factor 1; norm2 null: no sum)
    const double *w[kMaxDims];
    double *norm2;
};

// The block's sum of s added to *out (every thread of the block calls it).
__device__ void block_sum_add(double s, double *out)
{
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

// The weight of the orbit point whose index in direction v is r[v], or n[v] - 1 - r[v] where bit b
// of sp is set and v = pv[b].
template <typename R>
__device__ __forceinline__ double orbit_weight(const FoldDims &f, const R *r, const int *pv, int m, int sp)
{
    double w = 1.0;
#pragma unroll
    for (int v = 0; v < kMaxDims; ++v) {
        if (v >= f.d || !f.w[v]) continue;
        int64_t i = int64_t(r[v]);
        for (int b = 0; b < m; ++b)
            if (pv[b] == v && ((sp >> b) & 1)) i = f.n[v] - 1 - i;
        w *= f.w[v][i];
    }
    return w;
}

template <bool INV>
__global__ void fold_kernel(FoldDims f, int64_t reps, const float2 *__restrict__ in, float2 *__restrict__ out)
{
    double acc = 0.0;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < reps; t += int64_t(gridDim.x) * blockDim.x) {
        int64_t r[kMaxDims];
        int64_t q = t;
        int pv[kMaxDims], m = 0;  // the directions in which this orbit has a mirror pair
        for (int v = 0; v < f.d; ++v) {
            r[v] = q % f.rep[v];
            q /= f.rep[v];
            if (((f.mask >> v) & 1u) && r[v] < f.h[v]) pv[m++] = v;
        }
        const int cnt = 1 << m;
        float2 buf[1 << kMaxFold];
        // the original index of orbit pattern s (bit b: mirror in direction pv[b]) and the folded
        // index of pattern s (bit b: odd part in direction pv[b])
        auto orig = [&](int sp) {
            int64_t off = 0;
            for (int v = 0; v < f.d; ++v) off += r[v] * f.stride[v];
            for (int b = 0; b < m; ++b)
                if ((sp >> b) & 1) off += (f.n[pv[b]] - 1 - 2 * r[pv[b]]) * f.stride[pv[b]];
            return off;
        };
        auto folded = [&](int sp) {
            int64_t off = 0;
            for (int v = 0; v < f.d; ++v) off += r[v] * f.stride[v];
            for (int b = 0; b < m; ++b)
                if ((sp >> b) & 1) off += f.c[pv[b]] * f.stride[pv[b]];
            return off;
        };
        for (int sp = 0; sp < cnt; ++sp) buf[sp] = INV ? in[folded(sp)] : in[orig(sp)];
        for (int b = 0; b < m; ++b)
            for (int sp = 0; sp < cnt; ++sp)
                if (!((sp >> b) & 1)) {
                    const float2 a = buf[sp], z = buf[sp | (1 << b)];
                    if (INV) {
                        buf[sp] = make_float2(0.5f * (a.x + z.x), 0.5f * (a.y + z.y));
                        buf[sp | (1 << b)] = make_float2(0.5f * (a.x - z.x), 0.5f * (a.y - z.y));
                    } else {
                        buf[sp] = make_float2(a.x + z.x, a.y + z.y);
                        buf[sp | (1 << b)] = make_float2(a.x - z.x, a.y - z.y);
                    }
                }
        for (int sp = 0; sp < cnt; ++sp) out[INV ? orig(sp) : folded(sp)] = buf[sp];
        if (INV && f.norm2)
            for (int sp = 0; sp < cnt; ++sp)
                acc += (double(buf[sp].x) * buf[sp].x + double(buf[sp].y) * buf[sp].y) * orbit_weight(f, r, pv, m, sp);
    }
    if (INV && f.norm2) block_sum_add(acc, f.norm2);
}

// The same for at most three folded directions and 32-bit offsets: the orbit lives in registers.
// Orbit pattern sp (bit b: direction pv[b]) exists where every set bit's direction has a mirror
// pair at this orbit (pm); at the middle index of an odd length the direction has none and its
// butterfly is the identity.
template <int F, bool INV, bool NORM>
__global__ void fold_kernel_reg(FoldDims f, uint32_t reps, int p0, int p1, int p2, const float2 *__restrict__ in,
                                float2 *__restrict__ out)
{
    const int pv[3] = {p0, p1, p2};
    double acc = 0.0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < reps; t += gridDim.x * blockDim.x) {
        uint32_t q = t, base = 0, mir[3], odd[3], rv[kMaxDims], pm = 0;
#pragma unroll
        for (int v = 0; v < kMaxDims; ++v) {
            if (v >= f.d) break;
            const uint32_t rep = uint32_t(f.rep[v]), r = q % rep;
            rv[v] = r;
            q /= rep;
            base += r * uint32_t(f.stride[v]);
#pragma unroll
            for (int b = 0; b < F; ++b)
                if (pv[b] == v) {
                    mir[b] = (uint32_t(f.n[v]) - 1u - 2u * r) * uint32_t(f.stride[v]);
                    odd[b] = uint32_t(f.c[v]) * uint32_t(f.stride[v]);
                    if (r < uint32_t(f.h[v])) pm |= 1u << b;
                }
        }
        // the unfold's weighted norm: the weight of every orbit point (FP64), built as products
        // over the folded directions' weights at r and at the mirror and the other directions'
        double wsp[1 << F];
        if (NORM) {
            double wa[3] = {1.0, 1.0, 1.0}, wm[3] = {1.0, 1.0, 1.0}, wrest = 1.0;
#pragma unroll
            for (int v = 0; v < kMaxDims; ++v) {
                if (v >= f.d) break;
                if (!f.w[v]) continue;
                bool folded_v = false;
#pragma unroll
                for (int b = 0; b < F; ++b)
                    if (pv[b] == v) {
                        folded_v = true;
                        wa[b] = f.w[v][rv[v]];
                        wm[b] = f.w[v][uint32_t(f.n[v]) - 1u - rv[v]];
                    }
                if (!folded_v) wrest *= f.w[v][rv[v]];
            }
            wsp[0] = wrest;
#pragma unroll
            for (int b = 0; b < F; ++b)
#pragma unroll
                for (int sp = (1 << b) - 1; sp >= 0; --sp) {
                    wsp[sp | (1 << b)] = wsp[sp] * wm[b];
                    wsp[sp] *= wa[b];
                }
        }
        float2 buf[1 << F];
#pragma unroll
        for (int sp = 0; sp < (1 << F); ++sp) {
            buf[sp] = make_float2(0.0f, 0.0f);
            if (uint32_t(sp) & ~pm) continue;
            uint32_t off = base;
#pragma unroll
            for (int b = 0; b < F; ++b)
                if ((sp >> b) & 1) off += INV ? odd[b] : mir[b];
            buf[sp] = in[off];
        }
#pragma unroll
        for (int b = 0; b < F; ++b) {
            if (!((pm >> b) & 1u)) continue;
#pragma unroll
            for (int sp = 0; sp < (1 << F); ++sp)
                if (!((sp >> b) & 1)) {
                    const float2 a = buf[sp], z = buf[sp | (1 << b)];
                    const float h = INV ? 0.5f : 1.0f;
                    buf[sp] = make_float2(h * (a.x + z.x), h * (a.y + z.y));
                    buf[sp | (1 << b)] = make_float2(h * (a.x - z.x), h * (a.y - z.y));
                }
        }
#pragma unroll
        for (int sp = 0; sp < (1 << F); ++sp) {
            if (uint32_t(sp) & ~pm) continue;
            uint32_t off = base;
#pragma unroll
            for (int b = 0; b < F; ++b)
                if ((sp >> b) & 1) off += INV ? mir[b] : odd[b];
            out[off] = buf[sp];
            if (NORM)  // |out|^2 in FP32 (its rounding is unbiased), times the FP64 weight
                acc += wsp[sp] * double(buf[sp].x * buf[sp].x + buf[sp].y * buf[sp].y);
        }
    }
    if (NORM) block_sum_add(acc, f.norm2);
}

cudaError_t fold_state(int d, const int64_t *n, unsigned mask, bool inverse, const void *in, void *out, cudaStream_t s,
                       const double *const *w, double *norm2)
{
    if (d < 1 || d > kMaxDims || in == out || __builtin_popcount(mask) > kMaxFold || (norm2 && !inverse))
        return cudaErrorInvalidValue;
    FoldDims f;
    f.d = d;
    f.mask = mask;
    f.norm2 = norm2;
    for (int v = 0; v < kMaxDims; ++v) f.w[v] = (w && v < d) ? w[v] : nullptr;
    int64_t stride = 1, reps = 1;
    for (int v = 0; v < d; ++v) {
        f.n[v] = n[v];
        f.c[v] = (n[v] + 1) / 2;
        f.h[v] = n[v] / 2;
        f.stride[v] = stride;
        f.rep[v] = ((mask >> v) & 1u) ? f.c[v] : n[v];
        stride *= n[v];
        reps *= f.rep[v];
    }
    const int64_t blocks = (reps + 255) / 256 < 148 * 16 ? (reps + 255) / 256 : 148 * 16;
    // the fast form: at most three folded directions, 32-bit offsets
    int pv[3] = {0, 0, 0}, F = 0;
    const bool off32 = stride < (int64_t(1) << 31);
    for (int v = 0; v < d; ++v)
        if ((mask >> v) & 1u) {
            if (F < 3) pv[F] = v;
            ++F;
        }
    if (off32 && F >= 1 && F <= 3) {
        const float2 *i2 = (const float2 *)in;
        float2 *o2 = (float2 *)out;
        const uint32_t r32 = uint32_t(reps);
#define MM_FOLD(FF)                                                                                            \
    (norm2 ? (fold_kernel_reg<FF, true, true><<<unsigned(blocks), 256, 0, s>>>(f, r32, pv[0], pv[1], pv[2], i2, o2), 0) \
     : inverse ? (fold_kernel_reg<FF, true, false><<<unsigned(blocks), 256, 0, s>>>(f, r32, pv[0], pv[1], pv[2], i2, o2), 0) \
               : (fold_kernel_reg<FF, false, false><<<unsigned(blocks), 256, 0, s>>>(f, r32, pv[0], pv[1], pv[2], i2, o2), 0))
        if (F == 1) MM_FOLD(1);
        else if (F == 2) MM_FOLD(2);
        else MM_FOLD(3);
#undef MM_FOLD
    } else if (inverse) {
        fold_kernel<true><<<unsigned(blocks), 256, 0, s>>>(f, reps, (const float2 *)in, (float2 *)out);
    } else {
        fold_kernel<false><<<unsigned(blocks), 256, 0, s>>>(f, reps, (const float2 *)in, (float2 *)out);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t norm2_accumulate(mm_dtype dt, int64_t n1, int64_t n2, int64_t n3, const void *u,
                             const double *w1, const double *w2, const double *w3, double *out,
                             cudaStream_t s)
{
    const int64_t N = n1 * n2 * n3;
    const int blocks = int((N + 255) / 256 < 148 * 8 ? (N + 255) / 256 : 148 * 8);
    switch (dt) {
    case MM_R64: norm2_kernel<double><<<blocks, 256, 0, s>>>(n1, n2, n3, (const double *)u, w1, w2, w3, out); break;
    case MM_R32: norm2_kernel<float><<<blocks, 256, 0, s>>>(n1, n2, n3, (const float *)u, w1, w2, w3, out); break;
    case MM_C128: norm2_kernel<double2><<<blocks, 256, 0, s>>>(n1, n2, n3, (const double2 *)u, w1, w2, w3, out); break;
    default: norm2_kernel<float2><<<blocks, 256, 0, s>>>(n1, n2, n3, (const float2 *)u, w1, w2, w3, out); break;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace mm
