// Split-precision mu-mode product on the tcgen05 tensor cores (sm_103a).
//
// What is computed (Definition 2.1 with a complex n_out x n_in matrix
// E = C + iS):  Y[r][i][l] = sum_j E[i][j] X[r][j][l]  on complex data.
//
// State format between mode products.  The complex FP32 state is held as
// BF16 "pieces": x = x0 + x1 + x2 with x0 = bf16(x), x1 = bf16(x - x0),
// x2 = bf16(x - x0 - x1), which is exact for every normal FP32 x.  The real
// and imaginary parts live in separate planes, so the buffer is
// pieces[c][p][padded tensor] (c = re/im, p = piece).  Every direction is
// padded to a multiple of 16 with zeros, which keeps all TMA boxes aligned;
// the zero padding is invariant under the products (zero matrix rows and
// columns).  The last epilogue writes the pieces of its FP32 result, so a
// chain of mode products never leaves this format until the final merge.
//
// GEMM form.  For every direction the GEMM rows are 128 "points" (the
// non-contracted indices), the contraction runs over (plane c, j), the
// columns over (output part c', row i) of one tile of IT matrix rows:
//   D[pt][c'=re, i] = sum_j Xre[pt][j] C[i][j] + Xim[pt][j] (-S[i][j])
//   D[pt][c'=im, i] = sum_j Xre[pt][j] S[i][j] + Xim[pt][j]   C[i][j]
// The matrix tile is stored as the row blocks [C; S] (2 IT rows): the
// real-plane product is one MMA with N = 2 IT over [C; S]; the imaginary
// plane takes two MMAs with N = IT, -Xim S (the MMA's negate-A bit) into
// the real columns and Xim C into the imaginary ones.  For direction 1 (left == 1) the points are fibers and X is
// K-major in memory; for the other directions the points run along the
// contiguous index l and X is MN-major; both are loaded by TMA as they lie
// in HBM, with no permutation between directions (section 5).
//
// Precision.  The products e_a x_b with a + b <= P-1 (P pieces) are
// accumulated in FP32 in tensor memory; the leading product e0 x0 has an
// accumulator of its own so that the smaller corrections are not rounded
// against the large running sum; the epilogue adds the two in FP32.
// The tensor cores truncate (round toward zero) when they add to an FP32
// accumulator, so with floating BF16 pieces the leading sum carries a bias
// of about half an ulp per addition, which grows linearly over many steps.
// The fixed-point variant (MM_PREC_F16X6, template flag FX) removes it:
//   E_ij = rho_i (e0 + eR),  rho_i a power of two per row chosen so that
//          sum_j (|C_ij| + |S_ij|) / rho_i <= 4096, e0 = rint(E_ij / rho_i),
//   x    = s (x0 + xR),      s a power of two per state tensor chosen so
//          that max |x| / s <= 1024, x0 = rint(x / s),
// and the remainders eR, xR (|.| <= 1/2) are each carried by two FP16
// pieces.  The integer products e0 x0 then sum to integers below 2^24
// (4096 * 2048 * 2 planes), which the FP32 accumulator holds exactly, so
// truncation never acts on the leading sum; only the five correction
// products (about 2^-7 of the result) see it.  The state scale follows the
// state: each epilogue takes its output scale from the maximum that the
// same direction produced one sweep earlier (or from a bound in the first
// sweep) and accumulates the new maximum with atomicMax.
//
// Roles: warp 0 lane 0 issues TMA loads into a ring of stages, warp 1
// allocates tensor memory and its lane 0 issues tcgen05.mma, and the
// remaining (epilogue) warps drain tensor memory (warp w reads lanes
// 32 (w % 4) .. + 31).  The one-SM kernel (tc_mode_kernel) runs 576 threads
// with 16 epilogue warps and 4 stages; the CTA-pair kernel (tc_pair_kernel)
// sets its warps and stages per variant (pair_epi_warps, pair_stages).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mm {

int tc_pieces(mm_prec p)
{
    switch (p) {
    case MM_PREC_BF16X6: return 3;
    case MM_PREC_BF16X3: return 2;
    case MM_PREC_BF16: return 1;
    case MM_PREC_F16X6: return 3;
    case MM_PREC_TF32X3: return 2;
    default: return 0;
    }
}
bool tc_prec(mm_prec p) { return tc_pieces(p) > 0; }
bool tc_fixed(mm_prec p) { return p == MM_PREC_F16X6; }
bool tc_tf32(mm_prec p) { return p == MM_PREC_TF32X3; }
int tc_piece_bytes(mm_prec p) { return tc_tf32(p) ? 4 : 2; }

static inline int64_t round16(int64_t v) { return (v + 15) / 16 * 16; }

// Matrix blocks per piece and row tile: C = Re E and S = Im E.
constexpr int kBlocks = 2;

// ---- host: BF16 pieces of the matrix ----------------------------------------------

// Piece arithmetic shared by the host set-up and the device update kernel
// (tc_matrix_update), so that both produce the same bits.  rint rounds to
// nearest with ties to even (the default rounding mode on the host).

// Round a double to the nearest BF16 value (ties to even), returned as a double.
__host__ __device__ static double bf16_round(double v)
{
    if (v == 0.0 || !isfinite(v)) return 0.0;
    int e = ilogb(v);
    if (e < -126) return 0.0;  // below the BF16 normal range: flush
    double scaled = ldexp(v, 7 - e);  // |scaled| in [128, 256)
    double r = rint(scaled);
    return ldexp(r, e - 7);
}
__host__ __device__ static uint16_t bf16_bits(double exact_bf16_value)
{
    float f = float(exact_bf16_value);
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
#endif
    return uint16_t(u >> 16);
}

// Round a double to the nearest FP16 value (ties to even, subnormals kept).
__host__ __device__ static double f16_round(double v)
{
    if (v == 0.0 || !isfinite(v)) return 0.0;
    const int e = ilogb(v);
    if (e < -14) return rint(ldexp(v, 24)) * ldexp(1.0, -24);  // subnormal grid 2^-24
    return ldexp(rint(ldexp(v, 10 - e)), e - 10);
}
__host__ __device__ static uint16_t f16_bits(double exact)
{
    if (exact == 0.0) return 0;
    const uint16_t sign = exact < 0 ? 0x8000u : 0u;
    const double a = fabs(exact);
    if (a < ldexp(1.0, -14)) return uint16_t(sign | uint16_t(ldexp(a, 24)));
    const int e = ilogb(a);
    const uint16_t mant = uint16_t(ldexp(a, -e) * 1024.0 - 1024.0);
    return uint16_t(sign | uint16_t((e + 15) << 10) | mant);
}

// Round a double to the nearest TF32 value (10 explicit mantissa bits, ties to even; below the
// FP32 normal range: 0), returned as the FP32 bits.
static uint32_t tf32_bits_of(double v)
{
    if (v == 0.0 || !std::isfinite(v)) return 0u;
    const int e = std::ilogb(v);
    if (e < -126) return 0u;
    const float f = float(std::ldexp(std::rint(std::ldexp(v, 10 - e)), e - 10));  // 11 bits: exact in FP32
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

// Fixed-point row scale: the power of two 2^ceil(log2(sum_abs / 4096)) (1 for
// an empty row), by frexp so that host and device agree exactly.
__host__ __device__ static double row_scale(double sum_abs)
{
    if (!(sum_abs > 0.0)) return 1.0;
    int e = 0;
    const double mant = frexp(sum_abs / 4096.0, &e);  // sum / 4096 = mant 2^e, mant in [1/2, 1)
    return ldexp(1.0, mant == 0.5 ? e - 1 : e);
}

// Smallest power of two >= n.
__host__ __device__ static int64_t pow2_at_least(int64_t n)
{
    int64_t p = 1;
    while (p < n) p *= 2;
    return p;
}

// The pieces of one complex entry (C, S) / r: bits[p][0] (C), bits[p][1] (S).
__host__ __device__ static void entry_pieces(double c, double s, double r, int npieces, bool fixed, uint16_t bits[3][2])
{
    double rest[2] = {c, s};
    if (fixed) {  // r is a power of two: its reciprocal and the products are exact
        const double inv = 1.0 / r;
        rest[0] *= inv;
        rest[1] *= inv;
    }
    for (int p = 0; p < npieces; ++p)
        for (int q = 0; q < 2; ++q) {
            double piece;
            if (!fixed) piece = bf16_round(rest[q]);
            else if (p == 0) piece = f16_round(rint(rest[q]));  // integer, exact below 2048
            else piece = f16_round(rest[q]);
            rest[q] -= piece;
            bits[p][q] = fixed ? f16_bits(piece) : bf16_bits(piece);
        }
}

mm_status tc_matrix_host(const double *E, int64_t m, int64_t n, int npieces, bool fixed, TcMatrix *geom,
                         std::vector<uint16_t> &h, std::vector<float> &rho, bool tf32)
{
    if (m < 1 || n < 1 || m > 512 || n > 512) return fail(MM_ERR_SHAPE, "tensor-core matrices need sizes in 1..512");
    TcMatrix M;
    M.n_in = n;
    M.n_out = m;
    M.k_pad = round16(n);
    const int64_t m_pad = round16(m);
    M.ni = int((m_pad + 127) / 128);
    M.it = int(round16((m_pad + M.ni - 1) / M.ni));
    M.npieces = npieces;
    M.fixed = fixed;
    M.tf32 = tf32;
    if (tf32) {
        // two TF32 pieces, one-SM layout [piece][row tile][k-block of 8][C, S][it rows][8 x 4 bytes]
        // (as 16-bit halves, low half first); the same bytes per row as the 16-bit pieces
        if (npieces != 2 || fixed) return fail(MM_ERR_INVALID_ARG, "TF32 matrices take two floating pieces");
        const int64_t kbs = M.k_pad / 8;
        h.assign(size_t(int64_t(npieces) * M.ni * kbs * kBlocks * M.it * 16), 0);
        rho.assign(size_t(M.ni) * M.it, 1.0f);
        for (int64_t i = 0; i < m; ++i) {
            double sum_mod = 0.0;
            const int64_t tile = i / M.it, il = i % M.it;
            for (int64_t j = 0; j < n; ++j) {
                const double c = E[2 * (i * n + j)], sv = E[2 * (i * n + j) + 1];
                sum_mod += std::hypot(c, sv);
                const double val[2] = {c, sv};
                for (int w = 0; w < kBlocks; ++w) {
                    const uint32_t b0 = tf32_bits_of(val[w]);
                    float f0;
                    std::memcpy(&f0, &b0, 4);
                    const uint32_t b1 = tf32_bits_of(val[w] - double(f0));
                    const uint32_t bits[2] = {b0, b1};
                    const int64_t kb = j / 8, jj = j % 8;
                    for (int p = 0; p < npieces; ++p) {
                        const int64_t row = (((int64_t(p) * M.ni + tile) * kbs + kb) * kBlocks + w) * M.it + il;
                        h[size_t(row * 16 + 2 * jj)] = uint16_t(bits[p] & 0xffffu);
                        h[size_t(row * 16 + 2 * jj + 1)] = uint16_t(bits[p] >> 16);
                    }
                }
            }
            M.row_norm = std::max(M.row_norm, sum_mod);
        }
        for (int tile = 0; tile < M.ni; ++tile) {
            int lo = int(kbs), hi = 0;
            for (int p = 0; p < npieces; ++p)
                for (int64_t kb = 0; kb < kbs; ++kb) {
                    const int64_t row0 = (((int64_t(p) * M.ni + tile) * kbs + kb) * kBlocks) * M.it;
                    const uint16_t *blk = h.data() + size_t(row0 * 16);
                    bool any = false;
                    for (int64_t q = 0; q < int64_t(kBlocks) * M.it * 16 && !any; ++q) any = blk[q] != 0;
                    if (any) {
                        lo = std::min(lo, int(kb));
                        hi = std::max(hi, int(kb) + 1);
                    }
                }
            if (lo >= hi) {
                lo = 0;
                hi = 1;
            }
            M.kb_lo[tile] = lo;
            M.kb_hi[tile] = hi;
        }
        *geom = M;
        return MM_OK;
    }
    const int64_t rows = int64_t(npieces) * M.ni * kBlocks * M.it;
    h.assign(size_t(rows * M.k_pad), 0);
    rho.assign(size_t(M.ni) * M.it, 1.0f);
    // the row sums of |C| + |S| by a fixed pairwise tree (zero-padded to a power of two,
    // s[j] += s[j + h] for h = P/2 .. 1): matrix_update_kernel adds in the same order
    const int64_t P = pow2_at_least(n);
    std::vector<double> tree(size_t(P), 0.0);
    for (int64_t i = 0; i < m; ++i) {
        double sum_mod = 0.0;
        std::fill(tree.begin(), tree.end(), 0.0);
        for (int64_t j = 0; j < n; ++j) {
            const double c = E[2 * (i * n + j)], sv = E[2 * (i * n + j) + 1];
            tree[size_t(j)] = std::fabs(c) + std::fabs(sv);
            sum_mod += std::hypot(c, sv);
        }
        for (int64_t h = P / 2; h >= 1; h /= 2)
            for (int64_t j = 0; j < h; ++j) tree[size_t(j)] += tree[size_t(j + h)];
        const double sum_abs = tree[0];
        M.row_norm = std::max(M.row_norm, sum_mod);
        const double r = fixed ? row_scale(sum_abs) : 1.0;
        rho[size_t(i)] = float(r);
        const int64_t tile = i / M.it, il = i % M.it;
        for (int64_t j = 0; j < n; ++j) {
            uint16_t bits[3][2];
            entry_pieces(E[2 * (i * n + j)], E[2 * (i * n + j) + 1], r, npieces, fixed, bits);
            // blocks: 0 = C, 1 = S; stored tile by tile (see TcMatrix)
            const int64_t kb = j / 16, jj = j % 16, kbs = M.k_pad / 16;
            for (int p = 0; p < npieces; ++p)
                for (int w = 0; w < kBlocks; ++w) {
                    const int64_t row = (((int64_t(p) * M.ni + tile) * kbs + kb) * kBlocks + w) * M.it + il;
                    h[size_t(row * 16 + jj)] = bits[p][w];
                }
        }
    }
    // k-block band of each row tile: blocks outside it are exactly zero in
    // every piece, so their products add nothing and are skipped
    const int64_t kbs = M.k_pad / 16;
    for (int tile = 0; tile < M.ni; ++tile) {
        int lo = int(kbs), hi = 0;
        for (int p = 0; p < npieces; ++p)
            for (int64_t kb = 0; kb < kbs; ++kb) {
                const int64_t row0 = (((int64_t(p) * M.ni + tile) * kbs + kb) * kBlocks) * M.it;
                const uint16_t *blk = h.data() + size_t(row0 * 16);
                bool any = false;
                for (int64_t q = 0; q < int64_t(kBlocks) * M.it * 16 && !any; ++q) any = (blk[q] & 0x7fffu) != 0;
                if (any) {
                    lo = std::min(lo, int(kb));
                    hi = std::max(hi, int(kb) + 1);
                }
            }
        if (lo >= hi) {  // an all-zero tile still runs one block (of zeros) to define its accumulators
            lo = 0;
            hi = 1;
        }
        M.kb_lo[tile] = lo;
        M.kb_hi[tile] = hi;
    }
    *geom = M;
    return MM_OK;
}

// The bounded waits' limit and the stage-withholding test hook of a launch, from the environment:
// MM_WAIT_LIMIT_CYCLES (SM clocks, default 4e9, about two seconds) and MM_WITHHOLD_STAGE (the
// stage of each CTA whose loads the producers skip; unset or negative: none).  The hook lets a
// test make a wait run out and check that the launch ends with MM_ERR_TIMEOUT and leaves the
// context usable.
static void wait_hooks(long long *limit, int64_t *withhold)
{
    *limit = 4000000000LL;
    *withhold = -1;
    const char *l = std::getenv("MM_WAIT_LIMIT_CYCLES");
    if (l && l[0]) {
        const long long v = std::atoll(l);
        if (v > 0) *limit = v;
    }
    const char *w = std::getenv("MM_WITHHOLD_STAGE");
    if (w && w[0]) *withhold = std::atoll(w);
}

TcVariant tc_default_variant()
{
    const char *one = std::getenv("MM_TC_1SM");
    if (one && one[0] && !(one[0] == '0' && one[1] == 0)) return kTcOneSM;
    const char *v = std::getenv("MM_PAIR_TILE");
    return (v && std::atoi(v) == 128) ? kTcPair128 : kTcPair64;
}

// Rearrange the pieces for the CTA-pair kernel, which tiles the rows in
// ni2 tiles of it2 rows: per (row tile, k-block) CTA rank r of the pair
// gets, for each piece, the rows r it2/2 .. (r + 1) it2/2 - 1 of the tile as
// three blocks -S, C, S, so that [C; S] and [-S; C] are windows of it2 rows
// at the same offsets in both CTAs; the pieces of one (row tile, k-block,
// rank) are contiguous and arrive in one copy.  Each 32-byte block row holds two 16-byte
// halves, swapped in rows whose bit 2 is set: the order a TMA copy with
// 32-byte swizzling would produce, so a plain copy of 128-byte lines gives
// the MMA its layout.  Also sets the k-block band of every pair row tile.
static void tc_pair_layout(const TcMatrix &M, int64_t tmax, TcMatrix::TcPairTiles &P, const std::vector<uint16_t> &h,
                           std::vector<uint16_t> &h2)
{
    const int64_t kbs = M.k_pad / 16, m_pad = round16(M.n_out);
    P.ni = int((m_pad + tmax - 1) / tmax);
    P.it = int((m_pad + P.ni - 1) / P.ni + 31) / 32 * 32;
    const int64_t half = P.it / 2;
    h2.assign(size_t(int64_t(M.npieces) * P.ni * kbs * 2 * 3 * half * 16), 0);
    for (int tile = 0; tile < P.ni; ++tile) {
        int lo = int(kbs), hi = 0;
        for (int p = 0; p < M.npieces; ++p)
            for (int64_t kb = 0; kb < kbs; ++kb) {
                bool any = false;
                for (int r = 0; r < 2; ++r) {
                    const int64_t blk = (((int64_t(tile) * kbs + kb) * 2 + r) * M.npieces + p) * 3 * half;  // first row
                    for (int b = 0; b < 3; ++b)
                        for (int64_t j = 0; j < half; ++j) {
                            const int64_t i = int64_t(tile) * P.it + r * half + j;  // matrix row
                            if (i >= int64_t(M.ni) * M.it) continue;                 // padding: zero
                            const int w = b == 1 ? 0 : 1;  // C is block 0 of a tile, S block 1
                            const int64_t src =
                                ((((int64_t(p) * M.ni + i / M.it) * kbs + kb) * kBlocks + w) * M.it + i % M.it) * 16;
                            const int64_t row = b * half + j;
                            for (int e = 0; e < 16; ++e) {
                                uint16_t v = h[size_t(src + e)];
                                any = any || (v & 0x7fffu) != 0;
                                if (b == 0 && (v & 0x7fffu)) v ^= 0x8000u;  // -S
                                const int chunk = (e / 8) ^ int((row >> 2) & 1);
                                h2[size_t((blk + row) * 16 + chunk * 8 + e % 8)] = v;
                            }
                        }
                }
                if (any) {
                    lo = std::min(lo, int(kb));
                    hi = std::max(hi, int(kb) + 1);
                }
            }
        if (lo >= hi) {  // an all-zero tile still runs one block (of zeros) to define its accumulators
            lo = 0;
            hi = 1;
        }
        P.kb_lo[tile] = lo;
        P.kb_hi[tile] = hi;
    }
}

mm_status tc_matrix_create(const double *E, int64_t m, int64_t n, int npieces, bool fixed, TcMatrix *out, bool tf32)
{
    TcMatrix M;
    std::vector<uint16_t> h;
    std::vector<float> rho;
    mm_status st = tc_matrix_host(E, m, n, npieces, fixed, &M, h, rho, tf32);
    if (st) return st;
    auto release = [&]() { tc_matrix_destroy(&M); };
    auto upload = [&](void **dst, const void *src, size_t bytes) -> mm_status {
        if (cudaMalloc(dst, bytes) != cudaSuccess) {
            *dst = nullptr;
            release();
            return fail(MM_ERR_OOM, "cudaMalloc of %zu bytes for matrix pieces failed", bytes);
        }
        if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            release();
            return fail(MM_ERR_CUDA, "upload of matrix pieces failed");
        }
        return MM_OK;
    };
    if ((st = upload(&M.pieces, h.data(), h.size() * 2))) return st;
    const int64_t tmax[2] = {64, 128};
    for (int k = 0; k < 2 && !tf32; ++k) {  // TF32 runs on the one-SM kernel only: no pair tilings
        std::vector<uint16_t> h2;
        tc_pair_layout(M, tmax[k], M.pair[k], h, h2);
        if ((st = upload(&M.pair[k].pieces, h2.data(), h2.size() * 2))) return st;
    }
    if (fixed && (st = upload(reinterpret_cast<void **>(&M.rho), rho.data(), rho.size() * sizeof(float)))) return st;
    *out = M;
    return MM_OK;
}

void tc_matrix_destroy(TcMatrix *M)
{
    if (!M) return;
    if (M->pieces) cudaFree(M->pieces);
    for (auto &P : M->pair)
        if (P.pieces) cudaFree(P.pieces);
    if (M->rho) cudaFree(M->rho);
    M->pieces = nullptr;
    for (auto &P : M->pair) P.pieces = nullptr;
    M->rho = nullptr;
}

// ---- device: matrix pieces from a device matrix ----------------------------------

// One block per matrix row i < m: the row scale (one thread sums the row in
// the host's order, so the scale is the one tc_matrix_host picks), then the
// pieces of every entry into the one-SM layout and both pair layouts, at the
// positions tc_matrix_host and tc_pair_layout give them.  Entries of the
// padding are never written and keep the zeros of the matrix's creation.
__global__ void matrix_update_kernel(const double2 *__restrict__ E, int64_t m, int64_t n, int npieces, bool fixed,
                                     int ni, int it, int64_t kbs, uint16_t *pieces, float *rho, uint16_t *pp0,
                                     int it0, uint16_t *pp1, int it1)
{
    const int64_t i = blockIdx.x;
    if (i >= m) return;
    extern __shared__ double absrow[];  // |C_ij| + |S_ij| of the row, zero-padded to a power of two
    __shared__ double r_sh;
    const int64_t P = pow2_at_least(n);
    for (int64_t j = threadIdx.x; j < P; j += blockDim.x)
        absrow[j] = j < n ? fabs(E[i * n + j].x) + fabs(E[i * n + j].y) : 0.0;
    __syncthreads();
    for (int64_t h = P / 2; h >= 1; h /= 2) {  // the host's pairwise tree
        for (int64_t j = threadIdx.x; j < h; j += blockDim.x) absrow[j] += absrow[j + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sum_abs = absrow[0];
        const double r = fixed ? row_scale(sum_abs) : 1.0;
        r_sh = r;
        if (rho) rho[i] = float(r);
    }
    __syncthreads();
    const double r = r_sh;
    const int64_t tile = i / it, il = i % it;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        uint16_t bits[3][2];
        const double2 e = E[i * n + j];
        entry_pieces(e.x, e.y, r, npieces, fixed, bits);
        const int64_t kb = j / 16, jj = j % 16;
        if (pieces)
            for (int p = 0; p < npieces; ++p)
                for (int w = 0; w < kBlocks; ++w) {
                    const int64_t row = (((int64_t(p) * ni + tile) * kbs + kb) * kBlocks + w) * it + il;
                    pieces[row * 16 + jj] = bits[p][w];
                }
        for (int k = 0; k < 2; ++k) {
            uint16_t *pp = k == 0 ? pp0 : pp1;
            const int itk = k == 0 ? it0 : it1;
            if (!pp) continue;
            const int64_t half = itk / 2, tile2 = i / itk, i2 = i % itk, rr = i2 / half, jrow = i2 % half;
            for (int p = 0; p < npieces; ++p) {
                const int64_t blk = (((tile2 * kbs + kb) * 2 + rr) * npieces + p) * 3 * half;
                for (int b = 0; b < 3; ++b) {
                    uint16_t v = b == 1 ? bits[p][0] : bits[p][1];
                    if (b == 0 && (v & 0x7fffu)) v ^= 0x8000u;  // -S
                    const int64_t row = b * half + jrow;
                    const int64_t chunk = (jj / 8) ^ ((row >> 2) & 1);
                    pp[(blk + row) * 16 + chunk * 8 + jj % 8] = v;
                }
            }
        }
    }
}

static const TcMatrix::TcPairTiles *pair_tiles(const TcMatrix &M, TcVariant v);

cudaError_t tc_matrix_update(TcMatrix &M, const double2 *E, cudaStream_t s, const TcVariant *only_for)
{
    if (!M.pieces || !E || (M.fixed && !M.rho)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * size_t(pow2_at_least(M.n_in));
    if (smem > 48 * 1024) return cudaErrorInvalidValue;  // n_in <= 4096
    void *one = M.pieces, *pp0 = M.pair[0].pieces, *pp1 = M.pair[1].pieces;
    if (only_for) {  // the layout the variant's products read: its pair tiling, else the one-SM layout
        const TcMatrix::TcPairTiles *PT = pair_tiles(M, *only_for);
        one = PT ? nullptr : M.pieces;
        pp0 = PT == &M.pair[0] ? M.pair[0].pieces : nullptr;
        pp1 = PT == &M.pair[1] ? M.pair[1].pieces : nullptr;
    }
    matrix_update_kernel<<<unsigned(M.n_out), 128, smem, s>>>(
        E, M.n_out, M.n_in, M.npieces, M.fixed, M.ni, M.it, M.k_pad / 16, static_cast<uint16_t *>(one), M.rho,
        static_cast<uint16_t *>(pp0), M.pair[0].it, static_cast<uint16_t *>(pp1), M.pair[1].it);
    count_launch();
    return cudaGetLastError();
}

void tc_matrix_full_bands(TcMatrix &M)
{
    const int kbs = int(M.k_pad / 16);
    for (int t = 0; t < M.ni; ++t) {
        M.kb_lo[t] = 0;
        M.kb_hi[t] = kbs;
    }
    for (auto &P : M.pair)
        for (int t = 0; t < P.ni; ++t) {
            P.kb_lo[t] = 0;
            P.kb_hi[t] = kbs;
        }
}

// ---- device: splitting, merging -----------------------------------------------------

struct Dims {
    int d;
    int64_t n[kMaxDims];
    int64_t np[kMaxDims];
};

struct Bounds {
    double b[kMaxDims];
};

// Floating BF16 pieces: out[p * stride] = bf16 of what remains after p pieces.
__device__ __forceinline__ void split_bf16(float v, int np, uint16_t *out, int64_t stride)
{
    float r = v;
    for (int p = 0; p < np; ++p) {
        const __nv_bfloat16 b = __float2bfloat16_rn(r);
        out[p * stride] = __bfloat16_as_ushort(b);
        r -= __bfloat162float(b);
    }
}

// Fixed-point FP16 pieces of x on the grid s = 2^es: x / s = h0 + h1 + h2
// with h0 an integer (exact in FP16 below 2048) and h1, h2 the remainder.
// Every subtraction is exact (Sterbenz), so the pieces represent x / s to
// about 2^-22 of the grid unit.
__device__ __forceinline__ void split_fx(float x, int es, uint16_t &b0, uint16_t &b1, uint16_t &b2)
{
    const float xs = ldexpf(x, -es);
    const __half h0 = __float2half_rn(rintf(xs));
    const float r = xs - __half2float(h0);
    const __half h1 = __float2half_rn(r);
    const __half h2 = __float2half_rn(r - __half2float(h1));
    b0 = __half_as_ushort(h0);
    b1 = __half_as_ushort(h1);
    b2 = __half_as_ushort(h2);
}

// The same split for a value already divided by the grid spacing.
__device__ __forceinline__ void split_fx_scaled(float xs, uint16_t &b0, uint16_t &b1, uint16_t &b2)
{
    const __half h0 = __float2half_rn(rintf(xs));
    const float r = xs - __half2float(h0);
    const __half h1 = __float2half_rn(r);
    const __half h2 = __float2half_rn(r - __half2float(h1));
    b0 = __half_as_ushort(h0);
    b1 = __half_as_ushort(h1);
    b2 = __half_as_ushort(h2);
}

// split_fx_scaled of two values at once, the pieces packed as FP16 pairs (x in the low half):
// the same roundings, with paired conversions.
__device__ __forceinline__ void split_fx_pair(float x, float y, uint32_t &p0, uint32_t &p1, uint32_t &p2)
{
    const __half2 h0 = __floats2half2_rn(rintf(x), rintf(y));
    const float2 f0 = __half22float2(h0);
    const float rx = x - f0.x, ry = y - f0.y;
    const __half2 h1 = __floats2half2_rn(rx, ry);
    const float2 f1 = __half22float2(h1);
    const __half2 h2 = __floats2half2_rn(rx - f1.x, ry - f1.y);
    p0 = *reinterpret_cast<const uint32_t *>(&h0);
    p1 = *reinterpret_cast<const uint32_t *>(&h1);
    p2 = *reinterpret_cast<const uint32_t *>(&h2);
}

// Grid exponent for a tensor whose largest magnitude is m: s = 2^es with m / s < 1024.
__device__ __forceinline__ int grid_exponent(float m)
{
    if (!(m > 0.0f) || !(m < 3.0e38f)) return 0;
    int e;
    frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    return e - 10;
}

__global__ void max_abs_kernel(int64_t count, const float2 *__restrict__ u, unsigned *out)
{
    float m = 0.0f;
    // points [head, head + 2 pairs) two per 16-byte load; the first point (when u is not on a
    // 16-byte boundary) and an odd last point one by one
    const int64_t head = count > 0 && (reinterpret_cast<uintptr_t>(u) & 15) ? 1 : 0;
    const int64_t pairs = (count - head) / 2;
    const float4 *u4 = reinterpret_cast<const float4 *>(u + head);
    const int64_t t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x, stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t q = t0; q < pairs; q += stride) {
        const float4 v = u4[q];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    if (t0 == 0 && head) m = fmaxf(m, fmaxf(fabsf(u[0].x), fabsf(u[0].y)));
    if (t0 == 0 && count > head + 2 * pairs) m = fmaxf(m, fmaxf(fabsf(u[count - 1].x), fabsf(u[count - 1].y)));
    // one atomic per block: the warps' maxima meet in shared memory (blockDim.x = 256)
    __shared__ unsigned wmax[8];
    const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x / 32] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned c = __reduce_max_sync(0xffffffffu, threadIdx.x < 8 ? wmax[threadIdx.x] : 0u);
        if (threadIdx.x == 0 && c) atomicMax(out, c);
    }
}

// Logical offset of the first point of padded row r (the padded index over directions 2..d),
// and whether the row lies inside the logical tensor.  I: 32-bit when the padded plane fits.
template <typename I>
__device__ __forceinline__ I row_offset(const Dims &dm, I r, bool &inside)
{
    I lin = 0, mul = I(dm.n[0]);
    inside = true;
    for (int v = 1; v < dm.d; ++v) {
        const I np = I(dm.np[v]);
        const I c = r % np;
        r /= np;
        inside &= c < I(dm.n[v]);
        lin += c * mul;
        mul *= I(dm.n[v]);
    }
    return lin;
}

__device__ __forceinline__ uint4 pack8(const uint16_t (&b)[8])
{
    return make_uint4(uint32_t(b[0]) | (uint32_t(b[1]) << 16), uint32_t(b[2]) | (uint32_t(b[3]) << 16),
                      uint32_t(b[4]) | (uint32_t(b[5]) << 16), uint32_t(b[6]) | (uint32_t(b[7]) << 16));
}

// Reads the logical complex64 tensor, writes all pieces of the padded one.  Each thread takes
// 8 consecutive padded points of a row (the padded first direction is a multiple of 16): one
// index decomposition and one 16-byte store per piece plane for the 8.
template <bool FX, typename I>
__global__ void split_kernel(Dims dm, int64_t plane, int npieces, const float2 *__restrict__ u,
                             uint16_t *__restrict__ pieces, const unsigned *maxw, float *scale_out,
                             unsigned *bound_words, Bounds bounds, int nb)
{
    int es = 0;
    if (FX) {
        const float m = __uint_as_float(*maxw);
        es = grid_exponent(m);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *scale_out = ldexpf(1.0f, es);
            for (int q = 0; q < nb; ++q) {
                const double v = double(m) * bounds.b[q];
                bound_words[q] = __float_as_uint(float(v < 3.0e38 ? v : 3.0e38));
            }
        }
    }
    const I np0 = I(dm.np[0]), n0 = I(dm.n[0]), groups = I(plane / 8);
    for (I g = I(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += I(gridDim.x) * blockDim.x) {
        const I q0 = g * 8, c0 = q0 % np0;
        bool inside;
        const I lin = row_offset<I>(dm, q0 / np0, inside) + c0;
        float2 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = inside && c0 + I(k) < n0 ? u[lin + I(k)] : make_float2(0.f, 0.f);
        if (FX) {
            uint16_t b[6][8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                split_fx(x[k].x, es, b[0][k], b[1][k], b[2][k]);
                split_fx(x[k].y, es, b[3][k], b[4][k], b[5][k]);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) *reinterpret_cast<uint4 *>(pieces + int64_t(c) * plane + q0) = pack8(b[c]);
        } else {
            uint16_t br[3][8], bi[3][8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                split_bf16(x[k].x, npieces, &br[0][k], 8);
                split_bf16(x[k].y, npieces, &bi[0][k], 8);
            }
            for (int p = 0; p < npieces; ++p) {
                *reinterpret_cast<uint4 *>(pieces + int64_t(p) * plane + q0) = pack8(br[p]);
                *reinterpret_cast<uint4 *>(pieces + int64_t(npieces + p) * plane + q0) = pack8(bi[p]);
            }
        }
    }
}

// Sums the pieces back (exact for three BF16 pieces), 8 padded points per thread as in
// split_kernel; padding is skipped.
template <bool FX, typename I>
__global__ void merge_kernel(Dims dm, int64_t plane, int npieces, const uint16_t *__restrict__ pieces,
                             const float *scale, float2 *__restrict__ u)
{
    const float s = FX ? *scale : 1.0f;
    const I np0 = I(dm.np[0]), n0 = I(dm.n[0]), groups = I(plane / 8);
    for (I g = I(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += I(gridDim.x) * blockDim.x) {
        const I q0 = g * 8, c0 = q0 % np0;
        bool inside;
        const I lin = row_offset<I>(dm, q0 / np0, inside) + c0;
        if (!inside || c0 >= n0) continue;
        float re[8], im[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) re[k] = im[k] = 0.f;
        for (int p = npieces - 1; p >= 0; --p) {
            const uint4 wr = *reinterpret_cast<const uint4 *>(pieces + int64_t(p) * plane + q0);
            const uint4 wi = *reinterpret_cast<const uint4 *>(pieces + int64_t(npieces + p) * plane + q0);
            const uint32_t ar[4] = {wr.x, wr.y, wr.z, wr.w}, ai[4] = {wi.x, wi.y, wi.z, wi.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint16_t br = uint16_t(ar[k / 2] >> (16 * (k & 1))), bi = uint16_t(ai[k / 2] >> (16 * (k & 1)));
                if (FX) {
                    re[k] += __half2float(__ushort_as_half(br));
                    im[k] += __half2float(__ushort_as_half(bi));
                } else {
                    re[k] += __bfloat162float(__ushort_as_bfloat16(br));
                    im[k] += __bfloat162float(__ushort_as_bfloat16(bi));
                }
            }
        }
        // pairs of points as one 16-byte store where the pair starts on a 16-byte boundary
        const bool even = (reinterpret_cast<uintptr_t>(u + lin) & 15) == 0;
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            if (even && c0 + I(k + 1) < n0) {
                *reinterpret_cast<float4 *>(u + lin + I(k)) =
                    make_float4(re[k] * s, im[k] * s, re[k + 1] * s, im[k + 1] * s);
            } else {
                if (c0 + I(k) < n0) u[lin + I(k)] = make_float2(re[k] * s, im[k] * s);
                if (c0 + I(k + 1) < n0) u[lin + I(k + 1)] = make_float2(re[k + 1] * s, im[k + 1] * s);
            }
        }
    }
}

// FP32 -> the nearest TF32 value (10 explicit mantissa bits, ties to even), as FP32 bits.
__device__ __forceinline__ uint32_t tf32_rne_bits(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u + 0x0fffu + ((u >> 13) & 1u)) & 0xffffe000u;
}

// The two TF32 pieces of x: x0 = TF32(x), x1 = TF32(x - x0) (the difference is exact in FP32).
__device__ __forceinline__ void split_tf32(float x, uint32_t &b0, uint32_t &b1)
{
    b0 = tf32_rne_bits(x);
    b1 = tf32_rne_bits(x - __uint_as_float(b0));
}

// split_kernel for TF32 pieces: planes [re x0, re x1, im x0, im x1] of 4-byte elements, 8 padded
// points per thread (two 16-byte stores per plane).
template <typename I>
__global__ void split_tf32_kernel(Dims dm, int64_t plane, const float2 *__restrict__ u, uint32_t *__restrict__ pieces)
{
    const I np0 = I(dm.np[0]), n0 = I(dm.n[0]), groups = I(plane / 8);
    for (I g = I(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += I(gridDim.x) * blockDim.x) {
        const I q0 = g * 8, c0 = q0 % np0;
        bool inside;
        const I lin = row_offset<I>(dm, q0 / np0, inside) + c0;
        uint32_t b[4][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 x = inside && c0 + I(k) < n0 ? u[lin + I(k)] : make_float2(0.f, 0.f);
            split_tf32(x.x, b[0][k], b[1][k]);
            split_tf32(x.y, b[2][k], b[3][k]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint4 *dst = reinterpret_cast<uint4 *>(pieces + int64_t(c) * plane + q0);
            dst[0] = make_uint4(b[c][0], b[c][1], b[c][2], b[c][3]);
            dst[1] = make_uint4(b[c][4], b[c][5], b[c][6], b[c][7]);
        }
    }
}

// The sum of the two TF32 pieces (exact in FP32: they span at most 22 bits) back into complex64.
template <typename I>
__global__ void merge_tf32_kernel(Dims dm, int64_t plane, const uint32_t *__restrict__ pieces, float2 *__restrict__ u)
{
    const I np0 = I(dm.np[0]), n0 = I(dm.n[0]), groups = I(plane / 8);
    for (I g = I(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += I(gridDim.x) * blockDim.x) {
        const I q0 = g * 8, c0 = q0 % np0;
        bool inside;
        const I lin = row_offset<I>(dm, q0 / np0, inside) + c0;
        if (!inside || c0 >= n0) continue;
        float v[4][8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint4 *src = reinterpret_cast<const uint4 *>(pieces + int64_t(c) * plane + q0);
            const uint4 w0 = src[0], w1 = src[1];
            const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) v[c][k] = __uint_as_float(w[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (c0 + I(k) < n0) u[lin + I(k)] = make_float2(v[1][k] + v[0][k], v[3][k] + v[2][k]);
    }
}

static Dims make_dims(const TcState &st)
{
    Dims dm;
    dm.d = st.d;
    for (int v = 0; v < kMaxDims; ++v) {
        dm.n[v] = v < st.d ? st.n[v] : 1;
        dm.np[v] = v < st.d ? st.np[v] : 1;
    }
    return dm;
}

static int grid_for(int64_t count)
{
    int64_t b = (count + 255) / 256;
    return int(b < 148 * 32 ? (b > 0 ? b : 1) : 148 * 32);
}

cudaError_t tc_split(const TcState &st, int npieces, bool fixed, const void *u_c64, void *pieces, unsigned *work,
                     float *scale_out, unsigned *bound_words, const double *bounds, int nbounds, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(pieces) & 15) || st.plane % 8) return cudaErrorMisalignedAddress;
    Bounds bd{};
    for (int q = 0; q < nbounds && q < kMaxDims; ++q) bd.b[q] = bounds[q];
    if (fixed) {
        int64_t count = 1;
        for (int v = 0; v < st.d; ++v) count *= st.n[v];
        cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        max_abs_kernel<<<grid_for(count / 2 + 1), 256, 0, s>>>(count, (const float2 *)u_c64, work);
        count_launch();
        if (st.plane < (int64_t(1) << 31))
            split_kernel<true, uint32_t><<<grid_for(st.plane / 8), 256, 0, s>>>(
                make_dims(st), st.plane, npieces, (const float2 *)u_c64, (uint16_t *)pieces, work, scale_out,
                bound_words, bd, nbounds);
        else
            split_kernel<true, int64_t><<<grid_for(st.plane / 8), 256, 0, s>>>(
                make_dims(st), st.plane, npieces, (const float2 *)u_c64, (uint16_t *)pieces, work, scale_out,
                bound_words, bd, nbounds);
    } else {
        if (st.plane < (int64_t(1) << 31))
            split_kernel<false, uint32_t><<<grid_for(st.plane / 8), 256, 0, s>>>(
                make_dims(st), st.plane, npieces, (const float2 *)u_c64, (uint16_t *)pieces, nullptr, nullptr, nullptr,
                bd, 0);
        else
            split_kernel<false, int64_t><<<grid_for(st.plane / 8), 256, 0, s>>>(
                make_dims(st), st.plane, npieces, (const float2 *)u_c64, (uint16_t *)pieces, nullptr, nullptr, nullptr,
                bd, 0);
    }
    count_launch();
    return cudaGetLastError();
}

// The GPE nonlinear phase on a folded F16X6 piece state (even/odd folding in the directions of
// `mask`): each thread takes one orbit of the mirror maps, merges its points' pieces (input scale
// 2^grid_exponent(*max_in), the scale the product before wrote them with), unfolds them into point
// values, applies psi -> psi exp(-i tb |psi|^2) at each point, folds them back and splits them on
// the input's grid, and writes them to `out`.  The phase keeps every point's modulus, so a folded
// value grows by at most 2^f (f folded directions) and in practice hardly at all; the split takes
// values up to 16 times past the grid's bound of 1024 (the products' headroom for their predicted
// scales) and reports larger ones as MM_ERR_RANGE in *err.  Block 0 writes the scale to *s_out,
// which the next product reads as its input scale.
struct PhaseFoldDims {
    int d;
    int64_t n[kMaxDims], c[kMaxDims], h[kMaxDims], pstride[kMaxDims], rep[kMaxDims];
    unsigned mask;
};

__global__ void phase_fold_kernel(PhaseFoldDims g, int64_t reps, int64_t plane, const uint16_t *__restrict__ in,
                                  uint16_t *__restrict__ out, const unsigned *max_in, float *s_out, float tb,
                                  int *err)
{
    const int es = grid_exponent(__uint_as_float(*max_in));
    const float s_in = ldexpf(1.0f, es), inv_out = ldexpf(1.0f, -es);
    if (blockIdx.x == 0 && threadIdx.x == 0) *s_out = s_in;
    bool range_ok = true;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < reps; t += int64_t(gridDim.x) * blockDim.x) {
        int64_t r[kMaxDims], q = t, base = 0;
        int pv[5], m = 0;
        for (int v = 0; v < g.d; ++v) {
            r[v] = q % g.rep[v];
            q /= g.rep[v];
            base += r[v] * g.pstride[v];
            if (((g.mask >> v) & 1u) && r[v] < g.h[v] && m < 5) pv[m++] = v;
        }
        const int cnt = 1 << m;
        float2 z[32];
        int64_t off[32];
        for (int sp = 0; sp < cnt; ++sp) {
            int64_t o = base;
            for (int b = 0; b < m; ++b)
                if ((sp >> b) & 1) o += g.c[pv[b]] * g.pstride[pv[b]];
            off[sp] = o;
            float v2[2];
            for (int c = 0; c < 2; ++c) {
                const float x0 = __half2float(__ushort_as_half(in[(3 * c + 0) * plane + o]));
                const float x1 = __half2float(__ushort_as_half(in[(3 * c + 1) * plane + o]));
                const float x2 = __half2float(__ushort_as_half(in[(3 * c + 2) * plane + o]));
                v2[c] = s_in * (x0 + (x1 + x2));
            }
            z[sp] = make_float2(v2[0], v2[1]);
        }
        // unfold, phase at each point, fold
        for (int b = 0; b < m; ++b)
            for (int sp = 0; sp < cnt; ++sp)
                if (!((sp >> b) & 1)) {
                    const float2 a = z[sp], e = z[sp | (1 << b)];
                    z[sp] = make_float2(0.5f * (a.x + e.x), 0.5f * (a.y + e.y));
                    z[sp | (1 << b)] = make_float2(0.5f * (a.x - e.x), 0.5f * (a.y - e.y));
                }
        for (int sp = 0; sp < cnt; ++sp) {
            const float xr = z[sp].x, xi = z[sp].y;
            float sn, cs;
            sincosf(tb * (xr * xr + xi * xi), &sn, &cs);
            z[sp] = make_float2(xr * cs + xi * sn, xi * cs - xr * sn);
        }
        for (int b = 0; b < m; ++b)
            for (int sp = 0; sp < cnt; ++sp)
                if (!((sp >> b) & 1)) {
                    const float2 a = z[sp], e = z[sp | (1 << b)];
                    z[sp] = make_float2(a.x + e.x, a.y + e.y);
                    z[sp | (1 << b)] = make_float2(a.x - e.x, a.y - e.y);
                }
        for (int sp = 0; sp < cnt; ++sp) {
            uint16_t br[3], bi[3];
            const float xr = z[sp].x * inv_out, xi = z[sp].y * inv_out;
            range_ok &= fabsf(xr) < 16384.0f && fabsf(xi) < 16384.0f;
            split_fx_scaled(xr, br[0], br[1], br[2]);
            split_fx_scaled(xi, bi[0], bi[1], bi[2]);
            for (int p = 0; p < 3; ++p) {
                out[p * plane + off[sp]] = br[p];
                out[(3 + p) * plane + off[sp]] = bi[p];
            }
        }
    }
    if (!range_ok && err) atomicCAS(err, 0, MM_ERR_RANGE);
}

// The same for at most three folded directions and pieces that fit 32-bit offsets: the orbit
// lives in registers.  Orbit pattern sp (bit b: direction pv[b]) exists where every set bit's
// direction has a mirror pair at this orbit (pm); at the middle index of an odd length the
// direction has none and its butterflies are skipped.  Each thread takes the orbits of V
// consecutive points of direction 1 (V pieces per load and store: a warp's access to a plane
// covers 128 contiguous bytes for V = 2), which share pm.
template <int V>
struct PiecesV;
template <>
struct PiecesV<1> {
    using T = uint16_t;
};
template <>
struct PiecesV<2> {
    using T = uint32_t;
};

// sin and cos of the nonlinear phase: by their Taylor series about 0 for |a| <= 1/4 (the first
// omitted terms, a^11 / 11! and a^10 / 10!, are below 3e-13), else sincosf.  The phase tau beta
// |psi|^2 of a step is usually far below 1/4.
__device__ __forceinline__ void sincos_phase(float a, float &sn, float &cs)
{
    if (fabsf(a) <= 0.25f) {
        const float a2 = a * a;
        sn = a * (1.0f + a2 * (-1.0f / 6.0f + a2 * (1.0f / 120.0f + a2 * (-1.0f / 5040.0f + a2 * (1.0f / 362880.0f)))));
        cs = 1.0f + a2 * (-0.5f + a2 * (1.0f / 24.0f + a2 * (-1.0f / 720.0f + a2 * (1.0f / 40320.0f))));
    } else {
        sincosf(a, &sn, &cs);
    }
}

template <int F, int V>
__global__ void __launch_bounds__(256, 4) phase_fold_kernel_reg(PhaseFoldDims g, uint32_t reps, uint32_t plane, int p0, int p1, int p2,
                                       const uint16_t *__restrict__ in, uint16_t *__restrict__ out,
                                       const unsigned *max_in, float *s_out, float tb, int *err)
{
    using T = typename PiecesV<V>::T;
    const int pv[3] = {p0, p1, p2};
    const int es = grid_exponent(__uint_as_float(*max_in));
    const float s_in = ldexpf(1.0f, es), inv_out = ldexpf(1.0f, -es);
    if (blockIdx.x == 0 && threadIdx.x == 0) *s_out = s_in;
    bool range_ok = true;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < reps; t += gridDim.x * blockDim.x) {
        uint32_t q = t, base = 0, odd[3], pm = 0;
        for (int v = 0; v < g.d; ++v) {
            const uint32_t rep = uint32_t(v == 0 ? g.rep[0] / V : g.rep[v]), r = q % rep;
            q /= rep;
            base += (v == 0 ? r * V : r) * uint32_t(g.pstride[v]);
#pragma unroll
            for (int b = 0; b < F; ++b)
                if (pv[b] == v) {
                    odd[b] = uint32_t(g.c[v]) * uint32_t(g.pstride[v]);
                    if ((v == 0 ? r * V : r) < uint32_t(g.h[v])) pm |= 1u << b;
                }
        }
        uint32_t off[1 << F];
        float2 z[1 << F][V];
#pragma unroll
        for (int sp = 0; sp < (1 << F); ++sp) {
#pragma unroll
            for (int j = 0; j < V; ++j) z[sp][j] = make_float2(0.0f, 0.0f);
            off[sp] = 0;
            if (uint32_t(sp) & ~pm) continue;
            uint32_t o = base;
#pragma unroll
            for (int b = 0; b < F; ++b)
                if ((sp >> b) & 1) o += odd[b];
            off[sp] = o;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                T w[3];
#pragma unroll
                for (int p = 0; p < 3; ++p) w[p] = *reinterpret_cast<const T *>(in + (3 * c + p) * plane + o);
                float x[V];
                if constexpr (V >= 2) {  // paired conversions, the same values
                    const __half2 *q0 = reinterpret_cast<const __half2 *>(&w[0]);
                    const __half2 *q1 = reinterpret_cast<const __half2 *>(&w[1]);
                    const __half2 *q2 = reinterpret_cast<const __half2 *>(&w[2]);
#pragma unroll
                    for (int jp = 0; jp < V / 2; ++jp) {
                        const float2 f0 = __half22float2(q0[jp]), f1 = __half22float2(q1[jp]),
                                     f2 = __half22float2(q2[jp]);
                        x[2 * jp] = s_in * (f0.x + (f1.x + f2.x));
                        x[2 * jp + 1] = s_in * (f0.y + (f1.y + f2.y));
                    }
                } else {
                    const uint16_t *h0 = reinterpret_cast<const uint16_t *>(&w[0]);
                    const uint16_t *h1 = reinterpret_cast<const uint16_t *>(&w[1]);
                    const uint16_t *h2 = reinterpret_cast<const uint16_t *>(&w[2]);
#pragma unroll
                    for (int j = 0; j < V; ++j)
                        x[j] = s_in * (__half2float(__ushort_as_half(h0[j])) +
                                       (__half2float(__ushort_as_half(h1[j])) + __half2float(__ushort_as_half(h2[j]))));
                }
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    if (c == 0)
                        z[sp][j].x = x[j];
                    else
                        z[sp][j].y = x[j];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
#pragma unroll
            for (int b = 0; b < F; ++b) {
                if (!((pm >> b) & 1u)) continue;
#pragma unroll
                for (int sp = 0; sp < (1 << F); ++sp)
                    if (!((sp >> b) & 1)) {
                        const float2 a = z[sp][j], e = z[sp | (1 << b)][j];
                        z[sp][j] = make_float2(0.5f * (a.x + e.x), 0.5f * (a.y + e.y));
                        z[sp | (1 << b)][j] = make_float2(0.5f * (a.x - e.x), 0.5f * (a.y - e.y));
                    }
            }
#pragma unroll
            for (int sp = 0; sp < (1 << F); ++sp) {
                const float xr = z[sp][j].x, xi = z[sp][j].y;
                float sn, cs;
                sincos_phase(tb * (xr * xr + xi * xi), sn, cs);
                z[sp][j] = make_float2(xr * cs + xi * sn, xi * cs - xr * sn);
            }
#pragma unroll
            for (int b = 0; b < F; ++b) {
                if (!((pm >> b) & 1u)) continue;
#pragma unroll
                for (int sp = 0; sp < (1 << F); ++sp)
                    if (!((sp >> b) & 1)) {
                        const float2 a = z[sp][j], e = z[sp | (1 << b)][j];
                        z[sp][j] = make_float2(a.x + e.x, a.y + e.y);
                        z[sp | (1 << b)][j] = make_float2(a.x - e.x, a.y - e.y);
                    }
            }
        }
#pragma unroll
        for (int sp = 0; sp < (1 << F); ++sp) {
            if (uint32_t(sp) & ~pm) continue;
            T w[6];
            if constexpr (V >= 2) {  // paired conversions, the same pieces
                uint32_t *u[6];
#pragma unroll
                for (int p = 0; p < 6; ++p) u[p] = reinterpret_cast<uint32_t *>(&w[p]);
#pragma unroll
                for (int jp = 0; jp < V / 2; ++jp) {
                    const float r0 = z[sp][2 * jp].x * inv_out, r1 = z[sp][2 * jp + 1].x * inv_out;
                    const float i0 = z[sp][2 * jp].y * inv_out, i1 = z[sp][2 * jp + 1].y * inv_out;
                    range_ok &= fmaxf(fmaxf(fabsf(r0), fabsf(r1)), fmaxf(fabsf(i0), fabsf(i1))) < 16384.0f;
                    split_fx_pair(r0, r1, u[0][jp], u[1][jp], u[2][jp]);
                    split_fx_pair(i0, i1, u[3][jp], u[4][jp], u[5][jp]);
                }
            } else {
                uint16_t *hw = reinterpret_cast<uint16_t *>(w);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const float xr = z[sp][j].x * inv_out, xi = z[sp][j].y * inv_out;
                    range_ok &= fabsf(xr) < 16384.0f && fabsf(xi) < 16384.0f;
                    split_fx_scaled(xr, hw[0 * V + j], hw[1 * V + j], hw[2 * V + j]);
                    split_fx_scaled(xi, hw[3 * V + j], hw[4 * V + j], hw[5 * V + j]);
                }
            }
#pragma unroll
            for (int p = 0; p < 6; ++p) *reinterpret_cast<T *>(out + p * plane + off[sp]) = w[p];
        }
    }
    if (!range_ok && err) atomicCAS(err, 0, MM_ERR_RANGE);
}

cudaError_t tc_phase_fold(const TcState &st, unsigned mask, const void *in_pieces, void *out_pieces,
                          const unsigned *max_in, float *s_out, double tb, int *err, cudaStream_t s)
{
    if (st.d < 1 || st.d > kMaxDims || !mask || __builtin_popcount(mask) > 5 || in_pieces == out_pieces)
        return cudaErrorInvalidValue;
    PhaseFoldDims g;
    g.d = st.d;
    g.mask = mask;
    int64_t stride = 1, reps = 1;
    for (int v = 0; v < st.d; ++v) {
        const bool fv = (mask >> v) & 1u;
        g.n[v] = st.n[v];
        g.c[v] = (st.n[v] + 1) / 2;
        g.h[v] = st.n[v] / 2;
        g.pstride[v] = stride;
        g.rep[v] = fv ? g.c[v] : st.n[v];
        stride *= st.np[v];
        reps *= g.rep[v];
    }
    const int64_t blocks = (reps + 255) / 256 < 148 * 16 ? (reps + 255) / 256 : 148 * 16;
    int pv[3] = {0, 0, 0}, F = 0;
    const bool off32 = 6 * st.plane < (int64_t(1) << 31);
    for (int v = 0; v < st.d; ++v)
        if ((mask >> v) & 1u) {
            if (F < 3) pv[F] = v;
            ++F;
        }
    if (off32 && F >= 1 && F <= 3) {
        const uint16_t *i16 = (const uint16_t *)in_pieces;
        uint16_t *o16 = (uint16_t *)out_pieces;
        const uint32_t pl = uint32_t(st.plane);
        const float tf = float(tb);
        // two points a thread when every offset of a pair is even (direction 1's range and the
        // padded row even, the plane even, the buffers on 4-byte boundaries) and both points of a
        // pair have the same mirror pairs (direction 1 not folded, or of even length)
        const bool v2 = g.rep[0] % 2 == 0 && (!(mask & 1u) || st.n[0] % 2 == 0) && st.np[0] % 2 == 0 &&
                        st.plane % 2 == 0 && !(reinterpret_cast<uintptr_t>(in_pieces) & 3) &&
                        !(reinterpret_cast<uintptr_t>(out_pieces) & 3);
        const uint32_t r32 = uint32_t(v2 ? reps / 2 : reps);
        const int64_t nb = (int64_t(r32) + 255) / 256 < 148 * 16 ? (int64_t(r32) + 255) / 256 : 148 * 16;
#define MM_PHASE_FOLD(FF, VV)                                                                                  \
    phase_fold_kernel_reg<FF, VV><<<unsigned(nb), 256, 0, s>>>(g, r32, pl, pv[0], pv[1], pv[2], i16, o16, max_in, \
                                                               s_out, tf, err)
        if (v2) {
            if (F == 1) MM_PHASE_FOLD(1, 2);
            else if (F == 2) MM_PHASE_FOLD(2, 2);
            else MM_PHASE_FOLD(3, 2);
        } else {
            if (F == 1) MM_PHASE_FOLD(1, 1);
            else if (F == 2) MM_PHASE_FOLD(2, 1);
            else MM_PHASE_FOLD(3, 1);
        }
#undef MM_PHASE_FOLD
        count_launch();
        return cudaGetLastError();
    }
    phase_fold_kernel<<<unsigned(blocks), 256, 0, s>>>(g, reps, st.plane, (const uint16_t *)in_pieces,
                                                      (uint16_t *)out_pieces, max_in, s_out, float(tb), err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t tc_split_tf32(const TcState &st, const void *u_c64, void *pieces, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(pieces) & 15) || st.plane % 8) return cudaErrorMisalignedAddress;
    if (st.plane < (int64_t(1) << 31))
        split_tf32_kernel<uint32_t><<<grid_for(st.plane / 8), 256, 0, s>>>(make_dims(st), st.plane,
                                                                          (const float2 *)u_c64, (uint32_t *)pieces);
    else
        split_tf32_kernel<int64_t><<<grid_for(st.plane / 8), 256, 0, s>>>(make_dims(st), st.plane,
                                                                         (const float2 *)u_c64, (uint32_t *)pieces);
    count_launch();
    return cudaGetLastError();
}

cudaError_t tc_merge_tf32(const TcState &st, const void *pieces, void *u_c64, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(pieces) & 15) || st.plane % 8) return cudaErrorMisalignedAddress;
    if (st.plane < (int64_t(1) << 31))
        merge_tf32_kernel<uint32_t><<<grid_for(st.plane / 8), 256, 0, s>>>(make_dims(st), st.plane,
                                                                          (const uint32_t *)pieces, (float2 *)u_c64);
    else
        merge_tf32_kernel<int64_t><<<grid_for(st.plane / 8), 256, 0, s>>>(make_dims(st), st.plane,
                                                                         (const uint32_t *)pieces, (float2 *)u_c64);
    count_launch();
    return cudaGetLastError();
}

// out[p][r][b][a] = in[p][r][a][b] for 4-byte elements: each of the `planes` planes (plane elements
// apart) holds R matrices of A x B (B fastest); 32 x 32 tiles through shared memory.
__global__ void swap_last2_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t R, int64_t A,
                                  int64_t B, int planes, int64_t plane)
{
    __shared__ uint32_t t[32][33];
    const int64_t nz = R * planes;
    for (int64_t z = blockIdx.z; z < nz; z += gridDim.z) {
        const int64_t p = z / R, r = z % R;
        const uint32_t *src = in + p * plane + r * A * B;
        uint32_t *dst = out + p * plane + r * A * B;
        const int64_t a0 = int64_t(blockIdx.y) * 32, b0 = int64_t(blockIdx.x) * 32;
        for (int k = threadIdx.y; k < 32; k += blockDim.y) {
            const int64_t a = a0 + k, b = b0 + threadIdx.x;
            if (a < A && b < B) t[k][threadIdx.x] = src[a * B + b];
        }
        __syncthreads();
        for (int k = threadIdx.y; k < 32; k += blockDim.y) {
            const int64_t b = b0 + k, a = a0 + threadIdx.x;
            if (a < A && b < B) dst[b * A + a] = t[threadIdx.x][k];
        }
        __syncthreads();
    }
}

static cudaError_t swap_last2(const void *in, void *out, int64_t R, int64_t A, int64_t B, int planes, int64_t plane,
                              cudaStream_t s)
{
    const int64_t nz = R * planes;
    dim3 grid(unsigned((B + 31) / 32), unsigned((A + 31) / 32), unsigned(nz < 65535 ? nz : 65535));
    if ((B + 31) / 32 > 0x7fffffff || (A + 31) / 32 > 65535) return cudaErrorInvalidConfiguration;
    swap_last2_kernel<<<grid, dim3(32, 8), 0, s>>>((const uint32_t *)in, (uint32_t *)out, R, A, B, planes, plane);
    count_launch();
    return cudaGetLastError();
}

cudaError_t tc_merge(const TcState &st, int npieces, bool fixed, const void *pieces, const float *scale, void *u_c64,
                     cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(pieces) & 15) || st.plane % 8) return cudaErrorMisalignedAddress;
    const bool narrow = st.plane < (int64_t(1) << 31);
    const int grid = grid_for(st.plane / 8);
    if (fixed) {
        if (narrow)
            merge_kernel<true, uint32_t><<<grid, 256, 0, s>>>(make_dims(st), st.plane, npieces,
                                                              (const uint16_t *)pieces, scale, (float2 *)u_c64);
        else
            merge_kernel<true, int64_t><<<grid, 256, 0, s>>>(make_dims(st), st.plane, npieces,
                                                             (const uint16_t *)pieces, scale, (float2 *)u_c64);
    } else {
        if (narrow)
            merge_kernel<false, uint32_t><<<grid, 256, 0, s>>>(make_dims(st), st.plane, npieces,
                                                               (const uint16_t *)pieces, nullptr, (float2 *)u_c64);
        else
            merge_kernel<false, int64_t><<<grid, 256, 0, s>>>(make_dims(st), st.plane, npieces,
                                                              (const uint16_t *)pieces, nullptr, (float2 *)u_c64);
    }
    count_launch();
    return cudaGetLastError();
}

// ---- device: the tensor-core mode product ---------------------------------------------

constexpr int kStages = 4;
constexpr int kBK = 16;             // contraction elements per stage (one MMA K)
constexpr int kTileM = 128;         // points per CTA
constexpr int kDataTileBytes = kTileM * kBK * 2;  // 4 KB per (plane, piece)

struct TcArgs {
    int64_t left, right;    // padded sizes of the fast / slow index groups
    int64_t kp;             // padded contraction length
    int64_t mp;             // padded output length
    int64_t aps;            // 64-point atoms per slab (MN-major)
    int64_t plane_out;      // elements per output plane
    int64_t pairs;          // work items of a CTA pair: (pair of point tiles, row tile)
    int64_t tiles;          // point tiles
    int it, ni, kblocks;
    int kb_lo[8], kb_hi[8];  // k-blocks where the row tile's matrix pieces are not all zero
    int stage_bytes, tx_bytes, e_offset;
    float tb;               // tau * beta for the nonlinear epilogue
    const double2 *pl0, *pl1, *pr0, *pr1;  // point-phase epilogue (TcEpilogue kind 2)
    int64_t ldiv, rdiv;
    // weighted-norm epilogue (TcEpilogue kind 5): real weights of the points, in the point
    // phase's decomposition of (l, r), and of the outputs (zero past each direction's length),
    // and the FP64 sum of |y|^2 w that the launch adds to
    const double *wl0, *wl1, *wr0, *wr1, *wo;
    double *norm2;
    uint16_t *out;
    int *err;
    // bounded waits give up after this many SM clocks (MM_ERR_TIMEOUT)
    long long wait_limit;
    // test hook: the stage (counted over the launch, per CTA) whose loads the producers skip,
    // so that the MMA's wait for it runs out; -1: none
    int64_t withhold;
    // nonlinear epilogues of the GPE adjoint (TcEpilogue kinds 3, 4): the state before the
    // nonlinear stage, complex64 in the padded layout of one piece plane
    float2 *mid_out;
    const float2 *mid_in;
    // chained launches (one launch over a sequence of products): completion counters, one per
    // product, and the count that marks a product complete (one signal per CTA)
    unsigned *done;         // [product]: (CTA, item) signals received
    unsigned *gcnt;         // [product][kChainGroups]: signals received per slab group of the output
    // fixed-point mode
    const float *rho;
    TcScales sc;
};

// Piece pairs (a, b) of e_a x_b with a + b <= NP - 1, leading pair first.
__host__ __device__ constexpr int num_terms(int NP) { return NP == 3 ? 6 : (NP == 2 ? 3 : 1); }
__host__ __device__ constexpr int term_a(int t) { return t == 2 ? 1 : (t == 4 ? 1 : (t == 5 ? 2 : 0)); }
__host__ __device__ constexpr int term_b(int t) { return t == 1 ? 1 : (t == 3 ? 2 : (t == 4 ? 1 : 0)); }

// One problem of a batched CTA-pair launch: its tensor maps (read by TMA from
// global memory; CUtensorMap carries the alignment TMA needs), its kernel
// arguments and its first work item.
// Chained launches track their dependencies per slab group: groups of kChainSlabs consecutive
// values of the slowest index, at most kChainGroups of them (directions up to 512).
constexpr int kChainSlabs = 16, kChainGroups = 32;

struct TcPairProblem {
    CUtensorMap mapX, mapE, mapY;
    TcArgs a;
    int64_t pairs_begin;
    int km;    // chained launches: direction 1 (K-major data) or not
    int prod;  // chained launches: position of the product in the chain
    // chained launches: what completes this product's output, slab group by slab group (one
    // signal per CTA and item for each group its points or rows touch) and as a whole (one signal
    // per CTA and item)
    unsigned g_expect[kChainGroups];
    unsigned tot_target;
    int64_t slab_div;    // direction < d: "right" units per slab (the slowest index)
    int last_dir;        // direction d: the output rows are the slabs
    int hmajor;          // items in row-tile-major order (direction d, so that slabs complete in order)
    int wait_prod;       // product complete before any load of this one (-1: none)
    const unsigned *s_in_max;  // the word whose grid exponent is the input scale (null: read a.sc.s_in)
};

// Pair tile and row tile of item Pl of a problem: point-tile-major (row tile fastest), or, for
// the chained launches' last direction, row-tile-major.
__host__ __device__ __forceinline__ void chain_item(const TcArgs &A, bool hmajor, int64_t Pl, int64_t &pair, int &h)
{
    if (hmajor) {
        const int64_t np = A.pairs / A.ni;
        h = int(Pl / np);
        pair = Pl % np;
    } else {
        pair = Pl / A.ni;
        h = int(Pl % A.ni);
    }
}

// Slab groups [g_lo, g_hi] of the data one CTA of an item reads (reads = true) or writes; empty
// (g_lo > g_hi) when the CTA's tile holds no points.  Direction < d: the slabs of the CTA's points;
// direction d: its k-blocks (read) or its output rows (written).
__host__ __device__ __forceinline__ void chain_groups(const TcPairProblem &R, int64_t pair, int h, int rank,
                                                      bool reads, int &g_lo, int &g_hi)
{
    const TcArgs &A = R.a;
    int64_t s_lo, s_hi;
    if (R.last_dir) {
        if (reads) {
            s_lo = int64_t(A.kb_lo[h]) * 16;
            s_hi = int64_t(A.kb_hi[h]) * 16 - 1;
        } else {
            s_lo = int64_t(h) * A.it;
            s_hi = s_lo + A.it - 1;
            if (s_hi > A.mp - 1) s_hi = A.mp - 1;
        }
    } else {
        const int64_t tile = pair * 2 + rank;
        int64_t u_lo, u_hi;  // "right" units of the tile's points
        if (R.km) {
            u_lo = tile * 128;
            u_hi = u_lo + 127;
            if (u_hi > A.right - 1) u_hi = A.right - 1;
        } else {
            const int64_t a0 = 2 * tile, a1 = a0 + 1;
            u_lo = a0 / A.aps;
            u_hi = a1 / A.aps;
            if (u_hi > A.right - 1) u_hi = A.right - 1;
        }
        if (u_lo > u_hi) {
            g_lo = 1;
            g_hi = 0;
            return;
        }
        s_lo = u_lo / R.slab_div;
        s_hi = u_hi / R.slab_div;
    }
    g_lo = int(s_lo / kChainSlabs);
    g_hi = int(s_hi / kChainSlabs);
}

// The problem of work item P (records sorted by pairs_begin, the first at 0).
__device__ __forceinline__ const TcPairProblem &pair_problem(const TcPairProblem *many, int nprob, int64_t P)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (many[mid].pairs_begin <= P) lo = mid;
        else hi = mid - 1;
    }
    return many[lo];
}

// The same for a role that visits items in increasing order: `at` (start 0) is the record of its
// previous item, and the search moves forward from there (usually not at all, or by one record).
__device__ __forceinline__ const TcPairProblem &pair_problem_next(const TcPairProblem *many, int nprob, int64_t P,
                                                                  int &at)
{
    while (at + 1 < nprob && many[at + 1].pairs_begin <= P) ++at;
    return many[at];
}

constexpr int kEpiWarps = 16;      // four per TMEM lane quarter
constexpr int kThreads = 32 * (2 + kEpiWarps);  // warp 0 TMA, warp 1 TMEM + MMA, then the epilogue warps
constexpr int kChunksPerWarp = 2;  // 16-row chunks each epilogue warp drains (IT <= 128)

// Epilogue of one work item for one thread: its point is row `row` of
// point tile `tile`, and v[q] holds the drained sums of output rows
// i0 = h it + 16 (grp + 4 q) .. i0 + 15 (16 real, then 16 imaginary
// values).  Scales them (fixed point), applies the nonlinear phase (EPI 1),
// tracks the maximum and the range, splits them into pieces and stores.
template <int NP, bool KMAJOR, int EPI, bool FX, int CH, bool TF = false>
__device__ __forceinline__ void epi_store(const TcArgs &a, float (&v)[CH][32], int64_t tile, int h, int row, int grp,
                                          int nchunks, float s_in, float inv_out, float lim, float &local_max,
                                          bool &range_ok)
{
    // this thread's point (MN-major: atoms of 64 points, or 32 with TF32 pieces)
    constexpr int AW = TF ? 32 : 64;
    bool valid;
    int64_t r, l = 0;
    if (KMAJOR) {
        r = tile * kTileM + row;
        valid = r < a.right;
    } else {
        const int64_t atom = int64_t(kTileM / AW) * tile + row / AW;
        r = atom / a.aps;
        l = (atom % a.aps) * AW + row % AW;
        valid = r < a.right && l < a.left;
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        const int ch = grp + 4 * q;
        if (ch >= nchunks || !valid) continue;
        const int64_t i0 = int64_t(h) * a.it + ch * 16;
        if (i0 >= a.mp) continue;
        // scale (fixed point), nonlinear phase, range and maximum, in place; the 16 row scales
        // (powers of two, 64-byte aligned) come in four vector loads
        float g16[16];
        if (FX) {
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                const float4 r4 = __ldg(reinterpret_cast<const float4 *>(a.rho + i0) + k4);
                g16[4 * k4 + 0] = r4.x * s_in;
                g16[4 * k4 + 1] = r4.y * s_in;
                g16[4 * k4 + 2] = r4.z * s_in;
                g16[4 * k4 + 3] = r4.w * s_in;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float xr = v[q][k], xi = v[q][16 + k];
            if (FX) {
                xr *= g16[k];  // exact
                xi *= g16[k];
            }
            if (EPI == 1) {
                const float th = a.tb * (xr * xr + xi * xi);
                float sn, cs;
                sincosf(th, &sn, &cs);
                const float yr = xr * cs + xi * sn, yi = xi * cs - xr * sn;
                xr = yr;
                xi = yi;
            }
            if (FX) {
                const float ar = fabsf(xr), ai = fabsf(xi);
                local_max = fmaxf(local_max, fmaxf(ar, ai));
                range_ok &= ar < lim && ai < lim;
                xr *= inv_out;
                xi *= inv_out;
            }
            v[q][k] = xr;
            v[q][16 + k] = xi;
        }
        // pieces of one value: fixed point (already divided by the grid) or floating BF16
        auto pieces_of = [&](float x, uint16_t *b) {
            if (FX) {
                split_fx_scaled(x, b[0], b[1], b[2]);
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const __nv_bfloat16 h16 = __float2bfloat16_rn(x);
                    b[p] = __bfloat16_as_ushort(h16);
                    x -= __bfloat162float(h16);
                }
            }
        };
        if (TF) {
            // two TF32 pieces, 4 bytes each: K-major, 16 consecutive outputs of one row as two 32-byte
            // stores per (plane, piece); MN-major, one 4-byte store per value and piece
            uint32_t *out32 = reinterpret_cast<uint32_t *>(a.out);
            if (KMAJOR) {
                const int64_t base = r * a.mp + i0;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    uint32_t w[2][2][8];  // [piece][half][value]
#pragma unroll
                    for (int k = 0; k < 16; ++k) split_tf32(v[q][16 * c + k], w[0][k / 8][k % 8], w[1][k / 8][k % 8]);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        st_global_v8(out32 + int64_t(c * 2 + p) * a.plane_out + base, w[p][0]);
                        st_global_v8(out32 + int64_t(c * 2 + p) * a.plane_out + base + 8, w[p][1]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    uint32_t br[2], bi[2];
                    split_tf32(v[q][k], br[0], br[1]);
                    split_tf32(v[q][16 + k], bi[0], bi[1]);
                    const int64_t off = (r * a.mp + i0 + k) * a.left + l;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        out32[int64_t(p) * a.plane_out + off] = br[p];
                        out32[int64_t(2 + p) * a.plane_out + off] = bi[p];
                    }
                }
            }
        } else if (KMAJOR) {
            // 16 consecutive outputs of one row: one 32-byte store per (plane, piece)
            const int64_t base = r * a.mp + i0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t w[3][8];
#pragma unroll
                for (int k2 = 0; k2 < 8; ++k2) {
                    uint16_t b0[3], b1[3];
                    pieces_of(v[q][16 * c + 2 * k2], b0);
                    pieces_of(v[q][16 * c + 2 * k2 + 1], b1);
#pragma unroll
                    for (int p = 0; p < NP; ++p) w[p][k2] = uint32_t(b0[p]) | (uint32_t(b1[p]) << 16);
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) st_global_v8(a.out + int64_t(c * NP + p) * a.plane_out + base, w[p]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint16_t br[3], bi[3];
                pieces_of(v[q][k], br);
                pieces_of(v[q][16 + k], bi);
                const int64_t off = (r * a.mp + i0 + k) * a.left + l;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    a.out[int64_t(p) * a.plane_out + off] = br[p];
                    a.out[int64_t(NP + p) * a.plane_out + off] = bi[p];
                }
            }
        }
    }
}

// Persistent kernel in clusters of two CTAs.  Cluster c processes work
// items P = c, c + #clusters, ...; item P is the row tile h = P % ni of the
// point tiles 2 (P / ni) + rank, rank = 0, 1, so the two CTAs of a cluster
// need the same matrix tiles at the same time and read them through L2
// once between them.  Each CTA loads its own stages (data and the whole
// matrix tile) from this GPU's memory; no CTA touches the other's shared
// memory.  The TMA warp runs ahead across item boundaries; the epilogue warps copy the
// two accumulators into registers, release tensor memory to the MMA warp
// at once, and then scale, split and store while the next item's MMAs run.
template <int NP, bool KMAJOR, int EPI, bool FX, bool TF = false>
__global__ void __launch_bounds__(kThreads, 1)
    tc_mode_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapE, TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * a.stage_bytes);
    uint64_t *empty = full + kStages;
    uint64_t *accf = empty + kStages;
    uint64_t *tmem_empty = accf + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_empty + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint64_t *mma_fin = reinterpret_cast<uint64_t *>(tmem_slot + 2);  // abort: this CTA's MMAs have completed

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // TF: 4-byte pieces, K = 8 per MMA and per k-block (32-byte rows, as the 16-bit pieces' K = 16);
    // an MN-major data tile of 128 points is four 32-point atoms instead of two of 64
    constexpr int kKB = TF ? 8 : kBK;
    constexpr int kAtoms = TF ? 4 : 2, kAtomPoints = 128 / kAtoms, kAtomBytes = kDataTileBytes / kAtoms;
    const int acc_cols = 2 * a.it;
    const int need = NP > 1 ? 2 * acc_cols : acc_cols;
    const uint32_t ncols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);  // released by this CTA's MMA warp
        }
        mbar_init(accf, 1);
        mbar_init(tmem_empty, kEpiWarps);
        mbar_init(mma_fin, 1);
        *abort_flag = 0;
        mbar_fence_init();
        tma_prefetch_desc(&mapX);
        tma_prefetch_desc(&mapE);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // The next kernel of the stream may start its own set-up now; everything below reads or
    // writes data of the previous kernel (input pieces, scale words) only after it has completed.
    if (threadIdx.x == 0) griddep_launch_dependents();
    griddep_wait();
    if (FX && blockIdx.x == 0 && threadIdx.x == 0 && a.sc.zero_next) *a.sc.zero_next = 0u;
    uint32_t armed = 0, armed_ph = 0;  // producer: slots armed, and the parity of their last arming
    const int rank = int(blockIdx.x & 1);
    const int64_t cid = blockIdx.x / 2, nclusters = gridDim.x / 2;
    const int half_rows = a.it / 2;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t gk = 0;  // k-blocks issued by this CTA over all items
            for (int64_t P = cid; P < a.pairs && !*abort_flag; P += nclusters) {
                const int64_t tile = (P / a.ni) * 2 + rank;
                const int h = int(P % a.ni);
                // TMA coordinates of this item's atoms (MN-major: 128-byte rows, 64 points of 16-bit pieces
                // or 32 of TF32), fixed over k
                int ac_l[kAtoms] = {}, ac_r[kAtoms] = {};
                if (!KMAJOR) {
                    for (int q = 0; q < kAtoms; ++q) {
                        const int64_t atom = int64_t(kAtoms) * tile + q;
                        int64_t r = atom / a.aps;
                        if (r > a.right) r = a.right;  // past the end: zero fill
                        ac_r[q] = int(r);
                        ac_l[q] = int((atom % a.aps) * kAtomPoints);
                    }
                }
                // matrix tiles are stored contiguously per (piece, row tile, k-block): 3 it rows of 16
                const int e_row0 = h * a.kblocks * kBlocks * a.it;
                const int e_pstride = a.ni * a.kblocks * kBlocks * a.it;
                const int k_row = int(tile * kTileM);
                for (int kb = a.kb_lo[h]; kb < a.kb_hi[h]; ++kb, ++gk) {
                    const int s = int(gk % kStages);
                    const uint32_t ph = (gk / kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    if (int64_t(gk) == a.withhold) continue;
                    uint8_t *st = smem + s * a.stage_bytes;
                    mbar_arrive_expect_tx(&full[s], uint32_t(a.tx_bytes));
                    armed |= 1u << s;
                    armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
                    for (int c = 0; c < 2; ++c)
                        for (int p = 0; p < NP; ++p) {
                            uint8_t *dst = st + (c * NP + p) * kDataTileBytes;
                            if (KMAJOR) {
                                tma_load_3d(&mapX, &full[s], dst, kb * kKB, k_row, c * NP + p);
                            } else {
                                for (int q = 0; q < kAtoms; ++q)
                                    tma_load_4d(&mapX, &full[s], dst + q * kAtomBytes, ac_l[q], kb * kKB, ac_r[q],
                                                c * NP + p);
                            }
                        }
                    // every matrix block, in two boxes of half the rows each
                    uint8_t *est = st + a.e_offset;
                    for (int p = 0; p < NP; ++p)
                        for (int w = 0; w < kBlocks; ++w)
                            for (int hr = 0; hr < 2; ++hr)
                                tma_load_2d(&mapE, &full[s], est + (p * kBlocks + w) * a.it * 32 + hr * half_rows * 32,
                                            0, p * e_pstride + e_row0 + (kb * kBlocks + w) * a.it + hr * half_rows);
                }
            }
        }
        __syncwarp();  // the role's other lanes wait for it: the warp meets the block barrier converged
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc_full = TF   ? idesc_tf32_f32(kTileM, 2 * a.it, !KMAJOR, false)
                                        : FX ? idesc_f16_f32(kTileM, 2 * a.it, !KMAJOR, false)
                                             : idesc_bf16_f32(kTileM, 2 * a.it, !KMAJOR, false);
            const uint32_t idesc_half = TF   ? idesc_tf32_f32(kTileM, a.it, !KMAJOR, false)
                                        : FX ? idesc_f16_f32(kTileM, a.it, !KMAJOR, false)
                                             : idesc_bf16_f32(kTileM, a.it, !KMAJOR, false);
            auto mma = [&](uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
                if (TF) umma_tf32(d, ad, bd, id, acc);
                else umma_f16(d, ad, bd, id, acc);
            };
            const uint32_t idesc_half_neg = idesc_half | (1u << 13);  // negate A
            uint32_t gk = 0, lt = 0;
            for (int64_t P = cid; P < a.pairs && !*abort_flag; P += nclusters, ++lt) {
                const int h = int(P % a.ni);
                if (lt > 0 && !mbar_wait(tmem_empty, (lt - 1) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                bool started[2] = {false, false};
                for (int kb = a.kb_lo[h]; kb < a.kb_hi[h]; ++kb, ++gk) {
                    const int s = int(gk % kStages);
                    const uint32_t ph = (gk / kStages) & 1u;
                    if (!mbar_wait(&full[s], ph, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + s * a.stage_bytes);
                    const uint32_t est = st + a.e_offset;
                    // real plane: one MMA over the window [C; S] writes (re, im) columns;
                    // imaginary plane: -Xi S into the re columns (negated A), Xi C into the im columns
#pragma unroll
                    for (int t = 0; t < num_terms(NP); ++t) {
                        const int pa = term_a(t), pb = term_b(t);
                        const int acc = (NP > 1 && (pa != 0 || pb != 0)) ? 1 : 0;
                        const uint32_t dcol = tmem + uint32_t(acc * acc_cols);
                        const uint32_t eC = est + (pa * kBlocks + 0) * a.it * 32;
                        const uint32_t eS = est + (pa * kBlocks + 1) * a.it * 32;
                        const uint32_t xre = st + (0 * NP + pb) * kDataTileBytes;
                        const uint32_t xim = st + (1 * NP + pb) * kDataTileBytes;
                        // MN-major: the atoms of a plane tile lie kAtomBytes apart (leading byte offset),
                        // the 8-row groups along k 1024 bytes apart
                        const uint64_t are = KMAJOR ? smem_desc(xre, 16, 256, kSwz32) : smem_desc(xre, kAtomBytes, 1024, kSwz128);
                        const uint64_t aim = KMAJOR ? smem_desc(xim, 16, 256, kSwz32) : smem_desc(xim, kAtomBytes, 1024, kSwz128);
                        mma(dcol, are, smem_desc(eC, 16, 256, kSwz32), idesc_full, started[acc] ? 1u : 0u);
                        started[acc] = true;
                        mma(dcol, aim, smem_desc(eS, 16, 256, kSwz32), idesc_half_neg, 1u);
                        mma(dcol + uint32_t(a.it), aim, smem_desc(eC, 16, 256, kSwz32), idesc_half, 1u);
                    }
                    umma_commit(&empty[s]);
                }
                umma_commit(accf);
            }
            if (*abort_flag) {  // every MMA this thread issued completes before tensor memory is freed
                umma_commit(mma_fin);
                mbar_wait(mma_fin, 0u, nullptr, 0, a.wait_limit);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        const int ew = warp - 2;          // 0 .. kEpiWarps - 1
        const int quarter = warp % 4;     // TMEM lanes 32 quarter .. + 31
        const int grp = ew / 4;           // chunks of 16 rows: grp, grp + 4, ...
        const int row = quarter * 32 + lane;
        const uint32_t tbase = tmem + (uint32_t(quarter * 32) << 16);
        const int nchunks = a.it / 16;
        float s_in = 1.0f, inv_out = 1.0f, lim = 0.0f;
        int es_out = 0;
        if (FX) {
            s_in = *a.sc.s_in;
            es_out = grid_exponent(__uint_as_float(*a.sc.max_prev));
            inv_out = ldexpf(1.0f, -es_out);
            lim = ldexpf(16384.0f, es_out);
            if (blockIdx.x == 0 && ew == 0 && lane == 0) *a.sc.s_out = ldexpf(1.0f, es_out);
        }
        float local_max = 0.0f;
        bool range_ok = true;
        uint32_t lt = 0;
        for (int64_t P = cid; P < a.pairs; P += nclusters, ++lt) {
            const int64_t tile = (P / a.ni) * 2 + rank;
            const int h = int(P % a.ni);
            const bool acc_ready = !*abort_flag && mbar_wait(accf, lt & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit);
            if (!acc_ready) *abort_flag = 1;
            tc_fence_after();
            // drain: up to kChunksPerWarp chunks of 16 rows, real and imaginary, both accumulators summed
            float v[kChunksPerWarp][32];
#pragma unroll
            for (int q = 0; q < kChunksPerWarp; ++q) {
                const int ch = grp + 4 * q;
                if (ch < nchunks) {
                    float t0[16], t1[16];
                    tmem_ld16(tbase + uint32_t(ch * 16), t0);
                    if (NP > 1) tmem_ld16(tbase + uint32_t(acc_cols + ch * 16), t1);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[q][k] = NP > 1 ? t0[k] + t1[k] : t0[k];
                    tmem_ld16(tbase + uint32_t(a.it + ch * 16), t0);
                    if (NP > 1) tmem_ld16(tbase + uint32_t(acc_cols + a.it + ch * 16), t1);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[q][16 + k] = NP > 1 ? t0[k] + t1[k] : t0[k];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive(tmem_empty);
            if (!acc_ready) break;
            epi_store<NP, KMAJOR, EPI, FX, kChunksPerWarp, TF>(a, v, tile, h, row, grp, nchunks, s_in, inv_out,
                                                              lim, local_max, range_ok);
        }
        if (FX) {
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(local_max));
            if (lane == 0 && m) atomicMax(a.sc.max_cur, m);
            if (!range_ok && a.err) atomicCAS(a.err, 0, MM_ERR_RANGE);
        }
    }
    tc_fence_before();
    __syncthreads();
    // A wait ran out (the flag is final here): every load into this CTA lands before it exits (bounded).
    if (warp == 0 && lane == 0 && *abort_flag)
        for (int q = 0; q < kStages; ++q)
            if (armed & (1u << q)) mbar_wait(&full[q], (armed_ph >> q) & 1u, nullptr, 0, a.wait_limit);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// Point phase (EPI 2) of point `lane` of the warp's 32 points (TMEM lanes 32 quarter ..) in
// work item `tile`, formed in FP64 from the per-direction tables; 1 outside the tensor.
template <bool KMAJOR>
__device__ __forceinline__ float2 point_phase(const TcArgs &a, int64_t tile, int quarter, int lane)
{
    int64_t l, r;
    bool valid;
    if (KMAJOR) {
        l = 0;
        r = tile * kTileM + quarter * 32 + lane;
        valid = r < a.right;
    } else {
        const int64_t atom = 2 * tile + quarter / 2;
        r = atom / a.aps;
        l = (atom % a.aps) * 64 + (quarter & 1) * 32 + lane;
        valid = r < a.right && l < a.left;
    }
    if (!valid) return make_float2(1.0f, 0.0f);
    double fr = 1.0, fi = 0.0;
    auto mul = [&](const double2 *tab, int64_t i) {
        if (!tab) return;
        const double2 z = tab[i];
        const double nr = fr * z.x - fi * z.y;
        fi = fr * z.y + fi * z.x;
        fr = nr;
    };
    mul(a.pl0, l % a.ldiv);
    mul(a.pl1, l / a.ldiv);
    mul(a.pr0, r % a.rdiv);
    mul(a.pr1, r / a.rdiv);
    return make_float2(float(fr), float(fi));
}

// Weight (EPI 5) of point `lane` of the warp's 32 points in work item `tile`: the product of
// its directions' quadrature weights in FP64; 0 outside the tensor.
template <bool KMAJOR>
__device__ __forceinline__ double point_weight(const TcArgs &a, int64_t tile, int quarter, int lane)
{
    int64_t l, r;
    bool valid;
    if (KMAJOR) {
        l = 0;
        r = tile * kTileM + quarter * 32 + lane;
        valid = r < a.right;
    } else {
        const int64_t atom = 2 * tile + quarter / 2;
        r = atom / a.aps;
        l = (atom % a.aps) * 64 + (quarter & 1) * 32 + lane;
        valid = r < a.right && l < a.left;
    }
    if (!valid) return 0.0;
    double w = 1.0;
    if (a.wl0) w *= a.wl0[l % a.ldiv];
    if (a.wl1) w *= a.wl1[l / a.ldiv];
    if (a.wr0) w *= a.wr0[r % a.rdiv];
    if (a.wr1) w *= a.wr1[r / a.rdiv];
    return w;
}

// Per-warp staging of the pair kernel's output boxes: one plane's three pieces, 1 KB each.
constexpr int kStageBoxBytes = 1024;
constexpr int kStagingPerWarp = 3 * kStageBoxBytes;

// Epilogue of one work item for one warp of the pair kernel with row tiles of at most 64:
// the warp's 32 points (TMEM lanes 32 quarter ..) and output rows i0 = h it + 16 grp .. + 15.
// vr / vi[hh] hold the drained real / imaginary sums in the matrix-fragment order of
// tmem_ld_frag16 for the lanes 16 hh .. 16 hh + 15: value k is point 16 hh + t/4 + 8 ((k >> 1) & 1)
// at output 8 (k >> 2) + 2 (t % 4) + (k & 1) (t = lane).  The values are scaled, given the
// nonlinear phase (EPI 1), checked and split as in epi_store; each piece plane's 32 x 16 box is
// written to shared memory by stmatrix (two instructions per piece) and stored by TMA: for
// direction 1 (K-major output) as [point][output] rows of 32 bytes in the 32-byte swizzled order,
// otherwise transposed to [output][point] rows of 64 bytes in the 64-byte swizzled order.
// Parts of a box outside the padded tensor are clipped by the TMA unit; boxes wholly outside
// are not issued.
template <int NP, bool KMAJOR, int EPI, bool FX>
__device__ __forceinline__ int epi_frag_store(const TcArgs &a, const CUtensorMap *mapY, uint8_t *stg,
                                               float (&vr)[2][8], float (&vi)[2][8], int64_t tile, int h,
                                               int quarter, int lane, int grp, int nchunks, float s_in,
                                               float inv_out, float lim, float &local_max, bool &range_ok,
                                               float2 phl, double wpl, double &nacc)
{
    if (grp >= nchunks) return 0;
    const int i0 = h * a.it + grp * 16;
    if (i0 >= a.mp) return 0;
    const int t4 = lane / 4, tc = lane % 4;
    // the warp's box origin and the validity of this thread's four points (hh, s)
    bool box_ok, valid[2][2];
    int64_t rr;
    int l0 = 0;
    if (KMAJOR) {
        rr = tile * kTileM + quarter * 32;
        box_ok = rr < a.right;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int s = 0; s < 2; ++s) valid[hh][s] = rr + 16 * hh + 8 * s + t4 < a.right;
    } else {
        const int64_t atom = 2 * tile + quarter / 2;
        rr = atom / a.aps;
        l0 = int((atom % a.aps) * 64 + (quarter & 1) * 32);
        box_ok = rr < a.right && l0 < a.left;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int s = 0; s < 2; ++s) valid[hh][s] = rr < a.right && l0 + 16 * hh + 8 * s + t4 < a.left;
    }
    // point phases of this thread's four points (EPI 2): lane 16 hh + 8 s + t4 holds that point's
    float2 ph[2][2] = {{{1.0f, 0.0f}, {1.0f, 0.0f}}, {{1.0f, 0.0f}, {1.0f, 0.0f}}};
    if (EPI == 2) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                ph[hh][s].x = __shfl_sync(0xffffffffu, phl.x, 16 * hh + 8 * s + t4);
                ph[hh][s].y = __shfl_sync(0xffffffffu, phl.y, 16 * hh + 8 * s + t4);
            }
    }
    // output weights (EPI 5) of this thread's four outputs and the per-point sums of |y|^2 w over them
    float wout[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, psum[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    if (EPI == 5) {
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            const double2 w2 = __ldg(reinterpret_cast<const double2 *>(a.wo + i0 + 8 * cb + 2 * tc));
            wout[cb][0] = float(w2.x);
            wout[cb][1] = float(w2.y);
        }
    }
    // row scales of this thread's four outputs (pairs at 2 tc and 8 + 2 tc)
    float g[2][2] = {{1.0f, 1.0f}, {1.0f, 1.0f}};
    if (FX) {
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            const float2 r2 = __ldg(reinterpret_cast<const float2 *>(a.rho + i0 + 8 * cb + 2 * tc));
            g[cb][0] = r2.x * s_in;
            g[cb][1] = r2.y * s_in;
        }
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float xr = vr[hh][k], xi = vi[hh][k];
            if (FX) {
                xr *= g[k >> 2][k & 1];  // power of two: exact
                xi *= g[k >> 2][k & 1];
            }
            if (EPI == 3 || EPI == 4) {
                // this value's place in the padded plane (the pieces' offset): the state before the
                // nonlinear stage is stored there (3) or read from there (4)
                const int s8 = (k >> 1) & 1;
                const int64_t i = i0 + 8 * (k >> 2) + 2 * tc + (k & 1);
                const int64_t off = KMAJOR ? (rr + 16 * hh + 8 * s8 + t4) * a.mp + i
                                           : (rr * a.mp + i) * a.left + l0 + 16 * hh + 8 * s8 + t4;
                if (EPI == 3) {
                    if (valid[hh][s8]) a.mid_out[off] = make_float2(xr, xi);
                } else {
                    // adjoint of psi -> psi exp(-i tb |psi|^2) at psi (conjugate-Wirtinger gradient
                    // convention): g = exp(i th) g' + 2 tb Im(conj(g') psi') psi, psi' = exp(-i th) psi
                    const float2 ps = valid[hh][s8] ? a.mid_in[off] : make_float2(0.0f, 0.0f);
                    const float th = a.tb * (ps.x * ps.x + ps.y * ps.y);
                    float sn, cs;
                    sincosf(th, &sn, &cs);
                    const float pr = ps.x * cs + ps.y * sn, pi = ps.y * cs - ps.x * sn;  // psi'
                    const float im = xr * pi - xi * pr;                                  // Im(conj(g') psi')
                    const float f = 2.0f * a.tb * im;
                    const float yr = xr * cs - xi * sn + f * ps.x, yi = xr * sn + xi * cs + f * ps.y;
                    xr = yr;
                    xi = yi;
                }
            }
            if (EPI == 1 || EPI == 3) {
                const float th = a.tb * (xr * xr + xi * xi);
                float sn, cs;
                sincosf(th, &sn, &cs);
                const float yr = xr * cs + xi * sn, yi = xi * cs - xr * sn;
                xr = yr;
                xi = yi;
            }
            if (EPI == 2) {
                const float2 f = ph[hh][(k >> 1) & 1];
                const float yr = xr * f.x - xi * f.y, yi = xr * f.y + xi * f.x;
                xr = yr;
                xi = yi;
            }
            if (EPI == 5) psum[hh][(k >> 1) & 1] += (xr * xr + xi * xi) * wout[k >> 2][k & 1];
            if (FX) {
                const float ar = fabsf(xr), ai = fabsf(xi);
                if (valid[hh][(k >> 1) & 1]) {
                    local_max = fmaxf(local_max, fmaxf(ar, ai));
                    range_ok &= ar < lim && ai < lim;
                }
                xr *= inv_out;
                xi *= inv_out;
            }
            vr[hh][k] = xr;
            vi[hh][k] = xi;
        }
    if (EPI == 5) {
        // the four points' weights (lane 16 hh + 8 s + t4 holds that point's; 0 outside the tensor)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int s = 0; s < 2; ++s)
                nacc += __shfl_sync(0xffffffffu, wpl, 16 * hh + 8 * s + t4) * double(psum[hh][s]);
    }
    auto pieces_of = [&](float x, uint16_t *b) {
        if (FX) {
            split_fx_scaled(x, b[0], b[1], b[2]);
        } else {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const __nv_bfloat16 h16 = __float2bfloat16_rn(x);
                b[p] = __bfloat16_as_ushort(h16);
                x -= __bfloat162float(h16);
            }
        }
    };
    // the shared-memory row this thread addresses for stmatrix: matrix j = lane / 8 is (s, cb) =
    // (j & 1, j >> 1), row r = lane % 8
    const int mj = lane / 8, mr = lane % 8, ms = mj & 1, mcb = mj >> 1;
    const uint32_t sbase = smem_u32(stg);
    uint32_t row_off[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        if (KMAJOR) {
            const int pr = 16 * hh + 8 * ms + mr;  // point row of the [32][16] box
            row_off[hh] = uint32_t(pr * 32 + ((mcb ^ ((pr >> 2) & 1)) * 16));
        } else {
            const int ir = 8 * mcb + mr;  // output row of the [16][32] box
            row_off[hh] = uint32_t(ir * 64 + (((2 * hh + ms) ^ ((ir >> 1) & 3)) * 16));
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (lane == 0) bulk_wait_read0();  // the previous boxes have left the staging buffer
        __syncwarp();
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            // pack the pieces of output pairs (2 tc, 2 tc + 1): pk[p][j], matrix j = s + 2 cb
            uint32_t pk[3][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = 2 * j;  // values k, k + 1: s = j & 1, cb = j >> 1
                const float x0 = c == 0 ? vr[hh][k] : vi[hh][k], x1 = c == 0 ? vr[hh][k + 1] : vi[hh][k + 1];
                if (FX) {
                    split_fx_pair(x0, x1, pk[0][j], pk[1][j], pk[2][j]);
                } else {
                    uint16_t b0[3], b1[3];
                    pieces_of(x0, b0);
                    pieces_of(x1, b1);
#pragma unroll
                    for (int p = 0; p < NP; ++p) pk[p][j] = uint32_t(b0[p]) | (uint32_t(b1[p]) << 16);
                }
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const uint32_t ad = sbase + uint32_t(p * kStageBoxBytes) + row_off[hh];
                if (KMAJOR) stmatrix_x4(ad, pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
                else stmatrix_x4_trans(ad, pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0 && box_ok) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                if (KMAJOR) tma_store_3d(mapY, stg + p * kStageBoxBytes, i0, int(rr), c * NP + p);
                else tma_store_4d(mapY, stg + p * kStageBoxBytes, l0, i0, int(rr), c * NP + p);
            }
            bulk_commit();
        }
    }
    return box_ok ? 2 : 0;  // bulk groups committed (by lane 0)
}

// Epilogue warps of the pair kernel: 8 (two per tensor-memory lane quarter, two chunks of 16
// output rows each) for row tiles of 64, which spreads their shared-memory traffic over the
// item and leaves the MMA issue freer; 16 for row tiles of 128, for the nonlinear-phase
// epilogue (EPI 1), whose per-value arithmetic needs the extra warps, and for batches (BATCH),
// whose small problems give short items with much epilogue work per MMA.
__host__ __device__ constexpr int pair_epi_warps(int CH, int EPI, bool BATCH)
{
    return CH == 1 && (EPI == 0 || EPI == 2 || EPI == 5) && !BATCH ? 8 : 16;
}
// With row tiles of 64 outside batches the MMAs of a CTA pair come from two threads in two
// warps (the leading accumulator's from warp 1, the correction accumulator's from the warp after
// the epilogue warps), so that neither issue stream waits for the other.
__host__ __device__ constexpr bool pair_two_issuers(int CH, bool BATCH) { return CH == 1 && !BATCH; }
__host__ __device__ constexpr int pair_threads(int CH, int EPI, bool BATCH)
{
    return 32 * (2 + pair_epi_warps(CH, EPI, BATCH) + (pair_two_issuers(CH, BATCH) ? 1 : 0));
}
// k-blocks of 16 per pipeline stage: 2 with 8 epilogue warps (K-major data boxes then have
// 64-byte rows, 64-byte swizzled: half as many row requests per byte as 32-byte rows; MN-major
// boxes 32 k-rows of 128 bytes), else 1.
__host__ __device__ constexpr int pair_kb_per_stage(int CH, int EPI, bool BATCH)
{
    return pair_epi_warps(CH, EPI, BATCH) == 8 ? 2 : 1;
}
// Pipeline stages: with row tiles of 64, 3 of 66 KB (8 epilogue warps, two k-blocks each, 24 KB
// of output staging) or 5 of 33 KB (16 warps, 48 KB); with row tiles of 128, 4 of 42 KB (48 KB
// of staging).
__host__ __device__ constexpr int pair_stages(int CH, int EPI, bool BATCH)
{
    return CH == 2 ? 4 : (pair_epi_warps(CH, EPI, BATCH) == 8 ? 3 : 5);
}
__host__ __device__ constexpr int pair_staging_bytes(int CH, int EPI, bool BATCH)
{
    return pair_epi_warps(CH, EPI, BATCH) * kStagingPerWarp;
}

// The same product with the tensor cores of the two SMs of a cluster
// working as one (tcgen05 cta_group::2): the leader CTA (rank 0) issues
// MMAs of M = 256 points, rows 0..127 from its own shared memory and
// 128..255 from its peer's at the same offsets; each CTA holds half of the
// N = 2 IT matrix columns and receives its own 128 x N accumulator in its
// tensor memory.  The rows are tiled in row tiles of IT <= 64 (TcMatrix
// ni2 / it2), which keeps one item's two accumulators within 256 of the
// 512 tensor-memory columns: items alternate between two accumulator sets,
// so the MMAs of an item run while the epilogue drains the previous one.
// The matrix half of rank r covers output rows r IT/2 .. (r + 1) IT/2 - 1
// of the tile as the blocks [-S; C; S], so the real plane is one MMA over
// the window [C; S] and the imaginary plane one over [-S; C]: two
// N = 2 IT MMAs per piece product, every MMA reading one half of B per SM.
// Accumulator columns of a CTA: [re | im] of rows 0 .. IT/2 - 1, then
// [re | im] of rows IT/2 .. IT - 1.  Both CTAs' TMA loads complete on the
// leader's stage barriers; the leader's commits release the stages and
// signal the accumulators in both CTAs.  The leader's MMAs reuse an
// accumulator set once the epilogue warps of both CTAs have drained it:
// the peer's warps arrive on their own barrier, which one thread of the
// peer relays to the leader's.
template <int NP, bool KMAJOR, int EPI, bool FX, int CH, bool BATCH, bool CHAIN = false>
__global__ void __launch_bounds__(pair_threads(CH, EPI, BATCH && !CHAIN) + (CHAIN ? 32 : 0), 1)
    tc_pair_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapE,
                   const __grid_constant__ CUtensorMap mapY, TcArgs a, const TcPairProblem *__restrict__ many,
                   int nprob, int64_t total)
{
    // BATCH: items P < total of many problems (records `many`, sorted by pairs_begin); `a` then
    // carries only what all problems share (row tiles of the same size, stage layout, error word).
    // CHAIN (with BATCH): the records are a sequence of products, each reading what the previous
    // one wrote; a product's loads wait until every epilogue warp of the grid has signalled the
    // previous product complete, and the records say per product whether its data is K-major.
    // Chained launches keep the single launch's warps and stages.
    static_assert(!CHAIN || (BATCH && EPI == 0), "a chain is a batched launch of plain products");
    constexpr bool BCFG = BATCH && !CHAIN;  // the batched launches' warp and stage configuration
    // the second MMA issuer (correction accumulator) and whether it issues (NP > 1); with one
    // piece it has nothing to issue and stays idle
    constexpr int kIssuer2 = pair_two_issuers(CH, BCFG) ? 2 + pair_epi_warps(CH, EPI, BCFG) : -1;
    constexpr bool kTwo = kIssuer2 >= 0 && NP > 1;
    // CHAIN: the warp that publishes the items this CTA has stored
    constexpr int kSignal = CHAIN ? pair_threads(CH, EPI, BCFG) / 32 : -1;
    const int64_t items = BATCH ? total : a.pairs;
    constexpr int kSt = pair_stages(CH, EPI, BCFG);
    constexpr int KB = pair_kb_per_stage(CH, EPI, BCFG);  // k-blocks per stage
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *staging = smem + kSt * a.stage_bytes;  // pair_epi_warps(CH, EPI, BCFG) x kStagingPerWarp
    uint64_t *full = reinterpret_cast<uint64_t *>(staging + pair_staging_bytes(CH, EPI, BCFG));
    uint64_t *empty = full + kSt;
    uint64_t *accf = empty + kSt;  // [2]: accumulator set b holds a finished item
    uint64_t *tmem_empty = accf + 2;       // [2]: accumulator set b has been drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint64_t *mma_fin = reinterpret_cast<uint64_t *>(tmem_slot + 2);  // [2] abort: an issuer's MMAs have completed
    uint64_t *item_done = mma_fin + 2;  // [8] CHAIN: this CTA's epilogue warps have stored item l (l mod 8)

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int rank = int(blockIdx.x & 1);
    const int acc_cols = 2 * a.it;                          // one accumulator: [re | im] of IT rows
    const int set_cols = NP > 1 ? 2 * acc_cols : acc_cols;  // leading and correction accumulators
    const int nsets = 2 * set_cols <= 512 ? 2 : 1;          // two sets when they fit in tensor memory
    const int need = nsets * set_cols;
    const uint32_t ncols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSt; ++s) {
            mbar_init(&full[s], 1);   // the leader's producer (expecting both CTAs' bytes)
            mbar_init(&empty[s], kTwo ? 2 : 1);  // the leader's commits (one per issuer)
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], kTwo ? 2 : 1);
            // this CTA's epilogue warps, and in the leader the peer's relay
            mbar_init(&tmem_empty[b], pair_epi_warps(CH, EPI, BCFG) + (rank == 0 ? 1 : 0));
        }
        mbar_init(mma_fin, 1);
        mbar_init(mma_fin + 1, 1);
        if (CHAIN)
            for (int q = 0; q < 8; ++q) mbar_init(&item_done[q], pair_epi_warps(CH, EPI, BCFG));
        *abort_flag = 0;
        mbar_fence_init();
        if (!BATCH) {
            tma_prefetch_desc(&mapX);
            tma_prefetch_desc(&mapE);
            tma_prefetch_desc(&mapY);
        }
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, ncols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers and tensor memory exist before either uses the other's
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // The next kernel of the stream may start its own set-up now; everything below reads or
    // writes data of the previous kernel (input pieces, scale words) only after it has completed.
    if (threadIdx.x == 0) griddep_launch_dependents();
    griddep_wait();
    if (FX && !CHAIN && blockIdx.x == 0 && threadIdx.x == 0) {
        if (!BATCH) {
            if (a.sc.zero_next) *a.sc.zero_next = 0u;
        } else {
            for (int q = 0; q < nprob; ++q)
                if (many[q].a.sc.zero_next) *many[q].a.sc.zero_next = 0u;
        }
    }
    const int64_t cid = blockIdx.x / 2, nclusters = gridDim.x / 2;
    const int half = a.it / 2;
    const int e_bytes = 3 * half * 32;  // one piece's [-S; C; S] blocks in a stage
    uint32_t armed = 0, armed_ph = 0;   // producer of the leader: slots armed, parity of their last arming
    const uint32_t full_lead = mapa_shared(smem_u32(full), 0);
    const uint32_t tmem_empty_lead = mapa_shared(smem_u32(tmem_empty), 0);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            int s = 0;
            uint32_t ph = 0;  // ring position
            int64_t g = 0;    // stages reached over the launch
            int ready = 0;         // CHAIN: the product whose loads have begun on this CTA
            uint32_t gready = 0;   // CHAIN: slab groups of the previous product known complete
            int rec_at = 0;   // BATCH: the record of the previous item
            const int e_rows = 3 * half / 4;  // 128-byte rows of one block triple
            for (int64_t P = cid; P < items && !*abort_flag; P += nclusters) {
                const TcPairProblem *pr = BATCH ? &pair_problem_next(many, nprob, P, rec_at) : nullptr;
                const TcArgs &A = BATCH ? pr->a : a;
                const CUtensorMap *mx = BATCH ? &pr->mapX : &mapX, *me = BATCH ? &pr->mapE : &mapE;
                const int64_t Pl = BATCH ? P - pr->pairs_begin : P;
                int64_t pairi;
                int h;
                chain_item(A, CHAIN && pr->hmajor, Pl, pairi, h);
                const int64_t tile = pairi * 2 + rank;
                const bool km = CHAIN ? pr->km != 0 : KMAJOR;
                if (CHAIN) {
                    bool ok = true, waited = false;
                    if (pr->prod != ready || P == cid) {
                        // a new product: its tensor maps are fetched while the waits below run, and
                        // the next product's as well; the product two back (whose input buffer this
                        // one overwrites, and whose maximum sets this one's scale) must be complete
                        tma_prefetch_desc(mx);
                        tma_prefetch_desc(me);
                        if (pr->prod + 1 < nprob) {
                            tma_prefetch_desc(&pr[1].mapX);
                            tma_prefetch_desc(&pr[1].mapE);
                        }
                        if (pr->wait_prod >= 0) {
                            ok = counter_wait(a.done + pr->wait_prod, many[pr->wait_prod].tot_target, a.err,
                                              MM_ERR_TIMEOUT, a.wait_limit);
                            waited = true;
                        }
                        ready = pr->prod;
                        gready = 0;
                    }
                    if (ok && pr->prod > 0) {
                        // the previous product's output is this one's input: every slab group this
                        // CTA reads must be complete (bounded waits), then the loads go through TMA
                        int g_lo, g_hi;
                        chain_groups(*pr, pairi, h, rank, true, g_lo, g_hi);
                        const TcPairProblem &Q = pr[-1];
                        const unsigned *cnt = a.gcnt + int64_t(pr->prod - 1) * kChainGroups;
                        for (int gq = g_lo; gq <= g_hi && ok; ++gq) {
                            if (gready & (1u << gq)) continue;
                            ok = counter_wait(cnt + gq, Q.g_expect[gq], a.err, MM_ERR_TIMEOUT, a.wait_limit);
                            gready |= 1u << gq;
                            waited = true;
                        }
                    }
                    if (!ok) {
                        *abort_flag = 1;
                        break;
                    }
                    if (waited) fence_proxy_async_global();  // the acquired data, read by TMA
                }
                // MN-major: the two 64-point atoms of the tile (slab row, first point), past the end zero fill
                int ac_l[2] = {0, 0}, ac_r[2] = {0, 0};
                if (!km) {
                    for (int q = 0; q < 2; ++q) {
                        const int64_t atom = 2 * tile + q;
                        int64_t r = atom / A.aps;
                        if (r > A.right) r = A.right;
                        ac_r[q] = int(r);
                        ac_l[q] = int((atom % A.aps) * 64);
                    }
                }
                const int k_row = int(tile * kTileM);
                // the matrix blocks of all pieces for (row tile h, k-block kb, rank): one box of 128-byte rows
                const int e_box_rows = NP * e_rows;
                const int e_row0 = (h * A.kblocks * 2 + rank) * e_box_rows;
                const int kb_end = A.kb_hi[h];
                for (int kb = A.kb_lo[h]; kb < kb_end; kb += KB) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int nk = KB == 1 || kb + 1 == kb_end ? 1 : 2;  // k-blocks of the item in this stage
                    uint8_t *st = smem + s * a.stage_bytes;
                    const uint32_t fb = full_lead + uint32_t(s) * 8u;
                    if (g++ != a.withhold) {
                        // both CTAs' bytes: the data box (always whole, zero-filled past the tensor) and the
                        // matrix boxes of the stage's k-blocks
                        if (rank == 0) {
                            mbar_arrive_expect_tx(&full[s], KB == 1 ? uint32_t(a.tx_bytes)
                                                                    : uint32_t(2 * (a.e_offset + nk * NP * e_bytes)));
                            armed |= 1u << s;
                            armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
                        }
                        // all 2 NP piece planes in one box (K-major: [plane][128 points][16 KB k]) or one box
                        // per atom (MN-major: [atom][plane][16 k][64 points])
                        if (km) {
                            tma_load_3d_pair(mx, fb, st, kb * kBK, k_row, 0);
                        } else {
                            tma_load_4d_pair(mx, fb, st, ac_l[0], kb * kBK, ac_r[0], 0);
                            tma_load_4d_pair(mx, fb, st + KB * 2 * NP * 2048, ac_l[1], kb * kBK, ac_r[1], 0);
                        }
                        for (int j = 0; j < nk; ++j)
                            tma_load_2d_pair(me, fb, st + a.e_offset + j * NP * e_bytes, 0,
                                             e_row0 + (kb + j) * 2 * e_box_rows);
                    }
                    if (++s == kSt) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
        __syncwarp();  // the role's other lanes wait for it: the warp meets the block barrier converged
    } else if (CHAIN && warp == kSignal) {
        if (lane == 0) {
            // ---------------- signaller (CHAIN) ----------------
            // Items in the cluster's order: once the CTA's epilogue warps have all reported item l
            // stored, one release fence at GPU scope, then one count for every slab group this
            // CTA's part of the item wrote and one for the product's total (relaxed adds after the
            // fence).  The fence waits here, off the epilogue warps' path.
            uint32_t lt = 0;
            int rec_at = 0;
            for (int64_t P = cid; P < items; P += nclusters, ++lt) {
                const TcPairProblem *pr = &pair_problem_next(many, nprob, P, rec_at);
                int64_t pairi;
                int h;
                chain_item(pr->a, pr->hmajor != 0, P - pr->pairs_begin, pairi, h);
                if (*abort_flag ||
                    !mbar_wait(&item_done[lt % 8u], (lt / 8u) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                    *abort_flag = 1;
                    break;
                }
                fence_acq_rel_gpu();
                int g_lo, g_hi;
                chain_groups(*pr, pairi, h, rank, false, g_lo, g_hi);
                unsigned *cnt = a.gcnt + int64_t(pr->prod) * kChainGroups;
                for (int gq = g_lo; gq <= g_hi; ++gq) red_relaxed_gpu_add(cnt + gq, 1u);
                red_relaxed_gpu_add(a.done + pr->prod, 1u);
            }
        }
        __syncwarp();
    } else if (warp == 1 || warp == kIssuer2) {
        if (lane == 0 && rank == 1 && warp == 1) {
            // ---------------- relay (peer only) ----------------
            // One cluster-scope arrival on the leader's barrier once all of this
            // CTA's epilogue warps have drained an accumulator set (their own
            // arrivals stay CTA-scope, which does not wait for their stores).
            uint32_t lt = 0;
            for (int64_t P = cid; P < items; P += nclusters, ++lt) {
                const int b = int(lt % uint32_t(nsets));
                if (!mbar_wait(&tmem_empty[b], (lt / uint32_t(nsets)) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_arrive_cluster(tmem_empty_lead + uint32_t(b) * 8u);
            }
        }
        if (lane == 0 && rank == 0 && (warp == 1 || kTwo)) {
            // ---------------- MMA issuers (leader only) ----------------
            // The operand descriptors of stage 0 are built once; stage s adds s stage_bytes / 16 to
            // their start-address field (bits 0..13, wide enough for every shared-memory address of
            // the CTA).  Each issuing thread shares its SM sub-partition with busy epilogue warps,
            // whose shared-memory instructions delay its MMAs, so few instructions per MMA keep the
            // tensor pipe fed.  With two issuers (kTwo), warp 1 issues the leading product's MMAs
            // and warp kIssuer2 the corrections': each accumulator still receives its MMAs from one
            // thread in the same order, both commit every stage and every item (the barriers
            // count two), and the two streams interleave in the tensor pipe.
            const int lead_part = !kTwo ? -1 : (warp == 1 ? 1 : 0);  // -1: all terms
            auto idesc_for = [&](bool km) {
                return FX ? idesc_f16_f32(2 * kTileM, 2 * a.it, !km, false) : idesc_bf16_f32(2 * kTileM, 2 * a.it, !km, false);
            };
            const uint32_t idesc = idesc_for(KMAJOR || CHAIN), idesc_mn = idesc_for(false);
            const uint32_t st0 = smem_u32(smem), est0 = st0 + uint32_t(a.e_offset);
            // [real plane, imaginary plane][piece]; CHAIN: adesc for K-major data, adesc_mn for MN-major
            uint64_t adesc[2][NP], adesc_mn[2][NP], bdesc[2][NP];
            auto data_descs = [&](bool km, uint64_t(&ad)[2][NP]) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    // K-major: plane tiles of KB x 4 KB (rows of 32 KB bytes, 8-row swizzle atoms of 256 KB
                    // bytes); MN-major: plane tiles of KB x 2 KB (16 KB k-rows of 128 bytes) per atom, atoms
                    // 2 NP KB x 2 KB apart
                    const uint32_t pb = km ? uint32_t(KB * kDataTileBytes) : uint32_t(KB * 2048);
                    const uint32_t xre = st0 + uint32_t(p) * pb, xim = st0 + uint32_t(NP + p) * pb;
                    constexpr uint32_t kmswz = KB == 2 ? kSwz64 : kSwz32;
                    ad[0][p] = km ? smem_desc(xre, 16, 256 * KB, kmswz) : smem_desc(xre, 2 * NP * 2048 * KB, 1024, kSwz128);
                    ad[1][p] = km ? smem_desc(xim, 16, 256 * KB, kmswz) : smem_desc(xim, 2 * NP * 2048 * KB, 1024, kSwz128);
                }
            };
            data_descs(KMAJOR || CHAIN, adesc);
            if (CHAIN) data_descs(false, adesc_mn);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const uint32_t eb = est0 + uint32_t(p * e_bytes);
                bdesc[0][p] = smem_desc(eb + uint32_t(half * 32), 16, 256, kSwz32);  // [C; S]
                bdesc[1][p] = smem_desc(eb, 16, 256, kSwz32);                        // [-S; C]
            }
            const uint64_t stage_step = uint64_t(uint32_t(a.stage_bytes) >> 4);
            int s = 0;
            uint32_t ph = 0, lt = 0;  // ring position, advanced with the producer's
            int rec_at = 0;           // BATCH: the record of the previous item
            for (int64_t P = cid; P < items && !*abort_flag; P += nclusters, ++lt) {
                const TcPairProblem *pr = BATCH ? &pair_problem_next(many, nprob, P, rec_at) : nullptr;
                const TcArgs &A = BATCH ? pr->a : a;
                int64_t pairi;
                int h;
                chain_item(A, CHAIN && pr->hmajor, BATCH ? P - pr->pairs_begin : P, pairi, h);
                const bool km = CHAIN ? pr->km != 0 : KMAJOR;
                const uint32_t id = CHAIN && !km ? idesc_mn : idesc;
                // the item's data descriptors (CHAIN: chosen once per item, outside the MMA loop)
                uint64_t ad[2][NP];
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int p = 0; p < NP; ++p) ad[c][p] = CHAIN && !km ? adesc_mn[c][p] : adesc[c][p];
                const int b = int(lt % uint32_t(nsets));
                const uint32_t use = lt / uint32_t(nsets);
                if (use > 0 && !mbar_wait<true>(&tmem_empty[b], (use - 1) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + uint32_t(b * set_cols), d1 = d0 + uint32_t(acc_cols);
                const int kb_lo = A.kb_lo[h], kb_hi = A.kb_hi[h];
                for (int kb = kb_lo; kb < kb_hi; kb += KB) {
                    if (!mbar_wait(&full[s], ph, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t so = uint64_t(s) * stage_step;
                    const int nk = KB == 1 || kb + 1 == kb_hi ? 1 : 2;
                    for (int j = 0; j < nk; ++j) {
                        // k-block kb + j: its 32 bytes of every data row (K-major) or its 16 k-rows of
                        // 128 bytes (MN-major), its matrix blocks
                        const uint64_t ao = so + uint64_t(j * (km ? 2 : 128)), bo = so + uint64_t(j * (NP * e_bytes >> 4));
                        const uint32_t first = kb + j == kb_lo ? 0u : 1u;  // each accumulator starts at its first product
#pragma unroll
                        for (int t = 0; t < num_terms(NP); ++t) {
                            if (lead_part >= 0 && (t == 0) != (lead_part == 1)) continue;
                            const int pa = term_a(t), pb = term_b(t);
                            const uint32_t dcol = (NP > 1 && (pa != 0 || pb != 0)) ? d1 : d0;
                            umma_f16_pair(dcol, ad[0][pb] + ao, bdesc[0][pa] + bo, id, t <= 1 ? first : 1u);
                            umma_f16_pair(dcol, ad[1][pb] + ao, bdesc[1][pa] + bo, id, 1u);
                        }
                    }
                    umma_commit_pair_mc(&empty[s], 0x3);
                    if (++s == kSt) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                umma_commit_pair_mc(&accf[b], 0x3);
            }
            if (*abort_flag) {
                // every MMA this thread issued (into both CTAs' tensor memory) completes before
                // either CTA frees it
                uint64_t *fin = mma_fin + (warp == 1 ? 0 : 1);
                umma_commit_pair_mc(fin, 0x1);
                mbar_wait(fin, 0u, nullptr, 0, a.wait_limit);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps (both CTAs) ----------------
        const int ew = warp - 2;
        const int quarter = warp % 4;
        constexpr int kGroups = pair_epi_warps(CH, EPI, BCFG) / 4;  // warps per lane quarter
        constexpr int kPerWarp = 4 * CH / kGroups;       // chunks of 16 output rows per warp
        const int grp = ew / 4;  // the warp's chunks: grp, grp + kGroups, ..
        const int nchunks = a.it / 16;
        float s_in = 1.0f, inv_out = 1.0f, lim = 0.0f;
        int es_out = 0;
        float local_max = 0.0f;
        bool range_ok = true;
        double nacc = 0.0;  // EPI 5: this thread's part of the weighted norm
        // the fixed-point scales of the problem being stored (BATCH: they change with the problem,
        // and the maximum gathered so far goes to the previous problem's word first)
        const TcArgs *cur = nullptr;
        auto flush_max = [&]() {
            if (!FX || !cur) return;
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(local_max));
            if (lane == 0 && m) atomicMax(cur->sc.max_cur, m);
            local_max = 0.0f;
        };
        // s_in_max (chains): the input scale is the grid exponent of that maximum word (the one the
        // previous product took its output scale from), not a word the previous product writes
        auto scales_for = [&](const TcArgs &A, bool first_item, const unsigned *s_in_max) {
            if (!FX || cur == &A) return;
            flush_max();
            cur = &A;
            s_in = s_in_max ? ldexpf(1.0f, grid_exponent(__uint_as_float(*s_in_max))) : *A.sc.s_in;
            es_out = grid_exponent(__uint_as_float(*A.sc.max_prev));
            inv_out = ldexpf(1.0f, -es_out);
            lim = ldexpf(16384.0f, es_out);
            if (first_item && ew == 0 && lane == 0) *A.sc.s_out = ldexpf(1.0f, es_out);
        };
        // CHAIN: a warp reports an item stored (its stores complete, then an arrival on the item's
        // barrier) after it has committed the stores of its next item, whose loads do not wait for
        // this one (both belong to the same product), except the last item of a product on this
        // cluster, which it reports at once, after merging its maximum.  The signalling warp
        // publishes the counters.
        auto signal_item = [&](const TcPairProblem *R, int64_t pairi, int hh, uint32_t l) {
            (void)R;
            (void)pairi;
            (void)hh;
            if (lane == 0) {
                fence_proxy_async_global();
                mbarrier_arrive(&item_done[l % 8u]);
            }
            __syncwarp();
        };
        const TcPairProblem *pend_pr = nullptr;  // CHAIN: the item stored but not yet signalled
        int64_t pend_pair = 0;
        int pend_h = 0;
        uint32_t pend_lt = 0;
        if (!BATCH) scales_for(a, blockIdx.x == 0, nullptr);
        uint32_t lt = 0;
        int rec_at = 0;  // BATCH: the record of the previous item
        for (int64_t P = cid; P < items; P += nclusters, ++lt) {
            const TcPairProblem *pr = BATCH ? &pair_problem_next(many, nprob, P, rec_at) : nullptr;
            const TcArgs &A = BATCH ? pr->a : a;
            const int64_t Pl = BATCH ? P - pr->pairs_begin : P;
            if (CHAIN && lane == 0 && cur != &A) tma_prefetch_desc(&pr->mapY);  // fetched while the item's MMAs run
            if (BATCH && !CHAIN) scales_for(A, Pl == 0 && rank == 0, nullptr);
            int64_t pairi;
            int h;
            chain_item(A, CHAIN && pr->hmajor, Pl, pairi, h);
            const int64_t tile = pairi * 2 + rank;
            const int b = int(lt % uint32_t(nsets));
            // the same decision in every lane: the warp stays converged for its collective instructions
            const bool acc_ready = __all_sync(
                0xffffffffu, !*abort_flag && mbar_wait(&accf[b], (lt / uint32_t(nsets)) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit));
            if (!acc_ready) *abort_flag = 1;
            tc_fence_after();
            if (CHAIN && acc_ready && cur != &A) {
                // a new product: its loads began after the product two back had completed (the
                // maximum words its scales come from are that product's or older); one lane
                // acquires that counter, and the warp follows
                bool ok = true;
                if (lane == 0 && pr->wait_prod >= 0)
                    ok = counter_wait(a.done + pr->wait_prod, many[pr->wait_prod].tot_target, a.err, MM_ERR_TIMEOUT,
                                      a.wait_limit);
                if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) *abort_flag = 1;
                scales_for(A, Pl == 0 && rank == 0, pr->s_in_max);
            }
            // drain in the matrix-fragment order: the warp's chunks of 16 output rows
            // (grp, grp + kGroups ..), each as two 16-lane halves, leading + corrections; tensor
            // memory is released before the values are scaled, split and stored
            float vr[kPerWarp][2][8], vi[kPerWarp][2][8];
#pragma unroll
            for (int q = 0; q < kPerWarp; ++q) {
                const int ch = grp + kGroups * q;
                if (ch < nchunks) {
                    const int i0 = ch * 16;
                    const int cre = i0 + (i0 >= half ? half : 0), cim = cre + half;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint32_t ta = tmem + (uint32_t(quarter * 32 + hh * 16) << 16) + uint32_t(b * set_cols);
                        float t1[8];
                        tmem_ld_frag16(ta + uint32_t(cre), vr[q][hh]);
                        if (NP > 1) tmem_ld_frag16(ta + uint32_t(acc_cols + cre), t1);
                        tmem_ld_wait();
                        if (NP > 1) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) vr[q][hh][k] += t1[k];
                        }
                        tmem_ld_frag16(ta + uint32_t(cim), vi[q][hh]);
                        if (NP > 1) tmem_ld_frag16(ta + uint32_t(acc_cols + cim), t1);
                        tmem_ld_wait();
                        if (NP > 1) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) vi[q][hh][k] += t1[k];
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive(&tmem_empty[b]);
            if (!acc_ready) break;
            const float2 phl = EPI == 2 ? point_phase<KMAJOR>(A, tile, quarter, lane) : make_float2(1.0f, 0.0f);
            const double wpl = EPI == 5 ? point_weight<KMAJOR>(A, tile, quarter, lane) : 0.0;
            int commits = 0;
            if (CHAIN && pr->km) {
#pragma unroll
                for (int q = 0; q < kPerWarp; ++q)
                    commits += epi_frag_store<NP, true, EPI, FX>(A, &pr->mapY, staging + ew * kStagingPerWarp, vr[q],
                                                                 vi[q], tile, h, quarter, lane, grp + kGroups * q,
                                                                 nchunks, s_in, inv_out, lim, local_max, range_ok,
                                                                 phl, wpl, nacc);
            } else {
#pragma unroll
                for (int q = 0; q < kPerWarp; ++q)
                    commits += epi_frag_store<NP, KMAJOR && !CHAIN, EPI, FX>(
                        A, BATCH ? &pr->mapY : &mapY, staging + ew * kStagingPerWarp, vr[q], vi[q], tile, h,
                        quarter, lane, grp + kGroups * q, nchunks, s_in, inv_out, lim, local_max, range_ok, phl,
                        wpl, nacc);
            }
            if (CHAIN) {
                if (pend_pr) {
                    // the previous item's stores (all but this item's groups) have completed
                    if (lane == 0) bulk_wait_but(commits);
                    signal_item(pend_pr, pend_pair, pend_h, pend_lt);
                    pend_pr = nullptr;
                }
                if (P + nclusters >= items || P + nclusters >= pr->pairs_begin + A.pairs) {
                    // this cluster's last item of the product
                    flush_max();
                    if (lane == 0) bulk_wait0();
                    signal_item(pr, pairi, h, lt);
                } else {
                    pend_pr = pr;
                    pend_pair = pairi;
                    pend_h = h;
                    pend_lt = lt;
                }
            }
        }
        if (lane == 0) bulk_wait0();  // this warp's stores are complete
        if (EPI == 5) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
            if (lane == 0 && nacc != 0.0) atomicAdd(a.norm2, nacc);
        }
        if (FX) {
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(local_max));
            if (lane == 0 && m && cur) atomicMax(cur->sc.max_cur, m);
            local_max = 0.0f;
            if (!range_ok && a.err) atomicCAS(a.err, 0, MM_ERR_RANGE);
        }
        if (CHAIN && pend_pr) signal_item(pend_pr, pend_pair, pend_h, pend_lt);  // only after an abort
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0 && *abort_flag) {
        // A wait ran out (the flag is final here: every role of this CTA has finished).  No stage
        // may still be receiving data when the CTAs exit: the leader waits (bounded) for the last
        // arming of every slot, which completes once both CTAs' loads into that stage have landed;
        // the peer, whose loads complete on the leader's barriers, gives its last loads the same time.
        if (rank == 0) {
            for (int q = 0; q < kSt; ++q)
                if (armed & (1u << q)) mbar_wait(&full[q], (armed_ph >> q) & 1u, nullptr, 0, a.wait_limit);
        } else {
            const long long t0 = clock64();
            while (clock64() - t0 < a.wait_limit) {
            }
        }
    }
    // Every MMA (waited through the accumulator barriers), every load into either CTA's shared
    // memory and every store has completed: the CTAs only wait for each other before freeing
    // tensor memory and exiting.
    cluster_sync_relaxed();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, ncols);
    }
}

struct TcBatchArgs {
    int64_t total_pairs;    // work items over all problems
    int nprob;
    int it_max;             // widest row tile of the launch (tensor-memory allocation)
    int stage_bytes, e_offset;
    float tb;               // tau * beta for the nonlinear epilogue
    int *err;
    long long wait_limit;   // bounded waits give up after this many SM clocks
};

// Problem of work item P: the last problem whose first item is <= P.
template <bool BATCH>
__device__ __forceinline__ const TcProblem &problem_of(int64_t P, const TcProblem &one, const TcProblem *many,
                                                      int nprob)
{
    if (!BATCH) return one;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (many[mid].pairs_begin <= P) lo = mid;
        else hi = mid - 1;
    }
    return many[lo];
}

// The kernel above generalised to a list of problems (BATCH): the same
// persistent cluster-pair structure, with every per-problem quantity read
// from the item's problem record.  Cluster c processes work
// items P = c, c + #clusters, ...; item P of a problem is the row tile
// h = P % ni of the point tiles 2 (P / ni) + rank, rank = 0, 1, so the two
// CTAs of a cluster need the same matrix tiles at the same time and read
// them through L2 once between them; each CTA loads its own stages.  The
// TMA warp runs ahead across item boundaries; the epilogue warps
// copy the two accumulators into registers, release tensor memory to the
// MMA warp at once, and then scale, split and store while the next item's
// MMAs run.  A batched launch (BATCH) covers the same direction of many
// independent problems of different sizes; their records are in global
// memory and each item looks its problem up.
template <int NP, bool KMAJOR, int EPI, bool FX, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
    tc_mode_kernel_batched(const __grid_constant__ TcProblem one, const TcProblem *__restrict__ many, TcBatchArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * a.stage_bytes);
    uint64_t *empty = full + kStages;
    uint64_t *accf = empty + kStages;
    uint64_t *tmem_empty = accf + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_empty + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint64_t *mma_fin = reinterpret_cast<uint64_t *>(tmem_slot + 2);  // abort: this CTA's MMAs have completed

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int acc_cols_max = 2 * a.it_max;
    const int need = NP > 1 ? 2 * acc_cols_max : acc_cols_max;
    const uint32_t ncols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);  // released by this CTA's MMA warp
        }
        mbar_init(accf, 1);
        mbar_init(tmem_empty, kEpiWarps);
        mbar_init(mma_fin, 1);
        *abort_flag = 0;
        mbar_fence_init();
        if (!BATCH) {
            tma_prefetch_desc(&one.mapX);
            tma_prefetch_desc(&one.mapE);
        } else if (blockIdx.x == 0) {
            for (int q = 0; q < a.nprob; ++q)
                if (many[q].zero_word) *many[q].zero_word = 0u;
        }
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t armed = 0, armed_ph = 0;  // producer: slots armed, and the parity of their last arming
    const int rank = int(blockIdx.x & 1);
    const int64_t cid = blockIdx.x / 2, nclusters = gridDim.x / 2;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t gk = 0;  // k-blocks issued by this CTA over all items
            for (int64_t P = cid; P < a.total_pairs && !*abort_flag; P += nclusters) {
                const TcProblem &pr = problem_of<BATCH>(P, one, many, a.nprob);
                const CUtensorMap *mx = &pr.mapX, *me = &pr.mapE;
                const int64_t right = pr.right, aps = pr.aps;
                const int ni = pr.ni, kblocks = pr.kblocks;
                const uint32_t tx = uint32_t(pr.tx_bytes);
                const int64_t pl = P - pr.pairs_begin;
                const int64_t tile = (pl / ni) * 2 + rank;
                const int h = int(pl % ni);
                const int it = pr.it, half_rows = it / 2;
                // TMA coordinates of this item's two 64-point atoms (MN-major), fixed over k
                int ac_l[2] = {0, 0}, ac_r[2] = {0, 0};
                if (!KMAJOR) {
                    for (int q = 0; q < 2; ++q) {
                        const int64_t atom = 2 * tile + q;
                        int64_t r = atom / aps;
                        if (r > right) r = right;  // past the end: zero fill
                        ac_r[q] = int(r);
                        ac_l[q] = int((atom % aps) * 64);
                    }
                }
                // matrix tiles are stored contiguously per (piece, row tile, k-block): C, S blocks of it rows
                const int e_row0 = h * kblocks * kBlocks * it;
                const int e_pstride = ni * kblocks * kBlocks * it;
                const int k_row = int(tile * kTileM);
                for (int kb = pr.kb_lo[h]; kb < pr.kb_hi[h]; ++kb, ++gk) {
                    const int s = int(gk % kStages);
                    const uint32_t ph = (gk / kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * a.stage_bytes;
                    mbar_arrive_expect_tx(&full[s], tx);
                    armed |= 1u << s;
                    armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
                    for (int c = 0; c < 2; ++c)
                        for (int p = 0; p < NP; ++p) {
                            uint8_t *dst = st + (c * NP + p) * kDataTileBytes;
                            if (KMAJOR) {
                                tma_load_3d(mx, &full[s], dst, kb * kBK, k_row, c * NP + p);
                            } else {
                                tma_load_4d(mx, &full[s], dst, ac_l[0], kb * kBK, ac_r[0], c * NP + p);
                                tma_load_4d(mx, &full[s], dst + 2048, ac_l[1], kb * kBK, ac_r[1], c * NP + p);
                            }
                        }
                    // every matrix block, in two boxes of half the rows each
                    uint8_t *est = st + a.e_offset;
                    for (int p = 0; p < NP; ++p)
                        for (int w = 0; w < kBlocks; ++w)
                            for (int hr = 0; hr < 2; ++hr)
                                tma_load_2d(me, &full[s], est + (p * kBlocks + w) * it * 32 + hr * half_rows * 32, 0,
                                            p * e_pstride + e_row0 + (kb * kBlocks + w) * it + hr * half_rows);
                }
            }
        }
        __syncwarp();  // the role's other lanes wait for it: the warp meets the block barrier converged
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t gk = 0, lt = 0;
            for (int64_t P = cid; P < a.total_pairs && !*abort_flag; P += nclusters, ++lt) {
                const TcProblem &pr = problem_of<BATCH>(P, one, many, a.nprob);
                const int it = pr.it, acc_cols = 2 * it;
                const int hh = int((P - pr.pairs_begin) % pr.ni);
                const int kb_lo = pr.kb_lo[hh], kb_hi = pr.kb_hi[hh];
                const uint32_t idesc_full = FX ? idesc_f16_f32(kTileM, 2 * it, !KMAJOR, false)
                                               : idesc_bf16_f32(kTileM, 2 * it, !KMAJOR, false);
                const uint32_t idesc_half = FX ? idesc_f16_f32(kTileM, it, !KMAJOR, false)
                                               : idesc_bf16_f32(kTileM, it, !KMAJOR, false);
                const uint32_t idesc_half_neg = idesc_half | (1u << 13);  // negate A
                if (lt > 0 && !mbar_wait(tmem_empty, (lt - 1) & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                bool started[2] = {false, false};
                for (int kb = kb_lo; kb < kb_hi; ++kb, ++gk) {
                    const int s = int(gk % kStages);
                    const uint32_t ph = (gk / kStages) & 1u;
                    if (!mbar_wait(&full[s], ph, a.err, MM_ERR_TIMEOUT, a.wait_limit)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + s * a.stage_bytes);
                    const uint32_t est = st + a.e_offset;
                    // real plane: one MMA over the window [C; S] writes (re, im) columns;
                    // imaginary plane: -Xi S into the re columns (negated A), Xi C into the im columns
#pragma unroll
                    for (int t = 0; t < num_terms(NP); ++t) {
                        const int pa = term_a(t), pb = term_b(t);
                        const int acc = (NP > 1 && (pa != 0 || pb != 0)) ? 1 : 0;
                        const uint32_t dcol = tmem + uint32_t(acc * acc_cols);
                        const uint32_t eC = est + (pa * kBlocks + 0) * it * 32;
                        const uint32_t eS = est + (pa * kBlocks + 1) * it * 32;
                        const uint32_t xre = st + (0 * NP + pb) * kDataTileBytes;
                        const uint32_t xim = st + (1 * NP + pb) * kDataTileBytes;
                        const uint64_t are = KMAJOR ? smem_desc(xre, 16, 256, kSwz32) : smem_desc(xre, 2048, 1024, kSwz128);
                        const uint64_t aim = KMAJOR ? smem_desc(xim, 16, 256, kSwz32) : smem_desc(xim, 2048, 1024, kSwz128);
                        umma_f16(dcol, are, smem_desc(eC, 16, 256, kSwz32), idesc_full, started[acc] ? 1u : 0u);
                        started[acc] = true;
                        umma_f16(dcol, aim, smem_desc(eS, 16, 256, kSwz32), idesc_half_neg, 1u);
                        umma_f16(dcol + uint32_t(it), aim, smem_desc(eC, 16, 256, kSwz32), idesc_half, 1u);
                    }
                    umma_commit(&empty[s]);
                }
                umma_commit(accf);
            }
            if (*abort_flag) {  // every MMA this thread issued completes before tensor memory is freed
                umma_commit(mma_fin);
                mbar_wait(mma_fin, 0u, nullptr, 0, a.wait_limit);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        const int ew = warp - 2;          // 0 .. kEpiWarps - 1
        const int quarter = warp % 4;     // TMEM lanes 32 quarter .. + 31
        const int grp = ew / 4;           // chunks of 16 rows: grp, grp + 4, ...
        const int row = quarter * 32 + lane;
        const uint32_t tbase = tmem + (uint32_t(quarter * 32) << 16);
        bool range_ok = true;
        uint32_t lt = 0;
        // running maximum of |output|, flushed (one atomicMax per warp) when the problem changes
        float local_max = 0.0f;
        unsigned *max_word = nullptr;
        auto flush_max = [&]() {
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(local_max));
            if (lane == 0 && m && max_word) atomicMax(max_word, m);
            local_max = 0.0f;
        };
        for (int64_t P = cid; P < a.total_pairs; P += nclusters, ++lt) {
            const TcProblem &pr = problem_of<BATCH>(P, one, many, a.nprob);
            const int64_t right = pr.right, aps = pr.aps, mp = pr.mp, left = pr.left, plane_out = pr.plane_out;
            uint16_t *const out = pr.out;
            const float *const rho = pr.rho;
            const int ni = pr.ni;
            if (FX && pr.sc.max_cur != max_word) {
                flush_max();
                max_word = pr.sc.max_cur;
            }
            const int64_t pl = P - pr.pairs_begin;
            const int64_t tile = (pl / ni) * 2 + rank;
            const int h = int(pl % ni);
            const int it = pr.it, acc_cols = 2 * it, nchunks = it / 16;
            float s_in = 1.0f, inv_out = 1.0f, lim = 0.0f;
            if (FX) {
                s_in = *pr.sc.s_in;
                const int es_out = grid_exponent(__uint_as_float(*pr.sc.max_prev));
                inv_out = ldexpf(1.0f, -es_out);
                lim = ldexpf(16384.0f, es_out);
                if (ew == 0 && lane == 0) *pr.sc.s_out = ldexpf(1.0f, es_out);  // same value from every CTA
            }
            const bool acc_ready = !*abort_flag && mbar_wait(accf, lt & 1u, a.err, MM_ERR_TIMEOUT, a.wait_limit);
            if (!acc_ready) *abort_flag = 1;
            tc_fence_after();
            // drain: up to kChunksPerWarp chunks of 16 rows, real and imaginary, both accumulators summed
            float v[kChunksPerWarp][32];
#pragma unroll
            for (int q = 0; q < kChunksPerWarp; ++q) {
                const int ch = grp + 4 * q;
                if (ch < nchunks) {
                    float t0[16], t1[16];
                    tmem_ld16(tbase + uint32_t(ch * 16), t0);
                    if (NP > 1) tmem_ld16(tbase + uint32_t(acc_cols + ch * 16), t1);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[q][k] = NP > 1 ? t0[k] + t1[k] : t0[k];
                    tmem_ld16(tbase + uint32_t(it + ch * 16), t0);
                    if (NP > 1) tmem_ld16(tbase + uint32_t(acc_cols + it + ch * 16), t1);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[q][16 + k] = NP > 1 ? t0[k] + t1[k] : t0[k];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive(tmem_empty);
            if (!acc_ready) break;
            // this thread's point
            bool valid;
            int64_t r, l = 0;
            if (KMAJOR) {
                r = tile * kTileM + row;
                valid = r < right;
            } else {
                const int64_t atom = 2 * tile + row / 64;
                r = atom / aps;
                l = (atom % aps) * 64 + row % 64;
                valid = r < right && l < left;
            }
#pragma unroll
            for (int q = 0; q < kChunksPerWarp; ++q) {
                const int ch = grp + 4 * q;
                if (ch >= nchunks || !valid) continue;
                const int64_t i0 = int64_t(h) * it + ch * 16;
                if (i0 >= mp) continue;
                // scale (fixed point), nonlinear phase, range and maximum, in place
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    float xr = v[q][k], xi = v[q][16 + k];
                    if (FX) {
                        const float g = __ldg(rho + i0 + k) * s_in;  // power of two: exact
                        xr *= g;
                        xi *= g;
                    }
                    if (EPI == 1) {
                        const float th = a.tb * (xr * xr + xi * xi);
                        float sn, cs;
                        sincosf(th, &sn, &cs);
                        const float yr = xr * cs + xi * sn, yi = xi * cs - xr * sn;
                        xr = yr;
                        xi = yi;
                    }
                    if (FX) {
                        const float ar = fabsf(xr), ai = fabsf(xi);
                        local_max = fmaxf(local_max, fmaxf(ar, ai));
                        range_ok &= ar < lim && ai < lim;
                        xr *= inv_out;
                        xi *= inv_out;
                    }
                    v[q][k] = xr;
                    v[q][16 + k] = xi;
                }
                // pieces of one value: fixed point (already divided by the grid) or floating BF16
                auto pieces_of = [&](float x, uint16_t *b) {
                    if (FX) {
                        split_fx_scaled(x, b[0], b[1], b[2]);
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const __nv_bfloat16 h16 = __float2bfloat16_rn(x);
                            b[p] = __bfloat16_as_ushort(h16);
                            x -= __bfloat162float(h16);
                        }
                    }
                };
                if (KMAJOR) {
                    // 16 consecutive outputs of one row: one 32-byte store per (plane, piece)
                    const int64_t base = r * mp + i0;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        uint32_t w[3][8];
#pragma unroll
                        for (int k2 = 0; k2 < 8; ++k2) {
                            uint16_t b0[3], b1[3];
                            pieces_of(v[q][16 * c + 2 * k2], b0);
                            pieces_of(v[q][16 * c + 2 * k2 + 1], b1);
#pragma unroll
                            for (int p = 0; p < NP; ++p) w[p][k2] = uint32_t(b0[p]) | (uint32_t(b1[p]) << 16);
                        }
#pragma unroll
                        for (int p = 0; p < NP; ++p) st_global_v8(out + int64_t(c * NP + p) * plane_out + base, w[p]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        uint16_t br[3], bi[3];
                        pieces_of(v[q][k], br);
                        pieces_of(v[q][16 + k], bi);
                        const int64_t off = (r * mp + i0 + k) * left + l;
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            out[int64_t(p) * plane_out + off] = br[p];
                            out[int64_t(NP + p) * plane_out + off] = bi[p];
                        }
                    }
                }
            }
        }
        if (FX) flush_max();
        if (FX && !range_ok && a.err) atomicCAS(a.err, 0, MM_ERR_RANGE);
    }
    tc_fence_before();
    __syncthreads();
    // A wait ran out (the flag is final here): every load into this CTA lands before it exits (bounded).
    if (warp == 0 && lane == 0 && *abort_flag)
        for (int q = 0; q < kStages; ++q)
            if (armed & (1u << q)) mbar_wait(&full[q], (armed_ph >> q) & 1u, nullptr, 0, a.wait_limit);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// ---- host: tensor maps and launch -------------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

static bool encode(CUtensorMap *map, void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
                   const cuuint32_t *box, CUtensorMapSwizzle swz, bool four_bytes = false)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    // 16-bit elements (BF16 or FP16 pieces: TMA copies them bit for bit; zero fill is +0 in both),
    // or 32-bit ones (TF32 pieces in FP32 containers)
    return fn(map, four_bytes ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, cuuint32_t(rank),
              base, dims, strides_bytes, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NP, bool KM, int EPI, bool FX, bool PAIR>
static cudaError_t launch_tc(const CUtensorMap &mx, const CUtensorMap &me, const CUtensorMap &my, const TcArgs &a,
                             int grid, int smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(PAIR ? pair_threads(a.it > 64 ? 2 : 1, EPI, false) : kThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // may overlap the tail of the previous kernel in the stream (the kernel waits for it, griddepcontrol)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e;
    if constexpr (PAIR) {
        auto kern = a.it > 64 ? tc_pair_kernel<NP, KM, EPI, FX, 2, false> : tc_pair_kernel<NP, KM, EPI, FX, 1, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        // persistent grid: no more clusters than can be resident at once
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && 2 * active < grid)
            cfg.gridDim = dim3(unsigned(2 * active));
        e = cudaLaunchKernelEx(&cfg, kern, mx, me, my, a, static_cast<const TcPairProblem *>(nullptr), 0,
                               int64_t(0));
    } else {
        auto kern = tc_mode_kernel<NP, KM, EPI, FX>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && 2 * active < grid)
            cfg.gridDim = dim3(unsigned(2 * active));
        e = cudaLaunchKernelEx(&cfg, kern, mx, me, a);
    }
    count_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The one-SM kernel on TF32 pieces (two pieces, plain epilogue).
template <bool KM>
static cudaError_t launch_tc_tf32(const CUtensorMap &mx, const CUtensorMap &me, const TcArgs &a, int grid, int smem,
                                  cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    auto kern = tc_mode_kernel<2, KM, 0, false, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && 2 * active < grid)
        cfg.gridDim = dim3(unsigned(2 * active));
    e = cudaLaunchKernelEx(&cfg, kern, mx, me, a);
    count_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int NP, bool FX, bool PAIR>
static cudaError_t dispatch_np(bool km, int epi, const CUtensorMap &mx, const CUtensorMap &me, const CUtensorMap &my,
                               const TcArgs &a, int grid, int smem, cudaStream_t s)
{
    if (epi >= 2) {  // point phase, GPE adjoint, weighted norm: CTA-pair kernel, F16X6 only
        if constexpr (PAIR && NP == 3 && FX) {
            if (epi == 2)
                return km ? launch_tc<NP, true, 2, FX, PAIR>(mx, me, my, a, grid, smem, s)
                          : launch_tc<NP, false, 2, FX, PAIR>(mx, me, my, a, grid, smem, s);
            if (epi == 3)
                return km ? launch_tc<NP, true, 3, FX, PAIR>(mx, me, my, a, grid, smem, s)
                          : launch_tc<NP, false, 3, FX, PAIR>(mx, me, my, a, grid, smem, s);
            if (epi == 4)
                return km ? launch_tc<NP, true, 4, FX, PAIR>(mx, me, my, a, grid, smem, s)
                          : launch_tc<NP, false, 4, FX, PAIR>(mx, me, my, a, grid, smem, s);
            if (epi == 5)
                return km ? launch_tc<NP, true, 5, FX, PAIR>(mx, me, my, a, grid, smem, s)
                          : launch_tc<NP, false, 5, FX, PAIR>(mx, me, my, a, grid, smem, s);
        }
        return cudaErrorNotSupported;
    }
    if (km)
        return epi ? launch_tc<NP, true, 1, FX, PAIR>(mx, me, my, a, grid, smem, s)
                   : launch_tc<NP, true, 0, FX, PAIR>(mx, me, my, a, grid, smem, s);
    return epi ? launch_tc<NP, false, 1, FX, PAIR>(mx, me, my, a, grid, smem, s)
               : launch_tc<NP, false, 0, FX, PAIR>(mx, me, my, a, grid, smem, s);
}

// The pair tiling a variant runs on, or null for the one-SM kernel (also where the matrix lacks it).
static const TcMatrix::TcPairTiles *pair_tiles(const TcMatrix &M, TcVariant v)
{
    if (v == kTcOneSM) return nullptr;
    const TcMatrix::TcPairTiles &P = M.pair[v == kTcPair128 ? 1 : 0];  // kTcChain: row tiles of 64
    return P.pieces ? &P : nullptr;
}

bool tc_pair_ready(const TcMatrix &M, TcVariant variant) { return pair_tiles(M, variant) != nullptr; }

// Everything a launch of one product needs: tensor maps, kernel arguments,
// which kernel (K-major or not, pair or one-SM), grid and shared memory.
struct TcLaunch {
    CUtensorMap mx, me, my;
    TcArgs a;
    bool km = false, pair = false, fx = false;
    int np = 0, grid = 0, smem = 0;
};

// batch: the launch is a record of a batched pair launch (its stage layout).
static cudaError_t tc_setup(const TcState &si, const TcState &so, int mu, const TcMatrix &M, mm_prec prec,
                            const void *in_pieces, void *out_pieces, const TcEpilogue &epi, const TcScales &sc,
                            int *d_err, TcVariant variant, TcLaunch *L, bool batch = false)
{
    const int NP = tc_pieces(prec);
    const bool fx = tc_fixed(prec);
    const bool tf = tc_tf32(prec);
    if (NP == 0 || NP != M.npieces || fx != M.fixed || tf != M.tf32) return cudaErrorInvalidValue;
    if (fx && (!sc.s_in || !sc.s_out || !sc.max_prev || !sc.max_cur || !M.rho)) return cudaErrorInvalidValue;
    if (tf && (epi.kind != 0 || batch)) return cudaErrorNotSupported;  // TF32: plain products, one-SM kernel
    TcArgs &a = L->a;
    a = TcArgs{};
    a.left = 1;
    a.right = 1;
    for (int v = 0; v < mu - 1; ++v) a.left *= si.np[v];
    for (int v = mu; v < si.d; ++v) a.right *= si.np[v];
    a.kp = si.np[mu - 1];
    a.mp = so.np[mu - 1];
    if (a.kp != M.k_pad) return cudaErrorInvalidValue;
    a.aps = (a.left + 63) / 64;
    a.plane_out = so.plane;
    a.it = M.it;
    a.ni = M.ni;
    a.kblocks = int(a.kp / kBK);
    for (int h = 0; h < 8; ++h) {
        a.kb_lo[h] = h < M.ni ? M.kb_lo[h] : 0;
        a.kb_hi[h] = h < M.ni ? M.kb_hi[h] : 1;
    }
    a.e_offset = 2 * NP * kDataTileBytes;
    a.tx_bytes = a.e_offset + NP * kBlocks * M.it * 32;
    a.stage_bytes = (a.tx_bytes + 1023) / 1024 * 1024;
    a.tb = float(epi.tb);
    a.pl0 = epi.pl0;
    a.pl1 = epi.pl1;
    a.pr0 = epi.pr0;
    a.pr1 = epi.pr1;
    a.ldiv = epi.ldiv > 0 ? epi.ldiv : 1;
    a.rdiv = epi.rdiv > 0 ? epi.rdiv : 1;
    a.mid_out = epi.mid_out;
    a.mid_in = epi.mid_in;
    a.wl0 = epi.wl0;
    a.wl1 = epi.wl1;
    a.wr0 = epi.wr0;
    a.wr1 = epi.wr1;
    a.wo = epi.wo;
    a.norm2 = epi.norm2;
    if ((epi.kind == 3 && !epi.mid_out) || (epi.kind == 4 && !epi.mid_in)) return cudaErrorInvalidValue;
    if (epi.kind == 5 && (!epi.wo || !epi.norm2)) return cudaErrorInvalidValue;
    a.out = (uint16_t *)out_pieces;
    a.err = d_err;
    wait_hooks(&a.wait_limit, &a.withhold);
    a.rho = M.rho;
    a.sc = sc;
    const bool km = a.left == 1;
    if (tf) {
        // TF32 pieces: 4-byte elements, k-blocks of 8 (32-byte rows, the same stage bytes as the 16-bit
        // pieces), MN-major tiles of four 32-point atoms; the one-SM kernel only
        a.kblocks = int(a.kp / 8);
        a.aps = (a.left + 31) / 32;
        CUtensorMap &mx = L->mx, &me = L->me;
        void *xin = const_cast<void *>(in_pieces);
        if (km) {
            cuuint64_t dims[3] = {cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[2] = {cuuint64_t(a.kp * 4), cuuint64_t(si.plane * 4)};
            cuuint32_t box[3] = {8, kTileM, 1};
            if (!encode(&mx, xin, 3, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B, true)) return cudaErrorInvalidValue;
        } else {
            cuuint64_t dims[4] = {cuuint64_t(a.left), cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[3] = {cuuint64_t(a.left * 4), cuuint64_t(a.left * a.kp * 4), cuuint64_t(si.plane * 4)};
            cuuint32_t box[4] = {32, 8, 1, 1};
            if (!encode(&mx, xin, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B, true)) return cudaErrorInvalidValue;
        }
        const int64_t rows = int64_t(NP) * M.ni * a.kblocks * kBlocks * M.it;
        cuuint64_t dims[2] = {8, cuuint64_t(rows)};
        cuuint64_t str[1] = {32};
        cuuint32_t box[2] = {8, cuuint32_t(M.it / 2)};
        if (!encode(&me, M.pieces, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B, true)) return cudaErrorInvalidValue;
        a.tiles = km ? (a.right + kTileM - 1) / kTileM : (a.right * a.aps + 3) / 4;
        a.pairs = (a.tiles + 1) / 2 * a.ni;
        std::memset(&L->my, 0, sizeof L->my);
        L->km = km;
        L->pair = false;
        L->fx = false;
        L->np = NP;
        L->grid = int(2 * (a.pairs < num_sms() / 2 ? a.pairs : num_sms() / 2));
        L->smem = kStages * a.stage_bytes + 1024 + 256;
        return cudaSuccess;
    }

    CUtensorMap &mx = L->mx, &me = L->me;
    void *xin = const_cast<void *>(in_pieces);
    if (km) {
        cuuint64_t dims[3] = {cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
        cuuint64_t str[2] = {cuuint64_t(a.kp * 2), cuuint64_t(si.plane * 2)};
        cuuint32_t box[3] = {kBK, kTileM, 1};
        if (!encode(&mx, xin, 3, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B)) return cudaErrorInvalidValue;
    } else {
        cuuint64_t dims[4] = {cuuint64_t(a.left), cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
        cuuint64_t str[3] = {cuuint64_t(a.left * 2), cuuint64_t(a.left * a.kp * 2), cuuint64_t(si.plane * 2)};
        cuuint32_t box[4] = {64, kBK, 1, 1};
        if (!encode(&mx, xin, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorInvalidValue;
    }
    const TcMatrix::TcPairTiles *PT = pair_tiles(M, variant);
    const bool pair = PT != nullptr;
    // pair kernel: k-blocks per stage (two with 8 epilogue warps: one data box covers both)
    const int kbs = pair ? pair_kb_per_stage(PT->it > 64 ? 2 : 1, epi.kind, batch) : 1;
    if (pair) {
        // the pair kernel loads all 2 NP piece planes of a tile in one box
        if (km) {
            cuuint64_t dims[3] = {cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[2] = {cuuint64_t(a.kp * 2), cuuint64_t(si.plane * 2)};
            cuuint32_t box[3] = {cuuint32_t(kBK * kbs), kTileM, cuuint32_t(2 * NP)};
            if (!encode(&mx, xin, 3, dims, str, box, kbs == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B))
                return cudaErrorInvalidValue;
            a.e_offset = kbs * 2 * NP * kDataTileBytes;
        } else {
            cuuint64_t dims[4] = {cuuint64_t(a.left), cuuint64_t(a.kp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[3] = {cuuint64_t(a.left * 2), cuuint64_t(a.left * a.kp * 2), cuuint64_t(si.plane * 2)};
            cuuint32_t box[4] = {64, cuuint32_t(kBK * kbs), 1, cuuint32_t(2 * NP)};
            if (!encode(&mx, xin, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorInvalidValue;
            a.e_offset = kbs * 2 * NP * kDataTileBytes;
        }
    }
    if (pair) {
        // the pair kernel's row tiles
        a.it = PT->it;
        a.ni = PT->ni;
        for (int h = 0; h < 8; ++h) {
            a.kb_lo[h] = h < PT->ni ? PT->kb_lo[h] : 0;
            a.kb_hi[h] = h < PT->ni ? PT->kb_hi[h] : 1;
        }
        // blocks [-S; C; S] of it / 2 rows per (piece, row tile, k-block, rank), copied as 128-byte lines
        const int e_bytes = 3 * (PT->it / 2) * 32;
        a.tx_bytes = 2 * (a.e_offset + NP * e_bytes);  // both CTAs' loads complete on the leader's barrier
        a.stage_bytes = (a.e_offset + kbs * NP * e_bytes + 1023) / 1024 * 1024;
        const int64_t lines = int64_t(NP) * PT->ni * (M.k_pad / 16) * 2 * e_bytes / 128;
        cuuint64_t dims[2] = {64, cuuint64_t(lines)};
        cuuint64_t str[1] = {128};
        cuuint32_t box[2] = {64, cuuint32_t(NP * e_bytes / 128)};  // all pieces of (row tile, k-block, rank)
        if (!encode(&me, PT->pieces, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_NONE)) return cudaErrorInvalidValue;
    } else {
        const int64_t rows = int64_t(NP) * M.ni * (M.k_pad / 16) * kBlocks * M.it;
        cuuint64_t dims[2] = {16, cuuint64_t(rows)};
        cuuint64_t str[1] = {32};
        cuuint32_t box[2] = {kBK, cuuint32_t(M.it / 2)};  // each CTA of a pair loads half the rows
        if (!encode(&me, M.pieces, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B)) return cudaErrorInvalidValue;
    }
    int64_t tiles;
    if (km) tiles = (a.right + kTileM - 1) / kTileM;
    else tiles = (a.right * a.aps + 1) / 2;
    a.tiles = tiles;
    a.pairs = (tiles + 1) / 2 * a.ni;
    int64_t grid = 2 * (a.pairs < num_sms() / 2 ? a.pairs : num_sms() / 2);
    // output map of the pair kernel's TMA stores: boxes of 32 points x 16 outputs per (plane, piece)
    CUtensorMap &my = L->my;
    std::memset(&my, 0, sizeof my);
    const int ch = a.it > 64 ? 2 : 1;
    if (pair) {
        if (km) {
            cuuint64_t dims[3] = {cuuint64_t(a.mp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[2] = {cuuint64_t(a.mp * 2), cuuint64_t(so.plane * 2)};
            cuuint32_t box[3] = {16, 32, 1};
            if (!encode(&my, out_pieces, 3, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B)) return cudaErrorInvalidValue;
        } else {
            cuuint64_t dims[4] = {cuuint64_t(a.left), cuuint64_t(a.mp), cuuint64_t(a.right), cuuint64_t(2 * NP)};
            cuuint64_t str[3] = {cuuint64_t(a.left * 2), cuuint64_t(a.left * a.mp * 2), cuuint64_t(so.plane * 2)};
            cuuint32_t box[4] = {32, 16, 1, 1};
            if (!encode(&my, out_pieces, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_64B)) return cudaErrorInvalidValue;
        }
    }
    const int smem = pair ? pair_stages(ch, epi.kind, batch) * a.stage_bytes + pair_staging_bytes(ch, epi.kind, batch) + 1024 + 256
                          : kStages * a.stage_bytes + 1024 + 256;
    L->km = km;
    L->pair = pair;
    L->fx = fx;
    L->np = NP;
    L->grid = int(grid);
    L->smem = smem;
    return cudaSuccess;
}

cudaError_t tc_mode_product(const TcState &si, const TcState &so, int mu, const TcMatrix &M, mm_prec prec,
                            const void *in_pieces, void *out_pieces, const TcEpilogue &epi, const TcScales &sc,
                            int *d_err, cudaStream_t s, TcVariant variant)
{
    if (tc_tf32(prec) && mu > 1) {
        // The tcgen05 TF32 MMA takes the data K-major only (measured: an MN-major TF32 operand gives
        // zeros), so directions after the first run as a first direction on swapped data: the
        // pieces [right][n_mu][left] are swapped to [right][left][n_mu] into the output buffer, the
        // product runs from there into the input buffer (whose contents are no longer needed), and
        // the result is swapped back into the output buffer.  Both buffers hold the larger state.
        int64_t left = 1, right = 1;
        for (int v = 0; v < mu - 1; ++v) left *= si.np[v];
        for (int v = mu; v < si.d; ++v) right *= si.np[v];
        TcState ti, to;
        ti.d = to.d = 3;
        ti.n[0] = si.n[mu - 1];
        ti.np[0] = si.np[mu - 1];
        to.n[0] = so.n[mu - 1];
        to.np[0] = so.np[mu - 1];
        ti.n[1] = ti.np[1] = to.n[1] = to.np[1] = left;
        ti.n[2] = ti.np[2] = to.n[2] = to.np[2] = right;
        ti.plane = si.plane;
        to.plane = so.plane;
        const int planes = 2 * tc_pieces(prec);
        cudaError_t e = swap_last2(in_pieces, out_pieces, right, si.np[mu - 1], left, planes, si.plane, s);
        if (e == cudaSuccess)
            e = tc_mode_product(ti, to, 1, M, prec, out_pieces, const_cast<void *>(in_pieces), epi, sc, d_err, s,
                                variant);
        if (e == cudaSuccess) e = swap_last2(in_pieces, out_pieces, right, left, so.np[mu - 1], planes, so.plane, s);
        return e;
    }
    TcLaunch L;
    cudaError_t e = tc_setup(si, so, mu, M, prec, in_pieces, out_pieces, epi, sc, d_err, variant, &L);
    if (e != cudaSuccess) return e;
    const TcArgs &a = L.a;
    const int kind = epi.kind;
    if (tc_tf32(prec))
        return L.km ? launch_tc_tf32<true>(L.mx, L.me, a, L.grid, L.smem, s)
                    : launch_tc_tf32<false>(L.mx, L.me, a, L.grid, L.smem, s);
    if (L.pair) {
        if (L.fx) return dispatch_np<3, true, true>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
        switch (L.np) {
        case 3: return dispatch_np<3, false, true>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
        case 2: return dispatch_np<2, false, true>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
        default: return dispatch_np<1, false, true>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
        }
    }
    if (L.fx) return dispatch_np<3, true, false>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
    switch (L.np) {
    case 3: return dispatch_np<3, false, false>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
    case 2: return dispatch_np<2, false, false>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
    default: return dispatch_np<1, false, false>(L.km, kind, L.mx, L.me, L.my, a, L.grid, L.smem, s);
    }
}

template <int NP, bool KM, int EPI, bool FX, bool BATCH>
static cudaError_t launch_tcb(const TcProblem &one, const TcProblem *many, const TcBatchArgs &a, int smem, cudaStream_t s)
{
    auto kern = tc_mode_kernel_batched<NP, KM, EPI, FX, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = 2 * (a.total_pairs < num_sms() / 2 ? a.total_pairs : num_sms() / 2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent grid: no more clusters than can be resident at once
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && 2 * active < grid)
        cfg.gridDim = dim3(unsigned(2 * active));
    e = cudaLaunchKernelEx(&cfg, kern, one, many, a);
    count_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int NP, bool FX, bool BATCH>
static cudaError_t dispatch_npb(bool km, int epi, const TcProblem &one, const TcProblem *many, const TcBatchArgs &a,
                                int smem, cudaStream_t s)
{
    if (km)
        return epi ? launch_tcb<NP, true, 1, FX, BATCH>(one, many, a, smem, s)
                   : launch_tcb<NP, true, 0, FX, BATCH>(one, many, a, smem, s);
    return epi ? launch_tcb<NP, false, 1, FX, BATCH>(one, many, a, smem, s)
               : launch_tcb<NP, false, 0, FX, BATCH>(one, many, a, smem, s);
}

cudaError_t tc_problem_build(const TcState &si, const TcState &so, int mu, const TcMatrix &M, mm_prec prec,
                             const void *in_pieces, void *out_pieces, const TcScales &sc, TcProblem *pr, bool *kmajor)
{
    const int NP = tc_pieces(prec);
    const bool fx = tc_fixed(prec);
    if (NP == 0 || NP != M.npieces || fx != M.fixed) return cudaErrorInvalidValue;
    if (fx && (!sc.s_in || !sc.s_out || !sc.max_prev || !sc.max_cur || !M.rho)) return cudaErrorInvalidValue;
    TcProblem q;
    std::memset(&q, 0, sizeof q);
    q.left = 1;
    q.right = 1;
    for (int v = 0; v < mu - 1; ++v) q.left *= si.np[v];
    for (int v = mu; v < si.d; ++v) q.right *= si.np[v];
    const int64_t kp = si.np[mu - 1];
    q.mp = so.np[mu - 1];
    if (kp != M.k_pad) return cudaErrorInvalidValue;
    q.aps = (q.left + 63) / 64;
    q.plane_out = so.plane;
    q.it = M.it;
    q.ni = M.ni;
    q.kblocks = int(kp / kBK);
    for (int h = 0; h < 4; ++h) {
        q.kb_lo[h] = h < M.ni ? M.kb_lo[h] : 0;
        q.kb_hi[h] = h < M.ni ? M.kb_hi[h] : 1;
    }
    q.tx_bytes = 2 * NP * kDataTileBytes + NP * kBlocks * M.it * 32;
    q.out = (uint16_t *)out_pieces;
    q.rho = M.rho;
    q.sc = sc;
    const bool km = q.left == 1;
    void *xin = const_cast<void *>(in_pieces);
    if (km) {
        cuuint64_t dims[3] = {cuuint64_t(kp), cuuint64_t(q.right), cuuint64_t(2 * NP)};
        cuuint64_t str[2] = {cuuint64_t(kp * 2), cuuint64_t(si.plane * 2)};
        cuuint32_t box[3] = {kBK, kTileM, 1};
        if (!encode(&q.mapX, xin, 3, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B)) return cudaErrorInvalidValue;
    } else {
        cuuint64_t dims[4] = {cuuint64_t(q.left), cuuint64_t(kp), cuuint64_t(q.right), cuuint64_t(2 * NP)};
        cuuint64_t str[3] = {cuuint64_t(q.left * 2), cuuint64_t(q.left * kp * 2), cuuint64_t(si.plane * 2)};
        cuuint32_t box[4] = {64, kBK, 1, 1};
        if (!encode(&q.mapX, xin, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_128B)) return cudaErrorInvalidValue;
    }
    {
        const int64_t rows = int64_t(NP) * M.ni * (M.k_pad / 16) * kBlocks * M.it;
        cuuint64_t dims[2] = {16, cuuint64_t(rows)};
        cuuint64_t str[1] = {32};
        cuuint32_t box[2] = {kBK, cuuint32_t(M.it / 2)};  // each CTA of a pair loads half the rows
        if (!encode(&q.mapE, M.pieces, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_32B)) return cudaErrorInvalidValue;
    }
    const int64_t tiles = km ? (q.right + kTileM - 1) / kTileM : (q.right * q.aps + 1) / 2;
    q.pairs = (tiles + 1) / 2 * q.ni;
    *pr = q;
    *kmajor = km;
    return cudaSuccess;
}

static cudaError_t launch_batched(int NP, bool fx, bool km, int epi, const TcProblem &one, const TcProblem *many,
                                  const TcBatchArgs &a, int smem, cudaStream_t s)
{
    if (fx) return dispatch_npb<3, true, true>(km, epi, one, many, a, smem, s);
    switch (NP) {
    case 3: return dispatch_npb<3, false, true>(km, epi, one, many, a, smem, s);
    case 2: return dispatch_npb<2, false, true>(km, epi, one, many, a, smem, s);
    default: return dispatch_npb<1, false, true>(km, epi, one, many, a, smem, s);
    }
}

static int stage_bytes_for(int tx_bytes) { return (tx_bytes + 1023) / 1024 * 1024; }

cudaError_t tc_mode_product_batched(const TcProblem *host_probs, const TcProblem *dev_probs, int nprob, bool kmajor,
                                    mm_prec prec, const TcEpilogue &epi, int *d_err, cudaStream_t s)
{
    if (nprob < 1) return cudaSuccess;
    const int NP = tc_pieces(prec);
    TcBatchArgs a{};
    int max_tx = 0;
    for (int q = 0; q < nprob; ++q) {
        a.total_pairs = std::max(a.total_pairs, host_probs[q].pairs_begin + host_probs[q].pairs);
        a.it_max = std::max(a.it_max, host_probs[q].it);
        max_tx = std::max(max_tx, host_probs[q].tx_bytes);
    }
    a.nprob = nprob;
    a.e_offset = 2 * NP * kDataTileBytes;
    a.stage_bytes = stage_bytes_for(max_tx);
    a.tb = float(epi.tb);
    a.err = d_err;
    int64_t unused_withhold = -1;
    wait_hooks(&a.wait_limit, &unused_withhold);
    const int smem = kStages * a.stage_bytes + 1024 + 256;
    return launch_batched(NP, tc_fixed(prec), kmajor, epi.kind, host_probs[0], dev_probs, a, smem, s);
}

// Tensor-core flops one product issues: every MMA counted as 2 M N K, per
// work item its k-block band times the products of the precision.
// ---- batched CTA-pair launches ---------------------------------------------------

size_t tc_pair_record_bytes() { return sizeof(TcPairProblem); }
size_t tc_pair_record_align() { return alignof(TcPairProblem); }

cudaError_t tc_pair_record_build(const TcState &si, const TcState &so, int mu, const TcMatrix &M, mm_prec prec,
                                 const void *in_pieces, void *out_pieces, const TcScales &sc, void *rec, bool *kmajor,
                                 int64_t *items, int chain_pos)
{
    TcLaunch L;
    cudaError_t e = tc_setup(si, so, mu, M, prec, in_pieces, out_pieces, TcEpilogue{}, sc, nullptr, kTcPair64, &L,
                             chain_pos < 0);
    if (e != cudaSuccess) return e;
    if (!L.pair || L.a.it > 64) return cudaErrorNotSupported;  // the batched pair kernel stores with TMA (CH = 1)
    if (chain_pos >= 0 && !L.fx) return cudaErrorNotSupported;  // chains: the fixed-point pieces only
    TcPairProblem r;
    std::memset(&r, 0, sizeof r);
    r.mapX = L.mx;
    r.mapE = L.me;
    r.mapY = L.my;
    r.a = L.a;
    r.pairs_begin = 0;
    r.km = L.km ? 1 : 0;
    r.prod = chain_pos < 0 ? 0 : chain_pos;
    r.last_dir = mu == si.d ? 1 : 0;
    r.slab_div = mu < si.d ? L.a.right / si.np[si.d - 1] : 1;
    r.wait_prod = -1;
    std::memcpy(rec, &r, sizeof r);
    *kmajor = L.km;
    *items = L.a.pairs;
    return cudaSuccess;
}

// The dependencies of a chain's products (records built with positions 0 .. nprod - 1 of a
// d-direction sweep sequence): items of the last direction in row-tile-major order, what
// completes each product and each of its slab groups, and the product that must be complete
// before a product's first load (two back, or one for d = 1: the buffer a product overwrites was
// read two products back, and its scale comes from the maximum of the product d back);
// s_in_max[k]: the maximum word whose grid exponent is product k's input scale (null: its s_in).
cudaError_t tc_pair_chain_plan(void *host_recs, int nprod, int d, const unsigned *const *s_in_max)
{
    auto *h = reinterpret_cast<TcPairProblem *>(host_recs);
    for (int q = 0; q < nprod; ++q) {
        TcPairProblem &R = h[q];
        const int64_t np = R.a.pairs / R.a.ni;
        if (R.a.ni < 1 || np * R.a.ni != R.a.pairs || R.a.mp > int64_t(kChainSlabs) * kChainGroups)
            return cudaErrorInvalidValue;
        R.hmajor = R.last_dir;
        std::memset(R.g_expect, 0, sizeof R.g_expect);
        for (int64_t Pl = 0; Pl < R.a.pairs; ++Pl) {
            int64_t pair;
            int hh;
            chain_item(R.a, R.hmajor != 0, Pl, pair, hh);
            for (int rank = 0; rank < 2; ++rank) {
                int g_lo, g_hi;
                chain_groups(R, pair, hh, rank, false, g_lo, g_hi);
                for (int g = g_lo; g <= g_hi; ++g) {
                    if (g < 0 || g >= kChainGroups) return cudaErrorInvalidValue;
                    ++R.g_expect[g];
                }
            }
        }
        R.tot_target = unsigned(2 * R.a.pairs);
        const int back = d >= 2 ? 2 : 1;
        R.wait_prod = q >= back ? q - back : -1;
        R.s_in_max = s_in_max[q];
    }
    return cudaSuccess;
}

void tc_pair_record_set_begin(void *rec, int64_t begin)
{
    reinterpret_cast<TcPairProblem *>(rec)->pairs_begin = begin;
}

bool tc_pair_batch_compatible(const void *host_recs, int nprob)
{
    const auto *h = reinterpret_cast<const TcPairProblem *>(host_recs);
    for (int q = 1; q < nprob; ++q)
        if (h[q].a.it != h[0].a.it || h[q].a.stage_bytes != h[0].a.stage_bytes) return false;
    return nprob >= 1;
}

// The records must agree on what the kernel's launch arguments fix: the row
// tile size (stage layout) and the input layout.
// One persistent launch over a chain of products (records built with chain positions 0, 1, ..,
// in that order, all with row tiles of the same size, then tc_pair_chain_plan): an item's loads
// wait until the slab groups it reads have been stored by the previous product.  `done` holds
// nprod counters and `gcnt` nprod x kChainGroups, all zeroed by the caller before the launch.
int tc_chain_ctas() { return num_sms(); }

cudaError_t tc_pair_chain_launch(const void *host_recs, const void *dev_recs, int nprod, unsigned *done,
                                 unsigned *gcnt, int *d_err, cudaStream_t s)
{
    const auto *h = reinterpret_cast<const TcPairProblem *>(host_recs);
    if (nprod < 1 || !done || !gcnt) return cudaErrorInvalidValue;
    TcArgs a = h[0].a;
    int64_t total = 0;
    for (int q = 0; q < nprod; ++q) {
        if (h[q].a.it != a.it || h[q].a.stage_bytes != a.stage_bytes || h[q].pairs_begin != total || h[q].prod != q)
            return cudaErrorInvalidValue;
        total += h[q].a.pairs;
    }
    a.err = d_err;
    wait_hooks(&a.wait_limit, &a.withhold);
    a.done = done;
    auto kern = tc_pair_kernel<3, false, 0, true, 1, true, true>;
    const int smem = pair_stages(1, 0, false) * a.stage_bytes + pair_staging_bytes(1, 0, false) + 1024 + 256;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(2 * (total < num_sms() / 2 ? total : num_sms() / 2)));
    cfg.blockDim = dim3(pair_threads(1, 0, false) + 32);  // + the signalling warp
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    // every cluster must be resident at once: a product's items wait for the whole previous product
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, kern, &cfg);
    if (e != cudaSuccess || active < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    if (2 * active < int(cfg.gridDim.x)) cfg.gridDim = dim3(unsigned(2 * active));
    a.gcnt = gcnt;
    e = cudaLaunchKernelEx(&cfg, kern, h[0].mapX, h[0].mapE, h[0].mapY, a,
                           reinterpret_cast<const TcPairProblem *>(dev_recs), nprod, total);
    count_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t tc_pair_batch_launch(const void *host_recs, const void *dev_recs, int nprob, bool kmajor, mm_prec prec,
                                 int *d_err, cudaStream_t s)
{
    const auto *h = reinterpret_cast<const TcPairProblem *>(host_recs);
    if (nprob < 1) return cudaErrorInvalidValue;
    TcArgs a = h[0].a;
    int64_t total = 0;
    for (int q = 0; q < nprob; ++q) {
        if (h[q].a.it != a.it || h[q].a.stage_bytes != a.stage_bytes || h[q].pairs_begin != total)
            return cudaErrorInvalidValue;
        total += h[q].a.pairs;
    }
    a.err = d_err;
    wait_hooks(&a.wait_limit, &a.withhold);
    const int NP = tc_pieces(prec);
    const bool fx = tc_fixed(prec);
    const int smem = pair_stages(1, 0, true) * a.stage_bytes + pair_staging_bytes(1, 0, true) + 1024 + 256;
    const int64_t grid = 2 * (total < num_sms() / 2 ? total : num_sms() / 2);
    const auto *dev = reinterpret_cast<const TcPairProblem *>(dev_recs);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(pair_threads(1, 0, true));
        cfg.dynamicSmemBytes = size_t(smem);
        cfg.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0 && 2 * active < grid)
            cfg.gridDim = dim3(unsigned(2 * active));
        e = cudaLaunchKernelEx(&cfg, kern, h[0].mapX, h[0].mapE, h[0].mapY, a, dev, nprob, total);
        count_launch();
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    };
    if (fx) return kmajor ? go(tc_pair_kernel<3, true, 0, true, 1, true>) : go(tc_pair_kernel<3, false, 0, true, 1, true>);
    switch (NP) {
    case 3: return kmajor ? go(tc_pair_kernel<3, true, 0, false, 1, true>) : go(tc_pair_kernel<3, false, 0, false, 1, true>);
    case 2: return kmajor ? go(tc_pair_kernel<2, true, 0, false, 1, true>) : go(tc_pair_kernel<2, false, 0, false, 1, true>);
    default: return kmajor ? go(tc_pair_kernel<1, true, 0, false, 1, true>) : go(tc_pair_kernel<1, false, 0, false, 1, true>);
    }
}

double tc_issued_flops(const TcState &si, int mu, const TcMatrix &M, mm_prec prec, TcVariant variant)
{
    const int NP = tc_pieces(prec);
    int64_t left = 1, right = 1;
    for (int v = 0; v < mu - 1; ++v) left *= si.np[v];
    for (int v = mu; v < si.d; ++v) right *= si.np[v];
    const bool tf = tc_tf32(prec);
    const int64_t aps = tf ? (left + 31) / 32 : (left + 63) / 64;
    const int64_t tiles = left == 1 ? (right + kTileM - 1) / kTileM : (tf ? (right * aps + 3) / 4 : (right * aps + 1) / 2);
    const int64_t tiles_run = (tiles + 1) / 2 * 2;  // CTA pairs
    // the kernel that runs and its row tiling
    const TcMatrix::TcPairTiles *PT = pair_tiles(M, variant);
    const int it = PT ? PT->it : M.it, ni = PT ? PT->ni : M.ni;
    const int *lo = PT ? PT->kb_lo : M.kb_lo, *hi = PT ? PT->kb_hi : M.kb_hi;
    // one k-block of one point tile: per piece product 2 M N K over N = 4 it columns (one-SM kernel: the
    // real plane with N = 2 it and the imaginary plane as two of N = it; pair kernel: two of N = 2 it)
    const double per_kb = double(num_terms(NP)) * 2.0 * kTileM * (4.0 * it) * (tf ? 8 : kBK);
    double total = 0.0;
    for (int h = 0; h < ni; ++h) total += double(tiles_run) * double(hi[h] - lo[h]) * per_kb;
    return total;
}

}  // namespace mm
