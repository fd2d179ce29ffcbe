// mumode_product_noalloc: the F16X6 mu-mode product for callers that must
// not allocate device memory.  Everything the product needs on the device
// besides the caller's input and output -- the split input and output
// states, the matrix pieces, the row scales and the scale / status words --
// lives in one file-scope device array of fixed size, reserved when the
// library's device code is loaded on a GPU and kept until the process
// exits.  The matrix pieces are built on the host in ordinary host memory
// (std::vector) and copied into that array; no device memory is allocated.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB on every GPU that loads the library
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a stand-in for the symbol,
// never a device address: host code uses the pointer from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
mm_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mm::fail(MM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return mm::fail(MM_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return mm::fail(MM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MM_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" mm_status mumode_product_noalloc(int d, const int64_t *n, int mu, const double *L, int64_t m,
                                           int L_is_complex, const void *u_dev, void *s_dev, void *stream)
{
    using mm::fail;
    if (d < 1 || d > mm::kMaxDims) return fail(MM_ERR_SHAPE, "d = %d outside 1..%d", d, mm::kMaxDims);
    if (!n || !L) return fail(MM_ERR_INVALID_ARG, "n or L is NULL");
    if (mu < 1 || mu > d) return fail(MM_ERR_INVALID_ARG, "mu = %d outside 1..%d", mu, d);
    for (int v = 0; v < d; ++v)
        if (n[v] < 1 || n[v] > (int64_t(1) << 24)) return fail(MM_ERR_SHAPE, "n[%d] out of range", v);
    if (m < 1 || m > 256 || n[mu - 1] > 256) return fail(MM_ERR_SHAPE, "n_mu and m must be in 1..256");
    if (!u_dev || !s_dev) return fail(MM_ERR_INVALID_ARG, "u_dev or s_dev is NULL");
    if (reinterpret_cast<uintptr_t>(u_dev) % 16 || reinterpret_cast<uintptr_t>(s_dev) % 16)
        return fail(MM_ERR_ALIGN, "u_dev and s_dev must be 16-byte aligned");

    // Padded sizes and the scratch layout: words | matrix pieces | row scales | input pieces | output pieces.
    int64_t nout[mm::kMaxDims];
    mm::TcState si, so;
    si.d = so.d = d;
    si.plane = so.plane = 1;
    int64_t cnt_in = 1, cnt_out = 1;
    // Every running product stays below the scratch's point capacity (12 bytes per padded point
    // and state), so none of them can overflow before the size check below.
    const int64_t cap_points = int64_t(kScratchBytes / 12);
    for (int v = 0; v < d; ++v) {
        nout[v] = (v == mu - 1) ? m : n[v];
        si.n[v] = n[v];
        so.n[v] = nout[v];
        si.np[v] = (n[v] + 15) / 16 * 16;
        so.np[v] = (nout[v] + 15) / 16 * 16;
        if (si.np[v] > cap_points / si.plane || so.np[v] > cap_points / so.plane)
            return fail(MM_ERR_SHAPE, "this product needs more than the %zu bytes of the static scratch", kScratchBytes);
        si.plane *= si.np[v];
        so.plane *= so.np[v];
        cnt_in *= n[v];
        cnt_out *= nout[v];
    }
    const char *u0 = (const char *)u_dev, *s0 = (const char *)s_dev;
    if (u0 < s0 + cnt_out * 8 && s0 < u0 + cnt_in * 8) return fail(MM_ERR_INVALID_ARG, "u_dev and s_dev overlap");
    const int NP = 3;
    const int64_t nmu = n[mu - 1];
    const int64_t k_pad = (nmu + 15) / 16 * 16, m_pad = (m + 15) / 16 * 16;
    const int64_t ni = (m_pad + 127) / 128, it = ((m_pad + ni - 1) / ni + 15) / 16 * 16;
    const size_t words = 256;
    const size_t mat_bytes = align256(size_t(NP * ni * 2 * it * k_pad) * 2);  // C and S blocks
    const size_t rho_bytes = align256(size_t(ni * it) * sizeof(float));
    const size_t in_bytes = align256(size_t(si.plane) * 2 * NP * 2);
    const size_t out_bytes = align256(size_t(so.plane) * 2 * NP * 2);
    const size_t need = words + mat_bytes + rho_bytes + in_bytes + out_bytes;
    if (need > kScratchBytes)
        return fail(MM_ERR_SHAPE, "this product needs %zu bytes of scratch; the static scratch holds %zu", need,
                    kScratchBytes);

    int dev = -1, major = 0, minor = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return fail(MM_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    if (!(major == 10 && minor == 3)) return fail(MM_ERR_UNSUPPORTED, "needs an sm_103 device");
    void *base = nullptr;
    mm_status st = scratch_address(&base);
    if (st) return st;

    // Matrix pieces built on the host, copied into the scratch.
    std::vector<double> Lc(size_t(2 * m * nmu));
    for (int64_t q = 0; q < m * nmu; ++q) {
        Lc[size_t(2 * q)] = L_is_complex ? L[2 * q] : L[q];
        Lc[size_t(2 * q + 1)] = L_is_complex ? L[2 * q + 1] : 0.0;
    }
    mm::TcMatrix M;
    std::vector<uint16_t> hp;
    std::vector<float> hr;
    if ((st = mm::tc_matrix_host(Lc.data(), m, nmu, NP, true, &M, hp, hr))) return st;
    char *b = static_cast<char *>(base);
    float *scales = reinterpret_cast<float *>(b);        // [0] input scale, [1] output scale
    unsigned *uw = reinterpret_cast<unsigned *>(b);      // [2] bound, [3] max, [4] work
    int *err = reinterpret_cast<int *>(b) + 5;           // status word of this call
    M.pieces = b + words;
    M.rho = reinterpret_cast<float *>(b + words + mat_bytes);
    void *pin = b + words + mat_bytes + rho_bytes;
    void *pout = b + words + mat_bytes + rho_bytes + in_bytes;

    cudaStream_t s = (cudaStream_t)stream;
    mm::TcScales sc;
    sc.s_in = scales;
    sc.s_out = scales + 1;
    sc.max_prev = uw + 2;
    sc.max_cur = uw + 3;
    const double bound = M.row_norm;
    // The scale and status words start at zero on every call; the piece
    // buffers are overwritten in full by the split and the product.
    e = cudaMemsetAsync(b, 0, words, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.pieces, hp.data(), hp.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.rho, hr.data(), hr.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = mm::tc_split(si, NP, true, u_dev, pin, uw + 4, scales, uw + 2, &bound, 1, s);
    if (e == cudaSuccess)
        e = mm::tc_mode_product(si, so, mu, M, MM_PREC_F16X6, pin, pout, mm::TcEpilogue{}, sc, err, s);
    if (e == cudaSuccess) e = mm::tc_merge(so, NP, true, pout, scales + 1, s_dev, s);
    cudaError_t e2 = cudaStreamSynchronize(s);  // also keeps hp / hr alive until their copies finish
    if (e != cudaSuccess) return fail(MM_ERR_CUDA, "no-alloc mode product: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(MM_ERR_CUDA, "no-alloc mode product (sync): %s", cudaGetErrorString(e2));
    int word = 0;
    e = cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MM_ERR_CUDA, "status word read: %s", cudaGetErrorString(e));
    if (word) return fail(mm_status(word), "a device-side check failed (status %d)", word);
    return MM_OK;
}
