// C ABI of the library (declared in include/mumode.h): argument checking,
// contexts, plans and the per-step launch sequences.
#include <cuda_runtime.h>

#include <atomic>
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

// An NVTX range over the scope: each public call and each mode-product launch is a named range
// that profilers show on the timeline and can filter on (ncu --nvtx --nvtx-include ...); without
// a tool attached the calls cost next to nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
static const char *const kModeRangeNames[] = {"mode product 1", "mode product 2", "mode product 3",
                                              "mode product 4", "mode product 5", "mode product 6",
                                              "mode product 7", "mode product 8"};


using cd = std::complex<double>;

struct mm_ctx {
    int device = 0;
    int sm_major = 0, sm_minor = 0;
    int *d_err = nullptr;
    double *d_scratch = nullptr;  // one double for reductions
    // optional CUDA-event timing of the mode-product kernels
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    std::vector<int> event_products;  // mode products each event pair brackets (a chained launch: many)
    size_t events_used = 0;
    mm::ExpmWorkspace expm;  // mm_expm_device, complex z
    mm::ExpmBatch expmb;     // mm_expm_device, imaginary z
};

struct AdjCache;  // split_step_gpe_adjoint's matrices and buffers, kept with the plan

struct mm_plan {
    mm_ctx *ctx = nullptr;
    bool hermite = false;
    int d = 0;
    int64_t n[mm::kMaxDims] = {};
    int64_t count = 0;
    mm_dtype dtype = MM_C64;
    mm_prec prec = MM_PREC_BF16X6;
    int order[mm::kMaxDims] = {};
    bool tc = false;
    bool fixed = false;  // MM_PREC_F16X6
    bool tf32 = false;   // MM_PREC_TF32X3 (4-byte pieces, one-SM kernel, Tucker plans only)
    int npieces = 0;
    mm::TcVariant variant = mm::kTcPair64;  // tensor-core kernel (mm_plan_autotune, mm_plan_set_config)
    // kTcChain: the records of a chained call (one launch for all products of nsteps steps) and its
    // completion counters, kept for the last nsteps used
    int64_t chain_steps = -1;
    int chain_order[mm::kMaxDims] = {};
    unsigned chain_fold = 0;  // the folded directions the records were built for
    int chain_nprod = 0;
    std::vector<uint8_t> chain_host;
    void *chain_dev = nullptr;
    // nprod completion counters, nprod x 32 slab-group counters, then nprod maximum words (one per
    // product: a chain's products never share a maximum word)
    unsigned *chain_done = nullptr;
    // fixed-point state scale words (device): scale[d], max[2][d], one work word
    float *d_scale = nullptr;
    unsigned *d_max = nullptr;
    unsigned *d_work = nullptr;
    int64_t sweep = 0;
    // Tucker matrices (one per direction) in the form of the precision
    void *Edev[mm::kMaxDims] = {};        // SIMT: element type of the state
    mm::TcMatrix Etc[mm::kMaxDims] = {};  // tensor cores
    // Even/odd folding (Tucker plans on the tensor cores): the directions whose matrix is
    // centrosymmetric hold it folded, block-diagonal (Dtc); a step call folds the state once,
    // runs its steps on the folded state and unfolds it once (fold_buf: a complex64 state)
    unsigned fold_mask = 0;   // the directions the steps run folded (0 when folding is off)
    unsigned fold_avail = 0;  // the directions that can fold (Tucker plans: Dtc built)
    bool fold_on = true;      // mm_plan_set_fold
    bool fold_force = false;  // MM_FOLD_ALWAYS at plan creation: fold every call, however short (tests)
    mm::TcMatrix Dtc[mm::kMaxDims] = {};
    void *fold_buf = nullptr;
    // workspace
    mm::TcState st;
    void *work[3] = {nullptr, nullptr, nullptr};  // TC: piece buffers (the third for chains); SIMT: work[0] state-sized
    size_t work_bytes = 0;
    void *staging = nullptr;  // device copy for host stepping
    // Hermite data
    std::vector<double> x[mm::kMaxDims], W[mm::kMaxDims];
    std::vector<double> fwd[mm::kMaxDims], bwd[mm::kMaxDims];
    double *Wdev[mm::kMaxDims] = {};
    double *Wpad[mm::kMaxDims] = {};  // the weights at padded length (zeros past n): the norm epilogue's
    double *d_norm = nullptr;         // the norm epilogue's FP64 sum
    void *Fdev[mm::kMaxDims] = {}, *Bdev[mm::kMaxDims] = {};      // SIMT forward/backward
    mm::TcMatrix Ftc[mm::kMaxDims] = {}, Btc[mm::kMaxDims] = {};  // TC forward/backward
    // cached harmonic propagators Psi D(s) Phi_W for up to two step sizes
    double prop_s[2] = {NAN, NAN};
    void *Pdev[2][mm::kMaxDims] = {};
    mm::TcMatrix Ptc[2][mm::kMaxDims] = {};
    // the same propagators folded (even/odd, block-diagonal) where they are centrosymmetric, for
    // the harmonic-oscillator steps (the GPE's pointwise nonlinearity needs the unfolded state)
    mm::TcMatrix PFtc[2][mm::kMaxDims] = {};
    unsigned pfold_mask[2] = {0u, 0u};
    // HKMP (hkmp_plan_create): per direction the Hamiltonian H0 and the
    // Galerkin matrix G of the time-dependent part (device, FP64), their
    // 1-norms, and the step's exponential exp(-i tau (H0 + f G))
    bool hkmp = false;
    double tau = 0.0;
    double *H0dev[mm::kMaxDims] = {}, *Gdev[mm::kMaxDims] = {};
    double h0norm[mm::kMaxDims] = {}, gnorm[mm::kMaxDims] = {};  // ||H0 - mu I||_1, ||G||_1
    double hshift[mm::kMaxDims] = {};  // mu: the middle of H0's diagonal range, taken out as a phase
    double2 *Ebatch[mm::kMaxDims] = {};  // the exponentials of a chunk of steps (expmb.cap matrices)
    // tensor-core plans: exponentials at kInterpNodes Chebyshev nodes in f per direction, and the
    // device interpolation weights of a chunk (cap x kInterpNodes)
    double2 *hk_nodesE[mm::kMaxDims] = {};
    double *hk_w = nullptr;
    // hkmp_set_f_range: the exponentials at hk_rK Chebyshev nodes of a declared f range
    // [hk_rlo, hk_rhi], kept with the plan (hk_rK = 0: none)
    double2 *hk_rangeE[mm::kMaxDims] = {};
    double hk_rlo = 0.0, hk_rhi = 0.0;
    int hk_rK = 0;
    void *coef = nullptr;  // coefficient tensor of hkmp_evolve
    mm::ExpmBatch expmb;
    // HKMP with one time-dependent direction and harmonic others: a step is that direction's
    // product with the others' phases e^{-i tau (k + 1/2)} multiplied in its epilogue
    int hk_fuse = -1;                           // the time-dependent direction (0-based), or -1
    double2 *hk_phase[mm::kMaxDims] = {};       // per harmonic direction, padded length
    bool full_bands[mm::kMaxDims] = {};  // a device update switched direction v's bands to full
    AdjCache *adj = nullptr;  // built by the first split_step_gpe_adjoint call (and again when tau changes)
    // CUDA graphs of whole step sequences, keyed by (call, tensor, nsteps, stream, tau, beta)
    bool use_graphs = true;
    std::map<std::tuple<int, const void *, int64_t, cudaStream_t, double, double>,
             std::pair<cudaGraphExec_t, long long>>
        graphs;
};

namespace mm {

static thread_local char g_err[512] = "no error";
static std::atomic<long long> g_launches{0};

mm_status fail(mm_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

void count_launch(int k) { g_launches += k; }

}  // namespace mm

using mm::fail;

namespace {

size_t elem_bytes(mm_dtype dt)
{
    switch (dt) {
    case MM_R64: return 8;
    case MM_C64: return 8;
    case MM_C128: return 16;
    case MM_R32: return 4;
    }
    return 0;
}
bool is_complex(mm_dtype dt) { return dt == MM_C64 || dt == MM_C128; }

mm_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(MM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

mm_status check_dims(int d, const int64_t *n)
{
    if (d < 1 || d > mm::kMaxDims) return fail(MM_ERR_SHAPE, "d = %d outside 1..%d", d, mm::kMaxDims);
    if (!n) return fail(MM_ERR_INVALID_ARG, "n is NULL");
    for (int v = 0; v < d; ++v)
        if (n[v] < 1 || n[v] > (int64_t(1) << 24)) return fail(MM_ERR_SHAPE, "n[%d] = %lld out of range", v, (long long)n[v]);
    return MM_OK;
}

mm_status check_ptr(const void *p, const char *name)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % 16) return fail(MM_ERR_ALIGN, "%s is not 16-byte aligned", name);
    return MM_OK;
}

// MM_PREC_AUTO -> a concrete precision for data type dt; tc_fits: every
// contraction and output length within the tensor-core limit (256).
mm_prec resolve_prec(mm_prec pr, mm_dtype dt, bool tc_fits)
{
    if (pr != MM_PREC_AUTO) return pr;
    switch (dt) {
    case MM_C64: return tc_fits ? MM_PREC_F16X6 : MM_PREC_FP32_SIMT;
    case MM_R32: return MM_PREC_FP32_SIMT;
    default: return MM_PREC_FP64_DMMA;
    }
}

mm_status check_combo(mm_dtype dt, mm_prec pr, bool matrix_complex)
{
    switch (pr) {
    case MM_PREC_FP64_SIMT:
    case MM_PREC_FP64_DMMA:
        if (dt == MM_C128 || (dt == MM_R64 && !matrix_complex)) return MM_OK;
        break;
    case MM_PREC_FP32_SIMT:
        if (dt == MM_C64 || (dt == MM_R32 && !matrix_complex)) return MM_OK;
        break;
    case MM_PREC_BF16X6:
    case MM_PREC_BF16X3:
    case MM_PREC_BF16:
    case MM_PREC_F16X6:
    case MM_PREC_TF32X3:
        if (dt == MM_C64) return MM_OK;
        break;
    default: return fail(MM_ERR_INVALID_ARG, "unknown precision %d", int(pr));
    }
    return fail(MM_ERR_DTYPE, "dtype %d is not supported with precision %d%s", int(dt), int(pr),
                matrix_complex ? " and a complex matrix" : "");
}

// Matrix (m x n, host FP64, complex interleaved or real) -> device copy in
// the element type of dt.  Real data types take the real part only.
mm_status upload_simt(const double *L, int64_t m, int64_t n, bool Lc, mm_dtype dt, void **out)
{
    const size_t cnt = size_t(m * n);
    std::vector<uint8_t> buf(cnt * elem_bytes(dt));
    for (size_t q = 0; q < cnt; ++q) {
        const double re = Lc ? L[2 * q] : L[q], im = Lc ? L[2 * q + 1] : 0.0;
        switch (dt) {
        case MM_R64: reinterpret_cast<double *>(buf.data())[q] = re; break;
        case MM_R32: reinterpret_cast<float *>(buf.data())[q] = float(re); break;
        case MM_C128:
            reinterpret_cast<double *>(buf.data())[2 * q] = re;
            reinterpret_cast<double *>(buf.data())[2 * q + 1] = im;
            break;
        case MM_C64:
            reinterpret_cast<float *>(buf.data())[2 * q] = float(re);
            reinterpret_cast<float *>(buf.data())[2 * q + 1] = float(im);
            break;
        }
    }
    cudaError_t e = cudaMalloc(out, buf.size());
    if (e != cudaSuccess) return fail(MM_ERR_OOM, "cudaMalloc(%zu) failed", buf.size());
    e = cudaMemcpy(*out, buf.data(), buf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "matrix upload");
    return MM_OK;
}

// complex interleaved copy of a real or complex host matrix
std::vector<double> as_complex(const double *L, int64_t cnt, bool Lc)
{
    std::vector<double> out(size_t(2 * cnt));
    for (int64_t q = 0; q < cnt; ++q) {
        out[2 * q] = Lc ? L[2 * q] : L[q];
        out[2 * q + 1] = Lc ? L[2 * q + 1] : 0.0;
    }
    return out;
}

mm::TcState make_state(int d, const int64_t *n)
{
    mm::TcState st;
    st.d = d;
    st.plane = 1;
    for (int v = 0; v < d; ++v) {
        st.n[v] = n[v];
        st.np[v] = (n[v] + 15) / 16 * 16;
        st.plane *= st.np[v];
    }
    return st;
}

void left_right(int d, const int64_t *n, int mu, int64_t *left, int64_t *right)
{
    *left = 1;
    *right = 1;
    for (int v = 0; v < mu - 1; ++v) *left *= n[v];
    for (int v = mu; v < d; ++v) *right *= n[v];
}

// Events bracketing one mode-product launch when timing is on (the end event records how many
// mode products the launch ran: one, or a chained call's all).
cudaEvent_t timing_event(mm_ctx *c, bool start, int products = 1)
{
    if (!c->timing) return nullptr;
    if (start) {
        if (c->events_used == c->events.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
            if (cudaEventCreate(&b) != cudaSuccess) {
                cudaEventDestroy(a);
                return nullptr;
            }
            c->events.push_back({a, b});
            c->event_products.push_back(1);
        }
        return c->events[c->events_used].first;
    }
    c->event_products[c->events_used] = products;
    return c->events[c->events_used++].second;
}

// The tensor-core matrix the steps of a Tucker plan use in direction v (0-based): the folded
// block-diagonal form where the plan folds that direction.
mm::TcMatrix *step_matrix(mm_plan *p, int v) { return ((p->fold_mask >> v) & 1u) ? &p->Dtc[v] : &p->Etc[v]; }
const mm::TcMatrix *step_matrix(const mm_plan *p, int v)
{
    return ((p->fold_mask >> v) & 1u) ? &p->Dtc[v] : &p->Etc[v];
}

// Whether a call of nsteps steps should run folded: the tensor-core work the folded matrices save
// (issued flops, at 1.5 PFLOP/s) must exceed the fold and unfold passes (two reads and two writes
// of the complex64 state, at 6.5 TB/s).  Banded matrices save a few blocks per row tile and fold
// from about four steps per call; dense ones save half of every product and fold from one.
double fold_saved_s(const mm_plan *p, unsigned mask, mm::TcMatrix *const *unfolded, mm::TcMatrix *const *folded)
{
    double saved = 0.0;
    for (int v = 0; v < p->d; ++v)
        if ((mask >> v) & 1u)
            saved += mm::tc_issued_flops(p->st, v + 1, *unfolded[v], p->prec, p->variant) -
                     mm::tc_issued_flops(p->st, v + 1, *folded[v], p->prec, p->variant);
    return saved / 1.5e15;
}

bool fold_pays(const mm_plan *p, unsigned mask, mm::TcMatrix *const *unfolded, mm::TcMatrix *const *folded,
               int64_t nsteps)
{
    if (!mask) return false;
    if (p->fold_force) return true;
    const double cost_s = 4.0 * double(p->count) * 8.0 / 6.5e12;
    return double(nsteps) * fold_saved_s(p, mask, unfolded, folded) > cost_s;
}

// One Tucker sweep on the TC piece state: modes in plan order with
// matrices M[mu-1]; cur is the index of the buffer holding the state.
mm_status tc_sweep(mm_plan *p, mm::TcMatrix *const *M, int &cur, const mm::TcEpilogue &last_epi, cudaStream_t s)
{
    for (int q = 0; q < p->d; ++q) {
        const int mu = p->order[q];
        mm::TcEpilogue epi;
        if (q == p->d - 1) epi = last_epi;
        mm::TcScales sc;
        if (p->fixed) {
            // Three sets of maximum words, W[t][q] = d_max[t d + q], rotate with the sweep k (t = k mod 3):
            // launch (k, q) reads W[t-1][q] (sweep k-1's maximum), accumulates into W[t][q] and clears
            // W[t+1][q] for sweep k+1.  That word was last read by launch (k-1, q), which has completed,
            // and the launch itself neither reads nor writes it, whatever d is (with two sets and
            // d = 1 it would be the word the launch reads).  tc_begin clears W[0][*] for sweep 0.
            const int t = int(p->sweep % 3), d = p->d, par = int(p->sweep & 1);
            // state scales S[par][q] = d_scale[par d + q]: launch (k, q) reads S[k mod 2][q] and writes
            // the next position's, S[k mod 2][q + 1] or, after the last position, S[k + 1 mod 2][0]
            // (never the word it reads, also for d = 1)
            sc.s_in = p->d_scale + par * d + q;
            sc.s_out = (q + 1 < d) ? p->d_scale + par * d + q + 1 : p->d_scale + (1 - par) * d;
            sc.max_prev = p->d_max + ((t + 2) % 3) * d + q;
            sc.max_cur = p->d_max + t * d + q;
            sc.zero_next = p->d_max + ((t + 1) % 3) * d + q;
        }
        NvtxRange range(kModeRangeNames[(mu - 1) & 7]);
        cudaEvent_t ev0 = timing_event(p->ctx, true);
        if (ev0) cudaEventRecord(ev0, s);
        cudaError_t e = mm::tc_mode_product(p->st, p->st, mu, *M[mu - 1], p->prec, p->work[cur], p->work[1 - cur],
                                            epi, sc, p->ctx->d_err, s, p->variant);
        if (ev0) cudaEventRecord(timing_event(p->ctx, false), s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core mode product launch");
        cur = 1 - cur;
    }
    ++p->sweep;
    return MM_OK;
}

// kTcChain: the records of a chained call of nsteps Tucker steps with the plan's matrices, in
// the plan's mode order: product k d + q of the call is position q of sweep k, with the buffers and
// scale words tc_sweep gives it (tc_begin precedes, so sweep 0 and buffer 0 come first).  Built
// once per (nsteps, order) and kept; a rebuild drops the plan's graphs, which point at the old
// records.  false: the products cannot be chained (no pair tiling with row tiles of at most 64,
// row tiles of different sizes, too many products); the caller launches them one by one.
void drop_graphs(mm_plan *p);

bool chain_prepare(mm_plan *p, int64_t nsteps, unsigned fold)
{
    const int d = p->d;
    if (p->chain_steps == nsteps && p->chain_fold == fold && std::equal(p->order, p->order + d, p->chain_order))
        return true;
    if (!p->tc || !p->fixed || p->hermite || nsteps < 1 || nsteps * d > (int64_t(1) << 20)) return false;
    const int nprod = int(nsteps * d);
    const size_t rb = mm::tc_pair_record_bytes(), al = mm::tc_pair_record_align();
    std::vector<uint8_t> host(rb * size_t(nprod) + al, 0);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(host.data()) + al - 1) / al * al);
    // Products overlap in a chain, so the state rotates through three buffers (product k reads
    // buffer k mod 3 and writes k + 1 mod 3, which product k - 2 read) and each product has a
    // maximum word of its own: product k's output scale comes from product k - d's maximum (sweep
    // 0: the bounds the split writes), its input scale from product k - 1's.
    if (!p->work[2]) {
        if (cudaMalloc(&p->work[2], p->work_bytes) != cudaSuccess) {
            p->work[2] = nullptr;
            return false;
        }
        if (cudaMemset(p->work[2], 0, p->work_bytes) != cudaSuccess) return false;
    }
    const size_t counters = size_t(nprod) * (mm::kChainCounters + 1);
    unsigned *done = nullptr;
    if (cudaMalloc(&done, sizeof(unsigned) * counters) != cudaSuccess) return false;
    unsigned *maxw = done + size_t(nprod) * mm::kChainCounters;
    std::vector<const unsigned *> s_in_max(size_t(nprod), nullptr);
    std::vector<const unsigned *> max_prev(size_t(nprod), nullptr);
    int64_t begin = 0;
    for (int64_t k = 0; k < nsteps; ++k)
        for (int q = 0; q < d; ++q) {
            const int pos = int(k * d + q), mu = p->order[q];
            const int par = int(k & 1);  // the state scale words as tc_sweep with p->sweep = k
            mm::TcScales sc;
            sc.s_in = p->d_scale + par * d + q;
            sc.s_out = (q + 1 < d) ? p->d_scale + par * d + q + 1 : p->d_scale + (1 - par) * d;
            sc.max_prev = pos >= d ? maxw + (pos - d) : p->d_max + 2 * d + q;
            sc.max_cur = maxw + pos;
            sc.zero_next = nullptr;
            max_prev[size_t(pos)] = sc.max_prev;
            s_in_max[size_t(pos)] = pos > 0 ? max_prev[size_t(pos - 1)] : nullptr;
            bool km = false;
            int64_t items = 0;
            void *rec = base + rb * size_t(pos);
            const mm::TcMatrix &Mq = ((fold >> (mu - 1)) & 1u) ? p->Dtc[mu - 1] : p->Etc[mu - 1];
            if (mm::tc_pair_record_build(p->st, p->st, mu, Mq, p->prec, p->work[pos % 3],
                                         p->work[(pos + 1) % 3], sc, rec, &km, &items, pos) != cudaSuccess) {
                cudaFree(done);
                return false;
            }
            mm::tc_pair_record_set_begin(rec, begin);
            begin += items;
        }
    if (!mm::tc_pair_batch_compatible(base, nprod) ||
        mm::tc_pair_chain_plan(base, nprod, d, s_in_max.data()) != cudaSuccess) {
        cudaFree(done);
        return false;
    }
    void *dev = nullptr;
    if (cudaMalloc(&dev, rb * size_t(nprod)) != cudaSuccess ||
        cudaMemcpy(dev, base, rb * size_t(nprod), cudaMemcpyHostToDevice) != cudaSuccess) {
        if (dev) cudaFree(dev);
        cudaFree(done);
        return false;
    }
    drop_graphs(p);
    if (p->chain_dev) cudaFree(p->chain_dev);
    if (p->chain_done) cudaFree(p->chain_done);
    p->chain_host.assign(base, base + rb * size_t(nprod));
    p->chain_dev = dev;
    p->chain_done = done;
    p->chain_nprod = nprod;
    p->chain_steps = nsteps;
    p->chain_fold = fold;
    std::copy(p->order, p->order + d, p->chain_order);
    return true;
}

// The products of a chained call (chain_prepare for nsteps has succeeded), between tc_begin and tc_end.
mm_status chain_run(mm_plan *p, int &cur, cudaStream_t s)
{
    const size_t counters = size_t(p->chain_nprod) * (mm::kChainCounters + 1);
    cudaError_t e = cudaMemsetAsync(p->chain_done, 0, sizeof(unsigned) * counters, s);
    if (e != cudaSuccess) return cuda_fail(e, "chain counters");
    cudaEvent_t ev0 = timing_event(p->ctx, true);
    if (ev0) cudaEventRecord(ev0, s);
    e = mm::tc_pair_chain_launch(p->chain_host.data(), p->chain_dev, p->chain_nprod, p->chain_done,
                                 p->chain_done + p->chain_nprod, p->ctx->d_err, s);
    if (ev0) cudaEventRecord(timing_event(p->ctx, false, p->chain_nprod), s);
    if (e != cudaSuccess) return cuda_fail(e, "chained tensor-core launch");
    p->sweep += p->chain_steps;
    cur = int(p->chain_nprod % 3);  // product k wrote buffer k + 1 mod 3, starting from buffer 0
    return MM_OK;
}

// Split the user's complex64 tensor into the plan's piece buffer 0.  The
// fixed-point mode also sets the state scale and, for the first sweep, the
// bounds max|u| * prod_{r<=q} ||E_{o_r}||_inf on each position's output.
mm_status tc_begin_bounds(mm_plan *p, const double *bounds, const void *u, cudaStream_t s);

mm_status tc_begin(mm_plan *p, mm::TcMatrix *const *M, const void *u, cudaStream_t s)
{
    double bounds[mm::kMaxDims];
    double acc = 1.0;
    for (int q = 0; q < p->d; ++q) {
        acc *= M[p->order[q] - 1]->row_norm;
        bounds[q] = acc;
    }
    return tc_begin_bounds(p, bounds, u, s);
}

// tc_begin with the first sweep's bounds given: bounds[q] >= max|output of position q| / max|u|.
mm_status tc_begin_bounds(mm_plan *p, const double *bounds, const void *u, cudaStream_t s)
{
    p->sweep = 0;
    if (p->d_max) {  // the maximum words of sweep 0 (later sweeps' words are cleared by the launches)
        cudaError_t e0 = cudaMemsetAsync(p->d_max, 0, sizeof(unsigned) * p->d, s);
        if (e0 != cudaSuccess) return cuda_fail(e0, "scale word reset");
    }
    // sweep 0 reads its maximum words from set 2: the split writes the bounds there
    cudaError_t e = p->tf32 ? mm::tc_split_tf32(p->st, u, p->work[0], s)
                            : mm::tc_split(p->st, p->npieces, p->fixed, u, p->work[0], p->d_work, p->d_scale,
                                           p->d_max ? p->d_max + 2 * p->d : nullptr, bounds, p->d, s);
    if (e != cudaSuccess) return cuda_fail(e, "split");
    return MM_OK;
}

mm_status tc_end(mm_plan *p, int cur, void *u, cudaStream_t s)
{
    // the state's scale after p->sweep sweeps (see tc_sweep)
    float *scale = p->d_scale ? p->d_scale + (p->sweep & 1) * p->d : nullptr;
    cudaError_t e = p->tf32 ? mm::tc_merge_tf32(p->st, p->work[cur], u, s)
                            : mm::tc_merge(p->st, p->npieces, p->fixed, p->work[cur], scale, u, s);
    if (e != cudaSuccess) return cuda_fail(e, "merge");
    return MM_OK;
}

// One Tucker sweep on the SIMT state: u holds the state on entry and exit.
mm_status simt_sweep(mm_plan *p, void *const *Ed, void *u, cudaStream_t s)
{
    const bool fp64 = p->dtype == MM_R64 || p->dtype == MM_C128;
    const bool cplx = is_complex(p->dtype);
    void *src = u, *dst = p->work[0];
    for (int q = 0; q < p->d; ++q) {
        const int mu = p->order[q];
        int64_t left, right;
        left_right(p->d, p->n, mu, &left, &right);
        cudaEvent_t ev0 = timing_event(p->ctx, true);
        if (ev0) cudaEventRecord(ev0, s);
        cudaError_t e = p->prec == MM_PREC_FP64_DMMA
                            ? mm::dmma_mode_product(cplx, left, p->n[mu - 1], right, p->n[mu - 1], Ed[mu - 1], src, dst, s)
                            : mm::simt_mode_product(fp64, cplx, left, p->n[mu - 1], right, p->n[mu - 1], Ed[mu - 1], src,
                                                    dst, s);
        if (ev0) cudaEventRecord(timing_event(p->ctx, false), s);
        if (e != cudaSuccess) return cuda_fail(e, "SIMT mode product launch");
        std::swap(src, dst);
    }
    if (src != u) {
        cudaError_t e = cudaMemcpyAsync(u, src, size_t(p->count) * elem_bytes(p->dtype), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "state copy");
    }
    return MM_OK;
}

mm_status alloc_workspace(mm_plan *p)
{
    cudaError_t e;
    if (p->tc) {
        p->st = make_state(p->d, p->n);
        p->work_bytes = size_t(p->st.plane) * 2 * p->npieces * size_t(mm::tc_piece_bytes(p->prec));
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&p->work[b], p->work_bytes);
            if (e != cudaSuccess) return fail(MM_ERR_OOM, "workspace cudaMalloc(%zu) failed", p->work_bytes);
            e = cudaMemset(p->work[b], 0, p->work_bytes);
            if (e != cudaSuccess) return cuda_fail(e, "workspace memset");
        }
        if (p->fixed) {
            e = cudaMalloc(&p->d_scale, sizeof(float) * 2 * p->d);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_max, sizeof(unsigned) * 3 * p->d);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_work, sizeof(unsigned));
            if (e == cudaSuccess) e = cudaMemset(p->d_max, 0, sizeof(unsigned) * 3 * p->d);
            if (e != cudaSuccess) return fail(MM_ERR_OOM, "scale words");
        }
    } else {
        p->work_bytes = size_t(p->count) * elem_bytes(p->dtype);
        e = cudaMalloc(&p->work[0], p->work_bytes);
        if (e != cudaSuccess) return fail(MM_ERR_OOM, "workspace cudaMalloc(%zu) failed", p->work_bytes);
    }
    return MM_OK;
}

mm_status upload_matrix(mm_plan *p, const double *E, int64_t m, int64_t n, bool Ec, void **simt, mm::TcMatrix *tcm)
{
    if (p->tc) {
        std::vector<double> c = as_complex(E, m * n, Ec);
        return mm::tc_matrix_create(c.data(), m, n, p->npieces, p->fixed, tcm, p->tf32);
    }
    return upload_simt(E, m, n, Ec, p->dtype, simt);
}

mm_status plan_common(mm_ctx *ctx, int d, const int64_t *n, mm_dtype dtype, mm_prec prec, const int *order,
                      bool matrix_complex, mm_plan **out, mm_plan **made)
{
    if (!ctx) return fail(MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(MM_ERR_INVALID_ARG, "out is NULL");
    mm_status st = check_dims(d, n);
    if (st) return st;
    bool fits = true;
    for (int v = 0; v < d; ++v) fits = fits && n[v] <= 512;
    prec = resolve_prec(prec, dtype, fits);
    st = check_combo(dtype, prec, matrix_complex);
    if (st) return st;
    const bool tc = mm::tc_prec(prec);
    if (tc) {
        if (!(ctx->sm_major == 10 && ctx->sm_minor == 3))
            return fail(MM_ERR_UNSUPPORTED, "tensor-core precisions need an sm_103 device (have sm_%d%d)", ctx->sm_major,
                        ctx->sm_minor);
        for (int v = 0; v < d; ++v)
            if (n[v] > 512) return fail(MM_ERR_SHAPE, "tensor-core path supports n_mu <= 512 (n[%d] = %lld)", v, (long long)n[v]);
    }
    bool seen[mm::kMaxDims] = {};
    auto *p = new mm_plan;
    p->ctx = ctx;
    p->d = d;
    p->count = 1;
    for (int v = 0; v < d; ++v) {
        p->n[v] = n[v];
        p->count *= n[v];
        p->order[v] = order ? order[v] : v + 1;
        if (p->order[v] < 1 || p->order[v] > d || seen[p->order[v] - 1]) {
            delete p;
            return fail(MM_ERR_INVALID_ARG, "mode_order is not a permutation of 1..%d", d);
        }
        seen[p->order[v] - 1] = true;
    }
    p->dtype = dtype;
    p->prec = prec;
    p->tc = tc;
    p->fixed = mm::tc_fixed(prec);
    p->tf32 = mm::tc_tf32(prec);
    p->npieces = mm::tc_pieces(prec);
    p->variant = p->tf32 ? mm::kTcOneSM : mm::tc_default_variant();
    {
        const char *fa = std::getenv("MM_FOLD_ALWAYS");
        p->fold_force = fa && fa[0] && !(fa[0] == '0' && fa[1] == 0);
    }
    *made = p;
    return MM_OK;
}

// Psi D(s) Phi_W for one direction: D = diag(exp(-i s (k + 1/2))).
std::vector<double> harmonic_propagator(const mm_plan *p, int v, double s)
{
    const int64_t m = p->n[v];
    std::vector<cd> tmp(size_t(m * m));
    for (int64_t k = 0; k < m; ++k) {
        const cd ph = std::exp(cd(0, -s * (double(k) + 0.5)));
        for (int64_t l = 0; l < m; ++l) tmp[size_t(k * m + l)] = ph * p->fwd[v][size_t(k * m + l)];
    }
    std::vector<double> P(size_t(2 * m * m), 0.0);
    std::vector<cd> row(static_cast<size_t>(m));
    for (int64_t a = 0; a < m; ++a) {  // row a of bwd tmp, accumulated along rows of tmp (contiguous)
        std::fill(row.begin(), row.end(), cd(0));
        for (int64_t k = 0; k < m; ++k) {
            const double c = p->bwd[v][size_t(a * m + k)];
            const cd *t = &tmp[size_t(k * m)];
            for (int64_t b = 0; b < m; ++b) row[size_t(b)] += c * t[b];
        }
        for (int64_t b = 0; b < m; ++b) {
            P[size_t(2 * (a * m + b))] = row[size_t(b)].real();
            P[size_t(2 * (a * m + b) + 1)] = row[size_t(b)].imag();
        }
    }
    return P;
}

// The folded form of a centrosymmetric n x n matrix E (interleaved complex, row-major): with F
// the even/odd fold (fold_state) D = F E F^-1 is block-diagonal, an even block of ceil(n/2) rows
// and an odd block of floor(n/2).  Returns false (D untouched) when E is not centrosymmetric to
// 1e-13 of its largest entry; the off-diagonal blocks of D, rounding-sized then, are set to zero.
bool fold_matrix(const double *E, int64_t n, std::vector<double> &D)
{
    using cd = std::complex<double>;
    const cd *e = reinterpret_cast<const cd *>(E);
    double amax = 0.0, asym = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            amax = std::max(amax, std::abs(e[i * n + j]));
            asym = std::max(asym, std::abs(e[i * n + j] - e[(n - 1 - i) * n + (n - 1 - j)]));
        }
    if (n < 2 || !(asym <= 1e-13 * amax)) return false;
    const int64_t c = (n + 1) / 2, h = n / 2;
    std::vector<cd> G(size_t(n * n)), R(size_t(n * n));
    for (int64_t j = 0; j < n; ++j) {  // G = F E (rows)
        for (int64_t k = 0; k < h; ++k) {
            G[size_t(k * n + j)] = e[k * n + j] + e[(n - 1 - k) * n + j];
            G[size_t((c + k) * n + j)] = e[k * n + j] - e[(n - 1 - k) * n + j];
        }
        if (n % 2) G[size_t(h * n + j)] = e[h * n + j];
    }
    for (int64_t i = 0; i < n; ++i) {  // R = G F^-1 (columns)
        for (int64_t k = 0; k < h; ++k) {
            R[size_t(i * n + k)] = 0.5 * (G[size_t(i * n + k)] + G[size_t(i * n + n - 1 - k)]);
            R[size_t(i * n + c + k)] = 0.5 * (G[size_t(i * n + k)] - G[size_t(i * n + n - 1 - k)]);
        }
        if (n % 2) R[size_t(i * n + h)] = G[size_t(i * n + h)];
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            if ((i < c) != (j < c)) R[size_t(i * n + j)] = 0.0;
    D.assign(reinterpret_cast<const double *>(R.data()), reinterpret_cast<const double *>(R.data()) + 2 * n * n);
    return true;
}

// Even/odd folding applies to tensor-core plans on complex64 data unless MM_NO_FOLD is set to
// other than 0.
bool fold_enabled(const mm_plan *p)
{
    const char *off = std::getenv("MM_NO_FOLD");
    return p->tc && p->dtype == MM_C64 && !(off && off[0] && !(off[0] == '0' && off[1] == 0));
}

void free_prop(mm_plan *p, int slot)
{
    for (int v = 0; v < p->d; ++v) {
        if (p->Pdev[slot][v]) cudaFree(p->Pdev[slot][v]);
        p->Pdev[slot][v] = nullptr;
        mm::tc_matrix_destroy(&p->Ptc[slot][v]);
        mm::tc_matrix_destroy(&p->PFtc[slot][v]);
    }
    p->pfold_mask[slot] = 0u;
    p->prop_s[slot] = NAN;
}

void drop_graphs(mm_plan *p);

// Make sure the propagators for step s are in a cache slot; returns the slot.
mm_status ensure_prop(mm_plan *p, double s, int avoid, int *slot)
{
    for (int k = 0; k < 2; ++k)
        if (p->prop_s[k] == s) {
            *slot = k;
            return MM_OK;
        }
    int k = (avoid == 0) ? 1 : 0;
    drop_graphs(p);  // captured graphs may point at the matrices being replaced
    free_prop(p, k);
    for (int v = 0; v < p->d; ++v) {
        std::vector<double> P = harmonic_propagator(p, v, s);
        mm_status st = upload_matrix(p, P.data(), p->n[v], p->n[v], true, &p->Pdev[k][v], &p->Ptc[k][v]);
        if (st) return st;
        std::vector<double> D;
        if (fold_enabled(p) && __builtin_popcount(p->pfold_mask[k]) < 5 && fold_matrix(P.data(), p->n[v], D)) {
            if ((st = mm::tc_matrix_create(D.data(), p->n[v], p->n[v], p->npieces, p->fixed, &p->PFtc[k][v], p->tf32)))
                return st;
            p->pfold_mask[k] |= 1u << v;
        }
    }
    if (p->pfold_mask[k] && !p->fold_buf && cudaMalloc(&p->fold_buf, size_t(p->count) * 8) != cudaSuccess) {
        p->fold_buf = nullptr;
        return fail(MM_ERR_OOM, "folded state buffer of %lld bytes", (long long)(p->count * 8));
    }
    p->prop_s[k] = s;
    *slot = k;
    return MM_OK;
}

void drop_graphs(mm_plan *p)
{
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second.first);
    p->graphs.clear();
}

// Run `body` (a sequence of launches on stream s) through a cached CUDA
// graph: the first call with a given key captures it, later calls replay
// it.  Plain launches when graphs are off, on the legacy default stream, or
// while kernel timing is on.
template <class F>
mm_status run_graphed(mm_plan *p, int kind, const void *ptr, int64_t nsteps, cudaStream_t s, double a, double b,
                      F &&body)
{
    if (!p->use_graphs || s == nullptr || p->ctx->timing) return body();
    const auto key = std::make_tuple(kind, ptr, nsteps, s, a, b);
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        if (p->graphs.size() >= 16) drop_graphs(p);
        const long long before = mm_launch_count();
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "begin stream capture");
        mm_status st = body();
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        const long long launches = mm_launch_count() - before;
        mm::count_launch(int(-launches));  // captured, not run: counted at each replay
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "end stream capture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        it = p->graphs.emplace(key, std::make_pair(ex, launches)).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.first, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    mm::count_launch(int(it->second.second));
    return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_plan_issued_flops(const mm_plan *p, double *flops_per_step)
{
    if (!p || !flops_per_step) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    if (!p->tc || p->hermite) return fail(MM_ERR_INVALID_ARG, "needs a tensor-core Tucker plan");
    double f = 0.0;
    for (int q = 0; q < p->d; ++q) {
        const int mu = p->order[q];
        f += mm::tc_issued_flops(p->st, mu, *step_matrix(p, mu - 1), p->prec, p->variant);
    }
    *flops_per_step = f;
    return MM_OK;
}

mm_status mm_plan_get_config(const mm_plan *p, int *variant, int *order_out)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    if (variant) *variant = int(p->variant);
    if (order_out)
        for (int v = 0; v < p->d; ++v) order_out[v] = p->order[v];
    return MM_OK;
}

mm_status mm_plan_set_config(mm_plan *p, int variant, const int *order)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    if (variant < 0 || variant >= mm::kTcVariants)
        return fail(MM_ERR_INVALID_ARG, "variant %d outside 0..%d", variant, mm::kTcVariants - 1);
    if (order) {
        if (p->hermite) return fail(MM_ERR_UNSUPPORTED, "the mode order of a Hermite plan is fixed");
        bool seen[mm::kMaxDims] = {};
        for (int v = 0; v < p->d; ++v) {
            if (order[v] < 1 || order[v] > p->d || seen[order[v] - 1])
                return fail(MM_ERR_INVALID_ARG, "order is not a permutation of 1..%d", p->d);
            seen[order[v] - 1] = true;
        }
    }
    drop_graphs(p);
    p->variant = mm::TcVariant(variant);
    if (order)
        for (int v = 0; v < p->d; ++v) p->order[v] = order[v];
    return MM_OK;
}

extern "C++" {

// The autotuner's cache key: what the timed work depends on.  The step kind, the GPU, the plan
// kind, sizes, element type and precision, and for tensor-core Tucker plans the k-block bands of
// each direction's matrix in both pair tilings (a banded propagator and a dense matrix of the
// same size favour different variants).
std::string autotune_key(const mm_plan *p, const char *kind)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->ctx->device) != cudaSuccess) prop.name[0] = 0;
    std::string k = std::string(kind) + "|" + prop.name + "|" + (p->hermite ? "hermite" : "tucker") + "|d";
    char buf[64];
    for (int v = 0; v < p->d; ++v) {
        std::snprintf(buf, sizeof buf, "%s%lld", v ? "x" : "=", (long long)p->n[v]);
        k += buf;
    }
    std::snprintf(buf, sizeof buf, "|dtype=%d|prec=%d", int(p->dtype), int(p->prec));
    k += buf;
    if (p->tc && !p->hermite) {
        uint64_t h = 1469598103934665603ull;  // FNV-1a over the band limits
        auto mix = [&](int x) {
            for (int b = 0; b < 4; ++b) {
                h ^= uint64_t((x >> (8 * b)) & 0xff);
                h *= 1099511628211ull;
            }
        };
        for (int v = 0; v < p->d; ++v)
            for (int t = 0; t < 2; ++t) {
                const auto &P = step_matrix(p, v)->pair[t];
                mix(P.ni);
                for (int r = 0; r < P.ni && r < 8; ++r) {
                    mix(P.kb_lo[r]);
                    mix(P.kb_hi[r]);
                }
            }
        std::snprintf(buf, sizeof buf, "|fold=%x|bands=%016llx", p->fold_mask, (unsigned long long)h);
        k += buf;
    }
    for (char &c : k)
        if (c == '"' || c == '\\' || c == '\n') c = '_';
    return k;
}

// A cached configuration for the key: sets the plan's variant and mode order and returns true.
bool autotune_cache_lookup(const char *path, const std::string &key, mm_plan *p)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string pat = "\"key\": \"" + key + "\"";
    char line[2048];
    bool found = false;
    int variant = -1, order[mm::kMaxDims] = {};
    while (std::fgets(line, sizeof line, f)) {
        const char *at = std::strstr(line, pat.c_str());
        if (!at) continue;
        const char *v = std::strstr(at, "\"variant\": ");
        const char *o = std::strstr(at, "\"order\": [");
        if (!v || !o || std::sscanf(v + 11, "%d", &variant) != 1) continue;
        o += 10;
        bool ok = true;
        for (int q = 0; q < p->d && ok; ++q) {
            char *end = nullptr;
            const long x = std::strtol(o, &end, 10);
            ok = end != o && x >= 1 && x <= p->d;
            order[q] = int(x);
            o = end;
            while (*o == ',' || *o == ' ') ++o;
        }
        if (ok && variant >= 0 && variant < mm::kTcVariants) found = true;  // the last matching line wins
    }
    std::fclose(f);
    if (!found) return false;
    bool perm = true;
    for (int q = 0; q < p->d; ++q)
        for (int r = q + 1; r < p->d; ++r) perm = perm && order[q] != order[r];
    if (!perm) return false;
    drop_graphs(p);
    p->variant = mm::TcVariant(variant);
    if (!p->hermite)
        for (int q = 0; q < p->d; ++q) p->order[q] = order[q];
    return true;
}

// Appends the plan's configuration under the key (one line, written in one call).
void autotune_cache_store(const char *path, const std::string &key, const mm_plan *p)
{
    std::string line = "{\"key\": \"" + key + "\", \"variant\": " + std::to_string(int(p->variant)) + ", \"order\": [";
    for (int q = 0; q < p->d; ++q) line += (q ? ", " : "") + std::to_string(p->order[q]);
    line += "]}\n";
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fwrite(line.data(), 1, line.size(), f);
    std::fclose(f);
}

// The tuner's loop; step(scratch, k) runs k steps of the kind being tuned on the scratch copy.
template <typename Step>
mm_status autotune_with(mm_plan *p, const void *u_dev, int64_t nsteps, void *stream, bool orders_too,
                               const char *kind, Step step)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    mm_status st = check_ptr(u_dev, "u_dev");
    if (st) return st;
    if (nsteps < 1 || nsteps > 1000) return fail(MM_ERR_INVALID_ARG, "nsteps = %lld outside 1..1000", (long long)nsteps);
    // MM_AUTOTUNE_CACHE: a file of earlier results (one JSON object per line); a plan whose key is
    // there takes that configuration without timing anything, and a new result is appended
    const char *cache = std::getenv("MM_AUTOTUNE_CACHE");
    std::string key;
    if (cache && cache[0]) {
        key = autotune_key(p, kind);
        if (autotune_cache_lookup(cache, key, p)) return MM_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = size_t(p->count) * elem_bytes(p->dtype);
    void *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) return fail(MM_ERR_OOM, "autotune scratch of %zu bytes", bytes);
    // candidates: kernel variants (tensor-core plans) x mode orders (Tucker plans, all orders for d <= 4)
    std::vector<int> variants;
    if (p->tc && p->tf32) variants = {mm::kTcOneSM};  // TF32 pieces run on the one-SM kernel only
    else if (p->tc) variants = {mm::kTcPair64, mm::kTcPair128, mm::kTcOneSM};
    else variants = {int(p->variant)};
    // kTcChain is opt-in (mm_plan_set_config): slower than one launch per product at every size
    // measured, and a profiler's fixed cost per launch would make it look faster
    std::vector<std::vector<int>> orders;
    std::vector<int> ord(p->order, p->order + p->d);
    if (orders_too && !p->hermite && p->d <= 4) {
        std::vector<int> o(size_t(p->d));
        for (int v = 0; v < p->d; ++v) o[size_t(v)] = v + 1;
        do orders.push_back(o);
        while (std::next_permutation(o.begin(), o.end()));
    } else {
        orders.push_back(ord);
    }
    const bool graphs = p->use_graphs;
    p->use_graphs = false;
    drop_graphs(p);
    const mm::TcVariant v0 = p->variant;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    int best_v = int(v0);
    std::vector<int> best_o = ord;
    auto run = [&](int64_t k) -> mm_status { return step(scratch, k); };
    // Two passes over the candidates, each keeping its faster time: the first pass also brings an
    // idle GPU up to its clocks, which would otherwise penalise the candidates timed first.
    std::vector<float> tbest(variants.size() * orders.size(), INFINITY);
    for (int pass = 0; pass < 2 && !st; ++pass)
        for (size_t iv = 0; iv < variants.size() && !st; ++iv)
            for (size_t io = 0; io < orders.size(); ++io) {
                const int v = variants[iv];
                const auto &o = orders[io];
                p->variant = mm::TcVariant(v);
                for (int q = 0; q < p->d; ++q) p->order[q] = o[size_t(q)];
                cudaError_t e = cudaMemcpyAsync(scratch, u_dev, bytes, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess && !(st = run(1))) {
                    cudaEventRecord(e0, s);
                    st = run(nsteps);
                    cudaEventRecord(e1, s);
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess && !st) st = cuda_fail(e, "autotune");
                if (st) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                float &tb = tbest[iv * orders.size() + io];
                tb = std::min(tb, ms);
                if (pass == 1 && tb < best) {
                    best = tb;
                    best_v = v;
                    best_o = o;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    p->variant = st ? v0 : mm::TcVariant(best_v);
    const std::vector<int> &keep = st ? ord : best_o;
    for (int q = 0; q < p->d; ++q) p->order[q] = keep[size_t(q)];
    p->use_graphs = graphs;
    if (!st && !key.empty()) autotune_cache_store(cache, key, p);
    return st;
}

}  // extern "C++"

mm_status mm_plan_autotune(mm_plan *p, const void *u_dev, int64_t nsteps, void *stream)
{
    NvtxRange range("mm_plan_autotune");
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    return autotune_with(p, u_dev, nsteps, stream, true, "steps", [&](void *u, int64_t k) {
        return p->hermite ? hermite_ho_step(p, u, 0.01, k, stream) : mumode_step(p, u, k, stream);
    });
}

mm_status split_step_gpe_autotune(mm_plan *p, const void *psi_dev, double beta, double tau, int64_t nsteps,
                                  void *stream)
{
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    if (!std::isfinite(beta) || !std::isfinite(tau)) return fail(MM_ERR_INVALID_ARG, "beta or tau is not finite");
    return autotune_with(p, psi_dev, nsteps, stream, false, "gpe",
                         [&](void *u, int64_t k) { return split_step_gpe(p, u, beta, tau, k, stream); });
}

mm_status mm_plan_set_graphs(mm_plan *p, int enable)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    p->use_graphs = enable != 0;
    if (!p->use_graphs) drop_graphs(p);
    return MM_OK;
}

mm_status mm_plan_get_fold(const mm_plan *p, int *mask_out)
{
    if (!p || !mask_out) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    unsigned m = p->fold_mask;
    if (p->hermite) m = p->fold_on ? (p->pfold_mask[0] | p->pfold_mask[1]) : 0u;
    *mask_out = int(m);
    return MM_OK;
}

mm_status mm_plan_set_fold(mm_plan *p, int enable)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    drop_graphs(p);
    p->fold_on = enable != 0;
    p->fold_mask = p->fold_on ? p->fold_avail : 0u;
    p->chain_steps = -1;  // the chained records hold the matrices of the previous setting
    return MM_OK;
}

const char *mm_last_error(void) { return mm::g_err; }

int64_t mm_launch_count(void) { return mm::g_launches.load(); }

mm_status mm_ctx_create(int device, mm_ctx **out)
{
    if (!out) return fail(MM_ERR_INVALID_ARG, "out is NULL");
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(MM_ERR_INVALID_ARG, "device %d not present (%d devices)", device, count);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto *c = new mm_ctx;
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&c->sm_minor, cudaDevAttrComputeCapabilityMinor, device);
    e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, sizeof(double));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "context allocation");
    }
    *out = c;
    return MM_OK;
}

mm_status mm_kernel_timing(mm_ctx *ctx, int enable)
{
    if (!ctx) return fail(MM_ERR_INVALID_ARG, "ctx is NULL");
    ctx->timing = enable != 0;
    ctx->events_used = 0;
    return MM_OK;
}

mm_status mm_kernel_timing_read(mm_ctx *ctx, double *total_ms, int64_t *launches)
{
    if (!ctx || !total_ms || !launches) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    double tot = 0.0;
    int64_t products = 0;
    for (size_t k = 0; k < ctx->events_used; ++k) {
        cudaError_t e = cudaEventSynchronize(ctx->events[k].second);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->events[k].first, ctx->events[k].second);
        if (e != cudaSuccess) return cuda_fail(e, "event timing");
        tot += ms;
        products += ctx->event_products[k];
    }
    *total_ms = tot;
    *launches = products;
    ctx->events_used = 0;
    return MM_OK;
}

void mm_ctx_destroy(mm_ctx *ctx)
{
    if (!ctx) return;
    for (auto &pr : ctx->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_scratch);
    mm::expm_workspace_destroy(&ctx->expm);
    mm::expm_batch_destroy(&ctx->expmb);
    delete ctx;
}

mm_status mm_device_status(mm_ctx *ctx, void *stream)
{
    if (!ctx) return fail(MM_ERR_INVALID_ARG, "ctx is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int word = 0;
    e = cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "error word read");
    if (word != 0) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (word == MM_ERR_TIMEOUT) return fail(MM_ERR_TIMEOUT, "a device-side bounded wait gave up");
        if (word == MM_ERR_RANGE)
            return fail(MM_ERR_RANGE, "the fixed-point state left its range (grew more than 16x within a sweep)");
        return fail(mm_status(word), "device error word %d", word);
    }
    return MM_OK;
}

mm_status mm_fd_laplacian_dirichlet(int n, double *A_out)
{
    if (n < 1) return fail(MM_ERR_SHAPE, "n = %d < 1", n);
    if (!A_out) return fail(MM_ERR_INVALID_ARG, "A_out is NULL");
    mm::fd_laplacian_dirichlet(n, A_out);
    return MM_OK;
}

mm_status mm_expm(int n, const double *A_re, const double *A_im, double z_re, double z_im, double *E_out)
{
    if (n < 1) return fail(MM_ERR_SHAPE, "n = %d < 1", n);
    if (!A_re || !E_out) return fail(MM_ERR_INVALID_ARG, "A_re or E_out is NULL");
    if (!mm::expm(n, A_re, A_im, cd(z_re, z_im), reinterpret_cast<cd *>(E_out)))
        return fail(MM_ERR_INVALID_ARG, "expm: singular Pade denominator");
    return MM_OK;
}

mm_status mm_gauss_hermite(int m, double *x_out, double *W_out)
{
    if (m < 1 || m > 4096) return fail(MM_ERR_SHAPE, "m = %d outside 1..4096", m);
    if (!x_out || !W_out) return fail(MM_ERR_INVALID_ARG, "x_out or W_out is NULL");
    mm::gauss_hermite(m, x_out, W_out);
    return MM_OK;
}

mm_status mm_hermite_matrices(int m, double *fwd, double *bwd)
{
    if (m < 1 || m > 4096) return fail(MM_ERR_SHAPE, "m = %d outside 1..4096", m);
    std::vector<double> x(m), W(m);
    mm::gauss_hermite(m, x.data(), W.data());
    mm::hermite_matrices(m, x.data(), W.data(), fwd, bwd);
    return MM_OK;
}

mm_status mm_hermite_hamiltonian(int m, const double *V_nodes, double *H_out)
{
    if (m < 1 || m > 4096) return fail(MM_ERR_SHAPE, "m = %d outside 1..4096", m);
    if (!H_out) return fail(MM_ERR_INVALID_ARG, "H_out is NULL");
    std::vector<double> x(m), W(m);
    mm::gauss_hermite(m, x.data(), W.data());
    mm::hermite_hamiltonian(m, x.data(), W.data(), V_nodes, H_out);
    return MM_OK;
}

mm_status hkp_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *V_nodes, double tau,
                          mm_dtype dtype, mm_prec prec, const int *mode_order, mm_plan **out)
{
    if (!ctx || !n || !out) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    if (d < 1 || d > mm::kMaxDims) return fail(MM_ERR_SHAPE, "d = %d outside 1..%d", d, mm::kMaxDims);
    if (!std::isfinite(tau)) return fail(MM_ERR_INVALID_ARG, "tau is not finite");
    if (!is_complex(dtype)) return fail(MM_ERR_DTYPE, "HKP plans need complex data");
    // the propagators Psi exp(-i tau H) Phi^W are built on the device (FP64: the Galerkin matrix
    // and the two foldings as cuBLAS products, the exponential as in mm_expm_device), then split
    // into the plan's form on the host like any Tucker matrix
    int nmax = 0;
    for (int v = 0; v < d; ++v) {
        if (n[v] < 1 || n[v] > 4096) return fail(MM_ERR_SHAPE, "n[%d] = %lld outside 1..4096", v, (long long)n[v]);
        nmax = std::max(nmax, int(n[v]));
    }
    cudaError_t e = mm::expm_workspace_init(&ctx->expm, nmax);
    if (e == cudaSuccess) e = mm::expm_batch_init(&ctx->expmb, nmax, 1);
    if (e != cudaSuccess) return fail(MM_ERR_OOM, "expm workspace (%s)", cudaGetErrorString(e));
    double2 *Md = nullptr;
    if (cudaMalloc(&Md, sizeof(double2) * size_t(nmax) * nmax) != cudaSuccess) return fail(MM_ERR_OOM, "HKP matrix");
    std::vector<std::vector<cd>> M(static_cast<size_t>(d));
    std::vector<const double *> ptr(static_cast<size_t>(d), nullptr);
    mm_status st = MM_OK;
    for (int v = 0; v < d && !st; ++v) {
        const int m = int(n[v]);
        std::vector<double> x(m), W(m), fwd(size_t(m) * m), bwd(size_t(m) * m), GP;
        mm::gauss_hermite(m, x.data(), W.data());
        mm::hermite_matrices(m, x.data(), W.data(), fwd.data(), bwd.data());  // bwd[l][k] = phi_k(x_l)
        const double *V = V_nodes ? V_nodes[v] : nullptr;
        if (V) {
            GP.resize(size_t(m) * m);
            for (int l = 0; l < m; ++l) {
                const double g = W[size_t(l)] * (V[l] - 0.5 * x[size_t(l)] * x[size_t(l)]);
                for (int k = 0; k < m; ++k) GP[size_t(l) * m + k] = g * bwd[size_t(l) * m + k];
            }
        }
        e = mm::hkp_propagator_device(&ctx->expm, &ctx->expmb, m, bwd.data(), V ? GP.data() : nullptr, fwd.data(), tau,
                                      Md, nullptr);
        M[size_t(v)].resize(size_t(m) * m);
        if (e == cudaSuccess)
            e = cudaMemcpy(M[size_t(v)].data(), Md, sizeof(double2) * size_t(m) * m, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "HKP propagator");
        ptr[size_t(v)] = reinterpret_cast<const double *>(M[size_t(v)].data());
    }
    cudaFree(Md);
    if (st) return st;
    return mumode_plan_create(ctx, d, n, ptr.data(), 1, dtype, prec, mode_order, out);
}

mm_status mumode_product(mm_ctx *ctx, int d, const int64_t *n, int mu, const double *L, int64_t m, int L_is_complex,
                         mm_dtype dtype, mm_prec prec, const void *u_dev, void *s_dev, void *stream)
{
    NvtxRange range("mumode_product");
    if (!ctx) return fail(MM_ERR_INVALID_ARG, "ctx is NULL");
    mm_status st = check_dims(d, n);
    if (st) return st;
    if (mu < 1 || mu > d) return fail(MM_ERR_INVALID_ARG, "mu = %d outside 1..%d", mu, d);
    if (m < 1 || m > (int64_t(1) << 24)) return fail(MM_ERR_SHAPE, "m = %lld out of range", (long long)m);
    if (!L) return fail(MM_ERR_INVALID_ARG, "L is NULL");
    if ((st = check_ptr(u_dev, "u_dev")) || (st = check_ptr(s_dev, "s_dev"))) return st;
    prec = resolve_prec(prec, dtype, n[mu - 1] <= 512 && m <= 512);
    if ((st = check_combo(dtype, prec, L_is_complex != 0))) return st;
    int64_t nout[mm::kMaxDims];
    int64_t cnt_in = 1, cnt_out = 1;
    for (int v = 0; v < d; ++v) {
        nout[v] = (v == mu - 1) ? m : n[v];
        cnt_in *= n[v];
        cnt_out *= nout[v];
    }
    const size_t eb = elem_bytes(dtype);
    const char *u0 = (const char *)u_dev, *s0 = (const char *)s_dev;
    if (u0 < s0 + cnt_out * eb && s0 < u0 + cnt_in * eb) return fail(MM_ERR_INVALID_ARG, "u_dev and s_dev overlap");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nmu = n[mu - 1];
    if (!mm::tc_prec(prec)) {
        void *Ld = nullptr;
        if ((st = upload_simt(L, m, nmu, L_is_complex != 0, dtype, &Ld))) return st;
        int64_t left, right;
        left_right(d, n, mu, &left, &right);
        const bool fp64 = dtype == MM_R64 || dtype == MM_C128;
        cudaError_t e = prec == MM_PREC_FP64_DMMA
                            ? mm::dmma_mode_product(is_complex(dtype), left, nmu, right, m, Ld, u_dev, s_dev, s)
                            : mm::simt_mode_product(fp64, is_complex(dtype), left, nmu, right, m, Ld, u_dev, s_dev, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(Ld);
        if (e != cudaSuccess) return cuda_fail(e, "SIMT mode product");
        if (e2 != cudaSuccess) return cuda_fail(e2, "SIMT mode product (sync)");
        return MM_OK;
    }
    if (!(ctx->sm_major == 10 && ctx->sm_minor == 3))
        return fail(MM_ERR_UNSUPPORTED, "tensor-core precisions need an sm_103 device");
    if (nmu > 512 || m > 512) return fail(MM_ERR_SHAPE, "tensor-core path supports n_mu, m <= 512");
    const int NP = mm::tc_pieces(prec);
    const bool fixed = mm::tc_fixed(prec), tf32 = mm::tc_tf32(prec);
    std::vector<double> Lc = as_complex(L, m * nmu, L_is_complex != 0);
    mm::TcMatrix M;
    if ((st = mm::tc_matrix_create(Lc.data(), m, nmu, NP, fixed, &M, tf32))) return st;
    mm::TcState si = make_state(d, n), so = make_state(d, nout);
    void *bi = nullptr, *bo = nullptr, *words = nullptr;
    const size_t eb_p = size_t(mm::tc_piece_bytes(prec));
    size_t bytes_i = size_t(si.plane) * 2 * NP * eb_p, bytes_o = size_t(so.plane) * 2 * NP * eb_p;
    if (tf32 && mu > 1) bytes_i = bytes_o = std::max(bytes_i, bytes_o);  // both hold either state (the swaps)
    cudaError_t e = cudaMalloc(&bi, bytes_i);
    if (e == cudaSuccess) e = cudaMalloc(&bo, bytes_o);
    if (e == cudaSuccess) e = cudaMalloc(&words, 64);
    if (e != cudaSuccess) {
        cudaFree(bi);
        cudaFree(bo);
        mm::tc_matrix_destroy(&M);
        return fail(MM_ERR_OOM, "temporary piece buffers (%zu + %zu bytes)", bytes_i, bytes_o);
    }
    // words: [0] scale in, [1] scale out (floats), [2] bound, [3] max, [4] work (unsigned)
    float *scales = reinterpret_cast<float *>(words);
    unsigned *uw = reinterpret_cast<unsigned *>(words);
    mm::TcScales sc;
    if (fixed) {
        sc.s_in = scales;
        sc.s_out = scales + 1;
        sc.max_prev = uw + 2;
        sc.max_cur = uw + 3;
    }
    const double bound = M.row_norm;
    e = cudaMemsetAsync(words, 0, 64, s);
    if (e == cudaSuccess)
        e = tf32 ? mm::tc_split_tf32(si, u_dev, bi, s)
                 : mm::tc_split(si, NP, fixed, u_dev, bi, uw + 4, scales, uw + 2, &bound, 1, s);
    if (e == cudaSuccess)
        e = mm::tc_mode_product(si, so, mu, M, prec, bi, bo, mm::TcEpilogue{}, sc, ctx->d_err, s, mm::tc_default_variant());
    if (e == cudaSuccess) e = tf32 ? mm::tc_merge_tf32(so, bo, s_dev, s) : mm::tc_merge(so, NP, fixed, bo, scales + 1, s_dev, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(bi);
    cudaFree(bo);
    cudaFree(words);
    mm::tc_matrix_destroy(&M);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core mode product");
    if (e2 != cudaSuccess) return cuda_fail(e2, "tensor-core mode product (sync)");
    return MM_OK;
}

// Fold the directions of a tensor-core Tucker plan whose matrices are centrosymmetric (at most
// five; MM_NO_FOLD set to other than 0 turns it off), and allocate the folded state's buffer.
mm_status fold_matrices(mm_plan *p, const double *const *E_host, bool Ec)
{
    p->fold_mask = 0;
    if (!fold_enabled(p) || p->hermite) return MM_OK;
    int folded = 0;
    for (int v = 0; v < p->d && folded < 5; ++v) {
        const int64_t n = p->n[v];
        std::vector<double> c = as_complex(E_host[v], n * n, Ec), D;
        if (!fold_matrix(c.data(), n, D)) continue;
        mm_status st = mm::tc_matrix_create(D.data(), n, n, p->npieces, p->fixed, &p->Dtc[v], p->tf32);
        if (st) return st;
        p->fold_mask |= 1u << v;
        ++folded;
    }
    p->fold_avail = p->fold_mask;
    if (p->fold_mask && cudaMalloc(&p->fold_buf, size_t(p->count) * 8) != cudaSuccess) {
        p->fold_buf = nullptr;
        return fail(MM_ERR_OOM, "folded state buffer of %lld bytes", (long long)(p->count * 8));
    }
    return MM_OK;
}

mm_status mumode_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *E_host, int E_is_complex,
                             mm_dtype dtype, mm_prec prec, const int *mode_order, mm_plan **out)
{
    mm_plan *p = nullptr;
    mm_status st = plan_common(ctx, d, n, dtype, prec, mode_order, E_is_complex != 0, out, &p);
    if (st) return st;
    if (!E_host) {
        delete p;
        return fail(MM_ERR_INVALID_ARG, "E_host is NULL");
    }
    for (int v = 0; v < d; ++v) {
        if (!E_host[v]) {
            mm_plan_destroy(p);
            return fail(MM_ERR_INVALID_ARG, "E_host[%d] is NULL", v);
        }
        st = upload_matrix(p, E_host[v], n[v], n[v], E_is_complex != 0, &p->Edev[v], &p->Etc[v]);
        if (st) {
            mm_plan_destroy(p);
            return st;
        }
    }
    if ((st = alloc_workspace(p)) || (st = fold_matrices(p, E_host, E_is_complex != 0))) {
        mm_plan_destroy(p);
        return st;
    }
    *out = p;
    return MM_OK;
}

mm_status mumode_step(mm_plan *p, void *u_dev, int64_t nsteps, void *stream)
{
    NvtxRange range("mumode_step");
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    mm_status st = check_ptr(u_dev, "u_dev");
    if (st) return st;
    if (nsteps < 0) return fail(MM_ERR_INVALID_ARG, "nsteps < 0");
    if (nsteps == 0) return MM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->hermite) return fail(MM_ERR_INVALID_ARG, "mumode_step needs a Tucker plan (use hermite_ho_step)");
    if (!p->tc) {
        return run_graphed(p, 0, u_dev, nsteps, s, 0.0, 0.0, [&]() -> mm_status {
            mm_status r;
            for (int64_t k = 0; k < nsteps; ++k)
                if ((r = simt_sweep(p, p->Edev, u_dev, s))) return r;
            return MM_OK;
        });
    }
    // folded directions (when the call is long enough to pay for it): the steps run on the folded
    // state, folded and unfolded once per call
    mm::TcMatrix *M[mm::kMaxDims], *U[mm::kMaxDims], *D[mm::kMaxDims];
    for (int v = 0; v < p->d; ++v) {
        U[v] = &p->Etc[v];
        D[v] = &p->Dtc[v];
    }
    const unsigned fm = fold_pays(p, p->fold_mask, U, D, nsteps) ? p->fold_mask : 0u;
    for (int v = 0; v < p->d; ++v) M[v] = ((fm >> v) & 1u) ? D[v] : U[v];
    // kTcChain: every product of the call in one persistent launch (records prepared outside any capture)
    const bool chained = p->variant == mm::kTcChain && chain_prepare(p, nsteps, fm);
    return run_graphed(p, 0, u_dev, nsteps, s, 0.0, 0.0, [&]() -> mm_status {
        mm_status r;
        int cur = 0;
        const void *src = u_dev;
        if (fm) {
            cudaError_t e = mm::fold_state(p->d, p->n, fm, false, u_dev, p->fold_buf, s);
            if (e != cudaSuccess) return cuda_fail(e, "fold");
            src = p->fold_buf;
        }
        if ((r = tc_begin(p, M, src, s))) return r;
        if (chained) {
            if ((r = chain_run(p, cur, s))) return r;
        } else {
            for (int64_t k = 0; k < nsteps; ++k)
                if ((r = tc_sweep(p, M, cur, mm::TcEpilogue{}, s))) return r;
        }
        if (!fm) return tc_end(p, cur, u_dev, s);
        if ((r = tc_end(p, cur, p->fold_buf, s))) return r;
        cudaError_t e = mm::fold_state(p->d, p->n, fm, true, p->fold_buf, u_dev, s);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "unfold");
    });
}

mm_status mumode_step_host(mm_plan *p, void *u_host, int64_t nsteps, void *stream)
{
    NvtxRange range("mumode_step_host");
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    if (!u_host) return fail(MM_ERR_INVALID_ARG, "u_host is NULL");
    const size_t bytes = size_t(p->count) * elem_bytes(p->dtype);
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->staging) {
        cudaError_t e = cudaMalloc(&p->staging, bytes);
        if (e != cudaSuccess) return fail(MM_ERR_OOM, "staging cudaMalloc(%zu) failed", bytes);
    }
    cudaError_t e = cudaMemcpyAsync(p->staging, u_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    mm_status st = mumode_step(p, p->staging, nsteps, stream);
    if (st) return st;
    e = cudaMemcpyAsync(u_host, p->staging, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return MM_OK;
}

void adj_release(mm_plan *p);

void mm_plan_destroy(mm_plan *p)
{
    if (!p) return;
    drop_graphs(p);
    adj_release(p);
    for (int v = 0; v < mm::kMaxDims; ++v) {
        if (p->Edev[v]) cudaFree(p->Edev[v]);
        mm::tc_matrix_destroy(&p->Etc[v]);
        mm::tc_matrix_destroy(&p->Dtc[v]);
        if (p->Wdev[v]) cudaFree(p->Wdev[v]);
        if (p->Wpad[v]) cudaFree(p->Wpad[v]);
        if (p->Fdev[v]) cudaFree(p->Fdev[v]);
        if (p->Bdev[v]) cudaFree(p->Bdev[v]);
        mm::tc_matrix_destroy(&p->Ftc[v]);
        mm::tc_matrix_destroy(&p->Btc[v]);
    }
    free_prop(p, 0);
    free_prop(p, 1);
    if (p->work[0]) cudaFree(p->work[0]);
    if (p->work[1]) cudaFree(p->work[1]);
    if (p->work[2]) cudaFree(p->work[2]);
    if (p->staging) cudaFree(p->staging);
    if (p->fold_buf) cudaFree(p->fold_buf);
    if (p->d_scale) cudaFree(p->d_scale);
    if (p->d_max) cudaFree(p->d_max);
    if (p->d_work) cudaFree(p->d_work);
    if (p->d_norm) cudaFree(p->d_norm);
    if (p->chain_dev) cudaFree(p->chain_dev);
    if (p->chain_done) cudaFree(p->chain_done);
    for (int v = 0; v < mm::kMaxDims; ++v) {
        if (p->H0dev[v]) cudaFree(p->H0dev[v]);
        if (p->Gdev[v]) cudaFree(p->Gdev[v]);
        if (p->Ebatch[v]) cudaFree(p->Ebatch[v]);
        if (p->hk_nodesE[v]) cudaFree(p->hk_nodesE[v]);
        if (p->hk_rangeE[v]) cudaFree(p->hk_rangeE[v]);
    }
    if (p->coef) cudaFree(p->coef);
    if (p->hk_w) cudaFree(p->hk_w);
    for (int v = 0; v < mm::kMaxDims; ++v)
        if (p->hk_phase[v]) cudaFree(p->hk_phase[v]);
    mm::expm_batch_destroy(&p->expmb);
    delete p;
}

static mm_status hermite_setup(mm_plan *p);

mm_status hermite_plan_create(mm_ctx *ctx, int d, const int64_t *n, mm_dtype dtype, mm_prec prec, mm_plan **out)
{
    mm_plan *p = nullptr;
    mm_status st = plan_common(ctx, d, n, dtype, prec, nullptr, true, out, &p);
    if (st) return st;
    if (!is_complex(dtype)) {
        delete p;
        return fail(MM_ERR_DTYPE, "Hermite plans need complex data");
    }
    if (p->tf32) {
        delete p;
        return fail(MM_ERR_UNSUPPORTED, "MM_PREC_TF32X3 serves Tucker plans and mumode_product only");
    }
    if ((st = hermite_setup(p))) {
        mm_plan_destroy(p);
        return st;
    }
    *out = p;
    return MM_OK;
}

// Nodes, weights and transform matrices of every direction, and the workspace.
static mm_status hermite_setup(mm_plan *p)
{
    mm_status st;
    p->hermite = true;
    for (int v = 0; v < p->d; ++v) {
        const int m = int(p->n[v]);
        p->x[v].resize(m);
        p->W[v].resize(m);
        p->fwd[v].resize(size_t(m) * m);
        p->bwd[v].resize(size_t(m) * m);
        mm::gauss_hermite(m, p->x[v].data(), p->W[v].data());
        mm::hermite_matrices(m, p->x[v].data(), p->W[v].data(), p->fwd[v].data(), p->bwd[v].data());
        if (cudaMalloc(&p->Wdev[v], sizeof(double) * m) != cudaSuccess ||
            cudaMemcpy(p->Wdev[v], p->W[v].data(), sizeof(double) * m, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(MM_ERR_OOM, "weights upload");
        std::vector<double> wp(size_t((m + 15) / 16 * 16), 0.0);
        std::copy(p->W[v].begin(), p->W[v].end(), wp.begin());
        if (cudaMalloc(&p->Wpad[v], sizeof(double) * wp.size()) != cudaSuccess ||
            cudaMemcpy(p->Wpad[v], wp.data(), sizeof(double) * wp.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(MM_ERR_OOM, "weights upload");
        if ((st = upload_matrix(p, p->fwd[v].data(), m, m, false, &p->Fdev[v], &p->Ftc[v])) ||
            (st = upload_matrix(p, p->bwd[v].data(), m, m, false, &p->Bdev[v], &p->Btc[v])))
            return st;
    }
    return alloc_workspace(p);
}

mm_status hermite_nodes(const mm_plan *p, int mu, double *x_out, double *W_out)
{
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    if (mu < 1 || mu > p->d) return fail(MM_ERR_INVALID_ARG, "mu = %d outside 1..%d", mu, p->d);
    if (x_out) std::memcpy(x_out, p->x[mu - 1].data(), sizeof(double) * p->n[mu - 1]);
    if (W_out) std::memcpy(W_out, p->W[mu - 1].data(), sizeof(double) * p->n[mu - 1]);
    return MM_OK;
}

static mm_status hermite_apply(mm_plan *p, bool forward, const void *in, void *out, void *stream)
{
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    mm_status st;
    if ((st = check_ptr(in, "input")) || (st = check_ptr(out, "output"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->tc) {
        cudaError_t e = cudaMemcpyAsync(out, in, size_t(p->count) * elem_bytes(p->dtype), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy");
        return simt_sweep(p, forward ? p->Fdev : p->Bdev, out, s);
    }
    int cur = 0;
    mm::TcMatrix *M[mm::kMaxDims];
    for (int v = 0; v < p->d; ++v) M[v] = forward ? &p->Ftc[v] : &p->Btc[v];
    if ((st = tc_begin(p, M, in, s))) return st;
    if ((st = tc_sweep(p, M, cur, mm::TcEpilogue{}, s))) return st;
    return tc_end(p, cur, out, s);
}

mm_status hermite_forward(mm_plan *p, const void *values_dev, void *coeffs_dev, void *stream)
{
    NvtxRange range("hermite_forward");
    return hermite_apply(p, true, values_dev, coeffs_dev, stream);
}

mm_status hermite_backward(mm_plan *p, const void *coeffs_dev, void *values_dev, void *stream)
{
    NvtxRange range("hermite_backward");
    return hermite_apply(p, false, coeffs_dev, values_dev, stream);
}

mm_status hermite_ho_step(mm_plan *p, void *psi, double tau, int64_t nsteps, void *stream)
{
    NvtxRange range("hermite_ho_step");
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    mm_status st = check_ptr(psi, "psi_dev");
    if (st) return st;
    if (nsteps < 0 || !std::isfinite(tau)) return fail(MM_ERR_INVALID_ARG, "bad nsteps or tau");
    if (nsteps == 0) return MM_OK;
    int slot;
    if ((st = ensure_prop(p, tau, -1, &slot))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->tc) {
        for (int64_t k = 0; k < nsteps; ++k)
            if ((st = simt_sweep(p, p->Pdev[slot], psi, s))) return st;
        return MM_OK;
    }
    return run_graphed(p, 1, psi, nsteps, s, tau, 0.0, [&]() -> mm_status {
        mm_status r;
        int cur = 0;
        mm::TcMatrix *M[mm::kMaxDims], *U[mm::kMaxDims], *D[mm::kMaxDims];
        for (int v = 0; v < p->d; ++v) {
            U[v] = &p->Ptc[slot][v];
            D[v] = &p->PFtc[slot][v];
        }
        const unsigned fm = p->fold_on && fold_pays(p, p->pfold_mask[slot], U, D, nsteps) ? p->pfold_mask[slot] : 0u;
        for (int v = 0; v < p->d; ++v) M[v] = ((fm >> v) & 1u) ? D[v] : U[v];
        // folded directions: the steps run on the folded state, folded and unfolded once per call
        const void *src = psi;
        if (fm) {
            cudaError_t e = mm::fold_state(p->d, p->n, fm, false, psi, p->fold_buf, s);
            if (e != cudaSuccess) return cuda_fail(e, "fold");
            src = p->fold_buf;
        }
        if ((r = tc_begin(p, M, src, s))) return r;
        for (int64_t k = 0; k < nsteps; ++k)
            if ((r = tc_sweep(p, M, cur, mm::TcEpilogue{}, s))) return r;
        if (!fm) return tc_end(p, cur, psi, s);
        if ((r = tc_end(p, cur, p->fold_buf, s))) return r;
        cudaError_t e = mm::fold_state(p->d, p->n, fm, true, p->fold_buf, psi, s);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "unfold");
    });
}

}  // extern "C"

namespace {

// Strang steps of the GPE; with d_norm (tensor cores, F16X6 on the CTA-pair kernel, pair tilings of
// the half-step propagators), *d_norm is also set to the weighted norm sum |psi|^2 W of the result:
// by the last product's epilogue (kind 5), or by the final unfold when the steps run folded.
mm_status gpe_steps(mm_plan *p, void *psi, double beta, double tau, int64_t nsteps, double *d_norm, cudaStream_t s)
{
    mm_status st;
    int half, full;
    if ((st = ensure_prop(p, 0.5 * tau, -1, &half))) return st;
    if (nsteps > 1) {
        if ((st = ensure_prop(p, tau, half, &full))) return st;
    } else {
        full = half;
    }
    const double tb = tau * beta;
    if (!p->tc) {
        const bool fp64 = p->dtype == MM_C128;
        for (int64_t k = 0; k < nsteps; ++k) {
            if ((st = simt_sweep(p, p->Pdev[k == 0 ? half : full], psi, s))) return st;
            cudaError_t e = mm::simt_nonlinear_phase(fp64, p->count, tb, psi, s);
            if (e != cudaSuccess) return cuda_fail(e, "nonlinear phase");
        }
        return simt_sweep(p, p->Pdev[half], psi, s);
    }
    // Folded (F16X6, the half and full propagators folded alike, and long enough to pay for it): the
    // linear sweeps run on the folded state with plain epilogues, the nonlinear phase is a pass on
    // the folded pieces between sweeps (unfold, phase, fold per orbit), and the weighted norm, when
    // asked for, is summed by the final unfold
    const unsigned fm = p->pfold_mask[half];
    bool folded = p->fixed && p->fold_on && fm && p->pfold_mask[full] == fm;
    if (folded) {
        mm::TcMatrix *U[mm::kMaxDims], *D[mm::kMaxDims];
        for (int v = 0; v < p->d; ++v) {
            U[v] = &p->Ptc[full][v];
            D[v] = &p->PFtc[full][v];
        }
        // the tensor work of nsteps + 1 sweeps saved against the fold and unfold (32 bytes a point)
        // and the nsteps phase passes: each reads and writes 24 bytes a point but takes about as
        // long as 40 would at the HBM rate (it is bound by its instructions and load latency)
        const double cost_s = double(32 + 40 * nsteps) * double(p->count) / 6.5e12;
        folded = p->fold_force || double(nsteps + 1) * fold_saved_s(p, fm, U, D) > cost_s;
    }
    if (folded) {
        return run_graphed(p, d_norm ? 7 : 6, psi, nsteps, s, tau, beta, [&]() -> mm_status {
            mm_status r;
            int cur = 0;
            mm::TcMatrix *Mh[mm::kMaxDims], *Mf[mm::kMaxDims];
            for (int v = 0; v < p->d; ++v) {
                Mh[v] = ((fm >> v) & 1u) ? &p->PFtc[half][v] : &p->Ptc[half][v];
                Mf[v] = ((fm >> v) & 1u) ? &p->PFtc[full][v] : &p->Ptc[full][v];
            }
            cudaError_t e = mm::fold_state(p->d, p->n, fm, false, psi, p->fold_buf, s);
            if (e != cudaSuccess) return cuda_fail(e, "fold");
            if ((r = tc_begin(p, Mh, p->fold_buf, s))) return r;
            for (int64_t k = 0; k < nsteps; ++k) {
                const int64_t sw = p->sweep;  // the sweep about to run (tc_sweep's word rotation)
                if ((r = tc_sweep(p, k == 0 ? Mh : Mf, cur, mm::TcEpilogue{}, s))) return r;
                // its last product took its output scale from the maximum word W[sw - 1 mod 3][d - 1],
                // and the next sweep's first product reads its input scale from S[sw + 1 mod 2][0]
                const int d = p->d, t = int(sw % 3);
                const unsigned *max_in = p->d_max + ((t + 2) % 3) * d + (d - 1);
                float *s_next = p->d_scale + int((sw + 1) & 1) * d;
                e = mm::tc_phase_fold(p->st, fm, p->work[cur], p->work[1 - cur], max_in, s_next, tb, p->ctx->d_err,
                                      s);
                if (e != cudaSuccess) return cuda_fail(e, "nonlinear phase on the folded state");
                cur = 1 - cur;
            }
            if ((r = tc_sweep(p, Mh, cur, mm::TcEpilogue{}, s))) return r;
            if ((r = tc_end(p, cur, p->fold_buf, s))) return r;
            const double *W[mm::kMaxDims] = {};
            if (d_norm) {
                for (int v = 0; v < p->d; ++v) W[v] = p->Wpad[v];
                if ((e = cudaMemsetAsync(d_norm, 0, sizeof(double), s)) != cudaSuccess)
                    return cuda_fail(e, "norm accumulator");
            }
            e = mm::fold_state(p->d, p->n, fm, true, p->fold_buf, psi, s, d_norm ? W : nullptr, d_norm);
            return e == cudaSuccess ? MM_OK : cuda_fail(e, "unfold");
        });
    }
    return run_graphed(p, d_norm ? 5 : 2, psi, nsteps, s, tau, beta, [&]() -> mm_status {
        mm_status r;
        int cur = 0;
        mm::TcMatrix *Mh[mm::kMaxDims], *Mf[mm::kMaxDims];
        for (int v = 0; v < p->d; ++v) {
            Mh[v] = &p->Ptc[half][v];
            Mf[v] = &p->Ptc[full][v];
        }
        if ((r = tc_begin(p, Mh, psi, s))) return r;
        mm::TcEpilogue nl;
        nl.kind = 1;
        nl.tb = tb;
        for (int64_t k = 0; k < nsteps; ++k)
            if ((r = tc_sweep(p, k == 0 ? Mh : Mf, cur, nl, s))) return r;
        mm::TcEpilogue last;
        if (d_norm) {
            // the weights of the last direction's points: the directions before it (left index) and
            // after it (right index), in the point phase's decomposition
            const int v = p->order[p->d - 1] - 1, d = p->d;
            const int64_t np0 = p->st.np[0], np1 = d > 1 ? p->st.np[1] : 1;
            last.kind = 5;
            last.wo = p->Wpad[v];
            last.norm2 = d_norm;
            if (v == 0) {
                last.wr0 = d > 1 ? p->Wpad[1] : nullptr;
                last.wr1 = d > 2 ? p->Wpad[2] : nullptr;
                last.rdiv = np1;
            } else if (v == 1) {
                last.wl0 = p->Wpad[0];
                last.ldiv = np0;
                last.wr0 = d > 2 ? p->Wpad[2] : nullptr;
            } else {
                last.wl0 = p->Wpad[0];
                last.wl1 = p->Wpad[1];
                last.ldiv = np0;
            }
            cudaError_t e = cudaMemsetAsync(d_norm, 0, sizeof(double), s);
            if (e != cudaSuccess) return cuda_fail(e, "norm accumulator");
        }
        if ((r = tc_sweep(p, Mh, cur, last, s))) return r;
        return tc_end(p, cur, psi, s);
    });
}

}  // namespace

extern "C" {

mm_status split_step_gpe_norm2(mm_plan *p, void *psi, double beta, double tau, int64_t nsteps, double *norm2_host,
                               void *stream)
{
    NvtxRange range("split_step_gpe_norm2");
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    if (p->d != 3) return fail(MM_ERR_INVALID_ARG, "weighted norm needs a 3D Hermite plan");
    if (!norm2_host) return fail(MM_ERR_INVALID_ARG, "norm2_host is NULL");
    mm_status st = check_ptr(psi, "psi_dev");
    if (st) return st;
    if (nsteps < 0 || !std::isfinite(tau) || !std::isfinite(beta)) return fail(MM_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    bool fused = nsteps > 0 && p->tc && p->fixed && p->variant != mm::kTcOneSM;
    if (fused) {
        // the half-step propagator (the last sweep's) must have its pair tiling
        int half;
        if ((st = ensure_prop(p, 0.5 * tau, -1, &half))) return st;
        for (int v = 0; v < p->d && fused; ++v) fused = mm::tc_pair_ready(p->Ptc[half][v], p->variant);
    }
    if (!fused) {
        if ((st = split_step_gpe(p, psi, beta, tau, nsteps, stream))) return st;
        return mm_norm2(p, psi, 1, norm2_host, stream);
    }
    if (!p->d_norm && cudaMalloc(&p->d_norm, sizeof(double)) != cudaSuccess)
        return fail(MM_ERR_OOM, "norm accumulator");
    if ((st = gpe_steps(p, psi, beta, tau, nsteps, p->d_norm, s))) return st;
    cudaError_t e = cudaMemcpyAsync(norm2_host, p->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "norm");
    return MM_OK;
}

mm_status split_step_gpe(mm_plan *p, void *psi, double beta, double tau, int64_t nsteps, void *stream)
{
    NvtxRange range("split_step_gpe");
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    mm_status st = check_ptr(psi, "psi_dev");
    if (st) return st;
    if (nsteps < 0 || !std::isfinite(tau) || !std::isfinite(beta)) return fail(MM_ERR_INVALID_ARG, "bad arguments");
    if (nsteps == 0) return MM_OK;
    return gpe_steps(p, psi, beta, tau, nsteps, nullptr, (cudaStream_t)stream);
}

mm_status mm_norm2(mm_plan *p, const void *u_dev, int weighted, double *out_host, void *stream)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    if (!out_host) return fail(MM_ERR_INVALID_ARG, "out_host is NULL");
    mm_status st = check_ptr(u_dev, "u_dev");
    if (st) return st;
    if (weighted && (!p->hermite || p->d != 3)) return fail(MM_ERR_INVALID_ARG, "weighted norm needs a 3D Hermite plan");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(p->ctx->d_scratch, 0, sizeof(double), s);
    int64_t n1 = p->n[0], n2 = p->d > 1 ? p->n[1] : 1, n3 = p->count / (n1 * n2);
    if (e == cudaSuccess)
        e = mm::norm2_accumulate(p->dtype, n1, n2, n3, u_dev, weighted ? p->Wdev[0] : nullptr,
                                 weighted ? p->Wdev[1] : nullptr, weighted ? p->Wdev[2] : nullptr, p->ctx->d_scratch, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, p->ctx->d_scratch, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "norm");
    return MM_OK;
}

}  // extern "C"

// ---- adjoint of the GPE Strang step ---------------------------------------------------

namespace {

// conjugate transpose of an m x m complex matrix (interleaved)
std::vector<double> conj_transpose(const std::vector<double> &P, int64_t m)
{
    std::vector<double> H(P.size());
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < m; ++b) {
            H[size_t(2 * (a * m + b))] = P[size_t(2 * (b * m + a))];
            H[size_t(2 * (a * m + b) + 1)] = -P[size_t(2 * (b * m + a) + 1)];
        }
    return H;
}

struct MatSet {  // one matrix per direction, in the plan's precision
    void *simt[mm::kMaxDims] = {};
    mm::TcMatrix tc[mm::kMaxDims] = {};
    void release()
    {
        for (int v = 0; v < mm::kMaxDims; ++v) {
            if (simt[v]) cudaFree(simt[v]);
            simt[v] = nullptr;
            mm::tc_matrix_destroy(&tc[v]);
        }
    }
};

mm_status make_set(mm_plan *p, double s, bool adjoint, MatSet *out)
{
    for (int v = 0; v < p->d; ++v) {
        std::vector<double> P = harmonic_propagator(p, v, s);
        if (adjoint) P = conj_transpose(P, p->n[v]);
        mm_status st = upload_matrix(p, P.data(), p->n[v], p->n[v], true, &out->simt[v], &out->tc[v]);
        if (st) return st;
    }
    return MM_OK;
}

// out = L in (one linear flow: a sweep of the set's matrices); in may equal out.
mm_status apply_set(mm_plan *p, MatSet &S, const void *in, void *out, cudaStream_t s)
{
    if (!p->tc) {
        if (in != out) {
            cudaError_t e = cudaMemcpyAsync(out, in, size_t(p->count) * elem_bytes(p->dtype), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "copy");
        }
        return simt_sweep(p, S.simt, out, s);
    }
    mm::TcMatrix *M[mm::kMaxDims];
    for (int v = 0; v < p->d; ++v) M[v] = &S.tc[v];
    int cur = 0;
    mm_status st = tc_begin(p, M, in, s);
    if (st) return st;
    if ((st = tc_sweep(p, M, cur, mm::TcEpilogue{}, s))) return st;
    return tc_end(p, cur, out, s);
}

}  // namespace

struct AdjCache {
    double tau = NAN;
    MatSet Fh, Ff, Ah, Af;
    void *ckpt = nullptr, *mid = nullptr, *tmp = nullptr;
    size_t ckpt_bytes = 0, mid_bytes = 0, tmp_bytes = 0;
    void release_sets()
    {
        Fh.release();
        Ff.release();
        Ah.release();
        Af.release();
        tau = NAN;
    }
    static bool grow(void *&buf, size_t &have, size_t need)
    {
        if (have >= need) return true;
        if (buf) cudaFree(buf);
        buf = nullptr;
        have = 0;
        if (cudaMalloc(&buf, need) != cudaSuccess) return false;
        have = need;
        return true;
    }
    bool reserve(size_t ck, size_t md, size_t tp)
    {
        return grow(ckpt, ckpt_bytes, ck) && grow(mid, mid_bytes, md) && grow(tmp, tmp_bytes, tp);
    }
    ~AdjCache()
    {
        release_sets();
        if (ckpt) cudaFree(ckpt);
        if (mid) cudaFree(mid);
        if (tmp) cudaFree(tmp);
    }
};

void adj_release(mm_plan *p)
{
    delete p->adj;
    p->adj = nullptr;
}

extern "C" mm_status split_step_gpe_adjoint(mm_plan *p, const void *psi0, const void *gT, void *g0, double beta,
                                            double tau, int64_t nsteps, int64_t ckpt_every, void *stream)
{
    NvtxRange range("split_step_gpe_adjoint");
    if (!p || !p->hermite) return fail(MM_ERR_INVALID_ARG, "not a Hermite plan");
    mm_status st;
    if ((st = check_ptr(psi0, "psi0_dev")) || (st = check_ptr(gT, "gT_dev")) || (st = check_ptr(g0, "g0_dev")))
        return st;
    if (nsteps < 0 || ckpt_every < 1 || !std::isfinite(tau) || !std::isfinite(beta))
        return fail(MM_ERR_INVALID_ARG, "bad nsteps, ckpt_every, tau or beta");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = size_t(p->count) * elem_bytes(p->dtype);
    const bool fp64 = p->dtype == MM_C128;
    const double tb = tau * beta, h = 0.5 * tau;
    if (nsteps == 0) {
        cudaError_t e = cudaMemcpyAsync(g0, gT, bytes, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "copy");
    }
    const int64_t nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    const int64_t seglen = std::min(ckpt_every, nsteps);
    // matrices of the forward and adjoint half / full steps, built once per tau; checkpoint
    // buffers grown as needed; both kept with the plan for the next call
    if (!p->adj) p->adj = new AdjCache;
    AdjCache &C = *p->adj;
    if (!(C.tau == tau)) {
        C.release_sets();
        if ((st = make_set(p, h, false, &C.Fh)) || (st = make_set(p, tau, false, &C.Ff)) ||
            (st = make_set(p, h, true, &C.Ah)) || (st = make_set(p, tau, true, &C.Af))) {
            C.release_sets();
            return st;
        }
        C.tau = tau;
    }
    MatSet &Fh = C.Fh, &Ff = C.Ff, &Ah = C.Ah, &Af = C.Af;
    // Fused form (F16X6 on the CTA-pair kernel): the recomputed states before the nonlinear stages
    // come from the epilogue of each forward sweep (kind 3, which applies the phase as well), the
    // nonlinear adjoint runs in the epilogue of each adjoint sweep (kind 4), and the state stays in
    // pieces through a segment: one split and one merge per segment instead of per step.  The
    // stored states are complex64 in the padded layout of a piece plane.
    bool fused = p->tc && p->fixed && p->variant != mm::kTcOneSM;
    for (int v = 0; v < p->d && fused; ++v)
        fused = mm::tc_pair_ready(Fh.tc[v], p->variant) && mm::tc_pair_ready(Ff.tc[v], p->variant) &&
                mm::tc_pair_ready(Ah.tc[v], p->variant) && mm::tc_pair_ready(Af.tc[v], p->variant);
    const size_t mid_state = fused ? size_t(p->st.plane) * sizeof(float2) : bytes;
    if (!C.reserve(bytes * size_t(nseg), mid_state * size_t(seglen), bytes))
        return fail(MM_ERR_OOM, "checkpoint storage (%lld states)", (long long)(nseg + seglen + 1));
    void *ckpt = C.ckpt, *mid = C.mid, *tmp = C.tmp;
    auto ck = [&](int64_t k) { return static_cast<char *>(ckpt) + bytes * size_t(k); };
    auto md = [&](int64_t k) { return static_cast<char *>(mid) + bytes * size_t(k); };
    auto nl = [&](void *x) -> mm_status {
        cudaError_t e = mm::simt_nonlinear_phase(fp64, p->count, tb, x, s);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "nonlinear phase");
    };
    // forward sweep: checkpoints psi_{k c}, each segment by split_step_gpe (the same Strang
    // steps, the nonlinear phase fused into the last product) on the plan's scratch state
    cudaError_t e = cudaMemcpyAsync(tmp, psi0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy");
    for (int64_t k = 0; k < nseg; ++k) {
        e = cudaMemcpyAsync(ck(k), tmp, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
        if (k == nseg - 1) break;
        if ((st = split_step_gpe(p, tmp, beta, tau, ckpt_every, stream))) return st;
    }
    if (fused) {
        // reverse sweep, segment by segment.  Adjoint sweeps, in order: L_h^H then the nonlinear
        // adjoint of the last step, L_tau^H then that of each earlier step, a last L_h^H.
        e = cudaMemcpyAsync(g0, gT, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy");
        mm::TcMatrix *Mfh[mm::kMaxDims], *Mff[mm::kMaxDims], *Mah[mm::kMaxDims], *Maf[mm::kMaxDims];
        for (int v = 0; v < p->d; ++v) {
            Mfh[v] = &Fh.tc[v];
            Mff[v] = &Ff.tc[v];
            Mah[v] = &Ah.tc[v];
            Maf[v] = &Af.tc[v];
        }
        auto mid_at = [&](int64_t j) { return reinterpret_cast<float2 *>(static_cast<char *>(mid) + mid_state * size_t(j)); };
        for (int64_t k = nseg - 1; k >= 0 && !st; --k) {
            const int64_t first = k * ckpt_every, last = std::min(nsteps, first + ckpt_every);
            // the states before the nonlinear stages of steps first .. last - 1, from the checkpoint
            int cur = 0;
            st = tc_begin(p, Mfh, ck(k), s);
            for (int64_t q = first; q < last && !st; ++q) {
                mm::TcEpilogue ep;
                ep.kind = 3;
                ep.tb = tb;
                ep.mid_out = mid_at(q - first);
                st = tc_sweep(p, q == first ? Mfh : Mff, cur, ep, s);
            }
            if (st) break;
            // the adjoint through the segment, its state in pieces from split to merge
            cur = 0;
            st = tc_begin(p, last == nsteps ? Mah : Maf, g0, s);
            for (int64_t q = last - 1; q >= first && !st; --q) {
                mm::TcEpilogue ep;
                ep.kind = 4;
                ep.tb = tb;
                ep.mid_in = mid_at(q - first);
                st = tc_sweep(p, q == nsteps - 1 ? Mah : Maf, cur, ep, s);
            }
            if (!st && k == 0) st = tc_sweep(p, Mah, cur, mm::TcEpilogue{}, s);
            if (!st) st = tc_end(p, cur, g0, s);
        }
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (st) return st;
        if (e2 != cudaSuccess) return cuda_fail(e2, "adjoint (sync)");
        return MM_OK;
    }
    // reverse sweep, segment by segment: recompute the states before each
    // nonlinear stage, then g <- L_h^H (N^adj (L_h^H g)) per step, with the
    // adjacent L_h^H of consecutive steps merged into L_tau^H.
    e = cudaMemcpyAsync(g0, gT, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) st = apply_set(p, Ah, g0, g0, s);
    else st = cuda_fail(e, "copy");
    for (int64_t k = nseg - 1; k >= 0 && !st; --k) {
        const int64_t first = k * ckpt_every, last = std::min(nsteps, first + ckpt_every);
        st = apply_set(p, Fh, ck(k), md(0), s);  // state before the nonlinear stage of step `first`
        for (int64_t q = first + 1; q < last && !st; ++q) {
            e = cudaMemcpyAsync(md(q - first), md(q - first - 1), bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "copy");
            if (!st) st = nl(md(q - first));
            if (!st) st = apply_set(p, Ff, md(q - first), md(q - first), s);
        }
        for (int64_t q = last - 1; q >= first && !st; --q) {
            e = mm::simt_nonlinear_adjoint(fp64, p->count, tb, md(q - first), g0, s);
            if (e != cudaSuccess) st = cuda_fail(e, "nonlinear adjoint");
            if (!st) st = apply_set(p, q > 0 ? Af : Ah, g0, g0, s);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (st) return st;
    if (e2 != cudaSuccess) return cuda_fail(e2, "adjoint (sync)");
    return MM_OK;
}

// ---- batches of independent problems ---------------------------------------------------

struct mm_batch {
    mm_ctx *ctx = nullptr;
    std::vector<mm_plan *> plans;
    std::vector<unsigned> fold;  // each plan's folded directions when the batch was made (its records)
    int d = 0;
    mm_prec prec = MM_PREC_F16X6;
    bool fixed = false;
    // problem records for sweep position q and sweep k mod 6 (the input buffer follows k d + q mod 2,
    // the maximum words k mod 3): host copy and device array
    static constexpr int kPhases = 6;
    std::vector<mm::TcProblem> host[mm::kMaxDims][kPhases];
    mm::TcProblem *dev[mm::kMaxDims][kPhases] = {};
    bool kmajor[mm::kMaxDims] = {};
    // the same for the CTA-pair kernel (records opaque, mm::tc_pair_record_bytes() each), used when
    // every problem has a pair tiling with row tiles of the same size
    bool pair = false;
    std::vector<uint8_t> phost[mm::kMaxDims][kPhases];  // records start at recs(), aligned for their type
    void *pdev[mm::kMaxDims][kPhases] = {};
    uint8_t *recs(int q, int ph)
    {
        const uintptr_t a = mm::tc_pair_record_align(), p = reinterpret_cast<uintptr_t>(phost[q][ph].data());
        return reinterpret_cast<uint8_t *>((p + a - 1) / a * a);
    }
};

// Pair-kernel records of all (position, phase) of a batch; false if some product has no such tiling.
static bool build_pair_records(mm_batch *b, mm_plan *const *plans, int nprob)
{
    if (mm::tc_default_variant() == mm::kTcOneSM) return false;
    const size_t rb = mm::tc_pair_record_bytes();
    const int d = b->d;
    for (int q = 0; q < d; ++q)
        for (int ph = 0; ph < mm_batch::kPhases; ++ph) {
            auto &store = b->phost[q][ph];
            store.assign(rb * size_t(nprob) + mm::tc_pair_record_align(), 0);
            uint8_t *buf = b->recs(q, ph);
            const int cur = (ph * d + q) % 2;
            const int t = ph % 3;
            int64_t begin = 0;
            for (int k = 0; k < nprob; ++k) {
                mm_plan *p = plans[k];
                const int mu = p->order[q];
                mm::TcScales sc;
                if (p->fixed) {
                    const int par = ph & 1;  // sweep parity (kPhases is even)
                    sc.s_in = p->d_scale + par * d + q;
                    sc.s_out = (q + 1 < d) ? p->d_scale + par * d + q + 1 : p->d_scale + (1 - par) * d;
                    sc.max_prev = p->d_max + ((t + 2) % 3) * d + q;
                    sc.max_cur = p->d_max + t * d + q;
                    sc.zero_next = p->d_max + ((t + 1) % 3) * d + q;  // sweep k+1's word (see tc_sweep)
                }
                bool km = false;
                int64_t items = 0;
                void *rec = buf + rb * size_t(k);
                if (mm::tc_pair_record_build(p->st, p->st, mu, *step_matrix(p, mu - 1), p->prec, p->work[cur], p->work[1 - cur],
                                             sc, rec, &km, &items) != cudaSuccess ||
                    km != b->kmajor[q])
                    return false;
                mm::tc_pair_record_set_begin(rec, begin);
                begin += items;
            }
            if (!mm::tc_pair_batch_compatible(buf, nprob)) return false;
        }
    for (int q = 0; q < d; ++q)
        for (int ph = 0; ph < mm_batch::kPhases; ++ph) {
            const size_t bytes = rb * size_t(nprob);
            if (cudaMalloc(&b->pdev[q][ph], bytes) != cudaSuccess ||
                cudaMemcpy(b->pdev[q][ph], b->recs(q, ph), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
                return false;
        }
    return true;
}

extern "C" mm_status mumode_batch_create(mm_ctx *ctx, mm_plan *const *plans, int nprob, mm_batch **out)
{
    if (!ctx || !plans || !out) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    if (nprob < 1) return fail(MM_ERR_INVALID_ARG, "nprob = %d < 1", nprob);
    mm_plan *p0 = plans[0];
    if (!p0) return fail(MM_ERR_INVALID_ARG, "plans[0] is NULL");
    for (int k = 0; k < nprob; ++k) {
        mm_plan *p = plans[k];
        if (!p || p->hermite || !p->tc) return fail(MM_ERR_INVALID_ARG, "plan %d is not a tensor-core Tucker plan", k);
        if (p->tf32) return fail(MM_ERR_UNSUPPORTED, "plan %d: batches do not serve MM_PREC_TF32X3", k);
        if (p->ctx != ctx) return fail(MM_ERR_INVALID_ARG, "plan %d belongs to another context", k);
        if (p->prec != p0->prec || p->d != p0->d) return fail(MM_ERR_INVALID_ARG, "plan %d differs in precision or d", k);
        for (int v = 0; v < p->d; ++v)
            if (p->order[v] != p0->order[v]) return fail(MM_ERR_INVALID_ARG, "plan %d has another mode order", k);
        for (int j = 0; j < k; ++j)
            if (plans[j] == p) return fail(MM_ERR_INVALID_ARG, "plan %d appears twice", k);
    }
    auto *b = new mm_batch;
    b->ctx = ctx;
    b->plans.assign(plans, plans + nprob);
    for (int k = 0; k < nprob; ++k) b->fold.push_back(plans[k]->fold_mask);
    b->d = p0->d;
    b->prec = p0->prec;
    b->fixed = p0->fixed;
    const int d = b->d;
    for (int q = 0; q < d; ++q)
        for (int ph = 0; ph < mm_batch::kPhases; ++ph) {
            auto &vec = b->host[q][ph];
            vec.resize(size_t(nprob));
            int64_t begin = 0;
            const int cur = (ph * d + q) % 2;  // buffer holding the input of this launch
            const int t = ph % 3;              // maximum-word set (as in tc_sweep)
            for (int k = 0; k < nprob; ++k) {
                mm_plan *p = plans[k];
                const int mu = p->order[q];
                mm::TcScales sc;
                unsigned *zero = nullptr;
                if (p->fixed) {
                    const int par = ph & 1;  // sweep parity (kPhases is even)
                    sc.s_in = p->d_scale + par * d + q;
                    sc.s_out = (q + 1 < d) ? p->d_scale + par * d + q + 1 : p->d_scale + (1 - par) * d;
                    sc.max_prev = p->d_max + ((t + 2) % 3) * d + q;
                    sc.max_cur = p->d_max + t * d + q;
                    zero = p->d_max + ((t + 1) % 3) * d + q;  // sweep k+1's word (see tc_sweep)
                }
                bool km = false;
                cudaError_t e = mm::tc_problem_build(p->st, p->st, mu, *step_matrix(p, mu - 1), p->prec, p->work[cur],
                                                     p->work[1 - cur], sc, &vec[size_t(k)], &km);
                if (e != cudaSuccess) {
                    mm_batch_destroy(b);
                    return cuda_fail(e, "problem record");
                }
                vec[size_t(k)].pairs_begin = begin;
                vec[size_t(k)].zero_word = zero;
                begin += vec[size_t(k)].pairs;
                if (k == 0) b->kmajor[q] = km;
                else if (km != b->kmajor[q]) {
                    mm_batch_destroy(b);
                    return fail(MM_ERR_SHAPE, "plans disagree on the layout of direction %d", mu);
                }
            }
            const size_t bytes = sizeof(mm::TcProblem) * size_t(nprob);
            if (cudaMalloc(&b->dev[q][ph], bytes) != cudaSuccess) {
                mm_batch_destroy(b);
                return fail(MM_ERR_OOM, "problem records");
            }
            cudaError_t e = cudaMemcpy(b->dev[q][ph], vec.data(), bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                mm_batch_destroy(b);
                return cuda_fail(e, "problem records upload");
            }
        }
    b->pair = build_pair_records(b, plans, nprob);
    *out = b;
    return MM_OK;
}

extern "C" mm_status mumode_batch_step(mm_batch *b, void *const *u_dev, int64_t nsteps, void *stream)
{
    NvtxRange range("mumode_batch_step");
    if (!b || !u_dev) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    if (nsteps < 0) return fail(MM_ERR_INVALID_ARG, "nsteps < 0");
    mm_status st;
    for (size_t k = 0; k < b->plans.size(); ++k)
        if ((st = check_ptr(u_dev[k], "u_dev[k]"))) return st;
    if (nsteps == 0) return MM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int d = b->d;
    // split every problem (sets its state scale and first-sweep bounds)
    for (size_t k = 0; k < b->plans.size(); ++k) {
        mm_plan *p = b->plans[k];
        if (p->fixed) {
            cudaError_t e = cudaMemsetAsync(p->d_max, 0, sizeof(unsigned) * d, s);  // max words of sweep 0
            if (e != cudaSuccess) return cuda_fail(e, "max words");
        }
        const unsigned fm = b->fold[k];
        mm::TcMatrix *M[mm::kMaxDims];
        for (int v = 0; v < d; ++v) M[v] = ((fm >> v) & 1u) ? &p->Dtc[v] : &p->Etc[v];
        const void *src = u_dev[k];
        if (fm) {  // folded directions, as in mumode_step
            cudaError_t e = mm::fold_state(p->d, p->n, fm, false, u_dev[k], p->fold_buf, s);
            if (e != cudaSuccess) return cuda_fail(e, "fold");
            src = p->fold_buf;
        }
        if ((st = tc_begin(p, M, src, s))) return st;
    }
    for (int64_t t = 0; t < nsteps; ++t)
        for (int q = 0; q < d; ++q) {
            const int ph = int(t % mm_batch::kPhases);
            cudaEvent_t ev0 = timing_event(b->ctx, true);
            if (ev0) cudaEventRecord(ev0, s);
            cudaError_t e = b->pair ? mm::tc_pair_batch_launch(b->recs(q, ph), b->pdev[q][ph],
                                                               int(b->plans.size()), b->kmajor[q], b->prec,
                                                               b->ctx->d_err, s)
                                    : mm::tc_mode_product_batched(b->host[q][ph].data(), b->dev[q][ph],
                                                                  int(b->plans.size()), b->kmajor[q], b->prec,
                                                                  mm::TcEpilogue{}, b->ctx->d_err, s);
            if (ev0) cudaEventRecord(timing_event(b->ctx, false), s);
            if (e != cudaSuccess) return cuda_fail(e, "batched mode product");
        }
    const int cur = int((nsteps * d) % 2);
    for (size_t k = 0; k < b->plans.size(); ++k) {
        mm_plan *p = b->plans[k];
        const unsigned fm = b->fold[k];
        p->sweep = nsteps;  // the batched launches ran nsteps sweeps of every plan
        if (!fm) {
            if ((st = tc_end(p, cur, u_dev[k], s))) return st;
            continue;
        }
        if ((st = tc_end(p, cur, p->fold_buf, s))) return st;
        cudaError_t e = mm::fold_state(p->d, p->n, fm, true, p->fold_buf, u_dev[k], s);
        if (e != cudaSuccess) return cuda_fail(e, "unfold");
    }
    return MM_OK;
}

extern "C" void mm_batch_destroy(mm_batch *b)
{
    if (!b) return;
    for (int q = 0; q < mm::kMaxDims; ++q)
        for (int ph = 0; ph < mm_batch::kPhases; ++ph) {
            if (b->dev[q][ph]) cudaFree(b->dev[q][ph]);
            if (b->pdev[q][ph]) cudaFree(b->pdev[q][ph]);
        }
    delete b;
}

extern "C" mm_status mumode_step_batched(mm_ctx *ctx, mm_plan *const *plans, void *const *u_dev, int nprob,
                                          int64_t nsteps, void *stream)
{
    mm_batch *b = nullptr;
    mm_status st = mumode_batch_create(ctx, plans, nprob, &b);
    if (st) return st;
    st = mumode_batch_step(b, u_dev, nsteps, stream);
    // the batch's device records stay in use until its launches finish
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    mm_batch_destroy(b);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batched step (sync)");
    return MM_OK;
}

extern "C" mm_status mumode_batch_autotune(mm_ctx *ctx, mm_plan *const *plans, void *const *u_dev, int nprob,
                                           int64_t nsteps, int *order_out, void *stream)
{
    if (!ctx || !plans || !u_dev || nprob < 1) return fail(MM_ERR_INVALID_ARG, "ctx, plans or u_dev missing");
    if (nsteps < 1 || nsteps > 1000) return fail(MM_ERR_INVALID_ARG, "nsteps = %lld outside 1..1000", (long long)nsteps);
    for (int k = 0; k < nprob; ++k) {
        if (!plans[k] || !u_dev[k]) return fail(MM_ERR_INVALID_ARG, "plans[%d] or u_dev[%d] is NULL", k, k);
        if (plans[k]->hermite || !plans[k]->tc || plans[k]->d != plans[0]->d)
            return fail(MM_ERR_INVALID_ARG, "plan %d is not a tensor-core Tucker plan of plan 0's d", k);
    }
    const int d = plans[0]->d;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<void *> scratch(size_t(nprob), nullptr);
    auto release = [&]() {
        for (void *q : scratch)
            if (q) cudaFree(q);
    };
    for (int k = 0; k < nprob; ++k)
        if (cudaMalloc(&scratch[size_t(k)], size_t(plans[k]->count) * elem_bytes(plans[k]->dtype)) != cudaSuccess) {
            scratch[size_t(k)] = nullptr;
            release();
            return fail(MM_ERR_OOM, "batch autotune scratch");
        }
    std::vector<int> ord(plans[0]->order, plans[0]->order + d), best_o = ord;
    std::vector<std::vector<int>> orders;
    if (d <= 4) {
        std::vector<int> o(static_cast<size_t>(d), 0);
        for (int v = 0; v < d; ++v) o[size_t(v)] = v + 1;
        do orders.push_back(o);
        while (std::next_permutation(o.begin(), o.end()));
    } else {
        orders.push_back(ord);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    mm_status st = MM_OK;
    for (const auto &o : orders) {
        for (int k = 0; k < nprob && !st; ++k) st = mm_plan_set_config(plans[k], int(plans[k]->variant), o.data());
        mm_batch *b = nullptr;
        if (!st) st = mumode_batch_create(ctx, plans, nprob, &b);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < nprob && !st && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(scratch[size_t(k)], u_dev[k], size_t(plans[k]->count) * elem_bytes(plans[k]->dtype),
                                cudaMemcpyDeviceToDevice, s);
        if (!st && e == cudaSuccess && !(st = mumode_batch_step(b, scratch.data(), 1, stream))) {
            cudaEventRecord(e0, s);
            st = mumode_batch_step(b, scratch.data(), nsteps, stream);
            cudaEventRecord(e1, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (b) mm_batch_destroy(b);
        if (e != cudaSuccess && !st) st = cuda_fail(e, "batch autotune");
        if (st) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_o = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    const std::vector<int> &keep = st ? ord : best_o;
    for (int k = 0; k < nprob; ++k) mm_plan_set_config(plans[k], int(plans[k]->variant), keep.data());
    if (order_out && !st)
        for (int v = 0; v < d; ++v) order_out[v] = keep[size_t(v)];
    return st;
}

// ---------------------------------------------------------------------------
// Device exponentials, device matrix updates and HKMP (section 4.4)

static double norm1_host(int m, const double *A)
{
    double best = 0.0;
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += std::fabs(A[size_t(i) * m + j]);
        best = std::max(best, s);
    }
    return best;
}

extern "C" mm_status mm_expm_device(mm_ctx *ctx, int n, const double *A_dev, const double *B_dev, double f, double z_re,
                                    double z_im, double norm_bound, double *E_dev, void *stream)
{
    if (!ctx) return fail(MM_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 1 || n > 4096) return fail(MM_ERR_SHAPE, "n = %d outside 1..4096", n);
    mm_status st;
    if ((st = check_ptr(A_dev, "A_dev")) || (st = check_ptr(E_dev, "E_dev"))) return st;
    if (B_dev && (st = check_ptr(B_dev, "B_dev"))) return st;
    if (!std::isfinite(f) || !std::isfinite(z_re) || !std::isfinite(z_im) || !std::isfinite(norm_bound))
        return fail(MM_ERR_INVALID_ARG, "f, z or norm_bound is not finite");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = mm::expm_workspace_init(&ctx->expm, n);
    if (e != cudaSuccess) return fail(MM_ERR_OOM, "expm workspace (%s)", cudaGetErrorString(e));
    if (norm_bound <= 0.0) {
        e = mm::expm_norm1_device(&ctx->expm, n, A_dev, B_dev, f, &norm_bound, s);
        if (e != cudaSuccess) return cuda_fail(e, "expm norm");
    }
    if (z_re == 0.0 || z_im == 0.0) {  // real arithmetic: cos + i sin, or the real series
        if ((e = mm::expm_batch_init(&ctx->expmb, n, 1)) != cudaSuccess)
            return fail(MM_ERR_OOM, "expm workspace (%s)", cudaGetErrorString(e));
        e = z_re == 0.0 ? mm::expm_imag_batched(&ctx->expmb, n, A_dev, B_dev, &f, 1, z_im, norm_bound,
                                                reinterpret_cast<double2 *>(E_dev), s)
                        : mm::expm_real_device(&ctx->expmb, n, A_dev, B_dev, f, z_re, norm_bound,
                                               reinterpret_cast<double2 *>(E_dev), s);
    } else {
        e = mm::expm_device(&ctx->expm, n, A_dev, B_dev, f, z_re, z_im, norm_bound, reinterpret_cast<double2 *>(E_dev),
                            s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "device expm");
    return MM_OK;
}

// Replace direction mu's matrix by a device matrix, in stream order.
static mm_status set_matrix_device(mm_plan *p, int mu, const double2 *E, double row_norm_bound, cudaStream_t s)
{
    // the direction's new matrix is not folded: later steps use it as it is (the fold is per call)
    if ((p->fold_avail >> (mu - 1)) & 1u) {
        drop_graphs(p);
        p->fold_mask &= ~(1u << (mu - 1));
        p->fold_avail &= ~(1u << (mu - 1));
        p->chain_steps = -1;  // chained records point at the folded matrix
    }
    const int v = mu - 1;
    if (p->tf32) return fail(MM_ERR_UNSUPPORTED, "device matrix updates do not serve MM_PREC_TF32X3 plans");
    if (p->tc) {
        if (!p->full_bands[v]) {
            drop_graphs(p);  // captured launches carry the old bands
            mm::tc_matrix_full_bands(p->Etc[v]);
            p->full_bands[v] = true;
        }
        p->Etc[v].row_norm = row_norm_bound;
        cudaError_t e = mm::tc_matrix_update(p->Etc[v], E, s);
        if (e != cudaSuccess) return cuda_fail(e, "matrix update");
        return MM_OK;
    }
    if (p->dtype != MM_C128) return fail(MM_ERR_DTYPE, "device matrices need MM_C128 data on the FP64 paths");
    if (reinterpret_cast<const void *>(E) == p->Edev[v]) return MM_OK;
    cudaError_t e = cudaMemcpyAsync(p->Edev[v], E, sizeof(double2) * size_t(p->n[v] * p->n[v]), cudaMemcpyDeviceToDevice,
                                    s);
    if (e != cudaSuccess) return cuda_fail(e, "matrix copy");
    return MM_OK;
}

extern "C" mm_status mm_plan_set_matrix_device(mm_plan *p, int mu, const double *E_dev, double row_norm_bound,
                                               void *stream)
{
    if (!p) return fail(MM_ERR_INVALID_ARG, "plan is NULL");
    if (p->hermite) return fail(MM_ERR_INVALID_ARG, "needs a Tucker plan");
    if (mu < 1 || mu > p->d) return fail(MM_ERR_INVALID_ARG, "mu = %d outside 1..%d", mu, p->d);
    mm_status st = check_ptr(E_dev, "E_dev");
    if (st) return st;
    if (!std::isfinite(row_norm_bound)) return fail(MM_ERR_INVALID_ARG, "row_norm_bound is not finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (row_norm_bound <= 0.0 && p->tc) {
        // max_i sum_j |E_ij| from the device copy (synchronises the stream)
        const int64_t m = p->n[mu - 1];
        std::vector<double> h(size_t(2 * m * m));
        cudaError_t e = cudaMemcpyAsync(h.data(), E_dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "matrix read-back");
        for (int64_t i = 0; i < m; ++i) {
            double r = 0.0;
            for (int64_t j = 0; j < m; ++j) r += std::hypot(h[size_t(2 * (i * m + j))], h[size_t(2 * (i * m + j) + 1)]);
            row_norm_bound = std::max(row_norm_bound, r);
        }
    }
    return set_matrix_device(p, mu, reinterpret_cast<const double2 *>(E_dev), row_norm_bound, s);
}

extern "C" mm_status hkmp_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *V_nodes,
                                      const double *const *U_nodes, double tau, mm_dtype dtype, mm_prec prec,
                                      mm_plan **out)
{
    if (!std::isfinite(tau)) return fail(MM_ERR_INVALID_ARG, "tau is not finite");
    mm_plan *p = nullptr;
    mm_status st = plan_common(ctx, d, n, dtype, prec, nullptr, true, out, &p);
    if (st) return st;
    if (!(p->tc || (dtype == MM_C128 && (p->prec == MM_PREC_FP64_SIMT || p->prec == MM_PREC_FP64_DMMA)))) {
        delete p;
        return fail(MM_ERR_DTYPE, "HKMP plans need a tensor-core precision (MM_C64) or an FP64 one (MM_C128)");
    }
    if (p->tf32) {
        delete p;
        return fail(MM_ERR_UNSUPPORTED, "MM_PREC_TF32X3 serves Tucker plans and mumode_product only");
    }
    if ((st = hermite_setup(p))) {
        mm_plan_destroy(p);
        return st;
    }
    p->hkmp = true;
    p->tau = tau;
    int nmax = 0;
    for (int v = 0; v < d; ++v) {
        const int m = int(n[v]);
        std::vector<double> H(size_t(m) * m), G(size_t(m) * m, 0.0);
        mm::hermite_hamiltonian(m, p->x[v].data(), p->W[v].data(), V_nodes ? V_nodes[v] : nullptr, H.data());
        std::vector<cd> E(size_t(m) * m);
        if (!mm::expm(m, H.data(), nullptr, cd(0.0, -tau), E.data())) {
            mm_plan_destroy(p);
            return fail(MM_ERR_INVALID_ARG, "expm of direction %d failed", v + 1);
        }
        // the constant directions keep this exponential; the time-dependent
        // ones start from it (f = 0) and are rewritten every step
        if ((st = upload_matrix(p, reinterpret_cast<const double *>(E.data()), m, m, true, &p->Edev[v], &p->Etc[v]))) {
            mm_plan_destroy(p);
            return st;
        }
        const double *U = U_nodes ? U_nodes[v] : nullptr;
        if (!U) continue;
        mm::hermite_galerkin(m, p->x[v].data(), p->W[v].data(), U, G.data());
        double dmin = H[0], dmax = H[0];
        for (int k = 0; k < m; ++k) {
            dmin = std::min(dmin, H[size_t(k) * m + k]);
            dmax = std::max(dmax, H[size_t(k) * m + k]);
        }
        p->hshift[v] = 0.5 * (dmin + dmax);
        std::vector<double> Hs(H);
        for (int k = 0; k < m; ++k) Hs[size_t(k) * m + k] -= p->hshift[v];
        p->h0norm[v] = norm1_host(m, Hs.data());
        p->gnorm[v] = norm1_host(m, G.data());
        const size_t bytes = sizeof(double) * size_t(m) * m;
        if (cudaMalloc(&p->H0dev[v], bytes) != cudaSuccess || cudaMalloc(&p->Gdev[v], bytes) != cudaSuccess ||
            cudaMemcpy(p->H0dev[v], H.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p->Gdev[v], G.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            mm_plan_destroy(p);
            return fail(MM_ERR_OOM, "HKMP matrices");
        }
        if (p->tc) {
            mm::tc_matrix_full_bands(p->Etc[v]);
            p->full_bands[v] = true;
            p->Etc[v].row_norm = std::sqrt(double(m));  // bound for a unitary matrix: sum_j |E_ij| <= sqrt(m)
        }
        nmax = std::max(nmax, m);
    }
    // fusion: tensor cores, the pair kernel's tilings, d <= 3, one time-dependent direction, the
    // others harmonic (their exponentials are the diagonal phases)
    {
        int td = -1, ntd = 0;
        bool others_harmonic = true;
        for (int v = 0; v < d; ++v) {
            if (p->H0dev[v]) {
                td = v;
                ++ntd;
            } else if (V_nodes && V_nodes[v]) {
                others_harmonic = false;
            }
        }
        if (p->tc && d <= 3 && ntd == 1 && others_harmonic) {
            p->hk_fuse = td;
            for (int v = 0; v < d && p->hk_fuse >= 0; ++v) {
                if (v == td) continue;
                const int64_t np = (n[v] + 15) / 16 * 16;
                std::vector<double2> ph(size_t(np), make_double2(1.0, 0.0));
                for (int64_t k = 0; k < n[v]; ++k) {
                    const double a = -tau * (double(k) + 0.5);
                    ph[size_t(k)] = make_double2(std::cos(a), std::sin(a));
                }
                if (cudaMalloc(&p->hk_phase[v], sizeof(double2) * size_t(np)) != cudaSuccess ||
                    cudaMemcpy(p->hk_phase[v], ph.data(), sizeof(double2) * size_t(np), cudaMemcpyHostToDevice) !=
                        cudaSuccess) {
                    mm_plan_destroy(p);
                    return fail(MM_ERR_OOM, "HKMP phases");
                }
            }
        }
    }
    cudaError_t e = cudaMalloc(&p->coef, size_t(p->count) * elem_bytes(dtype));
    if (e == cudaSuccess && nmax > 0) {
        const int cap = mm::expm_batch_capacity(nmax);
        e = mm::expm_batch_init(&p->expmb, nmax, cap);
        for (int v = 0; v < d && e == cudaSuccess; ++v)
            if (p->H0dev[v])
                e = cudaMalloc(&p->Ebatch[v], sizeof(double2) * size_t(cap) * size_t(p->n[v] * p->n[v]));
        // interpolation in f (tensor-core plans, when a batch holds the nodes)
        const int K = mm::kInterpNodes;
        if (e == cudaSuccess && p->tc && cap > K) {
            e = cudaMalloc(&p->hk_w, sizeof(double) * size_t(cap) * K);
            for (int v = 0; v < d && e == cudaSuccess; ++v)
                if (p->H0dev[v])
                    e = cudaMalloc(&p->hk_nodesE[v], sizeof(double2) * size_t(K) * size_t(p->n[v] * p->n[v]));
        }
    }
    if (e != cudaSuccess) {
        mm_plan_destroy(p);
        return fail(MM_ERR_OOM, "HKMP workspace");
    }
    *out = p;
    return MM_OK;
}

namespace {

// The fewest Chebyshev nodes (4..kInterpNodes) whose interpolation error bound for
// exp(-i tau (H0 + f G)) over f in [flo, fhi], 2 (tau ||G|| (fhi - flo) / 4)^K / K!, is below
// 1e-14 in every time-dependent direction; kInterpNodes + 1 when none is.
int hk_nodes_for(const mm_plan *p, double flo, double fhi)
{
    int K = 0;
    for (int v = 0; v < p->d; ++v) {
        if (!p->H0dev[v]) continue;
        const double x = std::fabs(p->tau) * p->gnorm[v] * (fhi - flo) / 4.0;
        int k = 4;
        double bound = 2.0 * std::pow(x, 4) / 24.0;
        while (bound > 1e-14 && k < mm::kInterpNodes) {
            ++k;
            bound *= x / k;
        }
        if (bound > 1e-14) k = mm::kInterpNodes + 1;
        K = std::max(K, k);
    }
    return K;
}

// The K Chebyshev points of the first kind of [flo, fhi] and their barycentric weights.
void hk_cheb_nodes(double flo, double fhi, int K, double *nodes, double *bw)
{
    const double mid = 0.5 * (flo + fhi), half = 0.5 * (fhi - flo), pi = 3.14159265358979323846;
    for (int j = 0; j < K; ++j) {
        const double th = (2 * j + 1) * pi / (2 * K);
        nodes[j] = mid + half * std::cos(th);
        bw[j] = (j % 2 ? -1.0 : 1.0) * std::sin(th);
    }
}

// W[q K + j]: the Lagrange basis of the nodes at f[q] (barycentric form), q < cnt.
void hk_lagrange(const double *nodes, const double *bw, int K, const double *f, int cnt, double *W)
{
    for (int q = 0; q < cnt; ++q) {
        const double x = f[q];
        double *w = W + size_t(q) * K, sum = 0.0;
        int hit = -1;
        for (int j = 0; j < K && hit < 0; ++j)
            if (x == nodes[j]) hit = j;
        for (int j = 0; j < K; ++j) {
            w[j] = hit >= 0 ? (j == hit ? 1.0 : 0.0) : bw[j] / (x - nodes[j]);
            sum += w[j];
        }
        for (int j = 0; j < K; ++j) w[j] /= sum;
    }
}

}  // namespace

extern "C" mm_status hkmp_set_f_range(mm_plan *p, double f_lo, double f_hi, void *stream)
{
    NvtxRange range("hkmp_set_f_range");
    if (!p || !p->hkmp) return fail(MM_ERR_INVALID_ARG, "not an HKMP plan");
    if (!std::isfinite(f_lo) || !std::isfinite(f_hi)) return fail(MM_ERR_INVALID_ARG, "f range not finite");
    if (f_lo >= f_hi) {  // drop the range
        p->hk_rK = 0;
        return MM_OK;
    }
    if (!p->tc || !p->hk_w) return fail(MM_ERR_UNSUPPORTED, "a declared f range needs a tensor-core HKMP plan");
    const int K = hk_nodes_for(p, f_lo, f_hi);
    if (K > mm::kInterpNodes)
        return fail(MM_ERR_INVALID_ARG, "f range [%g, %g] needs more than %d interpolation nodes", f_lo, f_hi,
                    mm::kInterpNodes);
    cudaStream_t s = (cudaStream_t)stream;
    p->hk_rK = 0;  // invalid until the new nodes are in place
    double nodes[mm::kInterpNodes], bw[mm::kInterpNodes];
    hk_cheb_nodes(f_lo, f_hi, K, nodes, bw);
    const double fmax = std::max(std::fabs(f_lo), std::fabs(f_hi));
    for (int v = 0; v < p->d; ++v) {
        if (!p->H0dev[v]) continue;
        if (!p->hk_rangeE[v] && cudaMalloc(&p->hk_rangeE[v], sizeof(double2) * size_t(mm::kInterpNodes) *
                                                                  size_t(p->n[v] * p->n[v])) != cudaSuccess) {
            p->hk_rangeE[v] = nullptr;
            return fail(MM_ERR_OOM, "node exponentials of the f range");
        }
        const double bound = p->h0norm[v] + fmax * p->gnorm[v];
        cudaError_t e = mm::expm_imag_batched(&p->expmb, int(p->n[v]), p->H0dev[v], p->Gdev[v], nodes, K, -p->tau,
                                              bound, p->hk_rangeE[v], s, p->hshift[v], 2.0);
        if (e != cudaSuccess) return cuda_fail(e, "node exponentials of the f range");
    }
    // the nodes are read by asynchronous copies
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "node exponentials of the f range");
    p->hk_rlo = f_lo;
    p->hk_rhi = f_hi;
    p->hk_rK = K;
    return MM_OK;
}

extern "C" mm_status hkmp_evolve(mm_plan *p, void *psi, int64_t nsteps, const double *f_mid, void *stream)
{
    NvtxRange range("hkmp_evolve");
    if (!p || !p->hkmp) return fail(MM_ERR_INVALID_ARG, "not an HKMP plan");
    mm_status st = check_ptr(psi, "psi_dev");
    if (st) return st;
    if (nsteps < 0) return fail(MM_ERR_INVALID_ARG, "nsteps < 0");
    if (nsteps > 0 && !f_mid) return fail(MM_ERR_INVALID_ARG, "f_mid is NULL");
    for (int64_t k = 0; k < nsteps; ++k)
        if (!std::isfinite(f_mid[k])) return fail(MM_ERR_INVALID_ARG, "f_mid[%lld] is not finite", (long long)k);
    if (nsteps == 0) return MM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // The exponentials exp(-i tau (H0 + f G)) of the time-dependent directions
    // for a chunk of steps [k0, k0 + cnt), computed together (batched).
    const int cap = p->expmb.cap;
    // Tensor-core plans: E(f) = exp(-i tau (H0 + f G)) is an entire function of f whose k-th
    // derivative is at most (tau ||G||)^k in norm, so its interpolant at K Chebyshev points of
    // [f_lo, f_hi] errs by at most 2 (tau ||G|| (f_hi - f_lo) / 4)^K / K!.  K is the smallest
    // (4..12) that puts this below 1e-14 (the pieces hold 2^-34 of a row's scale); a chunk of more
    // than K steps then takes K exponentials and one combination instead of one exponential per
    // step.  The node values and weights stay in host memory until the call's final
    // synchronisation (their copies are asynchronous).
    const int Kmax = mm::kInterpNodes;
    const bool interp = p->tc && p->hk_w != nullptr;
    const int64_t nchunks = (nsteps + cap - 1) / cap;
    std::vector<double> ihost(interp ? size_t(nchunks) * size_t(Kmax + size_t(cap) * Kmax) : 0);
    auto chunk = [&](int64_t k0, int cnt) -> mm_status {
        double fmax = 0.0, flo = f_mid[k0], fhi = f_mid[k0];
        for (int q = 0; q < cnt; ++q) {
            fmax = std::max(fmax, std::fabs(f_mid[k0 + q]));
            flo = std::min(flo, f_mid[k0 + q]);
            fhi = std::max(fhi, f_mid[k0 + q]);
        }
        // a declared f range that holds the chunk: its node exponentials, combined only
        if (interp && p->hk_rK > 0 && flo >= p->hk_rlo && fhi <= p->hk_rhi) {
            const int K = p->hk_rK;
            double *nodes = ihost.data() + size_t(k0 / cap) * size_t(Kmax + size_t(cap) * Kmax);
            double *W = nodes + Kmax, bw[mm::kInterpNodes];
            hk_cheb_nodes(p->hk_rlo, p->hk_rhi, K, nodes, bw);
            hk_lagrange(nodes, bw, K, f_mid + k0, cnt, W);
            cudaError_t e = cudaMemcpyAsync(p->hk_w, W, sizeof(double) * size_t(cnt) * K, cudaMemcpyHostToDevice, s);
            for (int v = 0; v < p->d && e == cudaSuccess; ++v)
                if (p->H0dev[v])
                    e = mm::combine_interp_nodes(int(p->n[v]), cnt, K, p->hk_w, p->hk_rangeE[v], p->Ebatch[v], s);
            return e == cudaSuccess ? MM_OK : cuda_fail(e, "exponentials from the f range's nodes");
        }
        // the fewest nodes whose error bound is below 1e-14, over the time-dependent directions
        const int K = hk_nodes_for(p, flo, fhi);
        const bool use_interp = interp && K <= Kmax && cnt > K && fhi > flo;
        double *nodes = nullptr;
        if (use_interp) {
            nodes = ihost.data() + size_t(k0 / cap) * size_t(Kmax + size_t(cap) * Kmax);
            double *W = nodes + Kmax, bw[mm::kInterpNodes];
            hk_cheb_nodes(flo, fhi, K, nodes, bw);  // Chebyshev points of the first kind
            hk_lagrange(nodes, bw, K, f_mid + k0, cnt, W);
            cudaError_t e = cudaMemcpyAsync(p->hk_w, W, sizeof(double) * size_t(cnt) * K, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "interpolation weights");
        }
        for (int v = 0; v < p->d; ++v) {
            if (!p->H0dev[v]) continue;
            const double bound = p->h0norm[v] + fmax * p->gnorm[v];
            // tensor-core plans split the exponentials into pieces: scaled norms up to 2 suffice
            cudaError_t e;
            if (use_interp) {
                e = mm::expm_imag_batched(&p->expmb, int(p->n[v]), p->H0dev[v], p->Gdev[v], nodes, K, -p->tau, bound,
                                          p->hk_nodesE[v], s, p->hshift[v], 2.0);
                if (e == cudaSuccess)
                    e = mm::combine_interp_nodes(int(p->n[v]), cnt, K, p->hk_w, p->hk_nodesE[v], p->Ebatch[v], s);
            } else {
                e = mm::expm_imag_batched(&p->expmb, int(p->n[v]), p->H0dev[v], p->Gdev[v], f_mid + k0, cnt,
                                          -p->tau, bound, p->Ebatch[v], s, p->hshift[v], p->tc ? 2.0 : 1.0);
            }
            if (e != cudaSuccess) return cuda_fail(e, "device expm");
        }
        return MM_OK;
    };
    // step k's matrices: the batch slot of each time-dependent direction
    void *Ed[mm::kMaxDims];
    auto select = [&](int slot) -> mm_status {
        for (int v = 0; v < p->d; ++v) {
            Ed[v] = p->Edev[v];
            if (!p->H0dev[v]) continue;
            double2 *E = p->Ebatch[v] + size_t(slot) * size_t(p->n[v] * p->n[v]);
            if (!p->tc) {
                Ed[v] = E;
                continue;
            }
            // each step's matrix is split again before its product: only the variant's layout
            cudaError_t e = mm::tc_matrix_update(p->Etc[v], E, s, &p->variant);
            if (e != cudaSuccess) return cuda_fail(e, "matrix update");
        }
        return MM_OK;
    };
    if ((st = hermite_apply(p, true, psi, p->coef, stream))) return st;
    int cur = 0;
    mm::TcMatrix *M[mm::kMaxDims];
    for (int v = 0; v < p->d; ++v) M[v] = &p->Etc[v];
    const bool fused = p->hk_fuse >= 0 && p->variant != mm::kTcOneSM;
    mm::TcEpilogue epi2;  // fused: the other directions' phases at every output point
    if (fused) {
        const int v = p->hk_fuse, d = p->d;
        const int64_t np[3] = {p->st.np[0], d > 1 ? p->st.np[1] : 1, d > 2 ? p->st.np[2] : 1};
        epi2.kind = 2;
        if (v == 0) {  // points: right index over directions 2, 3
            epi2.pr0 = p->hk_phase[1];
            epi2.pr1 = d > 2 ? p->hk_phase[2] : nullptr;
            epi2.rdiv = np[1];
        } else if (v == 1) {  // left: direction 1; right: direction 3
            epi2.pl0 = p->hk_phase[0];
            epi2.ldiv = np[0];
            epi2.pr0 = d > 2 ? p->hk_phase[2] : nullptr;
            epi2.rdiv = d > 2 ? np[2] : 1;
        } else {  // left index over directions 1, 2
            epi2.pl0 = p->hk_phase[0];
            epi2.pl1 = p->hk_phase[1];
            epi2.ldiv = np[0];
        }
    }
    // one product per step (fused): a one-position sweep of direction hk_fuse + 1
    auto fused_step = [&]() -> mm_status {
        mm::TcScales sc;
        const int t = int(p->sweep % 3), par = int(p->sweep & 1), d = p->d;
        sc.s_in = p->d_scale + par * d;
        sc.s_out = p->d_scale + (1 - par) * d;
        sc.max_prev = p->d_max + ((t + 2) % 3) * d;
        sc.max_cur = p->d_max + t * d;
        sc.zero_next = p->d_max + ((t + 1) % 3) * d;
        const int mu = p->hk_fuse + 1;
        cudaError_t e = mm::tc_mode_product(p->st, p->st, mu, p->Etc[mu - 1], p->prec, p->work[cur], p->work[1 - cur],
                                            epi2, sc, p->ctx->d_err, s, p->variant);
        if (e != cudaSuccess) return cuda_fail(e, "HKMP fused product");
        cur = 1 - cur;
        ++p->sweep;
        return MM_OK;
    };
    for (int64_t k0 = 0; k0 < nsteps; k0 += cap) {
        const int cnt = int(std::min<int64_t>(cap, nsteps - k0));
        if ((st = chunk(k0, cnt))) return st;
        for (int q = 0; q < cnt; ++q) {
            if ((st = select(q))) return st;
            if (!p->tc) {
                if ((st = simt_sweep(p, Ed, p->coef, s))) return st;
                continue;
            }
            if (k0 == 0 && q == 0) {
                if (fused) {
                    double b[mm::kMaxDims];  // one position per sweep: its product; the phases have modulus 1
                    for (int v = 0; v < mm::kMaxDims; ++v) b[v] = p->Etc[p->hk_fuse].row_norm;
                    st = tc_begin_bounds(p, b, p->coef, s);
                } else {
                    st = tc_begin(p, M, p->coef, s);
                }
                if (st) return st;
            }
            if ((st = fused ? fused_step() : tc_sweep(p, M, cur, mm::TcEpilogue{}, s))) return st;
        }
    }
    if (p->tc && (st = tc_end(p, cur, p->coef, s))) return st;
    // f_mid is read by the batched exponentials' host-to-device copies, which
    // may still be queued: finish them before the caller may free the array
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "HKMP steps");
    return hermite_apply(p, false, p->coef, psi, stream);
}

// ---------------------------------------------------------------------------
// Pipe flow (section 4.2)

extern "C" mm_status mm_pipe_operators(int n_r, int n_z, double rmin, double rmax, double zmax, double alpha,
                                       const double *s_nodes, double *A_r, double *A_z)
{
    if (n_r < 2 || n_r > 4096 || n_z < 2 || n_z > 4096) return fail(MM_ERR_SHAPE, "n_r, n_z must be in 2..4096");
    if (!(rmin > 0.0) || !(rmax > rmin) || !(zmax > 0.0) || !(alpha > 0.0) || !std::isfinite(rmax) ||
        !std::isfinite(zmax) || !std::isfinite(alpha))
        return fail(MM_ERR_INVALID_ARG, "need 0 < r_min < r_max, z_max > 0, alpha > 0");
    if (A_r) mm::pipe_radial(n_r, rmin, rmax, alpha, A_r);
    if (A_z) mm::pipe_axial(n_z, zmax, alpha, s_nodes, A_z);
    return MM_OK;
}

extern "C" mm_status pipe_plan_create(mm_ctx *ctx, int n_r, int n_z, double rmin, double rmax, double zmax,
                                      double alpha, const double *s_nodes, double T, mm_prec prec, mm_plan **out)
{
    if (!ctx || !out) return fail(MM_ERR_INVALID_ARG, "NULL argument");
    if (!std::isfinite(T)) return fail(MM_ERR_INVALID_ARG, "T is not finite");
    if (prec != MM_PREC_FP64_SIMT && prec != MM_PREC_FP64_DMMA)
        return fail(MM_ERR_UNSUPPORTED, "pipe flow runs on the FP64 paths (MM_PREC_FP64_SIMT or MM_PREC_FP64_DMMA)");
    const int nn[2] = {n_r, n_z};
    std::vector<double> A[2] = {std::vector<double>(size_t(n_r) * n_r), std::vector<double>(size_t(n_z) * n_z)};
    mm_status st = mm_pipe_operators(n_r, n_z, rmin, rmax, zmax, alpha, s_nodes, A[0].data(), A[1].data());
    if (st) return st;
    // exp(T A) of both directions on the device (real Taylor series), then the plan's real matrices
    std::vector<double> E[2];
    cudaStream_t s = nullptr;
    for (int v = 0; v < 2; ++v) {
        const int m = nn[v];
        double *Ad = nullptr, *Ed = nullptr;
        cudaError_t e = cudaMalloc(&Ad, sizeof(double) * size_t(m) * m);
        if (e == cudaSuccess) e = cudaMalloc(&Ed, 2 * sizeof(double) * size_t(m) * m);
        if (e == cudaSuccess) e = cudaMemcpy(Ad, A[v].data(), sizeof(double) * size_t(m) * m, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            st = mm_expm_device(ctx, m, Ad, nullptr, 0.0, T, 0.0, norm1_host(m, A[v].data()), Ed, s);
        std::vector<double> Ec(size_t(2) * m * m);
        if (e == cudaSuccess && !st) e = cudaMemcpy(Ec.data(), Ed, sizeof(double) * Ec.size(), cudaMemcpyDeviceToHost);
        if (Ad) cudaFree(Ad);
        if (Ed) cudaFree(Ed);
        if (st) return st;
        if (e != cudaSuccess) return cuda_fail(e, "pipe-flow exponential");
        E[v].resize(size_t(m) * m);
        for (size_t q = 0; q < E[v].size(); ++q) E[v][q] = Ec[2 * q];
    }
    const int64_t n64[2] = {n_r, n_z};
    const double *Ep[2] = {E[0].data(), E[1].data()};
    return mumode_plan_create(ctx, 2, n64, Ep, 0, MM_R64, prec, nullptr, out);
}
