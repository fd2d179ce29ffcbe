// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <vector>

#include "mumode.h"

namespace mm {

// ---- host set-up (host_setup.cpp) ---------------------------------------
void fd_laplacian_dirichlet(int n, double *A);
bool expm(int n, const double *Are, const double *Aim, std::complex<double> z, std::complex<double> *E);
bool gauss_hermite(int m, double *x, double *W);
void hermite_matrices(int m, const double *x, const double *W, double *fwd, double *bwd);
void hermite_hamiltonian(int m, const double *x, const double *W, const double *V, double *H);
void hermite_galerkin(int m, const double *x, const double *W, const double *U, double *G);

// ---- error reporting (mumode_api.cu) --------------------------------------
mm_status fail(mm_status st, const char *fmt, ...);
void count_launch(int k = 1);

// ---- CUDA-core kernels (simt_kernels.cu) ----------------------------------
// Y[r][i][l] = sum_j L[i][j] X[r][j][l]; i < m, j < n, l < left, r < right.
// `complex_data` selects interleaved complex elements; L has the same
// element type as the data.  fp64 selects double, otherwise float.
cudaError_t simt_mode_product(bool fp64, bool complex_data, int64_t left, int64_t n, int64_t right,
                              int64_t m, const void *L, const void *X, void *Y, cudaStream_t s);
// The same contraction in FP64 on the tensor cores (warp MMA m8n8k4).
cudaError_t dmma_mode_product(bool complex_data, int64_t left, int64_t n, int64_t right, int64_t m, const void *L,
                              const void *X, void *Y, cudaStream_t s);
// psi *= exp(-i tb |psi|^2) for count complex elements.
cudaError_t simt_nonlinear_phase(bool fp64, int64_t count, double tb, void *psi, cudaStream_t s);
// Even/odd folding (inverse: unfolding) of a complex64 tensor with sizes n[0..d-1] (n[0] fastest)
// in the directions of mask (bit v: direction v + 1; at most five of them); in and out are distinct.
// With norm2 (inverse only) the unfold also adds sum |out|^2 w[0][i_1] ... w[d-1][i_d] over its
// outputs to *norm2 in FP64 (w null, or a null table: factor 1).
cudaError_t fold_state(int d, const int64_t *n, unsigned mask, bool inverse, const void *in, void *out, cudaStream_t s,
                       const double *const *w = nullptr, double *norm2 = nullptr);
// g <- adjoint of the nonlinear phase at psi (psi: state before the phase).
cudaError_t simt_nonlinear_adjoint(bool fp64, int64_t count, double tb, const void *psi, void *g, cudaStream_t s);
// out (device double) += sum |u|^2 w, w = w1[i1] w2[i2] w3[i3] if w1 != NULL.
cudaError_t norm2_accumulate(mm_dtype dt, int64_t n1, int64_t n2, int64_t n3, const void *u,
                             const double *w1, const double *w2, const double *w3, double *out,
                             cudaStream_t s);

// ---- tensor-core path (tc_kernels.cu) -------------------------------------
constexpr int kMaxDims = 8;

// Device layout of the split state: pieces[c][p][...] for c in {re, im},
// p < npieces, each plane the padded tensor (sizes np[]) in bf16.
struct TcState {
    int d = 0;
    int64_t n[kMaxDims] = {};   // logical sizes
    int64_t np[kMaxDims] = {};  // padded sizes (multiples of 16)
    int64_t plane = 0;          // elements per plane = prod np
};

// Per-direction matrix in the tensor-core form (device pieces).
struct TcMatrix {
    int64_t n_in = 0, n_out = 0;    // logical sizes (columns, rows)
    int64_t k_pad = 0;              // padded contraction length
    int ni = 0, it = 0;             // number of row tiles, rows per tile
    void *pieces = nullptr;         // [p][tile][k_pad/16][2 blocks (C, S)][it][16], bf16 or fp16
    // The same pieces for the CTA-pair kernel, in two tilings (see TcPairTiles):
    // pair[0] row tiles of at most 64 rows, pair[1] of at most 128.
    struct TcPairTiles {
        // [tile][k_pad/16][rank][p][3 blocks (-S, C, S)][it/2][16], rank r
        // holding rows r it/2 .. of the tile, each block row 32 bytes, stored
        // in the 32-byte swizzled order the MMA reads from shared memory
        void *pieces = nullptr;
        int ni = 0, it = 0;  // row tiles, rows per tile (a multiple of 32)
        int kb_lo[8] = {}, kb_hi[8] = {};  // per row tile (n_out <= 512: at most 8 tiles of 64)
    } pair[2];
    int npieces = 0;
    bool fixed = false;             // MM_PREC_F16X6 pieces
    bool tf32 = false;              // MM_PREC_TF32X3: 4-byte pieces ([..][8 elements] rows), k-blocks of 8
    float *rho = nullptr;           // fixed: power-of-two scale of each row (ni * it floats)
    double row_norm = 0.0;          // max_i sum_j |E_ij|, bounds the growth of one product
    int kb_lo[4] = {}, kb_hi[4] = {};  // per row tile (at most 4 of 128): k-blocks with a nonzero piece
};

// Device words that carry the state scale of MM_PREC_F16X6 through a sweep.
struct TcScales {
    const float *s_in = nullptr;          // scale of the input pieces
    float *s_out = nullptr;               // written: scale chosen for the output pieces
    const unsigned *max_prev = nullptr;   // max |output| of the previous sweep (float bits) or a bound
    unsigned *max_cur = nullptr;          // atomicMax of |output| (float bits), zero before the launch
    unsigned *zero_next = nullptr;        // if set: a word the kernel clears for the next launch's max_cur
};

// Kernel of a tensor-core product: the CTA-pair kernel with row tiles of at
// most 64 (two accumulator sets) or 128 rows (one set), or the one-SM kernel.
// kTcChain: the CTA-pair kernel with row tiles of at most 64, a whole call's products in one
// persistent launch (Tucker steps with F16X6; elsewhere it launches like kTcPair64).
enum TcVariant { kTcPair64 = 0, kTcPair128 = 1, kTcOneSM = 2, kTcChain = 3, kTcVariants = 4 };
// The variant a plan starts with: kTcPair64, or what the environment forces
// (MM_TC_1SM set to other than 0: kTcOneSM; MM_PAIR_TILE=128: kTcPair128).
TcVariant tc_default_variant();
// Whether a product with M runs on the CTA-pair kernel in this variant (else the one-SM kernel).
bool tc_pair_ready(const TcMatrix &M, TcVariant variant);

int tc_pieces(mm_prec p);
bool tc_prec(mm_prec p);
bool tc_fixed(mm_prec p);
bool tc_tf32(mm_prec p);       // MM_PREC_TF32X3: 4-byte pieces, k-blocks of 8, the one-SM kernel only
int tc_piece_bytes(mm_prec p);  // bytes of one piece element (2, or 4 for TF32)
// Build the pieces of an m x n complex matrix (interleaved FP64, row-major); tf32: two TF32
// pieces (npieces 2, not fixed), one-SM layout only.
mm_status tc_matrix_create(const double *E, int64_t m, int64_t n, int npieces, bool fixed, TcMatrix *out,
                           bool tf32 = false);
void tc_matrix_destroy(TcMatrix *M);
// Rewrite the pieces (all layouts) and row scales of M from a device
// matrix E (n_out x n_in complex FP64, row-major), in stream order.  The
// k-block bands are not touched: call tc_matrix_full_bands once first.
// With only_for set, only the layout that variant's products read is written (the others are
// then stale until the next full update); the row scales always are.
cudaError_t tc_matrix_update(TcMatrix &M, const double2 *E, cudaStream_t s, const TcVariant *only_for = nullptr);
void tc_matrix_full_bands(TcMatrix &M);
// Device FP64 matrix exponential E = exp(z (A + f B)) (expm_device.cu).
struct ExpmWorkspace {
    int n = 0;
    void *blas = nullptr;            // cublasHandle_t
    double2 *buf[6] = {};            // n x n complex each
    double *sums = nullptr;          // n column sums
};
cudaError_t expm_workspace_init(ExpmWorkspace *w, int n);
void expm_workspace_destroy(ExpmWorkspace *w);
// ||A + f B||_1 (max column sum), computed on the device; synchronises s.
cudaError_t expm_norm1_device(ExpmWorkspace *w, int n, const double *A, const double *B, double f, double *norm,
                              cudaStream_t s);
// norm_bound >= ||A + f B||_1; B may be null.  E (n x n complex) must not be a workspace buffer.
cudaError_t expm_device(ExpmWorkspace *w, int n, const double *A, const double *B, double f, double zr, double zi,
                        double norm_bound, double2 *E, cudaStream_t s);
// exp(i w (A + f_k B)) = cos + i sin for real A, B and count values f_k (host
// array), in real arithmetic, batched: E holds count n x n complex matrices.
// With count > 1 the f values are copied to the device in stream order (the
// host array must stay valid until that copy has run); a single f is passed
// by value.
struct ExpmBatch {
    int n = 0, cap = 0;
    double *buf[8] = {};     // cap real n x n matrices each
    double *f = nullptr;     // cap doubles
};
cudaError_t expm_batch_init(ExpmBatch *w, int n, int cap);
void expm_batch_destroy(ExpmBatch *w);
int expm_batch_capacity(int n);  // batch entries that keep the workspace near 1 GB (1..64)
// Interpolation of exp(z (A + f B)) in f: the exponentials at K <= kInterpNodes Chebyshev nodes
// of a range of f (nodes[j], n x n complex each) and, for cnt values f_k, weights W[k][j] (the
// Lagrange basis at f_k, device, cnt x K) give E_k = sum_j W[k][j] nodes[j].
constexpr int kInterpNodes = 12;
cudaError_t combine_interp_nodes(int n, int cnt, int K, const double *W_dev, const double2 *nodes, double2 *E,
                                 cudaStream_t s);
// mu: a diagonal shift taken out as the phase exp(i w mu); norm_bound then bounds ||A + f_k B - mu I||_1.
// theta: the largest scaled norm ||X||_1 the series may see.  1 gives full FP64 accuracy
// (truncation below 1e-19); 2 bounds the truncation by 2^20 / 20! < 5e-13, enough for matrices
// that are split into tensor-core pieces (about 2^-34 of a row's scale), with one doubling fewer.
cudaError_t expm_imag_batched(ExpmBatch *w, int n, const double *A, const double *B, const double *f_host, int count,
                              double wim, double norm_bound, double2 *E, cudaStream_t s, double mu = 0.0,
                              double theta = 1.0);
// HKP propagator of one direction on the device: M = Psi exp(-i tau H) Phi^W,
// H = diag(k + 1/2) + P^T GP (GP = diag(g) P, NULL for the harmonic case),
// P[l][k] = phi_k(x_l), fwd = Phi^W (host, m x m row-major).  Both workspaces
// must hold m x m matrices; synchronises the stream once (norm of H).
cudaError_t hkp_propagator_device(ExpmWorkspace *wz, ExpmBatch *wb, int m, const double *P_host, const double *GP_host,
                                  const double *fwd_host, double tau, double2 *M, cudaStream_t s);
// exp(z (A + f B)) for real z, Taylor series in real arithmetic; E complex with zero imaginary parts.
cudaError_t expm_real_device(ExpmBatch *w, int n, const double *A, const double *B, double f, double z,
                             double norm_bound, double2 *E, cudaStream_t s);
// Pipe-flow operators (host_setup.cpp)
void pipe_radial(int n, double rmin, double rmax, double alpha, double *A);
void pipe_axial(int n, double zmax, double alpha, const double *s, double *A);
// Host half of tc_matrix_create: geometry (pieces/rho left null) and the
// host images of the pieces and row scales.
mm_status tc_matrix_host(const double *E, int64_t m, int64_t n, int npieces, bool fixed, TcMatrix *geom,
                         std::vector<uint16_t> &pieces, std::vector<float> &rho, bool tf32 = false);
// Split an interleaved complex64 tensor into padded piece planes.  For the
// fixed-point mode the scale comes from the tensor's maximum: `work` (one
// unsigned, device) receives it, `scale_out` the chosen scale, and
// bound_words[q] = max * bounds[q] (float bits) for the first sweep.
cudaError_t tc_split(const TcState &st, int npieces, bool fixed, const void *u_c64, void *pieces, unsigned *work,
                     float *scale_out, unsigned *bound_words, const double *bounds, int nbounds, cudaStream_t s);
// The TF32 forms: two 4-byte pieces per plane element (x0 = TF32 of x, x1 = TF32 of x - x0).
cudaError_t tc_split_tf32(const TcState &st, const void *u_c64, void *pieces, cudaStream_t s);
// The GPE nonlinear phase psi exp(-i tb |psi|^2) on an F16X6 piece state folded in the directions of
// mask (at most five): unfold, phase, fold per orbit; input and output scale 2^grid_exponent(*max_in),
// written to *s_out; values past the split's range set MM_ERR_RANGE in *err; in and out distinct.
cudaError_t tc_phase_fold(const TcState &st, unsigned mask, const void *in_pieces, void *out_pieces,
                          const unsigned *max_in, float *s_out, double tb, int *err, cudaStream_t s);
cudaError_t tc_merge_tf32(const TcState &st, const void *pieces, void *u_c64, cudaStream_t s);
// Sum the piece planes back into an interleaved complex64 tensor
// (fixed-point mode: times *scale).
cudaError_t tc_merge(const TcState &st, int npieces, bool fixed, const void *pieces, const float *scale, void *u_c64,
                     cudaStream_t s);

// One problem of a tensor-core launch: its two tensor maps (64-byte
// aligned, as TMA requires of a tensor map in memory) and its sizes,
// buffers and scales.  Built by tc_problem_build.
struct TcProblem {  // the CUtensorMap members carry the 64-byte alignment TMA needs
    CUtensorMap mapX;       // split input state
    CUtensorMap mapE;       // matrix pieces
    int64_t left, right;    // padded sizes of the fast / slow index groups
    int64_t mp;             // padded output length
    int64_t aps;            // 64-point atoms per slab (MN-major)
    int64_t plane_out;      // elements per output plane
    int64_t pairs_begin;    // first work item of this problem in a batched launch
    int64_t pairs;          // work items: (pair of point tiles, row tile)
    int it, ni, kblocks, tx_bytes;
    int kb_lo[4], kb_hi[4];  // per row tile: k-blocks with a nonzero matrix piece
    uint16_t *out;
    const float *rho;       // fixed-point row scales
    TcScales sc;
    unsigned *zero_word;    // batched launches: a max word to clear at kernel start
};

struct TcEpilogue {
    // 0: store pieces, 1: nonlinear phase then store pieces, 2: point phase then store; 3: as 1,
    // and the value before the phase goes to mid_out; 4: the adjoint of that phase at the state in
    // mid_in (3 and 4: CTA-pair kernel, F16X6; mid buffers complex64 in the padded layout of one
    // piece plane of the output); 5: store, and the weighted norm of the output (below)
    int kind = 0;
    double tb = 0.0;   // tau * beta for kinds 1, 3, 4
    float2 *mid_out = nullptr;
    const float2 *mid_in = nullptr;
    // kind 2 (CTA-pair kernel with row tiles of at most 64): every output at point (l, r) (the
    // non-contracted index groups left and right of the direction) is multiplied by
    // pl0[l % ldiv] pl1[l / ldiv] pr0[r % rdiv] pr1[r / rdiv] (device tables, null: factor 1)
    const double2 *pl0 = nullptr, *pl1 = nullptr, *pr0 = nullptr, *pr1 = nullptr;
    int64_t ldiv = 1, rdiv = 1;
    // kind 5 (CTA-pair kernel with row tiles of at most 64, F16X6): plain store, and the launch
    // adds sum |y|^2 wl0[l % ldiv] wl1[l / ldiv] wr0[r % rdiv] wr1[r / rdiv] wo[i] over its outputs
    // y (point (l, r), output index i) to *norm2 in FP64 (real device tables, null: factor 1; wo
    // zero from the direction's length to its padded length)
    const double *wl0 = nullptr, *wl1 = nullptr, *wr0 = nullptr, *wr1 = nullptr, *wo = nullptr;
    double *norm2 = nullptr;
};
// One mu-mode product on the split state: in (sizes st_in) -> out (sizes
// st_out, equal except direction mu which becomes M.n_out).
// The variant falls back to the one-SM kernel where M lacks its tiling.
cudaError_t tc_mode_product(const TcState &st_in, const TcState &st_out, int mu, const TcMatrix &M,
                            mm_prec prec, const void *in_pieces, void *out_pieces,
                            const TcEpilogue &epi, const TcScales &sc, int *d_err, cudaStream_t s,
                            TcVariant variant = kTcPair64);
// Batched launches of the CTA-pair kernel: one record per problem (opaque,
// tc_pair_record_bytes() bytes, tc_pair_record_align() aligned), built for one direction,
// with its first work item set by tc_pair_record_set_begin (records in order,
// the first at 0).  cudaErrorNotSupported: the product has no pair tiling
// with row tiles of at most 64 (use tc_mode_product_batched).
size_t tc_pair_record_bytes();
size_t tc_pair_record_align();
// chain_pos < 0: a record of a batched launch; >= 0: the product's position in a chain (the
// single launch's stage layout, F16X6 only).
cudaError_t tc_pair_record_build(const TcState &si, const TcState &so, int mu, const TcMatrix &M, mm_prec prec,
                                 const void *in_pieces, void *out_pieces, const TcScales &sc, void *rec, bool *kmajor,
                                 int64_t *items, int chain_pos = -1);
// The dependencies of a chain's records (positions 0 .. nprod - 1 of sweeps over d directions):
// slab-group completion targets, row-tile-major items in the last direction, the product each
// must wait for before its first load, and s_in_max[k], the maximum word whose grid exponent is
// product k's input scale (null: its s_in word).
cudaError_t tc_pair_chain_plan(void *host_recs, int nprod, int d, const unsigned *const *s_in_max);
constexpr int kChainCounters = 33;  // words per product: its total, then its 32 slab groups
// One persistent launch over a chain of products (records built with chain positions 0, 1, ..,
// nprod - 1, their first items set in order, then tc_pair_chain_plan); `done`: nprod counters and
// `gcnt`: nprod x 32 slab-group counters, all zero at the launch.
cudaError_t tc_pair_chain_launch(const void *host_recs, const void *dev_recs, int nprod, unsigned *done,
                                 unsigned *gcnt, int *d_err, cudaStream_t s);
int tc_chain_ctas();  // the most CTAs a chained launch uses (the SM count)
void tc_pair_record_set_begin(void *rec, int64_t begin);
bool tc_pair_batch_compatible(const void *host_recs, int nprob);  // same row tile size in all records
cudaError_t tc_pair_batch_launch(const void *host_recs, const void *dev_recs, int nprob, bool kmajor, mm_prec prec,
                                 int *d_err, cudaStream_t s);
// Tensor-core flops (2 M N K per MMA) one product issues, padding and the
// skipped zero blocks included.
double tc_issued_flops(const TcState &st_in, int mu, const TcMatrix &M, mm_prec prec,
                       TcVariant variant = kTcPair64);
// The record of one such product, for a batched launch (kmajor: direction 1).
cudaError_t tc_problem_build(const TcState &st_in, const TcState &st_out, int mu, const TcMatrix &M, mm_prec prec,
                             const void *in_pieces, void *out_pieces, const TcScales &sc, TcProblem *pr, bool *kmajor);
// One launch over many problems (same direction kind and precision); the
// records are in device memory (dev_probs) with a host copy (host_probs),
// pairs_begin set to the running sum of pairs.
cudaError_t tc_mode_product_batched(const TcProblem *host_probs, const TcProblem *dev_probs, int nprob, bool kmajor,
                                    mm_prec prec, const TcEpilogue &epi, int *d_err, cudaStream_t s);

}  // namespace mm
