/*
 * FP64 CPU oracle for the mu-mode integrator (Caliari, Cassini, Einkemmer,
 * Ostermann, Zivcovich, "A mu-mode integrator for solving evolution equations
 * in Kronecker form", arXiv 2103.01691).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this file.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py load it, to check the CUDA path.
 *
 * Every routine is the plain definition (or the paper's algorithm, step by
 * step) written as straightforward loops in double / double complex.  There
 * is no blocking, fusion or reordering beyond what the definition states,
 * so each function can be checked against the paper by eye.
 *
 * Layout convention (paper section 4.1, after eq. (exactsol)): a tensor
 * U(i_1,...,i_d) is stored with i_1 fastest, offset
 * i_1 + n_1 (i_2 + n_2 (i_3 + ...)), all indices 0-based here.
 * Matrices are row-major: M[i*ncols + j].
 *
 * Pins (tests/test_oracle_*.py): dense expm of the full Kronecker sum,
 * scipy expm, closed-form sine-mode decay, mode-order independence, norm
 * conservation, the printed heat errors of section 4.1 and section 5.1,
 * numpy's Gauss-Hermite rule, discrete orthonormality, exact harmonic
 * oscillator phases, Strang reversibility and finite differences of the
 * adjoint.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------
 * One-dimensional operators A_mu (section 2, eq. (tensor-structure); the
 * heat problem of section 4.1 uses centered second-order differences).
 * ---------------------------------------------------------------------- */

/* Centered second-order FD Laplacian with homogeneous Dirichlet conditions
 * on (0,1): interior nodes x_j = j h, j = 1..n, h = 1/(n+1),
 * A = h^-2 tridiag(1, -2, 1). */
void or_fd_dirichlet(int n, double *A)
{
    double h = 1.0 / (n + 1);
    double s = 1.0 / (h * h);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            if (i == j) v = -2.0 * s;
            else if (i - j == 1 || j - i == 1) v = s;
            A[(size_t)i * n + j] = v;
        }
}

/* Centered second-order FD Laplacian on a periodic grid of n points over an
 * interval of given length, h = length / n (section 4.1, eq. (he)). */
void or_fd_periodic(int n, double length, double *A)
{
    double h = length / n;
    double s = 1.0 / (h * h);
    memset(A, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        A[(size_t)i * n + i] = -2.0 * s;
        A[(size_t)i * n + (i + 1) % n] += s;
        A[(size_t)i * n + (i + n - 1) % n] += s;
    }
}

/* ------------------------------------------------------------------------
 * One-dimensional exponentials E_mu = exp(z A_mu) (section 2: "d small
 * exponentials of sizes n_mu x n_mu").  The paper uses MATLAB's expm
 * (section 4 intro).  The oracle uses two methods of its own:
 * ---------------------------------------------------------------------- */

/* (a) Closed form for the Dirichlet FD Laplacian: it is diagonalised by the
 * orthogonal, symmetric sine matrix V_jk = sqrt(2/(n+1)) sin(j k pi/(n+1))
 * (j,k = 1..n) with eigenvalues lambda_k = -(4/h^2) sin^2(k pi / (2(n+1))),
 * so exp(zA) = V diag(exp(z lambda_k)) V.  z = zr + i zi; E is complex. */
void or_expm_dirichlet_fd(int n, double zr, double zi, cplx *E)
{
    double h = 1.0 / (n + 1);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * n);
    cplx *f = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    double c = sqrt(2.0 / (n + 1));
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k)
            V[(size_t)j * n + k] = c * sin((double)(j + 1) * (k + 1) * M_PI / (n + 1));
    for (int k = 0; k < n; ++k) {
        double s = sin((k + 1) * M_PI / (2.0 * (n + 1)));
        double lam = -4.0 * s * s / (h * h);
        f[k] = cexp((zr + I * zi) * lam);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx acc = 0;
            for (int k = 0; k < n; ++k)
                acc += V[(size_t)i * n + k] * f[k] * V[(size_t)k * n + j];
            E[(size_t)i * n + j] = acc;
        }
    free(V);
    free(f);
}

static void cmatmul(int n, const cplx *A, const cplx *B, cplx *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx acc = 0;
            for (int k = 0; k < n; ++k)
                acc += A[(size_t)i * n + k] * B[(size_t)k * n + j];
            C[(size_t)i * n + j] = acc;
        }
}

/* (b) General matrices: truncated Taylor series with scaling and squaring.
 * X = zA / 2^s with ||X||_1 <= 1/2, exp(X) ~ sum_{k<=30} X^k/k! (terms stop
 * once they fall below 1e-18 relative), then square s times.  A is complex
 * (A_re + i A_im; A_im may be NULL). */
void or_expm_taylor(int n, const double *Are, const double *Aim, double zr, double zi, cplx *E)
{
    size_t nn = (size_t)n * n;
    cplx *X = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *T = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *W = (cplx *)malloc(sizeof(cplx) * nn);
    cplx z = zr + I * zi;
    for (size_t q = 0; q < nn; ++q) X[q] = z * (Are[q] + (Aim ? I * Aim[q] : 0));
    double norm1 = 0;
    for (int j = 0; j < n; ++j) {
        double col = 0;
        for (int i = 0; i < n; ++i) col += cabs(X[(size_t)i * n + j]);
        if (col > norm1) norm1 = col;
    }
    int s = 0;
    while (norm1 > 0.5) { norm1 *= 0.5; ++s; }
    double scale = ldexp(1.0, -s);
    for (size_t q = 0; q < nn; ++q) X[q] *= scale;
    /* E = I, T = I; T <- T X / k; E += T */
    for (size_t q = 0; q < nn; ++q) { E[q] = 0; T[q] = 0; }
    for (int i = 0; i < n; ++i) { E[(size_t)i * n + i] = 1; T[(size_t)i * n + i] = 1; }
    for (int k = 1; k <= 30; ++k) {
        cmatmul(n, T, X, W);
        double tn = 0, en = 0;
        for (size_t q = 0; q < nn; ++q) {
            T[q] = W[q] / k;
            E[q] += T[q];
            tn += cabs(T[q]);
            en += cabs(E[q]);
        }
        if (tn <= 1e-18 * en) break;
    }
    for (int q = 0; q < s; ++q) {
        cmatmul(n, E, E, W);
        memcpy(E, W, sizeof(cplx) * nn);
    }
    free(X);
    free(T);
    free(W);
}

/* ------------------------------------------------------------------------
 * mu-mode product, Definition 2.1 (section 2):
 *   S(i_1..i_{mu-1}, i, i_{mu+1}..i_d) = sum_j L_{ij} U(i_1..j..i_d),
 * L is m x n_mu (row-major), S has n_mu replaced by m.  mu is 1-based.
 * With left = n_1...n_{mu-1} and right = n_{mu+1}...n_d, U is viewed as
 * U[r][j][l] (l fastest) and S as S[r][i][l].
 * ---------------------------------------------------------------------- */
void or_mode_product(int d, const int64_t *n, int mu, int64_t m, const cplx *L,
                     const cplx *U, cplx *S)
{
    int64_t left = 1, right = 1, nmu = n[mu - 1];
    for (int v = 0; v < mu - 1; ++v) left *= n[v];
    for (int v = mu; v < d; ++v) right *= n[v];
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t r = 0; r < right; ++r)
        for (int64_t i = 0; i < m; ++i) {
            cplx *srow = S + (r * m + i) * left;
            for (int64_t l = 0; l < left; ++l) srow[l] = 0;
            for (int64_t j = 0; j < nmu; ++j) {
                cplx lij = L[i * nmu + j];
                const cplx *urow = U + (r * nmu + j) * left;
                for (int64_t l = 0; l < left; ++l) srow[l] += lij * urow[l];
            }
        }
}

/* Tucker operator U x_{o_1} E_{o_1} x ... x_{o_d} E_{o_d} (section 2,
 * eq. (dd-tensor) and the Tucker form after Definition 2.1).  E[v] is the
 * n_{v+1} x n_{v+1} matrix for direction v+1; order lists the directions
 * (1-based) in application order, NULL means 1, 2, ..., d.  nsteps repeats
 * the whole operator (a marching scheme with constant step, section 2). */
void or_tucker(int d, const int64_t *n, const cplx *const *E, const int *order,
               int64_t nsteps, const cplx *U, cplx *out)
{
    int64_t N = 1;
    for (int v = 0; v < d; ++v) N *= n[v];
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    memcpy(out, U, sizeof(cplx) * (size_t)N);
    for (int64_t s = 0; s < nsteps; ++s)
        for (int q = 0; q < d; ++q) {
            int mu = order ? order[q] : q + 1;
            or_mode_product(d, n, mu, n[mu - 1], E[mu - 1], out, tmp);
            memcpy(out, tmp, sizeof(cplx) * (size_t)N);
        }
    free(tmp);
}

/* Single entries of U x_1 E_1 x_2 E_2 x_3 E_3 for d = 3, straight from the
 * definition: S(i1,i2,i3) = sum_{j1,j2,j3} E1[i1,j1] E2[i2,j2] E3[i3,j3]
 * U(j1,j2,j3).  Used at sizes where the full tensor is too costly.
 * idx holds npts triples (i1,i2,i3), 0-based. */
void or_tucker3_entries(const int64_t *n, const cplx *E1, const cplx *E2, const cplx *E3,
                        const cplx *U, int64_t npts, const int64_t *idx, cplx *out)
{
    int64_t n1 = n[0], n2 = n[1], n3 = n[2];
#pragma omp parallel for schedule(dynamic)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t i1 = idx[3 * p], i2 = idx[3 * p + 1], i3 = idx[3 * p + 2];
        cplx total = 0;
        for (int64_t j3 = 0; j3 < n3; ++j3) {
            cplx s2 = 0;
            for (int64_t j2 = 0; j2 < n2; ++j2) {
                const cplx *fiber = U + (j3 * n2 + j2) * n1;
                cplx s1 = 0;
                for (int64_t j1 = 0; j1 < n1; ++j1) s1 += E1[i1 * n1 + j1] * fiber[j1];
                s2 += E2[i2 * n2 + j2] * s1;
            }
            total += E3[i3 * n3 + j3] * s2;
        }
        out[p] = total;
    }
}

/* ------------------------------------------------------------------------
 * Hermite functions and Gauss-Hermite quadrature (section 3).
 * phi_k(x) = H_k(x) exp(-x^2/2) with H_k orthonormal w.r.t. exp(-x^2), so
 * the phi_k are orthonormal in L^2(R).  They satisfy the normalised
 * three-term recurrence
 *   phi_0 = pi^{-1/4} e^{-x^2/2},  phi_1 = sqrt(2) x phi_0,
 *   phi_{k+1} = sqrt(2/(k+1)) x phi_k - sqrt(k/(k+1)) phi_{k-1},
 * and phi_k' = sqrt(2k) phi_{k-1} - x phi_k.
 * ---------------------------------------------------------------------- */

/* phi_0..phi_{count-1} at one point x. */
static void hermite_column(int count, double x, double *out)
{
    double p0 = pow(M_PI, -0.25) * exp(-0.5 * x * x);
    out[0] = p0;
    if (count == 1) return;
    double p1 = sqrt(2.0) * x * p0;
    out[1] = p1;
    for (int k = 1; k + 1 < count; ++k) {
        double p2 = sqrt(2.0 / (k + 1)) * x * p1 - sqrt((double)k / (k + 1)) * p0;
        out[k + 1] = p2;
        p0 = p1;
        p1 = p2;
    }
}

/* H[k*npts + l] = phi_k(x_l), k < nfun. */
void or_hermite_functions(int nfun, int npts, const double *x, double *H)
{
    double *col = (double *)malloc(sizeof(double) * nfun);
    for (int l = 0; l < npts; ++l) {
        hermite_column(nfun, x[l], col);
        for (int k = 0; k < nfun; ++k) H[(size_t)k * npts + l] = col[k];
    }
    free(col);
}

/* Gauss-Hermite rule with m nodes: the zeros of phi_m, found by Newton's
 * method on the recurrence above, started from the classical asymptotic
 * guesses for the largest zeros (Stroud and Secrest; the same start values
 * appear in Numerical Recipes' Gauss-Hermite routine) and extrapolated
 * from the previous two zeros further in.  Outputs, ascending in x:
 *   x[l]  nodes,
 *   W[l]  weights for integrals of plain functions, sum_l W_l f(x_l) ~
 *         int f dx, obtained from the Christoffel function,
 *         W_l = 1 / sum_{k<m} phi_k(x_l)^2,
 *   w[l]  weights for exp(-x^2), w_l = W_l exp(-x_l^2) (may underflow).
 * Returns 0 on success, -1 if some Newton iteration did not converge. */
int or_gauss_hermite(int m, double *x, double *w, double *W)
{
    double *col = (double *)malloc(sizeof(double) * (m + 1));
    int half = (m + 1) / 2, status = 0;
    double z = 0, z1 = 0;
    double *pos = (double *)malloc(sizeof(double) * half);
    for (int i = 0; i < half; ++i) {
        /* guesses for the i-th largest zero */
        if (i == 0) z = sqrt(2.0 * m + 1) - 1.85575 * pow(2.0 * m + 1, -0.16667);
        else if (i == 1) z = z - 1.14 * pow((double)m, 0.426) / z;
        else if (i == 2) z = 1.86 * z - 0.86 * pos[0];
        else if (i == 3) z = 1.91 * z - 0.91 * pos[1];
        else z = 2.0 * z - pos[i - 2];
        int it;
        for (it = 0; it < 100; ++it) {
            hermite_column(m + 1, z, col);
            double pm = col[m], dpm = sqrt(2.0 * m) * col[m - 1] - z * col[m];
            z1 = z;
            z = z1 - pm / dpm;
            if (fabs(z - z1) <= 1e-15 * fmax(1.0, fabs(z))) break;
        }
        if (it == 100) status = -1;
        pos[i] = z;
    }
    for (int i = 0; i < half; ++i) {
        x[m - 1 - i] = pos[i];
        x[i] = -pos[i];
    }
    if (m % 2 == 1) x[m / 2] = 0.0;
    for (int l = 0; l < m; ++l) {
        hermite_column(m, x[l], col);
        double s = 0;
        for (int k = 0; k < m; ++k) s += col[k] * col[k];
        W[l] = 1.0 / s;
        w[l] = W[l] * exp(-x[l] * x[l]);
    }
    free(pos);
    free(col);
    return status;
}

/* ------------------------------------------------------------------------
 * Harmonic oscillator in a Hermite basis (section 3 eqs. (real2spec),
 * (spec2real); section 4.3, the HKP method, with the harmonic potential
 * x^2/2 in every direction so that the Hamiltonian is diagonal).
 * d = 3, m nodes per direction.  Phi_W[k][l] = phi_k(x_l) W_l is the
 * forward (values -> coefficients) matrix with the weights folded in,
 * Psi[l][k] = phi_k(x_l) the backward matrix (Psi = Phi^*, section 3).
 * The eigenvalues are lambda_k = sum_mu (1/2 + k_mu) (section 3).
 * ---------------------------------------------------------------------- */

typedef struct {
    int m;
    cplx *fwd; /* m x m, Phi_W */
    cplx *bwd; /* m x m, Psi */
} ho_basis;

static void ho_basis_make(int m, const double *x, const double *W, ho_basis *b)
{
    b->m = m;
    b->fwd = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    b->bwd = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    double *H = (double *)malloc(sizeof(double) * (size_t)m * m);
    or_hermite_functions(m, m, x, H);
    for (int k = 0; k < m; ++k)
        for (int l = 0; l < m; ++l) {
            b->fwd[(size_t)k * m + l] = H[(size_t)k * m + l] * W[l];
            b->bwd[(size_t)l * m + k] = H[(size_t)k * m + l];
        }
    free(H);
}

static void ho_basis_free(ho_basis *b)
{
    free(b->fwd);
    free(b->bwd);
}

/* values -> coefficients, eq. (real2spec) with F_W = f w folded into Phi_W */
void or_hermite_forward(int m, const double *x, const double *W, const cplx *vals, cplx *coef)
{
    ho_basis b;
    ho_basis_make(m, x, W, &b);
    int64_t n[3] = {m, m, m};
    const cplx *E[3] = {b.fwd, b.fwd, b.fwd};
    or_tucker(3, n, E, NULL, 1, vals, coef);
    ho_basis_free(&b);
}

/* coefficients -> values at the nodes, eq. (spec2real) with Psi = Phi^* */
void or_hermite_backward(int m, const double *x, const double *W, const cplx *coef, cplx *vals)
{
    ho_basis b;
    ho_basis_make(m, x, W, &b);
    int64_t n[3] = {m, m, m};
    const cplx *E[3] = {b.bwd, b.bwd, b.bwd};
    or_tucker(3, n, E, NULL, 1, coef, vals);
    ho_basis_free(&b);
}

/* c(k1,k2,k3) *= exp(-i s (k1 + k2 + k3 + 3/2)): the exact flow of the
 * diagonal Hamiltonian over time s. */
static void ho_phase(int m, double s, cplx *c)
{
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m; ++k3)
        for (int k2 = 0; k2 < m; ++k2)
            for (int k1 = 0; k1 < m; ++k1)
                c[((size_t)k3 * m + k2) * m + k1] *= cexp(-I * s * (k1 + k2 + k3 + 1.5));
}

/* Linear flow over time s: forward, exact phase, backward. */
static void ho_linear(const ho_basis *b, double s, cplx *psi, cplx *tmp)
{
    int m = b->m;
    int64_t n[3] = {m, m, m};
    const cplx *F[3] = {b->fwd, b->fwd, b->fwd};
    const cplx *B[3] = {b->bwd, b->bwd, b->bwd};
    or_tucker(3, n, F, NULL, 1, psi, tmp);
    ho_phase(m, s, tmp);
    or_tucker(3, n, B, NULL, 1, tmp, psi);
}

/* nsteps steps of the HKP scheme for i psi_t = -1/2 Lap psi + |x|^2/2 psi. */
void or_ho_steps(int m, const double *x, const double *W, double tau, int64_t nsteps, cplx *psi)
{
    ho_basis b;
    ho_basis_make(m, x, W, &b);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)m * m * m);
    for (int64_t s = 0; s < nsteps; ++s) ho_linear(&b, tau, psi, tmp);
    free(tmp);
    ho_basis_free(&b);
}

/* ------------------------------------------------------------------------
 * Gross-Pitaevskii equation with a harmonic trap,
 *   i psi_t = -1/2 Lap psi + |x|^2/2 psi + beta |psi|^2 psi,
 * Strang splitting (section 4.5): a linear half step by the mu-mode
 * integrator, the nonlinear subflow solved exactly
 * (|psi| is constant along it, so psi <- psi exp(-i tau beta |psi|^2)),
 * another linear half step.  Applied literally, with no merging of
 * adjacent half steps.
 * ---------------------------------------------------------------------- */
static void gpe_nonlinear(int64_t N, double tb, cplx *psi)
{
#pragma omp parallel for
    for (int64_t q = 0; q < N; ++q) {
        double a2 = creal(psi[q]) * creal(psi[q]) + cimag(psi[q]) * cimag(psi[q]);
        psi[q] *= cexp(-I * tb * a2);
    }
}

void or_gpe_steps(int m, const double *x, const double *W, double beta, double tau,
                  int64_t nsteps, cplx *psi)
{
    ho_basis b;
    ho_basis_make(m, x, W, &b);
    int64_t N = (int64_t)m * m * m;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    for (int64_t s = 0; s < nsteps; ++s) {
        ho_linear(&b, 0.5 * tau, psi, tmp);
        gpe_nonlinear(N, tau * beta, psi);
        ho_linear(&b, 0.5 * tau, psi, tmp);
    }
    free(tmp);
    ho_basis_free(&b);
}

/* Adjoint of the Strang scheme (not in the paper; reverse-mode derivative
 * of a real loss J(psi_T)).  Convention: g = dJ/dRe + i dJ/dIm, so that
 * dJ = Re <g, delta>.  psi0 is the initial state, gT the gradient at the
 * final state; on return g0 holds the gradient at psi0.
 *  - linear, complex-linear map L:  g <- L^H g
 *    (L = B P F with F = x_mu Phi_W, P = diag phase, B = x_mu Psi, so
 *     L^H = F^H P^H B^H: mode products with Psi^H = Phi^T-shaped real
 *     matrices, the conjugate phase, then Phi_W^H);
 *  - nonlinear psi' = psi e^{-i theta}, theta = tau beta |psi|^2:
 *    g = e^{i theta} g' + 2 tau beta Im(conj(g') psi') psi.
 * Forward states are recomputed from psi0 (no checkpointing here). */
void or_gpe_adjoint(int m, const double *x, const double *W, double beta, double tau,
                    int64_t nsteps, const cplx *psi0, const cplx *gT, cplx *g0)
{
    ho_basis b;
    ho_basis_make(m, x, W, &b);
    int64_t N = (int64_t)m * m * m;
    size_t bytes = sizeof(cplx) * (size_t)N;
    /* stored states before the nonlinear stage of every step */
    cplx *mid = (cplx *)malloc(bytes * (size_t)(nsteps > 0 ? nsteps : 1));
    cplx *psi = (cplx *)malloc(bytes);
    cplx *tmp = (cplx *)malloc(bytes);
    memcpy(psi, psi0, bytes);
    for (int64_t s = 0; s < nsteps; ++s) {
        ho_linear(&b, 0.5 * tau, psi, tmp);
        memcpy(mid + s * N, psi, bytes);
        gpe_nonlinear(N, tau * beta, psi);
        ho_linear(&b, 0.5 * tau, psi, tmp);
    }
    /* adjoint matrices: fwd^H and bwd^H (real, so transposes) */
    cplx *fH = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    cplx *bH = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            fH[(size_t)i * m + j] = conj(b.fwd[(size_t)j * m + i]);
            bH[(size_t)i * m + j] = conj(b.bwd[(size_t)j * m + i]);
        }
    int64_t n[3] = {m, m, m};
    const cplx *FH[3] = {fH, fH, fH};
    const cplx *BH[3] = {bH, bH, bH};
    cplx *g = g0;
    memcpy(g, gT, bytes);
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        /* second linear half step: g <- F^H P^H B^H g */
        or_tucker(3, n, BH, NULL, 1, g, tmp);
        ho_phase(m, -0.5 * tau, tmp);
        or_tucker(3, n, FH, NULL, 1, tmp, g);
        /* nonlinear stage */
        const cplx *pin = mid + s * N;
        double tb = tau * beta;
        for (int64_t q = 0; q < N; ++q) {
            double a2 = creal(pin[q]) * creal(pin[q]) + cimag(pin[q]) * cimag(pin[q]);
            cplx e = cexp(I * tb * a2);
            cplx pout = pin[q] / e;
            double im = cimag(conj(g[q]) * pout);
            g[q] = e * g[q] + 2.0 * tb * im * pin[q];
        }
        /* first linear half step */
        or_tucker(3, n, BH, NULL, 1, g, tmp);
        ho_phase(m, -0.5 * tau, tmp);
        or_tucker(3, n, FH, NULL, 1, tmp, g);
    }
    free(fH);
    free(bH);
    free(mid);
    free(psi);
    free(tmp);
    ho_basis_free(&b);
}

/* ------------------------------------------------------------------------
 * Hermite Kronecker pseudospectral method (HKP, section 4.3) for a
 * potential in Kronecker form, V(x) = V_1(x_1) + V_2(x_2) + V_3(x_3), in
 * i psi_t = -1/2 Lap psi + V psi.
 *
 * Reading of section 4.3 (the paper gives no formula for the matrices):
 * each direction's Hamiltonian -1/2 d^2/dx^2 + V_mu is split as the
 * harmonic part -1/2 d^2/dx^2 + x^2/2, diagonal in the Hermite functions
 * with eigenvalues k + 1/2 (section 3), plus the multiplication by
 * V_mu - x^2/2, whose Galerkin matrix is taken by the Gauss-Hermite
 * quadrature of eq. (quadrature):
 *   H[j][k] = (k + 1/2) delta_jk + sum_l W_l phi_j(x_l) (V(x_l) - x_l^2/2) phi_k(x_l).
 * The flow over time tau in coefficient space is then c <- c x_mu
 * exp(-i tau H_mu) for every mu, exact in time; a step is the forward
 * transform (eq. (real2spec)), the three exponentials, and the backward
 * transform (eq. (spec2real)).
 * ---------------------------------------------------------------------- */

/* H (m x m, row-major) of one direction from the potential's values V[l]
 * at the m nodes x[l] with plain-integral weights W[l]. */
void or_hkp_hamiltonian(int m, const double *x, const double *W, const double *V, double *H)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)m * m);
    or_hermite_functions(m, m, x, P);
    for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) {
            double acc = 0;
            for (int l = 0; l < m; ++l)
                acc += W[l] * P[(size_t)j * m + l] * (V[l] - 0.5 * x[l] * x[l]) * P[(size_t)k * m + l];
            H[(size_t)j * m + k] = acc + (j == k ? k + 0.5 : 0.0);
        }
    free(P);
}

/* nsteps HKP steps of length tau on psi, sizes n[0..2] (n[0] fastest).
 * x[mu], W[mu], V[mu] hold the nodes, weights and potential values of
 * direction mu+1.  Each exponential is or_expm_taylor of -i tau H_mu. */
void or_hkp_steps(const int64_t *n, const double *const *x, const double *const *W,
                  const double *const *V, double tau, int64_t nsteps, cplx *psi)
{
    cplx *fwd[3], *bwd[3], *E[3];
    for (int v = 0; v < 3; ++v) {
        int m = (int)n[v];
        size_t mm = (size_t)m * m;
        double *P = (double *)malloc(sizeof(double) * mm);
        double *H = (double *)malloc(sizeof(double) * mm);
        or_hermite_functions(m, m, x[v], P);
        fwd[v] = (cplx *)malloc(sizeof(cplx) * mm);
        bwd[v] = (cplx *)malloc(sizeof(cplx) * mm);
        E[v] = (cplx *)malloc(sizeof(cplx) * mm);
        for (int k = 0; k < m; ++k)
            for (int l = 0; l < m; ++l) {
                fwd[v][(size_t)k * m + l] = P[(size_t)k * m + l] * W[v][l];
                bwd[v][(size_t)l * m + k] = P[(size_t)k * m + l];
            }
        or_hkp_hamiltonian(m, x[v], W[v], V[v], H);
        or_expm_taylor(m, H, NULL, 0.0, -tau, E[v]);
        free(P);
        free(H);
    }
    int64_t N = n[0] * n[1] * n[2];
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    const cplx *F[3] = {fwd[0], fwd[1], fwd[2]};
    const cplx *G[3] = {E[0], E[1], E[2]};
    const cplx *B[3] = {bwd[0], bwd[1], bwd[2]};
    for (int64_t s = 0; s < nsteps; ++s) {
        or_tucker(3, n, F, NULL, 1, psi, a);
        or_tucker(3, n, G, NULL, 1, a, b);
        or_tucker(3, n, B, NULL, 1, b, psi);
    }
    for (int v = 0; v < 3; ++v) {
        free(fwd[v]);
        free(bwd[v]);
        free(E[v]);
    }
    free(a);
    free(b);
}

/* ------------------------------------------------------------------------
 * HKMP (section 4.4): Hermite pseudospectral discretisation with a
 * time-dependent potential in Kronecker form,
 *   i psi_t = -1/2 Lap psi + sum_mu (V_mu(x_mu) + f(t) U_mu(x_mu)) psi,
 * advanced by the order-two Magnus integrator (eq. (mag2), the exponential
 * midpoint rule).  The Magnus operator at the midpoint t_n + tau/2 is in
 * Kronecker form, so its exponential is the Tucker operator of the
 * directions' exponentials exp(-i tau (H_mu + f_mid G_mu)), with H_mu the
 * Hamiltonian of or_hkp_hamiltonian and G_mu the Galerkin matrix of U_mu.
 * A run: forward transform, nsteps Magnus steps in coefficient space (all
 * exponentials recomputed every step), backward transform.
 * ---------------------------------------------------------------------- */

/* G[j][k] = sum_l W_l phi_j(x_l) U(x_l) phi_k(x_l) (eq. (quadrature)). */
void or_hermite_galerkin(int m, const double *x, const double *W, const double *U, double *G)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)m * m);
    or_hermite_functions(m, m, x, P);
    for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) {
            double acc = 0;
            for (int l = 0; l < m; ++l) acc += W[l] * P[(size_t)j * m + l] * U[l] * P[(size_t)k * m + l];
            G[(size_t)j * m + k] = acc;
        }
    free(P);
}

/* nsteps Magnus steps of length tau on the values psi (sizes n[0..2]).
 * V[mu], U[mu]: values of V_mu and U_mu at the nodes (U[mu] may be NULL:
 * no time dependence in that direction); f_mid[s] = f(t_s + tau/2). */
void or_hkmp_steps(const int64_t *n, const double *const *x, const double *const *W,
                   const double *const *V, const double *const *U, double tau, int64_t nsteps,
                   const double *f_mid, cplx *psi)
{
    cplx *fwd[3], *bwd[3], *E[3];
    double *H[3], *G[3], *A[3];
    for (int v = 0; v < 3; ++v) {
        int m = (int)n[v];
        size_t mm = (size_t)m * m;
        double *P = (double *)malloc(sizeof(double) * mm);
        or_hermite_functions(m, m, x[v], P);
        fwd[v] = (cplx *)malloc(sizeof(cplx) * mm);
        bwd[v] = (cplx *)malloc(sizeof(cplx) * mm);
        E[v] = (cplx *)malloc(sizeof(cplx) * mm);
        H[v] = (double *)malloc(sizeof(double) * mm);
        G[v] = (double *)calloc(mm, sizeof(double));
        A[v] = (double *)malloc(sizeof(double) * mm);
        for (int k = 0; k < m; ++k)
            for (int l = 0; l < m; ++l) {
                fwd[v][(size_t)k * m + l] = P[(size_t)k * m + l] * W[v][l];
                bwd[v][(size_t)l * m + k] = P[(size_t)k * m + l];
            }
        or_hkp_hamiltonian(m, x[v], W[v], V[v], H[v]);
        if (U[v]) or_hermite_galerkin(m, x[v], W[v], U[v], G[v]);
        free(P);
    }
    int64_t N = n[0] * n[1] * n[2];
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    const cplx *F[3] = {fwd[0], fwd[1], fwd[2]};
    const cplx *B[3] = {bwd[0], bwd[1], bwd[2]};
    const cplx *Ec[3] = {E[0], E[1], E[2]};
    or_tucker(3, n, F, NULL, 1, psi, a);
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int v = 0; v < 3; ++v) {
            size_t mm = (size_t)n[v] * n[v];
            for (size_t q = 0; q < mm; ++q) A[v][q] = H[v][q] + f_mid[s] * G[v][q];
            or_expm_taylor((int)n[v], A[v], NULL, 0.0, -tau, E[v]);
        }
        or_tucker(3, n, Ec, NULL, 1, a, b);
        memcpy(a, b, sizeof(cplx) * (size_t)N);
    }
    or_tucker(3, n, B, NULL, 1, a, psi);
    for (int v = 0; v < 3; ++v) {
        free(fwd[v]);
        free(bwd[v]);
        free(E[v]);
        free(H[v]);
        free(G[v]);
        free(A[v]);
    }
    free(a);
    free(b);
}

/* ------------------------------------------------------------------------
 * Pipe flow (section 4.2): c_t = alpha (c_rr + c_r / r + c_zz) - s(z) c_z,
 * radially symmetric, second-order centred differences with n nodes per
 * direction.  The operator is the Kronecker sum of a radial and an axial
 * one (the coefficient 1/r depends on r only, s on z only), so the
 * mu-mode integrator applies (section 2, eq. (tensor-structure)).
 *
 * Grids (the paper gives only "n points per direction"; this reading):
 *   r_j = r_min + j h_r, j = 0..n-1, h_r = (r_max - r_min)/(n-1), both ends
 *     Neumann (c_r = 0) by reflection: ghost c_{-1} = c_1, c_n = c_{n-2};
 *   z_j = j h_z, j = 1..n, h_z = z_max / n: z = 0 carries the Dirichlet
 *     value 0 and is not an unknown; z_max is Neumann by reflection
 *     (ghost c_{n+1} = c_{n-1}).
 * ---------------------------------------------------------------------- */

/* A = alpha (D2 + diag(1/r) D1) on the radial grid; first = 0 drops the
 * 1/r D1 term. */
void or_pipe_radial(int n, double rmin, double rmax, double alpha, int first, double *A)
{
    double h = (rmax - rmin) / (n - 1);
    memset(A, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double r = rmin + j * h;
        /* coefficients of c_{j-1}, c_j, c_{j+1} before reflection */
        double lo = 1.0 / (h * h), mid = -2.0 / (h * h), hi = 1.0 / (h * h);
        if (first) {
            lo -= 1.0 / (r * 2.0 * h);
            hi += 1.0 / (r * 2.0 * h);
        }
        int jl = j - 1, jh = j + 1;
        if (jl < 0) jl = 1;          /* ghost c_{-1} = c_1 */
        if (jh > n - 1) jh = n - 2;  /* ghost c_n = c_{n-2} */
        A[(size_t)j * n + j] += alpha * mid;
        A[(size_t)j * n + jl] += alpha * lo;
        A[(size_t)j * n + jh] += alpha * hi;
    }
}

/* A = alpha D2 - diag(s) D1 on the axial grid; s holds s(z_j), j = 1..n,
 * or is NULL (pure diffusion). */
void or_pipe_axial(int n, double zmax, double alpha, const double *s, double *A)
{
    double h = zmax / n;
    memset(A, 0, sizeof(double) * (size_t)n * n);
    for (int q = 0; q < n; ++q) { /* unknown q is z_{q+1} */
        double sv = s ? s[q] : 0.0;
        double lo = alpha / (h * h) + sv / (2.0 * h);
        double mid = -2.0 * alpha / (h * h);
        double hi = alpha / (h * h) - sv / (2.0 * h);
        A[(size_t)q * n + q] += mid;
        if (q > 0) A[(size_t)q * n + q - 1] += lo; /* q == 0: neighbour z_0 = 0 is the Dirichlet value */
        if (q < n - 1) A[(size_t)q * n + q + 1] += hi;
        else A[(size_t)q * n + q - 1] += hi; /* ghost c_{n+1} = c_{n-1} */
    }
}
