// FP64 host set-up of the mu-mode integrator: one-dimensional operators,
// their exponentials and the Hermite-function matrices.  These are the
// "d small exponentials" of section 2, computed once for a constant step
// (their cost is the "exp" column of the paper's section 5 tables), and the
// Gauss-Hermite / Hermite-function data of section 3.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mm {

using cd = std::complex<double>;

void fd_laplacian_dirichlet(int n, double *A)
{
    const double inv_h2 = double(n + 1) * double(n + 1);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            A[size_t(i) * n + j] = (i == j) ? -2.0 * inv_h2 : (std::abs(i - j) == 1 ? inv_h2 : 0.0);
}

namespace {

void matmul(int n, const cd *A, const cd *B, cd *C)
{
    std::vector<cd> tmp(size_t(n) * n, cd(0));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const cd a = A[size_t(i) * n + k];
            if (a == cd(0)) continue;
            const cd *brow = B + size_t(k) * n;
            cd *trow = tmp.data() + size_t(i) * n;
            for (int j = 0; j < n; ++j) trow[j] += a * brow[j];
        }
    std::memcpy(C, tmp.data(), sizeof(cd) * tmp.size());
}

double norm1(int n, const cd *A)
{
    double best = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < n; ++i) s += std::abs(A[size_t(i) * n + j]);
        best = std::max(best, s);
    }
    return best;
}

// Solve P X = Q for X (overwrites Q), LU with partial pivoting.
bool solve(int n, std::vector<cd> &P, std::vector<cd> &Q)
{
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::abs(P[size_t(k) * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = std::abs(P[size_t(i) * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                std::swap(P[size_t(k) * n + j], P[size_t(p) * n + j]);
                std::swap(Q[size_t(k) * n + j], Q[size_t(p) * n + j]);
            }
        }
        const cd inv = 1.0 / P[size_t(k) * n + k];
        for (int i = k + 1; i < n; ++i) {
            const cd f = P[size_t(i) * n + k] * inv;
            if (f == cd(0)) continue;
            for (int j = k; j < n; ++j) P[size_t(i) * n + j] -= f * P[size_t(k) * n + j];
            for (int j = 0; j < n; ++j) Q[size_t(i) * n + j] -= f * Q[size_t(k) * n + j];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        const cd inv = 1.0 / P[size_t(k) * n + k];
        for (int j = 0; j < n; ++j) {
            cd s = Q[size_t(k) * n + j];
            for (int i = k + 1; i < n; ++i) s -= P[size_t(k) * n + i] * Q[size_t(i) * n + j];
            Q[size_t(k) * n + j] = s * inv;
        }
    }
    return true;
}

}  // namespace

// exp(z A) by scaling and squaring with the [13/13] Pade approximant
// (N. J. Higham, "The scaling and squaring method for the matrix
// exponential revisited", SIAM J. Matrix Anal. Appl. 26 (2005)).  The Pade
// coefficients c_j = (26-j)! 13! / (26! j! (13-j)!) are generated from
// their definition; theta_13 = 5.37 is the published bound on ||A||_1 for
// which the [13/13] approximant is accurate to double precision.
bool expm(int n, const double *Are, const double *Aim, cd z, cd *E)
{
    const size_t nn = size_t(n) * n;
    std::vector<cd> A(nn);
    for (size_t q = 0; q < nn; ++q) A[q] = z * cd(Are[q], Aim ? Aim[q] : 0.0);
    const double theta13 = 5.371920351148152;
    const double nrm = norm1(n, A.data());
    int s = 0;
    if (nrm > theta13) s = std::max(0, int(std::ceil(std::log2(nrm / theta13))));
    const double scale = std::ldexp(1.0, -s);
    for (auto &v : A) v *= scale;

    double c[14];
    c[0] = 1.0;
    for (int j = 1; j <= 13; ++j) c[j] = c[j - 1] * double(13 - j + 1) / (double(j) * double(26 - j + 1));

    std::vector<cd> A2(nn), A4(nn), A6(nn), U(nn), V(nn), T(nn);
    matmul(n, A.data(), A.data(), A2.data());
    matmul(n, A2.data(), A2.data(), A4.data());
    matmul(n, A4.data(), A2.data(), A6.data());
    // U = A [A6 (c13 A6 + c11 A4 + c9 A2) + c7 A6 + c5 A4 + c3 A2 + c1 I]
    // V =    A6 (c12 A6 + c10 A4 + c8 A2) + c6 A6 + c4 A4 + c2 A2 + c0 I
    for (size_t q = 0; q < nn; ++q) T[q] = c[13] * A6[q] + c[11] * A4[q] + c[9] * A2[q];
    matmul(n, A6.data(), T.data(), U.data());
    for (size_t q = 0; q < nn; ++q) U[q] += c[7] * A6[q] + c[5] * A4[q] + c[3] * A2[q];
    for (int i = 0; i < n; ++i) U[size_t(i) * n + i] += c[1];
    matmul(n, A.data(), U.data(), U.data());
    for (size_t q = 0; q < nn; ++q) T[q] = c[12] * A6[q] + c[10] * A4[q] + c[8] * A2[q];
    matmul(n, A6.data(), T.data(), V.data());
    for (size_t q = 0; q < nn; ++q) V[q] += c[6] * A6[q] + c[4] * A4[q] + c[2] * A2[q];
    for (int i = 0; i < n; ++i) V[size_t(i) * n + i] += c[0];
    std::vector<cd> P(nn), Q(nn);
    for (size_t q = 0; q < nn; ++q) {
        P[q] = V[q] - U[q];
        Q[q] = V[q] + U[q];
    }
    if (!solve(n, P, Q)) return false;
    for (int k = 0; k < s; ++k) matmul(n, Q.data(), Q.data(), Q.data());
    std::memcpy(E, Q.data(), sizeof(cd) * nn);
    return true;
}

// Hermite functions phi_0..phi_{count-1} at x (section 3: H_k orthonormal
// for exp(-x^2), phi_k = H_k exp(-x^2/2)), by their normalised three-term
// recurrence phi_{k+1} = sqrt(2/(k+1)) x phi_k - sqrt(k/(k+1)) phi_{k-1}.
static void hermite_values(int count, double x, double *out)
{
    double prev = std::pow(M_PI, -0.25) * std::exp(-0.5 * x * x);
    out[0] = prev;
    if (count < 2) return;
    double cur = std::sqrt(2.0) * x * prev;
    out[1] = cur;
    for (int k = 1; k + 1 < count; ++k) {
        const double next = std::sqrt(2.0 / (k + 1)) * x * cur - std::sqrt(double(k) / (k + 1)) * prev;
        out[k + 1] = next;
        prev = cur;
        cur = next;
    }
}

// Gauss-Hermite nodes = eigenvalues of the symmetric tridiagonal Jacobi
// matrix of the Hermite recurrence (zero diagonal, off-diagonal sqrt(k/2))
// (Golub-Welsch), found one by one by bisection on the Sturm count; then
// W_l = 1 / sum_k phi_k(x_l)^2 (Christoffel function).
bool gauss_hermite(int m, double *x, double *W)
{
    std::vector<double> b2(m);  // squared off-diagonal, b2[k] = k/2 couples k-1, k
    for (int k = 1; k < m; ++k) b2[k] = 0.5 * k;
    auto count_below = [&](double t) {
        int cnt = 0;
        double dprev = 1.0;
        for (int k = 0; k < m; ++k) {
            double dk = -t - (k > 0 ? b2[k] / dprev : 0.0);
            if (dk == 0.0) dk = -1e-300;
            if (dk < 0) ++cnt;
            dprev = dk;
        }
        return cnt;
    };
    const double bound = std::sqrt(2.0 * m) + 1.0;
    for (int i = 0; i < m; ++i) {
        double lo = -bound, hi = bound;  // count_below(lo) <= i < count_below(hi)
        for (int it = 0; it < 200 && hi - lo > 0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (count_below(mid) > i) hi = mid;
            else lo = mid;
        }
        x[i] = 0.5 * (lo + hi);
    }
    std::vector<double> col(m);
    for (int l = 0; l < m; ++l) {
        hermite_values(m, x[l], col.data());
        double s = 0;
        for (int k = 0; k < m; ++k) s += col[k] * col[k];
        W[l] = 1.0 / s;
    }
    return true;
}

void hermite_matrices(int m, const double *x, const double *W, double *fwd, double *bwd)
{
    std::vector<double> col(m);
    for (int l = 0; l < m; ++l) {
        hermite_values(m, x[l], col.data());
        for (int k = 0; k < m; ++k) {
            if (fwd) fwd[size_t(k) * m + l] = col[k] * W[l];
            if (bwd) bwd[size_t(l) * m + k] = col[k];
        }
    }
}

// Hamiltonian of one direction of i psi_t = -1/2 Lap psi + V psi in the
// Hermite functions (section 4.3, HKP).  -1/2 d^2/dx^2 + x^2/2 is diagonal
// with eigenvalues k + 1/2 (section 3); the remainder V - x^2/2 enters by
// its Galerkin matrix under the Gauss-Hermite rule of eq. (quadrature):
//   H[j][k] = (k + 1/2) delta_jk + sum_l phi_j(x_l) W_l (V_l - x_l^2/2) phi_k(x_l).
// V == nullptr means the harmonic potential itself (H diagonal).
void hermite_hamiltonian(int m, const double *x, const double *W, const double *V, double *H)
{
    std::fill(H, H + size_t(m) * m, 0.0);
    for (int k = 0; k < m; ++k) H[size_t(k) * m + k] = k + 0.5;
    if (!V) return;
    std::vector<double> phi(size_t(m) * m), g(m), col(m);  // phi[l][k] = phi_k(x_l)
    for (int l = 0; l < m; ++l) {
        hermite_values(m, x[l], phi.data() + size_t(l) * m);
        g[l] = W[l] * (V[l] - 0.5 * x[l] * x[l]);
    }
    for (int l = 0; l < m; ++l) {
        const double *p = phi.data() + size_t(l) * m;
        if (g[l] == 0.0) continue;
        for (int j = 0; j < m; ++j) {
            const double a = g[l] * p[j];
            double *hrow = H + size_t(j) * m;
            for (int k = 0; k < m; ++k) hrow[k] += a * p[k];
        }
    }
}

// Galerkin matrix of the multiplication by U under the Gauss-Hermite rule:
// G[j][k] = sum_l phi_j(x_l) W_l U_l phi_k(x_l).
void hermite_galerkin(int m, const double *x, const double *W, const double *U, double *G)
{
    std::fill(G, G + size_t(m) * m, 0.0);
    std::vector<double> phi(static_cast<size_t>(m), 0.0);
    for (int l = 0; l < m; ++l) {
        hermite_values(m, x[l], phi.data());
        const double g = W[l] * U[l];
        if (g == 0.0) continue;
        for (int j = 0; j < m; ++j) {
            const double a = g * phi[size_t(j)];
            double *grow = G + size_t(j) * m;
            for (int k = 0; k < m; ++k) grow[k] += a * phi[size_t(k)];
        }
    }
}

// Pipe flow (section 4.2), centred second-order differences.  Radial
// operator alpha (d^2/dr^2 + (1/r) d/dr) on r_j = r_min + j h, j < n,
// h = (r_max - r_min)/(n - 1), with c_r = 0 at both ends imposed by
// mirroring the neighbour (the ghost value equals the value one node in).
void pipe_radial(int n, double rmin, double rmax, double alpha, double *A)
{
    std::fill(A, A + size_t(n) * n, 0.0);
    const double h = (rmax - rmin) / double(n - 1), d2 = alpha / (h * h);
    for (int j = 0; j < n; ++j) {
        const double d1 = alpha / ((rmin + j * h) * 2.0 * h);
        const int left = j == 0 ? 1 : j - 1, right = j == n - 1 ? n - 2 : j + 1;
        double *row = A + size_t(j) * n;
        row[j] += -2.0 * d2;
        row[left] += d2 - d1;
        row[right] += d2 + d1;
    }
}

// Axial operator alpha d^2/dz^2 - s(z) d/dz on z_j = j h, j = 1..n,
// h = z_max / n: c = 0 at z = 0 (not an unknown) and c_z = 0 at z_max by
// mirroring.  s holds s(z_j) for the n unknowns.
void pipe_axial(int n, double zmax, double alpha, const double *s, double *A)
{
    std::fill(A, A + size_t(n) * n, 0.0);
    const double h = zmax / double(n), d2 = alpha / (h * h);
    for (int q = 0; q < n; ++q) {
        const double d1 = (s ? s[q] : 0.0) / (2.0 * h);
        double *row = A + size_t(q) * n;
        row[q] += -2.0 * d2;
        if (q > 0) row[q - 1] += d2 + d1;
        const int right = q == n - 1 ? n - 2 : q + 1;
        if (right >= 0) row[right] += d2 - d1;
    }
}

}  // namespace mm
