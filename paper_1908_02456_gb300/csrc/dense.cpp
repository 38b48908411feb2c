// Dense complex<double> linear algebra for the FP64 host setup: a packed,
// register-blocked GEMM (C -= A B), a blocked right-looking LU with partial
// pivoting and the blocked solve with many right-hand sides.  Column-major
// throughout.  Plain C++ with GCC vector extensions (2 x double), no
// architecture-specific intrinsics, so it builds unchanged on x86-64 and aarch64
// and sums in the same order on both.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace abc {

typedef double v2d __attribute__((vector_size(16)));

namespace {

constexpr int MR = 4;    // complex rows per micro-tile
constexpr int NR = 4;    // complex columns per micro-tile
constexpr int KC = 256;
constexpr int MC = 96;
constexpr int NC = 2048;
constexpr int NSUB = 64; // columns per parallel task

inline v2d ld2(const double* p) {
    v2d v;
    std::memcpy(&v, p, sizeof(v));
    return v;
}

// acc(MR x NR) = sum_p A(:,p) B(p,:), then C -= acc on the valid mr x nr corner.
void micro(int kc, const double* __restrict Ap, const double* __restrict Bp, cd* C, int ldc,
           int mr, int nr) {
    v2d cr[NR][2], ci[NR][2];
    for (int j = 0; j < NR; ++j) {
        cr[j][0] = cr[j][1] = ci[j][0] = ci[j][1] = v2d{0.0, 0.0};
    }
    for (int p = 0; p < kc; ++p) {
        const double* a = Ap + 2 * MR * p;
        const double* b = Bp + 2 * NR * p;
        const v2d ar0 = ld2(a), ar1 = ld2(a + 2), ai0 = ld2(a + 4), ai1 = ld2(a + 6);
        for (int j = 0; j < NR; ++j) {
            const double br = b[j], bi = b[NR + j];
            cr[j][0] += ar0 * br - ai0 * bi;
            cr[j][1] += ar1 * br - ai1 * bi;
            ci[j][0] += ar0 * bi + ai0 * br;
            ci[j][1] += ar1 * bi + ai1 * br;
        }
    }
    for (int j = 0; j < nr; ++j) {
        cd* c = C + (size_t)j * ldc;
        for (int i = 0; i < mr; ++i) c[i] -= cd(cr[j][i >> 1][i & 1], ci[j][i >> 1][i & 1]);
    }
}

// Pack A(i0:i0+mc, p0:p0+kc) into MR-row strips: per k, MR reals then MR imags.
void pack_a(int mc, int kc, const cd* A, int lda, double* Ap) {
    for (int ir = 0; ir < mc; ir += MR) {
        double* dst = Ap + (size_t)ir * 2 * kc;
        const int mr = std::min(MR, mc - ir);
        for (int p = 0; p < kc; ++p) {
            const cd* col = A + (size_t)p * lda + ir;
            for (int i = 0; i < MR; ++i) {
                const cd v = i < mr ? col[i] : cd(0.0, 0.0);
                dst[2 * MR * p + i] = v.real();
                dst[2 * MR * p + MR + i] = v.imag();
            }
        }
    }
}

// Pack B(p0:p0+kc, j0:j0+nc) into NR-column strips: per k, NR reals then NR imags.
void pack_b(int kc, int nc, const cd* B, int ldb, double* Bp) {
#pragma omp parallel for schedule(static)
    for (int jr = 0; jr < nc; jr += NR) {
        double* dst = Bp + (size_t)jr * 2 * kc;
        const int nr = std::min(NR, nc - jr);
        for (int p = 0; p < kc; ++p) {
            for (int j = 0; j < NR; ++j) {
                const cd v = j < nr ? B[(size_t)(jr + j) * ldb + p] : cd(0.0, 0.0);
                dst[2 * NR * p + j] = v.real();
                dst[2 * NR * p + NR + j] = v.imag();
            }
        }
    }
}

}  // namespace

void zgemm_sub(int m, int n, int k, const cd* A, int lda, const cd* B, int ldb, cd* C, int ldc) {
    if (m <= 0 || n <= 0 || k <= 0) return;
    const int ncap = std::min(NC, n);
    std::vector<double> Bp((size_t)2 * KC * (ncap + NR));
    for (int pc = 0; pc < k; pc += KC) {
        const int kc = std::min(KC, k - pc);
        for (int jc = 0; jc < n; jc += NC) {
            const int nc = std::min(NC, n - jc);
            pack_b(kc, nc, B + (size_t)jc * ldb + pc, ldb, Bp.data());
            const int n_ib = (m + MC - 1) / MC, n_jb = (nc + NSUB - 1) / NSUB;
#pragma omp parallel
            {
                std::vector<double> Ap((size_t)2 * KC * (MC + MR));
                int packed_ib = -1;
#pragma omp for schedule(dynamic) collapse(2)
                for (int ib = 0; ib < n_ib; ++ib) {
                    for (int jb = 0; jb < n_jb; ++jb) {
                        const int ic = ib * MC, mc = std::min(MC, m - ic);
                        if (packed_ib != ib) {
                            pack_a(mc, kc, A + (size_t)pc * lda + ic, lda, Ap.data());
                            packed_ib = ib;
                        }
                        const int j0 = jb * NSUB, j1 = std::min(nc, j0 + NSUB);
                        for (int jr = j0; jr < j1; jr += NR) {
                            const int nr = std::min(NR, nc - jr);
                            for (int ir = 0; ir < mc; ir += MR) {
                                micro(kc, Ap.data() + (size_t)ir * 2 * kc, Bp.data() + (size_t)jr * 2 * kc,
                                      C + (size_t)(jc + jr) * ldc + ic + ir, ldc, std::min(MR, mc - ir), nr);
                            }
                        }
                    }
                }
            }
        }
    }
}

static inline double cabs1(cd z) { return std::fabs(z.real()) + std::fabs(z.imag()); }

int zgetrf(int n, cd* A, int lda, int* ipiv) {
    const int NB = 64;
    for (int j = 0; j < n; j += NB) {
        const int jb = std::min(NB, n - j);
        // unblocked factorisation of the panel A(j:n, j:j+jb)
        for (int jj = j; jj < j + jb; ++jj) {
            cd* colj = A + (size_t)jj * lda;
            int p = jj;
            double best = cabs1(colj[jj]);
            for (int i = jj + 1; i < n; ++i) {
                const double v = cabs1(colj[i]);
                if (v > best) { best = v; p = i; }
            }
            ipiv[jj] = p;
            if (best == 0.0) return jj + 1;
            if (p != jj) {
                for (int c = j; c < j + jb; ++c) std::swap(A[(size_t)c * lda + jj], A[(size_t)c * lda + p]);
            }
            const cd inv = 1.0 / colj[jj];
            for (int i = jj + 1; i < n; ++i) colj[i] *= inv;
            const int rows = n - jj - 1;
#pragma omp parallel for schedule(static) if (rows > 512)
            for (int c = jj + 1; c < j + jb; ++c) {
                cd* colc = A + (size_t)c * lda;
                const cd u = colc[jj];
                if (u != cd(0.0, 0.0)) {
                    for (int i = jj + 1; i < n; ++i) colc[i] -= colj[i] * u;
                }
            }
        }
        // row interchanges outside the panel
#pragma omp parallel for schedule(static)
        for (int c = 0; c < n; ++c) {
            if (c >= j && c < j + jb) continue;
            cd* col = A + (size_t)c * lda;
            for (int jj = j; jj < j + jb; ++jj)
                if (ipiv[jj] != jj) std::swap(col[jj], col[ipiv[jj]]);
        }
        if (j + jb < n) {
            // A12 <- L11^{-1} A12 (unit lower triangular)
#pragma omp parallel for schedule(static)
            for (int c = j + jb; c < n; ++c) {
                cd* col = A + (size_t)c * lda;
                for (int r = 0; r < jb; ++r) {
                    const cd v = col[j + r];
                    if (v == cd(0.0, 0.0)) continue;
                    const cd* l = A + (size_t)(j + r) * lda;
                    for (int rr = r + 1; rr < jb; ++rr) col[j + rr] -= l[j + rr] * v;
                }
            }
            // A22 -= A21 A12
            zgemm_sub(n - j - jb, n - j - jb, jb, A + (size_t)j * lda + j + jb, lda,
                      A + (size_t)(j + jb) * lda + j, lda, A + (size_t)(j + jb) * lda + j + jb, lda);
        }
    }
    return 0;
}

void zgetrs(int n, int nrhs, const cd* A, int lda, const int* ipiv, cd* B, int ldb) {
    const int NB = 128;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nrhs; ++c) {
        cd* col = B + (size_t)c * ldb;
        for (int i = 0; i < n; ++i)
            if (ipiv[i] != i) std::swap(col[i], col[ipiv[i]]);
    }
    // forward substitution with the unit lower factor
    for (int j = 0; j < n; j += NB) {
        const int jb = std::min(NB, n - j);
#pragma omp parallel for schedule(static)
        for (int c = 0; c < nrhs; ++c) {
            cd* col = B + (size_t)c * ldb;
            for (int r = 0; r < jb; ++r) {
                const cd v = col[j + r];
                const cd* l = A + (size_t)(j + r) * lda;
                for (int rr = r + 1; rr < jb; ++rr) col[j + rr] -= l[j + rr] * v;
            }
        }
        if (j + jb < n)
            zgemm_sub(n - j - jb, nrhs, jb, A + (size_t)j * lda + j + jb, lda, B + j, ldb, B + j + jb, ldb);
    }
    // back substitution with the upper factor
    const int last = ((n - 1) / NB) * NB;
    for (int j = last; j >= 0; j -= NB) {
        const int jb = std::min(NB, n - j);
#pragma omp parallel for schedule(static)
        for (int c = 0; c < nrhs; ++c) {
            cd* col = B + (size_t)c * ldb;
            for (int r = jb - 1; r >= 0; --r) {
                const cd* u = A + (size_t)(j + r) * lda;
                col[j + r] /= u[j + r];
                const cd v = col[j + r];
                for (int rr = 0; rr < r; ++rr) col[j + rr] -= u[j + rr] * v;
            }
        }
        if (j > 0) zgemm_sub(j, nrhs, jb, A + (size_t)j * lda, lda, B + j, ldb, B, ldb);
    }
}

// Householder QR with column pivoting of a square A (column-major n x n, overwritten)
// and the basic solution of A Z = B (B: n x nrhs, overwritten by Z).  Each step takes
// the remaining column of largest norm (norms downdated after each reflection and
// recomputed when cancellation has eaten half the digits), reflects it onto e_k with
// H = I - tau v v^H (v_0 = 1, beta = R_kk real: the convention of LAPACK's zlarfg) and
// applies H^H to the trailing columns.  The factorisation stops at the first pivot with
// |R_kk| <= abs_tol (every remaining column is that small): the numerical rank r.  Then
// Z = P [R_11^{-1} (Q^H B)_1 ; 0]: the free unknowns of a rank-deficient system are set
// to zero (Golub and Van Loan, Sec. 5.5, the basic solution).  Returns 0; *rank = r.
int zqrp_basic(int n, int nrhs, cd* A, int lda, cd* B, int ldb, double abs_tol, int* rank) {
    std::vector<int> perm(n);
    std::vector<double> cn(n), cn0(n);
    std::vector<cd> tau(n, cd(0.0, 0.0));
    const double tol3z = std::sqrt(2.220446049250313e-16);
    for (int j = 0; j < n; ++j) {
        perm[j] = j;
        double s2 = 0;
        const cd* c = A + (size_t)j * lda;
        for (int i = 0; i < n; ++i) s2 += std::norm(c[i]);
        cn[j] = cn0[j] = std::sqrt(s2);
    }
    int r = n;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int j = k + 1; j < n; ++j)
            if (cn[j] > cn[p]) p = j;
        if (p != k) {
            std::swap_ranges(A + (size_t)k * lda, A + (size_t)k * lda + n, A + (size_t)p * lda);
            std::swap(cn[k], cn[p]);
            std::swap(cn0[k], cn0[p]);
            std::swap(perm[k], perm[p]);
        }
        cd* col = A + (size_t)k * lda;
        const cd alpha = col[k];
        double xn = 0;
        for (int i = k + 1; i < n; ++i) xn += std::norm(col[i]);
        xn = std::sqrt(xn);
        double beta;
        cd t(0.0, 0.0);
        if (xn == 0.0 && alpha.imag() == 0.0) {
            beta = alpha.real();
        } else {
            beta = -std::copysign(std::sqrt(std::norm(alpha) + xn * xn), alpha.real());
            t = cd((beta - alpha.real()) / beta, -alpha.imag() / beta);
            const cd sc = 1.0 / (alpha - beta);
            for (int i = k + 1; i < n; ++i) col[i] *= sc;
        }
        col[k] = beta;
        tau[k] = t;
        if (std::fabs(beta) <= abs_tol) {
            r = k;
            break;
        }
        const cd ct = std::conj(t);
#pragma omp parallel for schedule(static) if (n - k > 96)
        for (int j = k + 1; j < n; ++j) {
            cd* cj = A + (size_t)j * lda;
            cd w = cj[k];
            for (int i = k + 1; i < n; ++i) w += std::conj(col[i]) * cj[i];
            w *= ct;
            cj[k] -= w;
            for (int i = k + 1; i < n; ++i) cj[i] -= col[i] * w;
            if (cn[j] > 0.0) {
                const double q = std::abs(cj[k]) / cn[j];
                const double temp = std::max(0.0, (1.0 + q) * (1.0 - q));
                const double ratio = cn[j] / cn0[j];
                if (temp * ratio * ratio <= tol3z) {
                    double s2 = 0;
                    for (int i = k + 1; i < n; ++i) s2 += std::norm(cj[i]);
                    cn[j] = cn0[j] = std::sqrt(s2);
                } else {
                    cn[j] *= std::sqrt(temp);
                }
            }
        }
    }
    *rank = r;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nrhs; ++c) {
        cd* b = B + (size_t)c * ldb;
        for (int k = 0; k < r; ++k) {                  // b <- H_k^H b
            const cd* v = A + (size_t)k * lda;
            cd w = b[k];
            for (int i = k + 1; i < n; ++i) w += std::conj(v[i]) * b[i];
            w *= std::conj(tau[k]);
            b[k] -= w;
            for (int i = k + 1; i < n; ++i) b[i] -= v[i] * w;
        }
        std::vector<cd> y(r);
        for (int i = r - 1; i >= 0; --i) {             // R_11 y = (Q^H b)_1
            cd acc = b[i];
            for (int j = i + 1; j < r; ++j) acc -= A[(size_t)j * lda + i] * y[j];
            y[i] = acc / A[(size_t)i * lda + i];
        }
        for (int i = 0; i < n; ++i) b[i] = cd(0.0, 0.0);
        for (int i = 0; i < r; ++i) b[perm[i]] = y[i];
    }
    return 0;
}

}  // namespace abc
