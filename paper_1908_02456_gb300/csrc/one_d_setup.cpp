// FP64 host set-up of the one-dimensional boundary blocks (Sec. 4.1, App. B).
//
// One end of the 1D box with the five-point scheme: Gamma = {0, 1} (local order),
// Sigma = {-1, -2}; H_{Gamma,Sigma} holds -c_m / (2 h^2) for every pair m = |x - x'| <= 2.
// The free lattice Green's function G = (H_0 - i s)^{-1} is, by App. B, a sum of two
// decaying powers: H_0 acts on u^n as -(1/(2h^2)) (c2 u^2 + c1 u + c0 + c1/u + c2/u^2),
// so (H_0 - i s) u^n = 0 where c2 u^4 + c1 u^3 + (c0 + 2 i s h^2) u^2 + c1 u + c2 = 0.
// The quartic is palindromic: with w = u + 1/u it becomes c2 w^2 + c1 w + (c0 - 2 c2 +
// 2 i s h^2) = 0, and each w gives the pair u, 1/u; the roots with |u| < 1 are kept.
// G_n = b1 u1^|n| + b2 u2^|n| solves the equation for |n| >= 2 by construction; b1, b2
// make it hold at n = 0 (the delta) and n = 1 (where the stencil reaches across 0).
// Then eq:eval, K = -(I - H_{Gamma,Sigma} G_{Sigma,Gamma})^{-1} H_{Gamma,Sigma}
// G_{Sigma,Sigma} H_{Sigma,Gamma}, and the order-0/1/2 coefficients of the 3D library,
// here as 2 x 2 blocks.
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "one_d.h"

namespace abc {
namespace oned {

namespace {
typedef std::complex<double> cd;
const double kC[3] = {-2.5, 4.0 / 3.0, -1.0 / 12.0};

// Gaussian elimination with partial pivoting: solves A X = B (A n x n, B n x m, row-major).
bool solve(std::vector<cd> A, std::vector<cd>& B, int n, int m) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::abs(A[r * n + col]) > std::abs(A[piv * n + col])) piv = r;
        if (std::abs(A[piv * n + col]) == 0.0) return false;
        if (piv != col) {
            for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
            for (int k = 0; k < m; ++k) std::swap(B[col * m + k], B[piv * m + k]);
        }
        for (int r = col + 1; r < n; ++r) {
            const cd f = A[r * n + col] / A[col * n + col];
            if (f == 0.0) continue;
            for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
            for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[col * m + k];
        }
    }
    for (int col = n - 1; col >= 0; --col) {
        for (int k = 0; k < m; ++k) {
            cd v = B[col * m + k];
            for (int j = col + 1; j < n; ++j) v -= A[col * n + j] * B[j * m + k];
            B[col * m + k] = v / A[col * n + col];
        }
    }
    return true;
}

// One-sided (Hestenes) Jacobi SVD of a square complex matrix B (row-major n x n):
// unitary plane rotations from the right make the columns of B V mutually orthogonal.
// On return B holds W = B V (column k has norm sigma_k), V the accumulated rotations
// (row-major, column k the right singular vector k).  Each rotation first turns the
// phase of column q so that the pair's Gram matrix is real, then applies the real
// symmetric Schur rotation of that 2 x 2 Gram matrix (Golub and Van Loan, Sec. 8.6).
void jacobi_svd(std::vector<cd>& B, std::vector<cd>& V, int n) {
    V.assign((size_t)n * n, cd(0.0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double al = 0, be = 0;
                cd ga = 0;
                for (int i = 0; i < n; ++i) {
                    const cd bp = B[(size_t)i * n + p], bq = B[(size_t)i * n + q];
                    al += std::norm(bp);
                    be += std::norm(bq);
                    ga += std::conj(bp) * bq;
                }
                const double g = std::abs(ga);
                if (g <= 1e-15 * std::sqrt(al * be) || g == 0.0) continue;
                rotated = true;
                const cd ph = std::conj(ga / g);
                const double zeta = (be - al) / (2.0 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (std::vector<cd>* m : {&B, &V})
                    for (int i = 0; i < n; ++i) {
                        cd& xp = (*m)[(size_t)i * n + p];
                        cd& xq = (*m)[(size_t)i * n + q];
                        const cd a = xp, b = xq * ph;
                        xp = c * a - sn * b;
                        xq = sn * a + c * b;
                    }
            }
        if (!rotated) break;
    }
}

// The order-2 interpolation conditions of one end, X M = Y with X = [B1 B0 A1 A0]
// (2 x 8), given as Mt = M^T and Yt = Y^T (row-major 8 x 8 and 8 x 2).  For the
// five-point scheme M has a one-dimensional null space: a fixed row combination of
// K(s) obeys a first-degree identity (s b1 + b0) K(s) = -(s a1 + a0) for every s, so
// the solutions X0 + w x (x the null row, w any 2-vector) share R_22(s) for every s and
// differ only in one hidden root of det(s^2 I - s B1 - B0), which rounding excites and
// which for some w lies in the right half-plane.  Here X0 is the minimum-norm solution
// (pseudo-inverse of rank 7) and w the shortest vector that puts the hidden root at
// s = -min(s_j): by the determinant lemma det(D0(l) - w r) = det D0(l) - r adj(D0(l)) w
// with D0(l) = l^2 I - l B1 - B0 of X0 and r = l x_B1 + x_B0, one linear condition.  A
// system of full numerical rank is solved as it stands.
int fit_order2_end(const std::vector<cd>& Mt, const std::vector<cd>& Yt, double lam, cd X[2][8],
                   std::string& err) {
    std::vector<cd> B(64), V;
    for (int i = 0; i < 64; ++i) B[i] = std::conj(Mt[i]);          // B = M^H
    jacobi_svd(B, V, 8);                                            // M = V diag(sigma) (B V / sigma)^H
    double sig[8];
    int order[8];
    for (int k = 0; k < 8; ++k) {
        double v = 0;
        for (int i = 0; i < 8; ++i) v += std::norm(B[i * 8 + k]);
        sig[k] = std::sqrt(v);
        order[k] = k;
    }
    std::sort(order, order + 8, [&](int a, int b) { return sig[a] > sig[b]; });
    const int kmin = order[7];
    if (sig[kmin] > 1e-6 * sig[order[6]]) {
        std::vector<cd> Y = Yt;
        if (!solve(Mt, Y, 8, 2)) { err = "order-2 interpolation system singular"; return ABC_ERR_SINGULAR; }
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 8; ++k) X[r][k] = Y[k * 2 + r];
        return ABC_OK;
    }
    if (!(sig[order[6]] > 1e-14 * sig[order[0]])) {
        err = "order-2 interpolation system has more than one null direction";
        return ABC_ERR_SINGULAR;
    }
    cd x[8];
    for (int k = 0; k < 8; ++k) x[k] = std::conj(V[k * 8 + kmin]);      // x M = 0
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 8; ++k) X[r][k] = 0.0;
    for (int kk = 0; kk < 8; ++kk) {
        if (kk == kmin) continue;
        for (int r = 0; r < 2; ++r) {
            cd yw = 0;                                                  // Y w_kk
            for (int col = 0; col < 8; ++col) yw += Yt[col * 2 + r] * B[col * 8 + kk];
            yw /= sig[kk] * sig[kk];
            for (int k = 0; k < 8; ++k) X[r][k] += yw * std::conj(V[k * 8 + kk]);
        }
    }
    cd D0[2][2];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k) D0[r][k] = (r == k ? lam * lam : 0.0) - lam * X[r][k] - X[r][2 + k];
    const cd adj[2][2] = {{D0[1][1], -D0[0][1]}, {-D0[1][0], D0[0][0]}};
    const cd det = D0[0][0] * D0[1][1] - D0[0][1] * D0[1][0];
    const cd rv[2] = {lam * x[0] + x[2], lam * x[1] + x[3]};
    cd c[2];
    for (int j = 0; j < 2; ++j) c[j] = rv[0] * adj[0][j] + rv[1] * adj[1][j];
    const double cn = std::norm(c[0]) + std::norm(c[1]);
    if (!(cn > 0.0)) { err = "order-2 hidden root cannot be placed"; return ABC_ERR_SINGULAR; }
    for (int r = 0; r < 2; ++r) {
        const cd w = std::conj(c[r]) * det / cn;
        for (int k = 0; k < 8; ++k) X[r][k] += w * x[k];
    }
    return ABC_OK;
}

Mat2 mul(const Mat2& a, const Mat2& b) {
    Mat2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.v[i][j] = a.v[i][0] * b.v[0][j] + a.v[i][1] * b.v[1][j];
    return r;
}
Mat2 inv(const Mat2& a, bool& ok) {
    const cd det = a.v[0][0] * a.v[1][1] - a.v[0][1] * a.v[1][0];
    ok = std::abs(det) > 0.0;
    Mat2 r{};
    if (!ok) return r;
    r.v[0][0] = a.v[1][1] / det;
    r.v[0][1] = -a.v[0][1] / det;
    r.v[1][0] = -a.v[1][0] / det;
    r.v[1][1] = a.v[0][0] / det;
    return r;
}
Mat2 eye(cd d) {
    Mat2 r{};
    r.v[0][0] = r.v[1][1] = d;
    return r;
}
Mat2 sub(const Mat2& a, const Mat2& b) {
    Mat2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.v[i][j] = a.v[i][j] - b.v[i][j];
    return r;
}
Mat2 scale(const Mat2& a, cd s) {
    Mat2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.v[i][j] = a.v[i][j] * s;
    return r;
}

// H_{Gamma,Sigma} of the left end: rows Gamma = {0, 1}, columns Sigma = {-1, -2}.
Mat2 h_gs(double h) {
    const double w = -0.5 / (h * h);
    Mat2 r{};
    r.v[0][0] = w * kC[1];     // 0 -- -1
    r.v[0][1] = w * kC[2];     // 0 -- -2
    r.v[1][0] = w * kC[2];     // 1 -- -1
    r.v[1][1] = 0.0;           // 1 -- -2: distance 3
    return r;
}
Mat2 transpose(const Mat2& a) {
    Mat2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.v[i][j] = a.v[j][i];
    return r;
}
}  // namespace

bool green5(double h, double s, cd u[2], cd b[2]) {
    const cd a2 = kC[2], a1 = kC[1], a0 = kC[0] - 2.0 * kC[2] + cd(0.0, 2.0 * s * h * h);
    const cd disc = std::sqrt(a1 * a1 - 4.0 * a2 * a0);
    const cd w[2] = {(-a1 + disc) / (2.0 * a2), (-a1 - disc) / (2.0 * a2)};
    for (int q = 0; q < 2; ++q) {
        const cd r = std::sqrt(w[q] * w[q] - 4.0);
        const cd u1 = 0.5 * (w[q] + r), u2 = 0.5 * (w[q] - r);
        u[q] = std::abs(u1) < 1.0 ? u1 : u2;
        if (!(std::abs(u[q]) < 1.0)) return false;
    }
    // the equation at n = 0 and n = 1 for G_n = sum_q b_q u_q^|n|
    std::vector<cd> A(4), B = {1.0, 0.0};
    for (int n = 0; n < 2; ++n)
        for (int q = 0; q < 2; ++q) {
            cd acc = cd(0.0, -s) * std::pow(u[q], n);
            for (int m = -2; m <= 2; ++m) acc += -kC[std::abs(m)] / (2.0 * h * h) * std::pow(u[q], std::abs(n + m));
            A[n * 2 + q] = acc;
        }
    if (!solve(A, B, 2, 1)) return false;
    b[0] = B[0];
    b[1] = B[1];
    return true;
}

cd green5_at(const cd u[2], const cd b[2], int n) {
    const int a = std::abs(n);
    return b[0] * std::pow(u[0], a) + b[1] * std::pow(u[1], a);
}

bool k_block(double h, double s, Mat2& K) {
    cd u[2], b[2];
    if (!green5(h, s, u, b)) return false;
    const int sig[2] = {-1, -2}, gam[2] = {0, 1};
    Mat2 Gsg{}, Gss{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Gsg.v[i][j] = green5_at(u, b, sig[i] - gam[j]);
            Gss.v[i][j] = green5_at(u, b, sig[i] - sig[j]);
        }
    const Mat2 H = h_gs(h), Ht = transpose(H);
    bool ok = true;
    const Mat2 L = inv(sub(eye(1.0), mul(H, Gsg)), ok);
    if (!ok) return false;
    K = scale(mul(L, mul(H, mul(Gss, Ht))), -1.0);
    return true;
}

int build_blocks(const abc1d_params& p, Blocks1D& out, std::string& err) {
    out = Blocks1D{};
    out.order = p.order;
    if (p.order == 0) {
        if (!k_block(p.h, p.s[0], out.K)) { err = "K(s0) failed"; return ABC_ERR_SINGULAR; }
        out.M = out.K;
        return ABC_OK;
    }
    if (p.order == 1) {
        Mat2 K1;
        if (!k_block(p.h, p.s[0], K1)) { err = "K(s1) failed"; return ABC_ERR_SINGULAR; }
        out.K = K1;
        bool ok = true;
        if (p.fit1 == ABC_FIT1_LIMIT) {
            // A = -i H_{Gamma,Sigma} H_{Sigma,Gamma}, B = s1 I - A K1^{-1}
            const Mat2 H = h_gs(p.h);
            out.A = scale(mul(H, transpose(H)), cd(0.0, -1.0));
            const Mat2 Ki = inv(K1, ok);
            if (!ok) { err = "K(s1) singular"; return ABC_ERR_SINGULAR; }
            out.B = sub(eye(p.s[0]), mul(out.A, Ki));
        } else {
            // B (K1 - K2) = s1 K1 - s2 K2, A = (s1 I - B) K1
            Mat2 K2;
            if (!k_block(p.h, p.s[1], K2)) { err = "K(s1b) failed"; return ABC_ERR_SINGULAR; }
            const Mat2 D = inv(sub(K1, K2), ok);
            if (!ok) { err = "K(s1) - K(s1b) singular"; return ABC_ERR_SINGULAR; }
            out.B = mul(sub(scale(K1, p.s[0]), scale(K2, p.s[1])), D);
            out.A = mul(sub(eye(p.s[0]), out.B), K1);
        }
        return ABC_OK;
    }
    // order 2: (s_j^2 I - s_j B1 - B0) K_j = s_j A1 + A0 for the four points, i.e. for
    // each row r: B1[r,:] (s_j K_j) + B0[r,:] K_j + A1[r,:] (s_j I) + A0[r,:] I = s_j^2 K_j[r,:]
    Mat2 Ks[4];
    for (int j = 0; j < 4; ++j)
        if (!k_block(p.h, p.s[j], Ks[j])) { err = "K(s) failed"; return ABC_ERR_SINGULAR; }
    out.K = Ks[0];
    // unknown row vector x (8) = [B1 row | B0 row | A1 row | A0 row]; x M = y with M 8 x 8
    std::vector<cd> Mt(64), Y(16);   // solve M^T x^T = y^T for both rows at once
    for (int j = 0; j < 4; ++j)
        for (int c = 0; c < 2; ++c) {
            const int col = 2 * j + c;
            for (int k = 0; k < 2; ++k) {
                Mt[col * 8 + 0 + k] = p.s[j] * Ks[j].v[k][c];
                Mt[col * 8 + 2 + k] = Ks[j].v[k][c];
                Mt[col * 8 + 4 + k] = k == c ? cd(p.s[j]) : cd(0.0);
                Mt[col * 8 + 6 + k] = k == c ? cd(1.0) : cd(0.0);
            }
            for (int r = 0; r < 2; ++r) Y[col * 2 + r] = p.s[j] * p.s[j] * Ks[j].v[r][c];
        }
    double smin = p.s[0];
    for (int j = 1; j < 4; ++j) smin = std::min(smin, p.s[j]);
    cd X[2][8];
    const int st = fit_order2_end(Mt, Y, -smin, X, err);
    if (st != ABC_OK) return st;
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k) {
            out.B1.v[r][k] = X[r][0 + k];
            out.B0.v[r][k] = X[r][2 + k];
            out.A1.v[r][k] = X[r][4 + k];
            out.A0.v[r][k] = X[r][6 + k];
        }
    return ABC_OK;
}

int check_params(const abc1d_params* p, std::string& err) {
    if (!p) { err = "null params"; return ABC_ERR_ARG; }
    if (p->n < 8 || p->n > ABC1D_MAX_NODES) { err = "n outside [8, ABC1D_MAX_NODES]"; return ABC_ERR_ARG; }
    if (!(p->h > 0)) { err = "h must be positive"; return ABC_ERR_ARG; }
    if (p->order < 0 || p->order > 2) { err = "order must be 0, 1 or 2"; return ABC_ERR_ARG; }
    if (p->precision != ABC_FP64 && p->precision != ABC_C64_FP32) {
        err = "precision must be ABC_FP64 or ABC_C64_FP32";
        return ABC_ERR_ARG;
    }
    const int npts = p->order == 2 ? 4 : (p->order == 1 && p->fit1 == ABC_FIT1_TWO_POINT) ? 2 : 1;
    if (p->order == 1 && p->fit1 != ABC_FIT1_LIMIT && p->fit1 != ABC_FIT1_TWO_POINT) {
        err = "order 1 takes ABC_FIT1_LIMIT or ABC_FIT1_TWO_POINT";
        return ABC_ERR_ARG;
    }
    for (int j = 0; j < npts; ++j) {
        if (!(p->s[j] > 0)) { err = "interpolation points must be positive"; return ABC_ERR_ARG; }
        for (int k = 0; k < j; ++k)
            if (p->s[k] == p->s[j]) { err = "interpolation points must be distinct"; return ABC_ERR_ARG; }
    }
    return ABC_OK;
}

}  // namespace oned
}  // namespace abc
