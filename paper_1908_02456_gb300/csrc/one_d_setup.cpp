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
    if (!solve(Mt, Y, 8, 2)) { err = "order-2 interpolation system singular"; return ABC_ERR_SINGULAR; }
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k) {
            out.B1.v[r][k] = Y[(0 + k) * 2 + r];
            out.B0.v[r][k] = Y[(2 + k) * 2 + r];
            out.A1.v[r][k] = Y[(4 + k) * 2 + r];
            out.A0.v[r][k] = Y[(6 + k) * 2 + r];
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
    if (p->order == 2 && p->precision != ABC_FP64) {
        // the second-order blocks at close interpolation points carry large, cancelling
        // entries: FP32 loses the result (measured 6e-2 relative after 2000 steps)
        err = "the 1D second-order ABC needs ABC_FP64";
        return ABC_ERR_UNSUPPORTED;
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
