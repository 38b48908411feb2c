// Symmetry-adapted basis of the boundary beyond the reflection parities (host, FP64).
//
// The box's lattice symmetries commute with the exterior operator H_{II,II} and
// with H_{II,Gamma} (V = 0 outside, Sec. 2), hence with the DtN map K(s) of eq:17
// and with everything built from it (M, S = K^{-1}, the eq:eval matrices).  The
// reflections Z2^3 are handled by the parity blocks (setup.cpp).  On a cube the six
// axis permutations are symmetries too; together with the reflections they form
// the full symmetry group of the cube (48 elements).  A permutation pi maps parity
// block b onto block pi(b) (used by the permutation classes), and the permutations
// with pi(b) = b act on block b by permuting its representatives, without signs.
// Here that action is decomposed into real irreducible representations:
//   all six permutations (b = 0, 7): trivial, sign, two-dimensional standard;
//   one transposition (the other b): trivial, sign;
//   none (non-cube): trivial.
// For an orbit with anchor A and stabiliser H_A, representation rho (dimension d)
// occurs once per vector u of an orthonormal basis of the H_A-fixed space of rho,
// with basis vectors (component a = 0..d-1)
//   w_a = sqrt(d |H_A| / |H|) sum over orbit nodes h.A of (D_rho(h) u)_a e_{h.A}.
// These transform by the same matrices D_rho in every orbit, so by Schur's lemma
// the block is, in this basis, a direct sum of I_d (x) K_rho over rho.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"

namespace abc {

namespace {

void apply_perm(const int* P, const int* co, int* out) {
    for (int a = 0; a < 3; ++a) out[P[a]] = co[a];
}

int perm_bits(const int* P, int b) {
    int img = 0;
    for (int a = 0; a < 3; ++a)
        if (b >> a & 1) img |= 1 << P[a];
    return img;
}

int perm_sign(const int* P) {
    int inv = 0;
    for (int a = 0; a < 3; ++a)
        for (int c = a + 1; c < 3; ++c) inv += P[a] > P[c];
    return (inv & 1) ? -1 : 1;
}

// D_rho(P): rho = 0 trivial, 1 sign, 2 standard (on the plane orthogonal to (1,1,1)
// with orthonormal basis f0 = (1,-1,0)/sqrt2, f1 = (1,1,-2)/sqrt6; P moves axis a to
// axis P[a]).
void irrep_matrix(int rho, const int* P, double D[2][2]) {
    D[0][0] = 1.0; D[0][1] = D[1][0] = D[1][1] = 0.0;
    if (rho == 1) D[0][0] = perm_sign(P);
    if (rho != 2) return;
    const double s2 = 1.0 / std::sqrt(2.0), s6 = 1.0 / std::sqrt(6.0);
    const double f[2][3] = {{s2, -s2, 0.0}, {s6, s6, -2.0 * s6}};
    for (int b = 0; b < 2; ++b) {
        double pf[3];
        for (int a = 0; a < 3; ++a) pf[P[a]] = f[b][a];
        for (int a = 0; a < 2; ++a) D[a][b] = f[a][0] * pf[0] + f[a][1] * pf[1] + f[a][2] * pf[2];
    }
}

int irrep_dim(int rho) { return rho == 2 ? 2 : 1; }

}  // namespace

int build_irreps(Geometry& g, std::string& err) {
    const int nx = g.nx, ny = g.ny;
    std::vector<int> node_rep((size_t)g.n_nodes, -1);
    for (int r = 0; r < g.n_rep; ++r) node_rep[g.rep_node[r]] = r;
    auto coords = [&](int r, int* co) {
        const int node = g.rep_node[r];
        co[0] = node % nx; co[1] = (node / nx) % ny; co[2] = node / (nx * ny);
    };
    auto rep_at = [&](const int* co) { return node_rep[((size_t)co[2] * ny + co[1]) * nx + co[0]]; };
    auto permuted_rep = [&](int k, int r) {
        int co[3], pc[3];
        coords(r, co);
        apply_perm(kAxisPerms[k], co, pc);
        return rep_at(pc);
    };

    g.cls.clear();
    for (int b = 0; b < 8; ++b) {
        if (g.base_of[b] != b || g.m[b] == 0) continue;
        const int mb = g.m[b];
        std::vector<int> H;
        for (int k = 0; k < 6; ++k)
            if (k == 0 || (g.cube && perm_bits(kAxisPerms[k], b) == b)) H.push_back(k);
        const int nH = (int)H.size();
        const int n_irr = nH == 6 ? 3 : (nH == 2 ? 2 : 1);
        if (nH != 1 && nH != 2 && nH != 6) { err = "internal: unexpected stabiliser of a parity block"; return ABC_ERR_ARG; }
        // columns per irrep and component: entries (local index, weight)
        struct Col { int l[6]; double w[6]; };
        std::vector<Col> cols[3][2];
        std::vector<char> seen(mb, 0);
        for (int l0 = 0; l0 < mb; ++l0) {
            if (seen[l0]) continue;
            const int A = g.adapted_rep[g.off[b] + l0];
            int lh[6];
            std::vector<int> orbit;
            for (int i = 0; i < nH; ++i) {
                const int r = permuted_rep(H[i], A);
                const int q = r < 0 ? -1 : g.rep_adapted[(size_t)r * 8 + b];
                if (q < 0) { err = "internal: permutation leaves the parity block"; return ABC_ERR_ARG; }
                lh[i] = q - g.off[b];
                if (std::find(orbit.begin(), orbit.end(), lh[i]) == orbit.end()) orbit.push_back(lh[i]);
            }
            for (int l : orbit) seen[l] = 1;
            int n_stab = 0;
            for (int i = 0; i < nH; ++i) n_stab += lh[i] == l0;
            for (int rho = 0; rho < n_irr; ++rho) {
                const int d = irrep_dim(rho);
                double P[2][2] = {{0, 0}, {0, 0}};
                for (int i = 0; i < nH; ++i) {
                    if (lh[i] != l0) continue;
                    double D[2][2];
                    irrep_matrix(rho, kAxisPerms[H[i]], D);
                    for (int a = 0; a < d; ++a)
                        for (int c = 0; c < d; ++c) P[a][c] += D[a][c] / n_stab;
                }
                // orthonormal basis of the fixed space (range of the projector P)
                std::vector<std::array<double, 2>> us;
                const int rank = (int)std::lround(d == 1 ? P[0][0] : P[0][0] + P[1][1]);
                if (rank == d) {
                    for (int c = 0; c < d; ++c) us.push_back({c == 0 ? 1.0 : 0.0, c == 1 ? 1.0 : 0.0});
                } else if (rank == 1) {                       // d = 2, projector u u^T
                    const int c = (P[0][0] >= P[1][1]) ? 0 : 1;
                    const double nrm = std::sqrt(P[0][c] * P[0][c] + P[1][c] * P[1][c]);
                    us.push_back({P[0][c] / nrm, P[1][c] / nrm});
                }
                const double c0 = std::sqrt((double)d * n_stab / nH);
                for (const auto& u : us) {
                    for (int a = 0; a < d; ++a) {
                        Col col;
                        for (int i = 0; i < 6; ++i) { col.l[i] = -1; col.w[i] = 0.0; }
                        int n = 0;
                        for (int i = 0; i < nH; ++i) {
                            double D[2][2];
                            irrep_matrix(rho, kAxisPerms[H[i]], D);
                            const double w = c0 * (D[a][0] * u[0] + (d == 2 ? D[a][1] * u[1] : 0.0));
                            int k = 0;
                            while (k < n && col.l[k] != lh[i]) ++k;
                            if (k < n) {
                                if (std::fabs(col.w[k] - w) > 1e-12) { err = "internal: irrep basis inconsistent"; return ABC_ERR_ARG; }
                                continue;
                            }
                            col.l[n] = lh[i];
                            col.w[n] = w;
                            ++n;
                        }
                        cols[rho][a].push_back(col);
                    }
                }
            }
        }
        int nmem = 0;
        for (int p = 0; p < 8; ++p) nmem += g.base_of[p] == b;
        for (int rho = 0; rho < n_irr; ++rho) {
            const int d = irrep_dim(rho);
            const int m = (int)cols[rho][0].size();
            if (m == 0) continue;
            Geometry::IrrepClass k;
            k.base = b;
            k.irrep = rho;
            k.dim = d;
            k.m = m;
            k.R = nmem * d;
            if (k.R > 3) { err = "internal: more than 3 right-hand sides in a class"; return ABC_ERR_ARG; }
            k.col_l.assign((size_t)d * m * 6, -1);
            k.col_w.assign((size_t)d * m * 6, 0.0);
            for (int a = 0; a < d; ++a)
                for (int c = 0; c < m; ++c)
                    for (int i = 0; i < 6; ++i) {
                        const double w = cols[rho][a][c].w[i];
                        const bool keep = cols[rho][a][c].l[i] >= 0 && std::fabs(w) > 1e-15;
                        k.col_l[((size_t)a * m + c) * 6 + i] = keep ? cols[rho][a][c].l[i] : -1;
                        k.col_w[((size_t)a * m + c) * 6 + i] = keep ? w : 0.0;
                    }
            g.cls.push_back(std::move(k));
        }
    }
    // adapted offsets: classes in order, then member parity, then component
    int acc = 0;
    for (auto& k : g.cls)
        for (int e = 0; e < k.R; ++e) { k.moff[e] = acc; acc += k.m; }
    if (acc != g.n_gamma) { err = "internal: irreducible blocks do not cover Gamma"; return ABC_ERR_ARG; }

    // cells
    std::vector<int> cell_of(g.n_rep, -1), slot_of(g.n_rep, -1);
    g.cell_rep.clear();
    int nc = 0;
    for (int r = 0; r < g.n_rep; ++r) {
        if (cell_of[r] >= 0) continue;
        std::vector<int> mem{r};
        if (g.cube)
            for (int k = 1; k < 6; ++k) {
                const int r2 = permuted_rep(k, r);
                if (r2 < 0) { err = "internal: permuted representative missing"; return ABC_ERR_ARG; }
                if (std::find(mem.begin(), mem.end(), r2) == mem.end()) mem.push_back(r2);
            }
        for (int s = 0; s < 8; ++s) g.cell_rep.push_back(s < (int)mem.size() ? mem[s] : -1);
        for (int s = 0; s < (int)mem.size(); ++s) { cell_of[mem[s]] = nc; slot_of[mem[s]] = s; }
        ++nc;
    }
    g.n_cells = nc;
    g.cell_out.assign((size_t)nc * 64, -1);
    std::vector<double> mats((size_t)nc * 8 * 64, 0.0);
    std::vector<int> cnt((size_t)nc * 8, 0);
    for (const auto& k : g.cls) {
        std::vector<int> mem;
        for (int p = 0; p < 8; ++p)
            if (g.base_of[p] == k.base) mem.push_back(p);
        for (int e = 0; e < k.R; ++e) {
            const int p = mem[e / k.dim], a = e % k.dim;
            const int perm = g.perm_of[p];
            for (int c = 0; c < k.m; ++c) {
                int cell = -1;
                int slots[6], nsl = 0;
                double ws[6];
                for (int i = 0; i < 6; ++i) {
                    const int l = k.col_l[((size_t)a * k.m + c) * 6 + i];
                    if (l < 0) continue;
                    const int r = g.adapted_rep[g.off[k.base] + l];
                    const int r2 = permuted_rep(perm, r);
                    if (r2 < 0 || g.rep_adapted[(size_t)r2 * 8 + p] < 0) { err = "internal: member parity missing"; return ABC_ERR_ARG; }
                    if (cell >= 0 && cell_of[r2] != cell) { err = "internal: basis vector spans two cells"; return ABC_ERR_ARG; }
                    cell = cell_of[r2];
                    slots[nsl] = slot_of[r2];
                    ws[nsl++] = k.col_w[((size_t)a * k.m + c) * 6 + i];
                }
                if (cell < 0) { err = "internal: empty basis vector"; return ABC_ERR_ARG; }
                int& o = cnt[(size_t)cell * 8 + p];
                if (o >= 8) { err = "internal: too many outputs in a cell"; return ABC_ERR_ARG; }
                g.cell_out[((size_t)cell * 8 + o) * 8 + p] = k.moff[e] + c;
                for (int i = 0; i < nsl; ++i) mats[(((size_t)cell * 8 + p) * 8 + o) * 8 + slots[i]] = ws[i];
                ++o;
            }
        }
    }
    g.cell_c.assign(nc, 0);
    for (int cidx = 0; cidx < nc; ++cidx) {
        for (int p = 0; p < 8; ++p) {
            int exist = 0;
            for (int s = 0; s < 8; ++s) {
                const int r = g.cell_rep[(size_t)cidx * 8 + s];
                if (r >= 0 && g.rep_adapted[(size_t)r * 8 + p] >= 0) ++exist;
            }
            if (exist != cnt[(size_t)cidx * 8 + p]) { err = "internal: cell outputs do not match its components"; return ABC_ERR_ARG; }
        }
        const int c0 = g.gamma_c[g.node_gamma[g.rep_node[g.cell_rep[(size_t)cidx * 8]]]];
        for (int s = 1; s < 8; ++s) {
            const int r = g.cell_rep[(size_t)cidx * 8 + s];
            if (r >= 0 && g.gamma_c[g.node_gamma[g.rep_node[r]]] != c0) { err = "internal: cell mixes boundary types"; return ABC_ERR_ARG; }
        }
        g.cell_c[cidx] = c0;
    }
    // distinct coefficient matrices (with the slots' parity-basis scales folded in)
    std::map<std::vector<double>, int> ids;
    g.cell_type.assign((size_t)nc * 8, 0);
    g.coef.clear();
    g.coef_f.clear();
    g.coef_bt.clear();
    for (size_t cp = 0; cp < (size_t)nc * 8; ++cp) {
        const size_t cell = cp / 8;
        std::vector<double> key(mats.begin() + cp * 64, mats.begin() + cp * 64 + 64);
        double stab[8];
        for (int sl = 0; sl < 8; ++sl) {
            const int r = g.cell_rep[cell * 8 + sl];
            stab[sl] = r >= 0 ? (double)g.rep_stab[r] : 1.0;
            key.push_back(stab[sl]);
        }
        auto it = ids.find(key);
        if (it == ids.end()) {
            it = ids.emplace(key, (int)ids.size()).first;
            g.coef.insert(g.coef.end(), key.begin(), key.begin() + 64);
            for (int o = 0; o < 8; ++o)
                for (int sl = 0; sl < 8; ++sl) g.coef_f.push_back(key[o * 8 + sl] / std::sqrt(8.0 * stab[sl]));
            for (int sl = 0; sl < 8; ++sl)
                for (int o = 0; o < 8; ++o) g.coef_bt.push_back(key[o * 8 + sl] * std::sqrt(stab[sl] / 8.0));
        }
        g.cell_type[cp] = it->second;
    }
    // flattened node tables
    g.cell_gi.assign((size_t)nc * 64, -1);
    g.cell_node.assign((size_t)nc * 64, -1);
    g.cell_wr.assign((size_t)nc * 64, -1);
    for (int cidx = 0; cidx < nc; ++cidx)
        for (int sl = 0; sl < 8; ++sl) {
            const int r = g.cell_rep[(size_t)cidx * 8 + sl];
            if (r < 0) continue;
            for (int gg = 0; gg < 8; ++gg) {
                const int gi = g.rep_gamma[(size_t)r * 8 + gg];
                const size_t e = (size_t)cidx * 64 + sl * 8 + gg;
                g.cell_gi[e] = gi;
                g.cell_node[e] = g.gamma_node[gi];
                bool first = true;
                for (int g2 = 0; g2 < gg; ++g2) first &= g.rep_gamma[(size_t)r * 8 + g2] != gi;
                g.cell_wr[e] = first ? gi : -1;
            }
        }
    return ABC_OK;
}

void expand_base_block(const Geometry& g, int b, const std::vector<std::vector<cd>>& blk, std::vector<cd>& out) {
    const int mb = g.m[b];
    out.assign((size_t)mb * mb, cd(0.0, 0.0));
    for (size_t ki = 0; ki < g.cls.size(); ++ki) {
        const auto& k = g.cls[ki];
        if (k.base != b) continue;
        const int m = k.m;
        for (int a = 0; a < k.dim; ++a)
            for (int c = 0; c < m; ++c) {
                const int* li = &k.col_l[((size_t)a * m + c) * 6];
                const double* wi = &k.col_w[((size_t)a * m + c) * 6];
                for (int c2 = 0; c2 < m; ++c2) {
                    const cd v = blk[ki][(size_t)c * m + c2];
                    const int* lj = &k.col_l[((size_t)a * m + c2) * 6];
                    const double* wj = &k.col_w[((size_t)a * m + c2) * 6];
                    for (int i = 0; i < 6; ++i) {
                        if (li[i] < 0) continue;
                        for (int j = 0; j < 6; ++j) {
                            if (lj[j] < 0) continue;
                            out[(size_t)li[i] * mb + lj[j]] += wi[i] * wj[j] * v;
                        }
                    }
                }
            }
    }
}

}  // namespace abc
