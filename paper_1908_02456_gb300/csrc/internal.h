// Host-side structures shared by the FP64 setup (setup.cpp, dense.cpp) and the
// device driver (api.cu).  Not part of the ABI.
#pragma once

#include <complex>
#include <string>
#include <vector>

#include "abc.h"

namespace abc {

typedef std::complex<double> cd;

// Index sets of Sec. 2 (eq:25, App. A) for the 3-point stencil, plus the
// decomposition of Gamma under the reflections of the box.
//
// The box is invariant under the three axis reflections i -> n-1-i; they form the
// group Z2^3 (element g: bit a set = reflect axis a).  The DtN map K(s) (eq:17)
// commutes with them because H_{II,II} and H_{II,Gamma} do (V = 0 outside the box),
// so in the basis of parity-adapted combinations of each orbit it splits into 8
// independent blocks, one per character chi_p(g) = (-1)^{popcount(p & g)}.  Each
// orbit is represented by its node in the low octant (2*i <= n-1 per axis); a node
// on a middle plane (odd n) is fixed by that reflection, and only the parities that
// are even on its stabiliser give a basis vector.
struct Geometry {
    int nx = 0, ny = 0, nz = 0;
    double h = 0.0;
    int R = 1;                          // stencil radius per axis (1 or 3)
    double cst[5] = {0, 0, 0, 0, 0};    // second-difference coefficients c_0 .. c_R
    long long n_nodes = 0;
    int n_gamma = 0;
    std::vector<int> gamma_node;        // Gamma index -> linear node index (ascending)
    std::vector<int> node_gamma;        // linear node index -> Gamma index or -1
    std::vector<int> gamma_c;           // number of exterior nodes coupled to the node (1..3 for R = 1)
    int n_rep = 0;
    std::vector<int> rep_node;          // representative -> linear node index
    std::vector<int> rep_gamma;         // [n_rep][8] Gamma index of g.r
    std::vector<int> rep_adapted;       // [n_rep][8] adapted index of parity p, or -1
    std::vector<int> rep_stab;          // |stabiliser of r| (1, 2, 4 or 8)
    int m[8] = {0}, off[8] = {0};       // block sizes / offsets in adapted numbering
    std::vector<int> adapted_rep;       // adapted index -> representative
    // Axis-permutation classes (cubes only).  A permutation pi of the axes maps the
    // parity-p basis onto the parity-pi(p) basis and commutes with K, so blocks whose
    // parities have the same number of odd axes are equal once their representatives
    // are numbered consistently (local index of r in block pi(b) = local index of
    // pi^{-1}(r) in block b).  base_of[p] is the block that stores the matrix of p.
    bool cube = false;
    int base_of[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    int perm_of[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // index in kAxisPerms with pi(base_of[p]) = p

    // Irreducible blocks.  Inside stored block b the axis permutations that fix b
    // (all six for b = 0 and 7, one transposition for the others, none on a
    // non-cube) permute the representatives and commute with K, so in a real
    // orthogonal basis adapted to their irreducible representations rho the block
    // splits again (Schur's lemma): one m x m matrix per (b, rho), the same for
    // every component of rho.  A class applies it to R = (parities of b's class) x
    // dim(rho) right-hand sides stored at adapted offsets moff[0..R-1] (index
    // member * dim + component).  Columns of the basis change W_b: for component a
    // and copy c, up to 6 (local index in block b, weight) pairs at
    // [(a * m + c) * 6 + i]; unused pairs have local index -1.
    struct IrrepClass {
        int base = 0, irrep = 0, dim = 1, m = 0, R = 0;
        int moff[3] = {0, 0, 0};
        std::vector<int> col_l;
        std::vector<double> col_w;
    };
    std::vector<IrrepClass> cls;
    // Cells: orbits of representatives under all axis permutations (cubes) or single
    // representatives.  The device transforms run cell by cell: parity components
    // of the cell's representatives (slots) in, adapted values out.
    int n_cells = 0;
    std::vector<int> cell_rep;      // [n_cells][8] representative per slot, -1 unused
    std::vector<int> cell_out;      // [n_cells][8 outputs][8 parities] adapted index or -1
    std::vector<int> cell_type;     // [n_cells][8 parities] coefficient matrix id
    std::vector<double> coef;       // [types][8 outputs][8 slots]: output = sum coef * slot value
    std::vector<int> cell_c;        // exterior-neighbour count of the cell's nodes (1..3)
    // Flattened tables of the device transforms, thread t = 8 slot + g of a cell:
    std::vector<int> cell_gi;       // [n_cells][64] Gamma index of reflection g of the slot, -1 unused
    std::vector<int> cell_node;     // [n_cells][64] its linear node index, -1 unused
    std::vector<int> cell_wr;       // [n_cells][64] Gamma index if lane g is the lowest lane of the
                                    //   slot reaching that node (the one that writes it), else -1
    // coefficient matrices with the parity-basis scale of each slot folded in:
    std::vector<double> coef_f;     // [types][8 o][8 s] = coef[o][s] / sqrt(8 |H_s|)   (forward)
    std::vector<double> coef_bt;    // [types][8 s][8 o] = coef[o][s] * sqrt(|H_s| / 8)  (back, transposed)
};

// Axis permutations: (pi . x)[kAxisPerms[pi][a]] = x[a]; the same map moves parity bit a
// to bit kAxisPerms[pi][a].  Entry 0 is the identity.
extern const int kAxisPerms[6][3];

// Irreducible blocks and cells of a geometry whose parity blocks are built.
int build_irreps(Geometry& g, std::string& err);

// Closed-form Gamma index of a boundary node (ascending linear order).
int gamma_index_closed(int i, int j, int k, int nx, int ny, int nz, int R = 1);

int build_geometry(int nx, int ny, int nz, double h, Geometry& g, std::string& err, int R = 1);

// FP64 coefficient blocks in the symmetry-adapted basis, one per irreducible class
// (row-major m x m each):
//   order 0: mat[k] = M_k = K_k(s0)
//   order 1: mat[k] = S_k = K_k(s1)^{-1}; B = s1 I - A S with A diagonal
// Both are complex symmetric.
struct Blocks {
    int order = 0;
    int fit = 0;          // order 1: ABC_FIT1_*
    bool rows1 = false;   // order 1 held as general class rows [B | A] in mat2[0], mat2[1]
                          // (the two-point and Hermite fits; every fit when R > 1, where
                          // A = -i H_{Gamma,II} H_{II,Gamma} is not diagonal)
    double s = 0.0, s1b = 0.0;
    std::vector<std::vector<cd>> mat;
    // order 2: per class the four coefficient blocks B1, B0, A1, A0; order 1 with a
    // two-point or Hermite fit: B, A in mat2[0], mat2[1] (row-major m x m, general
    // complex); and the interpolation points
    std::vector<std::vector<cd>> mat2[4];
    double s2[4] = {0, 0, 0, 0};
};

// Order-2 coefficients (Sec. 3.3): per class, K_k(s_j) at the four points by the
// order-0 route, then [B1 B0 A1 A0] from s_j^2 K_j = s_j B1 K_j + B0 K_j + s_j A1 + A0.
int compute_blocks2(const Geometry& g, const double s[4], Blocks& b, std::string& err);

// Dense block-b matrix (row-major m_b x m_b, parity-adapted numbering) from the
// irreducible blocks whose base is b: sum over classes and components of W blk W^T.
void expand_base_block(const Geometry& g, int b, const std::vector<std::vector<cd>>& blk, std::vector<cd>& out);

// Class blocks of K(s) (order 0: M = K(s); order 1: S = K(s)^{-1}).  dK (order 0 only):
// also the class blocks of K'(s) = dK/ds, row-major.  HH: also the class blocks of
// H_{Gamma,II} H_{II,Gamma} (real symmetric).
int compute_blocks(const Geometry& g, int order, double s, Blocks& b, std::string& err,
                   std::vector<std::vector<cd>>* dK = nullptr, std::vector<std::vector<cd>>* HH = nullptr);

// Order-1 coefficients fitted by two finite points or by value and derivative
// (ABC_FIT1_TWO_POINT / ABC_FIT1_HERMITE): per class B (mat2[0]) and A (mat2[1]).
int compute_blocks_fit1(const Geometry& g, int fit, double s1, double s1b, Blocks& b, std::string& err);

// The blocks a parameter set asks for (dispatch on order and fit).
int compute_param_blocks(const Geometry& g, const abc_params& p, Blocks& b, std::string& err);

// Dense natural-order (row-major n_gamma^2) reconstruction of ABC_MAT_* from blocks.
int dense_natural(const Geometry& g, const Blocks& b, int which, cd* out, std::string& err);

// Free lattice Green's function table G(|dx|,|dy|,|dz|) = [(H_0 - i s)^{-1}](dx,dy,dz)
// for 0 <= |d| < dims[a] with the geometry's (2R + 1)-point stencil and spacing;
// layout [(c*dy)+b]*dx + a.  deriv: dG/ds instead (= i G^2).
void free_green_table(const Geometry& g, double s, int dx, int dy, int dz, std::vector<cd>& table,
                      bool deriv = false);

// Dense complex LU with partial pivoting (column-major), and the solve with many
// right-hand sides.  Return 0, or k+1 if U(k,k) == 0.
int zgetrf(int n, cd* A, int lda, int* ipiv);
void zgetrs(int n, int nrhs, const cd* A, int lda, const int* ipiv, cd* B, int ldb);
// Column-pivoted Householder QR of a square A (column-major, overwritten) and the basic
// solution of A Z = B at numerical rank r = the number of pivots above abs_tol (the free
// unknowns set to zero); Z overwrites B.  Returns 0.
int zqrp_basic(int n, int nrhs, cd* A, int lda, cd* B, int ldb, double abs_tol, int* rank);
// C -= A * B (column-major, m x k times k x n)
void zgemm_sub(int m, int n, int k, const cd* A, int lda, const cd* B, int ldb, cd* C, int ldc);

}  // namespace abc
