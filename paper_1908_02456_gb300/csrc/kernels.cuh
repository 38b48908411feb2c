// Device kernels of the time-stepper (sm_103a).  Templated on the real type T
// (float for the complex64 forms, double for the FP64 form); complex values are
// interleaved (re, im) pairs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace abc {
namespace dev {

// Programmatic dependent launch: wait until the preceding kernel of the stream has
// completed and its writes are visible (a no-op without a programmatic dependency),
// and allow the next kernel to be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 t; };
template <> struct C2<double> { typedef double2 t; };

template <typename T> __device__ __forceinline__ typename C2<T>::t mk(T re, T im) {
    typename C2<T>::t v; v.x = re; v.y = im; return v;
}

// The adapted input of an order-1 back transform, x = s1 f + (-i a)(p - t), with one
// fixed rounding order (every form of the back transform and the contraction epilogue
// that can form it give the same bits): re = fma(s1, f.re, a di), im = fma(s1, f.im,
// -(a dr)), d = p - t.
__device__ __forceinline__ float2 back_x1(float s1, float a, float2 f, float2 p, float2 t) {
    const float dr = __fsub_rn(p.x, t.x), di = __fsub_rn(p.y, t.y);
    return make_float2(__fmaf_rn(s1, f.x, __fmul_rn(a, di)), __fmaf_rn(s1, f.y, -__fmul_rn(a, dr)));
}
__device__ __forceinline__ double2 back_x1(double s1, double a, double2 f, double2 p, double2 t) {
    const double dr = __dsub_rn(p.x, t.x), di = __dsub_rn(p.y, t.y);
    return make_double2(__fma_rn(s1, f.x, __dmul_rn(a, di)), __fma_rn(s1, f.y, -__dmul_rn(a, dr)));
}

// Block structure of the symmetry-adapted boundary matrices (kernel parameter).
// Entry e is one right-hand side of one irreducible class: the class's matrix
// (m x m at mat_off, row stride ld) maps adapted indices [off, off + m) to the same
// range.  Entries of one class share mat_off.
constexpr int MAX_ENTRIES = 24;
struct BlockInfo {
    int n;                            // number of entries
    int nseg;                         // input segments per row: 1, or 4 for order 2 ([B1 | B0 - iA1 | -iA1 | A0])
    int m[MAX_ENTRIES];               // block sizes
    int off[MAX_ENTRIES];             // first adapted index of each entry (ascending)
    int ld[MAX_ENTRIES];              // row stride (complex elements) of the matrix
    int segw[MAX_ENTRIES];            // stride of the segments inside a row (multiple of 4)
    long long mat_off[MAX_ENTRIES];   // first element of the matrix in the buffer
};

// The same blocks by irreducible class: class c owns the thread blocks rowbase[c] ..
// rowbase[c+1]-1 (GEMV_RB block rows each) and applies its block to its R right-hand
// sides, which start at adapted offsets moff[c][k].
constexpr int MAX_CLASSES = 16;
struct ClassInfo {
    int n;                            // classes
    int R[MAX_CLASSES];
    int m[MAX_CLASSES];
    int moff[MAX_CLASSES][3];
    int ld[MAX_CLASSES];
    int segw[MAX_CLASSES];
    long long mat_off[MAX_CLASSES];
    int rowbase[MAX_CLASSES + 1];     // first block of each class (ceil(m / GEMV_RB) blocks per class)
};

// Input vectors of the contraction: segment q of a row multiplies x.p[q] (adapted,
// orbital-major); only p[0] is used when nseg = 1.
template <typename V>
struct XSeg {
    const V* p[4];
};

// Cell tables of the boundary transforms (kernel parameter).  A cell is a set of
// representatives closed under the axis permutations (one representative on a
// non-cube); its slots hold the representatives, and for every parity p its
// adapted outputs are out[o] = sum_s coef[o][s] * (parity-p component of slot s).
// Thread t = 8 s + g of a cell's group reads entry t of the node tables.
template <typename T>
struct CellTab {
    int n_cells;
    int ng;                // adapted vectors are orbital-major: element (j, orbital) at orbital * ng + j
    int n_gamma;           // natural boundary vectors: [n_gamma][n_orb]
    const int* out;        // [n_cells][8 o][8 p] adapted index or -1
    const int* type;       // [n_cells][8 p] coefficient matrix id
    const T* coef_f;       // [types][8 o][8 s] forward coefficients, slot scale folded in
    const T* coef_bt;      // [types][8 s][8 o] back coefficients (transposed), slot scale folded in
    const int* cell_c;     // [n_cells] exterior-neighbour count
    const int* gi;         // [n_cells][64] Gamma index of reflection g of slot s, -1 unused
    const int* node;       // [n_cells][64] its linear node index
    const int* wr;         // [n_cells][64] Gamma index written by lane g of slot s, -1 if none
};

// Partial sums of the tiled one-orbital contraction, gathered by the back transform:
// t[j] = sum of the row parts of the segments of (class c, tile row I) + the column
// parts of the tiles (c, K, I), K > I (fixed order).  desc is indexed like the cell
// output table (cell * 64 + 8 o + p): x = row-part element of the first segment and
// warp 0 (the SYM_GATHER_WARPS warps' partials are 192 elements apart), y = number of row
// segments (consecutive, 192 * SYM_GATHER_WARPS elements apart), z = column-part element
// of K = I + 1,
// w = (number of K) | ((I + 2) << 16); the column-part element of K + 1 is that of K
// plus (K + 1) * 192.
// Row partials per segment of the tiled contraction: one per consumer warp (equal to
// its SYM_CONSUMERS, checked where both are visible).
constexpr int SYM_GATHER_WARPS = 8;

struct SymGather {
    const int4* desc;
    const float2* rowpart;       // [segment][SYM_GATHER_WARPS warps][3][64]
    const float2* colpart;       // [tile][3][64]
};

// Gamma index of a boundary node (Gamma = nodes within R of a face, ascending linear
// order, x fastest): the first and last R planes z are entirely on Gamma; a middle
// plane contributes its first and last R rows and the first and last R nodes of every
// other row.
template <int R = 1>
__device__ __forceinline__ int gamma_index(int i, int j, int k, int nx, int ny, int nz) {
    const int full = nx * ny, mid_rows = ny - 2 * R;
    const int plane = 2 * R * nx + mid_rows * 2 * R;
    if (k < R) return k * full + j * nx + i;
    if (k >= nz - R) return R * full + (nz - 2 * R) * plane + (k - (nz - R)) * full + j * nx + i;
    const int base = R * full + (k - R) * plane;
    if (j < R) return base + j * nx + i;
    if (j >= ny - R) return base + R * nx + mid_rows * 2 * R + (j - (ny - R)) * nx + i;
    return base + R * nx + (j - R) * 2 * R + (i < R ? i : R + (i - (nx - R)));
}

// Second-difference coefficients c_1 .. c_R of the (2R + 1)-point formula (c_0 enters
// through the diagonal -1/2 * 3 c_0 / h^2): R = 1: (1); R = 3: (3/2, -3/20, 1/90), the
// "7-point scheme in each direction" of Sec. 4.2.
template <int R> __device__ __forceinline__ double stencil_c(int m);
template <> __device__ __forceinline__ double stencil_c<1>(int) { return 1.0; }
template <> __device__ __forceinline__ double stencil_c<3>(int m) {
    return m == 1 ? 1.5 : m == 2 ? -0.15 : 1.0 / 90.0;
}
template <int R> __device__ __forceinline__ double stencil_c0() { return R == 1 ? -2.0 : -49.0 / 18.0; }

// True when the node lies within R of a face (on Gamma).
template <int R>
__device__ __forceinline__ bool on_gamma(int i, int j, int k, int nx, int ny, int nz) {
    return i < R || i >= nx - R || j < R || j >= ny - R || k < R || k >= nz - R;
}

// (H_{I,I} w)(node) = -1/(2h^2) [3 c_0 w + sum over axes and 1 <= m <= R of c_m (w(+m) +
// w(-m))] + V w, the neighbours outside the box omitted (eq:22, eq:32).  Sums in S.
template <typename S, int R, typename V>
__device__ __forceinline__ void apply_h(const V* wo, long long n, int i, int j, int k, int nx, int ny, int nz,
                                        S inv_h2, S vpot, V c, S& hr, S& hi) {
    const long long sy = nx, sz = (long long)nx * ny;
    S sr = 0, si = 0;
#pragma unroll
    for (int m = 1; m <= R; ++m) {
        S ar = 0, ai = 0;
        if (i >= m) { const V v = wo[n - m]; ar += v.x; ai += v.y; }
        if (i < nx - m) { const V v = wo[n + m]; ar += v.x; ai += v.y; }
        if (j >= m) { const V v = wo[n - m * sy]; ar += v.x; ai += v.y; }
        if (j < ny - m) { const V v = wo[n + m * sy]; ar += v.x; ai += v.y; }
        if (k >= m) { const V v = wo[n - m * sz]; ar += v.x; ai += v.y; }
        if (k < nz - m) { const V v = wo[n + m * sz]; ar += v.x; ai += v.y; }
        if (R == 1) {
            sr = ar;
            si = ai;
        } else {
            sr += (S)stencil_c<R>(m) * ar;
            si += (S)stencil_c<R>(m) * ai;
        }
    }
    const S diag = (S)(-1.5 * stencil_c0<R>()) * inv_h2 + vpot;
    hr = diag * c.x - (S)0.5 * inv_h2 * sr;
    hi = diag * c.y - (S)0.5 * inv_h2 * si;
}

// 8-point Walsh-Hadamard transform across the 8 lanes of an aligned lane group:
// lane g holds in[g] and receives out[g] = sum_h (-1)^{popcount(g&h)} in[h].
template <typename V> __device__ __forceinline__ V wht8_lanes(V v, int g) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
        const decltype(v.x) ox = __shfl_xor_sync(0xffffffffu, v.x, bit);
        const decltype(v.y) oy = __shfl_xor_sync(0xffffffffu, v.y, bit);
        if (g & bit) { v.x = ox - v.x; v.y = oy - v.y; }
        else { v.x = v.x + ox; v.y = v.y + oy; }
    }
    return v;
}

// --------------------------------------------------------------------------
// Boundary: natural Gamma order <-> symmetry-adapted order
// --------------------------------------------------------------------------
// Launch with 128 threads per block: two groups of 64 threads, one group per (cell,
// orbital j), orbital fastest.  In a group thread t = 8 s + g; every table load of a
// thread is issued before its first data load.
//
// Forward: thread (s, g) gathers the value at the reflection g of slot s's
// representative; the 8-lane group of the slot transforms them (Walsh-Hadamard),
// which leaves parity component g in lane g (unscaled); after the exchange through
// shared memory thread (o, p) = (s, g) forms adapted output o of parity p with the
// scaled coefficients.
//   MODE 0: hat_phi (and hat_f when w_f is given)
//   MODE 1: hat_phi, hat_f and u = (+i a_coef c) hat_f  (order-1 adjoint, A^H f)
//   MODE 2: order 2: hat_phi, hat_f, and (in o2) the transforms of H_{I,I} w_phi at the
//           boundary nodes (hat_h) and of the g part of the auxiliary state (hat_g)
// Order-2 data (MODE 2 only).
template <typename T>
struct Ord2Fwd {
    const typename C2<T>::t* w_g;   // g part of the stage input, natural [n_gamma][n_orb]
    const T* V;                      // potential [nz][ny][nx]
    typename C2<T>::t* hat_h;
    typename C2<T>::t* hat_g;
    int nx, ny, nz;
    T inv_h2;
    int R;                           // stencil radius (1 or 3)
};

// EARLY: the kernel lets its programmatic dependent (the one-orbital tiled contraction)
// launch as soon as it starts.
template <typename T, int MODE, bool EARLY = false>
__global__ void __launch_bounds__(128) bnd_forward(CellTab<T> ct, int n_orb, long long nvox,
                                                   const typename C2<T>::t* __restrict__ w_phi,
                                                   const typename C2<T>::t* __restrict__ w_f,
                                                   typename C2<T>::t* __restrict__ hat_phi,
                                                   typename C2<T>::t* __restrict__ hat_f,
                                                   typename C2<T>::t* __restrict__ u, T a_coef, Ord2Fwd<T> o2) {
    typedef typename C2<T>::t V;
    if constexpr (EARLY) pdl_trigger();        // the contraction's tile copies need nothing from here
    __shared__ V sp[2][8][8], sf[2][8][8];     // [group][slot][parity]
    __shared__ V sh[MODE == 2 ? 2 : 1][8][8], sg2[MODE == 2 ? 2 : 1][8][8];
    const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
    const long long gidx = (long long)blockIdx.x * 2 + grp;
    const bool live = gidx < (long long)ct.n_cells * n_orb;
    const int j = live ? (int)(gidx % n_orb) : 0;
    const int cell = live ? (int)(gidx / n_orb) : 0;
    const int s = t >> 3, g = t & 7;
    const int gi = live ? ct.gi[cell * 64 + t] : -1;
    const int node = live ? ct.node[cell * 64 + t] : 0;
    const int jj = live ? ct.out[cell * 64 + t] : -1;          // output o = s of parity p = g
    const int ty = live ? ct.type[cell * 8 + g] : 0;
    V xp = mk<T>(0, 0), xf = mk<T>(0, 0), xh = mk<T>(0, 0), xg = mk<T>(0, 0);
    if (gi >= 0) {
        const V* wo = w_phi + (long long)j * nvox;
        xp = wo[node];
        if (w_f) xf = w_f[(long long)gi * n_orb + j];
        if constexpr (MODE == 2) {
            // (H_{I,I} w)(node) with the neighbours outside the box omitted
            const int nx = o2.nx, ny = o2.ny, nxy = nx * ny;
            const int i = node % nx, jy = (node / nx) % ny, k = node / nxy;
            T hr, hi;
            if (o2.R == 3) apply_h<T, 3>(wo, node, i, jy, k, nx, ny, o2.nz, o2.inv_h2, o2.V[node], xp, hr, hi);
            else apply_h<T, 1>(wo, node, i, jy, k, nx, ny, o2.nz, o2.inv_h2, o2.V[node], xp, hr, hi);
            xh = mk<T>(hr, hi);
            xg = o2.w_g[(long long)gi * n_orb + j];
        }
    }
    T cf[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cf[q] = jj >= 0 ? ct.coef_f[(long long)ty * 64 + s * 8 + q] : (T)0;
    const T c_cell = (MODE == 1 && live) ? (T)ct.cell_c[cell] : (T)0;
    xp = wht8_lanes(xp, g);
    if (w_f) xf = wht8_lanes(xf, g);
    if constexpr (MODE == 2) {
        xh = wht8_lanes(xh, g);
        xg = wht8_lanes(xg, g);
        sh[grp][s][g] = xh;
        sg2[grp][s][g] = xg;
    }
    sp[grp][s][g] = xp;
    sf[grp][s][g] = xf;
    __syncthreads();
    if (jj < 0) return;
    V ap = mk<T>(0, 0), af = mk<T>(0, 0), ah = mk<T>(0, 0), ag = mk<T>(0, 0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        ap.x += cf[q] * sp[grp][q][g].x; ap.y += cf[q] * sp[grp][q][g].y;
        af.x += cf[q] * sf[grp][q][g].x; af.y += cf[q] * sf[grp][q][g].y;
        if constexpr (MODE == 2) {
            ah.x += cf[q] * sh[grp][q][g].x; ah.y += cf[q] * sh[grp][q][g].y;
            ag.x += cf[q] * sg2[grp][q][g].x; ag.y += cf[q] * sg2[grp][q][g].y;
        }
    }
    const long long e = (long long)j * ct.ng + jj;
    hat_phi[e] = ap;
    if (w_f) hat_f[e] = af;
    if constexpr (MODE == 2) {
        o2.hat_h[e] = ah;
        o2.hat_g[e] = ag;
    }
    if (MODE == 1) {
        const T ac = a_coef * c_cell;
        u[e] = mk<T>(-ac * af.y, ac * af.x);
    }
}

// bnd_forward MODE 0 for many orbitals: a group of 64 threads transforms one cell for
// FO consecutive orbitals (n_orb a multiple of FO), so the cell's tables and
// coefficients are read once per FO orbitals and each thread has FO independent value
// loads in flight.  Same arithmetic, order and outputs as bnd_forward<T, 0>.
constexpr int FO = 4;
// g_phi (optional): w on Gamma in the natural boundary layout [n_gamma][n_orb] (written
// by the previous stage's stencil); read instead of gathering from w_phi.
template <typename T>
__global__ void __launch_bounds__(128) bnd_forward_multi(CellTab<T> ct, int n_orb, long long nvox,
                                                         const typename C2<T>::t* __restrict__ w_phi,
                                                         const typename C2<T>::t* __restrict__ w_f,
                                                         typename C2<T>::t* __restrict__ hat_phi,
                                                         typename C2<T>::t* __restrict__ hat_f,
                                                         const typename C2<T>::t* __restrict__ g_phi) {
    typedef typename C2<T>::t V;
    __shared__ V sp[2][FO][8][8], sf[2][FO][8][8];     // [group][orbital][slot][parity]
    const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int nch = n_orb / FO;
    const long long gidx = (long long)blockIdx.x * 2 + grp;
    const bool live = gidx < (long long)ct.n_cells * nch;
    const int j0 = live ? (int)(gidx % nch) * FO : 0;
    const int cell = live ? (int)(gidx / nch) : 0;
    const int s = t >> 3, g = t & 7;
    const int gi = live ? ct.gi[cell * 64 + t] : -1;
    const int node = live ? ct.node[cell * 64 + t] : 0;
    const int jj = live ? ct.out[cell * 64 + t] : -1;          // output o = s of parity p = g
    const int ty = live ? ct.type[cell * 8 + g] : 0;
    V xp[FO], xf[FO];
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        xp[o] = gi < 0 ? mk<T>(0, 0)
                       : g_phi ? g_phi[(long long)gi * n_orb + j0 + o] : w_phi[(long long)(j0 + o) * nvox + node];
        xf[o] = (gi >= 0 && w_f) ? w_f[(long long)gi * n_orb + j0 + o] : mk<T>(0, 0);
    }
    T cf[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cf[q] = jj >= 0 ? ct.coef_f[(long long)ty * 64 + s * 8 + q] : (T)0;
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        sp[grp][o][s][g] = wht8_lanes(xp[o], g);
        if (w_f) sf[grp][o][s][g] = wht8_lanes(xf[o], g);
    }
    __syncthreads();
    if (jj < 0) return;
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        V ap = mk<T>(0, 0), af = mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ap.x += cf[q] * sp[grp][o][q][g].x; ap.y += cf[q] * sp[grp][o][q][g].y;
            if (w_f) { af.x += cf[q] * sf[grp][o][q][g].x; af.y += cf[q] * sf[grp][o][q][g].y; }
        }
        const long long e = (long long)(j0 + o) * ct.ng + jj;
        hat_phi[e] = ap;
        if (w_f) hat_f[e] = af;
    }
}

// w on Gamma in the natural boundary layout, g[gamma index][orbital], gathered from the
// full state: one thread per (cell slot, orbital), orbitals fastest so the writes are
// contiguous.  Fills the forward transform's Gamma copy before the first stage of a run.
template <typename T>
__global__ void gamma_gather(CellTab<T> ct, int n_orb, long long nvox, const typename C2<T>::t* __restrict__ w_phi,
                             typename C2<T>::t* __restrict__ g) {
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)ct.n_cells * 64 * n_orb) return;
    const int j = (int)(id % n_orb);
    const long long cs = id / n_orb;                     // cell * 64 + slot
    const int gi = ct.gi[cs];
    if (gi < 0) return;
    g[(long long)gi * n_orb + j] = w_phi[(long long)j * nvox + ct.node[cs]];
}

// bnd_forward_multi with the reflection transform done in registers instead of across
// lanes: in phase A thread (array, orbital o, slot s) of a 64-thread group loads the 8
// reflections of its slot (psi at the nodes, or f) and runs the 8-point Walsh-Hadamard
// butterfly on them (the butterfly of wht8_lanes, so the same sums in the same order);
// in phase B thread (output, parity) mixes the 8 slots' values of its parity, read as
// contiguous 16-byte words.  No shuffles; the shared-memory traffic is about a third of
// bnd_forward_multi's.  Same outputs, bit for bit.
template <typename T>
__global__ void __launch_bounds__(128) bnd_forward_multi_rw(CellTab<T> ct, int n_orb, long long nvox,
                                                            const typename C2<T>::t* __restrict__ w_phi,
                                                            const typename C2<T>::t* __restrict__ w_f,
                                                            typename C2<T>::t* __restrict__ hat_phi,
                                                            typename C2<T>::t* __restrict__ hat_f,
                                                            const typename C2<T>::t* __restrict__ g_phi) {
    typedef typename C2<T>::t V;
    __shared__ __align__(16) V sw[2][2][FO][8][8];        // [group][array][orbital][parity][slot]
    const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int nch = n_orb / FO;
    const long long gidx = (long long)blockIdx.x * 2 + grp;
    const bool live = gidx < (long long)ct.n_cells * nch;
    const int j0 = live ? (int)(gidx % nch) * FO : 0;
    const int cell = live ? (int)(gidx / nch) : 0;
    // phase A: t = 32 array + 8 orbital + slot
    {
        const int arr = t >> 5, o = (t >> 3) & 3, sl = t & 7;
        V x[8];
        int gi[8], nd[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            gi[g] = live ? ct.gi[cell * 64 + sl * 8 + g] : -1;
            nd[g] = live ? ct.node[cell * 64 + sl * 8 + g] : 0;
        }
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            x[g] = mk<T>(0, 0);
            if (gi[g] >= 0) {
                if (arr == 0)
                    x[g] = g_phi ? g_phi[(long long)gi[g] * n_orb + j0 + o] : w_phi[(long long)(j0 + o) * nvox + nd[g]];
                else if (w_f) x[g] = w_f[(long long)gi[g] * n_orb + j0 + o];
            }
        }
#pragma unroll
        for (int bit = 1; bit < 8; bit <<= 1) {
            V y[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const V ov = x[g ^ bit];
                if (g & bit) y[g] = mk<T>(ov.x - x[g].x, ov.y - x[g].y);
                else y[g] = mk<T>(x[g].x + ov.x, x[g].y + ov.y);
            }
#pragma unroll
            for (int g = 0; g < 8; ++g) x[g] = y[g];
        }
#pragma unroll
        for (int p = 0; p < 8; ++p) sw[grp][arr][o][p][sl] = x[p];
    }
    __syncthreads();
    // phase B: t = 8 output + parity
    const int oo = t >> 3, p = t & 7;
    const int jj = live ? ct.out[cell * 64 + t] : -1;
    if (jj < 0) return;
    const int ty = ct.type[cell * 8 + p];
    T cf[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cf[q] = ct.coef_f[(long long)ty * 64 + oo * 8 + q];
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        V ap = mk<T>(0, 0), af = mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const V vp = sw[grp][0][o][p][q], vf = sw[grp][1][o][p][q];
            ap.x += cf[q] * vp.x; ap.y += cf[q] * vp.y;
            if (w_f) { af.x += cf[q] * vf.x; af.y += cf[q] * vf.y; }
        }
        const long long e = (long long)(j0 + o) * ct.ng + jj;
        hat_phi[e] = ap;
        if (w_f) hat_f[e] = af;
    }
}

// t from the partial sums of the tiled contraction (see SymGather).  The loads of the
// first two row segments and the first 24 column parts are all issued before any
// of them is used (one memory round trip for the common case); the sums are then
// formed in a fixed order: eight accumulators (the row part of warp w into
// accumulator w % 8, column part K into accumulator (K - I - 1) % 8), added at the end.
__device__ __forceinline__ float2 sym_gather(const SymGather& sg, int4 d) {
    constexpr int RS = 2, CB = 3, NW = SYM_GATHER_WARPS;   // row segments and column batches hoisted
    constexpr int SEG = 192 * NW;
    const int nk = d.w & 0xffff;
    float2 rv[RS][NW], cv[CB][8];
#pragma unroll
    for (int q = 0; q < RS; ++q)
#pragma unroll
        for (int w = 0; w < NW; ++w)
            rv[q][w] = q < d.y ? sg.rowpart[d.x + (size_t)q * SEG + w * 192] : make_float2(0.f, 0.f);
    int e = d.z, step = d.w >> 16;
#pragma unroll
    for (int b = 0; b < CB; ++b)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cv[b][q] = b * 8 + q < nk ? sg.colpart[e] : make_float2(0.f, 0.f);
            e += step * 192;
            ++step;
        }
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < RS; ++q)
#pragma unroll
        for (int w = 0; w < NW; ++w) {                 // the warps' partials of the segment
            acc[w & 7].x += rv[q][w].x;
            acc[w & 7].y += rv[q][w].y;
        }
    for (int q = RS; q < d.y; ++q) {
        const float2* rp = sg.rowpart + d.x + (size_t)q * SEG;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float2 v = rp[w * 192];
            acc[w & 7].x += v.x;
            acc[w & 7].y += v.y;
        }
    }
#pragma unroll
    for (int b = 0; b < CB; ++b)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q].x += cv[b][q].x;
            acc[q].y += cv[b][q].y;
        }
    for (int i0 = CB * 8; i0 < nk; i0 += 8) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = i0 + q < nk ? sg.colpart[e] : make_float2(0.f, 0.f);
            e += step * 192;
            ++step;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q].x += v[q].x;
            acc[q].y += v[q].y;
        }
    }
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        acc[0].x += acc[q].x;
        acc[0].y += acc[q].y;
    }
    return acc[0];
}

// The next stage's adapted inputs, formed by the back transform of an order-1 stage
// (FUSE): at each node of the cell the lane has the stage outputs f' = y_f + cdt v and
// phi' = y_phi + cdt (-i)(H w + w_f) (the interior stencil's formula at that node), and
// applies bnd_forward's transform to them, so the next stage needs no forward kernel.
template <typename T>
struct FwdNext {
    const typename C2<T>::t* w_phi;  // stage input phi [n_orb][nvox]
    const typename C2<T>::t* y_phi;  // step-start phi
    const T* V;                      // potential
    const typename C2<T>::t* w_f;    // stage input f, natural [n_gamma][n_orb]
    typename C2<T>::t* hat_phi;      // next stage's adapted phi
    typename C2<T>::t* hat_f;        // next stage's adapted f
    int nx, ny, nz, R;
    T inv_h2;
    long long nvox;
};

// Back: thread (o, p) = (s, g) forms the adapted value x of output o of parity p:
//   MODE 0 (order-1 step):    x = s1 f_hat + (-i a)(phi_hat - t),  a = a_coef c
//                             (B f + A E phi with B = s1 I - A S, t = S f_hat)
//   MODE 1 (order 0):         x = t  (t = M phi_hat, or conj(M) phi_hat)
//   MODE 2 (order-1 adjoint): x = s1 f_hat - t + i phi_hat  (t = conj(S) u)
//   MODE 3 (order-2 step):    x = t  (t = B1 g + (B0 - i A1) f - i A1 E H w + A0 E phi, the
//                             derivative of g); y_f / out / acc are then the step-start,
//                             stage-output and stage-input auxiliary states [f | g]
//   MODE 4 (order-1 step, two-point or Hermite fit): x = t  (t = B f_hat + A phi_hat,
//                             both general class blocks)
// with t read from t_in (the sum of its nsplit arrays split_stride apart), or
// gathered from the tiled contraction's partial sums (GATHER);
// then thread (s, p) undoes the mixing with the scaled transposed coefficients, the
// slot's 8-lane group transforms back and lane g holds the value v at the
// reflection g of the slot's representative.  At that node's Gamma index e, the
// lane that owns the node (table wr) writes:
//   MODE 0, 4: out[e] = y_f[e] + cdt v   MODE 1: out[e] = v
//   MODE 2: out[e] = cdt v, acc[e] += cdt v
//   MODE 3: out_f[e] = y_f[e] + cdt w_g[e], out_g[e] = y_g[e] + cdt v  (f' = g, g' = v)
// (only the owner reads y_f / acc there, so the update in place is race-free).
template <typename T, int MODE, bool GATHER, bool FUSE = false>
__global__ void __launch_bounds__(128) bnd_back(CellTab<T> ct, int n_orb, T s1, T a_coef,
                                                const typename C2<T>::t* __restrict__ hat_phi,
                                                const typename C2<T>::t* __restrict__ hat_f,
                                                const typename C2<T>::t* __restrict__ t_in, int nsplit,
                                                long long split_stride, SymGather sg,
                                                const typename C2<T>::t* y_f, typename C2<T>::t* out,
                                                typename C2<T>::t* acc, T cdt, FwdNext<T> fn) {
    static_assert(!FUSE || MODE == 0 || MODE == 4, "the fused forward follows an order-1 step");
    typedef typename C2<T>::t V;
    __shared__ V sx[2][8][8];                  // [group][output][parity]
    __shared__ V sp[FUSE ? 2 : 1][8][8], sf[FUSE ? 2 : 1][8][8];
    const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
    const long long gidx = (long long)blockIdx.x * 2 + grp;
    const bool live = gidx < (long long)ct.n_cells * n_orb;
    const int j = live ? (int)(gidx % n_orb) : 0;
    const int cell = live ? (int)(gidx / n_orb) : 0;
    const int s = t >> 3, g = t & 7;
    const int jj = live ? ct.out[cell * 64 + t] : -1;          // output o = s of parity p = g
    const int ty = live ? ct.type[cell * 8 + g] : 0;
    const int wr = live ? ct.wr[cell * 64 + t] : -1;
    int4 gd = make_int4(0, 0, 0, 0);
    if constexpr (GATHER) gd = live ? sg.desc[cell * 64 + t] : gd;
    const T c_cell = (MODE == 0 && live) ? (T)ct.cell_c[cell] : (T)0;
    T cf[8], cff[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) cf[o] = live ? ct.coef_bt[(long long)ty * 64 + s * 8 + o] : (T)0;
    int fgi = -1, fnode = 0;
    if constexpr (FUSE) {
        fgi = live ? ct.gi[cell * 64 + t] : -1;
        fnode = live ? ct.node[cell * 64 + t] : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) cff[q] = jj >= 0 ? ct.coef_f[(long long)ty * 64 + s * 8 + q] : (T)0;
    }
    // FUSE: phi' at this lane's node (the interior stencil's formula) and y_f there; the
    // loads run while the partial sums are gathered below
    V fy = mk<T>(0, 0), pn = mk<T>(0, 0);
    if constexpr (FUSE) {
        if (fgi >= 0) {
            fy = y_f[(long long)fgi * n_orb + j];
            const V* wo = fn.w_phi + (long long)j * fn.nvox;
            const int fi = fnode % fn.nx, fj = (fnode / fn.nx) % fn.ny, fk = fnode / (fn.nx * fn.ny);
            T hr, hi;
            if (fn.R == 3) apply_h<T, 3>(wo, fnode, fi, fj, fk, fn.nx, fn.ny, fn.nz, fn.inv_h2, fn.V[fnode], wo[fnode], hr, hi);
            else apply_h<T, 1>(wo, fnode, fi, fj, fk, fn.nx, fn.ny, fn.nz, fn.inv_h2, fn.V[fnode], wo[fnode], hr, hi);
            const V b = fn.w_f[(long long)fgi * n_orb + j];
            hr += b.x;
            hi += b.y;
            const V yp = fn.y_phi[(long long)j * fn.nvox + fnode];
            pn = mk<T>(yp.x + cdt * hi, yp.y - cdt * hr);
        }
    }
    V yv = mk<T>(0, 0), yg = mk<T>(0, 0), wg = mk<T>(0, 0);
    const long long ew = (long long)(wr >= 0 ? wr : 0) * n_orb + j;
    const long long gofs = (long long)ct.n_gamma * n_orb;      // g part of an order-2 auxiliary state
    if (wr >= 0 && (MODE == 0 || MODE == 4)) yv = y_f[ew];
    if (wr >= 0 && MODE == 2) yv = acc[ew];
    if (wr >= 0 && MODE == 3) {
        yv = y_f[ew];
        yg = y_f[gofs + ew];
        wg = acc[gofs + ew];
    }
    V x = mk<T>(0, 0);
    if (jj >= 0) {
        const long long e = (long long)j * ct.ng + jj;
        // the adapted inputs are loaded before t, so their loads overlap the gather's
        V fv = mk<T>(0, 0), pv = mk<T>(0, 0);
        if (MODE == 0 || MODE == 2) {
            fv = hat_f[e];
            pv = hat_phi[e];
        }
        V tv;
        if constexpr (GATHER) {
            const float2 q = sym_gather(sg, gd);
            tv = mk<T>((T)q.x, (T)q.y);
        } else {
            tv = t_in[e];
            for (int q = 1; q < nsplit; ++q) {
                const V u = t_in[(long long)q * split_stride + e];
                tv.x += u.x;
                tv.y += u.y;
            }
        }
        if (MODE == 0) {
            x = back_x1(s1, a_coef * c_cell, fv, pv, tv);
        } else if (MODE == 1 || MODE == 3 || MODE == 4) {
            x = tv;
        } else {
            x = mk<T>(s1 * fv.x - tv.x - pv.y, s1 * fv.y - tv.y + pv.x);
        }
    }
    sx[grp][s][g] = x;
    __syncthreads();
    V v = mk<T>(0, 0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        v.x += cf[o] * sx[grp][o][g].x;
        v.y += cf[o] * sx[grp][o][g].y;
    }
    v = wht8_lanes(v, g);
    if (wr >= 0) {
        if (MODE == 0 || MODE == 4) {
            out[ew] = mk<T>(yv.x + cdt * v.x, yv.y + cdt * v.y);
        } else if (MODE == 1) {
            out[ew] = v;
        } else if (MODE == 2) {
            const T nr = cdt * v.x, ni = cdt * v.y;
            out[ew] = mk<T>(nr, ni);
            acc[ew] = mk<T>(yv.x + nr, yv.y + ni);
        } else {
            out[ew] = mk<T>(yv.x + cdt * wg.x, yv.y + cdt * wg.y);
            out[gofs + ew] = mk<T>(yg.x + cdt * v.x, yg.y + cdt * v.y);
        }
    }
    if constexpr (FUSE) {
        // bnd_forward<T, 0> on (phi', f') at the cell's nodes
        V xp = mk<T>(0, 0), xf = mk<T>(0, 0);
        if (fgi >= 0) {
            xp = pn;
            xf = mk<T>(fy.x + cdt * v.x, fy.y + cdt * v.y);
        }
        xp = wht8_lanes(xp, g);
        xf = wht8_lanes(xf, g);
        sp[grp][s][g] = xp;
        sf[grp][s][g] = xf;
        __syncthreads();
        if (jj >= 0) {
            V ap = mk<T>(0, 0), af = mk<T>(0, 0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ap.x += cff[q] * sp[grp][q][g].x; ap.y += cff[q] * sp[grp][q][g].y;
                af.x += cff[q] * sf[grp][q][g].x; af.y += cff[q] * sf[grp][q][g].y;
            }
            const long long e = (long long)j * ct.ng + jj;
            fn.hat_phi[e] = ap;
            fn.hat_f[e] = af;
        }
    }
}

// bnd_back<T, 0, false> for FO consecutive orbitals per cell group (n_orb a multiple of
// FO, 2 or 4): the cell's tables and coefficients are read once per FO orbitals and
// each thread has FO independent sets of loads in flight.  Same arithmetic and order as
// bnd_back<T, 0, false>, orbital by orbital.
template <typename T, int FO = dev::FO>
__global__ void __launch_bounds__(128) bnd_back_multi(CellTab<T> ct, int n_orb, T s1, T a_coef,
                                                      const typename C2<T>::t* __restrict__ hat_phi,
                                                      const typename C2<T>::t* __restrict__ hat_f,
                                                      const typename C2<T>::t* __restrict__ t_in, int nsplit,
                                                      long long split_stride, const typename C2<T>::t* y_f,
                                                      typename C2<T>::t* out, T cdt) {
    typedef typename C2<T>::t V;
    __shared__ V sx[2][FO][8][8];              // [group][orbital][output][parity]
    const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int nch = n_orb / FO;
    const long long gidx = (long long)blockIdx.x * 2 + grp;
    const bool live = gidx < (long long)ct.n_cells * nch;
    const int j0 = live ? (int)(gidx % nch) * FO : 0;
    const int cell = live ? (int)(gidx / nch) : 0;
    const int s = t >> 3, g = t & 7;
    const int jj = live ? ct.out[cell * 64 + t] : -1;
    const int ty = live ? ct.type[cell * 8 + g] : 0;
    const int wr = live ? ct.wr[cell * 64 + t] : -1;
    const T c_cell = live ? (T)ct.cell_c[cell] : (T)0;
    T cf[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) cf[o] = live ? ct.coef_bt[(long long)ty * 64 + s * 8 + o] : (T)0;
    V yv[FO], x[FO];
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        yv[o] = wr >= 0 ? y_f[(long long)wr * n_orb + j0 + o] : mk<T>(0, 0);
        x[o] = mk<T>(0, 0);
    }
    if (jj >= 0) {
        V fv[FO], pv[FO], tv[FO];
#pragma unroll
        for (int o = 0; o < FO; ++o) {
            const long long e = (long long)(j0 + o) * ct.ng + jj;
            fv[o] = hat_f[e];
            pv[o] = hat_phi[e];
            tv[o] = t_in[e];
        }
        for (int q = 1; q < nsplit; ++q)
#pragma unroll
            for (int o = 0; o < FO; ++o) {
                const V u = t_in[(long long)q * split_stride + (long long)(j0 + o) * ct.ng + jj];
                tv[o].x += u.x;
                tv[o].y += u.y;
            }
        const T a = a_coef * c_cell;
#pragma unroll
        for (int o = 0; o < FO; ++o) x[o] = back_x1(s1, a, fv[o], pv[o], tv[o]);
    }
#pragma unroll
    for (int o = 0; o < FO; ++o) sx[grp][o][s][g] = x[o];
    __syncthreads();
#pragma unroll
    for (int o = 0; o < FO; ++o) {
        V v = mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v.x += cf[q] * sx[grp][o][q][g].x;
            v.y += cf[q] * sx[grp][o][q][g].y;
        }
        v = wht8_lanes(v, g);
        if (wr >= 0) out[(long long)wr * n_orb + j0 + o] = mk<T>(yv[o].x + cdt * v.x, yv[o].y + cdt * v.y);
    }
}

// --------------------------------------------------------------------------
// Boundary contraction, one orbital: t = S_p x_p for every parity block p
// (GEMV; HBM-bound).  One warp per row; the row is streamed with 16-byte loads.
// --------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int find_block(const BlockInfo& bi, int q) {
    int p = 0;
    for (int k = 1; k < bi.n; ++k)
        if (q >= bi.off[k]) p = k;
    return p;
}

// One orbital, one block of GEMV_WARPS warps per GEMV_RB consecutive block rows of a
// class: each row is streamed once and applied to all R right-hand sides of the class
// (the matrix bytes are read once per launch, where gemv_blocks reads a class block
// once per right-hand side); each loaded slice of x serves GEMV_RB rows; the warps
// split the columns (more loads in flight) and their partial sums are added through
// shared memory in a fixed order.
constexpr int GEMV_RB = 4, GEMV_WARPS = 4;
template <typename T, int R>
__device__ __forceinline__ void gemv_class_rows(const ClassInfo& ci, int c, int a0, const typename C2<T>::t* mat,
                                                const XSeg<typename C2<T>::t>& xs, typename C2<T>::t* y, T cs,
                                                typename C2<T>::t (*red)[GEMV_RB][3]) {
    typedef typename C2<T>::t V;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = ci.m[c];
    const int nr = m - a0 < GEMV_RB ? m - a0 : GEMV_RB;    // rows of this block (the last may be short)
    T sr[GEMV_RB][R], si[GEMV_RB][R];
#pragma unroll
    for (int r = 0; r < GEMV_RB; ++r)
#pragma unroll
        for (int k = 0; k < R; ++k) sr[r][k] = si[r][k] = 0;
    for (int q = 0; q < 4; ++q) {
        if (!xs.p[q]) break;
        const V* row0 = mat + ci.mat_off[c] + (long long)a0 * ci.ld[c] + (long long)q * ci.segw[c];
        if constexpr (sizeof(T) == 4) {
            const int m2 = m >> 1;
#pragma unroll 2
            for (int cc = threadIdx.x; cc < m2; cc += 32 * GEMV_WARPS) {
                float4 sv[GEMV_RB];
#pragma unroll
                for (int r = 0; r < GEMV_RB; ++r)
                    sv[r] = r < nr ? __ldcs(reinterpret_cast<const float4*>(row0 + (long long)r * ci.ld[c]) + cc)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const V* xv = xs.p[q] + ci.moff[c][k];
                    const V x0 = xv[2 * cc], x1 = xv[2 * cc + 1];
#pragma unroll
                    for (int r = 0; r < GEMV_RB; ++r) {
                        const T sy0 = cs * sv[r].y, sy1 = cs * sv[r].w;
                        sr[r][k] += sv[r].x * x0.x - sy0 * x0.y + sv[r].z * x1.x - sy1 * x1.y;
                        si[r][k] += sv[r].x * x0.y + sy0 * x0.x + sv[r].z * x1.y + sy1 * x1.x;
                    }
                }
            }
            if ((m & 1) && threadIdx.x == 0) {
#pragma unroll
                for (int r = 0; r < GEMV_RB; ++r) {
                    if (r >= nr) break;
                    const V sv = row0[(long long)r * ci.ld[c] + m - 1];
                    const T sy = cs * sv.y;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const V xx = xs.p[q][ci.moff[c][k] + m - 1];
                        sr[r][k] += sv.x * xx.x - sy * xx.y;
                        si[r][k] += sv.x * xx.y + sy * xx.x;
                    }
                }
            }
        } else {
#pragma unroll 2
            for (int cc = threadIdx.x; cc < m; cc += 32 * GEMV_WARPS) {
                V sv[GEMV_RB];
#pragma unroll
                for (int r = 0; r < GEMV_RB; ++r) sv[r] = r < nr ? __ldcs(row0 + (long long)r * ci.ld[c] + cc) : mk<T>(0, 0);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const V xx = xs.p[q][ci.moff[c][k] + cc];
#pragma unroll
                    for (int r = 0; r < GEMV_RB; ++r) {
                        const T sy = cs * sv[r].y;
                        sr[r][k] += sv[r].x * xx.x - sy * xx.y;
                        si[r][k] += sv[r].x * xx.y + sy * xx.x;
                    }
                }
            }
        }
    }
    // the warp's 2 GEMV_RB R partial sums, reduced by halving exchanges (a reduce-scatter
    // over the lanes with the xor masks 16, 8, ... of warp_sum, so every total is the same
    // pairwise tree): after the L = log2(NV) levels lane l holds slot l >> (5 - L), summed
    // over the lanes that differ in the top L bits; the remaining masks finish it
    constexpr int NV0 = 2 * GEMV_RB * R;
    constexpr int NV = NV0 <= 8 ? 8 : NV0 <= 16 ? 16 : 32;
    constexpr int L = NV == 8 ? 3 : NV == 16 ? 4 : 5;
    T v[NV];
#pragma unroll
    for (int r = 0; r < GEMV_RB; ++r)
#pragma unroll
        for (int k = 0; k < R; ++k) {
            v[2 * (r * R + k)] = sr[r][k];
            v[2 * (r * R + k) + 1] = si[r][k];
        }
#pragma unroll
    for (int i = NV0; i < NV; ++i) v[i] = 0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int half = NV >> (l + 1), m = 16 >> l;
        const bool up = lane & m;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T keep = up ? v[i + half] : v[i], send = up ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
#pragma unroll
    for (int m = 16 >> L; m; m >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    {
        const int slot = lane >> (5 - L);
        if ((lane & ((1 << (5 - L)) - 1)) == 0 && slot < NV0) {
            const int rk = slot >> 1;
            T* dst = reinterpret_cast<T*>(&red[w][rk / R][rk % R]);
            dst[slot & 1] = v[0];
        }
    }
    __syncthreads();
    if (threadIdx.x < GEMV_RB * R) {
        const int r = threadIdx.x / R, k = threadIdx.x % R;
        if (r < nr) {
            V acc = red[0][r][k];
#pragma unroll
            for (int u = 1; u < GEMV_WARPS; ++u) {
                acc.x += red[u][r][k].x;
                acc.y += red[u][r][k].y;
            }
            y[ci.moff[c][k] + a0 + r] = acc;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * GEMV_WARPS) gemv_classes(ClassInfo ci, const typename C2<T>::t* __restrict__ mat,
                                                                XSeg<typename C2<T>::t> xs,
                                                                typename C2<T>::t* __restrict__ y, int conj) {
    __shared__ typename C2<T>::t red[GEMV_WARPS][GEMV_RB][3];
    const int blk = blockIdx.x;
    if (blk >= ci.rowbase[ci.n]) return;
    int c = 0;
    while (c + 1 < ci.n && blk >= ci.rowbase[c + 1]) ++c;
    const int a0 = (blk - ci.rowbase[c]) * GEMV_RB;
    const T cs = conj ? (T)-1 : (T)1;     // conj: y = conj(S) x
    switch (ci.R[c]) {
        case 1: gemv_class_rows<T, 1>(ci, c, a0, mat, xs, y, cs, red); break;
        case 2: gemv_class_rows<T, 2>(ci, c, a0, mat, xs, y, cs, red); break;
        default: gemv_class_rows<T, 3>(ci, c, a0, mat, xs, y, cs, red); break;
    }
}

template <typename T>
__global__ void gemv_blocks(BlockInfo bi, int n_rows, const typename C2<T>::t* __restrict__ mat,
                            XSeg<typename C2<T>::t> xs, typename C2<T>::t* __restrict__ y, int conj) {
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n_rows) return;
    const int p = find_block(bi, warp);
    const int a = warp - bi.off[p];
    const int m = bi.m[p];
    T sr = 0, si = 0;
    const T cs = conj ? (T)-1 : (T)1;     // conj: y = conj(S conj(x)) = conj(S) x
    for (int q = 0; q < bi.nseg; ++q) {
        const typename C2<T>::t* row = mat + bi.mat_off[p] + (long long)a * bi.ld[p] + (long long)q * bi.segw[p];
        const typename C2<T>::t* xv = xs.p[q] + bi.off[p];
        if constexpr (sizeof(T) == 4) {
            // two complex per lane per load (segment start 16-byte aligned: ld, segw, mat_off multiples of 4)
            const float4* row4 = reinterpret_cast<const float4*>(row);
            const int m2 = m >> 1;
            int c = lane;
#pragma unroll 4
            for (; c < m2; c += 32) {
                const float4 sv = __ldcs(row4 + c);
                const typename C2<T>::t x0 = xv[2 * c], x1 = xv[2 * c + 1];
                const T sy0 = cs * sv.y, sy1 = cs * sv.w;
                sr += sv.x * x0.x - sy0 * x0.y + sv.z * x1.x - sy1 * x1.y;
                si += sv.x * x0.y + sy0 * x0.x + sv.z * x1.y + sy1 * x1.x;
            }
            if ((m & 1) && lane == 0) {
                const typename C2<T>::t sv = row[m - 1], xx = xv[m - 1];
                const T sy = cs * sv.y;
                sr += sv.x * xx.x - sy * xx.y;
                si += sv.x * xx.y + sy * xx.x;
            }
        } else {
#pragma unroll 4
            for (int c = lane; c < m; c += 32) {
                const typename C2<T>::t sv = row[c], xx = xv[c];
                const T sy = cs * sv.y;
                sr += sv.x * xx.x - sy * xx.y;
                si += sv.x * xx.y + sy * xx.x;
            }
        }
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) y[warp] = mk<T>(sr, si);
}

// --------------------------------------------------------------------------
// Boundary contraction, many orbitals: T_p = S_p X_p (X_p: m_p x n_orb; adapted
// vectors orbital-major with stride ng).  CUDA-core form (shared-memory tiles).
// --------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK>
__global__ void gemm_blocks_simt(BlockInfo bi, int n_orb, int ng, const typename C2<T>::t* __restrict__ mat,
                                 XSeg<typename C2<T>::t> xs, typename C2<T>::t* __restrict__ Y,
                                 int conj, const int* __restrict__ tile_block, const int* __restrict__ tile_row) {
    typedef typename C2<T>::t V;
    __shared__ V As[BK][BM + 1];
    __shared__ V Bs[BK][BN];
    const int p = tile_block[blockIdx.x];
    const int row0 = tile_row[blockIdx.x];          // local row in block p
    const int col0 = blockIdx.y * BN;
    const int m = bi.m[p];
    const V* S0 = mat + bi.mat_off[p];
    const int tx = threadIdx.x % BN, ty = threadIdx.x / BN;   // BN columns, (nthr/BN) row groups
    constexpr int NT = 256;
    constexpr int RPT = BM / (NT / BN);                       // rows per thread
    T accr[RPT], acci[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) accr[i] = acci[i] = 0;
    const T cs = conj ? (T)-1 : (T)1;
    for (int q = 0; q < bi.nseg; ++q)
    for (int k0 = 0; k0 < m; k0 += BK) {
        const V* S = S0 + (long long)q * bi.segw[p];
        const V* Xp = xs.p[q] + bi.off[p];                // column gc at Xp[gc * ng]
        for (int e = threadIdx.x; e < BM * BK; e += NT) {
            const int rr = e / BK, kk = e % BK;
            const int gr = row0 + rr, gk = k0 + kk;
            V v = mk<T>(0, 0);
            if (gr < m && gk < m) v = S[(long long)gr * bi.ld[p] + gk];
            v.y *= cs;
            As[kk][rr] = v;
        }
        for (int e = threadIdx.x; e < BK * BN; e += NT) {
            const int kk = e / BN, cc = e % BN;
            const int gk = k0 + kk, gc = col0 + cc;
            V v = mk<T>(0, 0);
            if (gk < m && gc < n_orb) v = Xp[(long long)gc * ng + gk];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            const V b = Bs[kk][tx];
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const V a = As[kk][ty * RPT + i];
                accr[i] += a.x * b.x - a.y * b.y;
                acci[i] += a.x * b.y + a.y * b.x;
            }
        }
        __syncthreads();
    }
    const int gc = col0 + tx;
    if (gc >= n_orb) return;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int gr = row0 + ty * RPT + i;
        if (gr < m) Y[(long long)gc * ng + bi.off[p] + gr] = mk<T>(accr[i], acci[i]);
    }
}

// --------------------------------------------------------------------------
// Fused stencil + potential + boundary term + Horner stage
//   out = y + cdt * (-i) [ H_{I,I} w + E^T b ],  H = -1/2 Delta_h + V
// b = w_f (order 1) or M E w (order 0), natural Gamma order [n_gamma][n_orb].
// Grid (ceil(nx ny / blockDim), nz, n_orb): one thread per node of a z-plane.
// --------------------------------------------------------------------------
template <typename T, int R = 1>
__global__ void stencil_stage(int nx, int ny, int nz, int n_orb, T inv_h2, const typename C2<T>::t* __restrict__ w,
                              const typename C2<T>::t* y, const T* __restrict__ V,
                              const typename C2<T>::t* __restrict__ bterm, typename C2<T>::t* out, T cdt) {
    typedef typename C2<T>::t Vc;
    const long long nvox = (long long)nx * ny * nz;
    const int tp = blockIdx.x * blockDim.x + threadIdx.x;          // node in the z-plane
    if (tp >= nx * ny) return;
    const int i = tp % nx, jy = tp / nx, k = blockIdx.y, orb = blockIdx.z;
    const long long n = (long long)k * nx * ny + tp;
    const long long idx = (long long)orb * nvox + n;
    const Vc* wo = w + (long long)orb * nvox;
    T hr, hi;
    apply_h<T, R>(wo, n, i, jy, k, nx, ny, nz, inv_h2, V[n], wo[n], hr, hi);
    if (on_gamma<R>(i, jy, k, nx, ny, nz)) {
        const Vc b = bterm[(long long)gamma_index<R>(i, jy, k, nx, ny, nz) * n_orb + orb];
        hr += b.x;
        hi += b.y;
    }
    const Vc yv = y[idx];
    out[idx] = mk<T>(yv.x + cdt * hi, yv.y - cdt * hr);
}

// The radius-1 complex64 stage update for two x-adjacent nodes (i, i + 1), i even, per
// thread, with 16-byte loads of the pair and of its y and z neighbours (nx even, so a
// pair never crosses a row and every pair starts on a 16-byte boundary): 7 loads of w
// for two nodes instead of 14.  Same neighbour order and formula as stencil_stage.
// gout (optional): the outputs on Gamma also go to gout[gamma_index * n_orb + orb], the
// natural boundary layout the next stage's forward transform reads instead of gathering
// them from the whole state.
__device__ __forceinline__ void stencil_pair_x2(int nx, int ny, int nz, int n_orb, float inv_h2,
                                                const float2* __restrict__ w, const float2* y,
                                                const float* __restrict__ V, const float2* __restrict__ bterm,
                                                float2* out, float cdt, int tp2, int k, int orb,
                                                float2* __restrict__ gout) {
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const int jy = tp2 / (nx >> 1), i = 2 * (tp2 - jy * (nx >> 1));
    const long long n = (long long)k * nxy + (long long)jy * nx + i;
    const float2* wo = w + (long long)orb * nvox;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 c = *reinterpret_cast<const float4*>(wo + n);
    const float2 xm = i >= 1 ? wo[n - 1] : make_float2(0.f, 0.f);
    const float2 xp = i + 2 < nx ? wo[n + 2] : make_float2(0.f, 0.f);
    const float4 ym = jy >= 1 ? *reinterpret_cast<const float4*>(wo + n - nx) : zero;
    const float4 yp = jy + 1 < ny ? *reinterpret_cast<const float4*>(wo + n + nx) : zero;
    const float4 zm = k >= 1 ? *reinterpret_cast<const float4*>(wo + n - nxy) : zero;
    const float4 zp = k + 1 < nz ? *reinterpret_cast<const float4*>(wo + n + nxy) : zero;
    const float2 vv = *reinterpret_cast<const float2*>(V + n);
    const long long idx = (long long)orb * nvox + n;
    const float4 yv = *reinterpret_cast<const float4*>(y + idx);
    float hr[2], hi[2];
    {
        // node i: x- = xm, x+ = node i + 1
        float sr = 0.f, si = 0.f;
        sr += xm.x; si += xm.y;
        sr += c.z; si += c.w;
        sr += ym.x; si += ym.y;
        sr += yp.x; si += yp.y;
        sr += zm.x; si += zm.y;
        sr += zp.x; si += zp.y;
        const float dg = 3.f * inv_h2 + vv.x;
        hr[0] = dg * c.x - 0.5f * inv_h2 * sr;
        hi[0] = dg * c.y - 0.5f * inv_h2 * si;
    }
    {
        // node i + 1: x- = node i, x+ = xp
        float sr = 0.f, si = 0.f;
        sr += c.x; si += c.y;
        sr += xp.x; si += xp.y;
        sr += ym.z; si += ym.w;
        sr += yp.z; si += yp.w;
        sr += zm.z; si += zm.w;
        sr += zp.z; si += zp.w;
        const float dg = 3.f * inv_h2 + vv.y;
        hr[1] = dg * c.z - 0.5f * inv_h2 * sr;
        hi[1] = dg * c.w - 0.5f * inv_h2 * si;
    }
    long long gq[2] = {-1, -1};
#pragma unroll
    for (int q = 0; q < 2; ++q)
        if (on_gamma<1>(i + q, jy, k, nx, ny, nz)) {
            gq[q] = (long long)gamma_index<1>(i + q, jy, k, nx, ny, nz) * n_orb + orb;
            const float2 b = bterm[gq[q]];
            hr[q] += b.x;
            hi[q] += b.y;
        }
    const float4 o = make_float4(yv.x + cdt * hi[0], yv.y - cdt * hr[0], yv.z + cdt * hi[1], yv.w - cdt * hr[1]);
    *reinterpret_cast<float4*>(out + idx) = o;
    if (gout) {
        if (gq[0] >= 0) gout[gq[0]] = make_float2(o.x, o.y);
        if (gq[1] >= 0) gout[gq[1]] = make_float2(o.z, o.w);
    }
}

static __global__ void stencil_stage_x2(int nx, int ny, int nz, int n_orb, float inv_h2, const float2* __restrict__ w,
                                        const float2* y, const float* __restrict__ V,
                                        const float2* __restrict__ bterm, float2* out, float cdt,
                                        float2* __restrict__ gout) {
    const int tp2 = blockIdx.x * blockDim.x + threadIdx.x;         // pair in the z-plane
    if (tp2 >= (nx >> 1) * ny) return;
    stencil_pair_x2(nx, ny, nz, n_orb, inv_h2, w, y, V, bterm, out, cdt, tp2, blockIdx.y, blockIdx.z, gout);
}

// stencil_stage_x2 compiled for MINB resident blocks per SM (registers capped so that
// all of the SM's warp slots can be filled: the kernel waits on loads, and more warps
// keep more of them in flight).
template <int MINB>
__global__ void __launch_bounds__(256, MINB) stencil_stage_x2_lb(int nx, int ny, int nz, int n_orb, float inv_h2,
                                                                 const float2* __restrict__ w, const float2* y,
                                                                 const float* __restrict__ V,
                                                                 const float2* __restrict__ bterm, float2* out,
                                                                 float cdt, float2* __restrict__ gout) {
    const int tp2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (tp2 >= (nx >> 1) * ny) return;
    stencil_pair_x2(nx, ny, nz, n_orb, inv_h2, w, y, V, bterm, out, cdt, tp2, blockIdx.y, blockIdx.z, gout);
}

// stencil_stage_x2 with each thread marching through KZ consecutive planes of its node
// pair (grid y = groups of KZ planes): the pair's z column rolls through registers (the
// centre of plane k + 1 is the z+ neighbour of plane k), and the loads of plane k + 1
// are issued before plane k is computed, so two planes' loads are in flight per
// thread.  Same neighbour order and formula as stencil_stage_x2, node by node.
template <int KZ>
__global__ void __launch_bounds__(256) stencil_stage_x2zk(int nx, int ny, int nz, int n_orb, float inv_h2,
                                                          const float2* __restrict__ w, const float2* y,
                                                          const float* __restrict__ V,
                                                          const float2* __restrict__ bterm, float2* out, float cdt,
                                                          float2* __restrict__ gout) {
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const int tp2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (tp2 >= (nx >> 1) * ny) return;
    const int jy = tp2 / (nx >> 1), i = 2 * (tp2 - jy * (nx >> 1)), orb = blockIdx.z;
    const int k0 = blockIdx.y * KZ, k1 = min(nz, k0 + KZ);
    const float2* wo = w + (long long)orb * nvox;
    const float2* yo = y + (long long)orb * nvox;
    float2* oo = out + (long long)orb * nvox;
    const long long col = (long long)jy * nx + i;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 z2 = make_float2(0.f, 0.f);
    auto ld4 = [&](const float2* p, long long n) { return *reinterpret_cast<const float4*>(p + n); };
    // plane k0: its centre, in-plane neighbours, y and V; and the z- neighbour
    long long n = (long long)k0 * nxy + col;
    float4 zm = k0 >= 1 ? ld4(wo, n - nxy) : zero;
    float4 c = ld4(wo, n);
    float2 xm = i >= 1 ? wo[n - 1] : z2, xp = i + 2 < nx ? wo[n + 2] : z2;
    float4 ym = jy >= 1 ? ld4(wo, n - nx) : zero, yp = jy + 1 < ny ? ld4(wo, n + nx) : zero;
    float4 yv = ld4(yo, n);
    float2 vv = *reinterpret_cast<const float2*>(V + n);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk) {
        const int k = k0 + kk;
        if (k >= k1) break;
        // plane k + 1 (its centre is this plane's z+ neighbour)
        const long long nn = n + nxy;
        const bool more = k + 1 < nz;
        const float4 zp = more ? ld4(wo, nn) : zero;
        float2 xmn = z2, xpn = z2, vvn = z2;
        float4 ymn = zero, ypn = zero, yvn = zero;
        if (more && k + 1 < k1) {
            xmn = i >= 1 ? wo[nn - 1] : z2;
            xpn = i + 2 < nx ? wo[nn + 2] : z2;
            ymn = jy >= 1 ? ld4(wo, nn - nx) : zero;
            ypn = jy + 1 < ny ? ld4(wo, nn + nx) : zero;
            yvn = ld4(yo, nn);
            vvn = *reinterpret_cast<const float2*>(V + nn);
        }
        float hr[2], hi[2];
        {
            float sr = 0.f, si = 0.f;
            sr += xm.x; si += xm.y;
            sr += c.z; si += c.w;
            sr += ym.x; si += ym.y;
            sr += yp.x; si += yp.y;
            sr += zm.x; si += zm.y;
            sr += zp.x; si += zp.y;
            const float dg = 3.f * inv_h2 + vv.x;
            hr[0] = dg * c.x - 0.5f * inv_h2 * sr;
            hi[0] = dg * c.y - 0.5f * inv_h2 * si;
        }
        {
            float sr = 0.f, si = 0.f;
            sr += c.x; si += c.y;
            sr += xp.x; si += xp.y;
            sr += ym.z; si += ym.w;
            sr += yp.z; si += yp.w;
            sr += zm.z; si += zm.w;
            sr += zp.z; si += zp.w;
            const float dg = 3.f * inv_h2 + vv.y;
            hr[1] = dg * c.z - 0.5f * inv_h2 * sr;
            hi[1] = dg * c.w - 0.5f * inv_h2 * si;
        }
        long long gq[2] = {-1, -1};
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (on_gamma<1>(i + q, jy, k, nx, ny, nz)) {
                gq[q] = (long long)gamma_index<1>(i + q, jy, k, nx, ny, nz) * n_orb + orb;
                const float2 b = bterm[gq[q]];
                hr[q] += b.x;
                hi[q] += b.y;
            }
        const float4 o = make_float4(yv.x + cdt * hi[0], yv.y - cdt * hr[0], yv.z + cdt * hi[1], yv.w - cdt * hr[1]);
        *reinterpret_cast<float4*>(oo + n) = o;
        if (gout) {
            if (gq[0] >= 0) gout[gq[0]] = make_float2(o.x, o.y);
            if (gq[1] >= 0) gout[gq[1]] = make_float2(o.z, o.w);
        }
        zm = c;
        c = zp;
        xm = xmn; xp = xpn; ym = ymn; yp = ypn; yv = yvn; vv = vvn;
        n = nn;
    }
}

// stencil_stage_x2 on a grid of a fixed number of blocks per SM that strides over
// (orbital, plane, pair): launched at the start of a stage beside the boundary chain,
// it leaves thread slots and registers on every SM for the chain's kernels (the
// tensor-core GEMM keeps its one CTA per SM) instead of filling the GPU.
static __global__ void __launch_bounds__(256) stencil_stage_x2_gs(int nx, int ny, int nz, int n_orb, float inv_h2,
                                                                  const float2* __restrict__ w, const float2* y,
                                                                  const float* __restrict__ V,
                                                                  const float2* __restrict__ bterm, float2* out,
                                                                  float cdt, float2* __restrict__ gout) {
    const int pp = (nx >> 1) * ny;                                  // pairs per plane
    const long long total = (long long)pp * nz * n_orb;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const long long pl = it / pp;
        const int tp2 = (int)(it - pl * pp);
        const int orb = (int)(pl / nz), k = (int)(pl - (long long)orb * nz);
        stencil_pair_x2(nx, ny, nz, n_orb, inv_h2, w, y, V, bterm, out, cdt, tp2, k, orb, gout);
    }
}

// stencil_stage_x2 for two planes per thread as well (grid y = plane pairs): the pair's
// column at k - 1 .. k + 2 serves both planes.
static __global__ void stencil_stage_x2z2(int nx, int ny, int nz, int n_orb, float inv_h2,
                                          const float2* __restrict__ w, const float2* y,
                                          const float* __restrict__ V, const float2* __restrict__ bterm, float2* out,
                                          float cdt) {
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const int tp2 = blockIdx.x * blockDim.x + threadIdx.x;         // pair in the z-plane
    if (tp2 >= (nx >> 1) * ny) return;
    const int jy = tp2 / (nx >> 1), i = 2 * (tp2 - jy * (nx >> 1)), k0 = 2 * blockIdx.y, orb = blockIdx.z;
    const long long n0 = (long long)k0 * nxy + (long long)jy * nx + i;
    const float2* wo = w + (long long)orb * nvox;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool two = k0 + 1 < nz;
    // column k0 - 1 .. k0 + 2 of the pair
    float4 col[4];
    col[0] = k0 >= 1 ? *reinterpret_cast<const float4*>(wo + n0 - nxy) : zero;
    col[1] = *reinterpret_cast<const float4*>(wo + n0);
    col[2] = two ? *reinterpret_cast<const float4*>(wo + n0 + nxy) : zero;
    col[3] = k0 + 2 < nz ? *reinterpret_cast<const float4*>(wo + n0 + 2 * nxy) : zero;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q == 1 && !two) break;
        const int k = k0 + q;
        const long long n = n0 + q * nxy;
        const float4 c = col[q + 1], zm = col[q], zp = col[q + 2];
        const float2 xm = i >= 1 ? wo[n - 1] : make_float2(0.f, 0.f);
        const float2 xp = i + 2 < nx ? wo[n + 2] : make_float2(0.f, 0.f);
        const float4 ym = jy >= 1 ? *reinterpret_cast<const float4*>(wo + n - nx) : zero;
        const float4 yp = jy + 1 < ny ? *reinterpret_cast<const float4*>(wo + n + nx) : zero;
        const float2 vv = *reinterpret_cast<const float2*>(V + n);
        const long long idx = (long long)orb * nvox + n;
        const float4 yv = *reinterpret_cast<const float4*>(y + idx);
        float hr[2], hi[2];
        {
            float sr = 0.f, si = 0.f;
            sr += xm.x; si += xm.y;
            sr += c.z; si += c.w;
            sr += ym.x; si += ym.y;
            sr += yp.x; si += yp.y;
            sr += zm.x; si += zm.y;
            sr += zp.x; si += zp.y;
            const float dg = 3.f * inv_h2 + vv.x;
            hr[0] = dg * c.x - 0.5f * inv_h2 * sr;
            hi[0] = dg * c.y - 0.5f * inv_h2 * si;
        }
        {
            float sr = 0.f, si = 0.f;
            sr += c.x; si += c.y;
            sr += xp.x; si += xp.y;
            sr += ym.z; si += ym.w;
            sr += yp.z; si += yp.w;
            sr += zm.z; si += zm.w;
            sr += zp.z; si += zp.w;
            const float dg = 3.f * inv_h2 + vv.y;
            hr[1] = dg * c.z - 0.5f * inv_h2 * sr;
            hi[1] = dg * c.w - 0.5f * inv_h2 * si;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (on_gamma<1>(i + e, jy, k, nx, ny, nz)) {
                const float2 b = bterm[(long long)gamma_index<1>(i + e, jy, k, nx, ny, nz) * n_orb + orb];
                hr[e] += b.x;
                hi[e] += b.y;
            }
        *reinterpret_cast<float4*>(out + idx) =
            make_float4(yv.x + cdt * hi[0], yv.y - cdt * hr[0], yv.z + cdt * hi[1], yv.w - cdt * hr[1]);
    }
}

// --------------------------------------------------------------------------
// Mean field: V = V_ext + a rho + b rho^(1+alpha), rho = sum_j |phi_j|^2
// --------------------------------------------------------------------------
template <typename T>
__global__ void density_potential(long long nvox, int n_orb, const typename C2<T>::t* __restrict__ phi,
                                  const T* __restrict__ Vext, T a, T b, T alpha, T* __restrict__ Vout) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nvox) return;
    T rho = 0;
    for (int j = 0; j < n_orb; ++j) {
        const typename C2<T>::t v = phi[(long long)j * nvox + n];
        rho += v.x * v.x + v.y * v.y;
    }
    const T pw = rho > 0 ? pow(rho, (T)1 + alpha) : (T)0;
    Vout[n] = Vext[n] + a * rho + b * pw;
}

// --------------------------------------------------------------------------
// Diagnostics (FP64 sums): per orbital |phi|^2 and Re<phi, H phi>; f^* Q f.
// --------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

template <typename T, int R = 1>
__global__ void diag_phi(int nx, int ny, int nz, int n_orb, T inv_h2, const typename C2<T>::t* __restrict__ phi,
                         const T* __restrict__ V, double* __restrict__ out /* [n_orb][3] */) {
    __shared__ double sh[32];
    const long long nvox = (long long)nx * ny * nz;
    const int orb = blockIdx.y;
    const typename C2<T>::t* w = phi + (long long)orb * nvox;
    double s_norm = 0, s_en = 0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nvox; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % nx), jy = (int)((n / nx) % ny), k = (int)(n / ((long long)nx * ny));
        const typename C2<T>::t c = w[n];
        double hr, hi;
        apply_h<double, R>(w, n, i, jy, k, nx, ny, nz, (double)inv_h2, (double)V[n], c, hr, hi);
        s_norm += (double)c.x * c.x + (double)c.y * c.y;
        s_en += (double)c.x * hr + (double)c.y * hi;
    }
    s_norm = block_sum(s_norm, sh);
    s_en = block_sum(s_en, sh);
    if (threadIdx.x == 0) {
        atomicAdd(out + orb * 3 + 0, s_norm);
        atomicAdd(out + orb * 3 + 2, s_en);
    }
}

template <typename T>
__global__ void diag_aux(int n_gamma, int n_orb, const int* __restrict__ gamma_c, double q_coef,
                         const typename C2<T>::t* __restrict__ f, double* __restrict__ out) {
    __shared__ double sh[32];
    const int orb = blockIdx.y;
    double s = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_gamma; g += gridDim.x * blockDim.x) {
        const typename C2<T>::t v = f[(long long)g * n_orb + orb];
        s += q_coef / gamma_c[g] * ((double)v.x * v.x + (double)v.y * v.y);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(out + orb * 3 + 1, s);
}

// Divergence monitor over the raw diagnostic rows (sums before the h^3 weight:
// [norm, f^* Q f, energy] per orbital) of a run: row r is compared with row r - 1
// (proven forms: W may not grow by more than the slack, Thm 3.1 / Thm 3.2 after
// the time discretisation) or with row 0 (other forms: W may not exceed twice its
// start), and any non-finite W fails.  The first failing row goes to *bad
// (atomicMin; the caller initialises it to a large value), its orbital to bad[1].
static __global__ void diag_monitor(const double* __restrict__ rows, long long r, int n_orb, int proven, double slack,
                             int* __restrict__ bad) {
    for (int j = threadIdx.x; j < n_orb; j += blockDim.x) {
        const double* cur = rows + r * 3 * n_orb + 3 * j;
        const double* ref = rows + (proven ? r - 1 : 0) * 3 * n_orb + 3 * j;
        const double w = cur[0] + cur[1], w0 = ref[0] + ref[1];
        const bool ok = isfinite(w) && (proven ? w <= w0 * (1.0 + slack) : w <= 2.0 * w0);
        if (!ok && atomicMin(bad, (int)r) > (int)r) bad[1] = j;
    }
}

}  // namespace dev
}  // namespace abc

namespace abc {
namespace dev {

// ==========================================================================
// Adjoint (reverse sweep through the Horner stages)
// ==========================================================================
// The adjoint operator of eq:dynamics0 / eq:dynamics1 (H real symmetric):
//   order 0: L^H a = i H a_phi + i E^T M^H E a_phi
//   order 1: L^H (a_phi, a_f) = (i H a_phi + E^T A^H a_f,  i E a_phi + B^H a_f)
// with A^H = +i diag(c)/(4h^4) and B^H = s1 I - conj(S) A^H (S = K(s1)^{-1} symmetric).

// anew_phi = cdt * (i H a_phi + bt),  acc_phi += anew_phi, with the boundary term
//   order 1: bt = A^H a_f = (+i c_gamma a_coef) a_f[gamma]
//   order 0: bt = i cnat[gamma]   (cnat = E^T conj(M) E a_phi)
template <typename T>
__global__ void stencil_adj(int order, int nx, int ny, int nz, int n_orb, T inv_h2, T a_coef,
                            const typename C2<T>::t* __restrict__ a, const T* __restrict__ V,
                            const typename C2<T>::t* __restrict__ bsrc, typename C2<T>::t* acc,
                            typename C2<T>::t* __restrict__ anew, T cdt) {
    typedef typename C2<T>::t Vc;
    const long long nvox = (long long)nx * ny * nz;
    const int tp = blockIdx.x * blockDim.x + threadIdx.x;          // node in the z-plane
    if (tp >= nx * ny) return;
    const int i = tp % nx, jy = tp / nx, k = blockIdx.y, orb = blockIdx.z;
    const long long n = (long long)k * nx * ny + tp;
    const long long idx = (long long)orb * nvox + n;
    const Vc* wo = a + (long long)orb * nvox;
    const Vc c = wo[n];
    T sr = 0, si = 0;
    if (i > 0) { const Vc v = wo[n - 1]; sr += v.x; si += v.y; }
    if (i < nx - 1) { const Vc v = wo[n + 1]; sr += v.x; si += v.y; }
    if (jy > 0) { const Vc v = wo[n - nx]; sr += v.x; si += v.y; }
    if (jy < ny - 1) { const Vc v = wo[n + nx]; sr += v.x; si += v.y; }
    if (k > 0) { const Vc v = wo[n - (long long)nx * ny]; sr += v.x; si += v.y; }
    if (k < nz - 1) { const Vc v = wo[n + (long long)nx * ny]; sr += v.x; si += v.y; }
    const T diag = (T)3 * inv_h2 + V[n];
    const T hr = diag * c.x - (T)0.5 * inv_h2 * sr;
    const T hi = diag * c.y - (T)0.5 * inv_h2 * si;
    // i H a = (-hi, hr)
    T lr = -hi, li = hr;
    const int cnt = (i == 0) + (i == nx - 1) + (jy == 0) + (jy == ny - 1) + (k == 0) + (k == nz - 1);
    if (cnt) {
        const Vc b = bsrc[(long long)gamma_index(i, jy, k, nx, ny, nz) * n_orb + orb];
        if (order == 1) {
            const T ac = a_coef * (T)cnt;
            lr += -ac * b.y;
            li += ac * b.x;
        } else {
            lr += -b.y;
            li += b.x;
        }
    }
    const Vc av = acc[idx];
    const T nr = cdt * lr, ni = cdt * li;
    anew[idx] = mk<T>(nr, ni);
    acc[idx] = mk<T>(av.x + nr, av.y + ni);
}

// grad[x] += coef * sum_j 2 Im(conj(a_j[x]) w_j[x])   (FP64 accumulation, one thread per node)
template <typename T>
__global__ void grad_accum(long long nvox, int n_orb, const typename C2<T>::t* __restrict__ a,
                           const typename C2<T>::t* __restrict__ w, double coef, double* __restrict__ grad) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nvox) return;
    double s = 0;
    for (int j = 0; j < n_orb; ++j) {
        const typename C2<T>::t av = a[(long long)j * nvox + n], wv = w[(long long)j * nvox + n];
        s += (double)av.x * wv.y - (double)av.y * wv.x;
    }
    grad[n] += 2.0 * coef * s;
}

// y = i x
template <typename T>
__global__ void mul_i_into(long long n, const typename C2<T>::t* __restrict__ x, typename C2<T>::t* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const typename C2<T>::t v = x[i];
    y[i] = mk<T>(-v.y, v.x);
}

// adjoint of J = sum_j (1 - h^3 |phi_j|^2):  a_phi = -h^3 phi
template <typename T>
__global__ void scale_into(long long n, const typename C2<T>::t* __restrict__ x, T s, typename C2<T>::t* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const typename C2<T>::t v = x[i];
    y[i] = mk<T>(s * v.x, s * v.y);
}

template <typename T>
__global__ void to_real(long long n, const double* __restrict__ x, T* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (T)x[i];
}

}  // namespace dev
}  // namespace abc
