// Boundary transforms of an order-1 stage with the orbitals across the lanes (complex64,
// n_orb a multiple of 32, the many-orbital tensor-core contraction between them).
//
// The adapted vectors (hat_phi, hat_f) and the contraction output t are held node-major,
// [adapted index][orbital] (orbitals fastest), instead of orbital-major.  A warp takes
// one cell and 32 consecutive orbitals, lane = orbital, and does the cell's whole
// transform for its orbital in registers: the 8-point reflection butterflies of every
// slot and the per-parity 8 x 8 slot mixing (no lane shuffles, no shared memory).  The
// cell's tables and coefficients are the same for every lane of the warp (broadcast
// loads, uniform branches), and every array access of a warp instruction is 32
// consecutive orbitals of one node: 256 contiguous bytes, whether the array is
// node-major or in the natural boundary layout [n_gamma][orbital].  Only the gather of
// w at Gamma from the full state is still one 8-byte value per orbital plane.
//
// The sums are those of bnd_forward_multi / bnd_back_multi, in the same order, so the
// results are bit for bit the same as the orbital-major chain's.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace abc {
namespace dev {

constexpr int LANES_W = 4;          // warps per block

// The 8-point Walsh-Hadamard butterflies of wht8_lanes on eight values in registers
// (element g plays lane g): the same sums in the same order.
__device__ __forceinline__ void wht8_regs(float2 (&x)[8]) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
        float2 y[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float2 o = x[g ^ bit];
            y[g] = (g & bit) ? make_float2(o.x - x[g].x, o.y - x[g].y) : make_float2(x[g].x + o.x, x[g].y + o.y);
        }
#pragma unroll
        for (int g = 0; g < 8; ++g) x[g] = y[g];
    }
}

__device__ __forceinline__ void ld_int8(const int* p, int (&v)[8]) {
    const int4 a = __ldg(reinterpret_cast<const int4*>(p)), b = __ldg(reinterpret_cast<const int4*>(p + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void ld_float8(const float* p, float (&v)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Warp -> (cell, first orbital), chunks of 32 orbitals fastest; false for the idle
// warps of the last block.
__device__ __forceinline__ bool lanes_item(const CellTab<float>& ct, int n_orb, int& cell, int& j) {
    const int nch = n_orb >> 5;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)ct.n_cells * nch) return false;
    cell = (int)(wid / nch);
    j = (int)(wid - (long long)cell * nch) * 32 + (threadIdx.x & 31);
    return true;
}

// Forward transform (bnd_forward_multi's outputs, node-major): hat_phi[jj][j] from w at
// Gamma (gathered from the state w_phi [n_orb][nvox], or read from g_phi in the natural
// boundary layout), hat_f[jj][j] from w_f (natural layout; nullptr: none).  Grid
// ceil(n_cells * n_orb / 32 / LANES_W) blocks of 32 LANES_W threads.
__global__ void __launch_bounds__(32 * LANES_W, 3) bnd_forward_lanes(CellTab<float> ct, int n_orb, long long nvox,
                                                                     const float2* __restrict__ w_phi,
                                                                     const float2* __restrict__ w_f,
                                                                     float2* __restrict__ hat_phi,
                                                                     float2* __restrict__ hat_f,
                                                                     const float2* __restrict__ g_phi) {
    int cell, j;
    if (!lanes_item(ct, n_orb, cell, j)) return;
    const int* gic = ct.gi + (size_t)cell * 64;
    const int* ndc = ct.node + (size_t)cell * 64;
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
#pragma unroll 1
    for (int arr = 0; arr < 2; ++arr) {
        if (arr == 1 && !w_f) break;
        const bool gather = arr == 0 && !g_phi;          // w from the full state
        const float2* nat = arr == 0 ? g_phi : w_f;      // natural boundary layout
        float2 x[8][8];                                  // [slot][reflection, then parity]
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            int gis[8], nds[8];
            ld_int8(gic + s * 8, gis);
            if (gather) ld_int8(ndc + s * 8, nds);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                float2 v = make_float2(0.f, 0.f);
                if (gis[g] >= 0) v = gather ? w_phi[(long long)j * nvox + nds[g]] : nat[(size_t)gis[g] * n_orb + j];
                x[s][g] = v;
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) wht8_regs(x[s]);
        float2* hat = arr == 0 ? hat_phi : hat_f;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const float* cf = ct.coef_f + (size_t)__ldg(tyc + p) * 64;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int jj = __ldg(outc + o * 8 + p);
                if (jj < 0) continue;
                float c[8];
                ld_float8(cf + o * 8, c);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    a.x += c[q] * x[q][p].x;
                    a.y += c[q] * x[q][p].y;
                }
                hat[(size_t)jj * n_orb + j] = a;
            }
        }
    }
}

// Back transform of an order-1 stage (bnd_back_multi's formula, node-major inputs):
// x = s1 f_hat + (-i a)(phi_hat - t) at the cell's outputs, a = a_coef c, t the sum of
// the nsplit arrays t_in + q split_stride; mixed back per parity and transformed back
// per slot; out[e][j] = y_f[e][j] + cdt v at each Gamma index e the cell writes (y_f and
// out natural; out may be y_f: each element is read, then written, by one lane and by
// no other thread, so y_f is read through the read-only path, which leaves the compiler
// free to issue the next loads before the earlier stores).
// The 64 values of a lane pass through its own column of shared memory (LANES_SMEM
// bytes per block, [warp][output o * 8 + parity p][lane]): first x at every output (all
// loads independent of each other, so many are in flight), then the per-parity mixing
// in place (v[s][p] over x[.][p]), then per slot the butterflies and the writes.
constexpr size_t LANES_SMEM = (size_t)LANES_W * 64 * 32 * sizeof(float2);
__global__ void __launch_bounds__(32 * LANES_W, 3) bnd_back_lanes(CellTab<float> ct, int n_orb, float s1, float a_coef,
                                                                  const float2* __restrict__ hat_phi,
                                                                  const float2* __restrict__ hat_f,
                                                                  const float2* __restrict__ t_in, int nsplit,
                                                                  long long split_stride, const float2* y_f,
                                                                  float2* out, float cdt) {
    extern __shared__ float2 lsm[];
    int cell, j;
    if (!lanes_item(ct, n_orb, cell, j)) return;
    const int lane = threadIdx.x & 31;
    float2* xs = lsm + (size_t)(threadIdx.x >> 5) * 64 * 32 + lane;   // this lane's column, stride 32
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
    const int* wrc = ct.wr + (size_t)cell * 64;
    const float a = a_coef * (float)__ldg(ct.cell_c + cell);
#pragma unroll 16
    for (int t = 0; t < 64; ++t) {                       // t = o * 8 + p
        const int jj = __ldg(outc + t);
        float2 x = make_float2(0.f, 0.f);
        if (jj >= 0) {
            const size_t e = (size_t)jj * n_orb + j;
            const float2 fv = hat_f[e], pv = hat_phi[e];
            float2 tv = t_in[e];
            for (int q = 1; q < nsplit; ++q) {
                const float2 u = t_in[(long long)q * split_stride + e];
                tv.x += u.x;
                tv.y += u.y;
            }
            x = back_x1(s1, a, fv, pv, tv);
        }
        xs[t * 32] = x;
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        float2 x[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) x[o] = xs[(o * 8 + p) * 32];
        const float* cb = ct.coef_bt + (size_t)__ldg(tyc + p) * 64;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float c[8];
            ld_float8(cb + s * 8, c);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                acc.x += c[q] * x[q].x;
                acc.y += c[q] * x[q].y;
            }
            xs[(s * 8 + p) * 32] = acc;                  // v[s][p] over x[s][p] (column p read above)
        }
    }
#pragma unroll 2
    for (int s = 0; s < 8; ++s) {
        int wr[8];
        ld_int8(wrc + s * 8, wr);
        float2 y[8], v[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) y[g] = wr[g] >= 0 ? __ldg(y_f + (size_t)wr[g] * n_orb + j) : make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 8; ++p) v[p] = xs[(s * 8 + p) * 32];
        wht8_regs(v);
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (wr[g] >= 0) out[(size_t)wr[g] * n_orb + j] = make_float2(y[g].x + cdt * v[g].x, y[g].y + cdt * v[g].y);
    }
}

// Back transform from x formed by the contraction epilogue (XEpi; node-major): a lane
// loads the cell's 64 values of x into registers (all loads issued together) and mixes
// them back per parity in place; the results go to the lane's shared-memory column
// (LANES_SMEM bytes per block), which frees the registers for all y_f loads of the cell
// at once; then per slot the butterflies and out[e][j] = y_f[e][j] + cdt v (the same
// bits as bnd_back_lanes; y_f through the read-only path, as there).
__global__ void __launch_bounds__(32 * LANES_W, 3) bnd_back_lanes_x(CellTab<float> ct, int n_orb,
                                                                    const float2* __restrict__ x_in,
                                                                    const float2* y_f, float2* out, float cdt) {
    extern __shared__ float2 lsm[];
    int cell, j;
    if (!lanes_item(ct, n_orb, cell, j)) return;
    float2* xs = lsm + (size_t)(threadIdx.x >> 5) * 64 * 32 + (threadIdx.x & 31);
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
    const int* wrc = ct.wr + (size_t)cell * 64;
    {
        float2 v[8][8];                                  // x[o][p], then v[s][p]
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            int jj[8];
            ld_int8(outc + o * 8, jj);
#pragma unroll
            for (int p = 0; p < 8; ++p) v[o][p] = jj[p] >= 0 ? x_in[(size_t)jj[p] * n_orb + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            float2 x[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) x[o] = v[o][p];
            const float* cb = ct.coef_bt + (size_t)__ldg(tyc + p) * 64;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                float c[8];
                ld_float8(cb + s * 8, c);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    acc.x += c[q] * x[q].x;
                    acc.y += c[q] * x[q].y;
                }
                v[s][p] = acc;
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int p = 0; p < 8; ++p) xs[(s * 8 + p) * 32] = v[s][p];
    }
    asm volatile("" ::: "memory");
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        int wr[8];
        ld_int8(wrc + s * 8, wr);
        float2 y[8], v[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) y[g] = wr[g] >= 0 ? __ldg(y_f + (size_t)wr[g] * n_orb + j) : make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 8; ++p) v[p] = xs[(s * 8 + p) * 32];
        wht8_regs(v);
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (wr[g] >= 0) out[(size_t)wr[g] * n_orb + j] = make_float2(y[g].x + cdt * v[g].x, y[g].y + cdt * v[g].y);
    }
}

// ---------------------------------------------------------------------------------
// The same transforms with a cell split between two lanes (ABC_TUNE_LANES 2): a warp
// takes one cell and 16 consecutive orbitals; lanes l and l + 16 share orbital l and
// each holds half of the cell's 64 values, so a lane needs half the registers and twice
// as many warps stay resident.  The halves swap 16 values through one lane shuffle each
// between the reflection butterflies (per slot) and the mixing (per parity).  Every
// access of a warp instruction is two runs of 16 orbitals (128 contiguous bytes each).
// Same sums in the same order as the forms above.  MINB: blocks per SM the registers
// are capped for (4: 128 registers; 5: 96, with a few spilled).
// ---------------------------------------------------------------------------------

__device__ __forceinline__ bool pairs_item(const CellTab<float>& ct, int n_orb, int& cell, int& j, int& h) {
    const int nch = n_orb >> 4;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)ct.n_cells * nch) return false;
    cell = (int)(wid / nch);
    j = (int)(wid - (long long)cell * nch) * 16 + (threadIdx.x & 15);
    h = (threadIdx.x >> 4) & 1;
    return true;
}

__device__ __forceinline__ float2 shfl16(float2 v) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 16), __shfl_xor_sync(0xffffffffu, v.y, 16));
}

// Forward (bnd_forward_lanes's outputs): half h loads and transforms slots 4h .. 4h + 3,
// then mixes parities 4h .. 4h + 3 over all eight slots.  Grid ceil(n_cells * n_orb / 16
// / LANES_W) blocks of 32 LANES_W threads.
template <int MINB>
__global__ void __launch_bounds__(32 * LANES_W, MINB) bnd_forward_pairs(CellTab<float> ct, int n_orb, long long nvox,
                                                                  const float2* __restrict__ w_phi,
                                                                  const float2* __restrict__ w_f,
                                                                  float2* __restrict__ hat_phi,
                                                                  float2* __restrict__ hat_f,
                                                                  const float2* __restrict__ g_phi) {
    int cell, j, h;
    const bool live = pairs_item(ct, n_orb, cell, j, h);
    if (!__any_sync(0xffffffffu, live)) return;      // whole warps only (the shuffles)
    if (!live) return;
    const int* gic = ct.gi + (size_t)cell * 64 + 32 * h;     // this half's slots
    const int* ndc = ct.node + (size_t)cell * 64 + 32 * h;
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
#pragma unroll 1
    for (int arr = 0; arr < 2; ++arr) {
        if (arr == 1 && !w_f) break;
        const bool gather = arr == 0 && !g_phi;
        const float2* nat = arr == 0 ? g_phi : w_f;
        float2 x[4][8];                                  // [slot 4h + s][reflection, then parity]
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int gis[8], nds[8];
            ld_int8(gic + s * 8, gis);
            if (gather) ld_int8(ndc + s * 8, nds);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                float2 v = make_float2(0.f, 0.f);
                if (gis[g] >= 0) v = gather ? w_phi[(long long)j * nvox + nds[g]] : nat[(size_t)gis[g] * n_orb + j];
                x[s][g] = v;
            }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) wht8_regs(x[s]);
        // y[S][q]: slot S (0..7), parity 4h + q; own slots from x, the partner's by shuffle
        float2 y[8][4];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 keep = h ? x[s][4 + q] : x[s][q];
                const float2 got = shfl16(h ? x[s][q] : x[s][4 + q]);
                y[s][q] = h ? got : keep;                // slots 0..3
                y[4 + s][q] = h ? keep : got;            // slots 4..7
            }
        float2* hat = arr == 0 ? hat_phi : hat_f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = 4 * h + q;
            const float* cf = ct.coef_f + (size_t)__ldg(tyc + p) * 64;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int jj = __ldg(outc + o * 8 + p);
                if (jj < 0) continue;
                float c[8];
                ld_float8(cf + o * 8, c);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int S = 0; S < 8; ++S) {
                    a.x += c[S] * y[S][q].x;
                    a.y += c[S] * y[S][q].y;
                }
                hat[(size_t)jj * n_orb + j] = a;
            }
        }
    }
}

// Back from the epilogue's x (bnd_back_lanes_x's outputs): half h loads and mixes
// parities 4h .. 4h + 3, then transforms back slots 4h .. 4h + 3 over all eight
// parities and writes their nodes.
template <int MINB>
__global__ void __launch_bounds__(32 * LANES_W, MINB) bnd_back_pairs_x(CellTab<float> ct, int n_orb,
                                                                 const float2* __restrict__ x_in, const float2* y_f,
                                                                 float2* out, float cdt) {
    int cell, j, h;
    const bool live = pairs_item(ct, n_orb, cell, j, h);
    if (!__any_sync(0xffffffffu, live)) return;
    if (!live) return;
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
    const int* wrc = ct.wr + (size_t)cell * 64 + 32 * h;
    float2 v[8][4];                                      // x[o][q], then v[s][q] (parity 4h + q)
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int4 jq = __ldg(reinterpret_cast<const int4*>(outc + o * 8 + 4 * h));
        const int jj[4] = {jq.x, jq.y, jq.z, jq.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) v[o][q] = jj[q] >= 0 ? x_in[(size_t)jj[q] * n_orb + j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 x[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) x[o] = v[o][q];
        const float* cb = ct.coef_bt + (size_t)__ldg(tyc + 4 * h + q) * 64;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float c[8];
            ld_float8(cb + s * 8, c);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                acc.x += c[o] * x[o].x;
                acc.y += c[o] * x[o].y;
            }
            v[s][q] = acc;
        }
    }
    // u[s][p]: slot 4h + s, parity p (0..7); own parities from v, the partner's by shuffle
    float2 u[4][8];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 keep = h ? v[4 + s][q] : v[s][q];
            const float2 got = shfl16(h ? v[s][q] : v[4 + s][q]);
            u[s][q] = h ? got : keep;                    // parities 0..3
            u[s][4 + q] = h ? keep : got;                // parities 4..7
        }
#pragma unroll
    for (int s = 0; s < 4; ++s) wht8_regs(u[s]);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        int wr[8];
        ld_int8(wrc + s * 8, wr);
        float2 y[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) y[g] = wr[g] >= 0 ? __ldg(y_f + (size_t)wr[g] * n_orb + j) : make_float2(0.f, 0.f);
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (wr[g] >= 0) out[(size_t)wr[g] * n_orb + j] = make_float2(y[g].x + cdt * u[s][g].x, y[g].y + cdt * u[s][g].y);
    }
}

// ---------------------------------------------------------------------------------
// A cell split between four lanes (ABC_TUNE_LANES 4 and 5): a warp takes one cell and 8
// consecutive orbitals; lanes l, l + 8, l + 16, l + 24 share orbital l & 7 and each holds
// a quarter of the cell's values (two slots, then two parities).  The quarters swap
// their values through the warp's own tile of shared memory, laid out so that both the
// writes (one parity of two slots per quarter) and the reads (one slot of two parities
// per quarter) take the two wavefronts 32 eight-byte values need.  Every access of a
// warp instruction is four runs of 8 orbitals (64 contiguous bytes).  Same sums in the
// same order as the forms above.  MINB: blocks per SM the registers are capped for.
// ---------------------------------------------------------------------------------
constexpr int QS_P = 12, QS_S = 8 * QS_P + 4;         // float2 strides of a parity and a slot
constexpr int QS_WARP = 8 * QS_S;                       // float2 per warp

__device__ __forceinline__ bool quads_item(const CellTab<float>& ct, int n_orb, int& cell, int& j, int& r) {
    const int nch = n_orb >> 3;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)ct.n_cells * nch) return false;
    cell = (int)(wid / nch);
    j = (int)(wid - (long long)cell * nch) * 8 + (threadIdx.x & 7);
    r = (threadIdx.x >> 3) & 3;
    return true;
}

// Forward: quarter r loads and transforms slots 2r, 2r + 1, then mixes parities 2r,
// 2r + 1 over all eight slots.
template <int MINB>
__global__ void __launch_bounds__(32 * LANES_W, MINB) bnd_forward_quads(CellTab<float> ct, int n_orb, long long nvox,
                                                                        const float2* __restrict__ w_phi,
                                                                        const float2* __restrict__ w_f,
                                                                        float2* __restrict__ hat_phi,
                                                                        float2* __restrict__ hat_f,
                                                                        const float2* __restrict__ g_phi) {
    __shared__ float2 qs[LANES_W][QS_WARP];
    int cell, j, r;
    if (!quads_item(ct, n_orb, cell, j, r)) return;    // whole warps (the item is per warp)
    float2* sm = qs[threadIdx.x >> 5] + (threadIdx.x & 7);
    const int* gic = ct.gi + (size_t)cell * 64 + 16 * r;     // slots 2r, 2r + 1
    const int* ndc = ct.node + (size_t)cell * 64 + 16 * r;
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
#pragma unroll 1
    for (int arr = 0; arr < 2; ++arr) {
        if (arr == 1 && !w_f) break;
        const bool gather = arr == 0 && !g_phi;
        const float2* nat = arr == 0 ? g_phi : w_f;
        float2 x[2][8];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            int gis[8], nds[8];
            ld_int8(gic + a * 8, gis);
            if (gather) ld_int8(ndc + a * 8, nds);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                float2 v = make_float2(0.f, 0.f);
                if (gis[g] >= 0) v = gather ? w_phi[(long long)j * nvox + nds[g]] : nat[(size_t)gis[g] * n_orb + j];
                x[a][g] = v;
            }
            wht8_regs(x[a]);
        }
        __syncwarp();                                    // the previous array's reads are done
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int p = 0; p < 8; ++p) sm[(2 * r + a) * QS_S + p * QS_P] = x[a][p];
        __syncwarp();
        float2 y[8][2];                                  // slot S, parity 2r + b
#pragma unroll
        for (int S = 0; S < 8; ++S)
#pragma unroll
            for (int b = 0; b < 2; ++b) y[S][b] = sm[S * QS_S + (2 * r + b) * QS_P];
        float2* hat = arr == 0 ? hat_phi : hat_f;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int p = 2 * r + b;
            const float* cf = ct.coef_f + (size_t)__ldg(tyc + p) * 64;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int jj = __ldg(outc + o * 8 + p);
                if (jj < 0) continue;
                float c[8];
                ld_float8(cf + o * 8, c);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int S = 0; S < 8; ++S) {
                    acc.x += c[S] * y[S][b].x;
                    acc.y += c[S] * y[S][b].y;
                }
                hat[(size_t)jj * n_orb + j] = acc;
            }
        }
    }
}

// Back from the epilogue's x: quarter r loads and mixes parities 2r, 2r + 1, then
// transforms back slots 2r, 2r + 1 over all eight parities and writes their nodes.
template <int MINB>
__global__ void __launch_bounds__(32 * LANES_W, MINB) bnd_back_quads_x(CellTab<float> ct, int n_orb,
                                                                       const float2* __restrict__ x_in,
                                                                       const float2* y_f, float2* out, float cdt) {
    __shared__ float2 qs[LANES_W][QS_WARP];
    int cell, j, r;
    if (!quads_item(ct, n_orb, cell, j, r)) return;
    float2* sm = qs[threadIdx.x >> 5] + (threadIdx.x & 7);
    const int* outc = ct.out + (size_t)cell * 64;
    const int* tyc = ct.type + (size_t)cell * 8;
    const int* wrc = ct.wr + (size_t)cell * 64 + 16 * r;
    float2 v[8][2];                                      // x[o][b], then v[s][b] (parity 2r + b)
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int2 jq = __ldg(reinterpret_cast<const int2*>(outc + o * 8 + 2 * r));
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int jj = b ? jq.y : jq.x;
            v[o][b] = jj >= 0 ? x_in[(size_t)jj * n_orb + j] : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float2 x[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) x[o] = v[o][b];
        const float* cb = ct.coef_bt + (size_t)__ldg(tyc + 2 * r + b) * 64;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float c[8];
            ld_float8(cb + s * 8, c);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                acc.x += c[o] * x[o].x;
                acc.y += c[o] * x[o].y;
            }
            v[s][b] = acc;
        }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s)
#pragma unroll
        for (int b = 0; b < 2; ++b) sm[s * QS_S + (2 * r + b) * QS_P] = v[s][b];
    __syncwarp();
    float2 u[2][8];                                      // slot 2r + a, parity p
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int p = 0; p < 8; ++p) u[a][p] = sm[(2 * r + a) * QS_S + p * QS_P];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        wht8_regs(u[a]);
        int wr[8];
        ld_int8(wrc + a * 8, wr);
        float2 y[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) y[g] = wr[g] >= 0 ? __ldg(y_f + (size_t)wr[g] * n_orb + j) : make_float2(0.f, 0.f);
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (wr[g] >= 0) out[(size_t)wr[g] * n_orb + j] = make_float2(y[g].x + cdt * u[a][g].x, y[g].y + cdt * u[a][g].y);
    }
}

// tc_colexp for a node-major x ((moff + row) * n_orb + o): block (class member rm,
// 32 consecutive orbitals, row part) with lane = orbital and its 16 warps taking every
// 16th row of the part; the parts' maxima meet in colmax by atomicMax, and the block
// that completes a column group last (counter) turns them into the exponents and resets
// colmax and the counter for the next call (no block waits for another).  The same
// exponents as tc_colexp.  Grid tc_ncols * n_orb / 32 * CX_PARTS blocks of 512 threads;
// colmax [tc_ncols * n_orb] and count [tc_ncols * n_orb / 32] zero before the first call.
constexpr int CX_WARPS = 16, CX_DEPTH = 8, CX_PARTS = 8;
static __global__ void __launch_bounds__(32 * CX_WARPS) tc_colexp_nm(TcInfo info, int n_orb, const float2* __restrict__ x,
                                                                   int* __restrict__ colexp, unsigned* colmax,
                                                                   unsigned* count) {
    __shared__ uint32_t red[CX_WARPS][32];
    __shared__ bool last;
    const int nog = n_orb >> 5;
    const int part = blockIdx.x % CX_PARTS, grp = blockIdx.x / CX_PARTS;
    const int rm = grp / nog, og = grp - rm * nog;                  // class member (rsum index), orbital group
    int c = 0;
    while (c + 1 < info.ncls && rm >= info.rsum[c + 1]) ++c;
    const int k = rm - info.rsum[c], m = info.m[c];
    const int r_lo = (int)((long long)m * part / CX_PARTS), r_hi = (int)((long long)m * (part + 1) / CX_PARTS);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int o = og * 32 + lane;
    const float2* p = x + (size_t)info.moff[c][k] * n_orb + o;
    uint32_t mx = 0;
    for (int r0 = r_lo + w; r0 < r_hi; r0 += CX_WARPS * CX_DEPTH) {
        float2 v[CX_DEPTH];
#pragma unroll
        for (int u = 0; u < CX_DEPTH; ++u) {
            const int r = r0 + CX_WARPS * u;
            v[u] = r < r_hi ? __ldg(p + (size_t)r * n_orb) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < CX_DEPTH; ++u)
            mx = max(mx, max(__float_as_uint(v[u].x) & 0x7fffffffu, __float_as_uint(v[u].y) & 0x7fffffffu));
    }
    red[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 1; q < CX_WARPS; ++q) mx = max(mx, red[q][lane]);
        atomicMax(colmax + rm * n_orb + o, mx);
        __threadfence();
        __syncwarp();                                    // every lane's maximum before the count
        unsigned done = 0;
        if (lane == 0) done = atomicAdd(count + grp, 1u);
        done = __shfl_sync(0xffffffffu, done, 0);
        if (lane == 0) last = done == CX_PARTS - 1;
    }
    __syncthreads();
    if (w == 0 && last) {
        __threadfence();
        const uint32_t all = atomicExch(colmax + rm * n_orb + o, 0u);     // the final maximum; reset
        int e = 0;
        if (all != 0) {
            const int E = (int)(all >> 23) - 127;
            e = min(TC_COLEXP_MAX, max(-TC_COLEXP_MAX, TC_TARGET_EXP - 1 - E));
        }
        colexp[rm * n_orb + o] = e;
        if (lane == 0) count[grp] = 0u;
    }
}

}  // namespace dev
}  // namespace abc
