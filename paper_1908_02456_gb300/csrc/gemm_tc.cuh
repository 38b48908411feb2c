// Boundary DtN contraction for many orbitals on the 5th-generation tensor cores
// (tcgen05, sm_103a), complex64 in / out with FP32-level accuracy.
//
// Per irreducible class the contraction is T = S X: S the class's m x m complex
// block, X the m x (R b) matrix of its R right-hand sides for b orbitals (adapted
// vectors are orbital-major, so every column of X is contiguous in K).  With
// S = Sr + i Si and X = Xr + i Xi, one accumulator of 2N columns holds
// [Re T | Im T] for an output tile of N columns:
//     [Re T | Im T] = Sr [Xr | Xi] + Si [-Xi | Xr]        (conj(S): + Si [Xi | -Xr])
// so a K step is two real products of width 2N, each 3xTF32: with a = a_hi + a_lo
// (a_hi the operand rounded to TF32, a_lo the remainder as TF32),
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, i.e. 6 MMAs (kind::tf32, M = 128, N = 2N, K = 8).
//
// Operand layout in shared memory: K-major, no swizzle, canonical 8-row x 16-byte
// core matrices (row stride 16 B inside a core matrix, LBO = 128 B between core
// matrices along K, SBO = 512 B between 8-row groups, 16-deep K blocks).  The host
// pre-splits and pre-packs S in exactly that image (4 planes Sr_hi, Sr_lo, Si_hi,
// Si_lo of 128 x 16 FP32 = 32 KB per (class, 128-row tile, K block)); pack_x_tc packs
// X once per contraction as 6 planes of N rows x 16 per (column range, K block):
// (-Xi, Xr, Xi) for S and (Xr, Xi, -Xr) for conj(S), hi parts then lo parts, so both
// width-2N operands of a product are windows of two adjacent planes.
//
// The split-FP16 form (TC_F16) runs the same products with FP16 hi + lo operands on
// kind::f16 (twice the TF32 rate): a K block is then 32 elements deep in the same
// 64-byte rows, so one MMA (K = 16) still spans two core matrices along K.  FP16
// keeps TF32's 10 mantissa bits but not its exponent range, so each class block is
// scaled by a power of two 2^es (its largest part near 2^14, on the host) and each
// right-hand-side column by 2^ec (tc_colexp, per contraction); the epilogue
// multiplies by 2^-(es + ec).  Power-of-two scales are exact, so the products carry
// the same rounding as 3xTF32.
//
// gemm_tc is persistent: one CTA per SM works through its own list of (output tile,
// K split) items, balanced by the host.  Warp 0 streams the A and X chunks of all its
// items through one 3-stage ring with 1D bulk copies (mbarrier completion), warp 1
// issues the MMAs and frees each slot with tcgen05.commit, and warps 2-5 run the
// epilogue; the accumulators of consecutive items alternate between two TMEM buffers,
// so the epilogue of one item overlaps the MMAs of the next.  Split-K partials go to
// separate buffers that the back transform adds in a fixed order.  Every mbarrier wait
// is bounded: on a timeout the kernel raises the error flag, stops issuing, waits
// (bounded) for its own copies and MMAs, frees its TMEM and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_fp16.h>

#include "sym_gemv.cuh"

namespace abc {
namespace dev {

constexpr int TC_TF32 = 0;                         // kind::tf32, K block of 16 four-byte elements
constexpr int TC_F16 = 1;                          // kind::f16, K block of 32 two-byte elements
template <int KIND>
struct TcKind {
    static constexpr int KB = KIND == TC_F16 ? 32 : 16;     // K elements per 64-byte row
    static constexpr int EB = KIND == TC_F16 ? 2 : 4;       // bytes per element
};

constexpr int TC_M = 128;
constexpr int TC_KB = 16;                          // K elements per pipeline stage (TF32)
constexpr int TC_NMAX = 96;                        // largest output tile width (accumulator 2 TC_NMAX)
constexpr int TC_THREADS = 192;                    // producer, MMA issuer, four epilogue warps
constexpr uint32_t TC_A_PLANE = TC_M * TC_KB * 4;  // 8 KB
constexpr uint32_t TC_A_BYTES = 4 * TC_A_PLANE;    // 32 KB per (tile, K block)
constexpr int TC_B_PLANES = 6;
constexpr uint32_t TC_B_PLANE = TC_NMAX * TC_KB * 4;
constexpr uint32_t TC_B_BYTES = TC_B_PLANES * TC_B_PLANE;   // 36 KB: the packed X chunk stride in global memory
constexpr int TC_MAX_SPLIT = 8;
constexpr int TC_PACK_KB = 4;                      // K blocks packed per pack_x_tc block

// Tile configurations of the persistent GEMM (chosen per shape by the autotuner):
// NMX output columns at most per tile, STG ring stages, CPS resident CTAs per SM.
// TMEM holds two accumulators of 2 NMX columns (rounded up to a power of two).
// KARA = 1: the complex product by Karatsuba's three real products, P1 = Sr Xr,
// P2 = Si Xi, P3 = (Sr + Si)(Xr + Xi), Re T = P1 - P2, Im T = P3 - P1 - P2: 9 MMAs of
// width N per K step instead of 6 of width 2N (a quarter less tensor work), with a
// third pair of A planes (Sr + Si, hi and lo) and three accumulators of N columns.
template <int NMX, int STG, int CPS, int KARA = 0>
struct TcCfg {
    static constexpr int nmax = NMX, stages = STG, cps = CPS, kara = KARA;
    static constexpr uint32_t a_bytes = (KARA ? 6u : 4u) * TC_A_PLANE;
    static constexpr uint32_t b_stage = (uint32_t)TC_B_PLANES * NMX * 64;
    static constexpr uint32_t acc_cols = (KARA ? 3 : 2) * NMX;     // one item's accumulators
    static constexpr uint32_t tmem_cols = 2 * acc_cols > 256 ? 512 : 2 * acc_cols > 128 ? 256 : 128;
    static constexpr uint32_t buf_cols = tmem_cols / 2;
    static constexpr size_t smem = (size_t)STG * (a_bytes + b_stage) + 256;
};
typedef TcCfg<96, 3, 1> TcWide;                    // 96 columns, one CTA per SM
typedef TcCfg<64, 2, 2> TcNarrow;                  // 64 columns, two CTAs per SM
typedef TcCfg<64, 3, 1, 1> TcKara;                 // Karatsuba, 64 columns, one CTA per SM
constexpr long long TC_WAIT_LIMIT = 1ll << 24;

// Byte offset of element (row r, k) inside a K-major no-swizzle plane of 16-deep
// K blocks (core matrix (r / 8, k / 4), row r % 8, element k % 4).
__host__ __device__ inline uint32_t tc_core_offset(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
// The same for two-byte elements in 32-deep K blocks (8 elements per core-matrix row).
__host__ __device__ inline uint32_t tc_core_offset_f16(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// 2^e as a float for |e| <= 126 (exact: exponent bits only).
__host__ __device__ inline float tc_exp2i(int e) {
    union { uint32_t u; float f; } v;
    v.u = (uint32_t)(127 + e) << 23;
    return v.f;
}
constexpr int TC_COLEXP_MAX = 126;                 // |ec| bound of the column scales (float range)
constexpr int TC_TARGET_EXP = 14;                  // scaled parts below 2^14 (FP16 max 65504)

// Output tile: class, first row, first column of the class's R*b columns, width, and
// the first of its packed X chunks (one per K block).
struct TcTile {
    int cls, row0, col0, n, bchunk0;
};
// One column range of a class, packed by pack_x_tc into nkb chunks from bchunk0.
struct TcCols {
    int cls, col0, n, bchunk0;
};

struct TcInfo {
    int m[SYM_CMAX];
    int R[SYM_CMAX];
    int moff[SYM_CMAX][3];
    int nkb[SYM_CMAX];                 // K blocks of the class
    long long abase[SYM_CMAX];         // first A chunk (32 KB units) of the class
    int es[SYM_CMAX];                  // TC_F16: the class block is stored times 2^es
    int rsum[SYM_CMAX];                // right-hand sides of the classes before this one
    int ncls;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;   // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    return d;                                      // base offset 0, no swizzle
}

// D = F32, A = B = TF32 (kind::tf32) or F16 (kind::f16), both K-major, M = 128, N = n.
template <int KIND>
__device__ __forceinline__ uint32_t tc_idesc(int n) {
    const uint32_t fmt = KIND == TC_F16 ? 0u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == TC_F16)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint32_t tf32_hi(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One unit of a CTA's work list: an output tile over one K split.
struct TcItem {
    int tile, split;
};

// X -> packed TF32 planes of every K block of a column range, in the shared-memory
// image the GEMM copies with one bulk copy per K block: hi planes (-Xi, Xr, Xi), then
// lo planes in the same order (conj: (Xr, Xi, -Xr)).  Grid (column ranges, largest
// nkb / TC_PACK_KB), 128 threads, TC_PACK_KB consecutive K blocks per block; x
// orbital-major (o * ng + j), or node-major (j * n_orb + o) when nm is set.  TC_F16:
// FP16 hi + lo of the column scaled by 2^colexp[column], 8 elements per 16-byte
// core-matrix row.
template <int KIND, int KARA = 0>
__global__ void __launch_bounds__(128) pack_x_tc(TcInfo info, const TcCols* __restrict__ cols, int n_orb, int ng,
                                                 const float2* __restrict__ x, int conj, float* __restrict__ bpack,
                                                 const int* __restrict__ colexp, int nm = 0) {
    constexpr int EPR = 16 / TcKind<KIND>::EB;          // elements per 16-byte row
    const TcCols cr = cols[blockIdx.x];
    const int c = cr.cls;
    const int m = info.m[c], N = cr.n;
    for (int kbi = 0; kbi < TC_PACK_KB; ++kbi) {
    const int kb = blockIdx.y * TC_PACK_KB + kbi;
    if (kb >= info.nkb[c]) return;
    unsigned char* B = reinterpret_cast<unsigned char*>(bpack + (size_t)(cr.bchunk0 + kb) * (TC_B_BYTES / 4));
    for (int it = threadIdx.x; it < N * 4; it += blockDim.x) {
        const int cc = (it & 7) | ((it >> 5) << 3), q = (it >> 3) & 3;
        const int col = cr.col0 + cc;
        const int k = col / n_orb, o = col - k * n_orb;
        float sc = 1.0f;
        if constexpr (KIND == TC_F16)
            if (k < info.R[c]) sc = tc_exp2i(colexp[info.rsum[c] * n_orb + col]);
        float re[EPR], im[EPR];
#pragma unroll
        for (int e = 0; e < EPR; ++e) {
            const int row = kb * TcKind<KIND>::KB + EPR * q + e;
            float2 v = make_float2(0.f, 0.f);
            if (k < info.R[c] && row < m)
                v = __ldg(nm ? x + (size_t)(info.moff[c][k] + row) * n_orb + o : x + (size_t)o * ng + info.moff[c][k] + row);
            re[e] = v.x * sc;
            im[e] = v.y * sc;
        }
        // Karatsuba planes: (Xr, Xi, Xr + Xi), conj: the same of conj(X)
        if constexpr (KARA) {
#pragma unroll
            for (int e = 0; e < EPR; ++e) {
                if (conj) im[e] = -im[e];
            }
        }
        // planes 0-2 (hi) and 3-5 (lo) of this 16-byte row
        uint32_t w[6][4];
        if constexpr (KARA) {
            float sm[EPR];
#pragma unroll
            for (int e = 0; e < EPR; ++e) sm[e] = re[e] + im[e];
            if constexpr (KIND == TC_F16) {
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    const float* src[3] = {re, im, sm};
#pragma unroll
                    for (int pl = 0; pl < 3; ++pl) {
                        const __half2 hh = __floats2half2_rn(src[pl][2 * e2], src[pl][2 * e2 + 1]);
                        const float2 hf = __half22float2(hh);
                        const __half2 ll = __floats2half2_rn(src[pl][2 * e2] - hf.x, src[pl][2 * e2 + 1] - hf.y);
                        w[pl][e2] = *reinterpret_cast<const uint32_t*>(&hh);
                        w[3 + pl][e2] = *reinterpret_cast<const uint32_t*>(&ll);
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float* src[3] = {re, im, sm};
#pragma unroll
                    for (int pl = 0; pl < 3; ++pl) {
                        const uint32_t hh = tf32_hi(src[pl][e]);
                        w[pl][e] = hh;
                        w[3 + pl][e] = tf32_hi(src[pl][e] - __uint_as_float(hh));
                    }
                }
            }
        } else if constexpr (KIND == TC_F16) {
            const uint32_t sgn = 0x80008000u;
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const __half2 rh = __floats2half2_rn(re[2 * e2], re[2 * e2 + 1]);
                const __half2 ih = __floats2half2_rn(im[2 * e2], im[2 * e2 + 1]);
                const float2 rhf = __half22float2(rh), ihf = __half22float2(ih);
                const __half2 rl = __floats2half2_rn(re[2 * e2] - rhf.x, re[2 * e2 + 1] - rhf.y);
                const __half2 il = __floats2half2_rn(im[2 * e2] - ihf.x, im[2 * e2 + 1] - ihf.y);
                const uint32_t urh = *reinterpret_cast<const uint32_t*>(&rh), uih = *reinterpret_cast<const uint32_t*>(&ih);
                const uint32_t url = *reinterpret_cast<const uint32_t*>(&rl), uil = *reinterpret_cast<const uint32_t*>(&il);
                if (conj) {
                    w[0][e2] = urh; w[1][e2] = uih; w[2][e2] = urh ^ sgn;
                    w[3][e2] = url; w[4][e2] = uil; w[5][e2] = url ^ sgn;
                } else {
                    w[0][e2] = uih ^ sgn; w[1][e2] = urh; w[2][e2] = uih;
                    w[3][e2] = uil ^ sgn; w[4][e2] = url; w[5][e2] = uil;
                }
            }
        } else {
            const uint32_t sgn = 0x80000000u;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t rh = tf32_hi(re[e]), ih = tf32_hi(im[e]);
                const uint32_t rl = tf32_hi(re[e] - __uint_as_float(rh)), il = tf32_hi(im[e] - __uint_as_float(ih));
                if (conj) {
                    w[0][e] = rh; w[1][e] = ih; w[2][e] = rh ^ sgn;
                    w[3][e] = rl; w[4][e] = il; w[5][e] = rl ^ sgn;
                } else {
                    w[0][e] = ih ^ sgn; w[1][e] = rh; w[2][e] = ih;
                    w[3][e] = il ^ sgn; w[4][e] = rl; w[5][e] = il;
                }
            }
        }
        // planes of a chunk are N * 64 bytes apart (only the tile's N rows are stored);
        // the 16-byte row of column cc and row group q sits where element (cc, EPR q) does
        const uint32_t off = KIND == TC_F16 ? tc_core_offset_f16(cc, EPR * q) : tc_core_offset(cc, EPR * q);
        const uint32_t pb = (uint32_t)N * 64;
#pragma unroll
        for (int p = 0; p < 6; ++p)
            *reinterpret_cast<uint4*>(B + p * pb + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
    }
}

// TC_F16 column scales: for every right-hand-side column of every class (index
// rsum[c] * n_orb + k * n_orb + o) the exponent ec with max |part| * 2^ec in
// [2^13, 2^14), clamped to +-TC_COLEXP_MAX (0 for an all-zero column; the largest
// FP32 subnormals reach 2^-23 after the clamp, still an FP16 value).  One warp per
// column; x orbital-major.
static __global__ void __launch_bounds__(256) tc_colexp(TcInfo info, int n_orb, int ng, const float2* __restrict__ x,
                                                 int* __restrict__ colexp, int ncols) {
    const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gw >= ncols) return;
    int c = 0;
    while (c + 1 < info.ncls && gw >= info.rsum[c + 1] * n_orb) ++c;
    const int col = gw - info.rsum[c] * n_orb;
    const int k = col / n_orb, o = col - k * n_orb;
    const float2* p = x + (size_t)o * ng + info.moff[c][k];
    const int m = info.m[c];
    uint32_t mx = 0;
    // eight independent loads in flight per lane
    for (int r0 = 0; r0 < m; r0 += 256) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u * 32 + lane;
            v[u] = r < m ? __ldg(p + r) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            mx = max(mx, max(__float_as_uint(v[u].x) & 0x7fffffffu, __float_as_uint(v[u].y) & 0x7fffffffu));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if (lane == 0) {
        int e = 0;
        if (mx != 0) {
            const int E = (int)(mx >> 23) - 127;              // floor(log2(max)) (subnormals: -127)
            e = min(TC_COLEXP_MAX, max(-TC_COLEXP_MAX, TC_TARGET_EXP - 1 - E));
        }
        colexp[gw] = e;
    }
}

// One CTA per SM over the items item_off[blockIdx.x] .. item_off[blockIdx.x + 1] of
// items[]; out + split * split_stride receives each item's (split's) partial product,
// orbital-major (o * ng + j), or node-major (j * n_orb + o) when nm is set (n_orb a
// multiple of 16: each 16-column group of a tile is then 16 consecutive orbitals of one
// right-hand side, stored as 128 contiguous bytes).
// Order-1 back-transform input (xe.ac set; node-major, one split): instead of t the
// epilogue stores x = s1 f_hat + (-i a)(phi_hat - t) (back_x1), a = xe.ac[j] per adapted
// index, f_hat and phi_hat node-major.
struct XEpi {
    const float2* hf;
    const float2* hp;
    const float* ac;
    float s1;
};
template <int KIND, typename CFG>
__global__ void __launch_bounds__(TC_THREADS, CFG::cps)
gemm_tc(TcInfo info, const TcTile* __restrict__ tiles, const TcItem* __restrict__ items,
        const int* __restrict__ item_off, const float* __restrict__ apack, const float* __restrict__ bpack, int n_orb,
        int ng, int nsplit, long long split_stride, float2* __restrict__ out, int conj, int* __restrict__ err,
        const int* __restrict__ colexp, int nm = 0, XEpi xe = XEpi{}) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;                                       // [stage][4 or 6 planes]
    constexpr int TC_STAGES = CFG::stages;
    constexpr uint32_t SB = CFG::b_stage;                              // smem bytes of one X stage
    constexpr uint32_t SA = CFG::a_bytes;                              // smem bytes of one A stage
    unsigned char* sB = tc_smem + (size_t)TC_STAGES * SA;              // [stage][6 planes]
    uint64_t* full = reinterpret_cast<uint64_t*>(tc_smem + (size_t)TC_STAGES * (SA + SB));
    uint64_t* empty = full + TC_STAGES;
    uint64_t* tfull = empty + TC_STAGES;                               // [2] accumulators ready
    uint64_t* tempty = tfull + 2;                                      // [2] accumulators drained
    uint64_t* fin = tempty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(fin + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = item_off[blockIdx.x], i1 = item_off[blockIdx.x + 1];
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);                  // the four epilogue warps
        }
        mbar_init(fin, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(CFG::tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    bool ok = true;
    long long issued = 0;                              // producer: K blocks copied
    if (tid == 0) {
        // ---------------- producer ----------------
        for (int it = i0; it < i1 && ok; ++it) {
            const TcItem w = items[it];
            const TcTile tile = tiles[w.tile];
            const int c = tile.cls, nkb = info.nkb[c], N = tile.n;
            const int kb0 = (int)((long long)nkb * w.split / nsplit), kb1 = (int)((long long)nkb * (w.split + 1) / nsplit);
            const float* achunk = apack + (size_t)(info.abase[c] + (long long)(tile.row0 / TC_M) * nkb) * (SA / 4);
            const float* bchunk = bpack + (size_t)tile.bchunk0 * (TC_B_BYTES / 4);
            const uint32_t b_bytes = (uint32_t)N * 64 * TC_B_PLANES;
            for (int kb = kb0; kb < kb1 && ok; ++kb, ++issued) {
                const int st = (int)(issued % TC_STAGES);
                if (issued >= TC_STAGES) ok &= mbar_wait_bounded(&empty[st], (uint32_t)((issued / TC_STAGES - 1) & 1));
                mbar_expect_tx(&full[st], SA + b_bytes);
                bulk_g2s(sA + (size_t)st * SA, achunk + (size_t)kb * (SA / 4), SA, &full[st]);
                bulk_g2s(sB + (size_t)st * SB, bchunk + (size_t)kb * (TC_B_BYTES / 4), b_bytes, &full[st]);
            }
        }
    } else if (tid == 32) {
        // ---------------- MMA issuer ----------------
        long long g = 0;                               // K blocks consumed
        int q = 0;                                     // items with K blocks
        for (int it = i0; it < i1 && ok; ++it) {
            const TcItem w = items[it];
            const TcTile tile = tiles[w.tile];
            const int c = tile.cls, nkb = info.nkb[c], N = tile.n;
            const int kb0 = (int)((long long)nkb * w.split / nsplit), kb1 = (int)((long long)nkb * (w.split + 1) / nsplit);
            if (kb1 <= kb0) continue;
            const int buf = q & 1;
            if (q >= 2) ok &= mbar_wait_bounded(&tempty[buf], (uint32_t)((q / 2 - 1) & 1));
            tc_fence_after();
            const uint32_t idesc = tc_idesc<KIND>(CFG::kara ? N : 2 * N);
            const uint32_t d = tmem + buf * CFG::buf_cols;                // [Re | Im] (2N) or [P1 | P2 | P3] (3N)
            const uint32_t pb = (uint32_t)N * 64;                         // X plane stride in the chunk
            // windows of two planes: [Xr | Xi] and [-Xi | Xr] (conj: [Xr | Xi] and [Xi | -Xr])
            const uint32_t wr = conj ? 0u : pb, wi = conj ? pb : 0u, lo = 3 * pb;
            for (int kb = kb0; kb < kb1 && ok; ++kb, ++g) {
                const int st = (int)(g % TC_STAGES);
                ok &= mbar_wait_bounded(&full[st], (uint32_t)((g / TC_STAGES) & 1));
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + (size_t)st * SA), b0 = smem_u32(sB + (size_t)st * SB);
                if constexpr (CFG::kara) {
#pragma unroll
                    for (int ks = 0; ks < TC_KB / 8; ++ks) {
                        const uint32_t ko = ks * 256;
                        const uint32_t acc0 = (kb > kb0 || ks > 0) ? 1u : 0u;
#pragma unroll
                        for (int pr = 0; pr < 3; ++pr) {       // P1 = Sr Xr, P2 = Si Xi, P3 = Ss Xs
                            const uint64_t ah = tc_desc(a0 + (2 * pr) * TC_A_PLANE + ko);
                            const uint64_t al = tc_desc(a0 + (2 * pr + 1) * TC_A_PLANE + ko);
                            const uint64_t bh = tc_desc(b0 + pr * pb + ko), bl = tc_desc(b0 + lo + pr * pb + ko);
                            const uint32_t dp = d + pr * (uint32_t)N;
                            tc_mma<KIND>(dp, ah, bh, idesc, acc0);
                            tc_mma<KIND>(dp, ah, bl, idesc, 1u);
                            tc_mma<KIND>(dp, al, bh, idesc, 1u);
                        }
                    }
                    tc_commit(&empty[st]);
                    continue;
                }
#pragma unroll
                for (int ks = 0; ks < TC_KB / 8; ++ks) {
                    const uint32_t ko = ks * 256;      // two core matrices along K per MMA
                    const uint64_t srh = tc_desc(a0 + 0 * TC_A_PLANE + ko), srl = tc_desc(a0 + 1 * TC_A_PLANE + ko);
                    const uint64_t sih = tc_desc(a0 + 2 * TC_A_PLANE + ko), sil = tc_desc(a0 + 3 * TC_A_PLANE + ko);
                    const uint64_t brh = tc_desc(b0 + wr + ko), brl = tc_desc(b0 + lo + wr + ko);
                    const uint64_t bih = tc_desc(b0 + wi + ko), bil = tc_desc(b0 + lo + wi + ko);
                    const uint32_t acc0 = (kb > kb0 || ks > 0) ? 1u : 0u;
                    tc_mma<KIND>(d, srh, brh, idesc, acc0);
                    tc_mma<KIND>(d, srh, brl, idesc, 1u);
                    tc_mma<KIND>(d, srl, brh, idesc, 1u);
                    tc_mma<KIND>(d, sih, bih, idesc, 1u);
                    tc_mma<KIND>(d, sih, bil, idesc, 1u);
                    tc_mma<KIND>(d, sil, bih, idesc, 1u);
                }
                tc_commit(&empty[st]);                // the slot is free once these MMAs are done
            }
            tc_commit(&tfull[buf]);                   // the item's accumulators are complete
            ++q;
        }
        tc_commit(fin);
        ok &= mbar_wait_bounded(fin, 0);              // every MMA done before the TMEM is freed
    } else if (warp >= 2) {
        // ---------------- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 ----------------
        const int quad = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        int q = 0;
        for (int it = i0; it < i1 && ok; ++it) {
            const TcItem w = items[it];
            const TcTile tile = tiles[w.tile];
            const int c = tile.cls, nkb = info.nkb[c], N = tile.n, m = info.m[c];
            const int kb0 = (int)((long long)nkb * w.split / nsplit), kb1 = (int)((long long)nkb * (w.split + 1) / nsplit);
            const bool any = kb1 > kb0;
            const int buf = q & 1;
            if (any) {
                ok &= mbar_wait_bounded(&tfull[buf], (uint32_t)((q / 2) & 1));
                ok = __all_sync(0xffffffffu, ok);      // the warp stays converged for tcgen05.ld
                if (!ok) break;
                tc_fence_after();
            }
            const int row = tile.row0 + quad * 32 + lane;
            float2* dst = out + (size_t)w.split * split_stride;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float pr[16], pi[16];
                // x form: this row's f_hat and phi_hat over the 16 columns, loaded before
                // the accumulator is read
                float4 fh[8], ph[8];
                float ar = 0.f;
                const int colx = tile.col0 + c0, kx = colx / n_orb;
                const bool xrow = xe.ac && row < m && c0 < N && kx < info.R[c];
                if (xrow) {
                    const size_t rb = (size_t)(info.moff[c][kx] + row) * n_orb + (colx - kx * n_orb);
                    ar = __ldg(xe.ac + info.moff[c][kx] + row);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        fh[i] = __ldg(reinterpret_cast<const float4*>(xe.hf + rb) + i);
                        ph[i] = __ldg(reinterpret_cast<const float4*>(xe.hp + rb) + i);
                    }
                }
                if (any) {
                    tc_ld16(lane_base + buf * CFG::buf_cols + c0, pr);
                    tc_ld16(lane_base + buf * CFG::buf_cols + N + c0, pi);
                    if constexpr (CFG::kara) {
                        float p3[16];
                        tc_ld16(lane_base + buf * CFG::buf_cols + 2 * N + c0, p3);
                        tc_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; ++i) {       // Re = P1 - P2, Im = P3 - P1 - P2 (conj: -Im)
                            const float re = pr[i] - pi[i], im = p3[i] - pr[i] - pi[i];
                            pr[i] = re;
                            pi[i] = conj ? -im : im;
                        }
                    } else {
                        tc_wait_ld();
                    }
                }
                if (row < m && nm) {
                    const int col = tile.col0 + c0;
                    const int k = col / n_orb, o = col - k * n_orb;
                    if (c0 < N && k < info.R[c]) {
                        float4* d4 = reinterpret_cast<float4*>(dst + (size_t)(info.moff[c][k] + row) * n_orb + o);
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            float2 v0 = any ? make_float2(pr[i], pi[i]) : make_float2(0.f, 0.f);
                            float2 v1 = any ? make_float2(pr[i + 1], pi[i + 1]) : make_float2(0.f, 0.f);
                            if constexpr (KIND == TC_F16) {      // as below, element by element
                                const float sc = tc_exp2i(-info.es[c]);
                                const float s0 = tc_exp2i(-colexp[info.rsum[c] * n_orb + col + i]);
                                const float s1 = tc_exp2i(-colexp[info.rsum[c] * n_orb + col + i + 1]);
                                v0 = make_float2(v0.x * sc * s0, v0.y * sc * s0);
                                v1 = make_float2(v1.x * sc * s1, v1.y * sc * s1);
                            }
                            if (xrow) {
                                const float4 f4 = fh[i >> 1], p4 = ph[i >> 1];
                                v0 = back_x1(xe.s1, ar, make_float2(f4.x, f4.y), make_float2(p4.x, p4.y), v0);
                                v1 = back_x1(xe.s1, ar, make_float2(f4.z, f4.w), make_float2(p4.z, p4.w), v1);
                            }
                            d4[i >> 1] = make_float4(v0.x, v0.y, v1.x, v1.y);
                        }
                    }
                } else if (row < m) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int col = tile.col0 + c0 + i;
                        const int k = col / n_orb, o = col - k * n_orb;
                        if (c0 + i < N && k < info.R[c]) {
                            float2 v = any ? make_float2(pr[i], pi[i]) : make_float2(0.f, 0.f);
                            if constexpr (KIND == TC_F16) {      // undo the power-of-two scales, one at a time
                                const float sc = tc_exp2i(-info.es[c]);
                                const float sx = tc_exp2i(-colexp[info.rsum[c] * n_orb + col]);
                                v = make_float2(v.x * sc * sx, v.y * sc * sx);
                            }
                            dst[(size_t)o * ng + info.moff[c][k] + row] = v;
                        }
                    }
                }
            }
            if (any) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                ++q;
            }
        }
    }
    // the producer's last copies land before the CTA frees its shared memory (they have,
    // unless a wait gave up)
    if (tid == 0)
        for (long long g = issued > TC_STAGES ? issued - TC_STAGES : 0; g < issued; ++g)
            ok &= mbar_wait_bounded(&full[g % TC_STAGES], (uint32_t)((g / TC_STAGES) & 1));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CFG::tmem_cols)
                     : "memory");
    }
    if (!ok) atomicExch(err, 1);
}

}  // namespace dev
}  // namespace abc
