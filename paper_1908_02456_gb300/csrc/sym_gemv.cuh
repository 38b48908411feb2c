// Boundary DtN contraction for one orbital on symmetric packed tiles (sm_103a).
//
// Each irreducible class block S (complex symmetric, m x m, applied to the class's
// R <= 3 right-hand sides) is stored as its lower triangle of 64 x 64 tiles, each
// tile contiguous (32 KB in complex64).  A tile (I, J <= I) serves twice:
//     t_I += S_IJ x_J          (row part)
//     t_J += S_IJ^T x_I        (column part, J < I)
// for every right-hand side x of the class.  One producer warp streams the tiles
// with 1D bulk copies (cp.async.bulk) into a shared-memory ring ("full" mbarriers);
// its lanes also stage, next to each tile, the slices x_J (the tile's columns) and x_I
// (its rows) of every right-hand side, so the consumers never wait on global loads.
// Eight consumer warps in two groups of four take alternate tiles; within a group,
// thread (warp wq, lane l) owns the column pairs cp = 4 wq + l/8 and cp + 16 and the
// eight rows 8(l%8) .. 8(l%8)+7 of the tile.  The host packs each tile in exactly that
// order (sym_pack_index), so chunk i of one column-pair half is one contiguous 2 KB
// run and every 16-byte shared load is conflict-free.  A warp releases a slot through
// its group's "empty" mbarrier once the values are in registers, sums the column part
// over its 8 row groups by shuffles, and keeps the row part in registers until its
// (class, tile-row) segment ends, when each warp stores its own partial.
// Every wait is bounded: a wait that gives up raises an error flag, and all warps
// still follow the same control flow to the end, so no barrier can hang.  Partial
// sums go to global scratch; the back transform of the stage gathers them in a
// fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace abc {
namespace dev {

constexpr int SYM_T = 64;                        // tile edge
constexpr int SYM_CONSUMERS = 8;                 // consumer warps
constexpr int SYM_THREADS = (SYM_CONSUMERS + 1) * 32;
constexpr int SYM_STAGES = 6;
constexpr int SYM_RMAX = 3;
constexpr uint32_t SYM_TILE_BYTES = SYM_T * SYM_T * 8;
constexpr size_t SYM_XS_FLOAT2 = 2 * SYM_RMAX * SYM_T;   // per ring slot: x_J and x_I of the tile
constexpr size_t SYM_XS_BYTES = (size_t)SYM_STAGES * SYM_XS_FLOAT2 * 8;
constexpr int SYM_SEG_CACHE = 64;                // segments of a CTA kept in shared memory
constexpr size_t SYM_SMEM =
    SYM_STAGES * (size_t)SYM_TILE_BYTES + SYM_XS_BYTES + 2 * SYM_STAGES * 8 + SYM_SEG_CACHE * 20;
constexpr long long SYM_WAIT_LIMIT = 1ll << 24;  // try_wait polls before giving up

// Complex offset of tile element (row, col) in the packed tile: chunk row % 8 of
// consumer thread t = 32 (col / 8) + 8 ((col / 2) % 4) + row / 8, element col & 1.
__host__ __device__ inline int sym_pack_index(int row, int col) {
    const int t = (col >> 3) * 32 + ((col >> 1) & 3) * 8 + (row >> 3);
    return ((row & 7) * 256 + t) * 2 + (col & 1);
}

constexpr int SYM_CMAX = 16;
struct SymInfo {
    int nclass;
    int R[SYM_CMAX];              // right-hand sides of the class
    int m[SYM_CMAX];              // block size
    int nt[SYM_CMAX];             // tile rows
    int moff[SYM_CMAX][3];        // adapted offset of each right-hand side
    long long tbase[SYM_CMAX];    // first global tile of the class
    int rbase[SYM_CMAX];          // first (class, tile-row) index of the class
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Adds bytes to the barrier's expected transaction count without arriving.
__device__ __forceinline__ void mbar_add_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 8-byte asynchronous copy global -> shared; src_bytes = 0 fills the destination with zeros.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// One arrival on the barrier once this thread's earlier cp.async copies have landed.
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Same copy with an L2 eviction-priority hint (a policy from createpolicy).
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Tiles with a global index below `keep` are copied with the evict_last L2 policy
// (they outlast other traffic from one stage to the next), the rest with the
// default policy.
__device__ __forceinline__ void tile_copy(void* dst, const float2* tiles, long long t, uint64_t* bar, long long keep) {
    const float2* src = tiles + (size_t)t * 64 * 64;
    if (t < keep) bulk_g2s_hint(dst, src, 64 * 64 * 8, bar, policy_evict_last());
    else bulk_g2s(dst, src, 64 * 64 * 8, bar);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed, false after SYM_WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < SYM_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 16-byte shared-memory load.
__device__ __forceinline__ float4 lds128(const void* p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

// The FMAs of one column pair of a tile for thread (tq, cp): row part into racc,
// column part (OFFDIAG) into cacc.
template <int R, bool CONJ, bool OFFDIAG>
__device__ __forceinline__ void sym_pair_fma(const float4* T4, const float2* xsl, int tq, int cp,
                                             const float2 (&xi)[8][R], float2 (&racc)[8][R],
                                             float2 (&cacc)[2][R]) {
    float2 xj[2][R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float4 v = lds128(xsl + k * SYM_T + 2 * cp);
        xj[0][k] = make_float2(v.x, v.y);
        xj[1][k] = make_float2(v.z, v.w);
        cacc[0][k] = cacc[1][k] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 e = lds128(T4 + i * 256 + tq);     // (8 rg + i, 2 cp) and (8 rg + i, 2 cp + 1)
        const float a0r = e.x, a0i = CONJ ? -e.y : e.y, a1r = e.z, a1i = CONJ ? -e.w : e.w;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 r = racc[i][k];
            r.x = fmaf(a0r, xj[0][k].x, r.x); r.x = fmaf(-a0i, xj[0][k].y, r.x);
            r.y = fmaf(a0r, xj[0][k].y, r.y); r.y = fmaf(a0i, xj[0][k].x, r.y);
            r.x = fmaf(a1r, xj[1][k].x, r.x); r.x = fmaf(-a1i, xj[1][k].y, r.x);
            r.y = fmaf(a1r, xj[1][k].y, r.y); r.y = fmaf(a1i, xj[1][k].x, r.y);
            racc[i][k] = r;
            if (OFFDIAG) {
                const float2 v = xi[i][k];
                float2 c0 = cacc[0][k], c1 = cacc[1][k];
                c0.x = fmaf(a0r, v.x, c0.x); c0.x = fmaf(-a0i, v.y, c0.x);
                c0.y = fmaf(a0r, v.y, c0.y); c0.y = fmaf(a0i, v.x, c0.y);
                c1.x = fmaf(a1r, v.x, c1.x); c1.x = fmaf(-a1i, v.y, c1.x);
                c1.y = fmaf(a1r, v.y, c1.y); c1.y = fmaf(a1i, v.x, c1.y);
                cacc[0][k] = c0;
                cacc[1][k] = c1;
            }
        }
    }
}

// One (class c, tile row I) segment of R right-hand sides for consumer thread tid
// (0..255): tiles sg.z .. sg.w-1 of the ring, u counts the CTA's tiles so far.
// CONJ applies conj(S) instead of S.
//
// The consumers form two groups of four warps (group = warp / 4, one warp of each
// group per scheduler); group g takes the CTA's tiles u with u % 2 == g, so the two
// warps that share a scheduler are at different points of different tiles and one
// hides the other's latency.  Thread (group warp wq, lane) of a group owns the
// column pairs cp = 4 wq + lane / 8 and cp + 16 and the eight rows 8 rg .. 8 rg + 7
// (rg = lane % 8) of its tiles.
//
// Both partial sums are reduced by halving exchanges (a reduce-scatter over lanes):
// at each level a lane keeps half of its values, sends the other half to its partner
// and adds what the partner sent for the kept half, so every level moves half as
// much as the one before and the reduced values end up spread over the lanes, in
// the order the stores want them.
template <int R, bool CONJ>
__device__ __forceinline__ bool sym_segment(const SymInfo& si, int4 sg, int s, int& u, const float2* ring,
                                            const float2* xs, uint64_t* full, uint64_t* empty,
                                            float2* __restrict__ rowpart, float* __restrict__ colpart, int tid) {
    const int I = sg.y;
    const int warp = tid >> 5, lane = tid & 31, rg = lane & 7, grp = warp >> 2, wq = warp & 3;
    const int cp = wq * 4 + (lane >> 3), tq = wq * 32 + lane;      // tq: the pair's thread in the packing
    const bool b0 = lane & 1, b1 = lane & 2, b2 = lane & 4, b3 = lane & 8, b4 = lane & 16;
    float2 xi[8][R], racc[8][R];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int k = 0; k < R; ++k) xi[i][k] = racc[i][k] = make_float2(0.f, 0.f);
    bool ok = true;
    const long long tb = si.tbase[sg.x] + (long long)I * (I + 1) / 2;
    const int skip = (grp + u) & 1;                  // this group's first tile of the segment
    bool first = true;
    for (int t = sg.z + skip, uu = u + skip; t < sg.w; t += 2, uu += 2) {
        const int J = (int)(t - tb);
        const bool offdiag = J < I;
        const int slot = uu % SYM_STAGES;
        ok &= mbar_wait_bounded(&full[slot], (uint32_t)((uu / SYM_STAGES) & 1));
        const float2* xsl = xs + (size_t)slot * SYM_XS_FLOAT2;      // [0][k][64] x_J, [1][k][64] x_I
        if (first) {
            first = false;
#pragma unroll
            for (int k = 0; k < R; ++k)
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const float4 v = lds128(xsl + (SYM_RMAX + k) * SYM_T + rg * 8 + i);
                    xi[i][k] = make_float2(v.x, v.y);
                    xi[i + 1][k] = make_float2(v.z, v.w);
                }
        }
        const float4* T4 = reinterpret_cast<const float4*>(ring + (size_t)slot * SYM_T * SYM_T);
        // the two column pairs in turn (a rolled loop keeps the hot code small); one
        // straight-line body per tile kind, so loads and FMAs schedule freely
#pragma unroll 1
        for (int p = 0; p < 2; ++p) {
            const int cpp = cp + 16 * p;
            float2 cacc[2][R];                       // [column of the pair][k]
            if (offdiag) sym_pair_fma<R, CONJ, true>(T4, xsl, tq + 128 * p, cpp, xi, racc, cacc);
            else sym_pair_fma<R, CONJ, false>(T4, xsl, tq + 128 * p, cpp, xi, racc, cacc);
            if (offdiag) {
                // column part: sum over the 8 row groups (lane bits 0-2).  Bit 2 picks the
                // column of the pair, bit 1 the real or imaginary part; bit 0 adds the last pair.
                float w[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float2 snd = b2 ? cacc[0][k] : cacc[1][k], kp = b2 ? cacc[1][k] : cacc[0][k];
                    float2 v;
                    v.x = kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 4);
                    v.y = kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 4);
                    w[k] = (b1 ? v.y : v.x) + __shfl_xor_sync(0xffffffffu, b1 ? v.x : v.y, 2);
                    w[k] += __shfl_xor_sync(0xffffffffu, w[k], 1);
                }
                // colpart[t][k][64 columns] complex: the warp's 8 columns are 64 contiguous bytes per k
                float* dst = colpart + (((size_t)t * SYM_RMAX) * SYM_T + 2 * cpp + (b2 ? 1 : 0)) * 2 + (b1 ? 1 : 0);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (R == 1 ? !b0 : ((k & 1) != 0) == b0) dst[k * SYM_T * 2] = w[k];
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);          // the slot's data is in registers
    }
    u += sg.w - sg.z;
    // row part of the segment, summed over the warp's lanes that share rows (lane bits 3, 4):
    // bit 4 keeps rows 0-3 or 4-7 of the lane's eight, bit 3 a pair of those, so lane
    // (rg, q = lane / 8) ends with rows 8 rg + 2 q and 8 rg + 2 q + 1.  Each warp stores
    // its own partial (the back transform adds the 8 warps' values in a fixed order),
    // so segment ends need no block-wide barrier.
    float2 r4[4][R];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float2 snd = b4 ? racc[j][k] : racc[j + 4][k], kp = b4 ? racc[j + 4][k] : racc[j][k];
            r4[j][k].x = kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 16);
            r4[j][k].y = kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 16);
        }
    // rowpart[s][warp][k][64 rows] complex: one contiguous 512-byte store per k
    float4* dst = reinterpret_cast<float4*>(rowpart + (((size_t)s * SYM_CONSUMERS + warp) * SYM_RMAX) * SYM_T) +
                  (rg * 8 + 2 * (lane >> 3)) / 2;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        float2 r2[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float2 snd = b3 ? r4[j][k] : r4[j + 2][k], kp = b3 ? r4[j + 2][k] : r4[j][k];
            r2[j].x = kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 8);
            r2[j].y = kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 8);
        }
        dst[k * SYM_T / 2] = make_float4(r2[0].x, r2[0].y, r2[1].x, r2[1].y);
    }
    return ok;
}

// Segment s = (class c, tile row I, first tile, end tile), numbered by (class, row,
// first tile).  CTA b works on cta_cnt[b] <= SYM_SEG_CACHE segments, stored in order at
// rec[b * SYM_SEG_CACHE + i] as (16 s + c, I, first tile, end tile), so the CTA reads its
// whole work list with one round of independent loads (tiles of different segments need
// not be contiguous).  rowpart[s][8 warps][3][64] and colpart[t][3][64] (complex,
// right-hand side k of R at index k; slots k >= R are not written).
static __global__ void __launch_bounds__(SYM_THREADS, 1)
sym_gemv_tiles(SymInfo si, const float2* __restrict__ tiles, const int4* __restrict__ rec,
               const int* __restrict__ cta_cnt, const float2* __restrict__ x, float2* __restrict__ rowpart,
               float2* __restrict__ colpart, int conj, long long keep, int* __restrict__ err) {
    float* colf = reinterpret_cast<float*>(colpart);
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ring = reinterpret_cast<float2*>(smem);
    float2* xs = reinterpret_cast<float2*>(smem + SYM_STAGES * (size_t)SYM_TILE_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + SYM_STAGES * (size_t)SYM_TILE_BYTES + SYM_XS_BYTES);
    uint64_t* empty = full + SYM_STAGES;
    int4* segc = reinterpret_cast<int4*>(empty + SYM_STAGES);       // this CTA's segments
    int* sidc = reinterpret_cast<int*>(segc + SYM_SEG_CACHE);       // and their ids
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nseg = cta_cnt[blockIdx.x];
    const int4 r = tid < SYM_SEG_CACHE ? rec[(size_t)blockIdx.x * SYM_SEG_CACHE + tid] : make_int4(0, 0, 0, 0);
    if (nseg <= 0 || nseg > SYM_SEG_CACHE) return;               // the host guarantees <= SYM_SEG_CACHE
    if (tid < nseg) {
        sidc[tid] = r.x >> 4;
        segc[tid] = make_int4(r.x & 15, r.y, r.z, r.w);
    }
    if (tid == 0) {
        for (int i = 0; i < SYM_STAGES; ++i) {
            mbar_init(&full[i], 32);                 // the producer warp's lanes (one with the tile bytes)
            mbar_init(&empty[i], SYM_CONSUMERS / 2);     // the group that consumes the slot
        }
        fence_mbar_init();
    }
    __syncthreads();
    int ntl = 0;                                     // tiles of this CTA
    for (int i = 0; i < nseg; ++i) ntl += segc[i].w - segc[i].z;

    if (warp == SYM_CONSUMERS) {
        // ---------------- producer warp ----------------
        // per tile: lane 0 announces the tile's bytes and starts its bulk copy; every lane
        // copies its share of x_J (the tile's columns) and x_I (its rows) of each
        // right-hand side into the slot with cp.async (zeros past the class size) and
        // arrives on the slot's "full" barrier once its copies have landed (32 arrivals)
        bool ok = true;
        // the tiles do not depend on the preceding kernel: start the first copies before
        // waiting for it (the vector slices below do depend on it)
        const int early = ntl < SYM_STAGES ? ntl : SYM_STAGES;
        if (lane == 0) {
            int i = 0;
            long long t = segc[0].z;
            for (int u = 0; u < early; ++u) {
                while (t >= segc[i].w) t = segc[++i].z;
                mbar_add_tx(&full[u], SYM_TILE_BYTES);
                tile_copy(ring + (size_t)u * SYM_T * SYM_T, tiles, t, &full[u], keep);
                ++t;
            }
        }
        pdl_wait();
        int i = 0;
        int4 sg = segc[0];
        long long t = sg.z;
        for (int u = 0; u < ntl; ++u, ++t) {
            const int slot = u % SYM_STAGES;
            while (t >= sg.w) {
                sg = segc[++i];
                t = sg.z;
            }
            if (u >= SYM_STAGES) ok &= mbar_wait_bounded(&empty[slot], (uint32_t)((u / SYM_STAGES - 1) & 1));
            const int c = sg.x, I = sg.y, R = si.R[c], m = si.m[c];
            const int J = (int)(t - si.tbase[c] - (long long)I * (I + 1) / 2);
            if (lane == 0 && u >= early) {
                mbar_add_tx(&full[slot], SYM_TILE_BYTES);
                tile_copy(ring + (size_t)slot * SYM_T * SYM_T, tiles, t, &full[slot], keep);
            }
            float2* xsl = xs + (size_t)slot * SYM_XS_FLOAT2;
#pragma unroll
            for (int half = 0; half < 2; ++half)
#pragma unroll
                for (int k = 0; k < SYM_RMAX; ++k) {
                    if (k >= R) break;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = lane + 32 * h, idx = (half ? I : J) * SYM_T + q;
                        cp_async8(xsl + (half * SYM_RMAX + k) * SYM_T + q, x + si.moff[c][k] + (idx < m ? idx : 0),
                                  idx < m ? 8u : 0u);
                    }
                }
            cp_async_arrive(&full[slot]);
        }
        // the last copies land before the CTA can release its shared memory
        if (lane == 0)
            for (int u = ntl > SYM_STAGES ? ntl - SYM_STAGES : 0; u < ntl; ++u)
                ok &= mbar_wait_bounded(&full[u % SYM_STAGES], (uint32_t)((u / SYM_STAGES) & 1));
        if (!ok) atomicExch(err, 1);
        return;
    }

    // ---------------- consumer warps ----------------
    bool ok = true;
    int u = 0;
    for (int i = 0; i < nseg; ++i) {
        const int4 sg = segc[i];
        const int s = sidc[i];
        const int R = si.R[sg.x];
        if (conj) {
            if (R == 1) ok &= sym_segment<1, true>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
            else if (R == 2) ok &= sym_segment<2, true>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
            else ok &= sym_segment<3, true>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
        } else {
            if (R == 1) ok &= sym_segment<1, false>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
            else if (R == 2) ok &= sym_segment<2, false>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
            else ok &= sym_segment<3, false>(si, sg, s, u, ring, xs, full, empty, rowpart, colf, tid);
        }
    }
    if (!ok && lane == 0) atomicExch(err, 1);
}

}  // namespace dev
}  // namespace abc
