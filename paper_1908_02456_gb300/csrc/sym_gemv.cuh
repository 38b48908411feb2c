// Boundary DtN contraction for one orbital on symmetric packed tiles (sm_103a).
//
// Each distinct parity block S (complex symmetric, m x m; one per axis-permutation
// class, shared by the R in {1, 3} parities of the class) is stored as its lower
// triangle of 64 x 64 tiles, each tile contiguous (32 KB in complex64).  A tile
// (I, J <= I) serves twice:
//     t_I += S_IJ x_J          (row part)
//     t_J += S_IJ^T x_I        (column part, J < I)
// for every right-hand side x of the class.  Tiles are stored column-major.  One
// producer warp streams them from HBM with 1D bulk copies (cp.async.bulk) into a
// 4-slot shared-memory ring ("full" mbarriers); 16 consumer warps run decoupled,
// each owning 4 columns of every tile (lanes own rows l and l+32), release a slot
// through its "empty" mbarrier, reduce the column part inside the warp, and keep
// the row part in registers until their (class, tile-row) segment ends.  Every wait
// is bounded: a wait that gives up raises an error flag, and all warps still follow
// the same control flow to the end, so no barrier can hang.  Partial sums go to
// global scratch and a second kernel adds them in a fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace abc {
namespace dev {

constexpr int SYM_T = 64;                        // tile edge
constexpr int SYM_CONSUMERS = 16;                // consumer warps, 4 columns each
constexpr int SYM_THREADS = (SYM_CONSUMERS + 1) * 32;
constexpr int SYM_STAGES = 4;
constexpr int SYM_RMAX = 3;
constexpr uint32_t SYM_TILE_BYTES = SYM_T * SYM_T * 8;
constexpr int SYM_CR_STRIDE = 8 * SYM_RMAX + 1;  // floats per lane row of the column-reduction area
constexpr size_t SYM_FLUSH_BYTES = (size_t)SYM_CONSUMERS * SYM_T * SYM_RMAX * 8;
constexpr size_t SYM_CR_BYTES = (size_t)SYM_CONSUMERS * 32 * SYM_CR_STRIDE * 4;
constexpr size_t SYM_SMEM = SYM_STAGES * (size_t)SYM_TILE_BYTES + SYM_FLUSH_BYTES + SYM_CR_BYTES +
                            2 * SYM_STAGES * 8;
constexpr long long SYM_WAIT_LIMIT = 1ll << 24;  // try_wait polls before giving up

struct SymInfo {
    int nclass;
    int R[8];              // right-hand sides (parities) of the class
    int m[8];              // block size
    int nt[8];             // tile rows
    int moff[8][3];        // adapted offset of each member parity
    long long tbase[8];    // first global tile of the class
    int rbase[8];          // first (class, tile-row) index of the class
    long long obase[9];    // first output thread of the class (reduction kernel)
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
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(SYM_CONSUMERS * 32) : "memory"); }
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
// Tiles with a global index below `keep` are copied with evict_last (they stay in L2
// from one stage to the next), the rest with evict_first.
__device__ __forceinline__ void tile_copy(void* dst, const float2* tiles, long long t, uint64_t* bar, long long keep) {
    const float2* src = tiles + (size_t)t * 64 * 64;
    bulk_g2s_hint(dst, src, 64 * 64 * 8, bar, t < keep ? policy_evict_last() : policy_evict_first());
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

// seg[s] = (class, tile row I, first tile, end tile); cta_seg[b]..cta_seg[b+1] are
// the segments of CTA b (contiguous tiles).  rowpart[s][64][3], colpart[t][64][3].
static __global__ void __launch_bounds__(SYM_THREADS, 1)
sym_gemv_tiles(SymInfo si, const float2* __restrict__ tiles, const int4* __restrict__ seg,
               const int* __restrict__ cta_seg, const float2* __restrict__ x, float2* __restrict__ rowpart,
               float2* __restrict__ colpart, int conj, long long keep, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ring = reinterpret_cast<float2*>(smem);
    float2* flush = reinterpret_cast<float2*>(smem + SYM_STAGES * (size_t)SYM_TILE_BYTES);
    float* cred = reinterpret_cast<float*>(smem + SYM_STAGES * (size_t)SYM_TILE_BYTES + SYM_FLUSH_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + SYM_STAGES * (size_t)SYM_TILE_BYTES + SYM_FLUSH_BYTES +
                                                 SYM_CR_BYTES);
    uint64_t* empty = full + SYM_STAGES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s_begin = cta_seg[blockIdx.x], s_end = cta_seg[blockIdx.x + 1];
    if (s_begin >= s_end) return;
    const long long t_first = seg[s_begin].z;
    const int ntl = (int)(seg[s_end - 1].w - t_first);
    if (tid == 0) {
        for (int i = 0; i < SYM_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], SYM_CONSUMERS);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == SYM_CONSUMERS) {
        // ---------------- producer warp ----------------
        if (lane == 0) {
            bool ok = true;
            for (int u = 0; u < ntl; ++u) {
                const int slot = u % SYM_STAGES;
                if (u >= SYM_STAGES) ok &= mbar_wait_bounded(&empty[slot], (uint32_t)((u / SYM_STAGES - 1) & 1));
                fence_proxy_async();
                mbar_expect_tx(&full[slot], SYM_TILE_BYTES);
                tile_copy(ring + (size_t)slot * SYM_T * SYM_T, tiles, t_first + u, &full[slot], keep);
            }
            // the last copies land before the CTA can release its shared memory
            for (int u = ntl > SYM_STAGES ? ntl - SYM_STAGES : 0; u < ntl; ++u)
                ok &= mbar_wait_bounded(&full[u % SYM_STAGES], (uint32_t)((u / SYM_STAGES) & 1));
            if (!ok) atomicExch(err, 1);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const float cs = conj ? -1.f : 1.f;
    float* cr = cred + (size_t)warp * 32 * SYM_CR_STRIDE;
    bool ok = true;
    int u = 0;
    for (int s = s_begin; s < s_end; ++s) {
        const int4 sg = seg[s];
        const int c = sg.x, I = sg.y;
        const int R = si.R[c], m = si.m[c];
        float2 xi[2][SYM_RMAX], xis[2][SYM_RMAX], racc[2][SYM_RMAX];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = I * SYM_T + lane + 32 * h;
#pragma unroll
            for (int k = 0; k < SYM_RMAX; ++k) {
                racc[h][k] = make_float2(0.f, 0.f);
                xi[h][k] = (k < R && row < m) ? x[si.moff[c][k] + row] : make_float2(0.f, 0.f);
                xis[h][k] = make_float2(xi[h][k].y, xi[h][k].x);
            }
        }
        for (int t = sg.z; t < sg.w; ++t, ++u) {
            const int J = (int)(t - si.tbase[c]) - I * (I + 1) / 2;
            const int slot = u % SYM_STAGES;
            const bool offdiag = J < I;
            // x_J for this warp's 4 columns (same for all lanes), fetched before the wait
            float2 xj[4][SYM_RMAX];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int col = J * SYM_T + warp * 4 + cc;
#pragma unroll
                for (int k = 0; k < SYM_RMAX; ++k)
                    xj[cc][k] = (k < R && col < m) ? __ldg(x + si.moff[c][k] + col) : make_float2(0.f, 0.f);
            }
            ok &= mbar_wait_bounded(&full[slot], (uint32_t)((u / SYM_STAGES) & 1));
            const float2* T = ring + (size_t)slot * SYM_T * SYM_T;
            float2 sv[4][2];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                sv[cc][0] = T[(warp * 4 + cc) * SYM_T + lane];
                sv[cc][1] = T[(warp * 4 + cc) * SYM_T + lane + 32];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);     // the slot's data is in registers
            float2 cacc[4][SYM_RMAX];
            // complex a*b = (a.x,a.x)*(b.x,b.y) + (-a.y,a.y)*(b.y,b.x): two packed FMAs
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
                for (int k = 0; k < SYM_RMAX; ++k) cacc[cc][k] = make_float2(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 sa = make_float2(sv[cc][h].x, sv[cc][h].x);
                    const float2 sb = make_float2(-cs * sv[cc][h].y, cs * sv[cc][h].y);
#pragma unroll
                    for (int k = 0; k < SYM_RMAX; ++k) {
                        if (k >= R) break;
                        const float2 b = xj[cc][k], bs = make_float2(b.y, b.x);
                        racc[h][k] = __ffma2_rn(sa, b, racc[h][k]);
                        racc[h][k] = __ffma2_rn(sb, bs, racc[h][k]);
                        if (offdiag) {
                            cacc[cc][k] = __ffma2_rn(sa, xi[h][k], cacc[cc][k]);
                            cacc[cc][k] = __ffma2_rn(sb, xis[h][k], cacc[cc][k]);
                        }
                    }
                }
            }
            if (offdiag) {
                // column part: sum over the 32 lanes (rows) through this warp's own area
                const int nv = 8 * R;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                    for (int k = 0; k < SYM_RMAX; ++k) {
                        if (k >= R) break;
                        cr[lane * SYM_CR_STRIDE + (cc * R + k) * 2] = cacc[cc][k].x;
                        cr[lane * SYM_CR_STRIDE + (cc * R + k) * 2 + 1] = cacc[cc][k].y;
                    }
                __syncwarp();
                if (lane < nv) {
                    float acc = 0.f;
#pragma unroll 8
                    for (int l = 0; l < 32; ++l) acc += cr[l * SYM_CR_STRIDE + lane];
                    const int v = lane >> 1, comp = lane & 1;
                    const int cc = v / R, k = v % R;
                    reinterpret_cast<float*>(colpart)[2 * (((size_t)t * SYM_T + warp * 4 + cc) * SYM_RMAX + k) + comp] =
                        acc;
                }
                __syncwarp();
            }
        }
        // row part of this segment: sum over the 16 consumer warps
        float2* fb = flush;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < SYM_RMAX; ++k)
                if (k < R) fb[((size_t)warp * SYM_T + lane + 32 * h) * SYM_RMAX + k] = racc[h][k];
        consumer_sync();
        if (tid < SYM_T * R) {
            const int row = tid % SYM_T, k = tid / SYM_T;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int w = 0; w < SYM_CONSUMERS; ++w) {
                const float2 v = fb[((size_t)w * SYM_T + row) * SYM_RMAX + k];
                acc.x += v.x;
                acc.y += v.y;
            }
            rowpart[((size_t)s * SYM_T + row) * SYM_RMAX + k] = acc;
        }
        consumer_sync();
    }
    if (!ok && lane == 0) atomicExch(err, 1);
}

// t[moff[c][k] + I*64 + r] = sum of the row-part partials of (c, I) + column parts of
// the tiles (c, K, I), K > I.  Eight lanes per output (c, I, r, k) take every eighth
// term and combine by a fixed butterfly, so the order of the additions is fixed.
static __global__ void sym_reduce(SymInfo si, const int2* __restrict__ rowseg, const float2* __restrict__ rowpart,
                                  const float2* __restrict__ colpart, float2* __restrict__ t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long idx = gid >> 3;
    const int sub = (int)(gid & 7);
    const bool live = idx < si.obase[si.nclass];
    float2 acc = make_float2(0.f, 0.f);
    int c = 0, k = 0, r = 0, I = 0, row = 0;
    if (live) {
        while (c + 1 < si.nclass && idx >= si.obase[c + 1]) ++c;
        const long long loc = idx - si.obase[c];
        const int R = si.R[c];
        k = (int)(loc % R);
        r = (int)((loc / R) % SYM_T);
        I = (int)(loc / ((long long)R * SYM_T));
        row = I * SYM_T + r;
        const int2 rs = rowseg[si.rbase[c] + I];
        for (int s = rs.x + sub; s < rs.y; s += 8) {
            const float2 v = rowpart[((size_t)s * SYM_T + r) * SYM_RMAX + k];
            acc.x += v.x;
            acc.y += v.y;
        }
        for (int K = I + 1 + sub; K < si.nt[c]; K += 8) {
            const long long tt = si.tbase[c] + (long long)K * (K + 1) / 2 + I;
            const float2 v = colpart[((size_t)tt * SYM_T + r) * SYM_RMAX + k];
            acc.x += v.x;
            acc.y += v.y;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (live && sub == 0 && row < si.m[c]) t[si.moff[c][k] + row] = acc;
}

}  // namespace dev
}  // namespace abc
