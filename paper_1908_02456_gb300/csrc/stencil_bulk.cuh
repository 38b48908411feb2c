// Interior stencil stage with the state's planes staged in shared memory by bulk copies
// (complex64, radius 1, nx even; sm_103a).
//
// The same update as stencil_stage_x2 -- out = y + cdt (-i) [H w + E^T b] for two
// x-adjacent nodes per thread, the same neighbour order, so the results are bit for bit
// those of stencil_stage_x2 -- but the values arrive differently: a CTA owns one
// orbital, SB_TY rows of the y axis and a run of z planes.  It marches through the run
// keeping six plane slots in shared memory; each slot holds SB_TY + 2 rows of w (the
// tile and its y halo) and the tile's SB_TY rows of y, brought in by two 1D bulk copies
// (cp.async.bulk; the rows of a plane are contiguous), completing on the slot's
// mbarrier.  While plane z is computed from slots z - 1, z, z + 1, the copies of planes
// z + 2 .. z + 4 are in flight; after it, the slot of plane z - 1 takes plane z + 5.
// V is read from global memory one plane ahead.  Rows and planes outside the box are never
// copied and read as zero (the stencil omits neighbours outside the box).  Every wait
// is bounded; a wait that gives up raises the error flag and the CTA still follows the
// same control flow to the end.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "sym_gemv.cuh"

namespace abc {
namespace dev {

constexpr int SB_TY = 8;      // rows of a tile
constexpr int SB_NP = 6;      // plane slots: z - 1, z, z + 1 and three in flight
constexpr int SB_KZ = 24;     // planes per CTA (the last run of a column may be shorter)

// Shared memory of one CTA for rows of nx complex values.
__host__ __device__ inline size_t stencil_bulk_smem(int nx) {
    return (size_t)SB_NP * (2 * SB_TY + 2) * nx * sizeof(float2) + SB_NP * sizeof(uint64_t);
}

// Grid (ceil(ny / SB_TY), ceil(nz / SB_KZ), n_orb); block (nx / 2) * SB_TY threads (nx
// even, at most 256); dynamic shared memory stencil_bulk_smem(nx); w, y and out 16-byte
// aligned.  gout as in stencil_pair_x2.
static __global__ void __launch_bounds__(1024) stencil_stage_x2_bulk(int nx, int ny, int nz, int n_orb,
                                                                   float inv_h2, const float2* __restrict__ w,
                                                                   const float2* y, const float* __restrict__ V,
                                                                   const float2* __restrict__ bterm, float2* out,
                                                                   float cdt, float2* __restrict__ gout,
                                                                   int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char sb_smem[];
    constexpr int SR = 2 * SB_TY + 2;                            // rows per slot: w rows -1 .. SB_TY, y rows
    float2* pl = reinterpret_cast<float2*>(sb_smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(pl + (size_t)SB_NP * SR * nx);
    const int npair = nx >> 1, tid = threadIdx.x;
    const int ry = tid / npair, tp = tid - ry * npair;           // tile row, pair in the row
    const int y0 = blockIdx.x * SB_TY, z0 = blockIdx.y * SB_KZ, orb = blockIdx.z;
    const int rows = min(SB_TY, ny - y0), z1 = min(nz, z0 + SB_KZ);
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const float2* wo = w + (long long)orb * nvox;
    const float2* yo = y + (long long)orb * nvox;
    const long long obase = (long long)orb * nvox;
    // w rows copied: local rows rlo .. rhi (local row r is y0 + r, slot row r + 1)
    const int rlo = y0 > 0 ? -1 : 0, rhi = y0 + rows < ny ? rows : rows - 1;
    const uint32_t bytes = (uint32_t)((rhi - rlo + 1) + rows) * (uint32_t)nx * 8u;
    const int p_first = max(z0 - 1, 0), p_last = min(z1, nz - 1);   // planes this CTA reads
    for (int i = tid; i < SB_NP * SR * nx; i += blockDim.x) pl[i] = make_float2(0.f, 0.f);
    if (tid == 0) {
        for (int s = 0; s < SB_NP; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    fence_proxy_async();                 // the zeros before any bulk copy into the slots
    __syncthreads();
    auto issue = [&](int p) {            // plane p into slot p % SB_NP (thread 0): the tile's rows of
        const int s = p % SB_NP;         // w with their halo, then of y, each one contiguous run
        float2* base = pl + (size_t)s * SR * nx;
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(base + (size_t)(rlo + 1) * nx, wo + (long long)p * nxy + (long long)(y0 + rlo) * nx,
                 (uint32_t)(rhi - rlo + 1) * (uint32_t)nx * 8u, &full[s]);
        bulk_g2s(base + (size_t)(SB_TY + 2) * nx, yo + (long long)p * nxy + (long long)y0 * nx,
                 (uint32_t)rows * (uint32_t)nx * 8u, &full[s]);
    };
    int next = p_first;                  // next plane to copy
    if (tid == 0)
        for (; next <= p_last && next < p_first + SB_NP; ++next) issue(next);
    next = min(p_last + 1, p_first + SB_NP);
    int ready = p_first - 1;             // planes up to this one have landed
    bool ok = true;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int i = 2 * tp, jy = y0 + ry;
    const bool act = ry < rows;
    const float* Vc = V + (long long)jy * nx + i;
    float2 vnext = act ? *reinterpret_cast<const float2*>(Vc + (long long)z0 * nxy) : make_float2(0.f, 0.f);
    for (int z = z0; z < z1; ++z) {
        const float2 vv = vnext;          // this plane's V, loaded one plane ahead
        if (act && z + 1 < z1) vnext = *reinterpret_cast<const float2*>(Vc + (long long)(z + 1) * nxy);
        for (const int need = min(z + 1, p_last); ready < need;) {
            ++ready;
            ok &= mbar_wait_bounded(&full[ready % SB_NP], (uint32_t)(((ready - p_first) / SB_NP) & 1));
        }
        if (act) {
            const float2* sc = pl + (size_t)(z % SB_NP) * SR * nx;
            const float2* sm = pl + (size_t)((z + SB_NP - 1) % SB_NP) * SR * nx;
            const float2* sp = pl + (size_t)((z + 1) % SB_NP) * SR * nx;
            const int ro = (ry + 1) * nx + i;
            const float4 c = *reinterpret_cast<const float4*>(sc + ro);
            const float2 xm = i >= 1 ? sc[ro - 1] : make_float2(0.f, 0.f);
            const float2 xp = i + 2 < nx ? sc[ro + 2] : make_float2(0.f, 0.f);
            const float4 ym = *reinterpret_cast<const float4*>(sc + ro - nx);     // zero outside the box
            const float4 yp = *reinterpret_cast<const float4*>(sc + ro + nx);
            const float4 zm = z >= 1 ? *reinterpret_cast<const float4*>(sm + ro) : zero;
            const float4 zp = z + 1 < nz ? *reinterpret_cast<const float4*>(sp + ro) : zero;
            const float4 yv = *reinterpret_cast<const float4*>(sc + (SB_TY + 2 + ry) * nx + i);
            const long long n = (long long)z * nxy + (long long)jy * nx + i;
            float hr[2], hi[2];
            {
                // node i: x- = xm, x+ = node i + 1 (the neighbour order of stencil_pair_x2)
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
                if (on_gamma<1>(i + q, jy, z, nx, ny, nz)) {
                    gq[q] = (long long)gamma_index<1>(i + q, jy, z, nx, ny, nz) * n_orb + orb;
                    const float2 b = bterm[gq[q]];
                    hr[q] += b.x;
                    hi[q] += b.y;
                }
            const float4 o = make_float4(yv.x + cdt * hi[0], yv.y - cdt * hr[0], yv.z + cdt * hi[1],
                                         yv.w - cdt * hr[1]);
            *reinterpret_cast<float4*>(out + obase + n) = o;
            if (gout) {
                if (gq[0] >= 0) gout[gq[0]] = make_float2(o.x, o.y);
                if (gq[1] >= 0) gout[gq[1]] = make_float2(o.z, o.w);
            }
        }
        __syncthreads();                 // every read of plane z - 1's slot is done
        if (tid == 0) {                  // (only thread 0 keeps `next` up to date)
            fence_proxy_async();
            for (; next <= p_last && next - SB_NP <= z - 1; ++next) issue(next);
        }
    }
    if (!ok) {
        // a wait gave up: wait (bounded) for the copies still in flight before the CTA
        // releases its shared memory, and report
        if (tid == 0)
            for (int p = ready + 1; p < next; ++p)
                mbar_wait_bounded(&full[p % SB_NP], (uint32_t)(((p - p_first) / SB_NP) & 1));
        if ((tid & 31) == 0) atomicExch(err, 1);
    }
}

}  // namespace dev
}  // namespace abc
