// Interior stencil of the four Horner stages of one order-1 time step, fused in time
// (complex64, radius 1, nx even).
//
// The stage update of eq:dynamics1 in Horner form is u^{s+1} = y + c_s dt (-i)
// [H u^s + E^T f^s] (s = 0..3, u^0 = y, c = 1/4, 1/3, 1/2, 1): the boundary variable
// f^s enters the phi-part only on Gamma, and the stencil moves information by one node
// per stage.  f^0 is known when the step starts; f^1, f^2, f^3 come out of the
// boundary contractions of stages 0, 1, 2.  Hence u^{s+1} at a node whose distance d to
// the nearest face (d = 0 on Gamma) satisfies d >= s depends on y and f^0 alone:
// u^1 everywhere, u^2 for d >= 1, u^3 for d >= 2 and the step's result u^4 for d >= 3.
//
// stencil_bulk4 computes all of those in one pass over the state: each CTA owns an xy
// tile of one orbital and marches through z, keeping rings of planes of y (with a halo
// of four nodes) and of the intermediate stages u^1, u^2, u^3 (halos of three, two,
// one) in shared memory; the next y plane streams in with cp.async while the current
// one is processed.  HBM traffic is y once and u^4 once instead of three arrays per
// stage.  It also stores the band values the stage-by-stage remainder needs: u^1 for
// d <= 1, u^2 for d in {1, 2}, u^3 for d in {2, 3}.
//
// stencil_band then finishes the band once the boundary contraction of the stage
// before has produced f^s: u^2 on d = 0, u^3 on d <= 1 and u^4 on d <= 2.
//
// Both evaluate the same expression, in the same order, as the stage-by-stage kernels
// (neighbours x-, x+, y-, y+, z-, z+; diagonal 3/h^2 + V; boundary term on Gamma), so
// the two forms agree to FP32 rounding of fused multiply-adds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace abc {
namespace dev {

constexpr int FB_TX = 32, FB_TY = 16;              // output tile per CTA (x, y)
constexpr int FB_THREADS = 256;
constexpr int FB_YW = FB_TX + 8, FB_YH = FB_TY + 8;   // y planes: halo 4
constexpr int FB_YSLOTS = 6;                          // y planes t-5 .. t (+ the one in flight)
__host__ __device__ constexpr int fb_w(int lvl) { return FB_TX + 2 * (4 - lvl); }   // level region (halo 4 - lvl)
__host__ __device__ constexpr int fb_h(int lvl) { return FB_TY + 2 * (4 - lvl); }
constexpr size_t FB_SMEM = sizeof(float2) * ((size_t)FB_YSLOTS * FB_YW * FB_YH + 3ull * fb_w(1) * fb_h(1) +
                                              3ull * fb_w(2) * fb_h(2) + 3ull * fb_w(3) * fb_h(3));

__device__ __forceinline__ int fb_dist(int i, int j, int k, int nx, int ny, int nz) {
    return min(min(min(i, nx - 1 - i), min(j, ny - 1 - j)), min(k, nz - 1 - k));
}

// One node of a stage: y + cdt (-i) (dg c - 1/(2h^2) sum(neighbours) + b).
__device__ __forceinline__ float2 fb_node(float2 c, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm, float2 zp,
                                          float v, float inv_h2, float2 yb, float2 b, float cdt) {
    float sr = 0.f, si = 0.f;
    sr += xm.x; si += xm.y;
    sr += xp.x; si += xp.y;
    sr += ym.x; si += ym.y;
    sr += yp.x; si += yp.y;
    sr += zm.x; si += zm.y;
    sr += zp.x; si += zp.y;
    const float dg = 3.f * inv_h2 + v;
    float hr = dg * c.x - 0.5f * inv_h2 * sr;
    float hi = dg * c.y - 0.5f * inv_h2 * si;
    hr += b.x;
    hi += b.y;
    return make_float2(yb.x + cdt * hi, yb.y - cdt * hr);
}

__device__ __forceinline__ void fb_cp16(void* sdst, const void* gsrc, bool inside) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(sdst);
    const int bytes = inside ? 16 : 0;                       // 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fb_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void fb_cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct FusedBulkArgs {
    int nx, ny, nz, n_orb, n_gamma;
    float inv_h2;
    float cdt[4];
    const float2* y;          // step input [n_orb][nz][ny][nx]
    const float* V;           // potential [nz][ny][nx]
    const float2* f0;         // f at the step start [n_gamma][n_orb]
    float2* out;              // u^4 for d >= 3
    float2* u1;               // u^1 for d <= 1
    float2* u2;               // u^2 for d in {1, 2}
    float2* u3;               // u^3 for d in {2, 3}
};

// Persistent over (orbital, xy tile) items.  Every global address a thread forms is
// inside the arrays: loads of nodes outside the box are zero fills that read nothing
// (their source address is clamped to the plane's first node), stores are guarded.
static __global__ void __launch_bounds__(FB_THREADS) stencil_bulk4(FusedBulkArgs a) {
    extern __shared__ __align__(16) float2 fb_smem[];
    float2* Y = fb_smem;                                              // [6][YH][YW]
    float2* L1 = Y + FB_YSLOTS * FB_YW * FB_YH;                       // [3][h1][w1]
    float2* L2 = L1 + 3 * fb_w(1) * fb_h(1);
    float2* L3 = L2 + 3 * fb_w(2) * fb_h(2);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const int ntx = (nx + FB_TX - 1) / FB_TX, nty = (ny + FB_TY - 1) / FB_TY;
    const long long items = (long long)a.n_orb * ntx * nty;
    const int tid = threadIdx.x;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int orb = (int)(item / ((long long)ntx * nty));
        const int rem = (int)(item - (long long)orb * ntx * nty);
        const int x0 = (rem % ntx) * FB_TX, y0 = (rem / ntx) * FB_TY;
        const float2* yo = a.y + (long long)orb * nvox;
        // all rings start as zero planes (planes below the box)
        for (int e = tid; e < FB_YSLOTS * FB_YW * FB_YH + 3 * (fb_w(1) * fb_h(1) + fb_w(2) * fb_h(2) + fb_w(3) * fb_h(3));
             e += FB_THREADS)
            fb_smem[e] = make_float2(0.f, 0.f);
        __syncthreads();
        // y plane p (halo 4) into its ring slot; 16-byte chunks = two x-adjacent nodes,
        // never straddling the x edge (x0 - 4 and nx are even)
        auto load_y = [&](int p) {
            float2* dst = Y + (size_t)(((p % FB_YSLOTS) + FB_YSLOTS) % FB_YSLOTS) * FB_YW * FB_YH;
            for (int e = tid; e < FB_YH * (FB_YW / 2); e += FB_THREADS) {
                const int r = e / (FB_YW / 2), q = e - r * (FB_YW / 2);
                const int gx = x0 - 4 + 2 * q, gy = y0 - 4 + r;
                const bool in = p >= 0 && p < nz && gy >= 0 && gy < ny && gx >= 0 && gx < nx;
                const float2* src = in ? yo + (long long)p * nxy + (long long)gy * nx + gx : yo;
                fb_cp16(dst + r * FB_YW + 2 * q, src, in);
            }
            fb_cp_commit();
        };
        load_y(0);
        for (int t = 0; t <= nz + 3; ++t) {
            fb_cp_wait_all();
            __syncthreads();                         // y plane t landed; last iteration's reads done
            if (t + 1 < nz) load_y(t + 1);           // overlaps this iteration (slot of plane t - 5)
            else if (t + 1 <= nz + 3) {              // zero plane above the box
                float2* dst = Y + (size_t)((t + 1) % FB_YSLOTS) * FB_YW * FB_YH;
                for (int e = tid; e < FB_YW * FB_YH; e += FB_THREADS) dst[e] = make_float2(0.f, 0.f);
            }
            // level s computes u^s at plane p = t - s over its region (halo 4 - s)
#pragma unroll
            for (int lvl = 1; lvl <= 4; ++lvl) {
                const float cdt = lvl == 1 ? a.cdt[0] : lvl == 2 ? a.cdt[1] : lvl == 3 ? a.cdt[2] : a.cdt[3];
                const int p = t - lvl;
                const int W = fb_w(lvl), H = fb_h(lvl), hal = 4 - lvl;
                const float2* src;                   // level lvl - 1 ring (y for level 1)
                int sW, sslots, sh;                  // its width, ring slots, halo offset into it
                if (lvl == 1) { src = Y; sW = FB_YW; sslots = FB_YSLOTS; sh = 1; }
                else if (lvl == 2) { src = L1; sW = fb_w(1); sslots = 3; sh = 1; }
                else if (lvl == 3) { src = L2; sW = fb_w(2); sslots = 3; sh = 1; }
                else { src = L3; sW = fb_w(3); sslots = 3; sh = 1; }
                const int sH = lvl == 1 ? FB_YH : fb_h(lvl - 1);
                const float2* sm = src + (size_t)((((p - 1) % sslots) + sslots) % sslots) * sW * sH;
                const float2* sc = src + (size_t)(((p % sslots) + sslots) % sslots) * sW * sH;
                const float2* sp = src + (size_t)((((p + 1) % sslots) + sslots) % sslots) * sW * sH;
                const float2* yb = Y + (size_t)(((p % FB_YSLOTS) + FB_YSLOTS) % FB_YSLOTS) * FB_YW * FB_YH;
                float2* dstL = lvl == 1 ? L1 : lvl == 2 ? L2 : L3;
                float2* dring = dstL + (size_t)(((p % 3) + 3) % 3) * W * H;
                const bool plane_in = p >= 0 && p < nz;
                for (int e = tid; e < W * H; e += FB_THREADS) {
                    const int r = e / W, q = e - r * W;
                    const int gx = x0 - hal + q, gy = y0 - hal + r;
                    const bool in = plane_in && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
                    float2 u = make_float2(0.f, 0.f);
                    if (in) {
                        const int si = (r + sh) * sW + (q + sh);          // the node in the source ring
                        const int yi = (r + lvl) * FB_YW + (q + lvl);     // the node in the y ring
                        float2 b = make_float2(0.f, 0.f);
                        if (lvl == 1 && (gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1 || p == 0 || p == nz - 1))
                            b = a.f0[(long long)gamma_index<1>(gx, gy, p, nx, ny, nz) * a.n_orb + orb];
                        const float v = __ldg(a.V + (long long)p * nxy + (long long)gy * nx + gx);
                        u = fb_node(sc[si], sc[si - 1], sc[si + 1], sc[si - sW], sc[si + sW], sm[si], sp[si], v,
                                    a.inv_h2, yb[yi], b, cdt);
                        const bool own = q >= hal && q < hal + FB_TX && r >= hal && r < hal + FB_TY;
                        if (own) {
                            const int d = fb_dist(gx, gy, p, nx, ny, nz);
                            const long long gi = (long long)orb * nvox + (long long)p * nxy + (long long)gy * nx + gx;
                            if (lvl == 1 && d <= 1) a.u1[gi] = u;
                            else if (lvl == 2 && (d == 1 || d == 2)) a.u2[gi] = u;
                            else if (lvl == 3 && (d == 2 || d == 3)) a.u3[gi] = u;
                            else if (lvl == 4 && d >= 3) a.out[gi] = u;
                        }
                    }
                    if (lvl < 4) dring[e] = u;
                }
                __syncthreads();
            }
        }
        __syncthreads();                             // the rings are reset for the next item
    }
}

// Band nodes of one orbital for a given dmax (the band kernel's grid): nodes with
// d <= dmax.
__host__ __device__ inline long long band_nodes(int nx, int ny, int nz, int dmax) {
    const long long nxy = (long long)nx * ny;
    const int D = dmax + 1;
    if (nz <= 2 * D) return nxy * nz;
    const int fw = nx - 2 * D, fh = ny - 2 * D;
    const long long frame = nxy - (fw > 0 && fh > 0 ? (long long)fw * fh : 0);
    return 2 * (long long)D * nxy + (long long)(nz - 2 * D) * frame;
}

// The band: u^{j} = y + cdt (-i)[H u^{j-1} + E^T f^{j-1}] at every node with d <= dmax
// (j = 2, 3, 4 with dmax = 0, 1, 2), reading u^{j-1} from `w` (valid for d <= dmax + 1).
// Grid (ceil(band nodes / 256), n_orb); band nodes of an orbital in the order: the
// dmax + 1 lowest z planes, the frames of width dmax + 1 of the middle planes, the
// dmax + 1 highest planes.
static __global__ void __launch_bounds__(256) stencil_band(int nx, int ny, int nz, int n_orb, int dmax, float inv_h2,
                                                           const float2* __restrict__ w, const float2* y,
                                                           const float* __restrict__ V,
                                                           const float2* __restrict__ bterm, float2* out, float cdt) {
    const long long nxy = (long long)nx * ny, nvox = nxy * nz;
    const int D = dmax + 1;                                  // slab / frame width
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= band_nodes(nx, ny, nz, dmax)) return;
    int i, j, k;
    const int fw = nx - 2 * D, fh = ny - 2 * D;              // inner part of a middle plane
    const long long frame = nxy - (fw > 0 && fh > 0 ? (long long)fw * fh : 0);
    if (nz <= 2 * D || p < (long long)D * nxy) {             // whole planes: a thin box or the low slab
        k = (int)(p / nxy);
        const int r = (int)(p - (long long)k * nxy);
        j = r / nx; i = r - j * nx;
    } else if (p < (long long)D * nxy + (long long)(nz - 2 * D) * frame) {
        const long long q = p - (long long)D * nxy;
        k = D + (int)(q / frame);
        int r = (int)(q - (long long)(k - D) * frame);
        if (fw <= 0 || fh <= 0) { j = r / nx; i = r - j * nx; }
        else if (r < D * nx) { j = r / nx; i = r - j * nx; }
        else if (r < 2 * D * nx) { r -= D * nx; j = ny - D + r / nx; i = r % nx; }
        else { r -= 2 * D * nx; j = D + r / (2 * D); const int c = r % (2 * D); i = c < D ? c : nx - 2 * D + c; }
    } else {                                                 // the high slab
        const long long q = p - (long long)D * nxy - (long long)(nz - 2 * D) * frame;
        k = nz - D + (int)(q / nxy);
        const int r = (int)(q - (long long)(k - nz + D) * nxy);
        j = r / nx; i = r - j * nx;
    }
    if (fb_dist(i, j, k, nx, ny, nz) > dmax) return;         // (only for boxes thinner than the band)
    const int orb = blockIdx.y;
    const long long n = (long long)k * nxy + (long long)j * nx + i;
    const float2* wo = w + (long long)orb * nvox;
    const float2 z = make_float2(0.f, 0.f);
    const float2 c = wo[n];
    const float2 xm = i >= 1 ? wo[n - 1] : z, xp = i + 1 < nx ? wo[n + 1] : z;
    const float2 ym = j >= 1 ? wo[n - nx] : z, yp = j + 1 < ny ? wo[n + nx] : z;
    const float2 zm = k >= 1 ? wo[n - nxy] : z, zp = k + 1 < nz ? wo[n + nxy] : z;
    float2 b = z;
    if (on_gamma<1>(i, j, k, nx, ny, nz)) b = bterm[(long long)gamma_index<1>(i, j, k, nx, ny, nz) * n_orb + orb];
    const long long idx = (long long)orb * nvox + n;
    out[idx] = fb_node(c, xm, xp, ym, yp, zm, zp, V[n], inv_h2, y[idx], b, cdt);
}

}  // namespace dev
}  // namespace abc
