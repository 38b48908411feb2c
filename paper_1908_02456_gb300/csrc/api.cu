// C ABI of the time-stepper: context set-up and upload, the Horner-form step,
// graph-captured runs, diagnostics and kernel timing.  See include/abc.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "ctx.h"
#include "stencil_fused.cuh"
#include "cell_lanes.cuh"
#include "stencil_bulk.cuh"

namespace abc {
int fail(int status, const std::string& msg);
int check_params(const abc_grid* grid, const abc_params* params);
}  // namespace abc

using namespace abc;
using abc::dev::BlockInfo;

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(ABC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

inline size_t cplx_bytes(const abc_ctx* c) { return 2 * c->real_bytes; }

// Launch with a programmatic dependency on the preceding kernel of the stream: the
// kernel may start early and calls griddepcontrol.wait before it reads that kernel's
// results (inside a captured graph this becomes a programmatic edge).
// With pdl == false it is an ordinary launch.
template <typename... K, typename... A>
void launch_pdl(bool pdl, void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

int upload_tables(abc_ctx* c) {
    const Geometry& g = c->geo;
    struct { DevBuf* b; const int* src; size_t n; } t[] = {
        {&c->gamma_c, g.gamma_c.data(), g.gamma_c.size()},
        {&c->cell_out, g.cell_out.data(), g.cell_out.size()},
        {&c->cell_type, g.cell_type.data(), g.cell_type.size()},
        {&c->cell_c, g.cell_c.data(), g.cell_c.size()},
        {&c->cell_gi, g.cell_gi.data(), g.cell_gi.size()},
        {&c->cell_node, g.cell_node.data(), g.cell_node.size()},
        {&c->cell_wr, g.cell_wr.data(), g.cell_wr.size()},
    };
    for (auto& e : t) {
        int st = e.b->alloc(e.n * sizeof(int));
        if (st) return st;
        CUDA_TRY(cudaMemcpy(e.b->p, e.src, e.n * sizeof(int), cudaMemcpyHostToDevice));
    }
    int st;
    for (auto pr : {std::make_pair(&c->cell_coef_f, &g.coef_f), std::make_pair(&c->cell_coef_bt, &g.coef_bt)}) {
        const std::vector<double>& v = *pr.second;
        if (c->prec == ABC_FP64) {
            if ((st = pr.first->alloc(v.size() * sizeof(double)))) return st;
            CUDA_TRY(cudaMemcpy(pr.first->p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(v.begin(), v.end());
            if ((st = pr.first->alloc(f.size() * sizeof(float)))) return st;
            CUDA_TRY(cudaMemcpy(pr.first->p, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    return ABC_OK;
}

static_assert(abc::dev::SYM_CONSUMERS == abc::dev::SYM_GATHER_WARPS,
              "the back transform gathers one row partial per consumer warp of the contraction");

// Class blocks in the device format: row-major, rows padded to a multiple of 4
// complex elements so that every row starts on a 32-byte boundary.  One BlockInfo
// entry per (class, right-hand side), in ascending adapted offset.
int upload_matrices(abc_ctx* c) {
    const Geometry& g = c->geo;
    const bool o2 = c->params.order == 2;
    const bool f1 = c->params.order == 1 && c->blocks.rows1;
    const int nseg = o2 ? 4 : f1 ? 2 : 1;
    long long total = 0;
    std::vector<long long> moff(g.cls.size());
    std::vector<int> lds(g.cls.size()), segw(g.cls.size());
    for (size_t k = 0; k < g.cls.size(); ++k) {
        segw[k] = (g.cls[k].m + 3) & ~3;
        lds[k] = nseg * segw[k];
        moff[k] = total;
        total += (long long)lds[k] * g.cls[k].m;
    }
    struct E { int off, m, ld, sw; long long mo; };
    std::vector<E> es;
    for (size_t k = 0; k < g.cls.size(); ++k)
        for (int e = 0; e < g.cls[k].R; ++e) es.push_back({g.cls[k].moff[e], g.cls[k].m, lds[k], segw[k], moff[k]});
    std::sort(es.begin(), es.end(), [](const E& a, const E& b) { return a.off < b.off; });
    if ((int)es.size() > dev::MAX_ENTRIES) return fail(ABC_ERR_ARG, "internal: too many block entries");
    c->bi = BlockInfo{};
    c->bi.n = (int)es.size();
    c->bi.nseg = nseg;
    for (size_t i = 0; i < es.size(); ++i) {
        c->bi.m[i] = es[i].m;
        c->bi.off[i] = es[i].off;
        c->bi.ld[i] = es[i].ld;
        c->bi.segw[i] = es[i].sw;
        c->bi.mat_off[i] = es[i].mo;
    }
    if ((int)g.cls.size() > dev::MAX_CLASSES) return fail(ABC_ERR_ARG, "internal: too many classes");
    c->ci = dev::ClassInfo{};
    c->ci.n = (int)g.cls.size();
    c->ci.rowbase[0] = 0;
    for (size_t k = 0; k < g.cls.size(); ++k) {
        c->ci.R[k] = g.cls[k].R;
        c->ci.m[k] = g.cls[k].m;
        for (int e = 0; e < 3; ++e) c->ci.moff[k][e] = e < g.cls[k].R ? g.cls[k].moff[e] : 0;
        c->ci.ld[k] = lds[k];
        c->ci.segw[k] = segw[k];
        c->ci.mat_off[k] = moff[k];
        c->ci.rowbase[k + 1] = c->ci.rowbase[k] + (g.cls[k].m + dev::GEMV_RB - 1) / dev::GEMV_RB;
    }
    const size_t eb = cplx_bytes(c);
    int st = c->mat.alloc((size_t)total * eb);
    if (st) return st;
    CUDA_TRY(cudaMemset(c->mat.p, 0, (size_t)total * eb));
    for (size_t k = 0; k < g.cls.size(); ++k) {
        const int m = g.cls[k].m, ld = lds[k];
        // row a, segment q: order 2 [B1 | B0 - i A1 | -i A1 | A0] (the g equation with
        // E phidot = -i E H w - i f substituted); fitted order 1 [B | A]; otherwise the
        // single class block
        auto entry = [&](int q, int a, int b) -> cd {
            if (f1) return c->blocks.mat2[q][k][(size_t)a * m + b];
            if (!o2) return c->blocks.mat[k][(size_t)a * m + b];
            const size_t e = (size_t)a * m + b;
            const cd mi(0.0, -1.0);
            switch (q) {
                case 0: return c->blocks.mat2[0][k][e];
                case 1: return c->blocks.mat2[1][k][e] + mi * c->blocks.mat2[2][k][e];
                case 2: return mi * c->blocks.mat2[2][k][e];
                default: return c->blocks.mat2[3][k][e];
            }
        };
        std::vector<double> buf((size_t)2 * ld * m, 0.0);
        for (int a = 0; a < m; ++a)
            for (int q = 0; q < nseg; ++q)
                for (int b = 0; b < m; ++b) {
                    const cd v = entry(q, a, b);
                    buf[2 * ((size_t)a * ld + q * segw[k] + b)] = v.real();
                    buf[2 * ((size_t)a * ld + q * segw[k] + b) + 1] = v.imag();
                }
        if (c->prec == ABC_FP64) {
            CUDA_TRY(cudaMemcpy(c->mat.as<char>() + moff[k] * eb, buf.data(), buf.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> fb(buf.begin(), buf.end());
            CUDA_TRY(cudaMemcpy(c->mat.as<char>() + moff[k] * eb, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    return ABC_OK;
}

int ensure_gam(abc_ctx* c);

int ensure_workspace(abc_ctx* c) {
    const size_t cb = cplx_bytes(c);
    const size_t b = (size_t)c->params.max_orbitals;
    const size_t phi_b = (size_t)c->nvox * b * cb, aux_b = (size_t)c->geo.n_gamma * b * cb;
    const size_t state_aux_b = aux_b * (c->params.order == 2 ? 2 : 1);     // order 2: [f | g]
    int st;
    for (int i = 0; i < 2; ++i) {
        if ((st = c->Tp[i].alloc(phi_b))) return st;
        if ((st = c->Tf[i].alloc(state_aux_b))) return st;
    }
    if ((st = c->hat_phi.alloc(aux_b))) return st;
    if ((st = c->hat_f.alloc(aux_b))) return st;
    if (c->params.order == 1) {
        if ((st = c->hat2_phi.alloc(aux_b))) return st;
        if ((st = c->hat2_f.alloc(aux_b))) return st;
    }
    if (c->params.order == 2) {
        if ((st = c->hat_h.alloc(aux_b))) return st;
        if ((st = c->hat_g.alloc(aux_b))) return st;
    }
    if ((st = c->tvec.alloc(aux_b))) return st;
    if ((st = c->cnat.alloc(aux_b))) return st;
    if ((st = c->Veff.alloc((size_t)c->nvox * c->real_bytes))) return st;
    CUDA_TRY(cudaMemset(c->Tf[0].p, 0, state_aux_b));
    CUDA_TRY(cudaMemset(c->Tf[1].p, 0, state_aux_b));
    return ABC_OK;
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

void prof_begin(abc_ctx* c, int k, cudaStream_t s) {
    if (!c->profiling) return;
    ProfileSlot& ps = c->prof[k];
    if (ps.used + 2 > ps.ev.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ps.ev.push_back(e);
        }
    }
    cudaEventRecord(ps.ev[ps.used], s);
}
void prof_end(abc_ctx* c, int k, cudaStream_t s) {
    if (!c->profiling) return;
    ProfileSlot& ps = c->prof[k];
    cudaEventRecord(ps.ev[ps.used + 1], s);
    ps.used += 2;
}

}  // namespace

namespace {
int build_tiles(abc_ctx* c) {
    std::vector<int> tb, tr;
    for (int p = 0; p < c->bi.n; ++p)
        for (int r0 = 0; r0 < c->bi.m[p]; r0 += 32) { tb.push_back(p); tr.push_back(r0); }
    c->n_tiles = (int)tb.size();
    int st;
    if ((st = c->tile_blk.alloc(tb.size() * sizeof(int)))) return st;
    if ((st = c->tile_row.alloc(tr.size() * sizeof(int)))) return st;
    CUDA_TRY(cudaMemcpy(c->tile_blk.p, tb.data(), tb.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->tile_row.p, tr.data(), tr.size() * sizeof(int), cudaMemcpyHostToDevice));
    return ABC_OK;
}

// Packed lower-triangular 64x64 tiles of every distinct block (complex64), the
// per-CTA segment lists and the partial-sum scratch of sym_gemv_tiles.
int build_sym(abc_ctx* c) {
    using abc::dev::SYM_T;
    const Geometry& g = c->geo;
    abc::dev::SymInfo si{};
    int nc = 0;
    long long tb = 0;
    int rb = 0;
    if ((int)g.cls.size() > abc::dev::SYM_CMAX) return fail(ABC_ERR_ARG, "internal: too many classes");
    for (const auto& k : g.cls) {
        const int nt = (k.m + SYM_T - 1) / SYM_T;
        for (int e = 0; e < k.R; ++e) si.moff[nc][e] = k.moff[e];
        si.R[nc] = k.R;
        si.m[nc] = k.m;
        si.nt[nc] = nt;
        si.tbase[nc] = tb;
        si.rbase[nc] = rb;
        tb += (long long)nt * (nt + 1) / 2;
        rb += nt;
        ++nc;
    }
    si.nclass = nc;
    const long long NT = tb;
    // tiles
    std::vector<float> host((size_t)NT * SYM_T * SYM_T * 2, 0.0f);
    std::vector<int> tile_c(NT), tile_I(NT);
    for (int k = 0; k < nc; ++k) {
        const int m = si.m[k];
        const std::vector<cd>& S = c->blocks.mat[k];
        for (int I = 0; I < si.nt[k]; ++I)
            for (int J = 0; J <= I; ++J) {
                const long long t = si.tbase[k] + (long long)I * (I + 1) / 2 + J;
                tile_c[t] = k;
                tile_I[t] = I;
                float* dst = host.data() + (size_t)t * SYM_T * SYM_T * 2;
                for (int r = 0; r < SYM_T; ++r) {
                    const int row = I * SYM_T + r;
                    if (row >= m) break;
                    for (int col = 0; col < SYM_T; ++col) {
                        const int cc = J * SYM_T + col;
                        if (cc >= m) break;
                        const cd v = S[(size_t)row * m + cc];
                        const int q = abc::dev::sym_pack_index(r, col);
                        dst[2 * q] = (float)v.real();
                        dst[2 * q + 1] = (float)v.imag();
                    }
                }
            }
    }
    int st;
    if ((st = c->sym_tiles.alloc(host.size() * sizeof(float)))) return st;
    CUDA_TRY(cudaMemcpy(c->sym_tiles.p, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice));
    // Work units: tile rows of a class (row I has I + 1 tiles), split into segments (runs
    // of tiles of one row); a segment's row part stays in registers and is stored once at
    // its end.  Costs are a model fitted to per-CTA timings of this kernel on GB300 (us):
    // 1.0 per segment, and per tile 0.36 / 0.59 / 0.87 off the diagonal and 0.0 / 0.29 /
    // 0.41 on it for R = 1 / 2 / 3 right-hand sides.  Two kinds of partition are built
    // and the one with the smallest predicted makespan is kept: contiguous runs of tiles
    // cut at the per-CTA cost target (`contiguous`), and pieces of at most `cap` tiles
    // bin-packed over the CTAs longest first (`lpt`, a CTA takes any set of segments).
    // Segments are numbered by (class, row, first tile), so the segments of one row are
    // consecutive (the back transform's gather relies on it).
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int G = std::max(1, sms);
    struct Piece { int c, I, t0, t1; double cost; };
    static const double tile_off[4] = {0.0, 0.36, 0.59, 0.87}, tile_diag[4] = {0.0, 0.0, 0.29, 0.41};
    const double seg_cost = 1.0;
    auto make_pieces = [&](int cap, std::vector<Piece>& out) {
        out.clear();
        for (int k = 0; k < nc; ++k)
            for (int I = 0; I < si.nt[k]; ++I) {
                const int len = I + 1, np = (len + cap - 1) / cap;
                const int t0 = (int)(si.tbase[k] + (long long)I * (I + 1) / 2);
                for (int q = 0; q < np; ++q) {
                    const int a = t0 + q * len / np, b = t0 + (q + 1) * len / np;
                    const bool has_diag = q == np - 1;          // the row's last tile is its diagonal one
                    const int R = si.R[k];
                    const double cost = seg_cost + (b - a - (has_diag ? 1 : 0)) * tile_off[R] +
                                        (has_diag ? tile_diag[R] : 0.0);
                    out.push_back({k, I, a, b, cost});
                }
            }
    };
    auto lpt = [&](const std::vector<Piece>& ps, std::vector<int>& owner) {
        std::vector<int> order(ps.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ps[a].cost > ps[b].cost; });
        std::vector<double> load(G, 0.0);
        std::vector<int> cnt(G, 0);
        owner.assign(ps.size(), 0);
        for (int i : order) {
            // least loaded CTA that still has room in its segment cache
            int best = -1;
            for (int g2 = 0; g2 < G; ++g2)
                if (cnt[g2] < abc::dev::SYM_SEG_CACHE && (best < 0 || load[g2] < load[best])) best = g2;
            if (best < 0) return 1e300;
            owner[i] = best;
            load[best] += ps[i].cost;
            ++cnt[best];
        }
        return *std::max_element(load.begin(), load.end());
    };
    // Contiguous runs of tiles in (class, row, tile) order: a CTA takes tiles while its
    // cost (tiles plus one segment cost at every row start and at every cut) stays within
    // half a tile of the target (total + G segment costs) / G; its run is split at row
    // ends into its segments.
    auto contiguous = [&](std::vector<Piece>& out, std::vector<int>& own) {
        struct T1 { int k, I, t; double c; };
        std::vector<T1> tl;
        double total = 0.0;
        for (int k = 0; k < nc; ++k)
            for (int I = 0; I < si.nt[k]; ++I) {
                const int t0 = (int)(si.tbase[k] + (long long)I * (I + 1) / 2);
                for (int J = 0; J <= I; ++J) {
                    const double ct = (J < I ? tile_off[si.R[k]] : tile_diag[si.R[k]]) + (J == 0 ? seg_cost : 0.0);
                    tl.push_back({k, I, t0 + J, ct});
                    total += ct;
                }
            }
        const double target = (total + seg_cost * G) / G;
        out.clear();
        own.clear();
        std::vector<double> load(G, 0.0);
        int b = 0;
        size_t i = 0;
        while (i < tl.size()) {
            // one segment: tiles of the same row, within CTA b
            const size_t i0 = i;
            double c = (tl[i].t == (int)(si.tbase[tl[i].k] + (long long)tl[i].I * (tl[i].I + 1) / 2)) ? 0.0 : seg_cost;
            while (i < tl.size() && tl[i].k == tl[i0].k && tl[i].I == tl[i0].I) {
                if (b < G - 1 && load[b] + c + 0.5 * tl[i].c > target && i > i0) break;
                c += tl[i].c;
                ++i;
            }
            if (i == i0) {                                // the CTA is full before this segment starts
                ++b;
                continue;
            }
            out.push_back({tl[i0].k, tl[i0].I, tl[i0].t, tl[i - 1].t + 1, c});
            own.push_back(b);
            load[b] += c;
            if (i < tl.size() && b < G - 1 && load[b] + 0.5 * tl[i].c > target) ++b;
        }
        for (int g2 = 0; g2 < G; ++g2) {
            int n = 0;
            for (int o : own) n += o == g2;
            if (n > abc::dev::SYM_SEG_CACHE) return 1e300;
        }
        return *std::max_element(load.begin(), load.end());
    };
    std::vector<Piece> pieces, trial;
    std::vector<int> owner, trial_owner;
    double best_span = contiguous(pieces, owner);
    for (int cap : {4, 6, 8, 12, 16}) {
        make_pieces(cap, trial);
        const double span = lpt(trial, trial_owner);
        if (span < best_span - 1e-9) {
            best_span = span;
            pieces = trial;
            owner = trial_owner;
        }
    }
    if (best_span >= 1e300) return fail(ABC_ERR_ARG, "internal: too many segments for the tiled contraction");
    // pieces are generated in (class, row, first tile) order already: their index is the segment id
    std::vector<int4> segs(pieces.size());
    for (size_t i = 0; i < pieces.size(); ++i)
        segs[i] = make_int4(pieces[i].c, pieces[i].I, pieces[i].t0, pieces[i].t1);
    // per-CTA work lists at a fixed stride: (16 s + class, I, first tile, end tile)
    const int CAP = abc::dev::SYM_SEG_CACHE;
    static_assert(abc::dev::SYM_SEG_CACHE <= abc::dev::SYM_THREADS, "one record per thread");
    static_assert(abc::dev::SYM_CMAX <= 16, "class index packed in 4 bits");
    std::vector<int4> rec((size_t)G * CAP, make_int4(0, 0, 0, 0));
    std::vector<int> cta_cnt(G, 0);
    for (size_t i = 0; i < pieces.size(); ++i) {
        const int b = owner[i];
        if (cta_cnt[b] >= CAP) return fail(ABC_ERR_ARG, "internal: too many segments for one CTA of the tiled contraction");
        if (i >= (size_t)1 << 27) return fail(ABC_ERR_ARG, "internal: too many segments for the tiled contraction");
        rec[(size_t)b * CAP + cta_cnt[b]++] = make_int4(((int)i << 4) | segs[i].x, segs[i].y, segs[i].z, segs[i].w);
    }
    std::vector<int2> rowseg(rb, make_int2(0, 0));
    for (size_t s = 0; s < segs.size(); ++s) {
        const int cI = si.rbase[segs[s].x] + segs[s].y;
        if (rowseg[cI].y == 0) rowseg[cI].x = (int)s;
        rowseg[cI].y = (int)s + 1;
    }
    if ((st = c->sym_seg.alloc(rec.size() * sizeof(int4)))) return st;
    if ((st = c->sym_cta.alloc(cta_cnt.size() * sizeof(int)))) return st;
    if ((st = c->sym_rowseg.alloc(rowseg.size() * sizeof(int2)))) return st;
    if ((st = c->sym_rowpart.alloc(segs.size() * SYM_T * abc::dev::SYM_RMAX * abc::dev::SYM_CONSUMERS *
                                   sizeof(float2))))
        return st;
    if ((st = c->sym_colpart.alloc((size_t)NT * SYM_T * abc::dev::SYM_RMAX * sizeof(float2)))) return st;
    if ((st = c->err_flag.alloc(sizeof(int)))) return st;
    CUDA_TRY(cudaMemcpy(c->sym_seg.p, rec.data(), rec.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->sym_cta.p, cta_cnt.data(), cta_cnt.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->sym_rowseg.p, rowseg.data(), rowseg.size() * sizeof(int2), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(c->err_flag.p, 0, sizeof(int)));
    CUDA_TRY(cudaFuncSetAttribute(abc::dev::sym_gemv_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)abc::dev::SYM_SMEM));
    // the forward transform that precedes the one-orbital contraction runs with the largest
    // shared-memory carveout, so the contraction's CTAs (launched as its programmatic
    // dependents) fit on an SM beside its blocks
    CUDA_TRY(cudaFuncSetAttribute(abc::dev::bnd_forward<float, 0, true>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared));
    c->si = si;
    c->sym_grid = G;
    c->sym_tiles_n = NT;
    c->l2_keep_tiles = 0;
    // gather descriptors of the back transform, indexed like the cell output table
    std::vector<int4> gdesc((size_t)g.n_cells * 64, make_int4(0, 0, 0, 0));
    std::vector<int> cls_of(g.n_gamma, -1), rhs_of(g.n_gamma, -1);
    for (size_t k = 0; k < g.cls.size(); ++k)
        for (int e = 0; e < g.cls[k].R; ++e)
            for (int q = 0; q < g.cls[k].m; ++q) {
                cls_of[g.cls[k].moff[e] + q] = (int)k;
                rhs_of[g.cls[k].moff[e] + q] = e;
            }
    for (size_t i = 0; i < gdesc.size(); ++i) {
        const int jj = g.cell_out[i];
        if (jj < 0) continue;
        const int k = cls_of[jj], e = rhs_of[jj];
        const int row = jj - si.moff[k][e], I = row / SYM_T, r = row % SYM_T;
        const int2 rs = rowseg[si.rbase[k] + I];
        const long long t1 = si.tbase[k] + (long long)(I + 1) * (I + 2) / 2 + I;
        const int nk = si.nt[k] - 1 - I;
        gdesc[i] = make_int4((int)((((long long)rs.x * abc::dev::SYM_CONSUMERS) * 3 + e) * SYM_T + r), rs.y - rs.x,
                             nk > 0 ? (int)((t1 * 3 + e) * SYM_T + r) : 0, nk | ((I + 2) << 16));
    }
    if ((st = c->sym_gdesc.alloc(gdesc.size() * sizeof(int4)))) return st;
    CUDA_TRY(cudaMemcpy(c->sym_gdesc.p, gdesc.data(), gdesc.size() * sizeof(int4), cudaMemcpyHostToDevice));
    abc::dev::SymGather& sg = c->sym_gather;
    sg.desc = c->sym_gdesc.as<int4>();
    sg.rowpart = c->sym_rowpart.as<float2>();
    sg.colpart = c->sym_colpart.as<float2>();
    c->sym = true;
    return ABC_OK;
}

// TF32 with round-to-nearest, ties away from zero (the device's cvt.rna.tf32.f32).
float tf32_rna(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Output tiles and work lists of the persistent GEMM for every orbital count
// 1..max_orbitals (largest classes first), for the context's tile configuration
// (tc_cfg: 0 96 columns, one CTA per SM; 1 64 columns, two CTAs per SM; 2 the Karatsuba
// form, 64 columns, one CTA per SM) and split
// choice (tc_split = 0: about two items per CTA slot; else that many K splits).
int build_tc_plans(abc_ctx* c) {
    using namespace abc::dev;
    const Geometry& g = c->geo;
    const TcInfo& info = c->tci;
    const int nmax = c->tc_cfg == 0 ? TcWide::nmax : c->tc_cfg == 1 ? TcNarrow::nmax : TcKara::nmax;
    const int slots = c->tc_sms * (c->tc_cfg == 0 ? TcWide::cps : c->tc_cfg == 1 ? TcNarrow::cps : TcKara::cps);
    const double a_chunk = c->tc_cfg == 2 ? (double)TcKara::a_bytes : (double)TC_A_BYTES;
    std::vector<int> order(g.cls.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g.cls[a].m > g.cls[b].m; });
    std::vector<TcTile> tiles;
    std::vector<TcCols> cranges;
    std::vector<TcItem> items;
    std::vector<int> item_off;
    const int B = c->params.max_orbitals;
    c->tc_b.assign(B + 1, abc_ctx::TcPlan{});
    long long max_chunks = 0, max_part = 0;
    for (int b = 1; b <= B; ++b) {
        abc_ctx::TcPlan& pl = c->tc_b[b];
        pl.tile_off = (int)tiles.size();
        pl.cols_off = (int)cranges.size();
        int chunks = 0, maxnkb = 1;
        for (int k : order) {
            const int cols = g.cls[k].R * b;
            const int nch = (cols + nmax - 1) / nmax;
            const int w = ((cols + nch - 1) / nch + 15) / 16 * 16;
            maxnkb = std::max(maxnkb, info.nkb[k]);
            for (int col0 = 0; col0 < cols; col0 += w) {
                const int n = std::min(w, (cols - col0 + 15) / 16 * 16);
                cranges.push_back(TcCols{k, col0, n, chunks});
                for (int mt = 0; mt * TC_M < g.cls[k].m; ++mt) tiles.push_back(TcTile{k, mt * TC_M, col0, n, chunks});
                chunks += info.nkb[k];
            }
        }
        pl.tile_cnt = (int)tiles.size() - pl.tile_off;
        pl.cols_cnt = (int)cranges.size() - pl.cols_off;
        pl.max_nkb = maxnkb;
        // about two items per CTA slot unless fixed; partial sums of the splits are added
        // by the back transform
        pl.nsplit = c->tc_split > 0 ? std::min(c->tc_split, TC_MAX_SPLIT)
                                    : std::max(1, std::min(TC_MAX_SPLIT, (2 * slots + pl.tile_cnt - 1) / pl.tile_cnt));
        // persistent GEMM: items (tile, split) longest first, each given to the CTA with the
        // least work so far; cost = bytes streamed for the item (its K blocks of A and X,
        // plus two K blocks' worth for the fill and the epilogue).  Items of equal cost
        // stay in (class, row tile, split, column range) order, so the items that share an
        // A chunk go to different CTAs at about the same time.
        {
            std::vector<TcItem> its;
            for (int ti = pl.tile_off; ti < pl.tile_off + pl.tile_cnt; ++ti)
                for (int sp = 0; sp < pl.nsplit; ++sp) its.push_back(TcItem{ti, sp});
            auto item_cost = [&](const TcItem& w) {
                const TcTile& x = tiles[w.tile];
                const int nkb = info.nkb[x.cls];
                const int nk = (int)((long long)nkb * (w.split + 1) / pl.nsplit - (long long)nkb * w.split / pl.nsplit);
                return (nk + 2.0) * (a_chunk + (double)x.n * 64 * TC_B_PLANES);
            };
            std::stable_sort(its.begin(), its.end(), [&](const TcItem& a, const TcItem& b2) {
                const double ca = item_cost(a), cb = item_cost(b2);
                if (ca != cb) return ca > cb;
                const TcTile &x = tiles[a.tile], &y = tiles[b2.tile];
                if (x.cls != y.cls) return x.cls < y.cls;
                if (x.row0 != y.row0) return x.row0 < y.row0;
                if (a.split != b2.split) return a.split < b2.split;
                return x.col0 < y.col0;
            });
            const int G = std::min<int>(slots, (int)its.size());
            std::vector<std::vector<TcItem>> per(G);
            std::vector<double> load(G, 0.0);
            for (const TcItem& w : its) {
                int best = 0;
                for (int g2 = 1; g2 < G; ++g2)
                    if (load[g2] < load[best]) best = g2;
                per[best].push_back(w);
                load[best] += item_cost(w);
            }
            pl.grid = G;
            pl.off_base = (int)item_off.size();
            for (int g2 = 0; g2 < G; ++g2) {
                item_off.push_back((int)items.size());
                for (const TcItem& w : per[g2]) items.push_back(w);
            }
            item_off.push_back((int)items.size());
        }
        max_chunks = std::max<long long>(max_chunks, chunks);
        if (pl.nsplit > 1) max_part = std::max<long long>(max_part, (long long)pl.nsplit * g.n_gamma * b);
    }
    int st;
    if ((st = c->tc_tiles.alloc(tiles.size() * sizeof(TcTile)))) return st;
    CUDA_TRY(cudaMemcpy(c->tc_tiles.p, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice));
    if ((st = c->tc_cols.alloc(cranges.size() * sizeof(TcCols)))) return st;
    CUDA_TRY(cudaMemcpy(c->tc_cols.p, cranges.data(), cranges.size() * sizeof(TcCols), cudaMemcpyHostToDevice));
    if ((st = c->tc_items.alloc(items.size() * sizeof(TcItem)))) return st;
    CUDA_TRY(cudaMemcpy(c->tc_items.p, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice));
    if ((st = c->tc_item_off.alloc(item_off.size() * sizeof(int)))) return st;
    CUDA_TRY(cudaMemcpy(c->tc_item_off.p, item_off.data(), item_off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((size_t)max_chunks * TC_B_BYTES > c->tc_bpack.bytes && (st = c->tc_bpack.alloc((size_t)max_chunks * TC_B_BYTES)))
        return st;
    if ((size_t)max_part * sizeof(float2) > c->tc_part.bytes && (st = c->tc_part.alloc((size_t)max_part * sizeof(float2))))
        return st;
    return ABC_OK;
}

// The GEMM's A operand image: every class block split into hi / lo planes (TF32, or
// FP16 after the class scale 2^es) in the shared-memory image of gemm_tc, per (128-row
// tile, K block): 4 planes (Re hi, Re lo, Im hi, Im lo), or for the Karatsuba form 6
// (the same plus (Re + Im) hi, lo).
int pack_a_image(abc_ctx* c, bool kara) {
    using namespace abc::dev;
    const Geometry& g = c->geo;
    const TcInfo& info = c->tci;
    const bool f16 = c->tc_f16;
    const int KB = f16 ? TcKind<TC_F16>::KB : TcKind<TC_TF32>::KB;
    const int nplanes = kara ? 6 : 4;
    const size_t per = (size_t)nplanes * TC_A_PLANE / 4;
    const long long chunks = c->tc_chunks;
    std::vector<float> pack((size_t)chunks * per, 0.0f);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long ch = 0; ch < chunks; ++ch) {
        int k = 0;
        while (k + 1 < (int)g.cls.size() && ch >= info.abase[k + 1]) ++k;
        const int m = info.m[k], nkb = info.nkb[k];
        const long long loc = ch - info.abase[k];
        const int mt = (int)(loc / nkb), kb = (int)(loc % nkb);
        const std::vector<cd>& S = c->blocks.mat[k];
        float* dst = pack.data() + (size_t)ch * per;
        __half* dh = reinterpret_cast<__half*>(dst);
        const double sc = std::ldexp(1.0, info.es[k]);
        for (int r = 0; r < TC_M; ++r) {
            const int row = mt * TC_M + r;
            if (row >= m) break;
            for (int q = 0; q < KB; ++q) {
                const int col = kb * KB + q;
                if (col >= m) break;
                const cd v = S[(size_t)row * m + col];
                const double parts[3] = {v.real(), v.imag(), v.real() + v.imag()};
                for (int pp = 0; pp < nplanes / 2; ++pp) {
                    if (f16) {
                        const float x = (float)(parts[pp] * sc);
                        const __half xh = __float2half_rn(x);
                        const size_t o = tc_core_offset_f16(r, q) / 2;
                        dh[(2 * pp) * (TC_A_PLANE / 2) + o] = xh;
                        dh[(2 * pp + 1) * (TC_A_PLANE / 2) + o] = __float2half_rn(x - __half2float(xh));
                    } else {
                        const float x = (float)parts[pp];
                        const float xh = tf32_rna(x);
                        const size_t o = tc_core_offset(r, q) / 4;
                        dst[(2 * pp) * (TC_A_PLANE / 4) + o] = xh;
                        dst[(2 * pp + 1) * (TC_A_PLANE / 4) + o] = tf32_rna(x - xh);
                    }
                }
            }
        }
    }
    DevBuf& out = kara ? c->tc_apack_k : c->tc_apack;
    int st;
    if ((st = out.alloc(pack.size() * sizeof(float)))) return st;
    CUDA_TRY(cudaMemcpy(out.p, pack.data(), pack.size() * sizeof(float), cudaMemcpyHostToDevice));
    return ABC_OK;
}

// Tensor-core form of the many-orbital contraction: every class block split into
// hi / lo planes of its real and imaginary parts (TF32, or FP16 after scaling the
// block by 2^es), packed per (128-row tile, K block) in the shared-memory image of
// gemm_tc, and the output tiles for every orbital count 1..max_orbitals (largest
// classes first).
int build_tc(abc_ctx* c) {
    using namespace abc::dev;
    const Geometry& g = c->geo;
    if ((int)g.cls.size() > SYM_CMAX) return fail(ABC_ERR_ARG, "internal: too many classes");
    const bool f16 = c->prec == ABC_C64_SPLIT_FP16;
    const int KB = f16 ? TcKind<TC_F16>::KB : TcKind<TC_TF32>::KB;
    TcInfo info{};
    info.ncls = (int)g.cls.size();
    long long chunks = 0;
    int rsum = 0;
    for (size_t k = 0; k < g.cls.size(); ++k) {
        info.m[k] = g.cls[k].m;
        info.R[k] = g.cls[k].R;
        for (int e = 0; e < 3; ++e) info.moff[k][e] = g.cls[k].moff[e];
        info.nkb[k] = (g.cls[k].m + KB - 1) / KB;
        info.abase[k] = chunks;
        info.rsum[k] = rsum;
        rsum += g.cls[k].R;
        chunks += (long long)((g.cls[k].m + TC_M - 1) / TC_M) * info.nkb[k];
        // FP16: the block's largest real or imaginary part scaled into [2^13, 2^14)
        double mx = 0;
        for (const cd& v : c->blocks.mat[k]) mx = std::max(mx, std::max(std::fabs(v.real()), std::fabs(v.imag())));
        int ex = 0;
        if (mx > 0) std::frexp(mx, &ex);                 // mx = f 2^ex, f in [0.5, 1)
        info.es[k] = f16 && mx > 0 ? std::min(60, std::max(-60, TC_TARGET_EXP - ex)) : 0;
    }
    c->tc_f16 = f16;
    c->tci = info;
    c->tc_chunks = chunks;
    int st;
    if ((st = pack_a_image(c, false))) return st;
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (!c->err_flag.p) {
        if ((st = c->err_flag.alloc(sizeof(int)))) return st;
        CUDA_TRY(cudaMemset(c->err_flag.p, 0, sizeof(int)));
    }
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_TF32, TcWide>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcWide::smem));
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_F16, TcWide>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcWide::smem));
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_TF32, TcNarrow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TcNarrow::smem));
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_F16, TcNarrow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TcNarrow::smem));
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_TF32, TcKara>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcKara::smem));
    CUDA_TRY(cudaFuncSetAttribute(gemm_tc<TC_F16, TcKara>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcKara::smem));
    if (f16 && (st = c->tc_colexp.alloc(sizeof(int) * (size_t)rsum * c->params.max_orbitals))) return st;
    if (f16) {   // tc_colexp_nm's column maxima and completion counters (zero between calls)
        const size_t n = (size_t)rsum * c->params.max_orbitals;
        if ((st = c->tc_colmax.alloc(sizeof(unsigned) * (n + n / 32 + 1)))) return st;
        CUDA_TRY(cudaMemset(c->tc_colmax.p, 0, sizeof(unsigned) * (n + n / 32 + 1)));
    }
    c->tc_f16 = f16;
    c->tc_ncols = rsum;
    c->tc_sms = sms;
    c->tci = info;
    if ((st = build_tc_plans(c))) return st;
    c->tc = true;
    return ABC_OK;
}

// Waits on a barrier that nothing completes, at most `polls` polls, then raises the
// error flag the way the contraction's bounded waits do (the fault-free check of that
// path; nothing traps or spins without a bound).
__global__ void wait_selftest_kernel(long long polls, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);                // one arrival expected, none ever made
        dev::fence_mbar_init();
    }
    __syncthreads();
    bool done = false;
    for (long long i = 0; i < polls && !done; ++i) done = dev::mbar_try_wait(&bar, 0);
    if (!done && threadIdx.x == 0) atomicExch(err, 1);
}

// A device wait that gave up (bounded mbarrier waits) -> ABC_ERR_TIMEOUT; resets the flag.
int check_device_flag(abc_ctx* c, cudaStream_t s) {
    if (!c->err_flag.p) return ABC_OK;
    int v = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, c->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (v) {
        CUDA_TRY(cudaMemsetAsync(c->err_flag.p, 0, sizeof(int), s));
        return fail(ABC_ERR_TIMEOUT, "a bounded device wait in the boundary contraction gave up");
    }
    return ABC_OK;
}

// Where a contraction left its result: partial sums for the back transform to
// gather (packed tiles), or nsplit arrays t + s * stride to add (split-K tensor
// cores), or plain t (nsplit = 1).
struct TRes {
    bool gathered = false;
    bool xform = false;        // t holds the order-1 back transform's x (XEpi), node-major
    const void* t = nullptr;
    int nsplit = 1;
    long long stride = 0;
};

// The persistent tensor-core GEMM in the context's tile configuration.
template <int KIND>
void launch_gemm_tc(abc_ctx* c, const abc_ctx::TcPlan& pl, int n_orb, float2* out, int conj, const int* colexp,
                    cudaStream_t s, int nm = 0, dev::XEpi xe = dev::XEpi{}) {
    const long long n = c->geo.n_gamma;
    if (c->tc_cfg == 2)
        dev::gemm_tc<KIND, dev::TcKara><<<(unsigned)pl.grid, dev::TC_THREADS, dev::TcKara::smem, s>>>(
            c->tci, c->tc_tiles.as<dev::TcTile>(), c->tc_items.as<dev::TcItem>(), c->tc_item_off.as<int>() + pl.off_base,
            c->tc_apack_k.as<float>(), c->tc_bpack.as<float>(), n_orb, (int)n, pl.nsplit, n * n_orb, out, conj,
            c->err_flag.as<int>(), colexp, nm, xe);
    else if (c->tc_cfg == 0)
        dev::gemm_tc<KIND, dev::TcWide><<<(unsigned)pl.grid, dev::TC_THREADS, dev::TcWide::smem, s>>>(
            c->tci, c->tc_tiles.as<dev::TcTile>(), c->tc_items.as<dev::TcItem>(), c->tc_item_off.as<int>() + pl.off_base,
            c->tc_apack.as<float>(), c->tc_bpack.as<float>(), n_orb, (int)n, pl.nsplit, n * n_orb, out, conj,
            c->err_flag.as<int>(), colexp, nm, xe);
    else
        dev::gemm_tc<KIND, dev::TcNarrow><<<(unsigned)pl.grid, dev::TC_THREADS, dev::TcNarrow::smem, s>>>(
            c->tci, c->tc_tiles.as<dev::TcTile>(), c->tc_items.as<dev::TcItem>(), c->tc_item_off.as<int>() + pl.off_base,
            c->tc_apack.as<float>(), c->tc_bpack.as<float>(), n_orb, (int)n, pl.nsplit, n * n_orb, out, conj,
            c->err_flag.as<int>(), colexp, nm, xe);
}

// The boundary contraction t = S x (conj: conj(S) x).  nm: x and t node-major
// (tensor-core path, n_orb a multiple of 32).
template <typename T>
TRes contraction(abc_ctx* c, const void* x, void* t, int n_orb, int conj, cudaStream_t s,
                 const void* const* x4 = nullptr, bool nm = false, const dev::XEpi* xe = nullptr) {
    typedef typename dev::C2<T>::t V;
    dev::XSeg<V> xs{{(const V*)x, nullptr, nullptr, nullptr}};
    if (x4)
        for (int q = 0; q < 4; ++q) xs.p[q] = (const V*)x4[q];
    const int n = c->geo.n_gamma;
    TRes res;
    res.t = t;
    const bool tc_path = n_orb > 1 && sizeof(T) == 4 && c->tc;
    if (!tc_path) prof_begin(c, ABC_KERNEL_CONTRACTION, s);
    if (n_orb == 1 && sizeof(T) == 4 && c->sym) {
        // early start behind the forward transform, except when the launch is timed by
        // an event pair (profiling), which must bracket the kernel alone
        launch_pdl(c->pdl && !c->profiling, dev::sym_gemv_tiles, dim3(c->sym_grid), dim3(dev::SYM_THREADS), dev::SYM_SMEM, s, c->si,
                   c->sym_tiles.as<const float2>(), c->sym_seg.as<const int4>(), c->sym_cta.as<const int>(),
                   (const float2*)x, c->sym_rowpart.as<float2>(), c->sym_colpart.as<float2>(), conj,
                   (long long)c->l2_keep_tiles, c->err_flag.as<int>());
        res.gathered = true;
    } else if (n_orb == 1) {
        dev::gemv_classes<T><<<c->ci.rowbase[c->ci.n], 32 * dev::GEMV_WARPS, 0, s>>>(c->ci, c->mat.as<V>(), xs,
                                                                                  (V*)t, conj);
    } else if (tc_path) {
        const abc_ctx::TcPlan& pl = c->tc_b[n_orb];
        // the operand packing has its own timing slot, so the contraction slot times the GEMM alone
        prof_begin(c, ABC_KERNEL_PACK, s);
        const dim3 pgrid((unsigned)pl.cols_cnt, (unsigned)((pl.max_nkb + dev::TC_PACK_KB - 1) / dev::TC_PACK_KB));
        float2* out = pl.nsplit > 1 ? c->tc_part.as<float2>() : (float2*)t;
        const int* colexp = c->tc_colexp.as<int>();
        // the epilogue forms the back transform's x when the whole sum is in one item
        const dev::XEpi xep = nm && xe && pl.nsplit == 1 ? *xe : dev::XEpi{};
        res.xform = xep.ac != nullptr;
        if (c->tc_f16) {
            const int ncols = c->tc_ncols * n_orb;
            if (nm)
                dev::tc_colexp_nm<<<(unsigned)(ncols / 32 * dev::CX_PARTS), 32 * dev::CX_WARPS, 0, s>>>(
                    c->tci, n_orb, (const float2*)x, c->tc_colexp.as<int>(), c->tc_colmax.as<unsigned>(),
                    c->tc_colmax.as<unsigned>() + (size_t)c->tc_ncols * c->params.max_orbitals);
            else
                dev::tc_colexp<<<(unsigned)((ncols + 7) / 8), 256, 0, s>>>(c->tci, n_orb, n, (const float2*)x,
                                                                           c->tc_colexp.as<int>(), ncols);
            if (c->tc_cfg == 2)
                dev::pack_x_tc<dev::TC_F16, 1><<<pgrid, 128, 0, s>>>(c->tci, c->tc_cols.as<dev::TcCols>() + pl.cols_off,
                                                                      n_orb, n, (const float2*)x, conj,
                                                                      c->tc_bpack.as<float>(), colexp, (int)nm);
            else
                dev::pack_x_tc<dev::TC_F16><<<pgrid, 128, 0, s>>>(c->tci, c->tc_cols.as<dev::TcCols>() + pl.cols_off,
                                                                   n_orb, n, (const float2*)x, conj,
                                                                   c->tc_bpack.as<float>(), colexp, (int)nm);
            prof_end(c, ABC_KERNEL_PACK, s);
            prof_begin(c, ABC_KERNEL_CONTRACTION, s);
            launch_gemm_tc<dev::TC_F16>(c, pl, n_orb, out, conj, colexp, s, (int)nm, xep);
            c->launches += 2;
        } else {
            if (c->tc_cfg == 2)
                dev::pack_x_tc<dev::TC_TF32, 1><<<pgrid, 128, 0, s>>>(c->tci, c->tc_cols.as<dev::TcCols>() + pl.cols_off,
                                                                       n_orb, n, (const float2*)x, conj,
                                                                       c->tc_bpack.as<float>(), colexp, (int)nm);
            else
                dev::pack_x_tc<dev::TC_TF32><<<pgrid, 128, 0, s>>>(c->tci, c->tc_cols.as<dev::TcCols>() + pl.cols_off,
                                                                    n_orb, n, (const float2*)x, conj,
                                                                    c->tc_bpack.as<float>(), colexp, (int)nm);
            prof_end(c, ABC_KERNEL_PACK, s);
            prof_begin(c, ABC_KERNEL_CONTRACTION, s);
            launch_gemm_tc<dev::TC_TF32>(c, pl, n_orb, out, conj, colexp, s, (int)nm, xep);
            c->launches += 1;
        }
        res.t = out;
        res.nsplit = pl.nsplit;
        res.stride = (long long)n * n_orb;
    } else {
        dim3 grid(c->n_tiles, (n_orb + 31) / 32);
        dev::gemm_blocks_simt<T, 32, 32, 16><<<grid, 256, 0, s>>>(c->bi, n_orb, c->geo.n_gamma, c->mat.as<V>(), xs,
                                                                  (V*)t, conj, c->tile_blk.as<int>(), c->tile_row.as<int>());
    }
    prof_end(c, ABC_KERNEL_CONTRACTION, s);
    return res;
}

// Back transform of a stage, reading t directly, adding split partials, or gathering it.
// hat_phi / hat_f: the stage's adapted inputs (nullptr: the context's first set).  With
// fn.hat_phi set (order 1), the kernel also forms the next stage's adapted inputs.
template <typename T, int MODE>
void back(abc_ctx* c, const TRes& tr, int n_orb, T s1, T a_coef, const void* y_f, void* out, void* acc, T cdt,
          cudaStream_t s, const void* hat_phi = nullptr, const void* hat_f = nullptr,
          dev::FwdNext<T> fn = dev::FwdNext<T>{}, bool nm = false) {
    typedef typename dev::C2<T>::t Vc;
    const dev::CellTab<T> ct = cell_tab<T>(c);
    const unsigned nbk = cell_blocks(c, n_orb);
    const Vc* hp = (const Vc*)(hat_phi ? hat_phi : c->hat_phi.p);
    const Vc* hf = (const Vc*)(hat_f ? hat_f : c->hat_f.p);
    constexpr bool can_fuse = MODE == 0 || MODE == 4;
    const bool fuse = can_fuse && fn.hat_phi != nullptr;
    if constexpr (sizeof(T) == 4) {
        if (tr.gathered) {
            if (fuse)
                dev::bnd_back<T, MODE, true, can_fuse><<<nbk, 128, 0, s>>>(
                    ct, n_orb, s1, a_coef, hp, hf, (const Vc*)nullptr, 1, 0LL, c->sym_gather, (const Vc*)y_f,
                    (Vc*)out, (Vc*)acc, cdt, fn);
            else
                dev::bnd_back<T, MODE, true><<<nbk, 128, 0, s>>>(ct, n_orb, s1, a_coef, hp, hf, (const Vc*)nullptr, 1,
                                                                 0LL, c->sym_gather, (const Vc*)y_f, (Vc*)out,
                                                                 (Vc*)acc, cdt, fn);
            return;
        }
    }
    if constexpr (sizeof(T) == 4 && MODE == 0) {
        if (nm && tr.xform && c->lanes >= 4) {   // x formed by the contraction epilogue
            if (c->lanes == 5)
                dev::bnd_back_quads_x<8><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    ct, n_orb, (const Vc*)tr.t, (const Vc*)y_f, (Vc*)out, cdt);
            else
                dev::bnd_back_quads_x<6><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    ct, n_orb, (const Vc*)tr.t, (const Vc*)y_f, (Vc*)out, cdt);
            return;
        }
        if (nm && tr.xform && c->lanes >= 2) {
            if (c->lanes == 3)
                dev::bnd_back_pairs_x<5><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    ct, n_orb, (const Vc*)tr.t, (const Vc*)y_f, (Vc*)out, cdt);
            else
                dev::bnd_back_pairs_x<4><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    ct, n_orb, (const Vc*)tr.t, (const Vc*)y_f, (Vc*)out, cdt);
            return;
        }
        if (nm && tr.xform) {
            dev::bnd_back_lanes_x<<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, dev::LANES_SMEM, s>>>(
                ct, n_orb, (const Vc*)tr.t, (const Vc*)y_f, (Vc*)out, cdt);
            return;
        }
        if (nm) {                            // node-major adapted vectors and t (lanes_ok)
            dev::bnd_back_lanes<<<(unsigned)(((long long)c->geo.n_cells * (n_orb / 32) + 3) / 4), 32 * dev::LANES_W,
                                  dev::LANES_SMEM, s>>>(
                ct, n_orb, s1, a_coef, hp, hf, (const Vc*)tr.t, tr.nsplit, tr.stride, (const Vc*)y_f, (Vc*)out, cdt);
            return;
        }
    }
    if (MODE == 0 && !fuse && c->back_multi == 1 && n_orb % 4 == 0) {
        dev::bnd_back_multi<T, 4><<<cell_blocks(c, n_orb / 4), 128, 0, s>>>(
            ct, n_orb, s1, a_coef, hp, hf, (const Vc*)tr.t, tr.nsplit, tr.stride, (const Vc*)y_f, (Vc*)out, cdt);
        return;
    }
    if (MODE == 0 && !fuse && c->back_multi == 2 && n_orb % 2 == 0) {
        dev::bnd_back_multi<T, 2><<<cell_blocks(c, n_orb / 2), 128, 0, s>>>(
            ct, n_orb, s1, a_coef, hp, hf, (const Vc*)tr.t, tr.nsplit, tr.stride, (const Vc*)y_f, (Vc*)out, cdt);
        return;
    }
    if (fuse)
        dev::bnd_back<T, MODE, false, can_fuse><<<nbk, 128, 0, s>>>(ct, n_orb, s1, a_coef, hp, hf, (const Vc*)tr.t,
                                                                    tr.nsplit, tr.stride, c->sym_gather,
                                                                    (const Vc*)y_f, (Vc*)out, (Vc*)acc, cdt, fn);
    else
        dev::bnd_back<T, MODE, false><<<nbk, 128, 0, s>>>(ct, n_orb, s1, a_coef, hp, hf, (const Vc*)tr.t, tr.nsplit,
                                                          tr.stride, c->sym_gather, (const Vc*)y_f, (Vc*)out,
                                                          (Vc*)acc, cdt, fn);
}

// One Horner stage: out = y + cdt * L(w).  For order >= 1 the interior part (stencil,
// which needs only w) and the boundary chain (which writes only the f part) are
// independent: the stencil runs on the side stream, forked from and joined back
// to s (inside a captured graph they become parallel branches).  The fork follows
// the contraction: its CTAs each need a whole SM (shared memory), so stencil blocks
// resident at its launch would hold back its start; forked after it, the stencil
// overlaps the back transform instead.
// The staged stencil form applies to radius 1, nx even and at most 256 (a tile row of
// pairs per thread), several orbitals and 16-byte aligned state arrays (bulk copies).
// The node-major order-1 chain (ABC_TUNE_LANES): complex64 on the tensor cores, the
// limit fit (diagonal A), n_orb a multiple of 32.
bool lanes_ok(const abc_ctx* c, int n_orb) {
    return c->lanes && c->lanes_attr && c->prec != ABC_FP64 && c->tc && c->params.order == 1 && !c->blocks.rows1 && n_orb % 32 == 0;
}

bool staged_ok(const abc_ctx* c, const void* w, const void* y, const void* o) {
    const Geometry& g = c->geo;
    const uintptr_t a = (uintptr_t)w | (uintptr_t)y | (uintptr_t)o;
    return g.R == 1 && (g.nx & 1) == 0 && g.nx <= 256 && c->staged_attr && (a & 15) == 0;
}

// g_in / g_out (complex64 stages with the Gamma copy, else NULL): the forward transform
// reads w on Gamma from g_in, and the stencil writes the stage output on Gamma to g_out.
template <typename T>
void stage(abc_ctx* c, int n_orb, T cdt, const void* w_phi, const void* w_f, const void* y_phi, const void* y_f,
           void* o_phi, void* o_f, const T* V, cudaStream_t s, int st = -1, const void* g_in = nullptr,
           void* g_out = nullptr) {
    typedef typename dev::C2<T>::t Vc;
    const Geometry& g = c->geo;
    const int order = c->params.order;
    const dev::CellTab<T> ct = cell_tab<T>(c);
    const unsigned nbk = cell_blocks(c, n_orb);
    auto stencil = [&](cudaStream_t ss) {
        prof_begin(c, ABC_KERNEL_STENCIL, ss);
        const Vc* bt = order >= 1 ? (const Vc*)w_f : c->cnat.as<Vc>();
        if (g.R == 3)
            dev::stencil_stage<T, 3><<<stencil_grid(c, n_orb), 256, 0, ss>>>(
                g.nx, g.ny, g.nz, n_orb, (T)(1.0 / (g.h * g.h)), (const Vc*)w_phi, (const Vc*)y_phi, V, bt,
                (Vc*)o_phi, cdt);
        else if (sizeof(T) == 4 && (g.nx & 1) == 0 && n_orb == 1) {
            // one orbital: also two planes per thread (half the blocks beside the back
            // transform, which runs at the same time)
            dim3 gp = stencil_grid(c, n_orb);
            gp.x = (unsigned)(((g.nx / 2) * g.ny + 255) / 256);
            gp.y = (gp.y + 1) / 2;
            dev::stencil_stage_x2z2<<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, (float)(1.0 / (g.h * g.h)),
                                                        (const float2*)w_phi, (const float2*)y_phi, (const float*)V,
                                                        (const float2*)bt, (float2*)o_phi, (float)cdt);
        } else if (sizeof(T) == 4 && c->stencil_staged && staged_ok(c, w_phi, y_phi, o_phi)) {
            // complex64: planes staged in shared memory by bulk copies, marching through z
            const dim3 gb((unsigned)((g.ny + dev::SB_TY - 1) / dev::SB_TY), (unsigned)((g.nz + dev::SB_KZ - 1) / dev::SB_KZ),
                          (unsigned)n_orb);
            dev::stencil_stage_x2_bulk<<<gb, (g.nx / 2) * dev::SB_TY, dev::stencil_bulk_smem(g.nx), ss>>>(
                g.nx, g.ny, g.nz, n_orb, (float)(1.0 / (g.h * g.h)), (const float2*)w_phi, (const float2*)y_phi,
                (const float*)V, (const float2*)bt, (float2*)o_phi, (float)cdt, (float2*)g_out, c->err_flag.as<int>());
        } else if (sizeof(T) == 4 && (g.nx & 1) == 0 && c->stencil_bps > 0 && ss != s) {
            // beside the boundary chain: a bounded number of blocks per SM, grid-stride
            dev::stencil_stage_x2_gs<<<(unsigned)(c->tc_sms_all * c->stencil_bps), 256, 0, ss>>>(
                g.nx, g.ny, g.nz, n_orb, (float)(1.0 / (g.h * g.h)), (const float2*)w_phi, (const float2*)y_phi,
                (const float*)V, (const float2*)bt, (float2*)o_phi, (float)cdt, (float2*)g_out);
        } else if (sizeof(T) == 4 && (g.nx & 1) == 0 && c->stencil_kz == 1) {
            // complex64, even rows: two nodes per thread, registers capped for 8 blocks per SM
            dim3 gp = stencil_grid(c, n_orb);
            gp.x = (unsigned)(((g.nx / 2) * g.ny + 255) / 256);
            dev::stencil_stage_x2_lb<8><<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, (float)(1.0 / (g.h * g.h)),
                                                            (const float2*)w_phi, (const float2*)y_phi,
                                                            (const float*)V, (const float2*)bt, (float2*)o_phi,
                                                            (float)cdt, (float2*)g_out);
        } else if (sizeof(T) == 4 && (g.nx & 1) == 0 && c->stencil_kz >= 2) {
            // complex64, even rows: two nodes per thread marching through KZ planes
            dim3 gp = stencil_grid(c, n_orb);
            gp.x = (unsigned)(((g.nx / 2) * g.ny + 255) / 256);
            gp.y = (unsigned)((g.nz + c->stencil_kz - 1) / c->stencil_kz);
            const float ih2 = (float)(1.0 / (g.h * g.h));
            const float2 *wp = (const float2*)w_phi, *yp = (const float2*)y_phi, *btp = (const float2*)bt;
            if (c->stencil_kz == 2)
                dev::stencil_stage_x2zk<2><<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, ih2, wp, yp, (const float*)V,
                                                               btp, (float2*)o_phi, (float)cdt, (float2*)g_out);
            else if (c->stencil_kz == 4)
                dev::stencil_stage_x2zk<4><<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, ih2, wp, yp, (const float*)V,
                                                               btp, (float2*)o_phi, (float)cdt, (float2*)g_out);
            else if (c->stencil_kz == 8)
                dev::stencil_stage_x2zk<8><<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, ih2, wp, yp, (const float*)V,
                                                               btp, (float2*)o_phi, (float)cdt, (float2*)g_out);
            else
                dev::stencil_stage_x2zk<16><<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, ih2, wp, yp,
                                                                (const float*)V, btp, (float2*)o_phi, (float)cdt,
                                                                (float2*)g_out);
        } else if (sizeof(T) == 4 && (g.nx & 1) == 0) {       // complex64, even rows: two nodes per thread
            dim3 gp = stencil_grid(c, n_orb);
            gp.x = (unsigned)(((g.nx / 2) * g.ny + 255) / 256);
            dev::stencil_stage_x2<<<gp, 256, 0, ss>>>(g.nx, g.ny, g.nz, n_orb, (float)(1.0 / (g.h * g.h)),
                                                      (const float2*)w_phi, (const float2*)y_phi, (const float*)V,
                                                      (const float2*)bt, (float2*)o_phi, (float)cdt, (float2*)g_out);
        } else
            dev::stencil_stage<T, 1><<<stencil_grid(c, n_orb), 256, 0, ss>>>(
                g.nx, g.ny, g.nz, n_orb, (T)(1.0 / (g.h * g.h)), (const Vc*)w_phi, (const Vc*)y_phi, V, bt,
                (Vc*)o_phi, cdt);
        prof_end(c, ABC_KERNEL_STENCIL, ss);
    };
    // where the stencil of an order >= 1 stage runs (ABC_TUNE_STENCIL): 0 forked after the
    // contraction, 1 forked at the stage start, 2 on the main stream after the back transform
    const int smode = c->stencil_mode;
    auto fork_stencil = [&]() {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        stencil(c->side);
    };
    auto stencil_at = [&](int point) {       // point 0: after the contraction, 1: stage start, 2: stage end
        if (point == 2 && smode == 2) stencil(s);
        if (point < 2 && point == smode) fork_stencil();
    };
    auto join = [&]() {
        if (smode == 2) return;
        cudaEventRecord(c->ev_join, c->side);
        cudaStreamWaitEvent(s, c->ev_join, 0);
    };
    const T a_coef = (T)(1.0 / (4.0 * g.h * g.h * g.h * g.h));
    if (order == 2) {
        stencil_at(1);
        // g' = B1 g + (B0 - i A1) f - i A1 E H w + A0 E w  (eq:dynamics2 with E phidot substituted)
        const dev::Ord2Fwd<T> o2{(const Vc*)w_f + (long long)g.n_gamma * n_orb, V, c->hat_h.as<Vc>(),
                                 c->hat_g.as<Vc>(), g.nx, g.ny, g.nz, (T)(1.0 / (g.h * g.h)), g.R};
        dev::bnd_forward<T, 2><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)w_phi, (const Vc*)w_f,
                                                   c->hat_phi.as<Vc>(), c->hat_f.as<Vc>(), nullptr, (T)0, o2);
        const void* x4[4] = {c->hat_g.p, c->hat_f.p, c->hat_h.p, c->hat_phi.p};
        const TRes tr = contraction<T>(c, nullptr, c->tvec.p, n_orb, 0, s, x4);
        stencil_at(0);
        back<T, 3>(c, tr, n_orb, (T)0, (T)0, y_f, o_f, const_cast<void*>(w_f), cdt, s);
        stencil_at(2);
        join();
        return;
    }
    // Order 1 inside a step (st = stage 0..3): the back transform of stages 0-2 also forms
    // the next stage's adapted inputs (two alternating sets), so stages 1-3 skip the
    // forward transform.
    const bool chain = st >= 0 && order == 1 && c->chain;
    const bool nm = sizeof(T) == 4 && lanes_ok(c, n_orb) && !chain;
    if (order >= 1) stencil_at(1);
    void* hp = chain && (st & 1) ? c->hat2_phi.p : c->hat_phi.p;
    void* hf = chain && (st & 1) ? c->hat2_f.p : c->hat_f.p;
    dev::FwdNext<T> fn{};
    if (chain && st < 3)
        fn = dev::FwdNext<T>{(const Vc*)w_phi, (const Vc*)y_phi, V, (const Vc*)w_f,
                             (Vc*)((st & 1) ? c->hat_phi.p : c->hat2_phi.p), (Vc*)((st & 1) ? c->hat_f.p : c->hat2_f.p),
                             g.nx, g.ny, g.nz, g.R, (T)(1.0 / (g.h * g.h)), c->nvox};
    if (!(chain && st > 0)) {
        // ahead of the one-orbital tiled contraction, the variant that lets it start early
        const bool early = n_orb == 1 && sizeof(T) == 4 && c->sym && !(order == 1 && c->blocks.rows1);
        if (early)
            dev::bnd_forward<T, 0, true><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)w_phi,
                                                             order == 1 ? (const Vc*)w_f : nullptr, (Vc*)hp, (Vc*)hf,
                                                             nullptr, (T)0, dev::Ord2Fwd<T>{});
        else if (nm && c->lanes >= 4) {
            if (c->lanes == 5)
                dev::bnd_forward_quads<8><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    cell_tab<float>(c), n_orb, c->nvox, (const float2*)w_phi, (const float2*)w_f, (float2*)hp,
                    (float2*)hf, (const float2*)g_in);
            else
                dev::bnd_forward_quads<6><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                    cell_tab<float>(c), n_orb, c->nvox, (const float2*)w_phi, (const float2*)w_f, (float2*)hp,
                    (float2*)hf, (const float2*)g_in);
        } else if (nm && c->lanes == 3)
            dev::bnd_forward_pairs<5><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                cell_tab<float>(c), n_orb, c->nvox, (const float2*)w_phi, (const float2*)w_f, (float2*)hp, (float2*)hf,
                (const float2*)g_in);
        else if (nm && c->lanes == 2)
            dev::bnd_forward_pairs<4><<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                cell_tab<float>(c), n_orb, c->nvox, (const float2*)w_phi, (const float2*)w_f, (float2*)hp, (float2*)hf,
                (const float2*)g_in);
        else if (nm)
            dev::bnd_forward_lanes<<<lanes_blocks(c, n_orb), 32 * dev::LANES_W, 0, s>>>(
                cell_tab<float>(c), n_orb, c->nvox, (const float2*)w_phi, (const float2*)w_f, (float2*)hp, (float2*)hf,
                (const float2*)g_in);
        else if (n_orb % dev::FO == 0 && c->fwd_rw)
            dev::bnd_forward_multi_rw<T><<<cell_blocks(c, n_orb / dev::FO), 128, 0, s>>>(
                ct, n_orb, c->nvox, (const Vc*)w_phi, order == 1 ? (const Vc*)w_f : nullptr, (Vc*)hp, (Vc*)hf,
                (const Vc*)g_in);
        else if (n_orb % dev::FO == 0)
            dev::bnd_forward_multi<T><<<cell_blocks(c, n_orb / dev::FO), 128, 0, s>>>(
                ct, n_orb, c->nvox, (const Vc*)w_phi, order == 1 ? (const Vc*)w_f : nullptr, (Vc*)hp, (Vc*)hf,
                (const Vc*)g_in);
        else
            dev::bnd_forward<T, 0><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)w_phi,
                                                       order == 1 ? (const Vc*)w_f : nullptr, (Vc*)hp, (Vc*)hf,
                                                       nullptr, (T)0, dev::Ord2Fwd<T>{});
    } else {
        c->launches -= 1;                    // the forward kernel counted by step_impl did not run
    }
    if (order == 1 && c->blocks.rows1) {
        // general B and A: t = B f_hat + A phi_hat on the rows [B | A], f' = t
        const void* x2[4] = {hf, hp, nullptr, nullptr};
        const TRes tr = contraction<T>(c, nullptr, c->tvec.p, n_orb, 0, s, x2);
        stencil_at(0);
        back<T, 4>(c, tr, n_orb, (T)0, (T)0, y_f, o_f, nullptr, cdt, s, hp, hf, fn);
        stencil_at(2);
        join();
        return;
    }
    const dev::XEpi xe{(const float2*)hf, (const float2*)hp, c->lanes_ac.as<float>(), (float)c->blocks.s};
    const TRes gathered = contraction<T>(c, order == 1 ? hf : hp, c->tvec.p, n_orb, 0, s, nullptr, nm,
                                         nm && order == 1 ? &xe : nullptr);
    if (order == 1) {
        stencil_at(0);
        back<T, 0>(c, gathered, n_orb, (T)c->blocks.s, a_coef, y_f, o_f, nullptr, cdt, s, hp, hf, fn, nm);
        stencil_at(2);
        join();
    } else {
        back<T, 1>(c, gathered, n_orb, (T)0, (T)0, nullptr, c->cnat.p, nullptr, (T)0, s);
        stencil(s);
    }
}

// The Gamma copy (ABC_TUNE_GAMMA_COPY): complex64, radius 1, nx even, orders 0 and 1,
// n_orb a multiple of 4 (the four-orbital forward transform), the stage-by-stage step.
// Each stage's stencil also writes its output on Gamma, in the natural boundary layout,
// to gam[(stage + 1) % 2]; the forward transform of the next stage reads it there
// instead of gathering single values from the whole state (a quarter or less of each
// 32-byte sector it fetches is Gamma).  The last stage writes gam[0], the next step's
// input; gamma_prime fills gam[0] from psi before the first step of a call.
bool gam_ok(const abc_ctx* c, int n_orb) {
    return c->gam_mode && c->prec != ABC_FP64 && c->geo.R == 1 && (c->geo.nx & 1) == 0 && c->params.order <= 1 &&
           n_orb >= 2 && n_orb % dev::FO == 0 && !c->chain && !(c->params.order == 1 && c->blocks.rows1) &&
           c->gam[0].p && c->gam[1].p;
}

int ensure_gam(abc_ctx* c) {
    if (!c->gam_mode || c->prec == ABC_FP64 || c->gam[0].p) return ABC_OK;
    if (c->geo.R != 1 || (c->geo.nx & 1) || c->params.order > 1 || c->params.max_orbitals < dev::FO) return ABC_OK;
    const size_t b = (size_t)c->geo.n_gamma * c->params.max_orbitals * cplx_bytes(c);
    int st;
    for (int i = 0; i < 2; ++i)
        if ((st = c->gam[i].alloc(b))) return st;
    return ABC_OK;
}

void gamma_prime(abc_ctx* c, const void* psi, int n_orb, cudaStream_t s) {
    const long long n = (long long)c->geo.n_cells * 64 * n_orb;
    dev::gamma_gather<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cell_tab<float>(c), n_orb, c->nvox,
                                                                         (const float2*)psi, c->gam[0].as<float2>());
    c->launches += 1;
}

// One time step (4 Horner stages) in place on (psi, aux); gam: the Gamma copy is in use
// (gam[0] holds psi on Gamma).
template <typename T>
void step_impl(abc_ctx* c, void* psi, void* aux, const void* V, int n_orb, double dt, const abc_meanfield* mf,
               cudaStream_t s, bool gam = false) {
    const T* Vuse = (const T*)V;
    if (mf) {
        dev::density_potential<T><<<nblk(c->nvox, 256), 256, 0, s>>>(
            c->nvox, n_orb, (const typename dev::C2<T>::t*)psi, (const T*)V, (T)mf->a, (T)mf->b, (T)mf->alpha,
            c->Veff.as<T>());
        Vuse = c->Veff.as<T>();
    }
    c->launches += 16 + (mf ? 1 : 0);
    const double cs[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    const void* in_p = psi;
    const void* in_f = aux;
    for (int st = 0; st < 4; ++st) {
        void* op = st == 3 ? psi : c->Tp[st & 1].p;
        void* of = st == 3 ? aux : c->Tf[st & 1].p;
        stage<T>(c, n_orb, (T)(cs[st] * dt), in_p, in_f, psi, aux, op, of, Vuse, s, st,
                 gam ? c->gam[st & 1].p : nullptr, gam ? c->gam[(st + 1) & 1].p : nullptr);
        in_p = op;
        in_f = of;
    }
}

// ---------------------------------------------------------------------------
// Order-1 step with the interior stencil fused in time (complex64, radius 1, nx even):
// stencil_bulk4 computes the four stages' interior in one pass beside the first
// boundary chain; stencil_band finishes the boundary band stage by stage after each
// contraction (see stencil_fused.cuh).  The result goes to `out` (not `in`: the bulk
// pass reads the input with a halo while it writes).
// ---------------------------------------------------------------------------
bool fused_ok(const abc_ctx* c, int n_orb) {
    if (c->prec == ABC_FP64 || c->params.order != 1 || c->geo.R != 1 || (c->geo.nx & 1)) return false;
    if (c->geo.nx < 8 || c->geo.ny < 8 || c->geo.nz < 8) return false;
    return c->fused_mode == 1 || (c->fused_mode == -1 && n_orb >= 2);
}

int ensure_fused_workspace(abc_ctx* c) {
    if (c->alt.p) return ABC_OK;
    const size_t phi_b = (size_t)c->nvox * c->params.max_orbitals * cplx_bytes(c);
    int st;
    if ((st = c->Tp3.alloc(phi_b))) return st;
    if ((st = c->alt.alloc(phi_b))) return st;
    for (int i = 0; i < 8; ++i)
        if (!c->ev_fz[i]) CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fz[i], cudaEventDisableTiming));
    CUDA_TRY(cudaFuncSetAttribute(dev::stencil_bulk4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::FB_SMEM));
    int sms = 0, per_sm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dev::stencil_bulk4, dev::FB_THREADS, dev::FB_SMEM));
    c->fused_grid = sms * std::max(per_sm, 1);
    return ABC_OK;
}

// The boundary part of an order-1 stage: forward transform of (w_phi, w_f), the
// contraction and the back transform writing o_f = y_f + cdt (B w_f + A E w_phi).
void boundary_chain_f(abc_ctx* c, int n_orb, float cdt, const void* w_phi, const void* w_f, const void* y_f, void* o_f,
                      cudaStream_t s) {
    typedef float2 Vc;
    const dev::CellTab<float> ct = cell_tab<float>(c);
    const unsigned nbk = cell_blocks(c, n_orb);
    const float a_coef = (float)(1.0 / (4.0 * c->geo.h * c->geo.h * c->geo.h * c->geo.h));
    void* hp = c->hat_phi.p;
    void* hf = c->hat_f.p;
    if (n_orb % dev::FO == 0 && c->fwd_rw)
        dev::bnd_forward_multi_rw<float><<<cell_blocks(c, n_orb / dev::FO), 128, 0, s>>>(
            ct, n_orb, c->nvox, (const Vc*)w_phi, (const Vc*)w_f, (Vc*)hp, (Vc*)hf, nullptr);
    else if (n_orb % dev::FO == 0)
        dev::bnd_forward_multi<float><<<cell_blocks(c, n_orb / dev::FO), 128, 0, s>>>(
            ct, n_orb, c->nvox, (const Vc*)w_phi, (const Vc*)w_f, (Vc*)hp, (Vc*)hf, nullptr);
    else
        dev::bnd_forward<float, 0><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)w_phi, (const Vc*)w_f, (Vc*)hp,
                                                       (Vc*)hf, nullptr, 0.f, dev::Ord2Fwd<float>{});
    if (c->blocks.rows1) {
        const void* x2[4] = {hf, hp, nullptr, nullptr};
        const TRes tr = contraction<float>(c, nullptr, c->tvec.p, n_orb, 0, s, x2);
        back<float, 4>(c, tr, n_orb, 0.f, 0.f, y_f, o_f, nullptr, cdt, s, hp, hf);
    } else {
        const TRes tr = contraction<float>(c, hf, c->tvec.p, n_orb, 0, s);
        back<float, 0>(c, tr, n_orb, (float)c->blocks.s, a_coef, y_f, o_f, nullptr, cdt, s, hp, hf);
    }
}

void step_fused(abc_ctx* c, const void* in, void* out, void* aux, const void* V, int n_orb, double dt,
                const abc_meanfield* mf, cudaStream_t s) {
    const Geometry& g = c->geo;
    const float* Vuse = (const float*)V;
    if (mf) {
        dev::density_potential<float><<<nblk(c->nvox, 256), 256, 0, s>>>(
            c->nvox, n_orb, (const float2*)in, (const float*)V, (float)mf->a, (float)mf->b, (float)mf->alpha,
            c->Veff.as<float>());
        Vuse = c->Veff.as<float>();
    }
    const double cs[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    const float ih2 = (float)(1.0 / (g.h * g.h));
    float2* U[4] = {nullptr, c->Tp[0].as<float2>(), c->Tp[1].as<float2>(), c->Tp3.as<float2>()};
    void* F[4] = {aux, c->Tf[0].p, c->Tf[1].p, c->Tf[0].p};           // f^0 .. f^3
    cudaStream_t side = c->side;
    // the bulk pass beside the first boundary chain
    cudaEventRecord(c->ev_fz[0], s);
    cudaStreamWaitEvent(side, c->ev_fz[0], 0);
    dev::FusedBulkArgs ba{};
    ba.nx = g.nx; ba.ny = g.ny; ba.nz = g.nz; ba.n_orb = n_orb; ba.n_gamma = g.n_gamma; ba.inv_h2 = ih2;
    for (int q = 0; q < 4; ++q) ba.cdt[q] = (float)(cs[q] * dt);
    ba.y = (const float2*)in; ba.V = Vuse; ba.f0 = (const float2*)aux; ba.out = (float2*)out;
    ba.u1 = U[1]; ba.u2 = U[2]; ba.u3 = U[3];
    prof_begin(c, ABC_KERNEL_STENCIL, side);
    dev::stencil_bulk4<<<c->fused_grid, dev::FB_THREADS, dev::FB_SMEM, side>>>(ba);
    prof_end(c, ABC_KERNEL_STENCIL, side);
    cudaEventRecord(c->ev_fz[1], side);
    int launches = 1 + (mf ? 1 : 0);
    // events: ev_fz[1] bulk done; ev_fz[2 + st] band of u^{st+2} done (side);
    // ev_fz[5 + st] f^{st+1} ready (main), st = 0, 1, 2
    for (int st = 0; st < 4; ++st) {
        const void* w_phi = st == 0 ? in : (const void*)U[st];
        void* o_f = st == 3 ? aux : c->Tf[st & 1].p;
        if (st > 0) cudaStreamWaitEvent(s, c->ev_fz[st], 0);   // u^st on Gamma (bulk, then bands)
        boundary_chain_f(c, n_orb, (float)(cs[st] * dt), w_phi, F[st], aux, o_f, s);
        launches += 3;
        if (st == 3) break;
        // the band of u^{st+2} (d <= st) once f^{st+1} is out
        cudaEventRecord(c->ev_fz[5 + st], s);
        cudaStreamWaitEvent(side, c->ev_fz[5 + st], 0);
        const int j = st + 2, dmax = st;
        const dim3 gb((unsigned)nblk(dev::band_nodes(g.nx, g.ny, g.nz, dmax), 256), (unsigned)n_orb);
        dev::stencil_band<<<gb, 256, 0, side>>>(g.nx, g.ny, g.nz, n_orb, dmax, ih2, U[j - 1], (const float2*)in, Vuse,
                                                (const float2*)F[j - 1], j == 4 ? (float2*)out : U[j],
                                                (float)(cs[j - 1] * dt));
        cudaEventRecord(c->ev_fz[2 + st], side);
        launches += 1;
    }
    cudaStreamWaitEvent(s, c->ev_fz[4], 0);     // the last band (u^4 on d <= 2)
    c->launches += launches;
}

template <typename T>
void diag_impl(abc_ctx* c, const void* psi, const void* aux, const void* V, int n_orb, const abc_meanfield* mf,
               double* out_dev, cudaStream_t s) {
    typedef typename dev::C2<T>::t Vc;
    const Geometry& g = c->geo;
    const T* Vuse = (const T*)V;
    if (mf) {
        // the energy column weighs each orbital with V_ext + e(rho), e(rho) = (a/2) rho +
        // b/(2+alpha) rho^(1+alpha): the interaction energy per unit density, so the
        // orbitals' energies sum to the mean-field functional whose rho-derivative is V
        dev::density_potential<T><<<nblk(c->nvox, 256), 256, 0, s>>>(
            c->nvox, n_orb, (const Vc*)psi, (const T*)V, (T)(0.5 * mf->a), (T)(mf->b / (2.0 + mf->alpha)),
            (T)mf->alpha, c->Veff.as<T>());
        Vuse = c->Veff.as<T>();
    }
    // W's auxiliary term f*Qf uses the diagonal Q of radius 1 (Thm 3.2); with R = 3, W = |phi|^2
    const bool waux = c->params.order == 1 && aux && g.R == 1;
    c->launches += 1 + (mf ? 1 : 0) + (waux ? 1 : 0);
    cudaMemsetAsync(out_dev, 0, sizeof(double) * 3 * n_orb, s);
    dim3 gp((unsigned)std::min<long long>(nblk(c->nvox, 256), 1024), n_orb);
    const T ih2 = (T)(1.0 / (g.h * g.h));
    if (g.R == 3) dev::diag_phi<T, 3><<<gp, 256, 0, s>>>(g.nx, g.ny, g.nz, n_orb, ih2, (const Vc*)psi, Vuse, out_dev);
    else dev::diag_phi<T, 1><<<gp, 256, 0, s>>>(g.nx, g.ny, g.nz, n_orb, ih2, (const Vc*)psi, Vuse, out_dev);
    if (waux) {
        dim3 ga((unsigned)std::min<long long>(nblk(g.n_gamma, 256), 256), n_orb);
        dev::diag_aux<T><<<ga, 256, 0, s>>>(g.n_gamma, n_orb, c->gamma_c.as<int>(), 4.0 * std::pow(g.h, 4),
                                            (const Vc*)aux, out_dev);
    }
}

// raw sums -> [norm, W, energy] with the h^3 weight
void finish_diag(const abc_ctx* c, double* v, long long rows) {
    const double w = c->geo.h * c->geo.h * c->geo.h;
    for (long long r = 0; r < rows; ++r) {
        double* d = v + 3 * r;
        const double nrm = w * d[0];
        d[1] = nrm + w * d[1];
        d[0] = nrm;
        d[2] = w * d[2];
    }
}

int check_run_args(abc_ctx* c, const void* psi, const void* aux, const void* V, int n_orb, double dt) {
    if (!c) return fail(ABC_ERR_ARG, "null context");
    if (!psi || !V) return fail(ABC_ERR_ARG, "null psi or V");
    if (c->params.order >= 1 && !aux) return fail(ABC_ERR_ARG, "orders 1 and 2 need the auxiliary buffer");
    if (n_orb < 1 || n_orb > c->params.max_orbitals) return fail(ABC_ERR_ARG, "n_orb outside [1, max_orbitals]");
    if (!(dt > 0.0)) return fail(ABC_ERR_ARG, "dt must be positive");
    return ABC_OK;
}

int last_launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ABC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ABC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" int abc_setup(const abc_grid* grid, const abc_params* params, abc_ctx** out) {
    if (!out) return fail(ABC_ERR_ARG, "null output pointer");
    *out = nullptr;
    int st = check_params(grid, params);
    if (st) return st;
    std::unique_ptr<abc_ctx> c(new abc_ctx());
    c->grid = *grid;
    c->params = *params;
    c->prec = params->precision;
    c->real_bytes = c->prec == ABC_FP64 ? 8 : 4;
    std::string err;
    st = build_geometry(grid->nx, grid->ny, grid->nz, grid->h, c->geo, err, grid->radius);
    if (st) return fail(st, err);
    c->nvox = c->geo.n_nodes;
    st = compute_param_blocks(c->geo, *params, c->blocks, err);
    if (st) return fail(st, err);
    CUDA_TRY(cudaGetDevice(&c->device));
    CUDA_TRY(cudaDeviceGetAttribute(&c->tc_sms_all, cudaDevAttrMultiProcessorCount, c->device));
    if ((st = upload_tables(c.get()))) return st;
    if ((st = upload_matrices(c.get()))) return st;
    if ((st = ensure_workspace(c.get()))) return st;
    if ((st = ensure_gam(c.get()))) return st;
    if ((st = c->diag.alloc(sizeof(double) * 3 * params->max_orbitals))) return st;
    if ((st = build_tiles(c.get()))) return st;
    // the packed symmetric tiles and the tensor-core image hold one symmetric m x m block
    // per class (order 0, order 1 with the limit fit); the order-2 rows
    // [B1 | B0 - i A1 | -i A1 | A0] and the fitted order-1 rows [B | A] use the
    // full-block kernels
    const bool one_seg = params->order < 2 && !c->blocks.rows1;
    const bool tc_prec = c->prec == ABC_C64_3XTF32 || c->prec == ABC_C64_SPLIT_FP16;
    if (one_seg && (c->prec == ABC_C64_FP32 || tc_prec) && (st = build_sym(c.get()))) return st;
    if (one_seg && tc_prec && (st = build_tc(c.get()))) return st;
    if (!c->err_flag.p) {
        if ((st = c->err_flag.alloc(sizeof(int)))) return st;
        CUDA_TRY(cudaMemset(c->err_flag.p, 0, sizeof(int)));
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    *out = c.release();
    return ABC_OK;
}

extern "C" int abc_boundary_size(const abc_ctx* ctx, long long* n_gamma) {
    if (!ctx || !n_gamma) return fail(ABC_ERR_ARG, "null argument");
    *n_gamma = ctx->geo.n_gamma;
    return ABC_OK;
}

extern "C" int abc_step(abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt, void* stream) {
    int st = check_run_args(ctx, psi, aux, V, n_orb, dt);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == ABC_FP64) step_impl<double>(ctx, psi, aux, V, n_orb, dt, nullptr, s);
    else {
        const bool gam = gam_ok(ctx, n_orb);
        if (gam) gamma_prime(ctx, psi, n_orb, s);
        step_impl<float>(ctx, psi, aux, V, n_orb, dt, nullptr, s, gam);
    }
    ctx->steps_done += 1;
    ctx->t_done += dt;
    return last_launch_status();
}

namespace {
int run_impl(abc_ctx* c, void* psi, void* aux, const void* V, int n_orb, double dt, long long nsteps,
             const abc_meanfield* mf, int diag_every, double* diag_out, cudaStream_t user) {
    if (nsteps < 0) return fail(ABC_ERR_ARG, "nsteps must be >= 0");
    if (diag_every < 0) return fail(ABC_ERR_ARG, "diag_every must be >= 0");
    if (diag_every > 0 && !diag_out) return fail(ABC_ERR_ARG, "diag_out is NULL");
    const long long ndiag = diag_every > 0 ? nsteps / diag_every : 0;
    if (ndiag >= INT_MAX) return fail(ABC_ERR_ARG, "too many diagnostic rows");
    // diagnostic rows: row 0 is the start state (the monitor's reference), row n the
    // state after n * diag_every steps; mon = {first failing row, its orbital}
    DevBuf dd, mon;
    int st;
    if (ndiag > 0 && (st = dd.alloc(sizeof(double) * 3 * n_orb * (ndiag + 1)))) return st;
    if (ndiag > 0 && (st = mon.alloc(2 * sizeof(int)))) return st;
    // work on a non-blocking stream ordered after the caller's stream
    cudaStream_t s = user ? user : c->own;
    if (!user) {
        CUDA_TRY(cudaEventRecord(c->ev_a, 0));
        CUDA_TRY(cudaStreamWaitEvent(s, c->ev_a, 0));
    }
    const bool fused = fused_ok(c, n_orb);
    if (fused && (st = ensure_fused_workspace(c))) return st;
    const bool gam = !fused && gam_ok(c, n_orb);
    // fused steps alternate between psi and the context's alternate buffer: step n (from
    // 1) reads psi and writes alt when n is odd, the reverse when n is even
    auto one_step = [&](cudaStream_t ss, int parity) {
        if (fused) {
            if (parity) step_fused(c, psi, c->alt.p, aux, V, n_orb, dt, mf, ss);
            else step_fused(c, c->alt.p, psi, aux, V, n_orb, dt, mf, ss);
        } else if (c->prec == ABC_FP64) step_impl<double>(c, psi, aux, V, n_orb, dt, mf, ss);
        else step_impl<float>(c, psi, aux, V, n_orb, dt, mf, ss, gam);
    };
    auto state_after = [&](long long n) -> const void* { return fused && (n & 1) ? c->alt.p : psi; };
    // divergence monitor (Thm 3.1 / Thm 3.2 give W as the quantity that may not grow):
    // proven for order 0 and for the order-1 limit fit at radius 1 (W^{n+1} <= W^n up to
    // a per-step slack for rounding), otherwise W may not pass twice its start value
    const bool proven = c->params.order == 0 ||
                        (c->params.order == 1 && c->params.fit1 == ABC_FIT1_LIMIT && c->geo.R == 1);
    const double slack = (c->prec == ABC_FP64 ? 1e-12 : 1e-6) * diag_every;
    auto one_diag = [&](long long row, cudaStream_t ss) {
        double* o = dd.as<double>() + row * 3 * n_orb;
        const void* cur = state_after(row * diag_every);
        if (c->prec == ABC_FP64) diag_impl<double>(c, cur, aux, V, n_orb, mf, o, ss);
        else diag_impl<float>(c, cur, aux, V, n_orb, mf, o, ss);
        if (row > 0) {
            dev::diag_monitor<<<1, 128, 0, ss>>>(dd.as<double>(), row, n_orb, proven ? 1 : 0, slack, mon.as<int>());
            c->launches += 1;
        }
    };
    if (ndiag > 0) {
        const int init[2] = {INT_MAX, -1};
        CUDA_TRY(cudaMemcpyAsync(mon.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
        one_diag(0, s);
    }
    const bool use_graph = !c->profiling && nsteps >= 1;
    if (use_graph) {
        abc_ctx::Key k;
        std::memset(&k, 0, sizeof(k));              // padding included: the key is compared bytewise
        k.psi = psi; k.aux = aux; k.V = V; k.n_orb = n_orb; k.dt = dt; k.mf = mf != nullptr;
        k.a = mf ? mf->a : 0; k.b = mf ? mf->b : 0; k.alpha = mf ? mf->alpha : 0; k.s = s; k.fused = fused ? 1 : 0;
        const bool same = c->gexec && !std::memcmp(&k, &c->key, sizeof(k));
        if (!same) {
            for (cudaGraphExec_t* ge : {&c->gexec, &c->gexec_b})
                if (*ge) { cudaGraphExecDestroy(*ge); *ge = nullptr; }
            for (int par = 1; par >= (fused ? 0 : 1); --par) {
                cudaGraph_t graph;
                CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                const long long before = c->launches;
                one_step(s, par);
                c->graph_kernels = c->launches - before;
                c->launches = before;
                cudaError_t le = cudaGetLastError();
                cudaError_t ce = cudaStreamEndCapture(s, &graph);
                if (le != cudaSuccess || ce != cudaSuccess)
                    return fail(ABC_ERR_CUDA,
                                std::string("graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
                cudaGraphExec_t* ge = par ? &c->gexec : &c->gexec_b;
                cudaError_t ie = cudaGraphInstantiate(ge, graph, 0);
                cudaGraphDestroy(graph);
                if (ie != cudaSuccess) {
                    *ge = nullptr;
                    return fail(ABC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
                }
            }
            c->key = k;
        }
    }
    if (gam && nsteps >= 1) gamma_prime(c, psi, n_orb, s);
    for (long long n = 1; n <= nsteps; ++n) {
        const int par = (int)(n & 1) | (fused ? 0 : 1);
        if (use_graph) {
            CUDA_TRY(cudaGraphLaunch(par ? c->gexec : c->gexec_b, s));
            c->launches += c->graph_kernels;
        } else {
            one_step(s, par);
        }
        if (diag_every > 0 && n % diag_every == 0) one_diag(n / diag_every, s);
    }
    if (fused && (nsteps & 1))                   // the result of an odd count is in alt
        CUDA_TRY(cudaMemcpyAsync(psi, c->alt.p, (size_t)c->nvox * n_orb * cplx_bytes(c), cudaMemcpyDeviceToDevice, s));
    st = last_launch_status();
    if (st) return st;
    c->steps_done += nsteps;
    c->t_done += (double)nsteps * dt;
    if (ndiag > 0) {
        int bad[2] = {INT_MAX, -1};
        CUDA_TRY(cudaMemcpyAsync(diag_out, dd.as<double>() + 3 * n_orb, sizeof(double) * 3 * n_orb * ndiag,
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(bad, mon.p, sizeof(bad), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        finish_diag(c, diag_out, ndiag * n_orb);
        if ((st = check_device_flag(c, s))) return st;
        if (bad[0] != INT_MAX) {
            const double* d = diag_out + ((long long)(bad[0] - 1) * n_orb + bad[1]) * 3;
            char msg[256];
            std::snprintf(msg, sizeof(msg),
                          "divergence monitor: W of orbital %d %s at step %lld of the run (W = %.6e)", bad[1],
                          proven ? "grew" : "passed twice its start value", (long long)bad[0] * diag_every, d[1]);
            return fail(ABC_ERR_UNSTABLE, msg);
        }
    }
    if (!user) {
        CUDA_TRY(cudaEventRecord(c->ev_b, s));
        CUDA_TRY(cudaStreamWaitEvent(0, c->ev_b, 0));
    }
    return ABC_OK;
}
}  // namespace

extern "C" int abc_run(abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt, long long nsteps,
                       const abc_meanfield* mf, int diag_every, double* diag_out, void* stream) {
    int st = check_run_args(ctx, psi, aux, V, n_orb, dt);
    if (st) return st;
    return run_impl(ctx, psi, aux, V, n_orb, dt, nsteps, mf, diag_every, diag_out, (cudaStream_t)stream);
}

namespace {
template <typename T>
int aux_init_impl(abc_ctx* c, const void* psi, void* aux, int n_orb, cudaStream_t s) {
    typedef typename dev::C2<T>::t Vc;
    const size_t ab = (size_t)c->geo.n_gamma * n_orb * sizeof(Vc);
    CUDA_TRY(cudaMemsetAsync(aux, 0, ab * (c->params.order == 2 ? 2 : 1), s));
    if (c->params.order != 2) return ABC_OK;
    // g(0) = A1 E psi: the contraction row [B1 | B0 - i A1 | -i A1 | A0] applied to
    // (0, 0, E psi, 0) gives -i A1 E psi; then g = i * that
    const dev::CellTab<T> ct = cell_tab<T>(c);
    const unsigned nbk = cell_blocks(c, n_orb);
    const size_t hb = (size_t)c->geo.n_gamma * n_orb * sizeof(Vc);
    CUDA_TRY(cudaMemsetAsync(c->hat_g.p, 0, hb, s));
    dev::bnd_forward<T, 0><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)psi, nullptr, c->hat_h.as<Vc>(),
                                               c->hat_f.as<Vc>(), nullptr, (T)0, dev::Ord2Fwd<T>{});
    const void* x4[4] = {c->hat_g.p, c->hat_g.p, c->hat_h.p, c->hat_g.p};
    const TRes tr = contraction<T>(c, nullptr, c->tvec.p, n_orb, 0, s, x4);
    back<T, 1>(c, tr, n_orb, (T)0, (T)0, nullptr, c->cnat.p, nullptr, (T)0, s);
    const long long n = (long long)c->geo.n_gamma * n_orb;
    dev::mul_i_into<T><<<nblk(n, 256), 256, 0, s>>>(n, c->cnat.as<Vc>(), (Vc*)aux + n);
    c->launches += 4;
    return last_launch_status();
}
}  // namespace

extern "C" int abc_aux_init(abc_ctx* ctx, const void* psi, void* aux, int n_orb, void* stream) {
    if (!ctx || !psi) return fail(ABC_ERR_ARG, "null context or psi");
    if (n_orb < 1 || n_orb > ctx->params.max_orbitals) return fail(ABC_ERR_ARG, "n_orb outside [1, max_orbitals]");
    if (ctx->params.order == 0) return ABC_OK;
    if (!aux) return fail(ABC_ERR_ARG, "null aux");
    cudaStream_t s = (cudaStream_t)stream;
    return ctx->prec == ABC_FP64 ? aux_init_impl<double>(ctx, psi, aux, n_orb, s)
                                 : aux_init_impl<float>(ctx, psi, aux, n_orb, s);
}

extern "C" int abc_run_host(abc_ctx* ctx, void* psi_host, void* aux_host, const void* V_host, int n_orb, double dt,
                            long long nsteps, const abc_meanfield* mf, int diag_every, double* diag_out) {
    int st = check_run_args(ctx, psi_host, aux_host, V_host, n_orb, dt);
    if (st) return st;
    const size_t cb = cplx_bytes(ctx);
    const size_t pb = (size_t)ctx->nvox * n_orb * cb,
                 ab = (size_t)ctx->geo.n_gamma * n_orb * cb * (ctx->params.order == 2 ? 2 : 1),
                 vb = (size_t)ctx->nvox * ctx->real_bytes;
    if (ctx->host_psi.bytes < pb && (st = ctx->host_psi.alloc(pb))) return st;
    if (ctx->host_aux.bytes < ab && (st = ctx->host_aux.alloc(ab))) return st;
    if (ctx->host_V.bytes < vb && (st = ctx->host_V.alloc(vb))) return st;
    cudaStream_t s = ctx->own;
    CUDA_TRY(cudaMemcpyAsync(ctx->host_psi.p, psi_host, pb, cudaMemcpyHostToDevice, s));
    if (ctx->params.order >= 1) CUDA_TRY(cudaMemcpyAsync(ctx->host_aux.p, aux_host, ab, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->host_V.p, V_host, vb, cudaMemcpyHostToDevice, s));
    st = run_impl(ctx, ctx->host_psi.p, ctx->params.order >= 1 ? ctx->host_aux.p : nullptr, ctx->host_V.p, n_orb, dt,
                  nsteps, mf, diag_every, diag_out, s);
    if (st) return st;
    CUDA_TRY(cudaMemcpyAsync(psi_host, ctx->host_psi.p, pb, cudaMemcpyDeviceToHost, s));
    if (ctx->params.order >= 1) CUDA_TRY(cudaMemcpyAsync(aux_host, ctx->host_aux.p, ab, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return check_device_flag(ctx, s);
}

extern "C" int abc_diagnostics(abc_ctx* ctx, const void* psi, const void* aux, const void* V, int n_orb,
                               const abc_meanfield* mf, double* out, void* stream) {
    int st = check_run_args(ctx, psi, aux, V, n_orb, 1.0);
    if (st) return st;
    if (!out) return fail(ABC_ERR_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == ABC_FP64) diag_impl<double>(ctx, psi, aux, V, n_orb, mf, ctx->diag.as<double>(), s);
    else diag_impl<float>(ctx, psi, aux, V, n_orb, mf, ctx->diag.as<double>(), s);
    if ((st = last_launch_status())) return st;
    CUDA_TRY(cudaMemcpyAsync(out, ctx->diag.p, sizeof(double) * 3 * n_orb, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    finish_diag(ctx, out, n_orb);
    return check_device_flag(ctx, s);
}

namespace {

// One adjoint stage: anew = cdt L^H a, acc += anew (both parts).
template <typename T>
void adj_stage(abc_ctx* c, int n_orb, T cdt, const void* a_phi, const void* a_f, void* acc_phi, void* acc_f,
               void* anew_phi, void* anew_f, const T* V, cudaStream_t s) {
    typedef typename dev::C2<T>::t Vc;
    const Geometry& g = c->geo;
    const T a_coef = (T)(1.0 / (4.0 * g.h * g.h * g.h * g.h));
    const dev::CellTab<T> ct = cell_tab<T>(c);
    const unsigned nbk = cell_blocks(c, n_orb);
    if (c->params.order == 1) {
        dev::bnd_forward<T, 1><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)a_phi, (const Vc*)a_f,
                                                   c->hat_phi.as<Vc>(), c->hat_f.as<Vc>(), c->cnat.as<Vc>(), a_coef,
                                                   dev::Ord2Fwd<T>{});
        const TRes gathered = contraction<T>(c, c->cnat.p, c->tvec.p, n_orb, 1, s);
        back<T, 2>(c, gathered, n_orb, (T)c->blocks.s, a_coef, nullptr, anew_f, acc_f, cdt, s);
    } else {
        dev::bnd_forward<T, 0><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)a_phi, nullptr, c->hat_phi.as<Vc>(),
                                                   c->hat_f.as<Vc>(), nullptr, (T)0, dev::Ord2Fwd<T>{});
        const TRes gathered = contraction<T>(c, c->hat_phi.p, c->tvec.p, n_orb, 1, s);
        back<T, 1>(c, gathered, n_orb, (T)0, (T)0, nullptr, c->cnat.p, nullptr, (T)0, s);
    }
    dev::stencil_adj<T><<<stencil_grid(c, n_orb), 256, 0, s>>>(
        c->params.order, g.nx, g.ny, g.nz, n_orb, (T)(1.0 / (g.h * g.h)), a_coef, (const Vc*)a_phi, V,
        c->params.order == 1 ? (const Vc*)a_f : c->cnat.as<Vc>(), (Vc*)acc_phi, (Vc*)anew_phi, cdt);
    c->launches += 4;
}

// Discrete adjoint of the Horner step.  With a the adjoint of a stage's output and w
// its input, a stage out = y + c dt L(w) sends c dt L^H a to w's adjoint and a to y's,
// and contributes c dt 2 Im(conj(a_phi) w_phi) to dJ/dV (dL/dV = -i on the phi part).
template <typename T>
int adjoint_impl(abc_ctx* c, const void* psi0, const void* V, int n_orb, double dt, long long nsteps, int K,
                 double* J_out, void* dJdV, cudaStream_t s) {
    typedef typename dev::C2<T>::t Vc;
    const size_t cb = sizeof(Vc);
    const bool o1 = c->params.order == 1;
    const size_t np = (size_t)c->nvox * n_orb, na = o1 ? (size_t)c->geo.n_gamma * n_orb : 0;
    const size_t sb = (np + na) * cb;
    const long long nck = nsteps / K;
    const long long segmax = std::min<long long>(K, std::max<long long>(nsteps, 1));
    DevBuf ck, seg, work, grad;
    int st;
    if ((st = ck.alloc((size_t)(nck + 1) * sb))) return st;
    if ((st = seg.alloc((size_t)segmax * sb))) return st;
    if ((st = work.alloc(7 * sb))) return st;
    if ((st = grad.alloc((size_t)c->nvox * sizeof(double)))) return st;
    auto S = [&](char* base, long long i) { return base + (size_t)i * sb; };
    auto PH = [&](char* b) { return (void*)b; };
    auto AF = [&](char* b) { return o1 ? (void*)(b + np * cb) : (void*)nullptr; };
    char* W = work.as<char>();
    char *Y = S(W, 0), *W4 = S(W, 1), *W3 = S(W, 2), *W2 = S(W, 3), *A = S(W, 4), *An = S(W, 5), *Acc = S(W, 6);
    const T* Vt = (const T*)V;
    // forward sweep, checkpoints every K steps
    CUDA_TRY(cudaMemcpyAsync(PH(Y), psi0, np * cb, cudaMemcpyDeviceToDevice, s));
    if (o1) CUDA_TRY(cudaMemsetAsync(AF(Y), 0, na * cb, s));
    CUDA_TRY(cudaMemcpyAsync(S(ck.as<char>(), 0), Y, sb, cudaMemcpyDeviceToDevice, s));
    for (long long n = 1; n <= nsteps; ++n) {
        step_impl<T>(c, PH(Y), AF(Y), V, n_orb, dt, nullptr, s);
        if (n % K == 0) CUDA_TRY(cudaMemcpyAsync(S(ck.as<char>(), n / K), Y, sb, cudaMemcpyDeviceToDevice, s));
    }
    // J and its adjoint
    diag_impl<T>(c, PH(Y), AF(Y), V, n_orb, nullptr, c->diag.as<double>(), s);
    std::vector<double> dg(3 * n_orb);
    CUDA_TRY(cudaMemcpyAsync(dg.data(), c->diag.p, sizeof(double) * 3 * n_orb, cudaMemcpyDeviceToHost, s));
    const double h3 = c->geo.h * c->geo.h * c->geo.h;
    dev::scale_into<T><<<nblk((long long)np, 256), 256, 0, s>>>((long long)np, (const Vc*)PH(Y), (T)(-h3), (Vc*)PH(A));
    if (o1) CUDA_TRY(cudaMemsetAsync(AF(A), 0, na * cb, s));
    CUDA_TRY(cudaMemsetAsync(grad.p, 0, (size_t)c->nvox * sizeof(double), s));
    const double cs[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    for (long long sg = (nsteps - 1) / K; nsteps > 0 && sg >= 0; --sg) {
        const long long start = sg * K, end = std::min<long long>(start + K, nsteps);
        char* SB = seg.as<char>();
        CUDA_TRY(cudaMemcpyAsync(S(SB, 0), S(ck.as<char>(), sg), sb, cudaMemcpyDeviceToDevice, s));
        for (long long k = 1; k < end - start; ++k) {
            CUDA_TRY(cudaMemcpyAsync(S(SB, k), S(SB, k - 1), sb, cudaMemcpyDeviceToDevice, s));
            step_impl<T>(c, PH(S(SB, k)), AF(S(SB, k)), V, n_orb, dt, nullptr, s);
        }
        for (long long n = end - 1; n >= start; --n) {
            char* y = S(SB, n - start);
            stage<T>(c, n_orb, (T)(cs[0] * dt), PH(y), AF(y), PH(y), AF(y), PH(W4), AF(W4), Vt, s);
            stage<T>(c, n_orb, (T)(cs[1] * dt), PH(W4), AF(W4), PH(y), AF(y), PH(W3), AF(W3), Vt, s);
            stage<T>(c, n_orb, (T)(cs[2] * dt), PH(W3), AF(W3), PH(y), AF(y), PH(W2), AF(W2), Vt, s);
            c->launches += 12;
            CUDA_TRY(cudaMemcpyAsync(Acc, A, sb, cudaMemcpyDeviceToDevice, s));
            char* ws[4] = {y, W4, W3, W2};
            for (int stg = 3; stg >= 0; --stg) {
                dev::grad_accum<T><<<nblk(c->nvox, 256), 256, 0, s>>>(c->nvox, n_orb, (const Vc*)PH(A),
                                                                      (const Vc*)PH(ws[stg]), cs[stg] * dt,
                                                                      grad.as<double>());
                adj_stage<T>(c, n_orb, (T)(cs[stg] * dt), PH(A), AF(A), PH(Acc), AF(Acc), PH(An), AF(An), Vt, s);
                c->launches += 1;
                std::swap(A, An);
            }
            std::swap(A, Acc);
        }
    }
    dev::to_real<T><<<nblk(c->nvox, 256), 256, 0, s>>>(c->nvox, grad.as<double>(), (T*)dJdV);
    if ((st = last_launch_status())) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    double J = 0;
    for (int j = 0; j < n_orb; ++j) J += 1.0 - h3 * dg[3 * j];
    *J_out = J;
    return check_device_flag(c, s);
}

}  // namespace

extern "C" int abc_adjoint_run(abc_ctx* ctx, const void* psi0, const void* V, int n_orb, double dt, long long nsteps,
                               int ckpt_every, double* J_out, void* dJdV, void* stream) {
    if (!ctx) return fail(ABC_ERR_ARG, "null context");
    if (!psi0 || !V) return fail(ABC_ERR_ARG, "null psi0 or V");
    if (n_orb < 1 || n_orb > ctx->params.max_orbitals) return fail(ABC_ERR_ARG, "n_orb outside [1, max_orbitals]");
    if (!(dt > 0.0)) return fail(ABC_ERR_ARG, "dt must be positive");
    if (!J_out || !dJdV) return fail(ABC_ERR_ARG, "null J_out or dJdV");
    if (nsteps < 0) return fail(ABC_ERR_ARG, "nsteps must be >= 0");
    if (ckpt_every < 1) return fail(ABC_ERR_ARG, "ckpt_every must be >= 1");
    if (ctx->params.order == 2) return fail(ABC_ERR_UNSUPPORTED, "the adjoint covers orders 0 and 1");
    if (ctx->params.fit1 != ABC_FIT1_LIMIT)
        return fail(ABC_ERR_UNSUPPORTED, "the adjoint covers the limit fit of order 1 (Thm 3.2) only");
    if (ctx->geo.R != 1) return fail(ABC_ERR_UNSUPPORTED, "the adjoint covers the radius-1 stencil only");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == ABC_FP64) return adjoint_impl<double>(ctx, psi0, V, n_orb, dt, nsteps, ckpt_every, J_out, dJdV, s);
    return adjoint_impl<float>(ctx, psi0, V, n_orb, dt, nsteps, ckpt_every, J_out, dJdV, s);
}

// ---------------------------------------------------------------------------
// Checkpoint / resume
// ---------------------------------------------------------------------------
namespace {
struct StateHeader {
    char magic[8];                   // "ABCSTATE"
    uint32_t version, header_bytes;
    int32_t nx, ny, nz, radius, order, precision, fit1, n_orb, n_gamma, reserved;
    double h, s, s1b, s2[4];
    int64_t steps_done;
    double t_done;
    uint64_t psi_bytes, aux_bytes, checksum;
};
const char kStateMagic[8] = {'A', 'B', 'C', 'S', 'T', 'A', 'T', 'E'};

uint64_t aux_bytes_of(const abc_ctx* c, int n_orb) {
    const uint64_t per = c->params.order == 2 ? 2 : c->params.order == 1 ? 1 : 0;
    return per * (uint64_t)c->geo.n_gamma * n_orb * cplx_bytes(c);
}

// 64-bit FNV-1a over 8-byte words, then the tail bytes.
uint64_t payload_hash(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        std::memcpy(&w, p + i, 8);
        h = (h ^ w) * 1099511628211ull;
    }
    for (; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
    return h;
}

StateHeader make_header(const abc_ctx* c, int n_orb) {
    StateHeader hd{};
    std::memcpy(hd.magic, kStateMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof(StateHeader);
    hd.nx = c->grid.nx; hd.ny = c->grid.ny; hd.nz = c->grid.nz; hd.radius = c->geo.R;
    hd.order = c->params.order; hd.precision = c->prec; hd.fit1 = c->params.fit1;
    hd.n_orb = n_orb; hd.n_gamma = c->geo.n_gamma;
    hd.h = c->grid.h; hd.s = c->blocks.s; hd.s1b = c->params.s1b;
    for (int q = 0; q < 4; ++q) hd.s2[q] = c->params.order == 2 ? c->params.s2[q] : 0.0;
    hd.psi_bytes = (uint64_t)c->nvox * n_orb * cplx_bytes(c);
    hd.aux_bytes = aux_bytes_of(c, n_orb);
    return hd;
}
}  // namespace

extern "C" int abc_state_size(const abc_ctx* ctx, int n_orb, size_t* bytes) {
    if (!ctx || !bytes) return fail(ABC_ERR_ARG, "null argument");
    if (n_orb < 1 || n_orb > ctx->params.max_orbitals) return fail(ABC_ERR_ARG, "n_orb outside [1, max_orbitals]");
    const StateHeader hd = make_header(ctx, n_orb);
    *bytes = sizeof(StateHeader) + hd.psi_bytes + hd.aux_bytes;
    return ABC_OK;
}

extern "C" int abc_get_state(const abc_ctx* ctx, const void* psi, const void* aux, int n_orb, void* host_dst,
                             size_t bytes, void* stream) {
    size_t need = 0;
    int st = abc_state_size(ctx, n_orb, &need);
    if (st) return st;
    if (!psi || !host_dst) return fail(ABC_ERR_ARG, "null psi or destination");
    if (ctx->params.order >= 1 && !aux) return fail(ABC_ERR_ARG, "orders 1 and 2 need the auxiliary buffer");
    if (bytes < need) return fail(ABC_ERR_ARG, "destination smaller than abc_state_size");
    StateHeader hd = make_header(ctx, n_orb);
    hd.steps_done = ctx->steps_done;
    hd.t_done = ctx->t_done;
    unsigned char* dst = static_cast<unsigned char*>(host_dst);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(dst + sizeof(hd), psi, hd.psi_bytes, cudaMemcpyDeviceToHost, s));
    if (hd.aux_bytes) CUDA_TRY(cudaMemcpyAsync(dst + sizeof(hd) + hd.psi_bytes, aux, hd.aux_bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    hd.checksum = payload_hash(dst + sizeof(hd), hd.psi_bytes + hd.aux_bytes);
    std::memcpy(dst, &hd, sizeof(hd));
    return ABC_OK;
}

extern "C" int abc_set_state(abc_ctx* ctx, void* psi, void* aux, int n_orb, const void* host_src, size_t bytes,
                             void* stream) {
    size_t need = 0;
    int st = abc_state_size(ctx, n_orb, &need);
    if (st) return st;
    if (!psi || !host_src) return fail(ABC_ERR_ARG, "null psi or source");
    if (ctx->params.order >= 1 && !aux) return fail(ABC_ERR_ARG, "orders 1 and 2 need the auxiliary buffer");
    if (bytes < sizeof(StateHeader)) return fail(ABC_ERR_ARG, "state blob shorter than its header");
    StateHeader hd;
    std::memcpy(&hd, host_src, sizeof(hd));
    const StateHeader want = make_header(ctx, n_orb);
    if (std::memcmp(hd.magic, kStateMagic, 8) || hd.version != 1 || hd.header_bytes != sizeof(StateHeader))
        return fail(ABC_ERR_ARG, "not a state blob of this library version");
    if (hd.nx != want.nx || hd.ny != want.ny || hd.nz != want.nz || hd.radius != want.radius || hd.h != want.h ||
        hd.order != want.order || hd.precision != want.precision || hd.fit1 != want.fit1 || hd.s != want.s ||
        hd.s1b != want.s1b || std::memcmp(hd.s2, want.s2, sizeof(hd.s2)) || hd.n_orb != want.n_orb ||
        hd.n_gamma != want.n_gamma ||
        hd.psi_bytes != want.psi_bytes || hd.aux_bytes != want.aux_bytes)
        return fail(ABC_ERR_ARG, "state blob was written by a context with another grid, ABC, precision or orbital count");
    if (bytes < need) return fail(ABC_ERR_ARG, "state blob truncated");
    const unsigned char* src = static_cast<const unsigned char*>(host_src);
    if (payload_hash(src + sizeof(hd), hd.psi_bytes + hd.aux_bytes) != hd.checksum)
        return fail(ABC_ERR_ARG, "state blob checksum mismatch (corrupted)");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(psi, src + sizeof(hd), hd.psi_bytes, cudaMemcpyHostToDevice, s));
    if (hd.aux_bytes) CUDA_TRY(cudaMemcpyAsync(aux, src + sizeof(hd) + hd.psi_bytes, hd.aux_bytes, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    ctx->steps_done = hd.steps_done;
    ctx->t_done = hd.t_done;
    return ABC_OK;
}

extern "C" int abc_progress(const abc_ctx* ctx, long long* steps, double* t) {
    if (!ctx || !steps || !t) return fail(ABC_ERR_ARG, "null argument");
    *steps = ctx->steps_done;
    *t = ctx->t_done;
    return ABC_OK;
}

extern "C" int abc_get_matrices(const abc_ctx* ctx, int which, void* host_dst, size_t bytes) {
    if (!ctx || !host_dst) return fail(ABC_ERR_ARG, "null argument");
    const size_t n = ctx->geo.n_gamma;
    if (bytes < 16 * n * n) return fail(ABC_ERR_ARG, "destination too small");
    std::string err;
    int st = dense_natural(ctx->geo, ctx->blocks, which, reinterpret_cast<cd*>(host_dst), err);
    if (st) return fail(st, err);
    return ABC_OK;
}

extern "C" int abc_profile_enable(abc_ctx* ctx, int enable) {
    if (!ctx) return fail(ABC_ERR_ARG, "null context");
    ctx->profiling = enable != 0;
    for (auto& p : ctx->prof) p.used = 0;
    return ABC_OK;
}

extern "C" int abc_profile_read(abc_ctx* ctx, int kernel, double* ms, long long* launches) {
    if (!ctx || !ms || !launches || kernel < 0 || kernel > 2) return fail(ABC_ERR_ARG, "bad argument");
    ProfileSlot& ps = ctx->prof[kernel];
    double tot = 0;
    for (size_t i = 0; i + 1 < ps.used; i += 2) {
        CUDA_TRY(cudaEventSynchronize(ps.ev[i + 1]));
        float t = 0;
        CUDA_TRY(cudaEventElapsedTime(&t, ps.ev[i], ps.ev[i + 1]));
        tot += t;
    }
    *ms = tot;
    *launches = (long long)(ps.used / 2);
    return ABC_OK;
}

extern "C" int abc_profile_durations(abc_ctx* ctx, int kernel, float* ms_out, long long max_out,
                                     long long* launches) {
    if (!ctx || !launches || kernel < 0 || kernel > 2 || max_out < 0 || (max_out > 0 && !ms_out))
        return fail(ABC_ERR_ARG, "bad argument");
    ProfileSlot& ps = ctx->prof[kernel];
    const long long n = (long long)(ps.used / 2);
    for (long long i = 0; i < n && i < max_out; ++i) {
        CUDA_TRY(cudaEventSynchronize(ps.ev[2 * i + 1]));
        CUDA_TRY(cudaEventElapsedTime(&ms_out[i], ps.ev[2 * i], ps.ev[2 * i + 1]));
    }
    *launches = n;
    return ABC_OK;
}

extern "C" int abc_kernel_bytes(const abc_ctx* ctx, int kernel, int n_orb, double* bytes) {
    if (!ctx || !bytes || n_orb < 1) return fail(ABC_ERR_ARG, "bad argument");
    const double cb = (double)cplx_bytes(ctx);
    if (kernel == ABC_KERNEL_CONTRACTION) {
        double entries = 0;
        if (ctx->sym && n_orb == 1) {
            entries = (double)ctx->sym_tiles_n * abc::dev::SYM_T * abc::dev::SYM_T;   // stored tiles, read once
        } else if (n_orb == 1) {
            for (int k = 0; k < ctx->ci.n; ++k)                                        // class blocks, read once
                entries += (double)ctx->bi.nseg * ctx->ci.m[k] * ctx->ci.m[k];
        } else if (ctx->tc && n_orb <= ctx->params.max_orbitals) {
            // tensor-core GEMM: the split planes of every class block once (4 planes of
            // 4-byte TF32), the packed right-hand sides (6 planes) and the partial outputs
            double a = 0, x = 0;
            for (int k = 0; k < ctx->ci.n; ++k) {
                a += (double)ctx->tci.m[k] * ctx->tci.m[k];
                x += (double)ctx->tci.R[k] * ctx->tci.m[k] * n_orb;
            }
            const int ns = ctx->tc_b[n_orb].nsplit;
            const double eb = ctx->tc_f16 ? 2.0 : 4.0;        // bytes per split-plane element
            // the node-major chain's epilogue forming x also reads f_hat and phi_hat
            const bool xf = lanes_ok(ctx, n_orb) && ns == 1;
            *bytes = a * (ctx->tc_cfg == 2 ? 6 : 4) * eb + x * 6 * eb + x * ns * 8 + (xf ? 2.0 * x * 8 : 0.0);
            return ABC_OK;
        } else {
            for (int p = 0; p < ctx->bi.n; ++p) entries += (double)ctx->bi.nseg * ctx->bi.m[p] * ctx->bi.m[p];
        }
        *bytes = entries * cb + 2.0 * ctx->geo.n_gamma * n_orb * cb;
    } else if (kernel == ABC_KERNEL_STENCIL) {
        if (fused_ok(ctx, n_orb))   // the time-fused pass: y in, u^4 out, V, and the band values it stores
            *bytes = (double)ctx->nvox * (2.0 * n_orb * cb + ctx->real_bytes) +
                     (double)n_orb * cb *
                         (dev::band_nodes(ctx->geo.nx, ctx->geo.ny, ctx->geo.nz, 1) +
                          (dev::band_nodes(ctx->geo.nx, ctx->geo.ny, ctx->geo.nz, 2) - ctx->geo.n_gamma) +
                          (dev::band_nodes(ctx->geo.nx, ctx->geo.ny, ctx->geo.nz, 3) -
                           dev::band_nodes(ctx->geo.nx, ctx->geo.ny, ctx->geo.nz, 1)));
        else    // w, y in, out, V; with the Gamma copy also the output on Gamma
            *bytes = (double)ctx->nvox * (3.0 * n_orb * cb + ctx->real_bytes) +
                     (gam_ok(ctx, n_orb) ? (double)ctx->geo.n_gamma * n_orb * cb : 0.0);
    } else {
        return fail(ABC_ERR_ARG, "unknown kernel");
    }
    return ABC_OK;
}

extern "C" int abc_kernel_flops(const abc_ctx* ctx, int kernel, int n_orb, double* useful, double* issued) {
    if (!ctx || !useful || !issued || n_orb < 1) return fail(ABC_ERR_ARG, "bad argument");
    if (kernel != ABC_KERNEL_CONTRACTION) return fail(ABC_ERR_ARG, "flops are reported for the contraction only");
    // complex multiply-add = 8 real flops per stored class-block entry and right-hand side
    double u = 0;
    for (int k = 0; k < ctx->ci.n; ++k) u += 8.0 * ctx->bi.nseg * ctx->ci.R[k] * (double)ctx->ci.m[k] * ctx->ci.m[k];
    *useful = u * n_orb;
    if (ctx->tc && n_orb > 1) {
        *issued = (ctx->tc_cfg == 2 ? 2.25 : 3.0) * *useful;       // three products per split term (x 3/4: Karatsuba)
    } else if (n_orb > 1) {
        // the CUDA-core GEMM multiplies every entry of the stored blocks (bi) by each
        // orbital's right-hand side
        double e = 0;
        for (int p = 0; p < ctx->bi.n; ++p) e += (double)ctx->bi.nseg * ctx->bi.m[p] * ctx->bi.m[p];
        *issued = 8.0 * e * n_orb;
    } else {
        *issued = *useful;
    }
    return ABC_OK;
}

namespace {
void drop_graphs(abc_ctx* ctx) {
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    if (ctx->gexec_b) { cudaGraphExecDestroy(ctx->gexec_b); ctx->gexec_b = nullptr; }
}
}  // namespace

extern "C" int abc_set_tuning(abc_ctx* ctx, int key, long long value) {
    if (!ctx) return fail(ABC_ERR_ARG, "null context");
    if (key == ABC_TUNE_L2_KEEP_TILES) {
        if (value < 0) return fail(ABC_ERR_ARG, "keep count must be >= 0");
        ctx->l2_keep_tiles = value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_PDL) {
        ctx->pdl = value != 0;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_CHAIN) {
        ctx->chain = value != 0;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_STENCIL) {
        if (value < 0 || value > 2) return fail(ABC_ERR_ARG, "stencil placement must be 0, 1 or 2");
        ctx->stencil_mode = (int)value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_GEMM_TILE || key == ABC_TUNE_GEMM_SPLIT) {
        if (key == ABC_TUNE_GEMM_TILE && (value < 0 || value > 2)) return fail(ABC_ERR_ARG, "GEMM tile must be 0, 1 or 2");
        if (key == ABC_TUNE_GEMM_SPLIT && (value < 0 || value > 8)) return fail(ABC_ERR_ARG, "GEMM split must be 0..8");
        drop_graphs(ctx);
        if (ctx->tc) CUDA_TRY(cudaDeviceSynchronize());   // the old work lists may be in use
        if (key == ABC_TUNE_GEMM_TILE) ctx->tc_cfg = (int)value;
        else ctx->tc_split = (int)value;
        if (!ctx->tc) return ABC_OK;
        int st;
        if (ctx->tc_cfg == 2 && !ctx->tc_apack_k.p && (st = pack_a_image(ctx, true))) return st;
        return build_tc_plans(ctx);
    }
    if (key == ABC_TUNE_FORWARD_RW) {
        ctx->fwd_rw = value != 0;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_GAMMA_COPY) {
        ctx->gam_mode = value != 0;
        drop_graphs(ctx);
        return ensure_gam(ctx);
    }
    if (key == ABC_TUNE_STENCIL_STAGED) {
        ctx->stencil_staged = value != 0;
        drop_graphs(ctx);
        if (ctx->stencil_staged && !ctx->staged_attr && ctx->geo.nx <= 256) {
            CUDA_TRY(cudaFuncSetAttribute(abc::dev::stencil_stage_x2_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)abc::dev::stencil_bulk_smem(ctx->geo.nx)));
            ctx->staged_attr = true;
        }
        return ABC_OK;
    }
    if (key == ABC_TUNE_LANES) {
        if (value < 0 || value > 5) return fail(ABC_ERR_ARG, "ABC_TUNE_LANES takes 0 .. 5");
        ctx->lanes = (int)value;
        drop_graphs(ctx);
        if (ctx->lanes && !ctx->lanes_attr) {
            CUDA_TRY(cudaFuncSetAttribute(abc::dev::bnd_back_lanes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)abc::dev::LANES_SMEM));
            CUDA_TRY(cudaFuncSetAttribute(abc::dev::bnd_back_lanes_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)abc::dev::LANES_SMEM));
            // a_coef c per adapted index for the contraction epilogue's x (the back
            // transform's a = a_coef * c, in the same float arithmetic)
            const Geometry& g = ctx->geo;
            const float af = (float)(1.0 / (4.0 * g.h * g.h * g.h * g.h));
            std::vector<float> ac((size_t)g.n_gamma, 0.f);
            for (int cell = 0; cell < g.n_cells; ++cell)
                for (int t = 0; t < 64; ++t) {
                    const int jj = g.cell_out[(size_t)cell * 64 + t];
                    if (jj >= 0) ac[(size_t)jj] = af * (float)g.cell_c[cell];
                }
            int st;
            if ((st = ctx->lanes_ac.alloc(ac.size() * sizeof(float)))) return st;
            CUDA_TRY(cudaMemcpy(ctx->lanes_ac.p, ac.data(), ac.size() * sizeof(float), cudaMemcpyHostToDevice));
            ctx->lanes_attr = true;
        }
        return ABC_OK;
    }
    if (key == ABC_TUNE_BACK_MULTI) {
        if (value < 0 || value > 2) return fail(ABC_ERR_ARG, "ABC_TUNE_BACK_MULTI takes 0, 1 or 2");
        ctx->back_multi = (int)value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_STENCIL_KZ) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(ABC_ERR_ARG, "stencil form must be 0, 1, 2, 4, 8 or 16");
        ctx->stencil_kz = (int)value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_STENCIL_BPS) {
        if (value < 0 || value > 8) return fail(ABC_ERR_ARG, "stencil blocks per SM must be 0..8");
        ctx->stencil_bps = (int)value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    if (key == ABC_TUNE_FUSED) {
        if (value < -1 || value > 1) return fail(ABC_ERR_ARG, "fused stencil must be -1 (auto), 0 or 1");
        ctx->fused_mode = (int)value;
        drop_graphs(ctx);
        return ABC_OK;
    }
    return fail(ABC_ERR_ARG, "unknown tuning key");
}

extern "C" int abc_get_tuning(const abc_ctx* ctx, int key, long long* value) {
    if (!ctx || !value) return fail(ABC_ERR_ARG, "null argument");
    if (key == ABC_TUNE_L2_KEEP_TILES) { *value = ctx->l2_keep_tiles; return ABC_OK; }
    if (key == ABC_TUNE_TILE_COUNT) { *value = ctx->sym ? ctx->sym_tiles_n : 0; return ABC_OK; }
    if (key == ABC_TUNE_PDL) { *value = ctx->pdl ? 1 : 0; return ABC_OK; }
    if (key == ABC_TUNE_CHAIN) { *value = ctx->chain ? 1 : 0; return ABC_OK; }
    if (key == ABC_TUNE_STENCIL) { *value = ctx->stencil_mode; return ABC_OK; }
    if (key == ABC_TUNE_FUSED) { *value = ctx->fused_mode; return ABC_OK; }
    if (key == ABC_TUNE_GEMM_TILE) { *value = ctx->tc_cfg; return ABC_OK; }
    if (key == ABC_TUNE_STENCIL_BPS) { *value = ctx->stencil_bps; return ABC_OK; }
    if (key == ABC_TUNE_STENCIL_KZ) { *value = ctx->stencil_kz; return ABC_OK; }
    if (key == ABC_TUNE_BACK_MULTI) { *value = ctx->back_multi; return ABC_OK; }
    if (key == ABC_TUNE_FORWARD_RW) { *value = ctx->fwd_rw ? 1 : 0; return ABC_OK; }
    if (key == ABC_TUNE_GAMMA_COPY) { *value = ctx->gam_mode ? 1 : 0; return ABC_OK; }
    if (key == ABC_TUNE_LANES) { *value = ctx->lanes; return ABC_OK; }
    if (key == ABC_TUNE_STENCIL_STAGED) { *value = ctx->stencil_staged ? 1 : 0; return ABC_OK; }
    if (key == ABC_TUNE_GEMM_SPLIT) { *value = ctx->tc_split; return ABC_OK; }
    return fail(ABC_ERR_ARG, "unknown tuning key");
}

extern "C" int abc_launch_count(const abc_ctx* ctx, long long* launches) {
    if (!ctx || !launches) return fail(ABC_ERR_ARG, "null argument");
    *launches = ctx->launches;
    return ABC_OK;
}

extern "C" void abc_destroy(abc_ctx* ctx) {
    if (!ctx) return;
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gexec_b) cudaGraphExecDestroy(ctx->gexec_b);
    for (auto e : ctx->ev_fz)
        if (e) cudaEventDestroy(e);
    for (auto& p : ctx->prof)
        for (auto e : p.ev) cudaEventDestroy(e);
    if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
    if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    delete ctx;
}

extern "C" int abc_wait_selftest(abc_ctx* ctx, long long polls, void* stream) {
    if (!ctx) return fail(ABC_ERR_ARG, "null context");
    if (polls < 1 || polls > (1LL << 24)) return fail(ABC_ERR_ARG, "polls must be in [1, 2^24]");
    if (!ctx->err_flag.p) return fail(ABC_ERR_ARG, "context has no device error flag");
    cudaStream_t s = (cudaStream_t)stream;
    wait_selftest_kernel<<<1, 32, 0, s>>>(polls, ctx->err_flag.as<int>());
    int st = last_launch_status();
    if (st) return st;
    return check_device_flag(ctx, s);
}
