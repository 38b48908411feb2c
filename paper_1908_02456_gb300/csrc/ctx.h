// Definition of the context behind the opaque abc_ctx handle (internal; shared
// by the .cu files of the library).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "sym_gemv.cuh"
#include "gemm_tc.cuh"

namespace abc {
int fail(int status, const std::string& msg);
}  // namespace abc

namespace abc {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t b) {
        if (p) { cudaFree(p); p = nullptr; bytes = 0; }
        if (b == 0) return ABC_OK;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) { p = nullptr; return fail(ABC_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
        bytes = b;
        return ABC_OK;
    }
    template <typename X> X* as() const { return reinterpret_cast<X*>(p); }
};

struct ProfileSlot {
    std::vector<cudaEvent_t> ev;   // pairs
    size_t used = 0;
};

}  // namespace abc

struct abc_ctx {
    abc_grid grid;
    abc_params params;
    abc::Geometry geo;
    abc::Blocks blocks;          // FP64 blocks (kept for abc_get_matrices)
    int device = 0;
    int prec = 0;
    size_t real_bytes = 8;  // bytes of one real value of the state
    long long nvox = 0;
    abc::dev::BlockInfo bi;
    abc::dev::ClassInfo ci;           // the same blocks by class (one-orbital contraction)
    // device tables
    abc::DevBuf gamma_c;
    abc::DevBuf cell_out, cell_type, cell_coef_f, cell_coef_bt, cell_c, cell_gi, cell_node, cell_wr;
                                                              // boundary transform tables
    abc::DevBuf mat;             // irreducible-class blocks in device format
    abc::DevBuf tile_blk, tile_row;   // row tiles (block, first row) of the multi-orbital contraction
    int n_tiles = 0;
    // workspace
    abc::DevBuf Tp[2], Tf[2], hat_phi, hat_f, hat2_phi, hat2_f, hat_h, hat_g, tvec, cnat, Veff, diag;
    abc::DevBuf host_psi, host_aux, host_V;   // device copies for abc_run_host
    cudaStream_t own = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // order 1: the stencil of a stage runs on `side`, concurrently with the boundary chain
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // order-1 steps with the interior stencil fused in time (stencil_fused.cuh): the
    // third stage buffer, the alternate state buffer of abc_run, events, grid
    int fused_mode = 0;              // ABC_TUNE_FUSED: 0 off (default), 1 on, -1 on for n_orb >= 2
    abc::DevBuf Tp3, alt;
    cudaEvent_t ev_fz[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int fused_grid = 0;
    // graph cache (gexec_b: the second graph of a fused run, alt -> psi)
    cudaGraphExec_t gexec = nullptr, gexec_b = nullptr;
    struct Key { const void *psi, *aux, *V; int n_orb; double dt; int mf; double a, b, alpha; cudaStream_t s; int fused; } key{};
    // one-orbital complex64 contraction on symmetric packed tiles
    bool sym = false;
    abc::dev::SymInfo si{};
    int sym_grid = 0;
    long long sym_tiles_n = 0;
    long long l2_keep_tiles = 0;     // tiles streamed with evict_last (tuning)
    bool pdl = true;                 // the contraction is a programmatic dependent of the forward transform (tuning)
    bool chain = false;              // order-1 back transforms form the next stage's adapted inputs (tuning)
    int stencil_mode = 0;            // where the stencil runs in a stage (tuning, ABC_TUNE_STENCIL)
    int stencil_bps = 0;             // side-stream stencil: blocks per SM of a grid-stride grid (0: one per pair)
    int stencil_kz = 1;              // complex64 stencil form (ABC_TUNE_STENCIL_KZ): 1 capped registers (default)
    bool stencil_staged = false;     // complex64 stencil with planes staged by bulk copies (ABC_TUNE_STENCIL_STAGED)
    bool staged_attr = false;        // its shared-memory size attribute has been set
    int back_multi = 0;              // order-1 back transform: 0 one orbital per cell group, 1 four, 2 two (tuning)
    bool fwd_rw = false;             // four-orbital forward transform with the reflection transform in registers
    bool gam_mode = false;           // stencils write the next stage's w on Gamma for the forward transform (tuning)
    int lanes = 0;                   // order-1 tensor-core chain with node-major adapted vectors (tuning):
                                     // 1 warp per cell and 32 orbitals, 2 / 3 cell split between lane
                                     // pairs (registers for 4 / 5 blocks per SM), 4 / 5 between four
                                     // lanes (6 / 8 blocks per SM)
    bool lanes_attr = false;         // bnd_back_lanes's shared-memory size set, lanes_ac filled
    abc::DevBuf lanes_ac;            // [n_gamma] a_coef * c per adapted index (node-major chain)
    abc::DevBuf tc_colmax;           // tc_colexp_nm: column maxima [tc_ncols * max_orbitals], then counters
    abc::DevBuf gam[2];              // that Gamma copy, [n_gamma][max_orbitals], one per stage parity
    int tc_sms_all = 0;              // SMs of the device
    abc::DevBuf sym_tiles, sym_seg, sym_cta, sym_rowseg, sym_rowpart, sym_colpart, sym_gdesc, err_flag;
    abc::dev::SymGather sym_gather{};   // partial-sum view for the back transform
    // many-orbital complex64 contraction on the tensor cores (ABC_C64_3XTF32)
    bool tc = false;
    abc::dev::TcInfo tci{};
    abc::DevBuf tc_apack, tc_tiles, tc_cols, tc_bpack, tc_part;
    bool tc_f16 = false;             // ABC_C64_SPLIT_FP16: kind::f16 operands with power-of-two scales
    int tc_cfg = 0;                  // GEMM form (ABC_TUNE_GEMM_TILE): 0 96 columns x 1 CTA/SM, 1 64 x 2, 2 Karatsuba
    long long tc_chunks = 0;         // (128-row tile, K block) chunks of the A image
    abc::DevBuf tc_apack_k;          // the Karatsuba form's A image (built when first selected)
    int tc_split = 0;                // GEMM K splits: 0 = about two items per CTA slot
    int tc_ncols = 0;                // right-hand sides over all classes (column scales per orbital)
    abc::DevBuf tc_colexp;           // TC_F16: per-column scale exponents of the current contraction
    struct TcPlan {
        int tile_off = 0, tile_cnt = 0, cols_off = 0, cols_cnt = 0, max_nkb = 1, nsplit = 1;
        int grid = 0, off_base = 0;     // CTAs of the persistent GEMM and their item offsets in tc_item_off
    };
    abc::DevBuf tc_items, tc_item_off;
    std::vector<TcPlan> tc_b;                    // launch plan of each orbital count b (index b)
    int tc_sms = 0;
    // progress of the state the context last advanced (steps and time), kept by
    // abc_step / abc_run and restored by abc_set_state
    long long steps_done = 0;
    double t_done = 0.0;
    // launch accounting
    long long launches = 0;
    long long graph_kernels = 0;
    // profiling
    bool profiling = false;
    abc::ProfileSlot prof[3];
};

namespace abc {
// Kernel view of the context's boundary transform tables.
template <typename T>
inline dev::CellTab<T> cell_tab(const abc_ctx* c) {
    dev::CellTab<T> t;
    t.n_cells = c->geo.n_cells;
    t.ng = c->geo.n_gamma;
    t.n_gamma = c->geo.n_gamma;
    t.out = c->cell_out.as<int>();
    t.type = c->cell_type.as<int>();
    t.coef_f = c->cell_coef_f.as<T>();
    t.coef_bt = c->cell_coef_bt.as<T>();
    t.cell_c = c->cell_c.as<int>();
    t.gi = c->cell_gi.as<int>();
    t.node = c->cell_node.as<int>();
    t.wr = c->cell_wr.as<int>();
    return t;
}
// Blocks (of 128 threads) of the boundary transforms for n_orb orbitals.
inline unsigned cell_blocks(const abc_ctx* c, int n_orb) {
    return (unsigned)(((long long)c->geo.n_cells * n_orb + 1) / 2);
}
// Blocks of the lane-per-orbital transforms (one warp per cell and 32 orbitals, four
// warps per block; n_orb a multiple of 32).
inline unsigned lanes_blocks(const abc_ctx* c, int n_orb) {
    const int per = c->lanes >= 4 ? 8 : c->lanes >= 2 ? 16 : 32;   // orbitals per warp
    return (unsigned)(((long long)c->geo.n_cells * (n_orb / per) + 3) / 4);
}
}  // namespace abc

namespace abc {
// Grid of the stencil kernels (256 threads per block): x over a z-plane, y = z, z = orbital.
inline dim3 stencil_grid(const abc_ctx* c, int n_orb) {
    return dim3((unsigned)((c->geo.nx * c->geo.ny + 255) / 256), (unsigned)c->geo.nz, (unsigned)n_orb);
}
}  // namespace abc
