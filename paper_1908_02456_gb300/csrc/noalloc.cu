// abc_step_noalloc: one time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they step the system: code that runs
// inside a host framework which owns the whole device heap (a pool allocator that
// must not be bypassed), or that runs where an allocation could block or fail at a
// point the caller cannot handle (for example, while other work on the device has
// already reserved all free memory).  For them this entry point takes the step's
// per-stage scratch -- the two Horner stage buffers, the auxiliary-variable stage
// buffers and the boundary vectors in the parity-adapted basis -- from one array
// of static device memory defined in this file, instead of from the context's
// workspace or from any allocation.
//
// The array has a fixed size (ABC_NOALLOC_SCRATCH_BYTES, 16 MiB).  Every GPU that
// loads the library holds it until the process exits.  All calls share it, so two
// calls whose work overlaps on the GPU (on different streams, or on different
// contexts of the same device) race on it and give wrong results; serialise them.
// Each call fully overwrites every scratch element it reads before reading it, so
// nothing needs to be cleared between calls.
//
// Host code cannot use the array's name as a device address (on the host the
// symbol is only a stand-in).  Every call made outside stream capture therefore
// looks the address up with cudaGetSymbolAddress, with the context's device
// current, so the address always belongs to the device's current primary context
// (it changes after a cudaDeviceReset).  A call made while its stream is being
// captured cannot make that runtime call and uses the address the last uncaptured
// call on the device found; make at least one call on each device before any
// stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ctx.h"

namespace {

constexpr size_t kScratchBytes = ABC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_for_device(int dev, cudaStream_t s, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return abc::fail(ABC_ERR_ARG, "device ordinal out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return abc::fail(ABC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return abc::fail(ABC_ERR_ARG, "abc_step_noalloc: first call on this device made during stream capture "
                                      "(make one call outside capture first)");
    }
    *out = g_scratch_ptr[dev];
    return ABC_OK;
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// The stages of abc_step on scratch from the static array.  The one-orbital
// contraction uses the full-block kernel (no partial-sum scratch), so for complex64
// the summation order differs from abc_step's symmetric-tile kernel.
template <typename T>
void step_with_scratch(const abc_ctx* c, void* psi, void* aux, const void* V, int n_orb, double dt, char* scratch,
                       cudaStream_t s) {
    typedef typename abc::dev::C2<T>::t Vc;
    const abc::Geometry& g = c->geo;
    const size_t phi_n = (size_t)c->nvox * n_orb, aux_n = (size_t)g.n_gamma * n_orb;
    Vc* base = reinterpret_cast<Vc*>(scratch);
    Vc* Tp[2] = {base, base + phi_n};
    Vc* Tf[2] = {base + 2 * phi_n, base + 2 * phi_n + aux_n};
    Vc* hat_phi = base + 2 * phi_n + 2 * aux_n;
    Vc* hat_f = hat_phi + aux_n;
    Vc* tvec = hat_f + aux_n;
    Vc* cnat = tvec + aux_n;
    const int order = c->params.order;
    const abc::dev::CellTab<T> ct = abc::cell_tab<T>(c);
    const unsigned nbk = abc::cell_blocks(c, n_orb);
    const double cs[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    const void* in_p = psi;
    const void* in_f = aux;
    for (int st = 0; st < 4; ++st) {
        void* op = st == 3 ? psi : (void*)Tp[st & 1];
        void* of = st == 3 ? aux : (void*)Tf[st & 1];
        const T cdt = (T)(cs[st] * dt);
        abc::dev::bnd_forward<T, 0><<<nbk, 128, 0, s>>>(ct, n_orb, c->nvox, (const Vc*)in_p,
                                                        order == 1 ? (const Vc*)in_f : nullptr, hat_phi, hat_f,
                                                        nullptr, (T)0, abc::dev::Ord2Fwd<T>{});
        const Vc* x = order == 1 ? hat_f : hat_phi;
        if (n_orb == 1) {
            abc::dev::gemv_blocks<T><<<nblk((long long)g.n_gamma * 32, 256), 256, 0, s>>>(
                c->bi, g.n_gamma, c->mat.as<Vc>(), abc::dev::XSeg<Vc>{{x, nullptr, nullptr, nullptr}}, tvec, 0);
        } else {
            dim3 grid(c->n_tiles, (n_orb + 31) / 32);
            abc::dev::gemm_blocks_simt<T, 32, 32, 16><<<grid, 256, 0, s>>>(
                c->bi, n_orb, g.n_gamma, c->mat.as<Vc>(), abc::dev::XSeg<Vc>{{x, nullptr, nullptr, nullptr}}, tvec, 0,
                c->tile_blk.as<int>(), c->tile_row.as<int>());
        }
        const T a_coef = (T)(1.0 / (4.0 * g.h * g.h * g.h * g.h));
        if (order == 1)
            abc::dev::bnd_back<T, 0, false><<<nbk, 128, 0, s>>>(ct, n_orb, (T)c->blocks.s, a_coef, hat_phi, hat_f, tvec,
                                                                1, 0, c->sym_gather, (const Vc*)aux, (Vc*)of, nullptr,
                                                                cdt, abc::dev::FwdNext<T>{});
        else
            abc::dev::bnd_back<T, 1, false><<<nbk, 128, 0, s>>>(ct, n_orb, (T)0, (T)0, hat_phi, hat_f, tvec, 1, 0,
                                                                c->sym_gather, nullptr, cnat, nullptr, (T)0,
                                                                abc::dev::FwdNext<T>{});
        abc::dev::stencil_stage<T><<<abc::stencil_grid(c, n_orb), 256, 0, s>>>(
            g.nx, g.ny, g.nz, n_orb, (T)(1.0 / (g.h * g.h)), (const Vc*)in_p, (const Vc*)psi, (const T*)V,
            order == 1 ? (const Vc*)in_f : cnat, (Vc*)op, cdt);
        in_p = op;
        in_f = of;
    }
}

}  // namespace

extern "C" int abc_step_noalloc(const abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt,
                                void* stream) {
    if (!ctx) return abc::fail(ABC_ERR_ARG, "null context");
    if (!psi || !V) return abc::fail(ABC_ERR_ARG, "null psi or V");
    if (ctx->params.order == 1 && !aux) return abc::fail(ABC_ERR_ARG, "order 1 needs the auxiliary buffer");
    if (n_orb < 1 || n_orb > ctx->params.max_orbitals) return abc::fail(ABC_ERR_ARG, "n_orb outside [1, max_orbitals]");
    if (!(dt > 0.0)) return abc::fail(ABC_ERR_ARG, "dt must be positive");
    if (ctx->params.order == 2) return abc::fail(ABC_ERR_UNSUPPORTED, "abc_step_noalloc covers orders 0 and 1");
    if (ctx->params.fit1 != ABC_FIT1_LIMIT)
        return abc::fail(ABC_ERR_UNSUPPORTED, "abc_step_noalloc covers the limit fit of order 1 only");
    if (ctx->geo.R != 1) return abc::fail(ABC_ERR_UNSUPPORTED, "abc_step_noalloc covers the radius-1 stencil only");
    if (ctx->prec != ABC_FP64 && ctx->prec != ABC_C64_FP32)
        return abc::fail(ABC_ERR_UNSUPPORTED, "abc_step_noalloc covers the ABC_FP64 and ABC_C64_FP32 forms");
    const size_t cb = 2 * ctx->real_bytes;
    const size_t need = (2 * (size_t)ctx->nvox * n_orb + 6 * (size_t)ctx->geo.n_gamma * n_orb) * cb;
    if (need > kScratchBytes)
        return abc::fail(ABC_ERR_ARG, "abc_step_noalloc: this grid and orbital count need " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes) +
                                          " (use abc_step)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != ctx->device) return abc::fail(ABC_ERR_ARG, "the context belongs to another device");
    void* scratch = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    int st = scratch_for_device(dev, s, &scratch);
    if (st) return st;
    if (ctx->prec == ABC_FP64) step_with_scratch<double>(ctx, psi, aux, V, n_orb, dt, (char*)scratch, s);
    else step_with_scratch<float>(ctx, psi, aux, V, n_orb, dt, (char*)scratch, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ABC_OK;
}
