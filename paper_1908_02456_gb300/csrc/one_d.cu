// The one-dimensional time-stepper of Sec. 4.1 on the GPU (abc1d.h).
//
// A 1D box of the paper's experiment has ~1500 nodes: too small to fill a GPU with one
// kernel per stage, so the whole run is one launch of one thread block.  The step-start
// state y and the two stage buffers live in shared memory (three arrays of n complex
// values), the boundary variables in a few shared words; every Horner stage is one
// sweep of the five-point stencil over the nodes plus the 2 x 2 boundary blocks of
// each end applied by the first threads, with a block barrier between stages.
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "one_d.h"

namespace abc {
int fail(int status, const std::string& msg);
}

struct abc1d_ctx {
    abc1d_params p;
    abc::oned::Blocks1D blk;
    int device = 0;
};

namespace {

template <typename T>
struct Cx {
    T x, y;
};
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
    return Cx<T>{a.x + b.x, a.y + b.y};
}

enum { MM = 0, MA = 1, MB = 2, MB1 = 3, MB0 = 4, MA1 = 5, MA0 = 6, NMAT = 7 };

template <typename T>
struct OneDArgs {
    int n, order;
    T cw[3];                    // -c_m / (2 h^2), m = 0, 1, 2 (H's weights)
    Cx<T> mat[NMAT][2][2];      // the left end's blocks
    Cx<T>* psi;
    Cx<T>* aux;
    long long nsteps;
    T dt;
    double h;
    int diag_every;
    double* diag;
};

// Block of the matrix `m` seen from Gamma index g (0..3) towards Gamma index j of the
// same end: the left end uses the stored block, the right end its mirror image.
template <typename T>
__device__ __forceinline__ Cx<T> blk(const OneDArgs<T>& a, int m, int g, int j) {
    return g < 2 ? a.mat[m][g][j] : a.mat[m][1 - (g - 2)][1 - (j - 2)];
}

template <typename T>
__device__ __forceinline__ int gnode(int g, int n) {
    return g < 2 ? g : n - 4 + g;                // Gamma order [0, 1, n - 2, n - 1]
}

// (H w)_i, the neighbours outside the box omitted.
template <typename T>
__device__ __forceinline__ Cx<T> apply_h1(const OneDArgs<T>& a, const Cx<T>* w, int i) {
    Cx<T> acc{a.cw[0] * w[i].x, a.cw[0] * w[i].y};
    if (i >= 1) { acc.x += a.cw[1] * w[i - 1].x; acc.y += a.cw[1] * w[i - 1].y; }
    if (i + 1 < a.n) { acc.x += a.cw[1] * w[i + 1].x; acc.y += a.cw[1] * w[i + 1].y; }
    if (i >= 2) { acc.x += a.cw[2] * w[i - 2].x; acc.y += a.cw[2] * w[i - 2].y; }
    if (i + 2 < a.n) { acc.x += a.cw[2] * w[i + 2].x; acc.y += a.cw[2] * w[i + 2].y; }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(1024) oned_run(OneDArgs<T> a) {
    extern __shared__ __align__(16) unsigned char oned_smem[];
    Cx<T>* buf = reinterpret_cast<Cx<T>*>(oned_smem);                 // 3 arrays of n
    __shared__ Cx<T> fb[3][8];                                         // aux: step start and two stage buffers
    __shared__ Cx<T> bvec[4];                                          // order 0: M E w
    __shared__ double red[32];
    const int n = a.n, tid = threadIdx.x;
    const int nf = a.order == 2 ? 8 : a.order == 1 ? 4 : 0;
    for (int i = tid; i < n; i += blockDim.x) buf[i] = a.psi[i];
    if (tid < nf) fb[0][tid] = a.aux[tid];
    __syncthreads();
    int iy = 0, ia = 1, ib = 2;                                        // buffer roles
    const T cs[4] = {(T)0.25, (T)(1.0 / 3.0), (T)0.5, (T)1.0};
    long long row = 0;
    for (long long step = 0; step < a.nsteps; ++step) {
        int in = iy, out = ia;
        for (int st = 0; st < 4; ++st) {
            const T cdt = cs[st] * a.dt;
            const Cx<T>* w = buf + (size_t)in * n;
            const Cx<T>* y = buf + (size_t)iy * n;
            Cx<T>* o = buf + (size_t)out * n;
            const Cx<T>* wf = fb[in];
            const Cx<T>* yf = fb[iy];
            Cx<T>* of = fb[out];
            if (a.order == 0) {                                        // b = M E w
                if (tid < 4) {
                    Cx<T> acc{0, 0};
                    const int j0 = tid < 2 ? 0 : 2;
                    for (int j = j0; j < j0 + 2; ++j) acc = cadd(acc, cmul(blk(a, MM, tid, j), w[gnode<T>(j, n)]));
                    bvec[tid] = acc;
                }
                __syncthreads();
            }
            // phi-part: o = y + cdt (-i) (H w + E^T b)
            for (int i = tid; i < n; i += blockDim.x) {
                Cx<T> hw = apply_h1(a, w, i);
                const int g = i < 2 ? i : i >= n - 2 ? i - n + 4 : -1;
                if (g >= 0) {
                    const Cx<T> b = a.order == 0 ? bvec[g] : wf[g];
                    hw = cadd(hw, b);
                }
                o[i] = Cx<T>{y[i].x + cdt * hw.y, y[i].y - cdt * hw.x};
            }
            // f-part
            if (tid < nf) {
                const int g = tid & 3, j0 = g < 2 ? 0 : 2;
                Cx<T> acc{0, 0};
                if (a.order == 1) {                                    // B f + A E w
                    for (int j = j0; j < j0 + 2; ++j) {
                        acc = cadd(acc, cmul(blk(a, MB, g, j), wf[j]));
                        acc = cadd(acc, cmul(blk(a, MA, g, j), w[gnode<T>(j, n)]));
                    }
                    of[g] = Cx<T>{yf[g].x + cdt * acc.x, yf[g].y + cdt * acc.y};
                } else if (tid < 4) {                                  // f' = g
                    of[g] = Cx<T>{yf[g].x + cdt * wf[4 + g].x, yf[g].y + cdt * wf[4 + g].y};
                } else {                                               // g' = B1 g + B0 f + A1 E phidot + A0 E w
                    for (int j = j0; j < j0 + 2; ++j) {
                        const int nj = gnode<T>(j, n);
                        Cx<T> pd = cadd(apply_h1(a, w, nj), wf[j]);   // phidot = -i (H w + E^T f) at Gamma
                        pd = Cx<T>{pd.y, -pd.x};
                        acc = cadd(acc, cmul(blk(a, MB1, g, j), wf[4 + j]));
                        acc = cadd(acc, cmul(blk(a, MB0, g, j), wf[j]));
                        acc = cadd(acc, cmul(blk(a, MA1, g, j), pd));
                        acc = cadd(acc, cmul(blk(a, MA0, g, j), w[nj]));
                    }
                    of[4 + g] = Cx<T>{yf[4 + g].x + cdt * acc.x, yf[4 + g].y + cdt * acc.y};
                }
            }
            __syncthreads();
            in = out;
            out = out == ia ? ib : ia;
        }
        // the last stage wrote buffer `in`: it becomes the next step's start, the other
        // two the stage buffers
        const int ny = in, oy = iy, oa = ia;
        iy = ny;
        ia = oy;
        ib = oa;
        if (a.diag_every > 0 && (step + 1) % a.diag_every == 0) {
            const Cx<T>* y = buf + (size_t)iy * n;
            double s = 0;
            for (int i = tid; i < n; i += blockDim.x) s += (double)y[i].x * y[i].x + (double)y[i].y * y[i].y;
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            if ((tid & 31) == 0) red[tid >> 5] = s;
            __syncthreads();
            if (tid < 32) {
                double v = tid < (int)(blockDim.x >> 5) ? red[tid] : 0.0;
                for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
                if (tid == 0) a.diag[row] = a.h * v;
            }
            ++row;
            __syncthreads();
        }
    }
    const Cx<T>* y = buf + (size_t)iy * n;
    for (int i = tid; i < n; i += blockDim.x) a.psi[i] = y[i];
    if (tid < nf) a.aux[tid] = fb[iy][tid];
}

template <typename T>
__global__ void oned_aux_init(OneDArgs<T> a, const Cx<T>* psi) {
    // order 2: f = 0, g = A1 E psi
    const int t = threadIdx.x;
    if (t < 4) {
        a.aux[t] = Cx<T>{0, 0};
        Cx<T> acc{0, 0};
        const int j0 = t < 2 ? 0 : 2;
        for (int j = j0; j < j0 + 2; ++j) acc = cadd(acc, cmul(blk(a, MA1, t, j), psi[gnode<T>(j, a.n)]));
        a.aux[4 + t] = acc;
    }
}

template <typename T>
OneDArgs<T> make_args(const abc1d_ctx* c) {
    OneDArgs<T> a{};
    a.n = c->p.n;
    a.order = c->p.order;
    const double w = -0.5 / (c->p.h * c->p.h);
    const double cc[3] = {-2.5, 4.0 / 3.0, -1.0 / 12.0};
    for (int m = 0; m < 3; ++m) a.cw[m] = (T)(w * cc[m]);
    const abc::oned::Mat2* src[NMAT] = {&c->blk.M, &c->blk.A, &c->blk.B, &c->blk.B1, &c->blk.B0, &c->blk.A1, &c->blk.A0};
    for (int k = 0; k < NMAT; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                a.mat[k][i][j] = Cx<T>{(T)src[k]->v[i][j].real(), (T)src[k]->v[i][j].imag()};
    a.h = c->p.h;
    return a;
}

}  // namespace

extern "C" int abc1d_setup(const abc1d_params* params, abc1d_ctx** out) {
    if (!out) return abc::fail(ABC_ERR_ARG, "null output pointer");
    *out = nullptr;
    std::string err;
    int st = abc::oned::check_params(params, err);
    if (st) return abc::fail(st, err);
    std::unique_ptr<abc1d_ctx> c(new abc1d_ctx());
    c->p = *params;
    st = abc::oned::build_blocks(c->p, c->blk, err);
    if (st) return abc::fail(st, err);
    if (cudaGetDevice(&c->device) != cudaSuccess) return abc::fail(ABC_ERR_CUDA, "no CUDA device");
    const size_t smem = 3 * (size_t)c->p.n * (c->p.precision == ABC_FP64 ? 16 : 8);
    cudaError_t e = c->p.precision == ABC_FP64
                        ? cudaFuncSetAttribute(oned_run<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaFuncSetAttribute(oned_run<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, std::string("shared memory: ") + cudaGetErrorString(e));
    *out = c.release();
    return ABC_OK;
}

extern "C" int abc1d_aux_init(abc1d_ctx* ctx, const void* psi, void* aux, void* stream) {
    if (!ctx || !psi) return abc::fail(ABC_ERR_ARG, "null argument");
    if (ctx->p.order == 0) return ABC_OK;
    if (!aux) return abc::fail(ABC_ERR_ARG, "orders 1 and 2 need the auxiliary buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cb = ctx->p.precision == ABC_FP64 ? 16 : 8;
    if (ctx->p.order == 1) {
        if (cudaMemsetAsync(aux, 0, 4 * cb, s) != cudaSuccess) return abc::fail(ABC_ERR_CUDA, "memset");
    } else if (ctx->p.precision == ABC_FP64) {
        OneDArgs<double> a = make_args<double>(ctx);
        a.aux = (Cx<double>*)aux;
        oned_aux_init<double><<<1, 32, 0, s>>>(a, (const Cx<double>*)psi);
    } else {
        OneDArgs<float> a = make_args<float>(ctx);
        a.aux = (Cx<float>*)aux;
        oned_aux_init<float><<<1, 32, 0, s>>>(a, (const Cx<float>*)psi);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, cudaGetErrorString(e));
    return ABC_OK;
}

extern "C" int abc1d_run(abc1d_ctx* ctx, void* psi, void* aux, double dt, long long nsteps, int diag_every,
                         double* norm_out, void* stream) {
    if (!ctx || !psi) return abc::fail(ABC_ERR_ARG, "null argument");
    if (ctx->p.order >= 1 && !aux) return abc::fail(ABC_ERR_ARG, "orders 1 and 2 need the auxiliary buffer");
    if (!(dt > 0) || nsteps < 0 || diag_every < 0) return abc::fail(ABC_ERR_ARG, "bad dt, nsteps or diag_every");
    if (diag_every > 0 && !norm_out) return abc::fail(ABC_ERR_ARG, "norm_out is NULL");
    const long long ndiag = diag_every > 0 ? nsteps / diag_every : 0;
    cudaStream_t s = (cudaStream_t)stream;
    double* dd = nullptr;
    if (ndiag > 0 && cudaMalloc(&dd, sizeof(double) * ndiag) != cudaSuccess)
        return abc::fail(ABC_ERR_ALLOC, "cudaMalloc of the norm series");
    const size_t smem = 3 * (size_t)ctx->p.n * (ctx->p.precision == ABC_FP64 ? 16 : 8);
    if (ctx->p.precision == ABC_FP64) {
        OneDArgs<double> a = make_args<double>(ctx);
        a.psi = (Cx<double>*)psi; a.aux = (Cx<double>*)aux; a.nsteps = nsteps; a.dt = dt;
        a.diag_every = diag_every; a.diag = dd;
        oned_run<double><<<1, 1024, smem, s>>>(a);
    } else {
        OneDArgs<float> a = make_args<float>(ctx);
        a.psi = (Cx<float>*)psi; a.aux = (Cx<float>*)aux; a.nsteps = nsteps; a.dt = (float)dt;
        a.diag_every = diag_every; a.diag = dd;
        oned_run<float><<<1, 1024, smem, s>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ndiag > 0) {
        e = cudaMemcpyAsync(norm_out, dd, sizeof(double) * ndiag, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (dd) cudaFree(dd);
    if (e != cudaSuccess) return abc::fail(ABC_ERR_CUDA, cudaGetErrorString(e));
    return ABC_OK;
}

extern "C" int abc1d_host_block(const abc1d_params* params, int which, double* out8) {
    if (!out8) return abc::fail(ABC_ERR_ARG, "null output");
    std::string err;
    int st = abc::oned::check_params(params, err);
    if (st) return abc::fail(st, err);
    abc::oned::Blocks1D b;
    st = abc::oned::build_blocks(*params, b, err);
    if (st) return abc::fail(st, err);
    const abc::oned::Mat2* m = nullptr;
    switch (which) {
        case ABC_MAT_K: m = &b.K; break;
        case ABC_MAT_M: m = &b.M; break;
        case ABC_MAT_A: m = &b.A; break;
        case ABC_MAT_B: m = &b.B; break;
        case ABC_MAT_B1: m = &b.B1; break;
        case ABC_MAT_B0: m = &b.B0; break;
        case ABC_MAT_A1: m = &b.A1; break;
        case ABC_MAT_A0: m = &b.A0; break;
        default: return abc::fail(ABC_ERR_ARG, "unknown matrix");
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            out8[(i * 2 + j) * 2] = m->v[i][j].real();
            out8[(i * 2 + j) * 2 + 1] = m->v[i][j].imag();
        }
    return ABC_OK;
}

extern "C" void abc1d_destroy(abc1d_ctx* ctx) { delete ctx; }
