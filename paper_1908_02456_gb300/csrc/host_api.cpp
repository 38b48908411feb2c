// Host-only entry points of the C ABI (no CUDA calls): status strings, the
// per-thread error message and the FP64 setup for machines without a GPU.
#include <cstring>
#include <string>

#include "internal.h"

namespace abc {
thread_local std::string g_last_error;
int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}
}  // namespace abc

using namespace abc;

extern "C" const char* abc_status_string(int status) {
    switch (status) {
        case ABC_OK: return "ok";
        case ABC_ERR_ARG: return "invalid argument";
        case ABC_ERR_ALLOC: return "allocation failed";
        case ABC_ERR_CUDA: return "CUDA error";
        case ABC_ERR_SINGULAR: return "singular system";
        case ABC_ERR_TIMEOUT: return "device wait timed out";
        case ABC_ERR_UNSTABLE: return "Lyapunov functional grew";
        case ABC_ERR_UNSUPPORTED: return "not supported by this build";
        default: return "unknown status";
    }
}

extern "C" const char* abc_last_error(void) { return g_last_error.c_str(); }

namespace abc {
int check_params(const abc_grid* grid, const abc_params* params) {
    if (!grid || !params) return fail(ABC_ERR_ARG, "null grid or params");
    if (grid->radius != 1 && grid->radius != 3)
        return fail(ABC_ERR_UNSUPPORTED, "stencil radius 1 (3-point) or 3 (7-point, Sec. 4.2) only");
    if (params->order < 0 || params->order > 2) return fail(ABC_ERR_ARG, "order must be 0, 1 or 2");
    if (params->order == 2) {
        for (int j = 0; j < 4; ++j) {
            if (!(params->s2[j] > 0.0)) return fail(ABC_ERR_ARG, "interpolation point must be > 0");
            for (int i = 0; i < j; ++i)
                if (params->s2[i] == params->s2[j]) return fail(ABC_ERR_ARG, "order-2 points must be distinct");
        }
    } else {
        const double s = params->order == 0 ? params->s0 : params->s1;
        if (!(s > 0.0)) return fail(ABC_ERR_ARG, "interpolation point must be > 0");
    }
    if (params->fit1 < ABC_FIT1_LIMIT || params->fit1 > ABC_FIT1_HERMITE)
        return fail(ABC_ERR_ARG, "fit1 must be ABC_FIT1_LIMIT, ABC_FIT1_TWO_POINT or ABC_FIT1_HERMITE");
    if (params->fit1 != ABC_FIT1_LIMIT && params->order != 1)
        return fail(ABC_ERR_ARG, "fit1 applies to order 1 only");
    if (params->fit1 == ABC_FIT1_TWO_POINT && (!(params->s1b > 0.0) || params->s1b == params->s1))
        return fail(ABC_ERR_ARG, "the two-point fit needs s1b > 0 and s1b != s1");
    if (params->precision < ABC_FP64 || params->precision > ABC_C64_SPLIT_FP16)
        return fail(ABC_ERR_ARG, "unknown precision");
    // With radius 3 the order-2 fit (the basic solution of a nearly singular system)
    // carries entries near 1e5 whose products cancel: complex64 drifts from FP64 by
    // ~1e-4 over 200 steps (measured), above the 1e-5 bound of the reduced forms.
    if (grid->radius == 3 && params->order == 2 && params->precision != ABC_FP64)
        return fail(ABC_ERR_UNSUPPORTED, "the second-order ABC with radius 3 needs ABC_FP64");
    if (params->precision == ABC_C64_SPLIT_BF16)
        return fail(ABC_ERR_UNSUPPORTED,
                    "the split-bf16 form is not built (use ABC_C64_SPLIT_FP16 or ABC_C64_3XTF32)");
    if (params->max_orbitals < 1 || params->max_orbitals > 65535)
        return fail(ABC_ERR_ARG, "max_orbitals must be in [1, 65535]");
    return ABC_OK;
}
}  // namespace abc

extern "C" int abc_host_matrices(const abc_grid* grid, const abc_params* params, int which,
                                 void* host_dst, size_t bytes) {
    int st = check_params(grid, params);
    if (st) return st;
    if (!host_dst) return fail(ABC_ERR_ARG, "null destination");
    Geometry g;
    std::string err;
    st = build_geometry(grid->nx, grid->ny, grid->nz, grid->h, g, err, grid->radius);
    if (st) return fail(st, err);
    if (bytes < (size_t)16 * g.n_gamma * g.n_gamma) return fail(ABC_ERR_ARG, "destination too small");
    Blocks b;
    st = compute_param_blocks(g, *params, b, err);
    if (st) return fail(st, err);
    st = dense_natural(g, b, which, reinterpret_cast<cd*>(host_dst), err);
    if (st) return fail(st, err);
    return ABC_OK;
}
