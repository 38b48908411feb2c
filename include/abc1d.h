/*
 * abc1d.h -- C ABI of the one-dimensional time-stepper of Sec. 4.1 (the paper's 1D
 * experiment): the free Schroedinger equation on n interior nodes of spacing h with
 * the five-point second difference (c = -5/2, 4/3, -1/12, the radius-2 formula of
 * Sec. 2), closed at both ends by the discrete DtN absorbing boundary condition of
 * order 0, 1 or 2.
 *
 * Gamma is the two outermost nodes at each end (eq:25 with R = 2): Gamma order is
 * [0, 1, n-2, n-1].  The two ends see disjoint half-lines, so K(s) is block diagonal:
 * one 2 x 2 block per end, the right block the left one with its nodes mirrored.
 * K(s) comes from eq:eval with the free lattice Green's function of the five-point
 * scheme in closed form (App. B): G_n = b1 u1^|n| + b2 u2^|n|, u1, u2 the roots inside
 * the unit circle of c2 u^4 + c1 u^3 + (c0 + 2 i s h^2) u^2 + c1 u + c2 = 0, b1, b2 from
 * the equation (H_0 - i s) G = delta at n = 0 and n = 1.
 *
 *   order 0 (eq:dynamics0): M = K(s0)
 *   order 1 (eq:dynamics1): fit1 = ABC_FIT1_LIMIT (Thm 3.2: A = -i H_{Gamma,II}
 *            H_{II,Gamma}, B = s1 I - A K(s1)^{-1}) or ABC_FIT1_TWO_POINT
 *            ((s_j I - B) K(s_j) = A at s1 and s1b; Sec. 4.1 uses s = 10, 20)
 *   order 2 (eq:dynamics2): R_22(s) = (s^2 I - s B1 - B0)^{-1}(s A1 + A0) = K(s) at four
 *            points (Sec. 4.1 uses s = 10, 11, 20, 21); g(0) = A1 E phi(0).  For the
 *            five-point scheme these conditions are singular: a fixed row combination
 *            of K(s) obeys a first-degree identity at every s, so the solutions share
 *            R_22 and differ in one hidden root of det(s^2 I - s B1 - B0) that rounding
 *            excites (in the right half-plane the run diverges).  The library takes the
 *            minimum-norm solution plus the shortest correction along the null
 *            direction that puts that root at s = -min(s_j).
 *
 * One time step applies the degree-4 Taylor polynomial of exp(dt L) in Horner form
 * (eq:21 read as that series), the same integrator as the 3D library.  The whole run
 * is one launch of one thread block; the state stays in shared memory.
 *
 * psi: device array of n complex values (complex128 for ABC_FP64, complex64 for
 * ABC_C64_FP32); aux: device array of 4 (order 1) or 8 (order 2: f then g) complex
 * values of the same type, NULL for order 0.  The caller owns both.  Every function
 * returns ABC_OK or an ABC_ERR_* code of abc.h.
 */
#ifndef ABC1D_H
#define ABC1D_H

#include <stddef.h>

#include "abc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ABC1D_MAX_NODES 4096   /* n: 8 .. 4096 (the state is held in shared memory) */

typedef struct {
    int n;            /* interior nodes, 8 .. ABC1D_MAX_NODES                          */
    double h;         /* spacing > 0                                                   */
    int order;        /* 0, 1 or 2                                                     */
    double s[4];      /* order 0: s[0] = s0; order 1: s[0] = s1 (and s[1] = s1b for the
                         two-point fit); order 2: the four distinct points            */
    int fit1;         /* order 1: ABC_FIT1_LIMIT or ABC_FIT1_TWO_POINT                  */
    int precision;    /* ABC_FP64 or ABC_C64_FP32                                       */
} abc1d_params;

typedef struct abc1d_ctx abc1d_ctx;

/* FP64 host set-up of the boundary blocks, then a copy to the current device. */
int abc1d_setup(const abc1d_params* params, abc1d_ctx** out);

/* The consistent auxiliary state at t = 0 for psi (order 1: zero; order 2: f = 0,
 * g = A1 E psi); no-op for order 0.  Synchronises the stream. */
int abc1d_aux_init(abc1d_ctx* ctx, const void* psi, void* aux, void* stream);

/* nsteps time steps of (psi, aux) in place.  If diag_every > 0, the norm h |phi|^2
 * after every diag_every steps goes to norm_out (host, nsteps / diag_every doubles);
 * the call then synchronises the stream. */
int abc1d_run(abc1d_ctx* ctx, void* psi, void* aux, double dt, long long nsteps, int diag_every,
              double* norm_out, void* stream);

/* The left end's 2 x 2 block (row-major complex128, 8 doubles) of a matrix of
 * abc.h's ABC_MAT_* (K at the first point, M, A, B, B1, B0, A1, A0); the right
 * end's block is this one with rows and columns reversed.  GPU-free. */
int abc1d_host_block(const abc1d_params* params, int which, double* out8);

void abc1d_destroy(abc1d_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ABC1D_H */
