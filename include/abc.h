/*
 * abc.h -- C ABI of the GB300 time-stepper for the 3D Schroedinger equation
 * closed by the discrete Dirichlet-to-Neumann absorbing boundary condition of
 * Wu & Li, "Absorbing boundary conditions for the time-dependent
 * Schroedinger-type equations in R^3".
 *
 * Problem (Sec. 2, eq:22/eq:32, eq:omega1): interior box of nx*ny*nz nodes with
 * spacing h, H = -1/2 Delta_h + V with the 3-point second difference per axis
 * (the standard 7-point 3D stencil).  The exterior (V = 0, phi_II(0) = 0) enters
 * only through the boundary nodes Gamma (eq:25: nodes with a coordinate on a
 * face), either as
 *   order 0 (eq:dynamics0):  phi' = -i H phi - i E^T M E phi,      M = K(s0)
 *   order 1 (eq:dynamics1):  phi' = -i H phi - i E^T f,
 *                            f'   = B f + A E phi,
 *                            A = -i H_{Gamma,II} H_{II,Gamma}, B = s1 I - A K(s1)^{-1}
 *   order 2 (eq:dynamics2):  phi' = -i H phi - i E^T f,  f' = g,
 *                            g' = B1 g + B0 f + A1 E phi' + A0 E phi,
 *                            R_22(s) = (s^2 I - s B1 - B0)^{-1}(s A1 + A0) fitted to
 *                            K at four points (Sec. 3.3)
 * with K(s) the DtN map of eq:17, evaluated by eq:eval (App. A).  One time step
 * applies sum_{k=0..4} (dt L)^k / k! (eq:21, signs read as the Taylor series of
 * exp(dt L)) in Horner form.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Node order: x fastest, linear index (k*ny + j)*nx + i.  Node coordinates are
 *   not needed by the library (only h).
 * - psi: device array [n_orb][nz][ny][nx] of complex values, interleaved (re, im):
 *   complex128 when precision == ABC_FP64, complex64 otherwise.
 * - aux: device array [n_gamma][n_orb] (orbital fastest) of the same complex type,
 *   holding f_Gamma (order 1; pass NULL for order 0), or [2][n_gamma][n_orb] holding
 *   f_Gamma then g = df_Gamma/dt (order 2).  Gamma nodes are numbered by ascending
 *   linear index.  Start it with abc_aux_init (order 1: zero, f_Gamma(0) = 0, Sec. 2).
 * - V: device array [nz][ny][nx] of real values (double for ABC_FP64, float
 *   otherwise): the external potential.
 * - The caller owns psi, aux and V.  The context owns the boundary matrices and
 *   its workspace; nothing the caller passes is freed by the library.
 * - stream: a cudaStream_t passed as void*; NULL means the legacy default stream.
 *   Calls are asynchronous with respect to the host unless stated.
 * - Every function returns ABC_OK (0) or an ABC_ERR_* code; no exception crosses
 *   the ABI.  abc_last_error() gives a message for the last failure on the calling
 *   thread.
 */
#ifndef ABC_H
#define ABC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ABC_OK 0
#define ABC_ERR_ARG 1          /* invalid argument (size, pointer, order, ...) */
#define ABC_ERR_ALLOC 2        /* host or device allocation failed */
#define ABC_ERR_CUDA 3         /* a CUDA runtime call failed */
#define ABC_ERR_SINGULAR 4     /* eq:eval system or K(s1) not invertible */
#define ABC_ERR_TIMEOUT 5      /* a bounded device wait gave up */
#define ABC_ERR_UNSTABLE 6     /* the Lyapunov functional grew (divergence monitor) */
#define ABC_ERR_UNSUPPORTED 7  /* valid request this build does not implement */

/* arithmetic of the path */
#define ABC_FP64 0             /* complex128 state, complex128 boundary matrices   */
#define ABC_C64_FP32 1         /* complex64 state, complex64 matrices, FP32 FMA     */
#define ABC_C64_SPLIT_BF16 2   /* reserved (bf16 hi + lo tensor-core form); not
                                  built: abc_setup returns ABC_ERR_UNSUPPORTED      */
#define ABC_C64_3XTF32 3       /* complex64 state; for n_orb >= 2 the boundary
                                  contraction runs on the tensor cores (tcgen05,
                                  kind::tf32) with the matrices split as TF32 hi +
                                  lo and three products per term (FP32-level error),
                                  FP32 accumulation; n_orb = 1 as ABC_C64_FP32      */
#define ABC_C64_SPLIT_FP16 4   /* complex64 state; for n_orb >= 2 the boundary
                                  contraction runs on the tensor cores with FP16
                                  operands (kind::f16, twice the TF32 rate): every
                                  class block is scaled by a power of two and every
                                  right-hand-side column by a power of two found per
                                  contraction, both split as FP16 hi + lo (the same
                                  10 + 10 mantissa bits as 3xTF32), three products
                                  per term, FP32 accumulation, the scales undone in
                                  the epilogue (exact); n_orb = 1 as ABC_C64_FP32.
                                  Columns whose largest part is above ~2^78 overflow
                                  FP16 (a state that large has diverged)            */

/* how the order-1 coefficients of R_11(s) = (sI - B)^{-1} A are fitted to K(s) */
#define ABC_FIT1_LIMIT 0       /* Thm 3.2: R_11(s1) = K(s1) and the s -> infinity
                                  limit, A = -i H_{Gamma,II} H_{II,Gamma} (diagonal
                                  for radius 1), B = s1 I - A K(s1)^{-1}             */
#define ABC_FIT1_TWO_POINT 1   /* R_11(s1) = K(s1), R_11(s1b) = K(s1b), both finite
                                  (the variant Sec. 3.2 reports as still stable):
                                  B = (s1 K1 - s1b K2)(K1 - K2)^{-1},
                                  A = (s1 I - B) K1; B and A dense per class         */
#define ABC_FIT1_HERMITE 2     /* value and derivative at s1 (eq:39, App. C):
                                  (s1 I - B)^{-1} A = K(s1), (s1 I - B)^{-2} A =
                                  -K'(s1); B = s1 I + K1 K1'^{-1},
                                  A = -K1 K1'^{-1} K1                                */

/* matrices for abc_get_matrices / abc_host_matrices (dense, natural Gamma order) */
#define ABC_MAT_K 0            /* K(s) at the context's interpolation point (orders
                                  0 and 1 with the limit fit)                       */
#define ABC_MAT_M 1            /* order 0: M = K(s0)                                */
#define ABC_MAT_A 2            /* order 1: A                                        */
#define ABC_MAT_B 3            /* order 1: B                                        */
#define ABC_MAT_Q 4            /* order 1: Q = (H_{Gamma,II} H_{II,Gamma})^{-1}
                                  (the Lyapunov weight of Thm 3.2; with the
                                  two-point and Hermite fits it is the weight of
                                  the diagnostic W only, not a proven Lyapunov
                                  functional)                                       */
#define ABC_MAT_B1 5           /* order 2: B1 of R_22 (Sec. 3.3, eq:dynamics2)      */
#define ABC_MAT_B0 6           /* order 2: B0                                       */
#define ABC_MAT_A1 7           /* order 2: A1                                       */
#define ABC_MAT_A0 8           /* order 2: A0                                       */

typedef struct {
    int nx, ny, nz;   /* interior nodes per axis, each >= 3, nz <= 65535,
                         nx * ny * nz < 2^31                                       */
    int radius;       /* stencil radius per axis: 1 (the 3-point formula) or 3 (the
                         7-point formula of Sec. 4.2, c = -49/18, 3/2, -3/20, 1/90;
                         Gamma is then the nodes within 3 of a face, each axis needs
                         >= 7 nodes, A is block-sparse and order 1 runs on dense class
                         rows, order 2 needs ABC_FP64, the adjoint and
                         abc_step_noalloc refuse it, and W is |phi|^2)              */
    double h;         /* grid spacing > 0                                          */
} abc_grid;

typedef struct {
    int order;        /* 0, 1 or 2 (rational order m of eq:24)                      */
    double s0;        /* order 0 interpolation point, > 0 (Thm 3.1)                 */
    double s1;        /* order 1 interpolation point, > 0 (Thm 3.2)                 */
    int precision;    /* ABC_FP64 | ABC_C64_FP32 | ABC_C64_3XTF32 | ABC_C64_SPLIT_FP16 */
    int max_orbitals; /* largest n_orb later passed to step/run (sizes workspace),
                         1 .. 65535                                                 */
    double s2[4];     /* order 2 interpolation points, > 0 and distinct (Sec. 3.3:
                         R_22(s) = (s^2 I - s B1 - B0)^{-1}(s A1 + A0) = K(s) there) */
    int fit1;         /* order 1: ABC_FIT1_LIMIT (0, default), ABC_FIT1_TWO_POINT or
                         ABC_FIT1_HERMITE; must be 0 for orders 0 and 2.  The fitted
                         forms run on the dense class blocks [B | A] (no packed
                         symmetric tiles, no tensor-core image); the adjoint and
                         abc_step_noalloc cover the limit fit only                    */
    double s1b;       /* ABC_FIT1_TWO_POINT: the second point, > 0 and != s1        */
} abc_params;

typedef struct {
    double a, b, alpha;   /* V = V_ext + a rho + b rho^(1+alpha), rho = sum_j |phi_j|^2
                             (the density-dependent mean field of Sec. 4.3, eq:ham_tdhf,
                             in simplified form); rho^(1+alpha) := 0 at rho = 0        */
} abc_meanfield;

typedef struct abc_ctx abc_ctx;

/* Builds the context: index sets, K(s) by eq:eval with the free lattice Green's
 * function (App. A, App. D), the order-0 / order-1 coefficients (Thm 3.1 / 3.2) or
 * the order-2 fit (Sec. 3.3: four interpolation conditions per irreducible class; at
 * radius 3 the system is nearly singular and its basic solution by column-pivoted QR
 * is taken, pivots below 1e-13 of the largest column norm dropped), all in FP64 on
 * the host (untimed setup, OpenMP), then converts them to the device format of
 * `precision` and uploads them to the current CUDA device.  *out receives the context
 * (free with abc_destroy).  Errors: ABC_ERR_ARG for bad sizes/order/precision,
 * ABC_ERR_UNSUPPORTED (order 2 at radius 3 in a reduced precision; ABC_C64_SPLIT_BF16),
 * ABC_ERR_SINGULAR, ABC_ERR_ALLOC, ABC_ERR_CUDA. */
int abc_setup(const abc_grid* grid, const abc_params* params, abc_ctx** out);

/* n_gamma = |Gamma| = nx*ny*nz - (nx-2R)(ny-2R)(nz-2R) (eq:25, radius R). */
int abc_boundary_size(const abc_ctx* ctx, long long* n_gamma);

/* One time step of the augmented system in place on (psi, aux), static potential
 * V.  n_orb in [1, max_orbitals]; dt > 0. */
int abc_step(abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt,
             void* stream);

/* nsteps time steps.  mf == NULL: static V; else V is V_ext and the mean-field
 * potential is recomputed from the state before every step and held fixed within
 * it.  If diag_every > 0, after every diag_every steps the per-orbital
 * diagnostics [norm, W, energy] (see abc_diagnostics) are stored; diag_out (host,
 * [nsteps/diag_every][n_orb][3] doubles) is filled when the call returns, which
 * then synchronises the stream.  The step loop is replayed as a CUDA graph.
 *
 * Divergence monitor (with diag_every > 0): Thm 3.1 and Thm 3.2 make W (= |phi|^2
 * for order 0, |phi|^2 + f^* Q f for order 1) non-increasing, and the degree-4
 * Taylor step keeps that for stable dt.  On the device, every diagnostic row is
 * compared with the previous one (with the start state for the first): for order 0
 * and for the order-1 limit fit at radius 1 W may not grow by more than
 * diag_every * 1e-12 (FP64) or diag_every * 1e-6 (complex64) relative; for the
 * forms without a proof (order 2, the other order-1 fits, order 1 at radius 3) W
 * may not pass twice its start value; a non-finite W always fails.  The run still
 * completes its nsteps (the host learns of the failure when the call synchronises)
 * and then returns ABC_ERR_UNSTABLE, naming the first failing step and orbital in
 * abc_last_error(); diag_out is filled all the same. */
int abc_run(abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt,
            long long nsteps, const abc_meanfield* mf, int diag_every, double* diag_out,
            void* stream);

/* abc_run on HOST buffers (same layouts): copies psi, aux and V to device buffers
 * owned by the context, runs, copies psi and aux back, and synchronises. */
int abc_run_host(abc_ctx* ctx, void* psi_host, void* aux_host, const void* V_host, int n_orb,
                 double dt, long long nsteps, const abc_meanfield* mf, int diag_every,
                 double* diag_out);

/* Consistent auxiliary state at t = 0 for the wave function psi (device, [n_orb]
 * orbitals): order 1 aux = 0 (f(0) = 0 since phi_II(0) = 0, Sec. 2); order 2 aux =
 * [f | g] with f = 0 and g = A1 E psi (the value for which the Laplace transform of
 * eq:dynamics2 gives f = R_22(s) E phi); order 0 holds no auxiliary state (no-op).
 * aux: device [n_gamma][n_orb] complex (order 1) or [2][n_gamma][n_orb] (order 2:
 * f then g), overwritten.  Asynchronous on the stream. */
int abc_aux_init(abc_ctx* ctx, const void* psi, void* aux, int n_orb, void* stream);

/* Checkpoint / resume.  A state blob is a self-describing host buffer: a header
 * (format version, grid, radius, ABC order and interpolation points, precision,
 * orbital count, n_gamma, the context's step count and time, payload sizes and a
 * 64-bit checksum) followed by psi and aux exactly as they are stored on the device
 * (layouts above).  abc_state_size gives the blob size for n_orb orbitals.
 * abc_get_state copies psi and aux (device) into host_dst (at least that size),
 * recording the context's progress; it synchronises the stream.  abc_set_state
 * checks that the blob was written by a context with the same grid, radius, order,
 * fit, interpolation points, precision and orbital count and that its checksum
 * matches (else ABC_ERR_ARG, nothing copied), then copies psi and aux to the given
 * device buffers and sets the context's progress to the recorded one; it
 * synchronises the stream.  abc_progress reports the steps and the time the
 * context has advanced (abc_step, abc_run, abc_run_host; abc_set_state resets
 * them).  The paper has no counterpart (it defines the state y = (phi, f) that the
 * blob holds, Sec. 3). */
int abc_state_size(const abc_ctx* ctx, int n_orb, size_t* bytes);
int abc_get_state(const abc_ctx* ctx, const void* psi, const void* aux, int n_orb, void* host_dst, size_t bytes,
                  void* stream);
int abc_set_state(abc_ctx* ctx, void* psi, void* aux, int n_orb, const void* host_src, size_t bytes, void* stream);
int abc_progress(const abc_ctx* ctx, long long* steps, double* t);

/* Per-orbital diagnostics of the current state into host out[n_orb][3]:
 * norm_j = h^3 |phi_j|^2; W_j = norm_j + h^3 f_j^* Q f_j (eq:lyapunov1; = norm_j
 * for order 0, eq:lyapunov0); energy_j = h^3 Re <phi_j, H_{I,I}[V] phi_j> for a
 * static potential.  With a mean field (mf as in abc_run) energy_j =
 * h^3 Re <phi_j, (H_kin + V_ext + e(rho)) phi_j> with e(rho) = (a/2) rho +
 * b/(2+alpha) rho^(1+alpha), the interaction energy per unit density, so that
 * sum_j energy_j = E[phi] = h^3 sum_j Re <phi_j, H_kin phi_j> + h^3 sum_x [V_ext rho
 * + (a/2) rho^2 + b/(2+alpha) rho^(2+alpha)], the energy the mean-field dynamics
 * conserves in a closed box (its rho-derivative is the potential; Sec. 4.3 reports
 * the energy a run releases).  All sums in FP64.  Synchronises the stream. */
int abc_diagnostics(abc_ctx* ctx, const void* psi, const void* aux, const void* V, int n_orb,
                    const abc_meanfield* mf, double* out, void* stream);

/* Gradient of the absorbed probability J = sum_j (1 - h^3 |phi_j(T)|^2) after
 * nsteps steps from psi0 (aux starts at zero) with the static potential V, with
 * respect to V: dJdV (device, real [nz][ny][nx], same real type as V) is
 * overwritten; J_out (host) receives J.  Discrete adjoint of the Horner stages;
 * the forward states are checkpointed every ckpt_every steps and recomputed
 * segment by segment.  psi0 is not modified.  Synchronises the stream. */
int abc_adjoint_run(abc_ctx* ctx, const void* psi0, const void* V, int n_orb, double dt,
                    long long nsteps, int ckpt_every, double* J_out, void* dJdV, void* stream);

/* Dense FP64 copy (complex128, row-major n_gamma x n_gamma, natural Gamma order)
 * of a coefficient matrix held by the context (ABC_MAT_*).  bytes must be at
 * least 16*n_gamma^2.  Reconstructed on the host from the stored FP64 blocks. */
int abc_get_matrices(const abc_ctx* ctx, int which, void* host_dst, size_t bytes);

/* Host-only variant for machines without a GPU: runs the FP64 setup of abc_setup
 * and returns the dense matrix `which` without touching CUDA. */
int abc_host_matrices(const abc_grid* grid, const abc_params* params, int which,
                      void* host_dst, size_t bytes);

/* Kernel timing: when enabled, abc_run launches eagerly (no graph) and brackets
 * every launch of the dominant kernel `kernel` (ABC_KERNEL_*) with CUDA events on
 * the launching stream; abc_profile_read returns the summed milliseconds and the
 * launch count since the last enable, after synchronising. */
#define ABC_KERNEL_CONTRACTION 0   /* boundary DtN contraction (GEMV / GEMM; for the
                                      tensor-core forms the GEMM alone)              */
#define ABC_KERNEL_STENCIL 1       /* fused stencil + potential + Horner stage       */
#define ABC_KERNEL_PACK 2          /* tensor-core forms: packing of the right-hand
                                      sides into the GEMM's operand image            */
int abc_profile_enable(abc_ctx* ctx, int enable);
int abc_profile_read(abc_ctx* ctx, int kernel, double* ms, long long* launches);
/* Per-launch durations (milliseconds, launch order) of the same record: writes
 * min(max_out, launches) values to the host array ms_out and the launch count to
 * *launches.  The paper has no counterpart (measurement support). */
int abc_profile_durations(abc_ctx* ctx, int kernel, float* ms_out, long long max_out, long long* launches);

/* Algorithmic bytes of one launch of a kernel for n_orb orbitals (the roofline
 * numerator): boundary matrix bytes + vectors for the contraction (for the
 * tensor-core GEMM: its split operand planes of every class block once, the packed
 * right-hand sides and the partial outputs, plus f_hat and phi_hat when its epilogue
 * forms the back transform's input, ABC_TUNE_LANES); for the stencil 3 complex values
 * per point and orbital plus V per point (plus the output on Gamma with
 * ABC_TUNE_GAMMA_COPY), or, when abc_run fuses the stages in time
 * (ABC_TUNE_FUSED), the fused pass's 2 complex values per point and orbital plus V
 * plus the band values it stores. */
int abc_kernel_bytes(const abc_ctx* ctx, int kernel, int n_orb, double* bytes);

/* Floating-point operations of one contraction launch for n_orb orbitals (kernel
 * must be ABC_KERNEL_CONTRACTION): useful = 8 real flops per complex multiply-add of
 * the class blocks with their right-hand sides, sum_k nseg R_k m_k^2 n_orb of them;
 * issued = what the arithmetic performs: 3 x useful on the tensor-core split forms
 * (three products per term; 2.25 x with the Karatsuba GEMM form, three real products
 * per complex term), 8 flops per entry of the stored blocks and orbital on the
 * CUDA-core GEMM of n_orb >= 2 (FP64, ABC_C64_FP32), useful otherwise.  The paper has
 * no counterpart (measurement support). */
int abc_kernel_flops(const abc_ctx* ctx, int kernel, int n_orb, double* useful, double* issued);

/* abc_step without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc while they step the
 * system (a framework whose pool allocator owns the device heap, or code that must
 * not allocate at that point).  It computes what abc_step computes with the same
 * stages; for one complex64 orbital its boundary contraction runs the full-block
 * kernel instead of abc_step's symmetric-tile kernel (whose partial sums need extra
 * scratch), so results agree to rounding.  It takes all per-step scratch
 * from one static device array of ABC_NOALLOC_SCRATCH_BYTES defined in the
 * library (held by every GPU that loads the library until exit) instead of the
 * context's workspace.  The context is only read.  Needs
 *   (2*nx*ny*nz*n_orb + 6*n_gamma*n_orb) * complex bytes <= ABC_NOALLOC_SCRATCH_BYTES,
 * otherwise ABC_ERR_ARG with the required size in abc_last_error().  Calls share
 * the array: calls whose work overlaps on the GPU race and must be serialised.
 * Nothing needs clearing between calls (every scratch value is written before it
 * is read).  Every call outside stream capture looks up the array's device address
 * (cudaGetSymbolAddress) on the current device; a call during capture reuses the
 * address the last uncaptured call found, so make one call on each device before
 * any stream capture.  ABC_FP64 and ABC_C64_FP32 contexts only. */
#define ABC_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int abc_step_noalloc(const abc_ctx* ctx, void* psi, void* aux, const void* V, int n_orb, double dt,
                     void* stream);

/* Fault-free check of the bounded-wait error path: one block waits on a barrier that
 * nothing completes, gives up after `polls` (1 .. 2^24) polls and raises the context's
 * device error flag, exactly as a bounded wait of the contraction does; the call then
 * returns ABC_ERR_TIMEOUT (and clears the flag), synchronising `stream`.  The context
 * stays usable.  Nothing traps, faults or spins without a bound. */
int abc_wait_selftest(abc_ctx* ctx, long long polls, void* stream);

/* Tuning knobs of the kernels (chosen by the autotuner, paper_1908_02456_gb300/tune.py):
 *   ABC_TUNE_L2_KEEP_TILES  number of leading 64x64 boundary tiles that the one-orbital
 *                           complex64 contraction streams with an L2 evict_last hint so
 *                           that they stay in L2 from one Horner stage to the next
 *                           (the rest use evict_first); 0 = all evict_first.
 *   ABC_TUNE_TILE_COUNT     (read only) number of stored tiles.
 *   ABC_TUNE_PDL            1 (default): launch the one-orbital tiled contraction
 *                           as a programmatic dependent of the forward transform
 *                           before it, so its CTAs start and copy their first
 *                           boundary tiles while the forward transform runs (they
 *                           wait for it before reading its output); 0: ordinary
 *                           launch.
 *   ABC_TUNE_CHAIN          1: in an order-1 step the back transforms of stages 1-3
 *                           also form the next stage's symmetry-adapted inputs (the
 *                           stencil's formula at the boundary nodes plus the forward
 *                           transform), so stages 2-4 launch no forward transform;
 *                           0 (default): a forward transform in every stage (measured
 *                           as fast at one orbital and faster at 32 and 128).
 *   ABC_TUNE_STENCIL        where the interior stencil of an order >= 1 stage runs:
 *                           0 (default) on a second stream forked after the boundary
 *                           contraction, 1 forked at the stage start, 2 on the main
 *                           stream after the back transform.
 *   ABC_TUNE_FUSED          order 1, complex64, radius 1, nx even: abc_run computes the
 *                           interior stencil of the four Horner stages of a step in one
 *                           pass (shared-memory rings of planes, the stages' boundary band
 *                           finished stage by stage after each contraction; same formula,
 *                           FP32 rounding differences only) and alternates the state
 *                           between psi and a context-owned buffer (one copy back after an
 *                           odd step count).  0 (default) off; 1 on; -1 on for n_orb >= 2.
 *                           abc_step and the adjoint always step stage by stage.
 *   ABC_TUNE_STENCIL_BPS    complex64, nx even: when the stencil runs on the second
 *                           stream (ABC_TUNE_STENCIL 0 or 1), launch it as a grid-stride
 *                           kernel of this many 256-thread blocks per SM (1..8), which
 *                           leaves room on every SM for the boundary chain's kernels
 *                           (the tensor-core GEMM needs one CTA slot per SM); 0 (default):
 *                           one thread per node pair.
 *   ABC_TUNE_STENCIL_KZ     complex64, radius 1, nx even, n_orb >= 2: form of the
 *                           stage-by-stage stencil: 0 one node pair per thread; 1 (default)
 *                           the same with registers capped for 8 blocks per SM; 2, 4, 8
 *                           or 16: each thread marches through that many planes of its
 *                           node pair, the z neighbours rolling through registers and the
 *                           next plane's loads issued before the current one is computed
 *                           (same formula in every form).
 *   ABC_TUNE_STENCIL_STAGED complex64, radius 1, nx even and <= 256, n_orb >= 2: 1 runs the
 *                           stage-by-stage stencil with each CTA marching through 24 planes
 *                           of an 8-row tile of one orbital, the planes of w (with their y
 *                           halo) and of y staged in six shared-memory slots by 1D bulk
 *                           copies (cp.async.bulk, two per plane) on mbarriers, so that
 *                           planes z + 2 .. z + 4 are in flight while plane z is computed;
 *                           bit-identical to the other forms; 0 (default) direct loads.
 *                           Takes precedence
 *                           over ABC_TUNE_STENCIL_KZ and ABC_TUNE_STENCIL_BPS.
 *   ABC_TUNE_BACK_MULTI     order 1 (limit fit), unpacked contraction output: 1 runs the
 *                           back transform four orbitals per cell group (n_orb a multiple
 *                           of 4; its tables read once per four), 2 two orbitals per group
 *                           (n_orb even); 0 (default) one orbital per group.
 *   ABC_TUNE_FORWARD_RW     n_orb a multiple of 4: 1 runs the four-orbital forward
 *                           transform with each slot's 8-point reflection transform in
 *                           one thread's registers (no lane shuffles; bit-identical
 *                           outputs); 0 (default) across 8 lanes.
 *   ABC_TUNE_GAMMA_COPY     complex64, radius 1, nx even, orders 0 and 1, n_orb a multiple
 *                           of 4: 1 each stage's stencil also writes its output on Gamma in
 *                           the natural boundary layout (two copies, 2 n_gamma max_orbitals
 *                           complex values, allocated on first use), and the next stage's
 *                           forward transform reads it there instead of gathering single
 *                           values from the whole state; 0 (default) gathers from the
 *                           state.  Bit-identical results either way.
 *   ABC_TUNE_LANES          order 1 (limit fit), tensor-core forms, n_orb a multiple of 32:
 *                           1 holds the adapted vectors and the contraction output
 *                           node-major ([adapted index][orbital]) inside a stage, and runs
 *                           the forward and back transforms one warp per cell and 32
 *                           orbitals, lane = orbital, the cell's transform in registers;
 *                           every access of a warp is then 256 contiguous bytes (except
 *                           the gather of w at Gamma from the state).  With one K split
 *                           the GEMM epilogue also forms the back transform's input
 *                           x = s1 f_hat + (-i a)(phi_hat - t), so the back transform
 *                           reads one array.  2 and 3: the same chain with each cell split
 *                           between two lanes (a warp per cell and 16 orbitals, half the
 *                           values per lane, the halves exchanged by lane shuffles;
 *                           registers capped for 4 or 5 blocks per SM); 4 and 5: each
 *                           cell split between four lanes (a warp per cell and 8
 *                           orbitals, the quarters exchanged through the warp's own
 *                           shared-memory tile; 6 or 8 blocks per SM).  Bit-identical
 *                           results; takes precedence over ABC_TUNE_FORWARD_RW and
 *                           ABC_TUNE_BACK_MULTI.  0 (default) orbital-major.
 *   ABC_TUNE_GEMM_TILE      tensor-core forms, n_orb >= 2: 0 (default) output tiles of up
 *                           to 96 columns, three ring stages, one CTA per SM; 1: up to 64
 *                           columns, two stages, two CTAs per SM; 2: the complex products
 *                           by Karatsuba's three real products (P1 = Sr Xr, P2 = Si Xi,
 *                           P3 = (Sr + Si)(Xr + Xi); Re = P1 - P2, Im = P3 - P1 - P2: a
 *                           quarter less tensor work, a third more matrix bytes), 64
 *                           columns, three stages, one CTA per SM (its matrix image is
 *                           built on first use).  Rebuilds the work lists (synchronises
 *                           the device).
 *   ABC_TUNE_GEMM_SPLIT     tensor-core forms: number of K splits of every output tile
 *                           (1..8), or 0 (default) for about two work items per CTA slot.
 *                           Rebuilds the work lists (synchronises the device).
 * Setting a knob drops the cached CUDA graph.  The paper has no counterpart.
 */
#define ABC_TUNE_L2_KEEP_TILES 0
#define ABC_TUNE_TILE_COUNT 1
#define ABC_TUNE_PDL 2
#define ABC_TUNE_CHAIN 3
#define ABC_TUNE_STENCIL 4
#define ABC_TUNE_FUSED 5
#define ABC_TUNE_GEMM_TILE 6
#define ABC_TUNE_GEMM_SPLIT 7
#define ABC_TUNE_STENCIL_BPS 8
#define ABC_TUNE_STENCIL_KZ 9
#define ABC_TUNE_BACK_MULTI 10
#define ABC_TUNE_FORWARD_RW 11
#define ABC_TUNE_GAMMA_COPY 12
#define ABC_TUNE_STENCIL_STAGED 13
#define ABC_TUNE_LANES 14
int abc_set_tuning(abc_ctx* ctx, int key, long long value);
int abc_get_tuning(const abc_ctx* ctx, int key, long long* value);

/* Number of kernels this context has launched since set-up (eager launches plus
 * the kernels of every replayed graph). */
int abc_launch_count(const abc_ctx* ctx, long long* launches);

void abc_destroy(abc_ctx* ctx);
const char* abc_status_string(int status);
const char* abc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ABC_H */
