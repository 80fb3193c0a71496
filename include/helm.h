/*
 * helm.h - C-ABI of the GB300 (sm_103a) solver for the 3D Helmholtz equation with Sommerfeld
 * absorbing boundaries, preconditioned by the exact inverse of a second-order operator that includes
 * the absorbing boundary (EigT / PFFT), inside restarted (flexible) GMRES.
 *
 * Paper: Gryazin, Gonzales, Li, "High-Resolution Solvers for 3D Helmholtz Scattering Problems Using
 * PFFT and Eigenvector-Based Preconditioning", arXiv 2602.07711.
 *
 * Conventions shared by every entry point
 *   - Grid functions are complex arrays indexed [l][j][i] (z, y, x) with x fastest: the slice ordering
 *     U_l of Sec. 4.1.  complex64 = interleaved float (re, im); complex128 = interleaved double.
 *   - Buffers passed to a call belong to the caller.  A pointer may be host or device memory where a
 *     comment says "host or device"; the library asks the CUDA runtime which one it is.  Everywhere else
 *     it must be device memory.  The context (helm_ctx) owns its device workspace; helm_destroy frees it.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are stream-ordered and return
 *     before the GPU work finishes, except helm_setup and helm_gmres_solve, which synchronise `stream`.
 *   - Errors are returned as helm_status; the library never aborts or traps.  Device-side loops have
 *     iteration caps and report through a status word, read back by the synchronising calls.
 *   - A context must not be used from two host threads at once.  Process-wide state is limited to: the
 *     launch-shape cache of helm_autotune (per grid size and order, guarded by a mutex), the per-thread text
 *     of helm_last_error, and the static scratch array of helm_residual_noalloc (one per GPU, shared by
 *     every call, so that overlapping calls of that entry point race).  Everything else lives in a context.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx helm_ctx;

typedef enum {
    HELM_OK = 0,
    HELM_ERR_ARG = 1,            /* invalid argument (sizes, null pointers, unsupported combination)   */
    HELM_ERR_CUDA = 2,           /* a CUDA runtime/driver call failed                                   */
    HELM_ERR_NOMEM = 3,          /* device allocation failed                                            */
    HELM_ERR_EIG = 4,            /* 1D eigendecomposition failed its residual / orthogonality check     */
    HELM_ERR_PIVOT = 5,          /* a tridiagonal pivot fell below 1e-30 in magnitude                   */
    HELM_ERR_NAN = 6,            /* NaN or Inf met in a norm or a Hessenberg entry                      */
    HELM_ERR_BREAKDOWN = 7,      /* Arnoldi breakdown h_{j+1,j} = 0 before convergence                  */
    HELM_ERR_NOT_CONVERGED = 8,  /* max_iter reached; x holds the last iterate                         */
    HELM_ERR_ITER_LIMIT = 9,     /* a device wait exceeded its iteration cap                           */
    HELM_ERR_UNSUPPORTED = 10    /* configuration not built (see the comment of the option)             */
} helm_status;

/* Grid (Sec. 2.1 and Sec. 5.2).  N_x x N_y x N_z unknowns on [0,lx] x [0,ly] x [0,lz].
 * staggered = 1: nodes at h/2 + j h, h = L/N, ghosts eliminated by Eq. D_bc (the grid of Sec. 5.2).
 * staggered = 0: collocated nodes (i-1) h, h = L/(N-1), boundary nodes are unknowns; the ghosts follow
 *   the three-point second-order closure of the ABC, U_0 = U_2 + 2 i k0 h U_1 per direction (edge and
 *   corner ghosts: the one-dimensional rules applied in turn), and the preconditioner is EigT3 (Lbar with
 *   gamma = 2 i k0 h, zeta = 2; Sec. 4.1).  k^2 and f are reflected about the boundary node.  The matvec
 *   and the residual run on the general stencil kernels (the fast ones are staggered).  EigT (EigT3),
 *   PFFT (PFFT3: the boundary correction spans the two outer layers, since zeta = 2) and FFT2; the 1D
 *   eigensetup needs k0 h <= 1 (HELM_ERR_EIG beyond). */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    int staggered;
} helm_grid;

/* Preconditioner M^-1 = h_z^2 A_p^-1 (Sec. 4): none, EigT (Sec. 4.1) or PFFT (Sec. 4.2; needs N_x and N_y
 * powers of two <= 512; its sine solver uses the Dirichlet condition with the corner -1 of the staggered
 * face, and the boundary correction makes the result that of A_p^-1 on either grid).  FFT2 is the
 * Dirichlet solve alone, M^-1 = h_z^2 (A_p^F)^-1 (Eq. TFprec; step 1 of PFFT without the boundary
 * correction): the FFT-based second-order preconditioner the paper compares against (Sec. 5), same size
 * limits as PFFT. */
enum { HELM_PRECOND_NONE = 0, HELM_PRECOND_EIGT = 1, HELM_PRECOND_PFFT = 2, HELM_PRECOND_FFT2 = 3 };

/* Arithmetic of the eigenvector transforms (EigT steps 2 and 4).  The stencil is complex64 in every mode and
 * the Krylov vectors too, except in flexible single solves with HELM_PREC_FP16 (below); the z-solves compute
 * in FP32; the Hessenberg/Givens update and the 1D eigensetup are FP64, the true residual, the right-hand
 * side and the iterate double-float (about 44 bits) in every mode.
 *   HELM_PREC_FP32    complex64 on the CUDA cores (FFMA), the "plain complex64" method
 *   HELM_PREC_TF32    tcgen05 tensor cores, TF32 operands, FP32 accumulation in TMEM (one product); needs
 *                     even N_x.  Relative error of a transform about 8e-4.
 *   HELM_PREC_TF32X3  split precision on the same tensor cores: every operand a = hi + lo with hi its TF32
 *                     rounding and lo the TF32 rounding of the remainder, products hi hi + hi lo + lo hi
 *                     (three MMAs) with FP32 accumulation: FP32-level transforms at three times the tensor
 *                     work; needs even N_x.
 *   HELM_PREC_BF16    tcgen05 tensor cores with BF16 operands (round to nearest even, 8-bit significand)
 *                     and FP32 accumulation in TMEM, and the grids between the passes of the EigT chain
 *                     stored in BF16 (the z-solve reads and writes BF16 and computes in FP32): half the
 *                     bytes of the TF32 chain and twice its MMA rate; relative error of the whole
 *                     preconditioner about 1e-2.  EigT only (the PFFT and helm_precond_step passes run in
 *                     TF32); needs N_x a multiple of 4; in helm_gmres_solve_batched only with flexible GMRES
 *                     (HELM_ERR_UNSUPPORTED otherwise).
 *   HELM_PREC_FP16    the same chain with FP16 operands and grids (TF32's 11-bit significand, so about
 *                     TF32's accuracy): every stored grid carries a power-of-two scale that rules out
 *                     overflow for any input, from operator bounds computed at set-up (spectral norms of
 *                     the eigenvector matrices, kappa(V_z) / min |lambda| for the z-solves) times, after the
 *                     first pass, the Frobenius norm the producing pass measured; the last pass undoes
 *                     them.  Flexible single solves with EigT (one Gram-Schmidt pass, no learned
 *                     correction) also keep the Krylov basis in FP16, one scale per vector.  Same limits as
 *                     BF16, and k0z2 (helm_setup) must be constant.                                     */
enum { HELM_PREC_FP32 = 0, HELM_PREC_TF32 = 1, HELM_PREC_TF32X3 = 2, HELM_PREC_BF16 = 3, HELM_PREC_FP16 = 4 };

typedef struct {
    int order;       /* 2, 4 (Eq. scheme4, any h_x, h_y, h_z) or 6 (Eq. scheme6, needs h_x = h_y = h_z)  */
    int precond;     /* HELM_PRECOND_*                                                                    */
    int precision;   /* HELM_PREC_*                                                                       */
    int restart;     /* GMRES(m) restart length m, 1..64                                                  */
    int max_iter;    /* cap on inner iterations N0                                                        */
    double rtol;     /* stop when ||F - A U||_2 / ||F - A U^0||_2 <= rtol (rel-res of Sec. 5.1)            */
    int flexible;    /* 1 = flexible GMRES (stores z_j = M^-1 v_j), 0 = right-preconditioned GMRES        */
    int reorth;      /* 1 = classical Gram-Schmidt twice (CGS2), 0 = once                                 */
} helm_options;

typedef struct {
    int status;            /* helm_status of the solve                                          */
    int iterations;        /* N0: inner Arnoldi steps                                           */
    int restarts;          /* completed cycles                                                  */
    int reserved;
    double relres_true;    /* FP64 ||F - A U|| / ||F - A U^0|| at exit                           */
    double relres_est;     /* Givens estimate at the last step                                   */
    double beta0;          /* ||F - A U^0||_2                                                    */
    double seconds;        /* host wall time of the call                                         */
    int cycle_its[16];     /* inner steps of each of the first 16 cycles                        */
} helm_solve_info;

/* Data type selector for helm_apply_A. */
enum { HELM_C64 = 0, HELM_C128 = 1 };

/* helm_setup - build a solver context.
 *   grid     grid of the problem (Sec. 2.1 / Sec. 5.2); every N >= 4, N_z <= 512, N_x N_y N_z even and
 *            below 2^31; N_x even for the tensor-core modes.
 *   k2       k^2(x,y,z) samples, complex128, N_x*N_y*N_z, host or device (Eq. problem).
 *   k0       background wavenumber of the ABC and of the preconditioner, real (Eq. background).
 *   k0z2     optional depth profile k0^2(z_l), N_z doubles (host), for K_z of Sec. 4.1; NULL = k0^2.
 *   opt      scheme order, preconditioner, precision, GMRES parameters.
 *   stream   cudaStream_t used for the set-up work; synchronised before return.
 *   out      receives the context.
 * Work: coefficient fields of Eq. scheme6 (fourth-order differences of k^2), the 1D eigendecompositions
 * Lbar_nu = V D V^-1 for nu = x, y (EigT step 1) on the GPU in FP64, checked by residual and by V^-1 V = I.
 * Errors: HELM_ERR_ARG, HELM_ERR_UNSUPPORTED, HELM_ERR_NOMEM, HELM_ERR_EIG, HELM_ERR_CUDA; *out = NULL then. */
helm_status helm_setup(const helm_grid* grid, const void* k2, double k0, const double* k0z2,
                       const helm_options* opt, void* stream, helm_ctx** out);

/* Boundary closure of a collocated grid's operator (helm_set_closure). */
enum { HELM_CLOSURE_THREE_POINT = 0, HELM_CLOSURE_HIGH_ORDER = 1 };

/* helm_set_closure - choose how the operator A (helm_apply_A, the solver's matvec, helm_residual) fills
 * the ghosts of a collocated grid.  The preconditioner keeps the three-point rule (EigT3) either way.
 *   HELM_CLOSURE_THREE_POINT  U_0 = U_2 + 2 i k0 h U_1 per direction (the default).
 *   HELM_CLOSURE_HIGH_ORDER   the high-order closure of the constant-k test problems (Sec. 2.1; the paper
 *     gives no formula, this is our reading): per face, with B the boundary node, I its interior
 *     neighbour and h the normal step, U_ghost = U_I + i k0 sum_{m=0..2} c_m (-1)^m L^m U_B with
 *     c_m = 2 h^(2m+1)/(2m+1)! and L = k0^2 + the two tangential second derivatives (sixth-order
 *     differences along the face, one-sided over eight nodes near its edges); faces filled x, then y,
 *     then z, each covering the ghost columns filled before it.  This is the U part of the closure; the
 *     closure's f part (s sum_m c_m sum_{j<m} (-L)^j d_n^(2(m-j)-1) f, s = +-1 on the far/near face) does
 *     not involve U and belongs to the right-hand side the caller passes to helm_gmres_solve, which
 *     helm_build_rhs does not form.
 * Each matvec first copies its operand into a padded array and fills the ghosts (seven small launches).
 * Memory: three padded copies ((N_x+2)(N_y+2)(N_z+2) points as complex64, complex128 and double-float)
 * and two scratch faces, allocated here and freed by helm_destroy or by HELM_CLOSURE_THREE_POINT.  The
 * scratch is shared by every operator call of the context: issue them on one stream (or order them), and
 * do not put the context in a batch (HELM_ERR_UNSUPPORTED there).
 * Errors: HELM_ERR_ARG (bad value), HELM_ERR_UNSUPPORTED (staggered grid, or an N below 8),
 * HELM_ERR_NOMEM. */
helm_status helm_set_closure(helm_ctx* ctx, int closure);

/* helm_build_rhs_fields - right-hand side of Eq. scheme4 / scheme6 from fields the caller knows (e.g. an
 * analytic f), in FP64; device complex128 buffers.
 *   order 4: fields = f on the padded grid, (N_x+2)(N_y+2)(N_z+2) values, x fastest, node (i,j,l) of the
 *            grid at padded index (i+1, j+1, l+1); F = f + sum_d (f_{+d} - 2 f + f_{-d})/12.
 *   order 6: fields = 7 grid arrays back to back: f, lap f, f_xxxx + f_yyyy + f_zzzz,
 *            f_xxyy + f_xxzz + f_yyzz, f_x, f_y, f_z; F = f + h^2/12 lap f + h^4/360 (pure) + h^4/90 (mixed)
 *            - h^2/20 (k^2 f - h^2/3 sum_d (k^2)_d f_d) with the context's sampled (k^2)_d.
 *   order 2: fields = f, F = f.
 * Errors: HELM_ERR_ARG (null or host pointer). */
helm_status helm_build_rhs_fields(helm_ctx* ctx, const void* fields, void* F, void* stream);

/* helm_closure_face_count - number of complex128 values helm_closure_rhs reads (0 for a staggered grid). */
long long helm_closure_face_count(helm_ctx* ctx);

/* helm_closure_rhs - F_out = F_in - A(G_f): moves the f part of the high-order closure to the right-hand
 * side (needs HELM_CLOSURE_HIGH_ORDER).  G_f is the ghost layer the closure gives for a zero interior
 * and the caller's face data, filled x, then y, then z like the operator's ghosts; its f part on a face
 * is s [c_1 f_n + c_2 (f_nnn - k0^2 f_n - lap_T f_n)] with s = -1 (near face) or +1 (far face).
 *   faces  device complex128, for axis x, y, z in turn, side near then far, fields f_n, f_nnn,
 *          lap_T f_n (derivatives along the axis, at the boundary coordinate), each over the face:
 *          x faces [N_z][N_y] (nodes 1..N); y faces [N_z][N_x + 2]; z faces [N_y + 2][N_x + 2], where an
 *          extent of N + 2 runs over the ghost column, the N nodes and the far ghost column (coordinates
 *          -h .. L + h).  helm_closure_face_count gives the total.
 *   F_in, F_out  device complex128 grids (may alias).  Synchronises the stream; allocates one grid.
 * Errors: HELM_ERR_ARG, HELM_ERR_UNSUPPORTED (closure not selected), HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_closure_rhs(helm_ctx* ctx, const void* faces, const void* F_in, void* F_out, void* stream);

/* helm_build_rhs - modified right-hand side F of the scheme from samples of f (Eqs. scheme4, scheme6).
 *   f  complex128 samples, host or device;  F  complex128 device output.  Order 2: F = f.
 * Derivatives of f and k^2 are sampled-data readings (fourth-order differences, mirror extension). */
helm_status helm_build_rhs(helm_ctx* ctx, const void* f, void* F, void* stream);

/* helm_apply_A - y = A x, the high-order operator with the ABC ghosts eliminated (Eqs. scheme4/scheme6,
 * Eq. D_bc).  dtype HELM_C64: complex64 arithmetic; HELM_C128: complex128 arithmetic.  x, y device. */
helm_status helm_apply_A(helm_ctx* ctx, const void* x, void* y, int dtype, void* stream);

/* helm_apply_precond - z = M^-1 r = h_z^2 A_p^-1 r, complex64 device buffers (may alias).  A_p is the
 * second-order constant-k0 operator with the same ABC (Kronecker form of Sec. 4.1); EigT (Eq. EIG_SOLVER)
 * or PFFT (Eq. PFFT_SOLVER) per the context's options, transforms in the context's precision. */
helm_status helm_apply_precond(helm_ctx* ctx, const void* r, void* z, void* stream);

/* helm_precond_step - one step of EigT on complex64 device buffers, for step-by-step checks:
 *   step 1: Ybar_l = V_y^-1 Y_l V_x^-T for every slice (forward transform, EigT step 2)
 *   step 2: the N_x N_y tridiagonal z-solves of Eq. Indep_precond_system (EigT step 3); in may equal out
 *   step 3: U_l = V_y Ubar_l V_x^T (inverse transform, EigT step 4)                                  */
helm_status helm_precond_step(helm_ctx* ctx, int step, const void* in, void* out, void* stream);

/* helm_get_eig - copy the FP64 1D eigendecomposition of axis 0 (x) or 1 (y) to host memory:
 * D (N complex128), V and Vinv (N*N complex128, row-major [row][col]).  Any pointer may be NULL. */
helm_status helm_get_eig(helm_ctx* ctx, int axis, void* D, void* V, void* Vinv);

/* helm_gmres_solve - solve A x = b by restarted right-preconditioned (or flexible) GMRES(m).
 *   b     complex128 right-hand side F (from helm_build_rhs), host or device.
 *   x     complex128, host or device; on entry x^0, on exit the iterate (also on NOT_CONVERGED).
 *   info  filled on return (may be NULL).
 * Host buffers: page-locked host memory that is mapped into the device address space (cudaHostAlloc, or
 * cudaHostRegister with mapping; the default for page-locked memory under unified addressing) is read and
 * written by the kernels directly over the host link, without staging copies; any other host memory is
 * copied to device buffers of the context and back.  The caller must not touch b or x until the call
 * returns.
 * Krylov vectors are complex64; inner products accumulate in compensated FP32 per thread and FP64 across
 * threads; the Hessenberg matrix and Givens rotations are FP64 on the GPU; x accumulates in double-float
 * (~44 bits); the stopping test uses the true residual in double-float.  A restart cycle ends after m
 * steps, at rtol, or once its residual estimate has fallen 1e-4 below the cycle's starting true residual
 * (a complex64 cycle cannot lower the true residual much further); the next cycle restarts from the true
 * residual.  Synchronises `stream`. */
helm_status helm_gmres_solve(helm_ctx* ctx, const void* b, void* x, helm_solve_info* info, void* stream);

/* helm_gmres_solve_batched - nrhs right-hand sides for each of nprob problems, solved together (an
 * extension: the paper solves one problem at a time).
 *   ctxs   nprob distinct contexts (any sizes, orders and options; EigT or no preconditioner; no attached
 *          net; the three-point closure on collocated grids)
 *   b[p]   complex128 device array [nrhs][nz][ny][nx] of problem p
 *   x[p]   complex128 device array of the same shape: x^0 on entry, the iterates on exit
 *   infos  nprob*nrhs entries (problem-major), may be NULL; seconds = wall time of the whole batch
 * Each (problem, right-hand side) pair runs the same restarted (F)GMRES as helm_gmres_solve with its own
 * Krylov workspace; the pairs run concurrently as branches of one CUDA graph whose loops and branches
 * (iterations, restarts, convergence) are decided on the device, so the host launches the graph once and
 * synchronises once per group of pairs that fits in 60% of the free device memory.
 * Returns HELM_OK when every pair converged, else the status of the first pair that did not (each pair's
 * status is in infos).  Errors: HELM_ERR_ARG (NULL, host pointers, a context twice), HELM_ERR_UNSUPPORTED
 * (PFFT or FFT2 context, attached net, or the high-order closure), HELM_ERR_NOMEM, HELM_ERR_CUDA.
 * Synchronises `stream`. */
helm_status helm_gmres_solve_batched(helm_ctx* const* ctxs, int nprob, const void* const* b, void* const* x, int nrhs,
                                     helm_solve_info* infos, void* stream);

/* Batch plans: the lanes' workspaces and the instantiated restart-cycle graph of helm_gmres_solve_batched,
 * built once and run many times (the set-up stays out of repeated solves).
 * helm_batch_create - plan for the same arguments as helm_gmres_solve_batched; b and x are read and written
 *   by every helm_batch_run (their contents may change between runs, not their addresses).  All lanes must
 *   fit in 85% of the free device memory (else HELM_ERR_NOMEM; helm_gmres_solve_batched splits instead).
 * helm_batch_run - solve every lane from the current b and x0 (as helm_gmres_solve_batched; infos
 *   problem-major, seconds = this run).  Synchronises `stream`.
 * helm_batch_destroy - free the plan (NULL is a no-op); the contexts must outlive it. */
typedef struct helm_batch helm_batch;
helm_status helm_batch_create(helm_ctx* const* ctxs, int nprob, const void* const* b, void* const* x, int nrhs,
                              void* stream, helm_batch** out);
helm_status helm_batch_run(helm_batch* batch, helm_solve_info* infos, void* stream);
void helm_batch_destroy(helm_batch* batch);

/* helm_autotune - time, on this context's grid, the candidate CTA counts of the Arnoldi update and combine
 * kernels, the variants of the complex64 matvec (see helm_set_matvec_variant) and of the inner-product
 * kernel (0: groups of eight, 1/2:
 * software-pipelined groups of four/eight); in TF32 contexts the tensor-core transform passes (persistent
 * with double-buffered accumulators, or one tile per CTA), timed on a preconditioner application; in EigT
 * contexts with even N_x the factorised z-solve (the L2-resident kernel at 1-3 CTAs per SM, or one thread
 * per line).  The fastest of each is kept for the context's later solves; *nb_out, *variant_out and
 * *dots_out (any may be NULL) receive the first three choices.  Results are cached per grid size and order
 * for the process.  Uses temporary device memory; synchronous. */
helm_status helm_autotune(helm_ctx* ctx, int* nb_out, int* variant_out, int* dots_out, void* stream);

/* helm_residual - r = b - A x and its norms, the rel-res numerator of Sec. 5.1, computed with about 44
 * significant bits (double-float arithmetic on the FP32 pipes) from complex128 b and x.
 *   b, x   complex128 device buffers;  r  complex64 device output (may be NULL);
 *   nrm2   receives ||b - A x||_2, nrmi receives ||b - A x||_inf (either may be NULL).
 * Synchronises `stream`. */
helm_status helm_residual(helm_ctx* ctx, const void* b, const void* x, void* r, double* nrm2, double* nrmi,
                          void* stream);

/* helm_residual_noalloc - the same residual and norms as helm_residual, for callers that cannot allocate
 * device memory while they run: an application that has handed the whole device to its own memory pool
 * after warm-up, or a runtime that forbids cudaMalloc/cudaFree (which synchronise the device) between its
 * steps.  helm_residual allocates its double-float copies of b and x on first use; this entry point keeps
 * them in a fixed static device array instead.  The paper has no counterpart: this is a library
 * convenience.
 *   b, x   complex128 device buffers;  r  complex64 device output (required);  nrm2, nrmi as above.
 * Allocates nothing and calls no allocating library routine.  Its scratch (double-float copies of b and x,
 * per-CTA partial sums, two result words) is one static device array of 65 MiB + 256 B that every GPU
 * loading the library holds until the process exits.  Limit: at most 2^21 = 2,097,152 grid points (128^3)
 * and 65536 residual CTAs; larger problems return HELM_ERR_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current).  Every call shares the array
 * and rewrites each part of it that it reads before reading it, so calls whose GPU work overlaps (two
 * streams, two host threads) race and must be serialised by the caller.  Like helm_residual it copies the
 * two norms to host memory and synchronises `stream` before returning. */
helm_status helm_residual_noalloc(helm_ctx* ctx, const void* b, const void* x, void* r, double* nrm2,
                                  double* nrmi, void* stream);

/* helm_profile - enable (1) or disable (0) per-kernel timing on this context: CUDA events are recorded
 * on the launch stream around every kernel launch of the solver (adds no synchronisation).  The first
 * call allocates the event pool (host-side cost only). */
helm_status helm_profile(helm_ctx* ctx, int enable);

/* helm_profile_classes - as helm_profile, but events are recorded only around the launches of the kernel
 * classes whose bits are set in mask (bit i = class i in the order of helm_profile_read; mask 0 disables
 * timing).  Timing one class keeps the events off the rest of the solve, whose launches then follow one
 * another without them.  Measurement only: the paper has no counterpart. */
helm_status helm_profile_classes(helm_ctx* ctx, unsigned mask);

/* helm_profile_read - accumulated milliseconds and launch counts per kernel class since the last reset,
 * in the order: stencil (complex64 A), x-pass, y-pass, z-solve, Arnoldi dots, Arnoldi update,
 * small FP64 kernels (reductions, Givens, least squares), solution update, FP64 true residual, other,
 * learned correction.
 *   ms, launches  host arrays of n entries (either may be NULL);  reset != 0 clears the counters.
 * Synchronises on the recorded events. */
helm_status helm_profile_read(helm_ctx* ctx, double* ms, long long* launches, int n, int reset);

/* ---- Learned correction (an extension: the paper has no counterpart) ----------------------------------
 * A small 3D U-Net N, applied after M^-1 inside flexible GMRES:
 *     c = s N(x),   s = RMS(M^-1 v),
 *     x = [Re v, Im v]/RMS(v), [Re, Im](M^-1 v)/s, Re(k^2)/k0^2 - 1      (5 channels)
 *     z = M^-1 v + alpha c,   alpha = <A c, v - A M^-1 v>/<A c, A c>   (complex64 stencil A of the context)
 * alpha minimises |v - A z|_2, so the corrected z never has a larger preconditioned residual than M^-1 v
 * (plain EigT is the fallback).  The correction is dropped (z = M^-1 v) when A c = 0 or a sum is not finite.
 * Network of width c: a1 = relu(conv(x,5->c)), a2 = relu(conv(a1,c->c)), p = avgpool2(a2),
 * b1 = relu(conv(p,c->2c)), b2 = relu(conv(b1,2c->2c)), u = [upsample2(b2), a2],
 * d1 = relu(conv(u,3c->c)), N = conv(d1,c->2); 3x3x3 convolutions, zero padding.
 * Parameters (float32, in this order, per layer l = 1..6): weights [Cout][Cin][3][3][3], then bias [Cout].
 * Activations are stored in bfloat16 with float32 accumulation; training keeps float32 master weights.
 * Tensors are [B][C][Z][Y][X] (X fastest), Z, Y, X even.  A net is used by one stream at a time. */
typedef struct helm_net helm_net;

/* helm_net_create - new network of width c (1..64), He-normal weights from `seed` (last layer x0.1),
 * zero biases.  Errors: HELM_ERR_ARG, HELM_ERR_NOMEM, HELM_ERR_CUDA; *out = NULL then. */
helm_status helm_net_create(int width, unsigned long long seed, helm_net** out);
/* helm_net_destroy - free (NULL is a no-op).  Detach it from every context first. */
void helm_net_destroy(helm_net* net);
/* helm_net_num_params - number of float32 parameters (0 for NULL). */
size_t helm_net_num_params(const helm_net* net);
/* helm_net_set_params / get_params / get_grads - host float32 arrays of exactly num_params entries;
 * synchronous.  set_params also refreshes the bfloat16 copy.  Errors: HELM_ERR_ARG on a size mismatch. */
helm_status helm_net_set_params(helm_net* net, const float* host, size_t count);
helm_status helm_net_get_params(helm_net* net, float* host, size_t count);
helm_status helm_net_get_grads(helm_net* net, float* host, size_t count);
/* helm_net_zero_grad - clear the accumulated parameter gradients (stream-ordered). */
helm_status helm_net_zero_grad(helm_net* net, void* stream);
/* helm_net_forward - y = N(x) for a batch: x bfloat16 device [B][5][Z][Y][X], y float32 device
 * [B][2][Z][Y][X].  Keeps the activations for helm_net_backward.  Grows the workspace on demand. */
helm_status helm_net_forward(helm_net* net, const void* x, float* y, int B, int Z, int Y, int X, void* stream);
/* helm_net_backward - accumulates dL/dparams for dL/dy = gy (float32 device, shape of the last forward's y)
 * into the gradients.  Needs a preceding helm_net_forward on the same net. */
helm_status helm_net_backward(helm_net* net, const float* gy, void* stream);
/* helm_net_adam - one Adam step (Kingma and Ba) with bias correction for step number `step` (>= 1). */
helm_status helm_net_adam(helm_net* net, float lr, float beta1, float beta2, float eps, int step, void* stream);
/* helm_net_mse - loss += 0.5 mean((y - t)^2) into the device double *loss (caller zeroes it), and
 * gy = (y - t)/count; float32 device arrays of `count` entries. */
helm_status helm_net_mse(const float* y, const float* t, float* gy, size_t count, double* loss, void* stream);
/* helm_net_features - the 5 input channels x (bfloat16 device [5][nz][ny][nx]) for v and mv = M^-1 v
 * (complex64 device) on the context's grid and k^2. */
helm_status helm_net_features(helm_ctx* ctx, helm_net* net, const void* v, const void* mv, void* x, void* stream);
/* helm_net_target - the training target t = (xs - xk - mv)/RMS(mv) (float32 device [2][nz][ny][nx]) for
 * the pair v = b - A xk, A^-1 v = xs - xk, where xs solves A xs = b and mv = M^-1 v (complex64);
 * xs, xk complex128 device fields of the context's grid. */
helm_status helm_net_target(helm_ctx* ctx, helm_net* net, const void* xs, const void* xk, const void* mv, float* t,
                            void* stream);
/* helm_net_stats - six doubles: sum |v|^2 and sum |M^-1 v|^2 of the last correction, its |alpha|, the
 * numbers of corrections dropped and applied since the net was created, and the sum over the applied ones
 * of |v - A z|^2/|v - A M^-1 v|^2 (the residual reduction the correction bought).  Synchronous. */
helm_status helm_net_stats(helm_net* net, double* host6);
/* helm_attach_net - apply `net` after M^-1 in helm_apply_precond and helm_gmres_solve of this context
 * (NULL detaches).  The context does not own the net.  Requires a flexible context and even nx, ny, nz
 * (else HELM_ERR_ARG); sizes the net's workspace for one field of the grid. */
helm_status helm_attach_net(helm_ctx* ctx, helm_net* net);

/* helm_set_wait_limit - bound, in polls, of every mbarrier wait of this context's tensor-core transform
 * passes and of its TMA matvec (0 restores the default, 2^20).  A wait that runs out raises a device
 * status bit; the CTA then skips its remaining work, waits (under a separate fixed bound) for the TMA loads
 * and MMAs it still has in flight, frees its tensor memory and exits, and the next synchronising call
 * (helm_gmres_solve, helm_gmres_solve_batched, helm_batch_run) returns HELM_ERR_ITER_LIMIT; the context
 * stays usable.  A diagnosis and test hook: a limit of a few polls makes the waits run out on purpose.
 * The paper has no counterpart.  Errors: HELM_ERR_ARG (NULL context, negative limit). */
helm_status helm_set_wait_limit(helm_ctx* ctx, long long polls);

/* helm_set_matvec_variant - pin the kernel of the context's complex64 matvec (staggered grids of order 4
 * or 6; other contexts use the general stencil kernel whatever is set):
 *   0  cp.async plane ring, one output per thread, four CTAs per SM
 *   1  TMA plane ring (even N_x; else as 0)
 *   2  cp.async plane ring, three CTAs per SM (the default for complex k^2)
 *   3  two outputs per thread, k^2 U in registers (real k^2; the default for a real medium; else as 2)
 *   4  as 3 with the sixth-order fields formed from a two-point-halo k^2 ring (real k^2, order 6; else as 3)
 * All compute the same operator (Eqs. scheme4/scheme6) in complex64; they differ in speed and bytes moved.
 * helm_autotune overrides the choice with the fastest.  Errors: HELM_ERR_ARG (NULL, out of range). */
helm_status helm_set_matvec_variant(helm_ctx* ctx, int variant);

/* helm_destroy - free the context and its device workspace (NULL is a no-op). */
void helm_destroy(helm_ctx* ctx);

/* helm_status_str - static English text of a status code. */
const char* helm_status_str(int status);

/* helm_last_error - text of the last CUDA failure that made a call on this host thread return
 * HELM_ERR_CUDA or HELM_ERR_NOMEM ("" if none); static storage per thread. */
const char* helm_last_error(void);

/* helm_version - library version string. */
const char* helm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
