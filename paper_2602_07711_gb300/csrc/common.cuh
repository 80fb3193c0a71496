// Internal declarations shared by the translation units of libhelm (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include "../../include/helm.h"

#define HELM_CUDA_TRY(expr)                                          \
    do {                                                             \
        cudaError_t e__ = (expr);                                    \
        if (e__ != cudaSuccess) return helm_fail_cuda(e__, #expr);   \
    } while (0)

helm_status helm_fail_cuda(cudaError_t e, const char* what);

// Device status word bits (OR-ed by kernels, read by synchronising calls).
enum : unsigned {
    HELM_DEV_PIVOT = 1u,      // tiny tridiagonal pivot
    HELM_DEV_NAN = 2u,        // NaN/Inf in a reduction
    HELM_DEV_WAIT = 4u,       // a bounded device wait expired
    HELM_DEV_EIG = 8u         // eigen-setup check failed
};

// ---- complex helpers -------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { typedef float2 t; };
template <> struct cplx<double> { typedef double2 t; };

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ inline C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ inline C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C, typename R> __host__ __device__ inline C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __host__ __device__ inline C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ inline C cconjmul(C a, C b) {  // conj(a) * b
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> __host__ __device__ inline C cfma(C a, C b, C c) {  // a*b + c
    c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
    return c;
}
template <typename C> __host__ __device__ inline C cdiv(C a, C b) {
    // Smith's algorithm
    C r;
    if (fabs(b.x) >= fabs(b.y)) {
        auto t = b.y / b.x; auto d = b.x + b.y * t;
        r.x = (a.x + a.y * t) / d; r.y = (a.y - a.x * t) / d;
    } else {
        auto t = b.x / b.y; auto d = b.x * t + b.y;
        r.x = (a.x * t + a.y) / d; r.y = (a.y * t - a.x) / d;
    }
    return r;
}
template <typename C> __host__ __device__ inline double cabs2(C a) { return (double)a.x * a.x + (double)a.y * a.y; }

// ---- stencil coefficient bundle (passed by value to kernels) --------------------------------
template <typename R>
struct StencilParams {
    int nx, ny, nz;
    R hx, hy, hz;
    typename cplx<R>::t gx, gy, gz;      // ghost factors (Eq. D_bc)
    const typename cplx<R>::t* k2;       // k^2 samples
    const typename cplx<R>::t* dk2[3];   // (k^2)_x, (k^2)_y, (k^2)_z  (order 6)
    const typename cplx<R>::t* G;        // lap(k^2) - k^4             (order 6)
};

// ---- the context -----------------------------------------------------------------------------
struct KrylovWork;
struct helm_net;

// Optional per-kernel timing: CUDA events recorded on the launch stream around every launch.
enum ProfClass { PROF_STENCIL = 0, PROF_XPASS, PROF_YPASS, PROF_ZSOLVE, PROF_DOTS, PROF_UPDATE, PROF_SMALL,
                 PROF_COMBINE, PROF_RESIDUAL, PROF_OTHER, PROF_LEARNED, PROF_NCLASS };
struct Prof {
    int enabled = 0;
    unsigned mask = ~0u;   // classes that are timed
    int open = 0;          // the last prof_begin recorded an event
    int used = 0;
    static constexpr int CAP = 16384;
    cudaEvent_t ev[CAP];
    int cls[CAP / 2];
    double ms[PROF_NCLASS] = {0};
    long long launches[PROF_NCLASS] = {0};
    int created = 0;
};
void prof_begin(helm_ctx* c, cudaStream_t s, int cls);
void prof_end(helm_ctx* c, cudaStream_t s);
void prof_flush(helm_ctx* c);
void prof_release(helm_ctx* c);

struct helm_ctx {
    int device;
    helm_grid grid;
    helm_options opt;
    int nx, ny, nz;
    size_t npts;
    double h[3];
    double k0;
    double ax, ay;                 // alpha_d = h_z^2/h_d^2
    double2 gam[3];                // corner entry of Lbar: two-point ghost factor (staggered), 2 i k0 h (collocated)
    double zeta[3];                // corner neighbour of Lbar: 1 staggered, 2 collocated
    int colloc = 0;                // collocated grid: ghost U_0 = U_2 + 2 i k0 h U_1 per direction
    int ho = 0;                    // collocated high-order closure (helm_set_closure): padded operands
    float2* ho_P32 = nullptr;      // padded (nx+2)(ny+2)(nz+2) copies of the operand, per storage type
    double2* ho_P64 = nullptr;
    float4* ho_Pdf = nullptr;
    double2* ho_S = nullptr;       // scratch faces L U_B, both sides
    // coefficient fields
    double2* k2_d = nullptr;
    float2* k2_f = nullptr;
    double2* dk2_d[3] = {nullptr, nullptr, nullptr};
    float2* dk2_f[3] = {nullptr, nullptr, nullptr};
    double2* G_d = nullptr;
    float2* G_f = nullptr;
    float4* k2_df = nullptr;                // double-float k^2 and G for the true residual
    float4* G_df = nullptr;
    float4* rhs_scratch = nullptr;          // double-float copy of f for helm_build_rhs
    // 1D eigendecompositions, FP64 (row-major [row][col])
    double2 *Dx = nullptr, *Dy = nullptr, *Vx = nullptr, *Vxi = nullptr, *Vy = nullptr, *Vyi = nullptr;
    // complex64 transform operands
    float2 *XF = nullptr, *XI = nullptr;    // B of the x-pass: V_x^-T (forward), V_x^T (inverse)
    float2 *YF = nullptr, *YI = nullptr;    // A of the y-pass: V_y^-1 (forward), V_y (inverse)
    float2 *dxs = nullptr, *dys = nullptr;  // alpha_x D_x, alpha_y D_y
    float2 *cz = nullptr;                   // h_z^2 k0^2(z_l) - 2(alpha_x + alpha_y + 1)
    float2 *zfac = nullptr;                 // Thomas factors m of the EigT z-systems, one per point
    // tensor-core operands, allocated for the TF32 mode
    float *XFr = nullptr, *XIr = nullptr;   // real-embedded x-pass B, [2N][2K] K-major (hi, lo follow)
    float *YFr = nullptr, *YIr = nullptr;   // y-pass A: re and im planes [2][N][N] (hi, lo follow)
    void* tmaps = nullptr;                  // host copies of TMA descriptors (gemm_tc.cu)
    void* pfft = nullptr;                   // PFFT tables and scratch (pfft.cu)
    float* k2r = nullptr;                   // real k^2 and real (G, g_x, g_y, g_z) for media without attenuation
    float4* fr = nullptr;
    float2* rkq = nullptr;                  // sixth-order residual, real media: k^2 h^2 / 3 (double-float)
    float4* rg4 = nullptr;                  // ... (3/2) h^4 G (double-float), (3/2) h^3 (g_x, g_y) (FP32)
    float* rgz = nullptr;                   // ... (3/2) h^3 g_z
    int realk = 0;
    float h16s[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f};   // FP16 chain: input, four stage scales, final factor
    double* h16n = nullptr;                 // FP16 chain: 1/||r||, ||r|| and partial sums (helm_apply_precond)
    double* h16d = nullptr;                 // FP16 chain, per application: ||T1||^2, ||T2||^2, ||T3||^2, -, s2, s3, s4, 1/(s2 s3 s4)
    float h16g[3] = {1.f, 1.f, 1.f};        // FP16 chain: norm bounds of the y-pass forward, z-solve, y-pass inverse
    cudaEvent_t h16_join = nullptr;         // FP16 basis: an event the chain's last pass waits for (the step's scale)
    void* sfast = nullptr;                  // TMA descriptors of the stencil's fixed operands (stencil_fast.cu)
    // scratch
    float2* tmp = nullptr;                  // one complex64 grid vector
    unsigned* status_d = nullptr;           // device status word
    KrylovWork* kw = nullptr;
    helm_net* net = nullptr;                // attached learned correction (not owned)
    int tune_nb = 0;                        // CTAs of the Arnoldi kernels chosen by helm_autotune (0 = default)
    int tune_stencil = 0;                   // complex64 matvec variant chosen by helm_autotune (0 = cp.async ring)
    int zring_sms = 0;                      // SM count, set with the ring kernel's attributes at set-up
    int zpiv_ready = 0;                     // shared-memory attribute of the pivot-recomputing z-solve set
    void* zck = nullptr;                    // pivot checkpoints of that z-solve ([block][line pair] float4)
    int zpiv_off = 0;                       // set while capturing launches that may run concurrently (batch lanes)
    int zck_slot = 0;                       // first checkpoint slot of the z-solve launches being captured (batch plans)
    size_t zck_bytes = 0;
    int tune_zring = 2;                     // factorised z-solve: CTAs per SM of the L2-resident ring kernel (0 = one thread per line)
    int tune_ypers = 1;                     // y-pass: 1 persistent with double-buffered accumulators, 0 one tile per CTA
    int tune_tc = 1;                        // x-pass on the tensor cores: 1 persistent, 0 one tile per CTA
    int tune_dots = 2;                      // inner-product kernel variant (helm_autotune; 2 measured best)
    cudaStream_t last_stream = nullptr;
    Prof* prof = nullptr;
    long long wait_limit = 1LL << 20;       // polls of each bounded mbarrier wait (helm_set_wait_limit)
};

// ---- launchers shared across translation units -----------------------------------------------
// stencil.cu
helm_status launch_derived_fields(helm_ctx* c, cudaStream_t s);
// closure.cu: padded operand with the high-order collocated closure ghosts
helm_status closure_fill_f32(helm_ctx* c, const float2* U, cudaStream_t s);
helm_status closure_fill_f64(helm_ctx* c, const double2* U, cudaStream_t s);
helm_status closure_fill_df(helm_ctx* c, const float4* U, cudaStream_t s);
void closure_release(helm_ctx* c);
size_t closure_face_points(const helm_ctx* c);
helm_status closure_rhs(helm_ctx* c, const double2* faces, const double2* Fin, double2* Fout, cudaStream_t s);
helm_status launch_stencil_f64_padded(helm_ctx* c, const double2* P, double2* y, cudaStream_t s);
helm_status launch_rhs_fields(helm_ctx* c, const double2* fields, double2* F, cudaStream_t s);
helm_status launch_stencil_f32(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, cudaStream_t s);
helm_status launch_stencil_f32_cls(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, int cls,
                                   cudaStream_t s);   // timed under profiling class cls
// the complex64 matvec of nb vectors stored npts apart (the right-hand sides of a batch group)
helm_status launch_stencil_f32_nb(helm_ctx* c, const float2* x, float2* y, int nb, cudaStream_t s);
helm_status launch_stencil_f64(helm_ctx* c, const double2* x, double2* y, cudaStream_t s);
helm_status launch_residual(helm_ctx* c, const float4* x, const float4* F, float2* r, double* part, cudaStream_t s);
helm_status launch_rhs(helm_ctx* c, const double2* f, double2* F, float4* fdf, cudaStream_t s);
// stencil_fast.cu: the complex64 matvec of orders 4 and 6 (cp.async plane ring, plane-quantity form)
helm_status stencil_fast_prepare(helm_ctx* c);
helm_status stencil_real_prepare(helm_ctx* c, cudaStream_t s);
void stencil_fast_release(helm_ctx* c);
int stencil_variants(const helm_ctx* c);
helm_status residual_fast_prepare();
helm_status residual_real_prepare(helm_ctx* c, cudaStream_t s);
void residual_real_release(helm_ctx* c);
helm_status launch_residual_fast(helm_ctx* c, const float4* x, const float4* F, float2* r, double* part,
                                 cudaStream_t s);   // same grid (and partial count) as the generic residual
bool stencil_fast_supported(const helm_ctx* c);
helm_status launch_stencil_fast(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, cudaStream_t s,
                                int nb = 1);
// eig.cu
helm_status run_eig_setup(helm_ctx* c, cudaStream_t s);
// gemm_simt.cu
// rows of C: row r scales by alpha_dev[aidx + (r / rows_per) astride] (rows_per = 0: alpha_dev[aidx] for all)
void launch_cgemm_simt(int M, int N, int K, const float2* A, long lda, long sA, const float2* B, long ldb, long sB,
                       float2* C, long ldc, long sC, int batch, float alpha, const double* alpha_dev, int aidx,
                       cudaStream_t s, int rows_per = 0, int astride = 0);
// gemm_tc.cu
helm_status tc_prepare(helm_ctx* c, cudaStream_t s);
// nb > 1: nb grid vectors back to back (a batch group); the x-pass scales vector v by alpha_dev[aidx + v astride]
helm_status tc_xpass(helm_ctx* c, int inverse, const float2* in, float2* out, float alpha, const double* alpha_dev,
                     int aidx, cudaStream_t s, int nb = 1, int astride = 0);
helm_status tc_ypass(helm_ctx* c, int inverse, const float2* in, float2* out, cudaStream_t s, int nb = 1);
helm_status tc_xpass_h16(helm_ctx* c, int inverse, const void* in, void* out, int out_h16, float alpha,
                         const double* alpha_dev, int aidx, cudaStream_t s, int nb = 1, int astride = 0,
                         const double* alpha_dev2 = nullptr, double* nsq_out = nullptr);
helm_status tc_ypass_h16(helm_ctx* c, int inverse, const void* in, void* out, float alpha, cudaStream_t s, int nb = 1,
                         double* h16d = nullptr, float gain = 1.f);
helm_status h16_scales(helm_ctx* c, cudaStream_t s);
helm_status precond_h16_basis(helm_ctx* c, const uint16_t* V16, float2* z, const double* cs, int cidx, cudaStream_t s);
helm_status to_h16_basis(helm_ctx* c, const float2* r, uint16_t* V16, const double* sigma, int sidx, cudaStream_t s);
helm_status launch_zsolve_h16(helm_ctx* c, const void* in, void* out, float4* dscr, float oscale, cudaStream_t s,
                              int nb = 1, double* h16d = nullptr, float gain = 1.f);
// operand sets of tc_xpass/tc_ypass (`inverse`): 0/1 EigT forward/inverse, 2/3 PFFT sine forward/inverse
helm_status tc_prepare_sine(helm_ctx* c, const double2* Sx, const double2* Sy, const double2* SxT, const double2* SyT,
                            cudaStream_t s);
void tc_release(helm_ctx* c);
// thomas.cu
helm_status zsolve_reserve(helm_ctx* c, int nb);
helm_status launch_zsolve(helm_ctx* c, const float2* in, float2* out, cudaStream_t s, int nb = 1);
helm_status zsolve_factor(helm_ctx* c, cudaStream_t s);
helm_status zsolve_factor_with(helm_ctx* c, const float2* dxs, const float2* dys, float2** m, cudaStream_t s);
helm_status launch_zsolve_fact(helm_ctx* c, const float2* m, const float2* in, float2* out, const float2* P,
                               const float2* Q, cudaStream_t s, int nb = 1);
helm_status launch_zsolve_gen(helm_ctx* c, const float2* in, float2* out, const float2* dxs, const float2* dys,
                              const float2* P, const float2* Q, cudaStream_t s);
// pfft.cu
helm_status pfft_prepare(helm_ctx* c, cudaStream_t s);
helm_status pfft_apply(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s);
helm_status pfft_apply_dirichlet(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx,
                                 cudaStream_t s);
void pfft_release(helm_ctx* c);
// learned.cu: the two halves of the learned correction around M^-1 (features and a copy of
// v = sigma[sidx] r before, the correction of z after; r and z may alias)
helm_status learned_pre(helm_ctx* c, const float2* r, const double* sigma, int sidx, cudaStream_t s);
helm_status learned_post(helm_ctx* c, float2* z, cudaStream_t s);
// precond.cu
helm_status precond_apply(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s);
helm_status precond_step(helm_ctx* c, int step, const float2* in, float2* out, cudaStream_t s);
helm_status precond_apply_nb(helm_ctx* c, const float2* r, float2* z, int nb, const double* sigma, int sidx,
                             int sstride, cudaStream_t s);
// krylov.cu
helm_status gmres_run(helm_ctx* c, const double2* b, double2* x, helm_solve_info* info, cudaStream_t s);
void krylov_free(helm_ctx* c);
helm_status residual_run(helm_ctx* c, const double2* b, const double2* x, float2* r, double* nrm2, double* nrmi,
                         cudaStream_t s);
