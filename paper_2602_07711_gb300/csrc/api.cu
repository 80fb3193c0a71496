// C-ABI entry points (include/helm.h): argument checks, context set-up and teardown, dispatch.
#include "common.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

// text of the last CUDA failure seen on this host thread (helm_last_error)
static thread_local char g_last_error[512] = "";

helm_status helm_fail_cuda(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", what ? what : "?", cudaGetErrorString(e), (int)e);
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    cudaGetLastError();
    return HELM_ERR_CUDA;
}

extern "C" const char* helm_last_error(void) { return g_last_error; }

namespace {

bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
helm_status dalloc(T** p, size_t n) {
    if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    return HELM_OK;
}

void free_ctx(helm_ctx* c) {
    if (!c) return;
    krylov_free(c);
    tc_release(c);
    pfft_release(c);
    stencil_fast_release(c);
    closure_release(c);
    prof_release(c);
    void* ps[] = {c->k2_d, c->k2_f, c->dk2_d[0], c->dk2_d[1], c->dk2_d[2], c->dk2_f[0], c->dk2_f[1], c->dk2_f[2],
                  c->G_d, c->G_f, c->Dx, c->Dy, c->Vx, c->Vxi, c->Vy, c->Vyi, c->XF, c->XI, c->YF, c->YI,
                  c->dxs, c->dys, c->cz, c->tmp, c->status_d, c->k2_df, c->G_df, c->rhs_scratch, c->zfac, c->zck, c->h16n, c->h16d};
    for (void* p : ps) if (p) cudaFree(p);
    delete c;
}

#define TRY(x) do { helm_status s__ = (x); if (s__ != HELM_OK) { free_ctx(c); return s__; } } while (0)

}  // namespace

extern "C" {

const char* helm_version(void) { return "helm-gb300 0.1 (sm_103a)"; }

const char* helm_status_str(int s) {
    switch (s) {
        case HELM_OK: return "ok";
        case HELM_ERR_ARG: return "invalid argument";
        case HELM_ERR_CUDA: return "CUDA error";
        case HELM_ERR_NOMEM: return "out of device memory";
        case HELM_ERR_EIG: return "1D eigendecomposition failed its check";
        case HELM_ERR_PIVOT: return "tiny tridiagonal pivot";
        case HELM_ERR_NAN: return "NaN or Inf in the iteration";
        case HELM_ERR_BREAKDOWN: return "GMRES breakdown";
        case HELM_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case HELM_ERR_ITER_LIMIT: return "device wait exceeded its cap";
        case HELM_ERR_UNSUPPORTED: return "configuration not supported";
        default: return "unknown status";
    }
}

helm_status helm_setup(const helm_grid* grid, const void* k2, double k0, const double* k0z2, const helm_options* opt,
                       void* stream, helm_ctx** out) {
    if (!out) return HELM_ERR_ARG;
    *out = nullptr;
    if (!grid || !k2 || !opt) return HELM_ERR_ARG;
    if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4) return HELM_ERR_ARG;
    if (!(grid->lx > 0 && grid->ly > 0 && grid->lz > 0)) return HELM_ERR_ARG;
    if (opt->order != 2 && opt->order != 4 && opt->order != 6) return HELM_ERR_ARG;
    if (opt->restart < 1 || opt->restart > 64 || opt->max_iter < 1 || !(opt->rtol > 0)) return HELM_ERR_ARG;
    if (opt->precond < 0 || opt->precond > 3 || opt->precision < 0 || opt->precision > 4) return HELM_ERR_ARG;
    const int colloc = grid->staggered ? 0 : 1;
    // the Krylov kernels move two points per 16-byte access: the point count must be even
    if (((size_t)grid->nx * grid->ny * grid->nz) % 2 != 0) return HELM_ERR_UNSUPPORTED;
    if (grid->nz > 512) return HELM_ERR_UNSUPPORTED;
    // point indices fit a signed 32-bit integer (grid offsets themselves are size_t)
    if ((size_t)grid->nx * grid->ny * grid->nz >= ((size_t)1 << 31)) return HELM_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    helm_ctx* c = new helm_ctx();
    cudaGetDevice(&c->device);
    c->grid = *grid;
    c->opt = *opt;
    c->nx = grid->nx; c->ny = grid->ny; c->nz = grid->nz;
    c->npts = (size_t)c->nx * c->ny * c->nz;
    c->colloc = colloc;
    // staggered: nodes h/2 + j h, h = L/N (Sec. 5.2); collocated: nodes j h, h = L/(N-1) (Sec. 2.1)
    c->h[0] = grid->lx / (grid->nx - colloc); c->h[1] = grid->ly / (grid->ny - colloc);
    c->h[2] = grid->lz / (grid->nz - colloc);
    if (opt->order == 6) {
        const double tol = 1e-12 * c->h[0];
        if (fabs(c->h[1] - c->h[0]) > tol || fabs(c->h[2] - c->h[0]) > tol) { delete c; return HELM_ERR_ARG; }
    }
    c->k0 = k0;
    c->ax = c->h[2] * c->h[2] / (c->h[0] * c->h[0]);
    c->ay = c->h[2] * c->h[2] / (c->h[1] * c->h[1]);
    for (int d = 0; d < 3; ++d) {
        const double a = k0 * c->h[d], den = 4.0 + a * a;
        if (colloc) {
            // central difference of du/dn = i k0 u at the boundary node: U_0 = U_2 + 2 i k0 h U_1, which puts
            // gamma = 2 i k0 h on the corner of Lbar and zeta = 2 next to it (Sec. 4.1)
            c->gam[d] = make_double2(0.0, 2.0 * a);
            c->zeta[d] = 2.0;
        } else {
            // gamma = (2 + i k0 h)/(2 - i k0 h), Eq. D_bc
            c->gam[d] = make_double2((4.0 - a * a) / den, 4.0 * a / den);
            c->zeta[d] = 1.0;
        }
    }
    const size_t n = c->npts;
    TRY(dalloc(&c->k2_d, n));
    TRY(dalloc(&c->k2_f, n));
    TRY(dalloc(&c->k2_df, n));
    if (opt->order == 6) {
        for (int d = 0; d < 3; ++d) { TRY(dalloc(&c->dk2_d[d], n)); TRY(dalloc(&c->dk2_f[d], n)); }
        TRY(dalloc(&c->G_d, n));
        TRY(dalloc(&c->G_f, n));
        TRY(dalloc(&c->G_df, n));
    }
    TRY(dalloc(&c->tmp, n));
    TRY(dalloc(&c->status_d, 1));
    if (cudaMemsetAsync(c->status_d, 0, sizeof(unsigned), s) != cudaSuccess) { free_ctx(c); return HELM_ERR_CUDA; }
    if (cudaMemcpyAsync(c->k2_d, k2, n * sizeof(double2), dev_ptr(k2) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s) != cudaSuccess) { free_ctx(c); return HELM_ERR_CUDA; }
    TRY(launch_derived_fields(c, s));
    TRY(stencil_fast_prepare(c));
    TRY(stencil_real_prepare(c, s));
    TRY(residual_real_prepare(c, s));
    // eigen set-up
    TRY(dalloc(&c->Dx, c->nx)); TRY(dalloc(&c->Dy, c->ny));
    TRY(dalloc(&c->Vx, (size_t)c->nx * c->nx)); TRY(dalloc(&c->Vxi, (size_t)c->nx * c->nx));
    TRY(dalloc(&c->Vy, (size_t)c->ny * c->ny)); TRY(dalloc(&c->Vyi, (size_t)c->ny * c->ny));
    TRY(dalloc(&c->XF, (size_t)c->nx * c->nx)); TRY(dalloc(&c->XI, (size_t)c->nx * c->nx));
    TRY(dalloc(&c->YF, (size_t)c->ny * c->ny)); TRY(dalloc(&c->YI, (size_t)c->ny * c->ny));
    TRY(dalloc(&c->dxs, c->nx)); TRY(dalloc(&c->dys, c->ny)); TRY(dalloc(&c->cz, c->nz));
    TRY(run_eig_setup(c, s));
    {
        std::vector<float2> czh(c->nz);
        const double hz2 = c->h[2] * c->h[2];
        for (int l = 0; l < c->nz; ++l) {
            const double kz2 = k0z2 ? k0z2[l] : k0 * k0;
            czh[l] = make_float2((float)(hz2 * kz2 - 2.0 * (c->ax + c->ay + 1.0)), 0.f);
        }
        if (cudaMemcpyAsync(c->cz, czh.data(), c->nz * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            free_ctx(c); return HELM_ERR_CUDA;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) { free_ctx(c); return HELM_ERR_CUDA; }
    }
    if (opt->precision != HELM_PREC_FP32) {
        if (c->nx % 2 != 0) { free_ctx(c); return HELM_ERR_UNSUPPORTED; }
        if (opt->precision == HELM_PREC_FP16 && k0z2) {   // the FP16 stage bounds assume a constant k0 in z
            for (int l = 1; l < c->nz; ++l)
                if (k0z2[l] != k0z2[0]) { free_ctx(c); return HELM_ERR_UNSUPPORTED; }
        }
        TRY(tc_prepare(c, s));
    }
    if (opt->precond != HELM_PRECOND_NONE) TRY(zsolve_factor(c, s));
    if (opt->precond == HELM_PRECOND_PFFT || opt->precond == HELM_PRECOND_FFT2) TRY(pfft_prepare(c, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) { free_ctx(c); return HELM_ERR_CUDA; }
    *out = c;
    return HELM_OK;
}

helm_status helm_build_rhs(helm_ctx* c, const void* f, void* F, void* stream) {
    if (!c || !f || !F) return HELM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double2* fd = (const double2*)f;
    double2* buf = nullptr;
    if (!dev_ptr(f)) {
        if (cudaMalloc(&buf, c->npts * sizeof(double2)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
        HELM_CUDA_TRY(cudaMemcpyAsync(buf, f, c->npts * sizeof(double2), cudaMemcpyHostToDevice, s));
        fd = buf;
    }
    if (!c->rhs_scratch) {
        if (cudaMalloc(&c->rhs_scratch, c->npts * sizeof(float4)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    }
    helm_status st = launch_rhs(c, fd, (double2*)F, c->rhs_scratch, s);
    if (buf) { cudaStreamSynchronize(s); cudaFree(buf); }
    return st;
}

helm_status helm_apply_A(helm_ctx* c, const void* x, void* y, int dtype, void* stream) {
    if (!c || !x || !y) return HELM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == HELM_C64) return launch_stencil_f32(c, (const float2*)x, (float2*)y, nullptr, 0, s);
    if (dtype == HELM_C128) return launch_stencil_f64(c, (const double2*)x, (double2*)y, s);
    return HELM_ERR_ARG;
}

helm_status helm_apply_precond(helm_ctx* c, const void* r, void* z, void* stream) {
    if (!c || !r || !z) return HELM_ERR_ARG;
    if (r == (const void*)c->tmp || z == (void*)c->tmp) return HELM_ERR_ARG;
    return precond_apply(c, (const float2*)r, (float2*)z, nullptr, 0, (cudaStream_t)stream);
}

helm_status helm_precond_step(helm_ctx* c, int step, const void* in, void* out, void* stream) {
    if (!c || !in || !out || step < 1 || step > 3) return HELM_ERR_ARG;
    if (c->opt.precond != HELM_PRECOND_EIGT) return HELM_ERR_ARG;
    return precond_step(c, step, (const float2*)in, (float2*)out, (cudaStream_t)stream);
}

helm_status helm_get_eig(helm_ctx* c, int axis, void* D, void* V, void* Vinv) {
    if (!c || (axis != 0 && axis != 1)) return HELM_ERR_ARG;
    const int N = axis == 0 ? c->nx : c->ny;
    const double2* d = axis == 0 ? c->Dx : c->Dy;
    const double2* v = axis == 0 ? c->Vx : c->Vy;
    const double2* vi = axis == 0 ? c->Vxi : c->Vyi;
    if (D) HELM_CUDA_TRY(cudaMemcpy(D, d, N * sizeof(double2), cudaMemcpyDeviceToHost));
    if (V) HELM_CUDA_TRY(cudaMemcpy(V, v, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToHost));
    if (Vinv) HELM_CUDA_TRY(cudaMemcpy(Vinv, vi, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToHost));
    return HELM_OK;
}

helm_status helm_gmres_solve(helm_ctx* c, const void* b, void* x, helm_solve_info* info, void* stream) {
    if (!c || !b || !x) return HELM_ERR_ARG;
    return gmres_run(c, (const double2*)b, (double2*)x, info, (cudaStream_t)stream);
}

helm_status helm_residual(helm_ctx* c, const void* b, const void* x, void* r, double* nrm2, double* nrmi,
                          void* stream) {
    if (!c || !b || !x) return HELM_ERR_ARG;
    if (!dev_ptr(b) || !dev_ptr(x) || (r && !dev_ptr(r))) return HELM_ERR_ARG;
    return residual_run(c, (const double2*)b, (const double2*)x, (float2*)r, nrm2, nrmi, (cudaStream_t)stream);
}

helm_status helm_build_rhs_fields(helm_ctx* c, const void* fields, void* F, void* stream) {
    if (!c || !fields || !F) return HELM_ERR_ARG;
    if (!dev_ptr(fields) || !dev_ptr(F)) return HELM_ERR_ARG;
    return launch_rhs_fields(c, (const double2*)fields, (double2*)F, (cudaStream_t)stream);
}

long long helm_closure_face_count(helm_ctx* c) {
    if (!c || !c->colloc) return 0;
    return (long long)closure_face_points(c);
}

helm_status helm_closure_rhs(helm_ctx* c, const void* faces, const void* F_in, void* F_out, void* stream) {
    if (!c || !faces || !F_in || !F_out) return HELM_ERR_ARG;
    if (!c->ho) return HELM_ERR_UNSUPPORTED;
    if (!dev_ptr(faces) || !dev_ptr(F_in) || !dev_ptr(F_out)) return HELM_ERR_ARG;
    return closure_rhs(c, (const double2*)faces, (const double2*)F_in, (double2*)F_out, (cudaStream_t)stream);
}

helm_status helm_set_wait_limit(helm_ctx* c, long long polls) {
    if (!c || polls < 0) return HELM_ERR_ARG;
    c->wait_limit = polls == 0 ? (1LL << 20) : polls;
    return HELM_OK;
}

helm_status helm_set_matvec_variant(helm_ctx* c, int variant) {
    if (!c || variant < 0 || variant >= stencil_variants(c)) return HELM_ERR_ARG;
    c->tune_stencil = variant;
    return HELM_OK;
}

void helm_destroy(helm_ctx* c) { free_ctx(c); }

}  // extern "C"
