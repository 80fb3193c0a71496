// Preconditioner action z = M^-1 r = h_z^2 A_p^-1 r (Sec. 4.1): EigT steps 2-4 (Eq. EIG_SOLVER).
//   step 2  Ybar_l = V_y^-1 Y_l V_x^-T   x-pass (right multiply) then y-pass (left multiply)
//   step 3  z-solves of Eq. Indep_precond_system
//   step 4  U_l = V_y Ubar_l V_x^T       y-pass then x-pass; the last pass carries the factor h_z^2
// Buffers: r -> tmp -> z -> (in place) z -> tmp -> z, so r may alias z but neither may alias the
// context's scratch vector.  An optional device scale sigma[sidx] multiplies r (lazy normalisation
// of the Arnoldi vectors).
#include "common.cuh"

namespace {

__global__ void scale_copy_kernel(const float2* __restrict__ a, float2* __restrict__ b, size_t n, float al,
                                  const double* sigma, int sidx) {
    const float s = al * (sigma ? (float)sigma[sidx] : 1.f);
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        b[id] = make_float2(s * a[id].x, s * a[id].y);
}

bool use_tc(const helm_ctx* c) { return c->opt.precision != HELM_PREC_FP32; }

// nb > 1: nb grid vectors back to back (a batch group); vector v is scaled by sigma[sidx + v sstride]
helm_status xpass(helm_ctx* c, int inverse, const float2* in, float2* out, float alpha, const double* sigma, int sidx,
                  cudaStream_t s, int nb = 1, int sstride = 0) {
    prof_begin(c, s, PROF_XPASS);
    if (use_tc(c)) {
        helm_status st = tc_xpass(c, inverse, in, out, alpha, sigma, sidx, s, nb, sstride);
        prof_end(c, s);
        return st;
    }
    const int rows = c->ny * c->nz, M = rows * nb, N = c->nx;
    launch_cgemm_simt(M, N, N, in, N, 0, inverse ? c->XI : c->XF, N, 0, out, N, 0, 1, alpha, sigma, sidx, s, rows,
                      sstride);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status ypass(helm_ctx* c, int inverse, const float2* in, float2* out, cudaStream_t s, int nb = 1) {
    prof_begin(c, s, PROF_YPASS);
    if (use_tc(c)) {
        helm_status st = tc_ypass(c, inverse, in, out, s, nb);
        prof_end(c, s);
        return st;
    }
    const int nx = c->nx, ny = c->ny;
    const long slice = (long)nx * ny;
    launch_cgemm_simt(ny, nx, ny, inverse ? c->YI : c->YF, ny, 0, in, nx, slice, out, nx, slice, c->nz * nb, 1.f,
                      nullptr, 0, s);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

}  // namespace

helm_status precond_step(helm_ctx* c, int step, const float2* in, float2* out, cudaStream_t s) {
    helm_status st;
    if (step == 1) {
        if ((st = xpass(c, 0, in, c->tmp, 1.f, nullptr, 0, s)) != HELM_OK) return st;
        return ypass(c, 0, c->tmp, out, s);
    }
    if (step == 2) return launch_zsolve(c, in, out, s);
    if (step == 3) {
        if ((st = ypass(c, 1, in, c->tmp, s)) != HELM_OK) return st;
        return xpass(c, 1, c->tmp, out, 1.f, nullptr, 0, s);
    }
    return HELM_ERR_ARG;
}

static helm_status precond_base(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s) {
    helm_status st;
    if (c->opt.precond == HELM_PRECOND_NONE) {
        prof_begin(c, s, PROF_OTHER);
        scale_copy_kernel<<<1024, 256, 0, s>>>(r, z, c->npts, 1.f, sigma, sidx);
        prof_end(c, s);
        HELM_CUDA_TRY(cudaGetLastError());
        return HELM_OK;
    }
    if (c->opt.precond == HELM_PRECOND_PFFT || c->opt.precond == HELM_PRECOND_FFT2) {
        prof_begin(c, s, PROF_OTHER);
        st = c->opt.precond == HELM_PRECOND_PFFT ? pfft_apply(c, r, z, sigma, sidx, s)
                                                 : pfft_apply_dirichlet(c, r, z, sigma, sidx, s);
        prof_end(c, s);
        return st;
    }
    const float hz2 = (float)(c->h[2] * c->h[2]);
    if ((st = xpass(c, 0, r, c->tmp, 1.f, sigma, sidx, s)) != HELM_OK) return st;
    if ((st = ypass(c, 0, c->tmp, z, s)) != HELM_OK) return st;
    if ((st = launch_zsolve(c, z, z, s)) != HELM_OK) return st;
    if ((st = ypass(c, 1, z, c->tmp, s)) != HELM_OK) return st;
    return xpass(c, 1, c->tmp, z, hz2, nullptr, 0, s);
}

// M^-1 for nb vectors back to back (the right-hand sides of a batch group): one x-pass GEMM over all their
// rows, one y-pass over all their slices, one z-solve over all their lines.  Vector v is scaled by
// sigma[sidx + v sstride] on the way in.  EigT or no preconditioner; the context's scratch vector must hold
// nb vectors (the caller swaps in a scratch block).
helm_status precond_apply_nb(helm_ctx* c, const float2* r, float2* z, int nb, const double* sigma, int sidx,
                             int sstride, cudaStream_t s) {
    helm_status st;
    if (nb == 1) return precond_apply(c, r, z, sigma, sidx, s);
    if (c->opt.precond == HELM_PRECOND_NONE) {
        for (int v = 0; v < nb; ++v) {
            scale_copy_kernel<<<1024, 256, 0, s>>>(r + (size_t)v * c->npts, z + (size_t)v * c->npts, c->npts, 1.f, sigma,
                                                   sidx + v * sstride);
        }
        HELM_CUDA_TRY(cudaGetLastError());
        return HELM_OK;
    }
    if (c->opt.precond != HELM_PRECOND_EIGT || c->net) return HELM_ERR_UNSUPPORTED;
    const float hz2 = (float)(c->h[2] * c->h[2]);
    if ((st = xpass(c, 0, r, c->tmp, 1.f, sigma, sidx, s, nb, sstride)) != HELM_OK) return st;
    if ((st = ypass(c, 0, c->tmp, z, s, nb)) != HELM_OK) return st;
    if ((st = launch_zsolve(c, z, z, s, nb)) != HELM_OK) return st;
    if ((st = ypass(c, 1, z, c->tmp, s, nb)) != HELM_OK) return st;
    return xpass(c, 1, c->tmp, z, hz2, nullptr, 0, s, nb, 0);
}

// M^-1 r, followed by the learned correction when a network is attached (flexible GMRES only)
helm_status precond_apply(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s) {
    helm_status st;
    if (c->net && (st = learned_pre(c, r, sigma, sidx, s)) != HELM_OK) return st;
    if ((st = precond_base(c, r, z, sigma, sidx, s)) != HELM_OK) return st;
    if (c->net) return learned_post(c, z, s);
    return HELM_OK;
}
