// Preconditioner action z = M^-1 r = h_z^2 A_p^-1 r (Sec. 4.1): EigT steps 2-4 (Eq. EIG_SOLVER).
//   step 2  Ybar_l = V_y^-1 Y_l V_x^-T   x-pass (right multiply) then y-pass (left multiply)
//   step 3  z-solves of Eq. Indep_precond_system
//   step 4  U_l = V_y Ubar_l V_x^T       y-pass then x-pass; the last pass carries the factor h_z^2
// Buffers: r -> tmp -> z -> (in place) z -> tmp -> z, so r may alias z but neither may alias the
// context's scratch vector.  An optional device scale sigma[sidx] multiplies r (lazy normalisation
// of the Arnoldi vectors).
#include "common.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

__global__ void scale_copy_kernel(const float2* __restrict__ a, float2* __restrict__ b, size_t n, float al,
                                  const double* sigma, int sidx) {
    const float s = al * (sigma ? (float)sigma[sidx] : 1.f);
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        b[id] = make_float2(s * a[id].x, s * a[id].y);
}

bool use_tc(const helm_ctx* c) { return c->opt.precision != HELM_PREC_FP32; }

// complex64 -> 16-bit pairs (H = 1 BF16, 2 FP16 clamped to the finite range; round to nearest even), the
// entry of the 16-bit chain: two points per float4, times s0 and the Arnoldi scale sigma[sidx] (else inv[0])
template <int H>
__device__ __forceinline__ uint32_t cpack16(float lo, float hi) {
    if (H == 2) {
        const __half2 v = __floats2half2_rn(fminf(fmaxf(lo, -65504.f), 65504.f), fminf(fmaxf(hi, -65504.f), 65504.f));
        return *reinterpret_cast<const uint32_t*>(&v);
    }
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
// (nb vectors back to back, vector v scaled by sigma[sidx + v sstride]: blockIdx.y = v)
template <int H>
__global__ void c64_to_h16_kernel(const float4* __restrict__ a, uint2* __restrict__ b, size_t n2, float s0,
                                  const double* __restrict__ sigma, int sidx, const double* __restrict__ inv,
                                  int sstride = 0) {
    const float sc = s0 * (sigma ? (float)sigma[sidx + blockIdx.y * sstride] : inv ? (float)inv[0] : 1.f);
    a += (size_t)blockIdx.y * n2;
    b += (size_t)blockIdx.y * n2;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n2; i0 += 4 * stride) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t i = i0 + u * stride;
            v[u] = i < n2 ? a[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t i = i0 + u * stride;
            if (i < n2) b[i] = make_uint2(cpack16<H>(sc * v[u].x, sc * v[u].y), cpack16<H>(sc * v[u].z, sc * v[u].w));
        }
    }
}

// ||r||_2 of a complex64 grid: per-block FP64 partial sums, then one block writes 1/||r|| (0 for r = 0) and ||r||
constexpr int NRM_BLOCKS = 1024;
__global__ void norm_part_kernel(const float2* __restrict__ r, size_t n, double* __restrict__ part) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = r[i];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void norm_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nr = sqrt(sh[0]);
        out[0] = nr > 0.0 ? 1.0 / nr : 0.0;
        out[1] = nr;
    }
}

// The passes of the 16-bit chain from the 16-bit input In to the complex64 z (T0, T1: the halves of the
// context's scratch vector; In may be T0).  BF16: the static factors of c->h16s (all 1 but the last).  FP16:
// the x-pass forward scales statically (its input's norm is bounded by h16s[0]), every later stage by the
// bound of its input's measured norm (c->h16d, reset here), and the last pass undoes those scales.
helm_status h16_chain(helm_ctx* c, const uint16_t* In, uint16_t* T1, float2* z, float alpha_last, const double* adev,
                      int aidx, cudaStream_t s, int nb = 1) {
    helm_status st;
    uint16_t* T0 = reinterpret_cast<uint16_t*>(c->tmp);
    const float* sc = c->h16s;
    double* d = c->opt.precision == HELM_PREC_FP16 ? c->h16d : nullptr;
    if (d) HELM_CUDA_TRY(cudaMemsetAsync(d, 0, 3 * sizeof(double), s));
    prof_begin(c, s, PROF_XPASS);
    st = tc_xpass_h16(c, 0, In, T1, 1, sc[1], nullptr, 0, s, nb, 0, nullptr, d);
    prof_end(c, s);
    if (st != HELM_OK) return st;
    prof_begin(c, s, PROF_YPASS);
    st = tc_ypass_h16(c, 0, T1, T0, sc[2], s, nb, d, c->h16g[0]);
    prof_end(c, s);
    if (st != HELM_OK) return st;
    if ((st = launch_zsolve_h16(c, T0, T0, reinterpret_cast<float4*>(z), sc[3], s, nb, d, c->h16g[1])) != HELM_OK) return st;
    prof_begin(c, s, PROF_YPASS);
    st = tc_ypass_h16(c, 1, T0, T1, sc[4], s, nb, d, c->h16g[2]);
    prof_end(c, s);
    if (st != HELM_OK) return st;
    prof_begin(c, s, PROF_XPASS);
    if (c->h16_join) HELM_CUDA_TRY(cudaStreamWaitEvent(s, c->h16_join, 0));
    st = tc_xpass_h16(c, 1, T1, z, 0, alpha_last, adev, aidx, s, nb, 0, d ? d + 7 : nullptr, nullptr);
    prof_end(c, s);
    return st;
}

// EigT with 16-bit intermediate grids (HELM_PREC_BF16, HELM_PREC_FP16): r (complex64) -> 16 bits ->
// x-pass -> y-pass -> z-solve -> y-pass -> x-pass -> z (complex64), every stored grid times its power-of-two
// stage scale c->h16s (FP16; all 1 for BF16, whose range is FP32's), the last pass undoing them.  The two
// 16-bit grids live in the halves of the context's scratch vector (T0, T1); the z-solve keeps its FP32
// forward values in z, which is free until the last pass, so r may alias z.
helm_status precond_h16(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s) {
    const size_t n = c->npts;
    const int H = c->opt.precision == HELM_PREC_FP16 ? 2 : 1;
    uint16_t* T0 = reinterpret_cast<uint16_t*>(c->tmp);
    uint16_t* T1 = T0 + 2 * n;
    const float* sc = c->h16s;
    const double* inv = nullptr;
    const double* nrm = nullptr;
    prof_begin(c, s, PROF_XPASS);
    if (H == 2 && !sigma) {   // no Arnoldi scale: normalise by ||r|| here, restore it in the last pass
        norm_part_kernel<<<NRM_BLOCKS, 256, 0, s>>>(r, n, c->h16n + 2);
        norm_final_kernel<<<1, 256, 0, s>>>(c->h16n + 2, NRM_BLOCKS, c->h16n);
        inv = c->h16n;
        nrm = c->h16n + 1;
    }
    if (H == 2)
        c64_to_h16_kernel<2><<<2048, 256, 0, s>>>(reinterpret_cast<const float4*>(r), reinterpret_cast<uint2*>(T0), n / 2,
                                                  sc[0], sigma, sidx, inv);
    else
        c64_to_h16_kernel<1><<<2048, 256, 0, s>>>(reinterpret_cast<const float4*>(r), reinterpret_cast<uint2*>(T0), n / 2,
                                                  sc[0], sigma, sidx, inv);
    HELM_CUDA_TRY(cudaGetLastError());
    prof_end(c, s);
    return h16_chain(c, T0, T1, z, sc[5], nrm, 0, s);
}

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
    if (c->opt.precision == HELM_PREC_BF16 || c->opt.precision == HELM_PREC_FP16) return precond_h16(c, r, z, sigma, sidx, s);
    const float hz2 = (float)(c->h[2] * c->h[2]);
    if ((st = xpass(c, 0, r, c->tmp, 1.f, sigma, sidx, s)) != HELM_OK) return st;
    if ((st = ypass(c, 0, c->tmp, z, s)) != HELM_OK) return st;
    if ((st = launch_zsolve(c, z, z, s)) != HELM_OK) return st;
    if ((st = ypass(c, 1, z, c->tmp, s)) != HELM_OK) return st;
    return xpass(c, 1, c->tmp, z, hz2, nullptr, 0, s);
}

// z = M^-1 v for v = cs[cidx] V16 with V16 an FP16 grid whose Frobenius norm is at most the chain's input
// bound h16s[0] (the FP16 Krylov basis of HELM_PREC_FP16): the chain of precond_h16 without its conversion,
// the last pass scaled by cs[cidx] h16s[0] on top of the stage factor.  z is complex64 and must not alias V16.
helm_status precond_h16_basis(helm_ctx* c, const uint16_t* V16, float2* z, const double* cs, int cidx, cudaStream_t s) {
    if (c->opt.precision != HELM_PREC_FP16 || c->opt.precond != HELM_PRECOND_EIGT || c->net) return HELM_ERR_UNSUPPORTED;
    uint16_t* T1 = reinterpret_cast<uint16_t*>(c->tmp) + 2 * c->npts;
    return h16_chain(c, V16, T1, z, c->h16s[5] * c->h16s[0], cs, cidx, s);
}

// complex64 r -> FP16 grid scaled by s0 sigma[sidx] (the first basis vector of a cycle)
helm_status to_h16_basis(helm_ctx* c, const float2* r, uint16_t* V16, const double* sigma, int sidx, cudaStream_t s) {
    prof_begin(c, s, PROF_SMALL);
    c64_to_h16_kernel<2><<<2048, 256, 0, s>>>(reinterpret_cast<const float4*>(r), reinterpret_cast<uint2*>(V16), c->npts / 2,
                                              c->h16s[0], sigma, sidx, nullptr);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
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
    if (c->opt.precision == HELM_PREC_BF16 || c->opt.precision == HELM_PREC_FP16) {
        // the 16-bit chain over the nb vectors (each pass acts on every vector's rows, slices or lines on
        // their own, so each vector's stage bounds hold; the measured norms are the group's)
        const size_t n = c->npts;
        uint16_t* T0 = reinterpret_cast<uint16_t*>(c->tmp);
        uint16_t* T1 = T0 + 2 * n * nb;
        prof_begin(c, s, PROF_XPASS);
        if (c->opt.precision == HELM_PREC_FP16)
            c64_to_h16_kernel<2><<<dim3(512, nb), 256, 0, s>>>(reinterpret_cast<const float4*>(r), reinterpret_cast<uint2*>(T0),
                                                              n / 2, c->h16s[0], sigma, sidx, nullptr, sstride);
        else
            c64_to_h16_kernel<1><<<dim3(512, nb), 256, 0, s>>>(reinterpret_cast<const float4*>(r), reinterpret_cast<uint2*>(T0),
                                                              n / 2, c->h16s[0], sigma, sidx, nullptr, sstride);
        HELM_CUDA_TRY(cudaGetLastError());
        prof_end(c, s);
        return h16_chain(c, T0, T1, z, c->h16s[5], nullptr, 0, s, nb);
    }
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
