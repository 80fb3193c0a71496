// EigT step 1 (Sec. 4.1, Eq. EIG_SOLVER): FP64 eigendecomposition Lbar = V D V^-1 of the 1D matrix
// of Eq. lambda_mat_definition, on the GPU: the staggered two-point ABC (corner gamma, zeta = 1) and the
// collocated three-point ABC (gamma = 2 i k0 h, zeta = 2).
//
// Method (our own, for this structured matrix): with v_l = cos((l - (N+1)/2) theta) or
// sin((l - (N+1)/2) theta), the interior rows give lambda = 2 cos theta and the two corner rows collapse
// (by the mirror symmetry of Lbar) to one scalar equation per family:
//     symmetric:      cos((N+1) theta/2) = gamma cos((N-1) theta/2)
//     antisymmetric:  sin((N+1) theta/2) = gamma sin((N-1) theta/2)   (divided by sin(theta/2) to remove
//                                                                      the spurious root theta = 0)
// For gamma = 0 the roots are the Dirichlet angles pi j/(N+1) (Sec. 3.1, Eq. LMB_egv), odd j symmetric,
// even j antisymmetric.  Each thread follows one root by Newton's method along gamma_t = t gamma,
// t = 1/S .. 1.  Lbar is complex symmetric, so eigenvectors of distinct eigenvalues are orthogonal in
// the bilinear form v^T w; normalising v^T v = 1 gives V^-1 = V^T without an inverse.  The result is
// checked by the residual |Lbar v - d v| and by |V^-1 V - I|; a failure is retried with more
// continuation steps and then reported as HELM_ERR_EIG.
//
// zeta = 2: the same vectors satisfy the interior rows; with b = (N-1)/2 the corner rows become
//     symmetric:      -2 sin(b theta) sin(theta) = gamma cos(b theta)
//     antisymmetric:   2 cos(b theta) sin(theta) = gamma sin(b theta)       (divided by sin(theta/2))
// At gamma = 0 (the Neumann-like matrix) the roots are pi j/(N-1), j = 0..N-1, even j symmetric; j = 0
// and j = N-1 are double roots (theta = 0, pi), so their first continuation step starts from the
// small-gamma expansions theta^2 = -gamma/(2b) and (pi - theta)^2 = gamma/(2b).  Lbar = W S W^-1 with
// W = diag(sqrt 2, 1, .., 1, sqrt 2) and S complex symmetric, so V^-1 = V^T W^-2 once v^T W^-2 v = 1
// (the end entries weigh one half).  The straight continuation path is reliable for |gamma| <= 2
// (k0 h <= 1, at least six points per wavelength); beyond that the check reports HELM_ERR_EIG.
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

__device__ inline double2 c_sin(double2 z) {
    return make_double2(sin(z.x) * cosh(z.y), cos(z.x) * sinh(z.y));
}
__device__ inline double2 c_cos(double2 z) {
    return make_double2(cos(z.x) * cosh(z.y), -sin(z.x) * sinh(z.y));
}
__device__ inline double2 c_sqrt(double2 z) {
    const double r = hypot(z.x, z.y);
    if (r == 0.0) return make_double2(0.0, 0.0);
    const double t = sqrt(0.5 * (r + fabs(z.x)));
    if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
    return make_double2(fabs(z.y) / (2.0 * t), z.y >= 0 ? t : -t);
}

// F(theta) and F'(theta) for one family.
__device__ inline void family(double2 th, int N, double2 g, bool anti, double2& F, double2& dF) {
    const double a = 0.5 * (N + 1), b = 0.5 * (N - 1);
    const double2 ta = make_double2(a * th.x, a * th.y), tb = make_double2(b * th.x, b * th.y);
    if (!anti) {
        const double2 ca = c_cos(ta), cb = c_cos(tb), sa = c_sin(ta), sb = c_sin(tb);
        F = csub(ca, cmul(g, cb));
        dF = cadd(cscale(sa, -a), cscale(cmul(g, sb), b));
    } else {
        const double2 sa = c_sin(ta), sb = c_sin(tb), ca = c_cos(ta), cb = c_cos(tb);
        const double2 h = make_double2(0.5 * th.x, 0.5 * th.y);
        const double2 sh = c_sin(h), ch = c_cos(h);
        const double2 num = csub(sa, cmul(g, sb));
        const double2 dnum = csub(cscale(ca, a), cscale(cmul(g, cb), b));
        const double2 dden = cscale(ch, 0.5);
        F = cdiv(num, sh);
        dF = cdiv(csub(cmul(dnum, sh), cmul(num, dden)), cmul(sh, sh));
    }
}

// F(theta) and F'(theta) for one family of the zeta = 2 matrix.
__device__ inline void family_z2(double2 th, int N, double2 g, bool anti, double2& F, double2& dF) {
    const double b = 0.5 * (N - 1);
    const double2 tb = make_double2(b * th.x, b * th.y);
    const double2 sb = c_sin(tb), cb = c_cos(tb), s1 = c_sin(th), c1 = c_cos(th);
    if (!anti) {
        // F = -2 sin(b t) sin t - g cos(b t)
        F = csub(cscale(cmul(sb, s1), -2.0), cmul(g, cb));
        dF = cadd(cadd(cscale(cmul(cb, s1), -2.0 * b), cscale(cmul(sb, c1), -2.0)), cscale(cmul(g, sb), b));
    } else {
        // (2 cos(b t) sin t - g sin(b t)) / sin(t/2)
        const double2 num = csub(cscale(cmul(cb, s1), 2.0), cmul(g, sb));
        const double2 dnum = csub(cadd(cscale(cmul(sb, s1), -2.0 * b), cscale(cmul(cb, c1), 2.0)), cscale(cmul(g, cb), b));
        const double2 h = make_double2(0.5 * th.x, 0.5 * th.y);
        const double2 sh = c_sin(h), ch = c_cos(h);
        F = cdiv(num, sh);
        dF = cdiv(csub(cmul(dnum, sh), cmul(num, cscale(ch, 0.5))), cmul(sh, sh));
    }
}

__global__ void eig_newton_kernel(int N, double2 gamma, int z2, int steps, double2* __restrict__ D,
                                  double2* __restrict__ V, double2* __restrict__ Vinv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int jp = j + 1;
    const bool anti = z2 ? (j % 2) == 1 : (jp % 2) == 0;
    double2 th = make_double2(z2 ? M_PI * j / (N - 1.0) : M_PI * jp / (N + 1.0), 0.0);
    const double b = 0.5 * (N - 1);
    for (int s = 1; s <= steps; ++s) {
        const double t = (double)s / steps;
        const double2 g = make_double2(t * gamma.x, t * gamma.y);
        if (z2 && s == 1 && j == 0) th = c_sqrt(make_double2(-g.x / (2.0 * b), -g.y / (2.0 * b)));
        if (z2 && s == 1 && j == N - 1) th = csub(make_double2(M_PI, 0.0), c_sqrt(make_double2(g.x / (2.0 * b), g.y / (2.0 * b))));
        const int its = s < steps ? 3 : 30;
        for (int it = 0; it < its; ++it) {
            double2 F, dF;
            if (z2) family_z2(th, N, g, anti, F, dF);
            else family(th, N, g, anti, F, dF);
            const double2 step = cdiv(F, dF);
            if (!(isfinite(step.x) && isfinite(step.y))) break;
            th = csub(th, step);
        }
    }
    const double2 c = c_cos(th);
    D[j] = make_double2(2.0 * c.x, 2.0 * c.y);
    double2 nrm = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) {
        const double off = l - 0.5 * (N - 1);
        const double2 arg = make_double2(off * th.x, off * th.y);
        const double2 v = anti ? c_sin(arg) : c_cos(arg);
        const double wt = (z2 && (l == 0 || l == N - 1)) ? 0.5 : 1.0;
        nrm = cadd(nrm, cscale(cmul(v, v), wt));
    }
    const double2 inv = cdiv(make_double2(1.0, 0.0), c_sqrt(nrm));
    for (int l = 0; l < N; ++l) {
        const double off = l - 0.5 * (N - 1);
        const double2 arg = make_double2(off * th.x, off * th.y);
        const double2 v = cmul(anti ? c_sin(arg) : c_cos(arg), inv);
        const double wt = (z2 && (l == 0 || l == N - 1)) ? 0.5 : 1.0;
        V[(size_t)l * N + j] = v;
        Vinv[(size_t)j * N + l] = cscale(v, wt);
    }
}

__device__ inline void atomic_max_nonneg(unsigned long long* addr, double v) {
    if (!(v >= 0.0)) v = 1e300;  // NaN counts as failure
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// res[0] = max_j |Lbar v_j - d_j v_j|_inf,  res[1] = max_{j,k} |(V^-1 V)_{jk} - delta_jk|
__global__ void eig_check_kernel(int N, double2 gamma, double zeta, const double2* __restrict__ D,
                                 const double2* __restrict__ V, const double2* __restrict__ Vinv,
                                 unsigned long long* res) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * N) return;
    const int j = (int)(id / N), k = (int)(id % N);
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) acc = cadd(acc, cmul(Vinv[(size_t)j * N + l], V[(size_t)l * N + k]));
    if (j == k) acc.x -= 1.0;
    atomic_max_nonneg(&res[1], hypot(acc.x, acc.y));
    if (j == 0) {
        // residual of eigenpair k at row l = ... all rows
        double worst = 0.0;
        for (int l = 0; l < N; ++l) {
            double2 lv = make_double2(0.0, 0.0);
            if (l > 0) lv = cadd(lv, cscale(V[(size_t)(l - 1) * N + k], l == N - 1 ? zeta : 1.0));
            if (l < N - 1) lv = cadd(lv, cscale(V[(size_t)(l + 1) * N + k], l == 0 ? zeta : 1.0));
            if (l == 0 || l == N - 1) lv = cadd(lv, cmul(gamma, V[(size_t)l * N + k]));
            lv = csub(lv, cmul(D[k], V[(size_t)l * N + k]));
            worst = fmax(worst, hypot(lv.x, lv.y));
        }
        atomic_max_nonneg(&res[0], worst);
    }
}

__global__ void prep_operands_kernel(int N, double alpha, const double2* __restrict__ D, const double2* __restrict__ V,
                                     const double2* __restrict__ Vinv, float2* __restrict__ BF, float2* __restrict__ BI,
                                     float2* __restrict__ AF, float2* __restrict__ AI, float2* __restrict__ ds) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * N) return;
    const int r = (int)(id / N), q = (int)(id % N);
    // x-pass B operands: B[k][n] = Vinv[n][k] (forward), V[n][k] (inverse)
    if (BF) {
        const double2 f = Vinv[(size_t)q * N + r], b = V[(size_t)q * N + r];
        BF[id] = make_float2((float)f.x, (float)f.y);
        BI[id] = make_float2((float)b.x, (float)b.y);
    }
    // y-pass A operands: A = Vinv (forward), V (inverse)
    if (AF) {
        const double2 f = Vinv[id], b = V[id];
        AF[id] = make_float2((float)f.x, (float)f.y);
        AI[id] = make_float2((float)b.x, (float)b.y);
    }
    if (q == 0) ds[r] = make_float2((float)(alpha * D[r].x), (float)(alpha * D[r].y));
}

helm_status eig_one_axis(int N, double2 gamma, double zeta, double2* D, double2* V, double2* Vinv,
                         unsigned long long* chk, cudaStream_t s) {
    const int steps_try[2] = {32, 256};
    const int z2 = zeta != 1.0;
    for (int t = 0; t < 2; ++t) {
        eig_newton_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, gamma, z2, steps_try[t], D, V, Vinv);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemsetAsync(chk, 0, 2 * sizeof(unsigned long long), s));
        const size_t nn = (size_t)N * N;
        eig_check_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(N, gamma, zeta, D, V, Vinv, chk);
        HELM_CUDA_TRY(cudaGetLastError());
        unsigned long long h[2];
        HELM_CUDA_TRY(cudaMemcpyAsync(h, chk, sizeof(h), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        double res, orth;
        memcpy(&res, &h[0], 8);
        memcpy(&orth, &h[1], 8);
        if (res < 1e-9 && orth < 1e-8) return HELM_OK;
    }
    return HELM_ERR_EIG;
}

}  // namespace

helm_status run_eig_setup(helm_ctx* c, cudaStream_t s) {
    unsigned long long* chk = nullptr;
    HELM_CUDA_TRY(cudaMalloc(&chk, 2 * sizeof(unsigned long long)));
    helm_status st = eig_one_axis(c->nx, c->gam[0], c->zeta[0], c->Dx, c->Vx, c->Vxi, chk, s);
    if (st == HELM_OK) st = eig_one_axis(c->ny, c->gam[1], c->zeta[1], c->Dy, c->Vy, c->Vyi, chk, s);
    cudaFree(chk);
    if (st != HELM_OK) return st;
    {
        const size_t nn = (size_t)c->nx * c->nx;
        prep_operands_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->nx, c->ax, c->Dx, c->Vx, c->Vxi, c->XF,
                                                                          c->XI, nullptr, nullptr, c->dxs);
        HELM_CUDA_TRY(cudaGetLastError());
    }
    {
        const size_t nn = (size_t)c->ny * c->ny;
        prep_operands_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->ny, c->ay, c->Dy, c->Vy, c->Vyi, nullptr,
                                                                          nullptr, c->YF, c->YI, c->dys);
        HELM_CUDA_TRY(cudaGetLastError());
    }
    return HELM_OK;
}

// ---- stage scales of the FP16 transform chain (HELM_PREC_FP16) ------------------------------------------
// FP16 keeps TF32's 11-bit significand but overflows above 65504, so every grid the chain stores is scaled by a
// power of two from bounds that hold for any input: the chain's input is the unit vector times 2^12 (the
// conversion applies the Arnoldi normalisation, or 1 / ||r||), and the Frobenius norm of each stage's output
// is at most the spectral norm of its operator times that of its input.  The first pass's scale is fixed
// here; every later stage takes its scale at run time from its input's measured Frobenius norm times the
// operator bound computed here, so the worst cases of the stages do not compound.  The x-pass
// applies V_x^-T (or V_x^T), the y-pass V_y^-1 (or V_y), row- and slice-wise, so their gains are the
// largest singular values of those matrices; the z-systems T_ij = Lbar_z + s_ij I (constant k0) diagonalise
// as V_z (D_z + s_ij) V_z^-1, so ||T_ij^-1|| <= kappa(V_z) / min_m |d_zm + s_ij|, with s_ij = a_x d_xi +
// a_y d_yj + h_z^2 k0^2 - 2 (a_x + a_y).  The spectral norms come from 60 power iterations (which approach
// them from below) and take a safety factor 1.5; each stage's output bound is brought to at most 2^15 (the
// largest element of a grid is at most its Frobenius norm), and the last pass undoes the scales.
namespace {
double spec_norm_host(const std::vector<double2>& A, int n) {
    std::vector<double> xr(n), xi(n), yr(n), yi(n);
    for (int i = 0; i < n; ++i) { xr[i] = 1.0 + 0.37 * ((i * 7919) % 13); xi[i] = 0.11 * ((i * 104729) % 5); }
    double sig = 0.0;
    for (int it = 0; it < 60; ++it) {
        double nn = 0.0;
        for (int i = 0; i < n; ++i) nn += xr[i] * xr[i] + xi[i] * xi[i];
        nn = std::sqrt(nn);
        for (int i = 0; i < n; ++i) { xr[i] /= nn; xi[i] /= nn; }
        for (int r = 0; r < n; ++r) {          // y = A x
            double ar = 0.0, ai = 0.0;
            for (int k = 0; k < n; ++k) {
                const double2 a = A[(size_t)r * n + k];
                ar += a.x * xr[k] - a.y * xi[k];
                ai += a.x * xi[k] + a.y * xr[k];
            }
            yr[r] = ar; yi[r] = ai;
        }
        double ny = 0.0;
        for (int r = 0; r < n; ++r) ny += yr[r] * yr[r] + yi[r] * yi[r];
        sig = std::sqrt(ny);                    // ||A x|| for the unit x
        for (int k = 0; k < n; ++k) { xr[k] = 0.0; xi[k] = 0.0; }
        for (int r = 0; r < n; ++r)             // x = A^H y
            for (int k = 0; k < n; ++k) {
                const double2 a = A[(size_t)r * n + k];
                xr[k] += a.x * yr[r] + a.y * yi[r];
                xi[k] += a.x * yi[r] - a.y * yr[r];
            }
    }
    return sig;
}
std::vector<double2> to_host(const double2* d, size_t n) {
    std::vector<double2> h(n);
    if (cudaMemcpy(h.data(), d, n * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) h.clear();
    return h;
}
float pow2_scale(double bound) {   // 2^e with bound * 2^e <= 2^15
    const int e = 15 - (int)std::ceil(std::log2(bound));
    return std::ldexp(1.0f, e);
}
}  // namespace

helm_status h16_scales(helm_ctx* c, cudaStream_t s) {
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    double2 *Dz = nullptr, *Vz = nullptr, *Vzi = nullptr;
    unsigned long long* chk = nullptr;
    if (cudaMalloc(&Dz, nz * sizeof(double2)) != cudaSuccess || cudaMalloc(&Vz, (size_t)nz * nz * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&Vzi, (size_t)nz * nz * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&chk, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(Dz); cudaFree(Vz); cudaFree(Vzi); cudaFree(chk);
        return HELM_ERR_NOMEM;
    }
    helm_status st = eig_one_axis(nz, c->gam[2], c->zeta[2], Dz, Vz, Vzi, chk, s);
    if (st == HELM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = HELM_ERR_CUDA;
    std::vector<double2> hVxi, hVyi, hVy, hVz, hVzi, hDx, hDy, hDz;
    if (st == HELM_OK) {
        hVxi = to_host(c->Vxi, (size_t)nx * nx);
        hVyi = to_host(c->Vyi, (size_t)ny * ny); hVy = to_host(c->Vy, (size_t)ny * ny);
        hVz = to_host(Vz, (size_t)nz * nz); hVzi = to_host(Vzi, (size_t)nz * nz);
        hDx = to_host(c->Dx, nx); hDy = to_host(c->Dy, ny); hDz = to_host(Dz, nz);
        if (hVxi.empty() || hVyi.empty() || hVy.empty() || hVz.empty() || hVzi.empty() || hDx.empty() ||
            hDy.empty() || hDz.empty())
            st = HELM_ERR_CUDA;
    }
    cudaFree(Dz); cudaFree(Vz); cudaFree(Vzi); cudaFree(chk);
    if (st != HELM_OK) return st;
    const double safety = 1.5;
    const double sxi = safety * spec_norm_host(hVxi, nx), syi = safety * spec_norm_host(hVyi, ny);
    const double sy = safety * spec_norm_host(hVy, ny);
    const double kz = safety * spec_norm_host(hVz, nz) * safety * spec_norm_host(hVzi, nz);
    const double hz2 = c->h[2] * c->h[2];
    const double base = hz2 * c->k0 * c->k0 - 2.0 * (c->ax + c->ay);
    double lmin = 1e300;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j) {
            const double sr = c->ax * hDx[i].x + c->ay * hDy[j].x + base, si = c->ax * hDx[i].y + c->ay * hDy[j].y;
            for (int m = 0; m < nz; ++m) {
                const double lr = sr + hDz[m].x, li = si + hDz[m].y;
                lmin = std::min(lmin, lr * lr + li * li);
            }
        }
    lmin = std::sqrt(lmin);
    if (!(lmin > 0.0) || !std::isfinite(sxi * syi * sy * kz)) return HELM_ERR_EIG;
    const double gz = kz / lmin;
    // static: the input (2^12) and the x-pass forward (its input's norm is that bound); the later stages
    // scale at run time from their input's measured norm times the gains kept here (c->h16g)
    c->h16s[0] = 4096.f;
    c->h16s[1] = pow2_scale(sxi * 4096.0);
    c->h16s[2] = c->h16s[3] = c->h16s[4] = 1.f;
    c->h16s[5] = (float)(hz2 / (4096.0 * (double)c->h16s[1]));
    c->h16g[0] = (float)syi;
    c->h16g[1] = (float)gz;
    c->h16g[2] = (float)sy;
    return HELM_OK;
}
