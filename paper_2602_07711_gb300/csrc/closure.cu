// High-order closure of the Sommerfeld condition on collocated grids (the constant-k test problems of
// Sec. 2.1 close the fourth- and sixth-order schemes with a high-order three-point approximation of the
// ABC; the paper gives no formula, this is our reading).
//
// Per face, with B the boundary node, I its interior neighbour, G the ghost and h the normal step:
//     U_G = U_I + i k0 sum_{m=0..2} c_m (-1)^m L^m U_B,      c_m = 2 h^(2m+1) / (2m+1)!,
// L = k0^2 + (tangential second derivatives), from the Taylor series of u about B in the normal
// direction with every odd normal derivative reduced by the ABC and the equation (k = k0 on the face).
// m = 0 alone is the three-point rule of the preconditioner.  The tangential derivatives are sixth-order
// differences along the face: seven centred points where they fit, the eight nearest points otherwise.
// The faces are filled x, then y, then z; a face covers the ghost columns of the directions filled before
// it, so edge and corner ghosts come from the rule applied along an already-filled ghost line.
// The closure's f part (U-independent) belongs to the right-hand side the caller supplies.
//
// Layout: the operand is copied into a padded array (nx+2) x (ny+2) x (nz+2), x fastest; the general
// stencil kernels then read it with no ghost logic.  Per face two launches: V1 = L U_B into a scratch
// face, then the ghost from U_I, U_B, V1 and L V1 (formed on the fly).  The arithmetic is FP64 whatever
// the storage (complex64, complex128 or double-float): the faces are O(N^2) work.
#include "common.cuh"
#include <cmath>
#include <cstring>

namespace {

struct Wts {
    double wl[3][8];     // rows 0, 1, 2 of the one-sided stencils (second derivative, times 1/h^2)
    double wc[7];        // centred seven-point stencil
};

struct Face {
    int axis;            // 0 x, 1 y, 2 z
    int la, lb;          // face extents along the tangential axes ta, tb (array order: ta slower)
    int sa0, sb0;        // first padded coordinate along ta, tb
    long long sn, sa, sb;  // padded strides along the normal and the tangential axes
    int nb_lo, nb_hi;    // padded normal index of the two boundary planes (1 and n)
    double iha2, ihb2;   // 1/h_ta^2, 1/h_tb^2
    double c0, c1, c2;   // Taylor weights of the normal step
    double k0;
};

__device__ __forceinline__ double2 ld2(const float2* p, long long i) { const float2 v = p[i]; return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld2(const double2* p, long long i) { return p[i]; }
__device__ __forceinline__ double2 ld2(const float4* p, long long i) {
    const float4 v = p[i];
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
__device__ __forceinline__ void st2(float2* p, long long i, double2 v) { p[i] = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st2(double2* p, long long i, double2 v) { p[i] = v; }
__device__ __forceinline__ void st2(float4* p, long long i, double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    p[i] = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

// Stencil row of node i on a line of n nodes: fills idx/w, returns the count (7 centred or 8 one-sided).
__device__ __forceinline__ int lap_row(const Wts& W, int i, int n, int* idx, double* w) {
    if (i >= 3 && i <= n - 4) {
#pragma unroll
        for (int k = 0; k < 7; ++k) { idx[k] = i - 3 + k; w[k] = W.wc[k]; }
        return 7;
    }
    if (i < 3) {
#pragma unroll
        for (int k = 0; k < 8; ++k) { idx[k] = k; w[k] = W.wl[i][k]; }
        return 8;
    }
    // mirror image of the left rows
    const int r = n - 1 - i;
#pragma unroll
    for (int k = 0; k < 8; ++k) { idx[k] = n - 1 - k; w[k] = W.wl[r][k]; }
    return 8;
}

// L V at face point (ia, ib) for a face stored with strides (fa, fb) from base p
template <class M>
__device__ __forceinline__ double2 apply_L(const Face& f, const Wts& W, const M* p, long long base, long long fa,
                                           long long fb, int ia, int ib) {
    int idx[8];
    double w[8];
    double2 v = ld2(p, base + ia * fa + ib * fb);
    double2 acc = make_double2(f.k0 * f.k0 * v.x, f.k0 * f.k0 * v.y);
    int n = lap_row(W, ia, f.la, idx, w);
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
        const double2 u = ld2(p, base + idx[k] * fa + ib * fb);
        s.x += w[k] * u.x; s.y += w[k] * u.y;
    }
    acc.x += s.x * f.iha2; acc.y += s.y * f.iha2;
    n = lap_row(W, ib, f.lb, idx, w);
    s = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
        const double2 u = ld2(p, base + ia * fa + idx[k] * fb);
        s.x += w[k] * u.x; s.y += w[k] * u.y;
    }
    acc.x += s.x * f.ihb2; acc.y += s.y * f.ihb2;
    return acc;
}

__device__ __forceinline__ long long plane_base(const Face& f, int plane) {
    return plane * f.sn + f.sa0 * f.sa + f.sb0 * f.sb;
}

// copy the operand into the interior of the padded array
template <class M>
__global__ void ho_copy_kernel(int nx, int ny, int nz, const M* __restrict__ U, M* __restrict__ P) {
    const long long n = (long long)nx * ny * nz;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(id % nx);
        const long long r = id / nx;
        const int j = (int)(r % ny), l = (int)(r / ny);
        P[((long long)(l + 1) * (ny + 2) + (j + 1)) * (nx + 2) + (i + 1)] = U[id];
    }
}

// S[side][ia][ib] = L U_B on both boundary planes of one direction
template <class M>
__global__ void ho_lap_kernel(Face f, Wts W, const M* __restrict__ P, double2* __restrict__ S) {
    const long long per = (long long)f.la * f.lb;
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * per) return;
    const int side = (int)(id / per);
    const long long q = id - side * per;
    const int ia = (int)(q / f.lb), ib = (int)(q % f.lb);
    const long long base = plane_base(f, side ? f.nb_hi : f.nb_lo);
    S[id] = apply_L(f, W, P, base, f.sa, f.sb, ia, ib);
}

// U_G = U_I + i k0 (c0 U_B - c1 L U_B + c2 L^2 U_B) on both ghost planes of one direction, plus (when fd
// is given) the f part s [c1 f_n + c2 (f_nnn - k0^2 f_n - lap_T f_n)], s = -1 near face, +1 far face;
// fd holds [side][field][ia][ib] with the fields f_n, f_nnn, lap_T f_n (derivatives along the axis).
template <class M>
__global__ void ho_ghost_kernel(Face f, Wts W, M* __restrict__ P, const double2* __restrict__ S,
                                const double2* __restrict__ fd) {
    const long long per = (long long)f.la * f.lb;
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * per) return;
    const int side = (int)(id / per);
    const long long q = id - side * per;
    const int ia = (int)(q / f.lb), ib = (int)(q % f.lb);
    const int pb = side ? f.nb_hi : f.nb_lo;
    const int pi = side ? pb - 1 : pb + 1;
    const int pg = side ? pb + 1 : pb - 1;
    const long long off = ia * f.sa + ib * f.sb;
    const double2 ub = ld2(P, plane_base(f, pb) + off);
    const double2 ui = ld2(P, plane_base(f, pi) + off);
    const double2 v1 = S[id];
    const double2 v2 = apply_L(f, W, S, side * per, (long long)f.lb, 1LL, ia, ib);
    const double2 t = make_double2(f.c0 * ub.x - f.c1 * v1.x + f.c2 * v2.x, f.c0 * ub.y - f.c1 * v1.y + f.c2 * v2.y);
    // i k0 t
    double2 g = make_double2(ui.x - f.k0 * t.y, ui.y + f.k0 * t.x);
    if (fd) {
        const long long fb = (long long)side * 3 * per + q;
        const double2 fn = fd[fb], fnnn = fd[fb + per], flt = fd[fb + 2 * per];
        const double sg = side ? 1.0 : -1.0, kk = f.k0 * f.k0;
        g.x += sg * (f.c1 * fn.x + f.c2 * (fnnn.x - kk * fn.x - flt.x));
        g.y += sg * (f.c1 * fn.y + f.c2 * (fnnn.y - kk * fn.y - flt.y));
    }
    st2(P, plane_base(f, pg) + off, g);
}

// Second-derivative weights on offsets o_k (Taylor conditions sum_k w_k o_k^q / q! = [q == 2]), FP64
// Gaussian elimination with partial pivoting on the small Vandermonde system.
void fd_weights(const double* o, int n, double* w) {
    double A[8][9];
    for (int q = 0; q < n; ++q) {
        double fact = 1.0;
        for (int t = 2; t <= q; ++t) fact *= t;
        for (int k = 0; k < n; ++k) A[q][k] = std::pow(o[k], q) / fact;
        A[q][n] = q == 2 ? 1.0 : 0.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r) if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (piv != col) for (int k = 0; k <= n; ++k) std::swap(A[col][k], A[piv][k]);
        for (int r = col + 1; r < n; ++r) {
            const double m = A[r][col] / A[col][col];
            for (int k = col; k <= n; ++k) A[r][k] -= m * A[col][k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = A[r][n];
        for (int k = r + 1; k < n; ++k) s -= A[r][k] * w[k];
        w[r] = s / A[r][r];
    }
}

Wts make_weights() {
    Wts W;
    double o[8];
    for (int k = 0; k < 7; ++k) o[k] = k - 3;
    fd_weights(o, 7, W.wc);
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 8; ++k) o[k] = k - i;
        fd_weights(o, 8, W.wl[i]);
    }
    return W;
}

Face make_face(const helm_ctx* c, int axis) {
    const int n[3] = {c->nx, c->ny, c->nz};
    const long long st[3] = {1, (long long)(c->nx + 2), (long long)(c->nx + 2) * (c->ny + 2)};
    // tangential axes in array order: x-face (z, y), y-face (z, x), z-face (y, x)
    const int ta = axis == 2 ? 1 : 2, tb = axis == 0 ? 1 : 0;
    Face f;
    f.axis = axis;
    // a face covers the ghost columns of the directions filled before it
    f.la = ta < axis ? n[ta] + 2 : n[ta];
    f.lb = tb < axis ? n[tb] + 2 : n[tb];
    f.sa0 = ta < axis ? 0 : 1;
    f.sb0 = tb < axis ? 0 : 1;
    f.sn = st[axis]; f.sa = st[ta]; f.sb = st[tb];
    f.nb_lo = 1; f.nb_hi = n[axis];
    f.iha2 = 1.0 / (c->h[ta] * c->h[ta]);
    f.ihb2 = 1.0 / (c->h[tb] * c->h[tb]);
    const double h = c->h[axis];
    f.c0 = 2.0 * h;
    f.c1 = 2.0 * h * h * h / 6.0;
    f.c2 = 2.0 * h * h * h * h * h / 120.0;
    f.k0 = c->k0;
    return f;
}

// U = nullptr: the interior is zero (the f part of the closure alone); faces = nullptr: no f part.
template <class M>
helm_status fill(helm_ctx* c, const M* U, M* P, const double2* faces, cudaStream_t s) {
    if (U) {
        ho_copy_kernel<M><<<1024, 256, 0, s>>>(c->nx, c->ny, c->nz, U, P);
        HELM_CUDA_TRY(cudaGetLastError());
    } else {
        HELM_CUDA_TRY(cudaMemsetAsync(P, 0, (size_t)(c->nx + 2) * (c->ny + 2) * (c->nz + 2) * sizeof(M), s));
    }
    static const Wts W = make_weights();   // the same for every grid (weights times 1/h^2 per face)
    long long foff = 0;
    for (int axis = 0; axis < 3; ++axis) {
        const Face f = make_face(c, axis);
        const long long tot = 2LL * f.la * f.lb;
        const unsigned blocks = (unsigned)((tot + 255) / 256);
        ho_lap_kernel<M><<<blocks, 256, 0, s>>>(f, W, P, c->ho_S);
        HELM_CUDA_TRY(cudaGetLastError());
        ho_ghost_kernel<M><<<blocks, 256, 0, s>>>(f, W, P, c->ho_S, faces ? faces + foff : nullptr);
        HELM_CUDA_TRY(cudaGetLastError());
        foff += 3 * tot;
    }
    return HELM_OK;
}

__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out,
                           size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

}  // namespace

size_t closure_face_points(const helm_ctx* c) {
    size_t tot = 0;
    for (int axis = 0; axis < 3; ++axis) {
        const Face f = make_face(c, axis);
        tot += 2 * 3 * (size_t)f.la * f.lb;
    }
    return tot;
}

helm_status closure_fill_f32(helm_ctx* c, const float2* U, cudaStream_t s) { return fill(c, U, c->ho_P32, nullptr, s); }
helm_status closure_fill_f64(helm_ctx* c, const double2* U, cudaStream_t s) { return fill(c, U, c->ho_P64, nullptr, s); }
helm_status closure_fill_df(helm_ctx* c, const float4* U, cudaStream_t s) { return fill(c, U, c->ho_Pdf, nullptr, s); }

// F_out = F_in - A(G_f), G_f the ghosts of the closure's f part with a zero interior (FP64)
helm_status closure_rhs(helm_ctx* c, const double2* faces, const double2* Fin, double2* Fout, cudaStream_t s) {
    double2* y = nullptr;
    if (cudaMalloc(&y, c->npts * sizeof(double2)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    helm_status st = fill<double2>(c, nullptr, c->ho_P64, faces, s);
    if (st == HELM_OK) st = launch_stencil_f64_padded(c, c->ho_P64, y, s);
    if (st == HELM_OK) {
        sub_kernel<<<1024, 256, 0, s>>>(Fin, y, Fout, c->npts);
        if (cudaGetLastError() != cudaSuccess) st = HELM_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    cudaFree(y);
    return st;
}

void closure_release(helm_ctx* c) {
    void* ps[] = {c->ho_P32, c->ho_P64, c->ho_Pdf, c->ho_S};
    for (void* p : ps) if (p) cudaFree(p);
    c->ho_P32 = nullptr; c->ho_P64 = nullptr; c->ho_Pdf = nullptr; c->ho_S = nullptr;
    c->ho = 0;
}

extern "C" helm_status helm_set_closure(helm_ctx* c, int closure) {
    if (!c || (closure != HELM_CLOSURE_THREE_POINT && closure != HELM_CLOSURE_HIGH_ORDER)) return HELM_ERR_ARG;
    if (closure == HELM_CLOSURE_THREE_POINT) { closure_release(c); return HELM_OK; }
    // the one-sided rows need eight nodes on every face line
    if (!c->colloc || c->nx < 8 || c->ny < 8 || c->nz < 8) return HELM_ERR_UNSUPPORTED;
    if (c->ho) return HELM_OK;
    const size_t np = (size_t)(c->nx + 2) * (c->ny + 2) * (c->nz + 2);
    const int nmax = c->nx > c->ny ? (c->nx > c->nz ? c->nx : c->nz) : (c->ny > c->nz ? c->ny : c->nz);
    const size_t ns = 2 * (size_t)(nmax + 2) * (nmax + 2);
    if (cudaMalloc(&c->ho_P32, np * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&c->ho_P64, np * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->ho_Pdf, np * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&c->ho_S, ns * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        closure_release(c);
        return HELM_ERR_NOMEM;
    }
    // ghost planes are rewritten by every fill; zero once so that no word is ever undefined
    HELM_CUDA_TRY(cudaMemset(c->ho_P32, 0, np * sizeof(float2)));
    HELM_CUDA_TRY(cudaMemset(c->ho_P64, 0, np * sizeof(double2)));
    HELM_CUDA_TRY(cudaMemset(c->ho_Pdf, 0, np * sizeof(float4)));
    c->ho = 1;
    return HELM_OK;
}
