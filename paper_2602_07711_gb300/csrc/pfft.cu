// PFFT preconditioner (Sec. 4.2, Eq. PFFT_SOLVER): A_p U = Y solved with a sine-transform solver for A_p^F
// (Eq. TFprec) and a boundary correction.  Dirichlet at the face for A_p^F (ghost -U_1, corner -1): its x/y
// eigenvectors are S[l][j] = c_j sin(pi j (2l+1)/(2N)), eigenvalues 2 cos(pi j/N), j = 1..N (the DST-II
// basis: our reading of "Dirichlet" for N = 2^k).  Staggered grids (PFFT2: two-point ABC, zeta = 1) and
// collocated grids (PFFT3: three-point ABC, Lbar corner gamma = 2 i k0 h and corner neighbour zeta = 2).
//
//   1. Yh = S_y^T Y_l S_x (2D sine transform of every slice), Th = z-solve_F(Yh)
//   2. Theta on the boundary frame only (rows j = 0, N-1, columns i = 0, N-1; with zeta = 2 also the
//      second layer j = 1, N-2 and i = 1, N-2) from Th (sparse inverse transform); R = (A_p^F - A_p) Theta
//      lives on the frame: alpha [(-1 - gamma) Theta_boundary + (1 - zeta) Theta_second layer] there.
//      Rbar = V_y^-1 R V_x^-T is a sum of four outer products per slice; Wbar = z-solve_EigT(Rbar) takes
//      them as a generated right-hand side; W on the frame from Wbar (sparse inverse EigT transform).
//   3. R2 = (A_p^F - A_p)(Theta + W) on the frame; its sine transform is again four outer products,
//      added to the stored Yh inside the last z-solve; U = S_y Uh S_x^T.
// The sine transforms are hand-written batched FFTs: a length-N DST-II (DST-III) is a 2N-point complex
// FFT of the odd extension (z_n = x_n, z_{2N-1-n} = -x_n) with a post- (pre-) twiddle, done in shared
// memory by an in-place radix-2 Stockham iteration.  N_x, N_y must be powers of two (<= 512).
#include "common.cuh"
#include <cmath>
#include <vector>

namespace {

struct PfftState {
    int nx = 0, ny = 0, nz = 0;
    float2 *twx = nullptr, *twy = nullptr;          // e^{-2 pi i m/(2N)}, m < N
    float2 *fwx = nullptr, *fwy = nullptr;          // forward post-twiddle c_j (i/2) e^{-i pi j/(2N)}
    float2 *gpx = nullptr, *gpy = nullptr;          // inverse pre-twiddles c_j e^{+i pi j/(2N)}/(2i)
    float2 *gmx = nullptr, *gmy = nullptr;          //                    -c_j e^{-i pi j/(2N)}/(2i)
    float2 *Sx = nullptr, *Sy = nullptr;            // sine bases S[l][j] (row-major), complex64
    float2 *Vx = nullptr, *Vxi = nullptr, *Vy = nullptr, *Vyi = nullptr;   // EigT bases, complex64 row-major
    float2 *dxF = nullptr, *dyF = nullptr;          // alpha_x 2cos(pi j/N_x), alpha_y 2cos(pi j/N_y)
    float2* Yh = nullptr;                           // transformed right-hand side (kept for step 3)
    float2 *fa = nullptr, *fb = nullptr, *fc = nullptr;   // frame work vectors [4][nz][nmax]
    float2 *fb1 = nullptr, *fc1 = nullptr;          // second frame layer (zeta = 2): Theta, W
    float2 *P = nullptr, *Q = nullptr;              // outer-product factors [4][nz][ny], [4][nz][nx]
    float2* zfacF = nullptr;                        // Thomas factors of the z-systems of A_p^F
};

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ---- batched sine transforms ----------------------------------------------------------------------
// In-place radix-2 Stockham FFT of `lines` sequences of length n = 2N in shared memory (line stride ls).
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }   // v a power of two

__device__ void fft_smem(float2* buf, int lines, int n, int ls, const float2* tw) {
    const int half = n / 2, lh = ilog2(half);
    const int nb = lines * half;
    for (int lNs = 0; (1 << lNs) < n; ++lNs) {
        const int Ns = 1 << lNs;
        // read phase (at most MAXB butterflies per thread: the launch keeps lines * n/2 <= MAXB * blockDim)
        constexpr int MAXB = 8;
        float2 a[MAXB], b[MAXB];
#pragma unroll
        for (int c = 0; c < MAXB; ++c) {
            const int q = threadIdx.x + c * blockDim.x;
            if (q < nb) {
                const int line = q >> lh, j = q & (half - 1);
                const int k = j & (Ns - 1);
                const float2 x0 = buf[line * ls + j];
                const float2 x1 = cmul(buf[line * ls + j + half], tw[k << (lh - lNs)]);
                a[c] = cadd(x0, x1);
                b[c] = csub(x0, x1);
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MAXB; ++c) {
            const int q = threadIdx.x + c * blockDim.x;
            if (q < nb) {
                const int line = q >> lh, j = q & (half - 1);
                const int d = ((j >> lNs) << (lNs + 1)) + (j & (Ns - 1));
                buf[line * ls + d] = a[c];
                buf[line * ls + d + Ns] = b[c];
            }
        }
        __syncthreads();
    }
}

// x-direction lines (contiguous).  INV = 0: a = S^T x;  INV = 1: x = scale * S a.
template <int INV>
__global__ void __launch_bounds__(256) dst_x_kernel(const float2* __restrict__ in, float2* __restrict__ out, int N,
                                                    long lines, const float2* __restrict__ tw,
                                                    const float2* __restrict__ f1, const float2* __restrict__ f2,
                                                    int lpb, float scale, const double* sigma, int sidx) {
    extern __shared__ float2 sm[];
    const int n = 2 * N, ls = n + 1;
    float2* stw = sm;                 // N twiddles
    float2* buf = sm + N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = tw[m];
    const long l0 = (long)blockIdx.x * lpb;
    const int nl = (int)min((long)lpb, lines - l0);
    const float sc = scale * (sigma ? (float)sigma[sidx] : 1.f);
    const int lN = ilog2(N);
    for (int q = threadIdx.x; q < nl * N; q += blockDim.x) {
        const int line = q >> lN, e = q & (N - 1);
        const float2 v = in[(l0 + line) * N + e];
        float2* b = buf + line * ls;
        if (!INV) {
            b[e] = v;
            b[n - 1 - e] = make_float2(-v.x, -v.y);
        } else {
            // G_j = g+_j a_{j-1} (j = 1..N), G_{2N-j} += g-_j a_{j-1}; stored conjugated for the forward FFT
            const int j = e + 1;
            const float2 gp = cmul(f1[e], v), gm = cmul(f2[e], v);
            if (j < N) {
                b[j] = make_float2(gp.x, -gp.y);
                b[n - j] = make_float2(gm.x, -gm.y);
            } else {
                const float2 g = cadd(gp, gm);
                b[N] = make_float2(g.x, -g.y);
            }
            if (e == 0) b[0] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    fft_smem(buf, nl, n, ls, stw);
    for (int q = threadIdx.x; q < nl * N; q += blockDim.x) {
        const int line = q >> lN, e = q & (N - 1);
        const float2* b = buf + line * ls;
        float2 r;
        if (!INV) {
            r = cmul(f1[e], b[e + 1]);
        } else {
            const float2 z = b[e];
            r = make_float2(z.x, -z.y);
        }
        out[(l0 + line) * N + e] = make_float2(sc * r.x, sc * r.y);
    }
}

// y-direction lines: for slice l, columns i0..i0+ti-1, the line runs over j (stride nx).
template <int INV>
__global__ void __launch_bounds__(256) dst_y_kernel(const float2* __restrict__ in, float2* __restrict__ out, int nx,
                                                    int N, const float2* __restrict__ tw, const float2* __restrict__ f1,
                                                    const float2* __restrict__ f2, int ti, float scale) {
    extern __shared__ float2 sm[];
    const int n = 2 * N, ls = n + 1;
    float2* stw = sm;
    float2* buf = sm + N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = tw[m];
    const int i0 = blockIdx.x * ti, l = blockIdx.y;
    const int nt = min(ti, nx - i0);
    const size_t sbase = (size_t)l * N * nx;
    const int lt = ilog2(ti);
    for (int q = threadIdx.x; q < N * ti; q += blockDim.x) {
        const int e = q >> lt, t = q & (ti - 1);  // consecutive threads: consecutive columns (coalesced)
        if (t >= nt) continue;
        const float2 v = in[sbase + (size_t)e * nx + i0 + t];
        float2* b = buf + t * ls;
        if (!INV) {
            b[e] = v;
            b[n - 1 - e] = make_float2(-v.x, -v.y);
        } else {
            const int j = e + 1;
            const float2 gp = cmul(f1[e], v), gm = cmul(f2[e], v);
            if (j < N) {
                b[j] = make_float2(gp.x, -gp.y);
                b[n - j] = make_float2(gm.x, -gm.y);
            } else {
                const float2 g = cadd(gp, gm);
                b[N] = make_float2(g.x, -g.y);
            }
            if (e == 0) b[0] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    fft_smem(buf, nt, n, ls, stw);
    for (int q = threadIdx.x; q < N * ti; q += blockDim.x) {
        const int e = q >> lt, t = q & (ti - 1);
        if (t >= nt) continue;
        const float2* b = buf + t * ls;
        float2 r;
        if (!INV) r = cmul(f1[e], b[e + 1]);
        else { const float2 z = b[e]; r = make_float2(z.x, -z.y); }
        out[sbase + (size_t)e * nx + i0 + t] = make_float2(scale * r.x, scale * r.y);
    }
}

// ---- frame extraction ------------------------------------------------------------------------------
// TT[l][i] = sum_j wr0[j] C[l][j][i],  TB[l][i] = sum_j wr1[j] C[l][j][i]   (weights over rows)
__global__ void frame_cols_kernel(const float2* __restrict__ C, int nx, int ny, const float2* __restrict__ wr0,
                                  const float2* __restrict__ wr1, float2* __restrict__ TT, float2* __restrict__ TB,
                                  int ld) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, l = blockIdx.y;
    if (i >= nx) return;
    const float2* s = C + (size_t)l * nx * ny;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    for (int j = 0; j < ny; ++j) {
        const float2 v = s[(size_t)j * nx + i];
        a = cfma(wr0[j], v, a);
        b = cfma(wr1[j], v, b);
    }
    TT[(size_t)l * ld + i] = a;
    TB[(size_t)l * ld + i] = b;
}

// UL[l][j] = sum_i C[l][j][i] wc0[i],  UR[l][j] = sum_i C[l][j][i] wc1[i]   (one warp per row)
__global__ void frame_rows_kernel(const float2* __restrict__ C, int nx, int ny, const float2* __restrict__ wc0,
                                  const float2* __restrict__ wc1, float2* __restrict__ UL, float2* __restrict__ UR,
                                  int ld) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + warp, l = blockIdx.y;
    if (j >= ny) return;
    const float2* row = C + ((size_t)l * ny + j) * nx;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    for (int i = lane; i < nx; i += 32) {
        const float2 v = row[i];
        a = cfma(v, wc0[i], a);
        b = cfma(v, wc1[i], b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, o); a.y += __shfl_down_sync(0xffffffffu, a.y, o);
        b.x += __shfl_down_sync(0xffffffffu, b.x, o); b.y += __shfl_down_sync(0xffffffffu, b.y, o);
    }
    if (lane == 0) { UL[(size_t)l * ld + j] = a; UR[(size_t)l * ld + j] = b; }
}

// out[b][r] = alpha * sum_k M(r, k) in[b][k]; M(r, k) = Mat[r][k] (trans = 0) or Mat[k][r] (trans = 1).
// optional add: out += add (same layout).  Vectors of length n, stride ld; one CTA per vector.
// Batched dense matrix times vector: out_b = alpha Mat v_b (+ add_b) for the nvec vectors v_b = in[b ld ..],
// NV vectors per block (every row of Mat read from L2 serves NV of them).  trans = 0 reads Mat row by row
// (one warp per row, lanes along the row, warp-shuffle sums); trans = 1 multiplies by Mat^T (one thread per
// output, lanes along the row index), so both forms read Mat coalesced.
template <int NV>
__global__ void matvec_kernel(const float2* __restrict__ Mat, int n, int trans, const float2* __restrict__ in,
                              float2* __restrict__ out, int ld, float2 alpha, const float2* __restrict__ add, int nvec) {
    extern __shared__ float2 v[];   // [NV][n]
    const int b0 = blockIdx.x * NV;
    const int nb = min(NV, nvec - b0);
    for (int q = 0; q < NV; ++q)
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            v[q * n + k] = q < nb ? in[(size_t)(b0 + q) * ld + k] : make_float2(0.f, 0.f);
    __syncthreads();
    if (trans) {
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            float2 acc[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int k = 0; k < n; ++k) {
                const float2 m = Mat[(size_t)k * n + r];
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[q] = cfma(m, v[q * n + k], acc[q]);
            }
            for (int q = 0; q < nb; ++q) {
                float2 o = cmul(alpha, acc[q]);
                if (add) o = cadd(o, add[(size_t)(b0 + q) * ld + r]);
                out[(size_t)(b0 + q) * ld + r] = o;
            }
        }
    } else {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = threadIdx.x >> 5; r < n; r += nw) {
            float2 acc[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int k = lane; k < n; k += 32) {
                const float2 m = Mat[(size_t)r * n + k];
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[q] = cfma(m, v[q * n + k], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < NV; ++q)
                for (int o = 16; o > 0; o >>= 1) {
                    acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, o);
                    acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, o);
                }
            if (lane == 0)
                for (int q = 0; q < nb; ++q) {
                    float2 o = cmul(alpha, acc[q]);
                    if (add) o = cadd(o, add[(size_t)(b0 + q) * ld + r]);
                    out[(size_t)(b0 + q) * ld + r] = o;
                }
        }
    }
}

constexpr int MV_NV = 1;   // one vector per block: nz blocks fill the GPU
void launch_matvec(int nvec, cudaStream_t s, const float2* Mat, int n, int trans, const float2* in, float2* out, int ld,
                   float2 alpha, const float2* add) {
    matvec_kernel<MV_NV><<<(nvec + MV_NV - 1) / MV_NV, 256, MV_NV * n * sizeof(float2), s>>>(Mat, n, trans, in, out, ld,
                                                                                         alpha, add, nvec);
}

// out[t][l][m] = vec[m] for every slice l (t fixed): fills the slice-independent outer-product factors
__global__ void fill_kernel(float2* __restrict__ out, int nz, int n, const float2* __restrict__ vec, int vstride,
                            int voff) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)nz * n) return;
    const int m = (int)(id % n);
    out[id] = vec[(size_t)m * vstride + voff];
}

// c = s (a + b) + t (a1 + b1) elementwise (frame values -> correction vectors; b, b1 may be NULL, and a1
// is NULL for a one-layer frame)
__global__ void frame_scale_kernel(const float2* __restrict__ a, const float2* __restrict__ b, const float2* a1,
                                   const float2* b1, float2* c, size_t n, float2 s, float2 t) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= n) return;
    float2 v = a[id];
    if (b) v = cadd(v, b[id]);
    float2 o = cmul(s, v);
    if (a1) {
        float2 w = a1[id];
        if (b1) w = cadd(w, b1[id]);
        o = cfma(t, w, o);
    }
    c[id] = o;
}

__global__ void to_c64_kernel(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id < n) b[id] = make_float2((float)a[id].x, (float)a[id].y);
}

template <typename T>
helm_status dmal(T** p, size_t n) {
    if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    return HELM_OK;
}

helm_status upload(float2* d, const std::vector<float2>& h, cudaStream_t s) {
    HELM_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    return HELM_OK;
}

// host tables for one axis of length N
void axis_tables(int N, double alpha, std::vector<float2>& tw, std::vector<float2>& f1, std::vector<float2>& gp,
                 std::vector<float2>& gm, std::vector<float2>& S, std::vector<float2>& dF) {
    const int n = 2 * N;
    tw.resize(N); f1.resize(N); gp.resize(N); gm.resize(N); S.resize((size_t)N * N); dF.resize(N);
    for (int m = 0; m < N; ++m) tw[m] = make_float2((float)cos(-2.0 * M_PI * m / n), (float)sin(-2.0 * M_PI * m / n));
    for (int e = 0; e < N; ++e) {
        const int j = e + 1;
        const double c = j < N ? sqrt(2.0 / N) : sqrt(1.0 / N);
        const double ph = M_PI * j / (2.0 * N);
        // c (i/2) e^{-i ph}
        f1[e] = make_float2((float)(c * 0.5 * sin(ph)), (float)(c * 0.5 * cos(ph)));
        // c e^{i ph}/(2i) = (c/2)(sin ph - i cos ph);  -c e^{-i ph}/(2i) = (c/2)(sin ph + i cos ph)
        gp[e] = make_float2((float)(0.5 * c * sin(ph)), (float)(-0.5 * c * cos(ph)));
        gm[e] = make_float2((float)(0.5 * c * sin(ph)), (float)(0.5 * c * cos(ph)));
        dF[e] = make_float2((float)(alpha * 2.0 * cos(M_PI * j / N)), 0.f);
    }
    for (int l = 0; l < N; ++l)
        for (int e = 0; e < N; ++e) {
            const int j = e + 1;
            const double c = j < N ? sqrt(2.0 / N) : sqrt(1.0 / N);
            S[(size_t)l * N + e] = make_float2((float)(c * sin(M_PI * j * (2.0 * l + 1) / (2.0 * N))), 0.f);
        }
}

size_t xsmem(int N, int lpb) { return (size_t)(N + lpb * (2 * N + 1)) * sizeof(float2); }

// butterflies per stage = lines * N <= 8 * 256 (see fft_smem)
int lines_per_block(int N) { return 1024 / N; }
int cols_per_block(int N) { const int t = 2048 / N; return t > 64 ? 64 : t; }

}  // namespace

helm_status pfft_prepare(helm_ctx* c, cudaStream_t s) {
    if (!pow2(c->nx) || !pow2(c->ny) || c->nx > 512 || c->ny > 512 || c->nx < 4 || c->ny < 4)
        return HELM_ERR_UNSUPPORTED;
    PfftState* P = new PfftState();
    c->pfft = P;
    P->nx = c->nx; P->ny = c->ny; P->nz = c->nz;
    const int nx = c->nx, ny = c->ny, nz = c->nz, nm = nx > ny ? nx : ny;
    std::vector<float2> tw, f1, gp, gm, S, dF;
    helm_status st;
    axis_tables(nx, c->ax, tw, f1, gp, gm, S, dF);
    if ((st = dmal(&P->twx, nx)) || (st = dmal(&P->fwx, nx)) || (st = dmal(&P->gpx, nx)) || (st = dmal(&P->gmx, nx)) ||
        (st = dmal(&P->Sx, (size_t)nx * nx)) || (st = dmal(&P->dxF, nx))) return st;
    if ((st = upload(P->twx, tw, s)) || (st = upload(P->fwx, f1, s)) || (st = upload(P->gpx, gp, s)) ||
        (st = upload(P->gmx, gm, s)) || (st = upload(P->Sx, S, s)) || (st = upload(P->dxF, dF, s))) return st;
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    axis_tables(ny, c->ay, tw, f1, gp, gm, S, dF);
    if ((st = dmal(&P->twy, ny)) || (st = dmal(&P->fwy, ny)) || (st = dmal(&P->gpy, ny)) || (st = dmal(&P->gmy, ny)) ||
        (st = dmal(&P->Sy, (size_t)ny * ny)) || (st = dmal(&P->dyF, ny))) return st;
    if ((st = upload(P->twy, tw, s)) || (st = upload(P->fwy, f1, s)) || (st = upload(P->gpy, gp, s)) ||
        (st = upload(P->gmy, gm, s)) || (st = upload(P->Sy, S, s)) || (st = upload(P->dyF, dF, s))) return st;
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = dmal(&P->Vx, (size_t)nx * nx)) || (st = dmal(&P->Vxi, (size_t)nx * nx)) ||
        (st = dmal(&P->Vy, (size_t)ny * ny)) || (st = dmal(&P->Vyi, (size_t)ny * ny))) return st;
    to_c64_kernel<<<(unsigned)((nx * (size_t)nx + 255) / 256), 256, 0, s>>>(c->Vx, P->Vx, (size_t)nx * nx);
    to_c64_kernel<<<(unsigned)((nx * (size_t)nx + 255) / 256), 256, 0, s>>>(c->Vxi, P->Vxi, (size_t)nx * nx);
    to_c64_kernel<<<(unsigned)((ny * (size_t)ny + 255) / 256), 256, 0, s>>>(c->Vy, P->Vy, (size_t)ny * ny);
    to_c64_kernel<<<(unsigned)((ny * (size_t)ny + 255) / 256), 256, 0, s>>>(c->Vyi, P->Vyi, (size_t)ny * ny);
    HELM_CUDA_TRY(cudaGetLastError());
    if ((st = dmal(&P->Yh, c->npts))) return st;
    const size_t fv = (size_t)4 * nz * nm;
    if ((st = dmal(&P->fa, fv)) || (st = dmal(&P->fb, fv)) || (st = dmal(&P->fc, fv))) return st;
    if (c->zeta[0] != 1.0 || c->zeta[1] != 1.0)
        if ((st = dmal(&P->fb1, fv)) || (st = dmal(&P->fc1, fv))) return st;
    if ((st = dmal(&P->P, (size_t)4 * nz * ny)) || (st = dmal(&P->Q, (size_t)4 * nz * nx))) return st;
    if ((st = zsolve_factor_with(c, P->dxF, P->dyF, &P->zfacF, s))) return st;
    if (c->tmaps) {
        // TF32 contexts: the sine transforms run as dense products on the tensor cores (operand sets 2, 3)
        std::vector<double2> hS[4];
        const int nn[2] = {nx, ny};
        for (int a = 0; a < 2; ++a) {
            const int N = nn[a];
            hS[2 * a].resize((size_t)N * N);
            hS[2 * a + 1].resize((size_t)N * N);
            for (int l = 0; l < N; ++l)
                for (int e = 0; e < N; ++e) {
                    const int j = e + 1;
                    const double cc = j < N ? sqrt(2.0 / N) : sqrt(1.0 / N);
                    const double v = cc * sin(M_PI * j * (2.0 * l + 1) / (2.0 * N));
                    hS[2 * a][(size_t)l * N + e] = make_double2(v, 0.0);       // S[l][j]
                    hS[2 * a + 1][(size_t)e * N + l] = make_double2(v, 0.0);   // S^T
                }
        }
        double2* dS[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int k = 0; k < 4; ++k) {
            if (cudaMalloc(&dS[k], hS[k].size() * sizeof(double2)) != cudaSuccess) {
                cudaGetLastError();
                for (int q = 0; q < k; ++q) cudaFree(dS[q]);
                return HELM_ERR_NOMEM;
            }
            HELM_CUDA_TRY(cudaMemcpyAsync(dS[k], hS[k].data(), hS[k].size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        }
        st = tc_prepare_sine(c, dS[0], dS[2], dS[1], dS[3], s);
        cudaStreamSynchronize(s);
        for (int k = 0; k < 4; ++k) cudaFree(dS[k]);
        if (st != HELM_OK) return st;
    }
    const int lpbx = lines_per_block(nx), lpby = cols_per_block(ny);
    HELM_CUDA_TRY(cudaFuncSetAttribute(dst_x_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem(nx, lpbx)));
    HELM_CUDA_TRY(cudaFuncSetAttribute(dst_x_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem(nx, lpbx)));
    HELM_CUDA_TRY(cudaFuncSetAttribute(dst_y_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem(ny, lpby)));
    HELM_CUDA_TRY(cudaFuncSetAttribute(dst_y_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsmem(ny, lpby)));
    return HELM_OK;
}

void pfft_release(helm_ctx* c) {
    PfftState* P = (PfftState*)c->pfft;
    if (!P) return;
    void* ps[] = {P->twx, P->twy, P->fwx, P->fwy, P->gpx, P->gpy, P->gmx, P->gmy, P->Sx, P->Sy, P->Vx, P->Vxi,
                  P->Vy, P->Vyi, P->dxF, P->dyF, P->Yh, P->fa, P->fb, P->fc, P->fb1, P->fc1, P->P, P->Q, P->zfacF};
    for (void* p : ps) if (p) cudaFree(p);
    delete P;
    c->pfft = nullptr;
}

namespace {

helm_status dst2d(helm_ctx* c, PfftState* P, int inv, const float2* in, float2* out, float scale, const double* sigma,
                  int sidx, cudaStream_t s) {
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const long lines = (long)ny * nz;
    const int lpbx = lines_per_block(nx), tiy = cols_per_block(ny);
    const dim3 gy((nx + tiy - 1) / tiy, nz);
    if (c->tmaps) {
        // tensor-core products with the sine bases (same data flow as the EigT transforms)
        helm_status st;
        if (!inv) {
            if ((st = tc_xpass(c, 2, in, c->tmp, 1.f, sigma, sidx, s)) != HELM_OK) return st;
            return tc_ypass(c, 2, c->tmp, out, s);
        }
        if ((st = tc_ypass(c, 3, in, c->tmp, s)) != HELM_OK) return st;
        return tc_xpass(c, 3, c->tmp, out, scale, nullptr, 0, s);
    }
    if (!inv) {
        // x then y: in -> ctx tmp -> out
        dst_x_kernel<0><<<(unsigned)((lines + lpbx - 1) / lpbx), 256, xsmem(nx, lpbx), s>>>(
            in, c->tmp, nx, lines, P->twx, P->fwx, nullptr, lpbx, 1.f, sigma, sidx);
        dst_y_kernel<0><<<gy, 256, xsmem(ny, tiy), s>>>(c->tmp, out, nx, ny, P->twy, P->fwy, nullptr, tiy, scale);
    } else {
        dst_y_kernel<1><<<gy, 256, xsmem(ny, tiy), s>>>(in, c->tmp, nx, ny, P->twy, P->gpy, P->gmy, tiy, 1.f);
        dst_x_kernel<1><<<(unsigned)((lines + lpbx - 1) / lpbx), 256, xsmem(nx, lpbx), s>>>(
            c->tmp, out, nx, lines, P->twx, P->gpx, P->gmx, lpbx, scale, nullptr, 0);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// layer k of the frame of M_y C M_x^T (rows k, N-1-k and columns k, N-1-k of every slice) into fr: [0] row
// k, [1] row N-1-k (length nx), [2] column k, [3] column N-1-k (length ny); the row weights are rows k,
// N-1-k of M_y and of M_x; Mx, My full matrices.  Uses fa as scratch.
helm_status frame_of(helm_ctx* c, PfftState* P, const float2* C, const float2* Mx, const float2* My, float2* fr,
                     cudaStream_t s, int k = 0) {
    const int nx = P->nx, ny = P->ny, nz = P->nz, nm = nx > ny ? nx : ny;
    const size_t blk = (size_t)nz * nm;
    float2* TT = P->fa;
    float2* TB = P->fa + blk;
    float2* UL = P->fa + 2 * blk;
    float2* UR = P->fa + 3 * blk;
    frame_cols_kernel<<<dim3((nx + 127) / 128, nz), 128, 0, s>>>(C, nx, ny, My + (size_t)k * ny,
                                                                 My + (size_t)(ny - 1 - k) * ny, TT, TB, nm);
    frame_rows_kernel<<<dim3((ny + 7) / 8, nz), 256, 0, s>>>(C, nx, ny, Mx + (size_t)k * nx,
                                                             Mx + (size_t)(nx - 1 - k) * nx, UL, UR, nm);
    const float2 one = make_float2(1.f, 0.f);
    // rows: Theta[0][i] = sum_i' Mx[i][i'] TT[i'];  columns: Theta[j][0] = sum_j' My[j][j'] UL[j']
    launch_matvec(nz, s, Mx, nx, 0, TT, fr, nm, one, nullptr);
    launch_matvec(nz, s, Mx, nx, 0, TB, fr + blk, nm, one, nullptr);
    launch_matvec(nz, s, My, ny, 0, UL, fr + 2 * blk, nm, one, nullptr);
    launch_matvec(nz, s, My, ny, 0, UR, fr + 3 * blk, nm, one, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

}  // namespace

// FFT2: the Dirichlet solve alone, z = h_z^2 (A_p^F)^-1 r (step 1 of PFFT: sine transforms of every slice,
// the factorised z-solves with the Dirichlet lateral eigenvalues, inverse sine transforms)
helm_status pfft_apply_dirichlet(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx,
                                 cudaStream_t s) {
    PfftState* P = (PfftState*)c->pfft;
    if (!P) return HELM_ERR_UNSUPPORTED;
    helm_status st;
    if ((st = dst2d(c, P, 0, r, P->Yh, 1.f, sigma, sidx, s)) != HELM_OK) return st;
    if ((st = launch_zsolve_fact(c, P->zfacF, P->Yh, P->Yh, nullptr, nullptr, s)) != HELM_OK) return st;
    const float hz2 = (float)(c->h[2] * c->h[2]);
    return dst2d(c, P, 1, P->Yh, z, hz2, nullptr, 0, s);
}

helm_status pfft_apply(helm_ctx* c, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s) {
    PfftState* P = (PfftState*)c->pfft;
    if (!P) return HELM_ERR_UNSUPPORTED;
    const int nx = P->nx, ny = P->ny, nz = P->nz, nm = nx > ny ? nx : ny;
    const size_t blk = (size_t)nz * nm;
    helm_status st;
    const float2 one = make_float2(1.f, 0.f);
    // (A_p^F - A_p) on the frame: alpha_d (-1 - gamma_d) times the boundary layer, plus alpha_d (1 - zeta_d)
    // times the second layer (zeta = 2 on collocated grids; nothing for zeta = 1)
    const float2 ex = make_float2((float)(c->ax * (-1.0 - c->gam[0].x)), (float)(c->ax * (-c->gam[0].y)));
    const float2 ey = make_float2((float)(c->ay * (-1.0 - c->gam[1].x)), (float)(c->ay * (-c->gam[1].y)));
    const float2 tx = make_float2((float)(c->ax * (1.0 - c->zeta[0])), 0.f);
    const float2 ty = make_float2((float)(c->ay * (1.0 - c->zeta[1])), 0.f);
    const bool two = P->fb1 != nullptr;
    // 1. Yh = S_y^T Y S_x ; Th = z-solve_F(Yh) -> tmp2 (z is free until the end)
    if ((st = dst2d(c, P, 0, r, P->Yh, 1.f, sigma, sidx, s)) != HELM_OK) return st;
    if ((st = launch_zsolve_fact(c, P->zfacF, P->Yh, z, nullptr, nullptr, s)) != HELM_OK) return st;
    // 2. Theta on the frame (fb; second layer fb1), R vectors (fc): rows scaled by e_y, t_y, columns by e_x, t_x
    if ((st = frame_of(c, P, z, P->Sx, P->Sy, P->fb, s)) != HELM_OK) return st;
    if (two && (st = frame_of(c, P, z, P->Sx, P->Sy, P->fb1, s, 1)) != HELM_OK) return st;
    frame_scale_kernel<<<(unsigned)((2 * blk + 255) / 256), 256, 0, s>>>(P->fb, nullptr, two ? P->fb1 : nullptr,
                                                                        nullptr, P->fc, 2 * blk, ey, ty);
    frame_scale_kernel<<<(unsigned)((2 * blk + 255) / 256), 256, 0, s>>>(
        P->fb + 2 * blk, nullptr, two ? P->fb1 + 2 * blk : nullptr, nullptr, P->fc + 2 * blk, 2 * blk, ex, tx);
    // Rbar = sum of four outer products: (Vyi e_0)(Vxi ryT)^T + (Vyi e_N)(Vxi ryB)^T + (Vyi cxL)(Vxi e_0)^T + ...
    //   P[0] = Vyi[:, 0], P[1] = Vyi[:, N-1], P[2] = Vyi cxL, P[3] = Vyi cxR
    //   Q[0] = Vxi ryT,   Q[1] = Vxi ryB,     Q[2] = Vxi[:, 0], Q[3] = Vxi[:, N-1]
    fill_kernel<<<(unsigned)((nz * (size_t)ny + 255) / 256), 256, 0, s>>>(P->P, nz, ny, P->Vyi, ny, 0);
    fill_kernel<<<(unsigned)((nz * (size_t)ny + 255) / 256), 256, 0, s>>>(P->P + (size_t)nz * ny, nz, ny, P->Vyi, ny, ny - 1);
    fill_kernel<<<(unsigned)((nz * (size_t)nx + 255) / 256), 256, 0, s>>>(P->Q + 2 * (size_t)nz * nx, nz, nx, P->Vxi, nx, 0);
    fill_kernel<<<(unsigned)((nz * (size_t)nx + 255) / 256), 256, 0, s>>>(P->Q + 3 * (size_t)nz * nx, nz, nx, P->Vxi, nx, nx - 1);
    // matvec outputs are written with stride n of the factor arrays
    launch_matvec(nz, s, P->Vyi, ny, 0, P->fc + 2 * blk, P->fa, nm, one, nullptr);
    launch_matvec(nz, s, P->Vyi, ny, 0, P->fc + 3 * blk, P->fa + blk, nm, one, nullptr);
    launch_matvec(nz, s, P->Vxi, nx, 0, P->fc, P->fa + 2 * blk, nm, one, nullptr);
    launch_matvec(nz, s, P->Vxi, nx, 0, P->fc + blk, P->fa + 3 * blk, nm, one, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    // repack to the factor layouts P[t][l][j], Q[t][l][i]
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->P + 2 * (size_t)nz * ny, ny * sizeof(float2), P->fa, nm * sizeof(float2),
                                    ny * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->P + 3 * (size_t)nz * ny, ny * sizeof(float2), P->fa + blk, nm * sizeof(float2),
                                    ny * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->Q, nx * sizeof(float2), P->fa + 2 * blk, nm * sizeof(float2), nx * sizeof(float2),
                                    nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->Q + (size_t)nz * nx, nx * sizeof(float2), P->fa + 3 * blk, nm * sizeof(float2),
                                    nx * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    //    Wbar = z-solve_EigT(Rbar) into z; W on the frame (fc) from Wbar with the EigT bases
    if ((st = launch_zsolve_fact(c, c->zfac, nullptr, z, P->P, P->Q, s)) != HELM_OK) return st;
    if ((st = frame_of(c, P, z, P->Vx, P->Vy, P->fc, s)) != HELM_OK) return st;
    if (two && (st = frame_of(c, P, z, P->Vx, P->Vy, P->fc1, s, 1)) != HELM_OK) return st;
    // 3. R2 = (A_p^F - A_p)(Theta + W) on the frame -> fc (rows e_y, t_y, columns e_x, t_x)
    frame_scale_kernel<<<(unsigned)((2 * blk + 255) / 256), 256, 0, s>>>(
        P->fb, P->fc, two ? P->fb1 : nullptr, two ? P->fc1 : nullptr, P->fc, 2 * blk, ey, ty);
    frame_scale_kernel<<<(unsigned)((2 * blk + 255) / 256), 256, 0, s>>>(
        P->fb + 2 * blk, P->fc + 2 * blk, two ? P->fb1 + 2 * blk : nullptr, two ? P->fc1 + 2 * blk : nullptr,
        P->fc + 2 * blk, 2 * blk, ex, tx);
    //    sine transform of R2 as four outer products:
    //   P[0] = S_y[0][:], P[1] = S_y[N-1][:], P[2] = S_y^T c2L, P[3] = S_y^T c2R
    //   Q[0] = S_x^T r2T, Q[1] = S_x^T r2B,   Q[2] = S_x[0][:], Q[3] = S_x[N-1][:]
    fill_kernel<<<(unsigned)((nz * (size_t)ny + 255) / 256), 256, 0, s>>>(P->P, nz, ny, P->Sy, 1, 0);
    fill_kernel<<<(unsigned)((nz * (size_t)ny + 255) / 256), 256, 0, s>>>(P->P + (size_t)nz * ny, nz, ny,
                                                                        P->Sy + (size_t)(ny - 1) * ny, 1, 0);
    fill_kernel<<<(unsigned)((nz * (size_t)nx + 255) / 256), 256, 0, s>>>(P->Q + 2 * (size_t)nz * nx, nz, nx, P->Sx, 1, 0);
    fill_kernel<<<(unsigned)((nz * (size_t)nx + 255) / 256), 256, 0, s>>>(P->Q + 3 * (size_t)nz * nx, nz, nx,
                                                                        P->Sx + (size_t)(nx - 1) * nx, 1, 0);
    launch_matvec(nz, s, P->Sy, ny, 1, P->fc + 2 * blk, P->fa, nm, one, nullptr);
    launch_matvec(nz, s, P->Sy, ny, 1, P->fc + 3 * blk, P->fa + blk, nm, one, nullptr);
    launch_matvec(nz, s, P->Sx, nx, 1, P->fc, P->fa + 2 * blk, nm, one, nullptr);
    launch_matvec(nz, s, P->Sx, nx, 1, P->fc + blk, P->fa + 3 * blk, nm, one, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->P + 2 * (size_t)nz * ny, ny * sizeof(float2), P->fa, nm * sizeof(float2),
                                    ny * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->P + 3 * (size_t)nz * ny, ny * sizeof(float2), P->fa + blk, nm * sizeof(float2),
                                    ny * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->Q, nx * sizeof(float2), P->fa + 2 * blk, nm * sizeof(float2), nx * sizeof(float2),
                                    nz, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaMemcpy2DAsync(P->Q + (size_t)nz * nx, nx * sizeof(float2), P->fa + 3 * blk, nm * sizeof(float2),
                                    nx * sizeof(float2), nz, cudaMemcpyDeviceToDevice, s));
    //    Uh = z-solve_F(Yh + sine transform of R2) in place in Yh; U = h_z^2 S_y Uh S_x^T
    if ((st = launch_zsolve_fact(c, P->zfacF, P->Yh, P->Yh, P->P, P->Q, s)) != HELM_OK) return st;
    const float hz2 = (float)(c->h[2] * c->h[2]);
    return dst2d(c, P, 1, P->Yh, z, hz2, nullptr, 0, s);
}
