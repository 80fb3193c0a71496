// Stencil kernels: the compact 4th/6th-order operator A with the two-point ABC ghosts eliminated,
// its FP64 residual form, the coefficient fields of the sixth-order scheme and the modified
// right-hand sides.
//
//   Eq. scheme4 (P. Sec. 2.2): (dxx+dyy+dzz)U + sum_pairs (ha^2+hb^2)/12 da2 db2 U
//                               + (1 + sum_d hd^2/12 dd2)(k^2 U)
//   Eq. scheme6 (Sec. 2.3, uniform h), with the difference operators acting on the product grid
//   functions k^2 U and the U-free parts moved to the right-hand side:
//     L[(1 + h^2 k^2/30)U] + h^4/30 dxx dyy dzz U + k^2 U + h^2/6 M[(1 + h^2 k^2/15)U]
//     + h^2/20 { (lap k^2 - k^4) U + 2 sum_d (k^2)_d ( d_d[(1 + h^2 k^2/6)U] + h^2/6 d_d T_d U ) }
//   Ghosts (Eq. D_bc): U_0 = gamma U_1, U_{N+1} = gamma U_N per direction (edge and corner ghosts take
//   the product of the gammas); k^2 at a ghost is the mirror value of its neighbour.
//
// Design: 2.5D blocking.  A CTA owns a 32 x 8 column tile and marches along z through ZCH planes.
// Each plane (with a one-point halo) is staged once in shared memory; every thread lifts its 3 x 3
// neighbourhood into registers and keeps the previous two planes there, so a point costs 9 + 9
// shared-memory reads and one HBM read/write of each field (24 B/pt at order 4, 56 B/pt at order 6).
#include "common.cuh"

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int PX = TX + 2;
constexpr int PY = TY + 2;
constexpr int ZCH = 32;

template <typename C>
__device__ inline C czero() { C r; r.x = 0; r.y = 0; return r; }

// Fetch U at (X, Y, Z) with the ghost rule (at most one point outside in each direction).
template <typename R>
__device__ inline typename cplx<R>::t fetch_u(const StencilParams<R>& p, const typename cplx<R>::t* __restrict__ U,
                                              int X, int Y, int Z) {
    typedef typename cplx<R>::t C;
    int Xc = X < 0 ? 0 : (X >= p.nx ? p.nx - 1 : X);
    int Yc = Y < 0 ? 0 : (Y >= p.ny ? p.ny - 1 : Y);
    int Zc = Z < 0 ? 0 : (Z >= p.nz ? p.nz - 1 : Z);
    C v = U[((size_t)Zc * p.ny + Yc) * p.nx + Xc];
    if (Xc != X) v = cmul(v, p.gx);
    if (Yc != Y) v = cmul(v, p.gy);
    if (Zc != Z) v = cmul(v, p.gz);
    return v;
}

template <typename R>
__device__ inline typename cplx<R>::t fetch_k(const StencilParams<R>& p, int X, int Y, int Z) {
    int Xc = X < 0 ? 0 : (X >= p.nx ? p.nx - 1 : X);
    int Yc = Y < 0 ? 0 : (Y >= p.ny ? p.ny - 1 : Y);
    int Zc = Z < 0 ? 0 : (Z >= p.nz ? p.nz - 1 : Z);
    return p.k2[((size_t)Zc * p.ny + Yc) * p.nx + Xc];
}

// A at one point from its 3x3x3 neighbourhood u[c][b][a] (a = x offset + 1, b = y, c = z).
template <typename R, int ORDER>
__device__ inline typename cplx<R>::t apply_point(const StencilParams<R>& p, const typename cplx<R>::t (&u)[3][3][3],
                                                  const typename cplx<R>::t (&k)[3][3][3], size_t gidx) {
    typedef typename cplx<R>::t C;
    const C uc = u[1][1][1];
    const C kc = k[1][1][1];
    if (ORDER == 2 || ORDER == 4) {
        const R ihx = R(1) / (p.hx * p.hx), ihy = R(1) / (p.hy * p.hy), ihz = R(1) / (p.hz * p.hz);
        C fx = cadd(u[1][1][0], u[1][1][2]);
        C fy = cadd(u[1][0][1], u[1][2][1]);
        C fz = cadd(u[0][1][1], u[2][1][1]);
        C out;
        out.x = (fx.x - 2 * uc.x) * ihx + (fy.x - 2 * uc.x) * ihy + (fz.x - 2 * uc.x) * ihz;
        out.y = (fx.y - 2 * uc.y) * ihx + (fy.y - 2 * uc.y) * ihy + (fz.y - 2 * uc.y) * ihz;
        out = cadd(out, cmul(kc, uc));
        if (ORDER == 4) {
            // mixed fourth differences da2 db2 U
            C exy = cadd(cadd(u[1][0][0], u[1][0][2]), cadd(u[1][2][0], u[1][2][2]));
            C exz = cadd(cadd(u[0][1][0], u[0][1][2]), cadd(u[2][1][0], u[2][1][2]));
            C eyz = cadd(cadd(u[0][0][1], u[0][2][1]), cadd(u[2][0][1], u[2][2][1]));
            const R wxy = (p.hx * p.hx + p.hy * p.hy) / R(12) * ihx * ihy;
            const R wxz = (p.hx * p.hx + p.hz * p.hz) / R(12) * ihx * ihz;
            const R wyz = (p.hy * p.hy + p.hz * p.hz) / R(12) * ihy * ihz;
            C t;
            t.x = exy.x - 2 * (fx.x + fy.x) + 4 * uc.x; t.y = exy.y - 2 * (fx.y + fy.y) + 4 * uc.y;
            out = cadd(out, cscale(t, wxy));
            t.x = exz.x - 2 * (fx.x + fz.x) + 4 * uc.x; t.y = exz.y - 2 * (fx.y + fz.y) + 4 * uc.y;
            out = cadd(out, cscale(t, wxz));
            t.x = eyz.x - 2 * (fy.x + fz.x) + 4 * uc.x; t.y = eyz.y - 2 * (fy.y + fz.y) + 4 * uc.y;
            out = cadd(out, cscale(t, wyz));
            // (hd^2/12) dd2 (k^2 U) = (1/12)(kU+ - 2 kU0 + kU-)
            C kuc = cmul(kc, uc);
            C s = cadd(cadd(cmul(k[1][1][0], u[1][1][0]), cmul(k[1][1][2], u[1][1][2])),
                       cadd(cmul(k[1][0][1], u[1][0][1]), cmul(k[1][2][1], u[1][2][1])));
            s = cadd(s, cadd(cmul(k[0][1][1], u[0][1][1]), cmul(k[2][1][1], u[2][1][1])));
            t.x = (s.x - 6 * kuc.x) / R(12); t.y = (s.y - 6 * kuc.y) / R(12);
            out = cadd(out, t);
        }
        return out;
    } else {
        const R h = p.hx, h2 = h * h, ih2 = R(1) / h2;
        const R c30 = h2 / R(30), c15 = h2 / R(15), c6 = h2 / R(6);
        // P_c = (1 + c k^2) U at the needed points
        auto P = [&](int c, int b, int a, R cc) -> C { return cadd(u[c][b][a], cscale(cmul(k[c][b][a], u[c][b][a]), cc)); };
        // faces
        C f30 = czero<C>(), f15 = czero<C>(), fu = czero<C>();
        const int FA[6][3] = {{1, 1, 0}, {1, 1, 2}, {1, 0, 1}, {1, 2, 1}, {0, 1, 1}, {2, 1, 1}};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int c = FA[q][0], b = FA[q][1], a = FA[q][2];
            f30 = cadd(f30, P(c, b, a, c30));
            f15 = cadd(f15, P(c, b, a, c15));
            fu = cadd(fu, u[c][b][a]);
        }
        C e15 = czero<C>(), eu = czero<C>();
        const int ED[12][3] = {{1, 0, 0}, {1, 0, 2}, {1, 2, 0}, {1, 2, 2}, {0, 1, 0}, {0, 1, 2},
                               {2, 1, 0}, {2, 1, 2}, {0, 0, 1}, {0, 2, 1}, {2, 0, 1}, {2, 2, 1}};
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const int c = ED[q][0], b = ED[q][1], a = ED[q][2];
            e15 = cadd(e15, P(c, b, a, c15));
            eu = cadd(eu, u[c][b][a]);
        }
        C cu = czero<C>();
#pragma unroll
        for (int c = 0; c < 3; c += 2)
#pragma unroll
            for (int b = 0; b < 3; b += 2)
#pragma unroll
                for (int a = 0; a < 3; a += 2) cu = cadd(cu, u[c][b][a]);
        const C p30c = P(1, 1, 1, c30), p15c = P(1, 1, 1, c15);
        C out;
        // L[(1 + h^2 k^2/30)U]
        out.x = (f30.x - 6 * p30c.x) * ih2; out.y = (f30.y - 6 * p30c.y) * ih2;
        // h^4/30 dxx dyy dzz U
        out.x += (cu.x - 2 * eu.x + 4 * fu.x - 8 * uc.x) * (ih2 / R(30));
        out.y += (cu.y - 2 * eu.y + 4 * fu.y - 8 * uc.y) * (ih2 / R(30));
        // k^2 U
        out = cadd(out, cmul(kc, uc));
        // h^2/6 M[(1 + h^2 k^2/15)U]
        out.x += (e15.x - 4 * f15.x + 12 * p15c.x) * (ih2 / R(6));
        out.y += (e15.y - 4 * f15.y + 12 * p15c.y) * (ih2 / R(6));
        // h^2/20 { G U + 2 sum_d g_d inner_d }
        const C G = p.G[gidx];
        C acc = cmul(G, uc);
        const R i2h = R(1) / (R(2) * h), i12h = R(1) / (R(12) * h);
        // S_a = sum of the four transverse neighbours of the side point a minus 4 * that point
        // x direction: side points (1,1,0) and (1,1,2)
        {
            C sp = csub(cadd(cadd(u[1][0][2], u[1][2][2]), cadd(u[0][1][2], u[2][1][2])), cscale(u[1][1][2], R(4)));
            C sm = csub(cadd(cadd(u[1][0][0], u[1][2][0]), cadd(u[0][1][0], u[2][1][0])), cscale(u[1][1][0], R(4)));
            C in = cadd(cscale(csub(P(1, 1, 2, c6), P(1, 1, 0, c6)), i2h), cscale(csub(sp, sm), i12h));
            acc = cadd(acc, cscale(cmul(p.dk2[0][gidx], in), R(2)));
        }
        {   // y direction: side points (1,2,1) and (1,0,1)
            C sp = csub(cadd(cadd(u[1][2][0], u[1][2][2]), cadd(u[0][2][1], u[2][2][1])), cscale(u[1][2][1], R(4)));
            C sm = csub(cadd(cadd(u[1][0][0], u[1][0][2]), cadd(u[0][0][1], u[2][0][1])), cscale(u[1][0][1], R(4)));
            C in = cadd(cscale(csub(P(1, 2, 1, c6), P(1, 0, 1, c6)), i2h), cscale(csub(sp, sm), i12h));
            acc = cadd(acc, cscale(cmul(p.dk2[1][gidx], in), R(2)));
        }
        {   // z direction: side points (2,1,1) and (0,1,1)
            C sp = csub(cadd(cadd(u[2][1][0], u[2][1][2]), cadd(u[2][0][1], u[2][2][1])), cscale(u[2][1][1], R(4)));
            C sm = csub(cadd(cadd(u[0][1][0], u[0][1][2]), cadd(u[0][0][1], u[0][2][1])), cscale(u[0][1][1], R(4)));
            C in = cadd(cscale(csub(P(2, 1, 1, c6), P(0, 1, 1, c6)), i2h), cscale(csub(sp, sm), i12h));
            acc = cadd(acc, cscale(cmul(p.dk2[2][gidx], in), R(2)));
        }
        out = cadd(out, cscale(acc, h2 / R(20)));
        return out;
    }
}

// MODE 0: y = scale * A x.  MODE 1: r = F - A x written as complex64, with per-CTA partial sums of
// |r|^2 and max |r| (FP64) in part[2*cta], part[2*cta+1].
template <typename R, int ORDER, int MODE>
__global__ void __launch_bounds__(TX * TY)
stencil_kernel(StencilParams<R> p, const typename cplx<R>::t* __restrict__ U, typename cplx<R>::t* __restrict__ Y,
               const double* __restrict__ sigma, int sidx, const double2* __restrict__ F, float2* __restrict__ rout,
               double* __restrict__ part) {
    typedef typename cplx<R>::t C;
    __shared__ C sU[2][PY][PX];
    __shared__ C sK[2][PY][PX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZCH;
    const int z1 = min(z0 + ZCH, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < p.nx && gy < p.ny;
    C u[3][3][3], k[3][3][3];
    double ssum = 0.0, smax = 0.0;

    auto stage = [&](int buf, int Z) {
        for (int q = tid; q < PX * PY; q += TX * TY) {
            const int ly = q / PX, lx = q - ly * PX;
            sU[buf][ly][lx] = fetch_u<R>(p, U, x0 + lx - 1, y0 + ly - 1, Z);
            sK[buf][ly][lx] = fetch_k<R>(p, x0 + lx - 1, y0 + ly - 1, Z);
        }
    };
    auto lift = [&](int buf, int slot) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                u[slot][b][a] = sU[buf][ty + b][tx + a];
                k[slot][b][a] = sK[buf][ty + b][tx + a];
            }
    };
    int buf = 0;
    stage(buf, z0 - 1); __syncthreads(); lift(buf, 0); buf ^= 1;
    stage(buf, z0);     __syncthreads(); lift(buf, 1); buf ^= 1;
    for (int z = z0; z < z1; ++z) {
        stage(buf, z + 1);
        __syncthreads();
        lift(buf, 2);
        buf ^= 1;
        if (active) {
            const size_t gidx = ((size_t)z * p.ny + gy) * p.nx + gx;
            C v = apply_point<R, ORDER>(p, u, k, gidx);
            if (MODE == 0) {
                if (sigma) v = cscale(v, (R)sigma[sidx]);
                Y[gidx] = v;
            } else {
                const double2 f = F[gidx];
                const double rx = f.x - (double)v.x, ry = f.y - (double)v.y;
                rout[gidx] = make_float2((float)rx, (float)ry);
                const double a2 = rx * rx + ry * ry;
                ssum += a2;
                smax = fmax(smax, a2);
            }
        }
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                u[0][b][a] = u[1][b][a]; u[1][b][a] = u[2][b][a];
                k[0][b][a] = k[1][b][a]; k[1][b][a] = k[2][b][a];
            }
    }
    if (MODE == 1) {
        __shared__ double rs[TX * TY / 32], rm[TX * TY / 32];
        for (int o = 16; o > 0; o >>= 1) {
            ssum += __shfl_down_sync(0xffffffffu, ssum, o);
            smax = fmax(smax, __shfl_down_sync(0xffffffffu, smax, o));
        }
        if ((tid & 31) == 0) { rs[tid >> 5] = ssum; rm[tid >> 5] = smax; }
        __syncthreads();
        if (tid == 0) {
            double s = 0, m = 0;
            for (int w = 0; w < TX * TY / 32; ++w) { s += rs[w]; m = fmax(m, rm[w]); }
            const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            part[2 * cta] = s;
            part[2 * cta + 1] = sqrt(m);
        }
    }
}

template <typename R>
StencilParams<R> make_params(const helm_ctx* c, int f64) {
    StencilParams<R> p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.hx = (R)c->h[0]; p.hy = (R)c->h[1]; p.hz = (R)c->h[2];
    p.gx = mk((R)c->gam[0].x, (R)c->gam[0].y);
    p.gy = mk((R)c->gam[1].x, (R)c->gam[1].y);
    p.gz = mk((R)c->gam[2].x, (R)c->gam[2].y);
    for (int d = 0; d < 3; ++d) p.dk2[d] = nullptr;
    p.G = nullptr;
    return p;
}

dim3 stencil_grid(const helm_ctx* c) {
    return dim3((c->nx + TX - 1) / TX, (c->ny + TY - 1) / TY, (c->nz + ZCH - 1) / ZCH);
}

// ---- coefficient fields of Eq. scheme6 (set-up, FP64) ----------------------------------------
__device__ inline int mirror_stag(int i, int n) { return i < 0 ? -i - 1 : (i >= n ? 2 * n - 1 - i : i); }

__global__ void derived_kernel(int nx, int ny, int nz, double hx, double hy, double hz, const double2* __restrict__ k2,
                               double2* dkx, double2* dky, double2* dkz, double2* G, float2* fdkx, float2* fdky,
                               float2* fdkz, float2* fG, float2* fk2) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(id % nx), j = (int)((id / nx) % ny), l = (int)(id / ((size_t)nx * ny));
        auto at = [&](int a, int b, int c) {
            return k2[((size_t)mirror_stag(l + c, nz) * ny + mirror_stag(j + b, ny)) * nx + mirror_stag(i + a, nx)];
        };
        double2 g[3];
        double2 lap = make_double2(0, 0);
        const double hh[3] = {hx, hy, hz};
        for (int d = 0; d < 3; ++d) {
            int o[3] = {0, 0, 0};
            double2 v[5];
            for (int s = -2; s <= 2; ++s) { o[d] = s; v[s + 2] = at(o[0], o[1], o[2]); }
            g[d].x = (-v[4].x + 8 * v[3].x - 8 * v[1].x + v[0].x) / (12 * hh[d]);
            g[d].y = (-v[4].y + 8 * v[3].y - 8 * v[1].y + v[0].y) / (12 * hh[d]);
            lap.x += (-v[4].x + 16 * v[3].x - 30 * v[2].x + 16 * v[1].x - v[0].x) / (12 * hh[d] * hh[d]);
            lap.y += (-v[4].y + 16 * v[3].y - 30 * v[2].y + 16 * v[1].y - v[0].y) / (12 * hh[d] * hh[d]);
        }
        const double2 kc = k2[id];
        const double2 gg = csub(lap, cmul(kc, kc));
        dkx[id] = g[0]; dky[id] = g[1]; dkz[id] = g[2]; G[id] = gg;
        fdkx[id] = make_float2((float)g[0].x, (float)g[0].y);
        fdky[id] = make_float2((float)g[1].x, (float)g[1].y);
        fdkz[id] = make_float2((float)g[2].x, (float)g[2].y);
        fG[id] = make_float2((float)gg.x, (float)gg.y);
        fk2[id] = make_float2((float)kc.x, (float)kc.y);
    }
}

__global__ void to_f32_kernel(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        b[id] = make_float2((float)a[id].x, (float)a[id].y);
}

// ---- modified right-hand side (set-up, FP64) -------------------------------------------------
__global__ void rhs_kernel(int order, int nx, int ny, int nz, double hx, double hy, double hz,
                           const double2* __restrict__ f, const double2* __restrict__ k2,
                           const double2* __restrict__ dkx, const double2* __restrict__ dky,
                           const double2* __restrict__ dkz, double2* __restrict__ F) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(id % nx), j = (int)((id / nx) % ny), l = (int)(id / ((size_t)nx * ny));
        auto at = [&](int a, int b, int c) {
            return f[((size_t)mirror_stag(l + c, nz) * ny + mirror_stag(j + b, ny)) * nx + mirror_stag(i + a, nx)];
        };
        const double2 fc = f[id];
        if (order == 2) { F[id] = fc; continue; }
        const double hh[3] = {hx, hy, hz};
        if (order == 4) {
            double2 out = fc;
            for (int d = 0; d < 3; ++d) {
                int o[3] = {0, 0, 0};
                o[d] = 1; double2 p = at(o[0], o[1], o[2]);
                o[d] = -1; double2 m = at(o[0], o[1], o[2]);
                out.x += (p.x - 2 * fc.x + m.x) / 12.0;
                out.y += (p.y - 2 * fc.y + m.y) / 12.0;
            }
            F[id] = out;
            continue;
        }
        // order 6 (uniform h)
        const double h = hx, h2 = h * h;
        double2 lap = make_double2(0, 0), s4 = make_double2(0, 0), fd[3];
        for (int d = 0; d < 3; ++d) {
            int o[3] = {0, 0, 0};
            double2 v[5];
            for (int s = -2; s <= 2; ++s) { o[d] = s; v[s + 2] = at(o[0], o[1], o[2]); }
            lap.x += (-v[4].x + 16 * v[3].x - 30 * v[2].x + 16 * v[1].x - v[0].x) / (12 * hh[d] * hh[d]);
            lap.y += (-v[4].y + 16 * v[3].y - 30 * v[2].y + 16 * v[1].y - v[0].y) / (12 * hh[d] * hh[d]);
            const double h4 = hh[d] * hh[d] * hh[d] * hh[d];
            s4.x += (v[4].x - 4 * v[3].x + 6 * v[2].x - 4 * v[1].x + v[0].x) / h4;
            s4.y += (v[4].y - 4 * v[3].y + 6 * v[2].y - 4 * v[1].y + v[0].y) / h4;
            fd[d].x = (v[3].x - v[1].x) / (2 * hh[d]);
            fd[d].y = (v[3].y - v[1].y) / (2 * hh[d]);
        }
        double2 mix = make_double2(0, 0);
        const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        const double w[3] = {1.0, -2.0, 1.0};
        for (int q = 0; q < 3; ++q) {
            double2 acc = make_double2(0, 0);
            for (int s1 = -1; s1 <= 1; ++s1)
                for (int s2 = -1; s2 <= 1; ++s2) {
                    int o[3] = {0, 0, 0};
                    o[pairs[q][0]] = s1; o[pairs[q][1]] = s2;
                    const double2 v = at(o[0], o[1], o[2]);
                    acc.x += w[s1 + 1] * w[s2 + 1] * v.x;
                    acc.y += w[s1 + 1] * w[s2 + 1] * v.y;
                }
            const double den = hh[pairs[q][0]] * hh[pairs[q][0]] * hh[pairs[q][1]] * hh[pairs[q][1]];
            mix.x += acc.x / den; mix.y += acc.y / den;
        }
        double2 out;
        out.x = fc.x + h2 / 12.0 * lap.x + h2 * h2 / 360.0 * s4.x + h2 * h2 / 90.0 * mix.x;
        out.y = fc.y + h2 / 12.0 * lap.y + h2 * h2 / 360.0 * s4.y + h2 * h2 / 90.0 * mix.y;
        const double2 kc = k2[id];
        double2 kf = cmul(kc, fc);
        double2 gf = cadd(cadd(cmul(dkx[id], fd[0]), cmul(dky[id], fd[1])), cmul(dkz[id], fd[2]));
        out.x -= h2 / 20.0 * (kf.x - h2 / 3.0 * gf.x);
        out.y -= h2 / 20.0 * (kf.y - h2 / 3.0 * gf.y);
        F[id] = out;
    }
}

}  // namespace

helm_status launch_derived_fields(helm_ctx* c, cudaStream_t s) {
    const int blocks = 1024;
    if (c->opt.order == 6) {
        derived_kernel<<<blocks, 256, 0, s>>>(c->nx, c->ny, c->nz, c->h[0], c->h[1], c->h[2], c->k2_d, c->dk2_d[0],
                                              c->dk2_d[1], c->dk2_d[2], c->G_d, c->dk2_f[0], c->dk2_f[1], c->dk2_f[2],
                                              c->G_f, c->k2_f);
    } else {
        to_f32_kernel<<<blocks, 256, 0, s>>>(c->k2_d, c->k2_f, c->npts);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

template <typename R, int MODE>
static void launch_stencil(helm_ctx* c, StencilParams<R> p, const typename cplx<R>::t* x, typename cplx<R>::t* y,
                           const double* sigma, int sidx, const double2* F, float2* r, double* part, cudaStream_t s) {
    dim3 grid = stencil_grid(c), block(TX, TY);
    switch (c->opt.order) {
        case 2: stencil_kernel<R, 2, MODE><<<grid, block, 0, s>>>(p, x, y, sigma, sidx, F, r, part); break;
        case 4: stencil_kernel<R, 4, MODE><<<grid, block, 0, s>>>(p, x, y, sigma, sidx, F, r, part); break;
        default: stencil_kernel<R, 6, MODE><<<grid, block, 0, s>>>(p, x, y, sigma, sidx, F, r, part); break;
    }
}

helm_status launch_stencil_f32(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, cudaStream_t s) {
    StencilParams<float> p = make_params<float>(c, 0);
    p.k2 = c->k2_f;
    for (int d = 0; d < 3; ++d) p.dk2[d] = c->dk2_f[d];
    p.G = c->G_f;
    prof_begin(c, s, PROF_STENCIL);
    launch_stencil<float, 0>(c, p, x, y, sigma, sidx, nullptr, nullptr, nullptr, s);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status launch_stencil_f64(helm_ctx* c, const double2* x, double2* y, cudaStream_t s) {
    StencilParams<double> p = make_params<double>(c, 1);
    p.k2 = c->k2_d;
    for (int d = 0; d < 3; ++d) p.dk2[d] = c->dk2_d[d];
    p.G = c->G_d;
    prof_begin(c, s, PROF_OTHER);
    launch_stencil<double, 0>(c, p, x, y, nullptr, 0, nullptr, nullptr, nullptr, s);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// Number of CTAs of the residual launch (one partial pair per CTA).
int residual_ctas(const helm_ctx* c) {
    dim3 g = stencil_grid(c);
    return (int)(g.x * g.y * g.z);
}

helm_status launch_residual(helm_ctx* c, const double2* x, const double2* F, float2* r, double* part, int nblk,
                            cudaStream_t s) {
    (void)nblk;
    StencilParams<double> p = make_params<double>(c, 1);
    p.k2 = c->k2_d;
    for (int d = 0; d < 3; ++d) p.dk2[d] = c->dk2_d[d];
    p.G = c->G_d;
    prof_begin(c, s, PROF_RESIDUAL);
    launch_stencil<double, 1>(c, p, x, (double2*)nullptr, nullptr, 0, F, r, part, s);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status launch_rhs(helm_ctx* c, const double2* f, double2* F, cudaStream_t s) {
    rhs_kernel<<<1024, 256, 0, s>>>(c->opt.order, c->nx, c->ny, c->nz, c->h[0], c->h[1], c->h[2], f, c->k2_d,
                                    c->dk2_d[0], c->dk2_d[1], c->dk2_d[2], F);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
