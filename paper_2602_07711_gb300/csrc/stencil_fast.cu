// Complex64 stencil matvec w = A z of the Krylov iteration (Eqs. scheme4 and scheme6 with the ghosts of
// Eq. D_bc eliminated), restructured for throughput.
//
// The operator at a point couples three z-planes.  Each plane enters through a few plane quantities of
// the 3 x 3 patch around the point's column: for the sixth-order scheme, with c the centre, fx, fy the
// in-plane face pairs, e the in-plane corners and KU = k^2 U,
//   as the z-neighbour plane (lo or hi):
//     A_s = (1/h^2)[(7/15) c + (1/10)(fx + fy) + (1/30) e] + (1/90)(KU faces - KU centre)
//     D_x += (1/6)(U_{x+} - U_{x-}),  D_y likewise,  D_z += +-[c + (h^2/6) KU_c + (1/6)(fx + fy - 4c)]
//   as the point's own plane (mid):
//     A_m = (1/h^2)[(7/15)(fx + fy) + (1/10) e - (64/15) c] + (14/15) KU_c + (1/90)(KU corners - KU faces)
//           + (h^2/20) G c
//     D_x += (U_{x+} - U_{x-}) + (h^2/6)(KU_{x+} - KU_{x-}) + (1/6)(T_{x+} - T_{x-})|_mid,   D_y likewise
//   A z = A_s(lo) + A_m + A_s(hi) + (h/20) sum_d g_d D_d            (g_d = (k^2)_d, G = lap k^2 - k^4),
// which is the collected form of Eq. scheme6 (the fourth-order scheme splits the same way without D).
// A thread therefore keeps two pending sums (the outputs of planes P and P+1) instead of three planes of
// its patch, and every plane is read from shared memory once.
//
// Data movement: a CTA owns a 32 x 8 column tile and marches through a z-chunk.  Planes of U and k^2
// with a one-point halo, and the per-point fields G, g_x, g_y, g_z, stream into a four-slot shared
// memory ring by cp.async, two planes ahead of the arithmetic; one barrier per plane.  Halo points
// outside the grid are loaded from the clamped position and multiplied by the ghost factors gamma_d
// (products at edges and corners) when lifted; k^2 there is the mirror (clamped) value.
#include "common.cuh"

namespace {

constexpr int FTX = 32, FTY = 8;
constexpr int FPX = FTX + 2, FPY = FTY + 2;
constexpr int FHALO = FPX * FPY;   // 340
constexpr int FNT = FTX * FTY;     // 256 threads
constexpr int FNS = 4;             // ring slots
constexpr int FZCH = 32;           // planes per CTA

template <int ORDER>
struct FStage {
    float2 u[FHALO];
    float2 k[FHALO];
    float2 f[ORDER == 6 ? 4 : 1][ORDER == 6 ? FNT : 2];   // G, g_x, g_y, g_z at the tile's points
};

struct FParams {
    int nx, ny, nz;
    float2 gx, gy, gz;
    float ihx, ihy, ihz;          // 1/h_d^2
    float wxy, wxz, wyz;          // order 4 mixed weights
    float h2_20, h_20, hh6;       // order 6: h^2/20, h/20, h^2/6
    const float2* k2;
    const float2* fld[4];         // G, g_x, g_y, g_z (order 6)
};

__device__ __forceinline__ void cp8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2scl(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 f2fma(float s, float2 a, float2 b) {   // s a + b
    return make_float2(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y));
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <int ORDER>
__global__ void __launch_bounds__(FNT, 4)
stencil_fast_kernel(FParams p, const float2* __restrict__ U, float2* __restrict__ Y, const double* __restrict__ sigma,
                    int sidx) {
    extern __shared__ __align__(16) unsigned char fsm[];
    FStage<ORDER>* ring = reinterpret_cast<FStage<ORDER>*>(fsm);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < p.nx && gy < p.ny;
    const bool xyedge = gx == 0 || gx == p.nx - 1 || gy == 0 || gy == p.ny - 1;
    const float sg = sigma ? (float)sigma[sidx] : 1.f;

    // stage plane P (ghost planes P = -1, nz come from the clamped plane) into its ring slot
    auto issue = [&](int P) {
        if (P <= z1) {
            FStage<ORDER>& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const size_t pbase = (size_t)Pc * p.ny;
            for (int q = tid; q < FHALO; q += FNT) {
                const int ly = q / FPX, lx = q - ly * FPX;
                const int X = min(max(x0 + lx - 1, 0), p.nx - 1);
                const int Yc = min(max(y0 + ly - 1, 0), p.ny - 1);
                const size_t g = (pbase + Yc) * p.nx + X;
                cp8(&S.u[q], U + g);
                cp8(&S.k[q], p.k2 + g);
            }
            if (ORDER == 6 && P >= z0 && P < z1 && active) {
                const size_t g = (pbase + gy) * p.nx + gx;
#pragma unroll
                for (int f = 0; f < 4; ++f) cp8(&S.f[f][tid], p.fld[f] + g);
            }
        }
        cp_commit();   // one group per plane, empty ones included, so that wait_group counts planes
    };

    // pending sums of the outputs at planes P (cur) and P+1 (nxt): A, D_x, D_y, D_z
    float2 cA = make_float2(0, 0), cX = cA, cY = cA, cZ = cA;
    float2 nA = cA, nX = cA, nY = cA, nZ = cA;

    issue(z0 - 1);
    issue(z0);
    for (int P = z0 - 1; P <= z1; ++P) {
        cp_wait1();          // plane P has landed (only plane P+1 may still be in flight)
        __syncthreads();     // ... for every thread; and every thread is done with plane P-2's slot
        issue(P + 2);
        const FStage<ORDER>& S = ring[(P + FNS) % FNS];
        // the 3x3 patch of U (ghost factors applied) and the sums of KU = k^2 U the scheme needs
        const bool zghost = P < 0 || P >= p.nz;
        const bool fix = xyedge || zghost;
        const float2 one = make_float2(1.f, 0.f);
        const float2 fz = zghost ? p.gz : one;
        const float2 fxm = gx == 0 ? p.gx : one, fxp = gx == p.nx - 1 ? p.gx : one;
        const float2 fym = gy == 0 ? p.gy : one, fyp = gy == p.ny - 1 ? p.gy : one;
        float2 u[3][3];
        float2 kc = make_float2(0, 0), kf4 = kc, kcs = kc, dkx = kc, dky = kc;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float2 v = S.u[(ty + b) * FPX + tx + a];
                if (fix) {
                    float2 f = fz;
                    if (a == 0) f = f2mul(f, fxm);
                    if (a == 2) f = f2mul(f, fxp);
                    if (b == 0) f = f2mul(f, fym);
                    if (b == 2) f = f2mul(f, fyp);
                    v = f2mul(v, f);
                }
                u[b][a] = v;
                if (ORDER == 6 || a == 1 || b == 1) {
                    const float2 kv = f2mul(S.k[(ty + b) * FPX + tx + a], v);
                    if (a == 1 && b == 1) kc = kv;
                    else if (a == 1 || b == 1) kf4 = f2add(kf4, kv);
                    else kcs = f2add(kcs, kv);
                    if (b == 1 && a == 0) dkx = f2sub(dkx, kv);
                    if (b == 1 && a == 2) dkx = f2add(dkx, kv);
                    if (a == 1 && b == 0) dky = f2sub(dky, kv);
                    if (a == 1 && b == 2) dky = f2add(dky, kv);
                }
            }
        const float2 c = u[1][1];
        const float2 fx = f2add(u[1][0], u[1][2]), fy = f2add(u[0][1], u[2][1]);
        const float2 e = f2add(f2add(u[0][0], u[0][2]), f2add(u[2][0], u[2][2]));
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;   // finish the output at plane P-1
        const bool do_mid = P >= z0 && P < z1;             // the output at plane P
        if (ORDER == 6) {
            const float ih = p.ihx;
            // as a z-neighbour plane
            float2 As = f2scl(f2fma(1.f / 30.f, e, f2fma(0.1f, f2add(fx, fy), f2scl(c, 7.f / 15.f))), ih);
            As = f2fma(1.f / 90.f, f2sub(kf4, kc), As);
            const float2 dx1 = f2sub(u[1][2], u[1][0]), dy1 = f2sub(u[2][1], u[0][1]);
            const float2 Xs = f2scl(dx1, 1.f / 6.f), Ys = f2scl(dy1, 1.f / 6.f);
            const float2 Zs = f2add(f2fma(p.hh6, kc, c), f2scl(f2fma(-4.f, c, f2add(fx, fy)), 1.f / 6.f));
            if (out_prev) {
                const FStage<ORDER>& Sp = ring[(P - 1 + FNS) % FNS];
                const float2 A = f2add(cA, As);
                float2 g = f2mul(Sp.f[1][tid], f2add(cX, Xs));
                g = f2add(g, f2mul(Sp.f[2][tid], f2add(cY, Ys)));
                g = f2add(g, f2mul(Sp.f[3][tid], f2add(cZ, Zs)));
                const float2 v = f2fma(p.h_20, g, A);
                if (active) Y[((size_t)(P - 1) * p.ny + gy) * p.nx + gx] = f2scl(v, sg);
            }
            // the output at plane P: lo part (already in nxt) + this plane as mid
            cA = nA; cX = nX; cY = nY; cZ = nZ;
            if (do_mid) {
                float2 Am = f2scl(f2fma(-64.f / 15.f, c, f2fma(0.1f, e, f2scl(f2add(fx, fy), 7.f / 15.f))), ih);
                Am = f2fma(14.f / 15.f, kc, Am);
                Am = f2fma(1.f / 90.f, f2sub(kcs, kf4), Am);
                Am = f2fma(p.h2_20, f2mul(S.f[0][tid], c), Am);
                const float2 tdx = f2sub(f2add(u[0][2], u[2][2]), f2add(u[0][0], u[2][0]));
                const float2 tdy = f2sub(f2add(u[2][0], u[2][2]), f2add(u[0][0], u[0][2]));
                const float2 Xm = f2add(f2fma(p.hh6, dkx, dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                const float2 Ym = f2add(f2fma(p.hh6, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                cA = f2add(cA, Am); cX = f2add(cX, Xm); cY = f2add(cY, Ym);
            }
            // this plane as the lo neighbour of the output at plane P+1
            nA = As; nX = Xs; nY = Ys; nZ = make_float2(-Zs.x, -Zs.y);
        } else {
            const float2 As = f2fma(1.f / 12.f, kc,
                                    f2add(f2scl(c, p.ihz),
                                          f2add(f2scl(f2fma(-2.f, c, fx), p.wxz), f2scl(f2fma(-2.f, c, fy), p.wyz))));
            if (out_prev && active)
                Y[((size_t)(P - 1) * p.ny + gy) * p.nx + gx] = f2scl(f2add(cA, As), sg);
            cA = nA;
            if (do_mid) {
                const float2 c2 = f2add(c, c), c4 = f2add(c2, c2);
                float2 Am = f2add(f2scl(f2sub(fx, c2), p.ihx), f2scl(f2sub(fy, c2), p.ihy));
                Am = f2fma(-2.f * p.ihz, c, Am);
                Am = f2fma(p.wxy, f2add(f2fma(-2.f, f2add(fx, fy), e), c4), Am);
                Am = f2fma(p.wxz, f2fma(-2.f, fx, c4), Am);
                Am = f2fma(p.wyz, f2fma(-2.f, fy, c4), Am);
                Am = f2fma(0.5f, kc, Am);
                Am = f2fma(1.f / 12.f, kf4, Am);
                cA = f2add(cA, Am);
            }
            nA = As;
        }
    }
}

template <int ORDER>
size_t fast_smem() { return FNS * sizeof(FStage<ORDER>); }

}  // namespace

// Set the shared-memory limit of the kernels once per device (set-up time, not inside a capture).
helm_status stencil_fast_prepare() {
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<4>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<6>()));
    return HELM_OK;
}

bool stencil_fast_supported(const helm_ctx* c) { return c->opt.order == 4 || c->opt.order == 6; }

helm_status launch_stencil_fast(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, cudaStream_t s) {
    FParams p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.gx = make_float2((float)c->gam[0].x, (float)c->gam[0].y);
    p.gy = make_float2((float)c->gam[1].x, (float)c->gam[1].y);
    p.gz = make_float2((float)c->gam[2].x, (float)c->gam[2].y);
    const double hx = c->h[0], hy = c->h[1], hz = c->h[2];
    const double ihx = 1.0 / (hx * hx), ihy = 1.0 / (hy * hy), ihz = 1.0 / (hz * hz);
    p.ihx = (float)ihx; p.ihy = (float)ihy; p.ihz = (float)ihz;
    p.wxy = (float)((hx * hx + hy * hy) / 12.0 * ihx * ihy);
    p.wxz = (float)((hx * hx + hz * hz) / 12.0 * ihx * ihz);
    p.wyz = (float)((hy * hy + hz * hz) / 12.0 * ihy * ihz);
    p.h2_20 = (float)(hx * hx / 20.0);
    p.h_20 = (float)(hx / 20.0);
    p.hh6 = (float)(hx * hx / 6.0);
    p.k2 = c->k2_f;
    p.fld[0] = c->G_f;
    for (int d = 0; d < 3; ++d) p.fld[d + 1] = c->dk2_f[d];
    dim3 grid((c->nx + FTX - 1) / FTX, (c->ny + FTY - 1) / FTY, (c->nz + FZCH - 1) / FZCH), block(FTX, FTY);
    if (c->opt.order == 6)
        stencil_fast_kernel<6><<<grid, block, fast_smem<6>(), s>>>(p, x, y, sigma, sidx);
    else
        stencil_fast_kernel<4><<<grid, block, fast_smem<4>(), s>>>(p, x, y, sigma, sidx);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
