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
// memory ring two planes ahead of the arithmetic, one barrier per plane:
//   TMA kernel (even N_x): one thread issues cp.async.bulk.tensor tile loads per plane (a 36 x 10 tile of
//     U and of k^2 starting two points left of the tile so that the 16-byte rule holds, four 32 x 8 field
//     tiles), completion counted by one mbarrier per slot with bounded waits.  A prepare pass turns the
//     landed k^2 into KU = k^2 U in place; out-of-grid halo points (TMA fills them with zeros) are then
//     written as gamma-multiples of their interior neighbours, U and KU alike (KU is linear in U and k^2
//     at a ghost is the mirror value), and the ghost planes z = -1, N_z come from the clamped plane times
//     gamma_z.
//   cp.async kernel: 8-byte cp.async of the clamped halo points (each thread stages the same points of
//     every plane, so their offsets and ghost factors are computed once); a prepare pass per plane
//     applies the ghost factors and forms KU = k^2 U once per staged point.
#include "common.cuh"
#include "packed.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>

namespace {

constexpr int FTX = 32, FTY = 8;
constexpr int FPX = FTX + 2, FPY = FTY + 2;
constexpr int FHALO = FPX * FPY;   // 340
constexpr int FNT = FTX * FTY;     // 256 threads
constexpr int FNS = 4;             // ring slots
constexpr int FZCH = 32;           // planes per CTA

template <int ORDER, bool RK = false>
struct FStage {
    float2 u[FHALO];
    float2 k[FHALO];
    float2 f[ORDER == 6 ? 4 : 1][ORDER == 6 ? FNT : 2];   // G, g_x, g_y, g_z at the tile's points
};
// real k^2 (no attenuation): k^2 staged as float, KU formed from it; the four order-6 fields are real and
// interleaved (G, g_x, g_y, g_z) in one float4 per point
template <int ORDER>
struct FStage<ORDER, true> {
    float2 u[FHALO];
    float2 k[FHALO];   // KU
    float kr[FHALO];
    float4 f4[ORDER == 6 ? FNT : 1];
};

struct FParams {
    int nx, ny, nz;
    float2 gx, gy, gz;
    float ihx, ihy, ihz;          // 1/h_d^2
    float wxy, wxz, wyz;          // order 4 mixed weights
    float h2_20, h_20, hh6;       // order 6: h^2/20, h/20, h^2/6
    const float2* k2;
    const float2* fld[4];         // G, g_x, g_y, g_z (order 6)
    const float* k2r;             // real k^2 (real-medium kernels)
    const float4* fr;             // real (G, g_x, g_y, g_z) per point (real-medium kernels, order 6)
    int nb = 1;                   // vectors in one launch (the right-hand sides of a batch group), npts apart;
                                  // blockIdx.z = z chunk * nb + vector
    float i12h[3], i12h2[3];      // 1/(12 h_d), 1/(12 h_d^2): the in-kernel sixth-order fields
};

__device__ __forceinline__ void cp8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp16f(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// complex64 helpers on packed pairs (one f32x2 instruction per operation, two for the product)
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 f2scl(float2 a, float s) { return mul2(a, bc2(s)); }
__device__ __forceinline__ float2 f2fma(float s, float2 a, float2 b) { return fma2(bc2(s), a, b); }   // s a + b
// a b = a.x (b.x, b.y) + (-a.y, a.y) (b.y, b.x)
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    return fma2(make_float2(-a.y, a.y), swap2(b), mul2(bc2(a.x), b));
}

template <int ORDER, int MINB, bool RK = false>
__global__ void __launch_bounds__(FNT, MINB)
stencil_fast_kernel(FParams p, const float2* __restrict__ U, float2* __restrict__ Y, const double* __restrict__ sigma,
                    int sidx) {
    extern __shared__ __align__(16) unsigned char fsm[];
    using Stage = FStage<ORDER, RK>;
    Stage* ring = reinterpret_cast<Stage*>(fsm);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int vb = blockIdx.z % p.nb;   // the vector of the batch this CTA works on
    const int z0 = (blockIdx.z / p.nb) * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < p.nx && gy < p.ny;
    const float sg = sigma ? (float)sigma[sidx] : 1.f;
    if (vb) {
        const size_t off = (size_t)vb * p.nx * p.ny * p.nz;
        U += off;
        Y += off;
    }
    // this thread's staging slots (fixed across planes): clamped in-plane offset in the low 30 bits,
    // bit 30 = x ghost, bit 31 = y ghost
    unsigned sl[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int q = tid + k * FNT;
        if (q < FHALO) {
            const int ly = q / FPX, lx = q - ly * FPX;
            const int Xg = x0 + lx - 1, Yg = y0 + ly - 1;
            const int Xc = min(max(Xg, 0), p.nx - 1), Yc = min(max(Yg, 0), p.ny - 1);
            sl[k] = (unsigned)(Yc * p.nx + Xc) | (Xc != Xg ? 1u << 30 : 0u) | (Yc != Yg ? 1u << 31 : 0u);
        }
    }
    const size_t plane = (size_t)p.nx * p.ny;
    const int poff = gy * p.nx + gx;

    auto issue = [&](int P) {
        if (P <= z1) {
            Stage& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const float2* Ub = U + (size_t)Pc * plane;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (tid + k * FNT < FHALO) {
                    cp8(&S.u[tid + k * FNT], Ub + (sl[k] & 0x3FFFFFFFu));
                    if constexpr (RK) cp4(&S.kr[tid + k * FNT], p.k2r + (size_t)Pc * plane + (sl[k] & 0x3FFFFFFFu));
                    else cp8(&S.k[tid + k * FNT], p.k2 + (size_t)Pc * plane + (sl[k] & 0x3FFFFFFFu));
                }
            if (ORDER == 6 && P >= z0 && P < z1 && active) {
                const size_t g = (size_t)P * plane + poff;
                if constexpr (RK) {
                    cp16f(&S.f4[tid], p.fr + g);
                } else {
#pragma unroll
                    for (int f = 0; f < 4; ++f) cp8(&S.f[f][tid], p.fld[f] + g);
                }
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
        Stage& S = ring[(P + FNS) % FNS];
        cp_wait1();          // plane P has landed (only plane P+1 may still be in flight)
        __syncthreads();     // ... for every thread; and every thread is done with plane P-1
        // prepare this thread's staged points: ghost factors, then KU = k^2 U once per point
        const bool zghost = P < 0 || P >= p.nz;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q = tid + k * FNT;
            if (q < FHALO) {
                float2 u = S.u[q];
                if ((sl[k] >> 30) || zghost) {
                    if (sl[k] & (1u << 30)) u = f2mul(u, p.gx);
                    if (sl[k] & (1u << 31)) u = f2mul(u, p.gy);
                    if (zghost) u = f2mul(u, p.gz);
                    S.u[q] = u;
                }
                if constexpr (RK) S.k[q] = f2scl(u, S.kr[q]);
                else S.k[q] = f2mul(S.k[q], u);
            }
        }
        __syncthreads();     // U and KU of plane P ready for every thread
        issue(P + 2);        // into the slot of plane P-2, which nobody reads any more
        float2 u[3][3];
        float2 kc = make_float2(0, 0), kf4 = kc, kcs = kc, dkx = kc, dky = kc;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = (ty + b) * FPX + tx + a;
                u[b][a] = S.u[i];
                if (ORDER == 6 || a == 1 || b == 1) {
                    const float2 kv = S.k[i];
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
                const Stage& Sp = ring[(P - 1 + FNS) % FNS];
                const float2 A = f2add(cA, As);
                float2 g;
                if constexpr (RK) {
                    const float4 fv = Sp.f4[tid];
                    g = f2scl(f2add(cX, Xs), fv.y);
                    g = f2fma(fv.z, f2add(cY, Ys), g);
                    g = f2fma(fv.w, f2add(cZ, Zs), g);
                } else {
                    g = f2mul(Sp.f[1][tid], f2add(cX, Xs));
                    g = f2add(g, f2mul(Sp.f[2][tid], f2add(cY, Ys)));
                    g = f2add(g, f2mul(Sp.f[3][tid], f2add(cZ, Zs)));
                }
                const float2 v = f2fma(p.h_20, g, A);
                if (active) Y[(size_t)(P - 1) * plane + poff] = f2scl(v, sg);
            }
            // the output at plane P: lo part (already in nxt) + this plane as mid
            cA = nA; cX = nX; cY = nY; cZ = nZ;
            if (do_mid) {
                float2 Am = f2scl(f2fma(-64.f / 15.f, c, f2fma(0.1f, e, f2scl(f2add(fx, fy), 7.f / 15.f))), ih);
                Am = f2fma(14.f / 15.f, kc, Am);
                Am = f2fma(1.f / 90.f, f2sub(kcs, kf4), Am);
                if constexpr (RK) Am = f2fma(p.h2_20 * S.f4[tid].x, c, Am);
                else Am = f2fma(p.h2_20, f2mul(S.f[0][tid], c), Am);
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
            if (out_prev && active) Y[(size_t)(P - 1) * plane + poff] = f2scl(f2add(cA, As), sg);
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

// Two rows per thread (real media): the kernel above is bound by shared-memory traffic (each point reads a
// 3 x 3 patch of U and of KU per plane, and KU is written once per staged point).  Here a thread computes
// the points (x, 2 t) and (x, 2 t + 1) of the same 32 x 8 tile from one 4 x 3 patch of U and of the real
// k^2 (a third fewer reads per point) and forms k^2 U itself, so no KU plane is written; the ghost factors
// are applied in shared memory only by tiles that touch the boundary (and on the ghost planes), so interior
// tiles take one barrier per plane.  128 threads per CTA, each staging three halo points.
template <int ORDER>
struct F2Stage {
    float2 u[FHALO];
    float kr[FHALO];
    float4 f4[ORDER == 6 ? FNT : 1];   // G, g_x, g_y, g_z at the tile's points
};
constexpr int F2T = FNT / 2;
template <int ORDER>
size_t fast2_smem() { return FNS * sizeof(F2Stage<ORDER>); }

template <int ORDER, int MINB>
__global__ void __launch_bounds__(F2T, MINB)
stencil_fast2_kernel(FParams p, const float2* __restrict__ U, float2* __restrict__ Y, const double* __restrict__ sigma,
                     int sidx) {
    extern __shared__ __align__(16) unsigned char fsm[];
    using Stage = F2Stage<ORDER>;
    Stage* ring = reinterpret_cast<Stage*>(fsm);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;   // ty = 0 .. 3
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int vb = blockIdx.z % p.nb;
    const int z0 = (blockIdx.z / p.nb) * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy0 = y0 + 2 * ty;
    const bool act[2] = {gx < p.nx && gy0 < p.ny, gx < p.nx && gy0 + 1 < p.ny};
    // the tile's halo reaches a ghost point in x or y (its interior points never need a ghost factor)
    const bool edge = x0 == 0 || y0 == 0 || x0 + FTX >= p.nx || y0 + FTY >= p.ny;
    const float sg = sigma ? (float)sigma[sidx] : 1.f;
    if (vb) {
        const size_t off = (size_t)vb * p.nx * p.ny * p.nz;
        U += off;
        Y += off;
    }
    unsigned sl[3] = {0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = tid + k * F2T;
        if (q < FHALO) {
            const int ly = q / FPX, lx = q - ly * FPX;
            const int Xg = x0 + lx - 1, Yg = y0 + ly - 1;
            const int Xc = min(max(Xg, 0), p.nx - 1), Yc = min(max(Yg, 0), p.ny - 1);
            sl[k] = (unsigned)(Yc * p.nx + Xc) | (Xc != Xg ? 1u << 30 : 0u) | (Yc != Yg ? 1u << 31 : 0u);
        }
    }
    const size_t plane = (size_t)p.nx * p.ny;
    const int poff = gy0 * p.nx + gx;
    const int fi = (2 * ty) * FTX + tx;   // the fields of point r at f4[fi + r FTX]

    auto issue = [&](int P) {
        if (P <= z1) {
            Stage& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const float2* Ub = U + (size_t)Pc * plane;
            const float* Kb = p.k2r + (size_t)Pc * plane;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (tid + k * F2T < FHALO) {
                    cp8(&S.u[tid + k * F2T], Ub + (sl[k] & 0x3FFFFFFFu));
                    cp4(&S.kr[tid + k * F2T], Kb + (sl[k] & 0x3FFFFFFFu));
                }
            if (ORDER == 6 && P >= z0 && P < z1) {
                const size_t g = (size_t)P * plane + poff;
                if (act[0]) cp16f(&S.f4[fi], p.fr + g);
                if (act[1]) cp16f(&S.f4[fi + FTX], p.fr + g + p.nx);
            }
        }
        cp_commit();
    };

    float2 cA[2], cX[2], cY[2], cZ[2], nA[2], nX[2], nY[2], nZ[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        cA[r] = cX[r] = cY[r] = cZ[r] = make_float2(0, 0);
        nA[r] = nX[r] = nY[r] = nZ[r] = make_float2(0, 0);
    }
    issue(z0 - 1);
    issue(z0);
    for (int P = z0 - 1; P <= z1; ++P) {
        Stage& S = ring[(P + FNS) % FNS];
        cp_wait1();
        __syncthreads();          // plane P landed for everyone; everyone is done with planes P-1 and P-2
        const bool zghost = P < 0 || P >= p.nz;
        if (edge || zghost) {     // uniform per CTA and plane
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int q = tid + k * F2T;
                if (q < FHALO && ((sl[k] >> 30) || zghost)) {
                    float2 u = S.u[q];
                    if (sl[k] & (1u << 30)) u = f2mul(u, p.gx);
                    if (sl[k] & (1u << 31)) u = f2mul(u, p.gy);
                    if (zghost) u = f2mul(u, p.gz);
                    S.u[q] = u;
                }
            }
            __syncthreads();
        }
        issue(P + 2);             // into the slot of plane P-2
        float2 u[4][3], kv[4][3];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = (2 * ty + b) * FPX + tx + a;
                u[b][a] = S.u[i];
                kv[b][a] = f2scl(u[b][a], S.kr[i]);   // KU = k^2 U (k^2 at a ghost point is the mirror value)
            }
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;
        const bool do_mid = P >= z0 && P < z1;
        const Stage& Sp = ring[(P - 1 + FNS) % FNS];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float2 c = u[r + 1][1];
            const float2 fx = f2add(u[r + 1][0], u[r + 1][2]), fy = f2add(u[r][1], u[r + 2][1]);
            const float2 e = f2add(f2add(u[r][0], u[r][2]), f2add(u[r + 2][0], u[r + 2][2]));
            const float2 kc = kv[r + 1][1];
            const float2 kf4 = f2add(f2add(kv[r + 1][0], kv[r + 1][2]), f2add(kv[r][1], kv[r + 2][1]));
            if (ORDER == 6) {
                const float2 kcs = f2add(f2add(kv[r][0], kv[r][2]), f2add(kv[r + 2][0], kv[r + 2][2]));
                const float2 dkx = f2sub(kv[r + 1][2], kv[r + 1][0]), dky = f2sub(kv[r + 2][1], kv[r][1]);
                const float ih = p.ihx;
                float2 As = f2scl(f2fma(1.f / 30.f, e, f2fma(0.1f, f2add(fx, fy), f2scl(c, 7.f / 15.f))), ih);
                As = f2fma(1.f / 90.f, f2sub(kf4, kc), As);
                const float2 dx1 = f2sub(u[r + 1][2], u[r + 1][0]), dy1 = f2sub(u[r + 2][1], u[r][1]);
                const float2 Xs = f2scl(dx1, 1.f / 6.f), Ys = f2scl(dy1, 1.f / 6.f);
                const float2 Zs = f2add(f2fma(p.hh6, kc, c), f2scl(f2fma(-4.f, c, f2add(fx, fy)), 1.f / 6.f));
                if (out_prev) {
                    const float2 A = f2add(cA[r], As);
                    const float4 fv = Sp.f4[fi + r * FTX];
                    float2 g = f2scl(f2add(cX[r], Xs), fv.y);
                    g = f2fma(fv.z, f2add(cY[r], Ys), g);
                    g = f2fma(fv.w, f2add(cZ[r], Zs), g);
                    const float2 v = f2fma(p.h_20, g, A);
                    if (act[r]) Y[(size_t)(P - 1) * plane + poff + r * p.nx] = f2scl(v, sg);
                }
                cA[r] = nA[r]; cX[r] = nX[r]; cY[r] = nY[r]; cZ[r] = nZ[r];
                if (do_mid) {
                    float2 Am = f2scl(f2fma(-64.f / 15.f, c, f2fma(0.1f, e, f2scl(f2add(fx, fy), 7.f / 15.f))), ih);
                    Am = f2fma(14.f / 15.f, kc, Am);
                    Am = f2fma(1.f / 90.f, f2sub(kcs, kf4), Am);
                    Am = f2fma(p.h2_20 * S.f4[fi + r * FTX].x, c, Am);
                    const float2 tdx = f2sub(f2add(u[r][2], u[r + 2][2]), f2add(u[r][0], u[r + 2][0]));
                    const float2 tdy = f2sub(f2add(u[r + 2][0], u[r + 2][2]), f2add(u[r][0], u[r][2]));
                    const float2 Xm = f2add(f2fma(p.hh6, dkx, dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                    const float2 Ym = f2add(f2fma(p.hh6, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                    cA[r] = f2add(cA[r], Am); cX[r] = f2add(cX[r], Xm); cY[r] = f2add(cY[r], Ym);
                }
                nA[r] = As; nX[r] = Xs; nY[r] = Ys; nZ[r] = make_float2(-Zs.x, -Zs.y);
            } else {
                const float2 As = f2fma(1.f / 12.f, kc,
                                        f2add(f2scl(c, p.ihz),
                                              f2add(f2scl(f2fma(-2.f, c, fx), p.wxz), f2scl(f2fma(-2.f, c, fy), p.wyz))));
                if (out_prev && act[r]) Y[(size_t)(P - 1) * plane + poff + r * p.nx] = f2scl(f2add(cA[r], As), sg);
                cA[r] = nA[r];
                if (do_mid) {
                    const float2 c2 = f2add(c, c), c4 = f2add(c2, c2);
                    float2 Am = f2add(f2scl(f2sub(fx, c2), p.ihx), f2scl(f2sub(fy, c2), p.ihy));
                    Am = f2fma(-2.f * p.ihz, c, Am);
                    Am = f2fma(p.wxy, f2add(f2fma(-2.f, f2add(fx, fy), e), c4), Am);
                    Am = f2fma(p.wxz, f2fma(-2.f, fx, c4), Am);
                    Am = f2fma(p.wyz, f2fma(-2.f, fy, c4), Am);
                    Am = f2fma(0.5f, kc, Am);
                    Am = f2fma(1.f / 12.f, kf4, Am);
                    cA[r] = f2add(cA[r], Am);
                }
                nA[r] = As;
            }
        }
    }
}

// Sixth order, real medium, fields formed in the kernel: the four order-6 fields g_d = d(k^2)/dx_d and
// G = lap(k^2) - k^4 (fourth-order five-point differences, the staggered mirror extension at the faces,
// exactly the definitions of the set-up's derived_kernel, here in FP32) are computed from a second ring of
// k^2 planes with a two-point halo, so the kernel streams U, k^2 and w only: 20 instead of 36 bytes per
// point.  Otherwise the two-row form above.  The k^2 ring holds the planes P-3 .. P+4 (eight slots; a plane
// is fetched four iterations ahead and read for the last time two iterations later); at iteration P the
// fields of plane P are formed (G is used at once, g one iteration later, in registers).
constexpr int K2X = FTX + 4, K2Y = FTY + 4, K2PTS = K2X * K2Y;   // 36 x 12
constexpr int K2NS = 8;
struct F3Stage {
    float2 u[FHALO];
};
constexpr size_t F3_SMEM = FNS * sizeof(F3Stage) + K2NS * K2PTS * sizeof(float);

template <int MINB>
__global__ void __launch_bounds__(F2T, MINB)
stencil_fast3_kernel(FParams p, const float2* __restrict__ U, float2* __restrict__ Y, const double* __restrict__ sigma,
                     int sidx) {
    extern __shared__ __align__(16) unsigned char fsm[];
    F3Stage* ring = reinterpret_cast<F3Stage*>(fsm);
    float* kring = reinterpret_cast<float*>(fsm + FNS * sizeof(F3Stage));   // [K2NS][K2PTS]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;   // ty = 0 .. 3
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int vb = blockIdx.z % p.nb;
    const int z0 = (blockIdx.z / p.nb) * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy0 = y0 + 2 * ty;
    const bool act[2] = {gx < p.nx && gy0 < p.ny, gx < p.nx && gy0 + 1 < p.ny};
    const bool edge = x0 == 0 || y0 == 0 || x0 + FTX >= p.nx || y0 + FTY >= p.ny;
    const float sg = sigma ? (float)sigma[sidx] : 1.f;
    if (vb) {
        const size_t off = (size_t)vb * p.nx * p.ny * p.nz;
        U += off;
        Y += off;
    }
    // U staging slots (one-point halo, clamped, ghost flags) and k^2 staging slots (two-point halo, the
    // staggered mirror: -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2; points beyond are never read)
    unsigned sl[3] = {0u, 0u, 0u};
    int kl[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = tid + k * F2T;
        if (q < FHALO) {
            const int ly = q / FPX, lx = q - ly * FPX;
            const int Xg = x0 + lx - 1, Yg = y0 + ly - 1;
            const int Xc = min(max(Xg, 0), p.nx - 1), Yc = min(max(Yg, 0), p.ny - 1);
            sl[k] = (unsigned)(Yc * p.nx + Xc) | (Xc != Xg ? 1u << 30 : 0u) | (Yc != Yg ? 1u << 31 : 0u);
        }
    }
    auto mir = [](int i, int n) { i = min(i, n + 1); return i < 0 ? -i - 1 : (i >= n ? 2 * n - 1 - i : i); };
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = tid + k * F2T;
        if (q < K2PTS) {
            const int ly = q / K2X, lx = q - ly * K2X;
            kl[k] = mir(y0 + ly - 2, p.ny) * p.nx + mir(x0 + lx - 2, p.nx);
        }
    }
    const size_t plane = (size_t)p.nx * p.ny;
    const int poff = gy0 * p.nx + gx;

    auto issue = [&](int P, int Pk) {   // U plane P (if in the window) and k^2 plane Pk (if in the window)
        if (P <= z1) {
            F3Stage& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const float2* Ub = U + (size_t)Pc * plane;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (tid + k * F2T < FHALO) cp8(&S.u[tid + k * F2T], Ub + (sl[k] & 0x3FFFFFFFu));
        }
        if (Pk >= z0 - 2 && Pk <= z1 + 1) {
            float* K = kring + ((Pk + 2 * K2NS) % K2NS) * K2PTS;
            const float* Kb = p.k2r + (size_t)mir(Pk, p.nz) * plane;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (tid + k * F2T < K2PTS) cp4(&K[tid + k * F2T], Kb + kl[k]);
        }
        cp_commit();
    };
    auto kp = [&](int P) -> const float* { return kring + ((P + 2 * K2NS) % K2NS) * K2PTS; };

    float2 cA[2], cX[2], cY[2], cZ[2], nA[2], nX[2], nY[2], nZ[2];
    float gpx[2], gpy[2], gpz[2];   // the gradient fields of the previous plane
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        cA[r] = cX[r] = cY[r] = cZ[r] = make_float2(0, 0);
        nA[r] = nX[r] = nY[r] = nZ[r] = make_float2(0, 0);
        gpx[r] = gpy[r] = gpz[r] = 0.f;
    }
    // first group: U(z0-1) and k^2 planes z0-2 .. z0+1; second: U(z0), k^2(z0+2); iteration P: U(P+2), k^2(P+4)
    {
        if (z0 - 1 <= z1) {
            F3Stage& S = ring[(z0 - 1 + FNS) % FNS];
            const int Pc = min(max(z0 - 1, 0), p.nz - 1);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (tid + k * F2T < FHALO) cp8(&S.u[tid + k * F2T], U + (size_t)Pc * plane + (sl[k] & 0x3FFFFFFFu));
        }
        for (int Pk = z0 - 2; Pk <= z0 + 1; ++Pk) {
            if (Pk > z1 + 1) break;
            float* K = kring + ((Pk + 2 * K2NS) % K2NS) * K2PTS;
            const float* Kb = p.k2r + (size_t)mir(Pk, p.nz) * plane;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (tid + k * F2T < K2PTS) cp4(&K[tid + k * F2T], Kb + kl[k]);
        }
        cp_commit();
    }
    issue(z0, z0 + 2);
    const int c0 = (2 * ty + 2) * K2X + tx + 2;   // the k^2 tile index of this thread's first point
    for (int P = z0 - 1; P <= z1; ++P) {
        F3Stage& S = ring[(P + FNS) % FNS];
        cp_wait1();
        __syncthreads();          // U(P) and k^2 up to P+2 landed for everyone; planes P-2 (U), P-4 (k^2) free
        const bool zghost = P < 0 || P >= p.nz;
        if (edge || zghost) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int q = tid + k * F2T;
                if (q < FHALO && ((sl[k] >> 30) || zghost)) {
                    float2 u = S.u[q];
                    if (sl[k] & (1u << 30)) u = f2mul(u, p.gx);
                    if (sl[k] & (1u << 31)) u = f2mul(u, p.gy);
                    if (zghost) u = f2mul(u, p.gz);
                    S.u[q] = u;
                }
            }
            __syncthreads();
        }
        issue(P + 2, P + 4);
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;
        const bool do_mid = P >= z0 && P < z1;
        // k^2 of plane P at the patch (clamped plane: a ghost plane takes its mirror plane's values)
        const float* K0 = kp(min(max(P, z0 - 2), z1 + 1));
        float2 u[4][3];
        float kk[4][3];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                u[b][a] = S.u[(2 * ty + b) * FPX + tx + a];
                kk[b][a] = K0[(2 * ty + b + 1) * K2X + tx + a + 1];
            }
        const float* Km1 = kp(P - 1);
        const float* Kp1 = kp(P + 1);
        const float* Km2 = kp(P - 2);
        const float* Kp2 = kp(P + 2);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // the fields of plane P at point r (patch row r + 1 is the point's row; the +-1 neighbours in x
            // and y and one +-2 neighbour in y are patch values)
            float Gf = 0.f, gfx = 0.f, gfy = 0.f, gfz = 0.f;
            if (do_mid) {
                const int c = c0 + r * K2X;
                const float kc0 = kk[r + 1][1];
                const float xm1 = kk[r + 1][0], xp1 = kk[r + 1][2], ym1 = kk[r][1], yp1 = kk[r + 2][1];
                const float xm2 = K0[c - 2], xp2 = K0[c + 2];
                const float ym2 = r == 1 ? kk[0][1] : K0[c - 2 * K2X];
                const float yp2 = r == 0 ? kk[3][1] : K0[c + 2 * K2X];
                const float zm1 = Km1[c], zp1 = Kp1[c], zm2 = Km2[c], zp2 = Kp2[c];
                gfx = (8.f * (xp1 - xm1) - (xp2 - xm2)) * p.i12h[0];
                gfy = (8.f * (yp1 - ym1) - (yp2 - ym2)) * p.i12h[1];
                gfz = (8.f * (zp1 - zm1) - (zp2 - zm2)) * p.i12h[2];
                const float lap = (16.f * (xp1 + xm1) - (xp2 + xm2) - 30.f * kc0) * p.i12h2[0] +
                                  (16.f * (yp1 + ym1) - (yp2 + ym2) - 30.f * kc0) * p.i12h2[1] +
                                  (16.f * (zp1 + zm1) - (zp2 + zm2) - 30.f * kc0) * p.i12h2[2];
                Gf = fmaf(-kc0, kc0, lap);
            }
            const float2 c = u[r + 1][1];
            const float2 fx = f2add(u[r + 1][0], u[r + 1][2]), fy = f2add(u[r][1], u[r + 2][1]);
            const float2 e = f2add(f2add(u[r][0], u[r][2]), f2add(u[r + 2][0], u[r + 2][2]));
            // KU = k^2 U at the 3 x 3 patch of point r, formed where it is needed
            const float2 kxm = f2scl(u[r + 1][0], kk[r + 1][0]), kxp = f2scl(u[r + 1][2], kk[r + 1][2]);
            const float2 kym = f2scl(u[r][1], kk[r][1]), kyp = f2scl(u[r + 2][1], kk[r + 2][1]);
            const float2 kc = f2scl(c, kk[r + 1][1]);
            const float2 kf4 = f2add(f2add(kxm, kxp), f2add(kym, kyp));
            const float2 kcs = f2fma(kk[r][0], u[r][0], f2fma(kk[r][2], u[r][2], f2fma(kk[r + 2][0], u[r + 2][0],
                                                                                 f2scl(u[r + 2][2], kk[r + 2][2]))));
            const float2 dkx = f2sub(kxp, kxm), dky = f2sub(kyp, kym);
            const float ih = p.ihx;
            float2 As = f2scl(f2fma(1.f / 30.f, e, f2fma(0.1f, f2add(fx, fy), f2scl(c, 7.f / 15.f))), ih);
            As = f2fma(1.f / 90.f, f2sub(kf4, kc), As);
            const float2 dx1 = f2sub(u[r + 1][2], u[r + 1][0]), dy1 = f2sub(u[r + 2][1], u[r][1]);
            const float2 Xs = f2scl(dx1, 1.f / 6.f), Ys = f2scl(dy1, 1.f / 6.f);
            const float2 Zs = f2add(f2fma(p.hh6, kc, c), f2scl(f2fma(-4.f, c, f2add(fx, fy)), 1.f / 6.f));
            if (out_prev) {
                const float2 A = f2add(cA[r], As);
                float2 g = f2scl(f2add(cX[r], Xs), gpx[r]);
                g = f2fma(gpy[r], f2add(cY[r], Ys), g);
                g = f2fma(gpz[r], f2add(cZ[r], Zs), g);
                const float2 v = f2fma(p.h_20, g, A);
                if (act[r]) Y[(size_t)(P - 1) * plane + poff + r * p.nx] = f2scl(v, sg);
            }
            cA[r] = nA[r]; cX[r] = nX[r]; cY[r] = nY[r]; cZ[r] = nZ[r];
            if (do_mid) {
                float2 Am = f2scl(f2fma(-64.f / 15.f, c, f2fma(0.1f, e, f2scl(f2add(fx, fy), 7.f / 15.f))), ih);
                Am = f2fma(14.f / 15.f, kc, Am);
                Am = f2fma(1.f / 90.f, f2sub(kcs, kf4), Am);
                Am = f2fma(p.h2_20 * Gf, c, Am);
                const float2 tdx = f2sub(f2add(u[r][2], u[r + 2][2]), f2add(u[r][0], u[r + 2][0]));
                const float2 tdy = f2sub(f2add(u[r + 2][0], u[r + 2][2]), f2add(u[r][0], u[r][2]));
                const float2 Xm = f2add(f2fma(p.hh6, dkx, dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                const float2 Ym = f2add(f2fma(p.hh6, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                cA[r] = f2add(cA[r], Am); cX[r] = f2add(cX[r], Xm); cY[r] = f2add(cY[r], Ym);
            }
            nA[r] = As; nX[r] = Xs; nY[r] = Ys; nZ[r] = make_float2(-Zs.x, -Zs.y);
            gpx[r] = gfx; gpy[r] = gfy; gpz[r] = gfz;
        }
    }
}

template <int ORDER, bool RK = false>
size_t fast_smem() { return FNS * sizeof(FStage<ORDER, RK>); }

// ---- TMA kernel --------------------------------------------------------------------------------
constexpr int TPX = 36;                          // tile row of the TMA halo: x0-2 .. x0+33
constexpr int TU_BYTES = TPX * FPY * 8;          // 2880
constexpr int TU_PAD = 2944;                     // 128-byte multiple
constexpr int TF_BYTES = FNT * 8;                // 2048 per field
template <int ORDER>
struct TLayout {
    static constexpr int U_OFF = 0, K_OFF = TU_PAD, F_OFF = 2 * TU_PAD;
    static constexpr int STAGE = 2 * TU_PAD + (ORDER == 6 ? 4 * TF_BYTES : 0);
    static constexpr int BAR_OFF = FNS * STAGE;
    static constexpr int SMEM = BAR_OFF + FNS * 8 + 128;   // + alignment slack
};
constexpr long TDRAIN_LIMIT = 1L << 22;   // bound of the drain waits after an expired wait

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool tbar_wait(uint32_t bar, uint32_t parity, long limit) {
    for (long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tload3(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

template <int ORDER>
__global__ void __launch_bounds__(FNT, 4)
stencil_tma_kernel(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mK,
                   const __grid_constant__ CUtensorMap mG, const __grid_constant__ CUtensorMap mGx,
                   const __grid_constant__ CUtensorMap mGy, const __grid_constant__ CUtensorMap mGz, FParams p,
                   float2* __restrict__ Y, const double* __restrict__ sigma, int sidx, unsigned* status, long wlim) {
    typedef TLayout<ORDER> L;
    extern __shared__ unsigned char traw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)traw + 127) & ~(uintptr_t)127);
    const uint32_t sbase = s32(base);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < p.nx && gy < p.ny;
    const bool edge = x0 == 0 || p.nx <= x0 + FTX || y0 == 0 || p.ny <= y0 + FTY;   // the halo leaves the grid
    const float sg = sigma ? (float)sigma[sidx] : 1.f;
    if (tid == 0) {
        for (int sl = 0; sl < FNS; ++sl) tbar_init(sbase + L::BAR_OFF + 8 * sl);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // thread 0: stage plane P (relative index r = P - z0 + 1) into slot r % 4
    auto issue = [&](int P) {
        const int r = P - z0 + 1, sl = r & (FNS - 1);
        const uint32_t st = sbase + sl * L::STAGE, bar = sbase + L::BAR_OFF + 8 * sl;
        const int Pc = min(max(P, 0), p.nz - 1);
        const bool fields = ORDER == 6 && P >= z0 && P < z1;
        tbar_expect(bar, 2 * TU_BYTES + (fields ? 4 * TF_BYTES : 0));
        tload3(st + L::U_OFF, &mU, bar, 2 * (x0 - 2), y0 - 1, Pc);
        tload3(st + L::K_OFF, &mK, bar, 2 * (x0 - 2), y0 - 1, Pc);
        if (fields) {
            tload3(st + L::F_OFF, &mG, bar, 2 * x0, y0, P);
            tload3(st + L::F_OFF + TF_BYTES, &mGx, bar, 2 * x0, y0, P);
            tload3(st + L::F_OFF + 2 * TF_BYTES, &mGy, bar, 2 * x0, y0, P);
            tload3(st + L::F_OFF + 3 * TF_BYTES, &mGz, bar, 2 * x0, y0, P);
        }
    };
    bool failed = false;
    int r_fail = 0, r_last = 1;   // thread 0: relative index of its first unconfirmed plane, of its last issued one
    if (tid == 0) { issue(z0 - 1); issue(z0); }

    float2 cA = make_float2(0, 0), cX = cA, cY = cA, cZ = cA;
    float2 nA = cA, nX = cA, nY = cA, nZ = cA;
    for (int P = z0 - 1; P <= z1; ++P) {
        const int r = P - z0 + 1, sl = r & (FNS - 1);
        if (!failed && !tbar_wait(sbase + L::BAR_OFF + 8 * sl, (r >> 2) & 1, wlim)) {
            failed = true;
            r_fail = r;
            if (tid == 0) atomicOr(status, HELM_DEV_WAIT);
        }
        float2* sU = reinterpret_cast<float2*>(base + sl * L::STAGE + L::U_OFF);
        float2* sK = reinterpret_cast<float2*>(base + sl * L::STAGE + L::K_OFF);
        // prepare: KU = k^2 U in place; ghost planes are gamma_z times the clamped plane
        const bool zghost = P < 0 || P >= p.nz;
        for (int q = tid; q < FHALO; q += FNT) {
            const int ly = q / FPX, lx = q - ly * FPX + 1;
            const int i = ly * TPX + lx;
            float2 u = sU[i];
            if (zghost) { u = f2mul(u, p.gz); sU[i] = u; }
            sK[i] = f2mul(sK[i], u);
        }
        if (edge) {
            __syncthreads();
            // out-of-grid halo points next to the grid: gamma multiples of the interior neighbour
            for (int q = tid; q < FHALO; q += FNT) {
                const int ly = q / FPX, lx = q - ly * FPX + 1;
                const int X = x0 + lx - 2, Yy = y0 + ly - 1;
                const bool xo = X == -1 || X == p.nx, yo = Yy == -1 || Yy == p.ny;
                if ((xo || yo) && X >= -1 && X <= p.nx && Yy >= -1 && Yy <= p.ny) {
                    const int sx = lx + (X == -1 ? 1 : (X == p.nx ? -1 : 0));
                    const int sy = ly + (Yy == -1 ? 1 : (Yy == p.ny ? -1 : 0));
                    float2 f = make_float2(1.f, 0.f);
                    if (xo) f = p.gx;
                    if (yo) f = f2mul(f, p.gy);
                    sU[ly * TPX + lx] = f2mul(f, sU[sy * TPX + sx]);
                    sK[ly * TPX + lx] = f2mul(f, sK[sy * TPX + sx]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes before later TMA writes
        __syncthreads();   // slot P prepared; every thread is done with plane P-1 (and the slot of P-2)
        if (tid == 0 && P + 2 <= z1 && !failed) {
            issue(P + 2);
            r_last = P + 2 - z0 + 1;
        }
        float2 u[3][3];
        float2 kc, kf4 = make_float2(0, 0), kcs = kf4, dkx = kf4, dky = kf4;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = (ty + b) * TPX + tx + 1 + a;
                u[b][a] = sU[i];
                if (ORDER == 6 || a == 1 || b == 1) {
                    const float2 kv = sK[i];
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
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;
        const bool do_mid = P >= z0 && P < z1;
        if (ORDER == 6) {
            const float2* F = reinterpret_cast<const float2*>(base + sl * L::STAGE + L::F_OFF);
            const float2* Fp = reinterpret_cast<const float2*>(base + ((r - 1) & (FNS - 1)) * L::STAGE + L::F_OFF);
            const float ih = p.ihx;
            float2 As = f2scl(f2fma(1.f / 30.f, e, f2fma(0.1f, f2add(fx, fy), f2scl(c, 7.f / 15.f))), ih);
            As = f2fma(1.f / 90.f, f2sub(kf4, kc), As);
            const float2 dx1 = f2sub(u[1][2], u[1][0]), dy1 = f2sub(u[2][1], u[0][1]);
            const float2 Xs = f2scl(dx1, 1.f / 6.f), Ys = f2scl(dy1, 1.f / 6.f);
            const float2 Zs = f2add(f2fma(p.hh6, kc, c), f2scl(f2fma(-4.f, c, f2add(fx, fy)), 1.f / 6.f));
            if (out_prev) {
                const float2 A = f2add(cA, As);
                float2 g = f2mul(Fp[FNT + tid], f2add(cX, Xs));
                g = f2add(g, f2mul(Fp[2 * FNT + tid], f2add(cY, Ys)));
                g = f2add(g, f2mul(Fp[3 * FNT + tid], f2add(cZ, Zs)));
                const float2 v = f2fma(p.h_20, g, A);
                if (active) Y[((size_t)(P - 1) * p.ny + gy) * p.nx + gx] = f2scl(v, sg);
            }
            cA = nA; cX = nX; cY = nY; cZ = nZ;
            if (do_mid) {
                float2 Am = f2scl(f2fma(-64.f / 15.f, c, f2fma(0.1f, e, f2scl(f2add(fx, fy), 7.f / 15.f))), ih);
                Am = f2fma(14.f / 15.f, kc, Am);
                Am = f2fma(1.f / 90.f, f2sub(kcs, kf4), Am);
                Am = f2fma(p.h2_20, f2mul(F[tid], c), Am);
                const float2 tdx = f2sub(f2add(u[0][2], u[2][2]), f2add(u[0][0], u[2][0]));
                const float2 tdy = f2sub(f2add(u[2][0], u[2][2]), f2add(u[0][0], u[0][2]));
                const float2 Xm = f2add(f2fma(p.hh6, dkx, dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                const float2 Ym = f2add(f2fma(p.hh6, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                cA = f2add(cA, Am); cX = f2add(cX, Xm); cY = f2add(cY, Ym);
            }
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
    if (failed && tid == 0) {
        // thread 0 stopped at plane r_fail: the planes it issued from there on may still be in flight; let
        // them land before the CTA's shared memory goes away (at most four planes, one per slot, so every
        // barrier phase is unambiguous; bounded).  A thread other than 0 that gave up leaves thread 0
        // waiting for every plane it issued, as in a normal run.
        for (int r = r_fail; r <= r_last; ++r)
            tbar_wait(sbase + L::BAR_OFF + 8 * (r & (FNS - 1)), (r >> 2) & 1, TDRAIN_LIMIT);
    }
}

struct FastMaps {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    CUtensorMap mK, mF[4];
};

helm_status encode3(FastMaps* m, CUtensorMap* map, const void* ptr, int nx, int ny, int nz, int boxw, int boxh) {
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * nx * sizeof(float), (cuuint64_t)2 * nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)boxw, (cuuint32_t)boxh, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = m->encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HELM_OK : HELM_ERR_CUDA;
}

}  // namespace

// Set-up (not inside a capture): the kernels' shared-memory limits and, for even N_x, the TMA descriptors
// of the fixed operands (k^2 and the sixth-order fields).
helm_status stencil_fast_prepare(helm_ctx* c) {
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<4>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<6, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<6>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<4, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<4>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<6, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<6>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<4, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<4, true>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<6, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<6, true>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<4, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<4, true>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast_kernel<6, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast_smem<6, true>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast2_kernel<6, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast2_smem<6>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast2_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fast2_smem<4>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_fast3_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)F3_SMEM));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_tma_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TLayout<4>::SMEM));
    HELM_CUDA_TRY(cudaFuncSetAttribute(stencil_tma_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TLayout<6>::SMEM));
    if (residual_fast_prepare() != HELM_OK) return HELM_ERR_CUDA;
    // measured default: the sixth-order kernel needs about 80 registers (three CTAs per SM, no spills)
    c->tune_stencil = c->opt.order == 6 ? 2 : 0;
    if (c->nx % 2 != 0 || !stencil_fast_supported(c)) return HELM_OK;
    FastMaps* m = new FastMaps();
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&m->encode, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !m->encode) {
        cudaGetLastError();
        delete m;
        return HELM_OK;   // no TMA descriptors: the cp.async kernel serves
    }
    helm_status st = encode3(m, &m->mK, c->k2_f, c->nx, c->ny, c->nz, 2 * TPX, FPY);
    if (st == HELM_OK && c->opt.order == 6) {
        const float2* f[4] = {c->G_f, c->dk2_f[0], c->dk2_f[1], c->dk2_f[2]};
        for (int i = 0; i < 4 && st == HELM_OK; ++i) st = encode3(m, &m->mF[i], f[i], c->nx, c->ny, c->nz, 2 * FTX, FTY);
    } else if (st == HELM_OK) {
        for (int i = 0; i < 4; ++i) m->mF[i] = m->mK;   // unused by the fourth-order kernel
    }
    if (st != HELM_OK) { delete m; return HELM_OK; }
    c->sfast = m;
    return HELM_OK;
}

void stencil_fast_release(helm_ctx* c) {
    delete (FastMaps*)c->sfast;
    c->sfast = nullptr;
    cudaFree(c->k2r);
    cudaFree(c->fr);
    c->k2r = nullptr;
    c->fr = nullptr;
    c->realk = 0;
    residual_real_release(c);
}

namespace {
__global__ void imag_any_kernel(const double2* __restrict__ k2, size_t n, unsigned* flag) {
    unsigned any = 0;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        any |= k2[id].y != 0.0;
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}
__global__ void real_fields_kernel(size_t n, int order, const float2* __restrict__ k2f, const float2* __restrict__ G,
                                   const float2* __restrict__ gx, const float2* __restrict__ gy,
                                   const float2* __restrict__ gz, float* __restrict__ kr, float4* __restrict__ fr) {
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        kr[id] = k2f[id].x;
        if (order == 6) fr[id] = make_float4(G[id].x, gx[id].x, gy[id].x, gz[id].x);
    }
}
}  // namespace

// Set-up of the real-medium matvec: when Im k^2 vanishes everywhere (a medium without attenuation), the
// complex64 matvec stages k^2 as float and reads the four order-6 fields as one real float4 per point
// (36 instead of 56 bytes per point, real instead of complex products).  Synchronises s.
helm_status stencil_real_prepare(helm_ctx* c, cudaStream_t s) {
    if (!stencil_fast_supported(c)) return HELM_OK;
    unsigned* flag = nullptr;
    unsigned h = 1;
    HELM_CUDA_TRY(cudaMalloc(&flag, sizeof(unsigned)));
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        imag_any_kernel<<<1024, 256, 0, s>>>(c->k2_d, c->npts, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    HELM_CUDA_TRY(e);
    if (h) return HELM_OK;   // complex k^2: the general kernels
    if (cudaMalloc(&c->k2r, c->npts * sizeof(float)) != cudaSuccess ||
        (c->opt.order == 6 && cudaMalloc(&c->fr, c->npts * sizeof(float4)) != cudaSuccess)) {
        cudaGetLastError();
        cudaFree(c->k2r);
        c->k2r = nullptr;
        return HELM_ERR_NOMEM;
    }
    real_fields_kernel<<<1024, 256, 0, s>>>(c->npts, c->opt.order, c->k2_f, c->G_f, c->dk2_f[0], c->dk2_f[1],
                                            c->dk2_f[2], c->k2r, c->fr);
    HELM_CUDA_TRY(cudaGetLastError());
    c->realk = 1;
    if (c->opt.order == 6) c->tune_stencil = 3;   // two rows per thread (variant 4, the fields formed in the kernel, moves half the bytes but issues 40% more instructions: slower alone)
    return HELM_OK;
}

bool stencil_fast_supported(const helm_ctx* c) { return !c->colloc && (c->opt.order == 4 || c->opt.order == 6); }

// Variants of the complex64 matvec a context can run: 0 = cp.async ring at four CTAs per SM, 1 = TMA ring
// (even N_x, else the same as 0), 2 = cp.async ring at three CTAs per SM with more registers, 3 = two rows
// per thread (real media; else the same as 2), 4 = two rows with the sixth-order fields formed in the kernel
// (real media, order 6; else the same as 3).
int stencil_variants(const helm_ctx* c) { (void)c; return 5; }

helm_status launch_stencil_fast(helm_ctx* c, const float2* x, float2* y, const double* sigma, int sidx, cudaStream_t s,
                                int nb) {
    if (nb > 1 && c->sfast && c->tune_stencil == 1) {
        // the TMA form stages one vector: one launch per vector of the batch
        helm_status st;
        for (int v = 0; v < nb; ++v)
            if ((st = launch_stencil_fast(c, x + (size_t)v * c->npts, y + (size_t)v * c->npts, sigma, sidx, s, 1)) !=
                HELM_OK)
                return st;
        return HELM_OK;
    }
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
    p.nb = nb;
    for (int d = 0; d < 3; ++d) {
        p.i12h[d] = (float)(1.0 / (12.0 * c->h[d]));
        p.i12h2[d] = (float)(1.0 / (12.0 * c->h[d] * c->h[d]));
    }
    dim3 grid((c->nx + FTX - 1) / FTX, (c->ny + FTY - 1) / FTY, (c->nz + FZCH - 1) / FZCH * nb), block(FTX, FTY);
    if (c->sfast && c->tune_stencil == 1) {
        FastMaps* m = (FastMaps*)c->sfast;
        CUtensorMap mU;
        if (encode3(m, &mU, x, c->nx, c->ny, c->nz, 2 * TPX, FPY) == HELM_OK) {
            if (c->opt.order == 6)
                stencil_tma_kernel<6><<<grid, block, TLayout<6>::SMEM, s>>>(mU, m->mK, m->mF[0], m->mF[1], m->mF[2],
                                                                           m->mF[3], p, y, sigma, sidx, c->status_d,
                                                                           (long)c->wait_limit);
            else
                stencil_tma_kernel<4><<<grid, block, TLayout<4>::SMEM, s>>>(mU, m->mK, m->mF[0], m->mF[1], m->mF[2],
                                                                           m->mF[3], p, y, sigma, sidx, c->status_d,
                                                                           (long)c->wait_limit);
            HELM_CUDA_TRY(cudaGetLastError());
            return HELM_OK;
        }
    }
    const bool three = c->tune_stencil >= 2;   // the variant with up to 85 registers, three CTAs per SM
    if (c->realk) {
        p.k2r = c->k2r;
        p.fr = c->fr;
        if (c->tune_stencil == 4 && c->opt.order == 6) {   // two rows per thread, fields formed in the kernel
            const dim3 block2(FTX, FTY / 2);
            stencil_fast3_kernel<4><<<grid, block2, F3_SMEM, s>>>(p, x, y, sigma, sidx);
            HELM_CUDA_TRY(cudaGetLastError());
            return HELM_OK;
        }
        if (c->tune_stencil >= 3) {   // two rows per thread
            const dim3 block2(FTX, FTY / 2);
            if (c->opt.order == 6) stencil_fast2_kernel<6, 4><<<grid, block2, fast2_smem<6>(), s>>>(p, x, y, sigma, sidx);
            else stencil_fast2_kernel<4, 4><<<grid, block2, fast2_smem<4>(), s>>>(p, x, y, sigma, sidx);
            HELM_CUDA_TRY(cudaGetLastError());
            return HELM_OK;
        }
        if (c->opt.order == 6) {
            if (three) stencil_fast_kernel<6, 3, true><<<grid, block, fast_smem<6, true>(), s>>>(p, x, y, sigma, sidx);
            else stencil_fast_kernel<6, 4, true><<<grid, block, fast_smem<6, true>(), s>>>(p, x, y, sigma, sidx);
        } else {
            if (three) stencil_fast_kernel<4, 3, true><<<grid, block, fast_smem<4, true>(), s>>>(p, x, y, sigma, sidx);
            else stencil_fast_kernel<4, 4, true><<<grid, block, fast_smem<4, true>(), s>>>(p, x, y, sigma, sidx);
        }
        HELM_CUDA_TRY(cudaGetLastError());
        return HELM_OK;
    }
    if (c->opt.order == 6) {
        if (three) stencil_fast_kernel<6, 3><<<grid, block, fast_smem<6>(), s>>>(p, x, y, sigma, sidx);
        else stencil_fast_kernel<6, 4><<<grid, block, fast_smem<6>(), s>>>(p, x, y, sigma, sidx);
    } else {
        if (three) stencil_fast_kernel<4, 3><<<grid, block, fast_smem<4>(), s>>>(p, x, y, sigma, sidx);
        else stencil_fast_kernel<4, 4><<<grid, block, fast_smem<4>(), s>>>(p, x, y, sigma, sidx);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// ---- the true residual r = F - A x in double-float -------------------------------------------
// Same plane-quantity form and z-march as the complex64 matvec, with x, k^2, G and F in double-float
// (float4: re.hi, im.hi, re.lo, im.lo) and every term of A in double-float except the gradient terms
// (h/20) g_d D_d, below 1e-3 of the total, which take the leading parts in FP32.  Planes stream into a
// four-slot ring by 16-byte cp.async of the clamped halo points; a prepare pass per plane applies the
// ghost factors (double-float) and forms KU = k^2 U once per staged point.  Writes r rounded to complex64
// and per-CTA partial sums of |r|^2 and max |r| in FP64.
#include "dfloat.cuh"

namespace {

template <int ORDER>
struct RStage {
    float4 u[FHALO];
    float4 k[FHALO];
    float4 F[FNT];
    float4 G[ORDER == 6 ? FNT : 1];
    float2 g[ORDER == 6 ? 3 : 1][ORDER == 6 ? FNT : 1];
};

struct RParams {
    int nx, ny, nz;
    cdf gx, gy, gz;
    df ihx, ihy, ihz, wxy, wxz, wyz, h2_20;
    float h_20, hh6;
    const float4* k2;
    const float4* G;
    const float2* g[3];
    const float4* F;
};

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// double-float constants, evaluated by the compiler
constexpr df dfc(double v) { return df{(float)v, (float)(v - (double)(float)v)}; }
template <int NUM, int DEN>
__device__ __forceinline__ cdf cdf_sc(cdf a) {
    constexpr df s = dfc((double)NUM / (double)DEN);
    return cdf_scale(a, s);
}
__device__ __forceinline__ float2 hi2(cdf a) { return a.hi; }

template <int ORDER>
__global__ void __launch_bounds__(FNT, 2)
residual_fast_kernel(RParams p, const float4* __restrict__ X, float2* __restrict__ rout, double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char rsm[];
    RStage<ORDER>* ring = reinterpret_cast<RStage<ORDER>*>(rsm);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < p.nx && gy < p.ny;
    // this thread's staging slots (fixed across planes): clamped in-plane offset and the x/y ghost factor
    size_t soff[2] = {0, 0};
    int sfix[2] = {0, 0};
    cdf sgam[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int q = tid + k * FNT;
        sgam[k] = cdf{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
        if (q < FHALO) {
            const int ly = q / FPX, lx = q - ly * FPX;
            const int Xg = x0 + lx - 1, Yg = y0 + ly - 1;
            const int Xc = min(max(Xg, 0), p.nx - 1), Yc = min(max(Yg, 0), p.ny - 1);
            soff[k] = (size_t)Yc * p.nx + Xc;
            if (Xc != Xg) { sgam[k] = p.gx; sfix[k] = 1; }
            if (Yc != Yg) { sgam[k] = sfix[k] ? cdf_mul(sgam[k], p.gy) : p.gy; sfix[k] = 1; }
        }
    }
    const size_t poff = (size_t)gy * p.nx + gx;
    const size_t plane = (size_t)p.nx * p.ny;
    auto issue = [&](int P) {
        if (P <= z1) {
            RStage<ORDER>& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const size_t pb = (size_t)Pc * plane;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = tid + k * FNT;
                if (q < FHALO) {
                    cp16(&S.u[q], X + pb + soff[k]);
                    cp16(&S.k[q], p.k2 + pb + soff[k]);
                }
            }
            if (P >= z0 && P < z1 && active) {
                const size_t g = (size_t)P * plane + poff;
                cp16(&S.F[tid], p.F + g);
                if (ORDER == 6) {
                    cp16(&S.G[tid], p.G + g);
#pragma unroll
                    for (int d = 0; d < 3; ++d) cp8(&S.g[d][tid], p.g[d] + g);
                }
            }
        }
        cp_commit();
    };

    cdf cA = cdf_zero(), nA = cdf_zero();
    float2 cX = make_float2(0, 0), cY = cX, cZ = cX, nX = cX, nY = cX, nZ = cX;
    float fsum = 0.f, fcmp = 0.f, fmx = 0.f;   // per-thread compensated FP32 sum and max of |r|^2
    issue(z0 - 1);
    issue(z0);
    for (int P = z0 - 1; P <= z1; ++P) {
        RStage<ORDER>& S = ring[(P + FNS) % FNS];
        cp_wait1();
        __syncthreads();          // plane P landed for every thread; everyone is done with plane P-1
        const bool zghost = P < 0 || P >= p.nz;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q = tid + k * FNT;
            if (q < FHALO) {
                cdf u = cdf_from4(S.u[q]);
                if (sfix[k]) u = cdf_mul(u, sgam[k]);
                if (zghost) u = cdf_mul(u, p.gz);
                if (sfix[k] || zghost) S.u[q] = cdf_to4(u);
                S.k[q] = cdf_to4(cdf_mul(cdf_from4(S.k[q]), u));
            }
        }
        __syncthreads();          // U with ghosts and KU of plane P ready
        issue(P + 2);             // into the slot of plane P-2, which nobody reads any more
        cdf c, fx, fy, e, kc, kf4, kcs;
        float2 dx1, dy1, tdx, tdy, dkx, dky;
        {
            auto U = [&](int b, int a) { return cdf_from4(S.u[(ty + b) * FPX + tx + a]); };
            auto K = [&](int b, int a) { return cdf_from4(S.k[(ty + b) * FPX + tx + a]); };
            const cdf u10 = U(1, 0), u12 = U(1, 2), u01 = U(0, 1), u21 = U(2, 1);
            const cdf u00 = U(0, 0), u02 = U(0, 2), u20 = U(2, 0), u22 = U(2, 2);
            c = U(1, 1);
            fx = cdf_add(u10, u12);
            fy = cdf_add(u01, u21);
            e = cdf_add(cdf_add(u00, u02), cdf_add(u20, u22));
            dx1 = f2sub(hi2(u12), hi2(u10));
            dy1 = f2sub(hi2(u21), hi2(u01));
            tdx = f2sub(f2add(hi2(u02), hi2(u22)), f2add(hi2(u00), hi2(u20)));
            tdy = f2sub(f2add(hi2(u20), hi2(u22)), f2add(hi2(u00), hi2(u02)));
            const cdf k10 = K(1, 0), k12 = K(1, 2), k01 = K(0, 1), k21 = K(2, 1);
            kc = K(1, 1);
            kf4 = cdf_add(cdf_add(k10, k12), cdf_add(k01, k21));
            dkx = f2sub(hi2(k12), hi2(k10));
            dky = f2sub(hi2(k21), hi2(k01));
            if (ORDER == 6) kcs = cdf_add(cdf_add(K(0, 0), K(0, 2)), cdf_add(K(2, 0), K(2, 2)));
        }
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;
        const bool do_mid = P >= z0 && P < z1;
        const RStage<ORDER>& Sp = ring[(P - 1 + FNS) % FNS];
        const cdf fxy = cdf_add(fx, fy);
        cdf As;
        float2 Xs = make_float2(0, 0), Ys = Xs, Zs = Xs;
        if (ORDER == 6) {
            As = cdf_scale(cdf_add(cdf_add(cdf_sc<7, 15>(c), cdf_sc<1, 10>(fxy)), cdf_sc<1, 30>(e)), p.ihx);
            As = cdf_add(As, cdf_sc<1, 90>(cdf_sub(kf4, kc)));
            Xs = f2scl(dx1, 1.f / 6.f);
            Ys = f2scl(dy1, 1.f / 6.f);
            const float2 ch = hi2(c);
            Zs = f2add(f2fma(p.hh6, hi2(kc), ch), f2scl(f2fma(-4.f, ch, hi2(fxy)), 1.f / 6.f));
        } else {
            const cdf c2 = cdf_add(c, c);
            As = cdf_add(cdf_add(cdf_scale(c, p.ihz), cdf_scale(cdf_sub(fx, c2), p.wxz)),
                         cdf_add(cdf_scale(cdf_sub(fy, c2), p.wyz), cdf_sc<1, 12>(kc)));
        }
        if (out_prev) {
            cdf A = cdf_add(cA, As);
            if (ORDER == 6) {
                float2 g = f2mul(Sp.g[0][tid], f2add(cX, Xs));
                g = f2add(g, f2mul(Sp.g[1][tid], f2add(cY, Ys)));
                g = f2add(g, f2mul(Sp.g[2][tid], f2add(cZ, Zs)));
                A = cdf_add(A, cdf_from_f2(f2scl(g, p.h_20)));
            }
            if (active) {
                const cdf r = cdf_sub(cdf_from4(Sp.F[tid]), A);
                const float2 rf = cdf_round(r);
                rout[(size_t)(P - 1) * plane + poff] = rf;
                const float a2 = fmaf(rf.x, rf.x, rf.y * rf.y);
                kahan_add(fsum, fcmp, a2);
                fmx = fmaxf(fmx, a2);
            }
        }
        cA = nA; cX = nX; cY = nY; cZ = nZ;
        if (do_mid) {
            if (ORDER == 6) {
                cdf Am = cdf_scale(cdf_sub(cdf_add(cdf_sc<7, 15>(fxy), cdf_sc<1, 10>(e)), cdf_sc<64, 15>(c)),
                                   p.ihx);
                Am = cdf_add(Am, cdf_add(cdf_sc<14, 15>(kc), cdf_sc<1, 90>(cdf_sub(kcs, kf4))));
                Am = cdf_add(Am, cdf_scale(cdf_mul(cdf_from4(S.G[tid]), c), p.h2_20));
                const float2 Xm = f2add(f2fma(p.hh6, dkx, dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                const float2 Ym = f2add(f2fma(p.hh6, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                cA = cdf_add(cA, Am);
                cX = f2add(cX, Xm);
                cY = f2add(cY, Ym);
            } else {
                const cdf c2 = cdf_add(c, c), c4 = cdf_add(c2, c2);
                cdf Am = cdf_add(cdf_scale(cdf_sub(fx, c2), p.ihx), cdf_scale(cdf_sub(fy, c2), p.ihy));
                Am = cdf_sub(Am, cdf_scale(c2, p.ihz));
                Am = cdf_add(Am, cdf_scale(cdf_add(cdf_sub(e, cdf_add(fxy, fxy)), c4), p.wxy));
                Am = cdf_add(Am, cdf_scale(cdf_sub(c4, cdf_add(fx, fx)), p.wxz));
                Am = cdf_add(Am, cdf_scale(cdf_sub(c4, cdf_add(fy, fy)), p.wyz));
                Am = cdf_add(Am, cdf_add(cdf_sc<1, 2>(kc), cdf_sc<1, 12>(kf4)));
                cA = cdf_add(cA, Am);
            }
        }
        nA = As; nX = Xs; nY = Ys; nZ = make_float2(-Zs.x, -Zs.y);
    }
    __shared__ double rs[FNT / 32], rm[FNT / 32];
    double ssum = (double)fsum - (double)fcmp, smax = (double)fmx;   // FP64 across threads
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_down_sync(0xffffffffu, ssum, o);
        smax = fmax(smax, __shfl_down_sync(0xffffffffu, smax, o));
    }
    if ((tid & 31) == 0) { rs[tid >> 5] = ssum; rm[tid >> 5] = smax; }
    __syncthreads();
    if (tid == 0) {
        double s = 0, m = 0;
        for (int w = 0; w < FNT / 32; ++w) { s += rs[w]; m = fmax(m, rm[w]); }
        const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * cta] = s;
        part[2 * cta + 1] = sqrt(m);
    }
}

template <int ORDER>
int rsmem() { return (int)(FNS * sizeof(RStage<ORDER>)); }

cdf cdf_host(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return cdf{make_float2(rh, ih), make_float2((float)(v.x - (double)rh), (float)(v.y - (double)ih))};
}
df df_host(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}

// ---- the true residual, sixth order, real media: two rows per thread, compensated sums ------------
// For a medium without attenuation the sixth-order operator, divided by c_L = 1/(30 h^2), contributes per
// plane Q of the z-march (the factors of the kernel above times 30 h^2):
//   as a neighbour plane (Q = P -+ 1):  14 c + 3 f + e + (kf - kc)
//   as the centre plane (Q = P):        14 f + 3 e - 128 c + (84 kc + kcs - kf) + Gq c
// with c, f, e the centre value, the sum of the four in-plane face neighbours and of the four in-plane
// corners of U, kc, kf, kcs the same sums of Kq U, Kq = k^2 h^2 / 3, Gq = (3/2) h^4 G; the gradient terms
// (h/20) g_d D_d become (3/2) h^3 g_d D_d, taken in FP32 from the leading parts as above.  Then A x =
// c_L S and r = F - c_L S.  Every sum is an unnormalised double-float pair (one two-sum per addition, the
// errors gathered in the low part), every product by a constant one FMA-exact product: about half the
// instructions of the renormalised form.  A thread computes the points (x, 2t) and (x, 2t + 1) of the
// 32 x 8 tile from one 4 x 3 patch of U and Kq; x, Kq, F and the per-point fields stream into a four-slot
// cp.async ring; the ghost factors are applied in shared memory only by tiles touching the boundary and on
// the ghost planes.  Same grid and per-CTA partial sums as the kernel above.
struct R6Stage {
    float4 u[FHALO];     // x on the halo (re.hi, im.hi, re.lo, im.lo)
    float2 kq[FHALO];    // Kq on the halo (hi, lo)
    float4 F[FNT];       // F at the tile's points
    float4 g4[FNT];      // (Gq hi, Gq lo, gq_x, gq_y)
    float gz[FNT];       // gq_z
};
constexpr size_t R6_SMEM = FNS * sizeof(R6Stage);   // 69,504 bytes: three CTAs per SM

struct R6Params {
    int nx, ny, nz;
    cdf gx, gy, gz;      // ghost factors
    df cL;               // 1 / (30 h^2)
    const float2* kq;
    const float4* g4;
    const float* gzq;
    const float4* F;
};

__global__ void __launch_bounds__(F2T, 3)
residual_real6_kernel(R6Params p, const float4* __restrict__ X, float2* __restrict__ rout, double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char r6sm[];
    R6Stage* ring = reinterpret_cast<R6Stage*>(r6sm);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;   // ty = 0 .. 3
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * FZCH;
    const int z1 = min(z0 + FZCH, p.nz);
    const int gx = x0 + tx, gy0 = y0 + 2 * ty;
    const bool act[2] = {gx < p.nx && gy0 < p.ny, gx < p.nx && gy0 + 1 < p.ny};
    const bool edge = x0 == 0 || y0 == 0 || x0 + FTX >= p.nx || y0 + FTY >= p.ny;
    unsigned sl[3] = {0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = tid + k * F2T;
        if (q < FHALO) {
            const int ly = q / FPX, lx = q - ly * FPX;
            const int Xg = x0 + lx - 1, Yg = y0 + ly - 1;
            const int Xc = min(max(Xg, 0), p.nx - 1), Yc = min(max(Yg, 0), p.ny - 1);
            sl[k] = (unsigned)(Yc * p.nx + Xc) | (Xc != Xg ? 1u << 30 : 0u) | (Yc != Yg ? 1u << 31 : 0u);
        }
    }
    const size_t plane = (size_t)p.nx * p.ny;
    const int poff = gy0 * p.nx + gx;
    const int fi = (2 * ty) * FTX + tx;   // point r of this thread at index fi + r FTX of the per-point arrays

    auto issue = [&](int P) {
        if (P <= z1) {
            R6Stage& S = ring[(P + FNS) % FNS];
            const int Pc = min(max(P, 0), p.nz - 1);
            const float4* Xb = X + (size_t)Pc * plane;
            const float2* Kb = p.kq + (size_t)Pc * plane;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (tid + k * F2T < FHALO) {
                    cp16f(&S.u[tid + k * F2T], Xb + (sl[k] & 0x3FFFFFFFu));
                    cp8(&S.kq[tid + k * F2T], Kb + (sl[k] & 0x3FFFFFFFu));
                }
            if (P >= z0 && P < z1) {
                const size_t g = (size_t)P * plane + poff;
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (act[r]) {
                        cp16f(&S.F[fi + r * FTX], p.F + g + r * p.nx);
                        cp16f(&S.g4[fi + r * FTX], p.g4 + g + r * p.nx);
                        cp4(&S.gz[fi + r * FTX], p.gzq + g + r * p.nx);
                    }
            }
        }
        cp_commit();
    };

    cdf cS[2], nS[2];
    float2 cX[2], cY[2], cZ[2], nX[2], nY[2], nZ[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        cS[r] = nS[r] = cdf_zero();
        cX[r] = cY[r] = cZ[r] = nX[r] = nY[r] = nZ[r] = make_float2(0.f, 0.f);
    }
    float fsum = 0.f, fcmp = 0.f, fmx = 0.f;
    issue(z0 - 1);
    issue(z0);
    for (int P = z0 - 1; P <= z1; ++P) {
        R6Stage& S = ring[(P + FNS) % FNS];
        cp_wait1();
        __syncthreads();          // plane P landed for everyone; everyone is done with planes P-1 and P-2
        const bool zghost = P < 0 || P >= p.nz;
        if (edge || zghost) {     // uniform per CTA and plane
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int q = tid + k * F2T;
                if (q < FHALO && ((sl[k] >> 30) || zghost)) {
                    cdf u = cdf_from4(S.u[q]);
                    if (sl[k] & (1u << 30)) u = cdf_mul(u, p.gx);
                    if (sl[k] & (1u << 31)) u = cdf_mul(u, p.gy);
                    if (zghost) u = cdf_mul(u, p.gz);
                    S.u[q] = cdf_to4(u);
                }
            }
            __syncthreads();
        }
        issue(P + 2);             // into the slot of plane P-2
        // per patch row b (halo row 2t + b): centre column, the pair sum of the side columns and their
        // leading-part difference, for U and for Kq U
        cdf um[4], hu[4], km[4], hk[4];
        float2 du[4], dk[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = (2 * ty + b) * FPX + tx;
            const cdf u0 = cdf_from4(S.u[i]), u1 = cdf_from4(S.u[i + 1]), u2 = cdf_from4(S.u[i + 2]);
            const float2 q0 = S.kq[i], q1 = S.kq[i + 1], q2 = S.kq[i + 2];
            const cdf k0 = cp_mul(u0, df{q0.x, q0.y}), k1 = cp_mul(u1, df{q1.x, q1.y}), k2 = cp_mul(u2, df{q2.x, q2.y});
            um[b] = u1;
            hu[b] = cp_add(u0, u2);
            du[b] = sub2(u2.hi, u0.hi);
            km[b] = k1;
            hk[b] = cp_add(k0, k2);
            dk[b] = sub2(k2.hi, k0.hi);
        }
        const bool out_prev = P - 1 >= z0 && P - 1 < z1;
        const bool do_mid = P >= z0 && P < z1;
        const R6Stage& Sp = ring[(P - 1 + FNS) % FNS];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const cdf c = um[r + 1];
            const cdf f = cp_add(hu[r + 1], cp_add(um[r], um[r + 2]));
            const cdf e = cp_add(hu[r], hu[r + 2]);
            const cdf kc = km[r + 1];
            const cdf kf = cp_add(hk[r + 1], cp_add(km[r], km[r + 2]));
            // this plane as a neighbour plane
            const cdf nb = cp_add(cp_add(cp_mulk(c, 14.f), cp_mulk(f, 3.f)), cp_add(e, cp_sub(kf, kc)));
            const float2 dx1 = du[r + 1], dy1 = sub2(um[r + 2].hi, um[r].hi);
            const float2 Xs = f2scl(dx1, 1.f / 6.f), Ys = f2scl(dy1, 1.f / 6.f);
            const float2 Zs = f2add(f2fma(0.5f, kc.hi, c.hi), f2scl(f2fma(-4.f, c.hi, f.hi), 1.f / 6.f));
            if (out_prev && act[r]) {
                const int j = fi + r * FTX;
                const float4 gv = Sp.g4[j];
                float2 g = f2scl(f2add(cX[r], Xs), gv.z);
                g = f2fma(gv.w, f2add(cY[r], Ys), g);
                g = f2fma(Sp.gz[j], f2add(cZ[r], Zs), g);
                const cdf Ssum = cp_add_f2(cp_add(cS[r], nb), g);
                const cdf R = cp_sub(cdf_from4(Sp.F[j]), cp_mul(Ssum, p.cL));
                const float2 rf = add2(R.hi, R.lo);
                rout[(size_t)(P - 1) * plane + poff + r * p.nx] = rf;
                const float a2 = fmaf(rf.x, rf.x, rf.y * rf.y);
                kahan_add(fsum, fcmp, a2);
                fmx = fmaxf(fmx, a2);
            }
            cS[r] = nS[r]; cX[r] = nX[r]; cY[r] = nY[r]; cZ[r] = nZ[r];
            if (do_mid) {
                const cdf kcs = cp_add(hk[r], hk[r + 2]);
                const float4 gv = S.g4[fi + r * FTX];
                cdf ce = cp_sub(cp_add(cp_mulk(f, 14.f), cp_mulk(e, 3.f)), cdf{f2scl(c.hi, 128.f), f2scl(c.lo, 128.f)});
                ce = cp_add(ce, cp_sub(cp_add(cp_mulk(kc, 84.f), kcs), kf));
                ce = cp_add(ce, cp_mul(c, df{gv.x, gv.y}));
                const float2 tdx = f2add(du[r], du[r + 2]), tdy = f2sub(hu[r + 2].hi, hu[r].hi);
                const float2 dky = sub2(km[r + 2].hi, km[r].hi);
                const float2 Xm = f2add(f2fma(0.5f, dk[r + 1], dx1), f2scl(f2fma(-4.f, dx1, tdx), 1.f / 6.f));
                const float2 Ym = f2add(f2fma(0.5f, dky, dy1), f2scl(f2fma(-4.f, dy1, tdy), 1.f / 6.f));
                cS[r] = cp_add(cS[r], ce);
                cX[r] = f2add(cX[r], Xm);
                cY[r] = f2add(cY[r], Ym);
            }
            nS[r] = nb; nX[r] = Xs; nY[r] = Ys; nZ[r] = make_float2(-Zs.x, -Zs.y);
        }
    }
    __shared__ double rs[F2T / 32], rm[F2T / 32];
    double ssum = (double)fsum - (double)fcmp, smax = (double)fmx;
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_down_sync(0xffffffffu, ssum, o);
        smax = fmax(smax, __shfl_down_sync(0xffffffffu, smax, o));
    }
    if ((tid & 31) == 0) { rs[tid >> 5] = ssum; rm[tid >> 5] = smax; }
    __syncthreads();
    if (tid == 0) {
        double s = 0, m = 0;
        for (int w = 0; w < F2T / 32; ++w) { s += rs[w]; m = fmax(m, rm[w]); }
        const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * cta] = s;
        part[2 * cta + 1] = sqrt(m);
    }
}

// the residual's real-medium fields from the FP64 set-up fields (real parts; Im k^2 = 0 everywhere)
__global__ void resid6_fields_kernel(size_t n, double h, const double2* __restrict__ k2, const double2* __restrict__ G,
                                     const double2* __restrict__ gx, const double2* __restrict__ gy,
                                     const double2* __restrict__ gz, float2* __restrict__ kq, float4* __restrict__ g4,
                                     float* __restrict__ gzq) {
    const double h2 = h * h, cq = h2 / 3.0, cg = 1.5 * h2 * h2, cd = 1.5 * h2 * h;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const double k = k2[id].x * cq, g = G[id].x * cg;
        const float kh = (float)k, gh = (float)g;
        kq[id] = make_float2(kh, (float)(k - (double)kh));
        g4[id] = make_float4(gh, (float)(g - (double)gh), (float)(gx[id].x * cd), (float)(gy[id].x * cd));
        gzq[id] = (float)(gz[id].x * cd);
    }
}

}  // namespace

helm_status residual_fast_prepare() {
    HELM_CUDA_TRY(cudaFuncSetAttribute(residual_fast_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, rsmem<4>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(residual_fast_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, rsmem<6>()));
    HELM_CUDA_TRY(cudaFuncSetAttribute(residual_real6_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R6_SMEM));
    return HELM_OK;
}

// Fields of the sixth-order real-medium residual (after stencil_real_prepare found Im k^2 = 0): 28 bytes
// per point.  Without them the residual takes the complex-medium kernel.
helm_status residual_real_prepare(helm_ctx* c, cudaStream_t s) {
    if (!c->realk || c->opt.order != 6) return HELM_OK;
    if (cudaMalloc(&c->rkq, c->npts * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&c->rg4, c->npts * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&c->rgz, c->npts * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        residual_real_release(c);
        return HELM_ERR_NOMEM;
    }
    resid6_fields_kernel<<<1024, 256, 0, s>>>(c->npts, c->h[0], c->k2_d, c->G_d, c->dk2_d[0], c->dk2_d[1], c->dk2_d[2],
                                              c->rkq, c->rg4, c->rgz);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

void residual_real_release(helm_ctx* c) {
    cudaFree(c->rkq);
    cudaFree(c->rg4);
    cudaFree(c->rgz);
    c->rkq = nullptr;
    c->rg4 = nullptr;
    c->rgz = nullptr;
}

// grid of the residual kernels: 32 x 8 columns, 32-plane chunks (one partial pair per CTA)
helm_status launch_residual_fast(helm_ctx* c, const float4* x, const float4* F, float2* r, double* part,
                                 cudaStream_t s) {
    RParams p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.gx = cdf_host(c->gam[0]); p.gy = cdf_host(c->gam[1]); p.gz = cdf_host(c->gam[2]);
    const double hx = c->h[0], hy = c->h[1], hz = c->h[2];
    const double ihx = 1.0 / (hx * hx), ihy = 1.0 / (hy * hy), ihz = 1.0 / (hz * hz);
    p.ihx = df_host(ihx); p.ihy = df_host(ihy); p.ihz = df_host(ihz);
    p.wxy = df_host((hx * hx + hy * hy) / 12.0 * ihx * ihy);
    p.wxz = df_host((hx * hx + hz * hz) / 12.0 * ihx * ihz);
    p.wyz = df_host((hy * hy + hz * hz) / 12.0 * ihy * ihz);
    p.h2_20 = df_host(hx * hx / 20.0);
    p.h_20 = (float)(hx / 20.0);
    p.hh6 = (float)(hx * hx / 6.0);
    p.k2 = c->k2_df;
    p.G = c->G_df;
    for (int d = 0; d < 3; ++d) p.g[d] = c->dk2_f[d];
    p.F = F;
    dim3 grid((c->nx + FTX - 1) / FTX, (c->ny + FTY - 1) / FTY, (c->nz + FZCH - 1) / FZCH), block(FTX, FTY);
    if (c->opt.order == 6 && c->rkq) {
        R6Params q;
        q.nx = c->nx; q.ny = c->ny; q.nz = c->nz;
        q.gx = p.gx; q.gy = p.gy; q.gz = p.gz;
        q.cL = df_host(1.0 / (30.0 * hx * hx));
        q.kq = c->rkq; q.g4 = c->rg4; q.gzq = c->rgz; q.F = F;
        residual_real6_kernel<<<grid, dim3(FTX, FTY / 2), R6_SMEM, s>>>(q, x, r, part);
    } else if (c->opt.order == 6)
        residual_fast_kernel<6><<<grid, block, rsmem<6>(), s>>>(p, x, r, part);
    else
        residual_fast_kernel<4><<<grid, block, rsmem<4>(), s>>>(p, x, r, part);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
