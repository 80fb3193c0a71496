// EigT step 3 (Sec. 4.1): the N_x N_y independent complex tridiagonal systems of
// Eq. Indep_precond_system along z,
//   (gamma_z + b_1) u_1 + zeta_z u_2 = y_1
//   u_{l-1} + b_l u_l + u_{l+1} = y_l
//   zeta_z u_{N-1} + (gamma_z + b_N) u_N = y_N,
//   b_l = alpha_x d_{x,i} + alpha_y d_{y,j} + h_z^2 k0^2(z_l) - 2(alpha_x + alpha_y + 1).
//
// Design (ours): the systems are lines of stride N_x N_y through HBM, so a CTA takes L consecutive
// lines (consecutive i: every access is a contiguous L x 8-byte row) and cuts each line into W chunks
// of at most MCH rows, one chunk per thread.  Each thread keeps its chunk in registers and eliminates
// it twice without pivoting (down, then up), which expresses the chunk's end values through its
// neighbours' end values.  One thread per line solves that small block-tridiagonal interface system
// (2 unknowns per chunk) from shared memory, and every thread then finishes its chunk by a Thomas sweep
// with known boundary values.  HBM traffic is one read and one write per point (16 B/pt).
// This partitioned kernel solves the systems when no set-up factors exist; every EigT and PFFT context
// factorises its systems at set-up, so the factorised forms below serve the solver.
#include "common.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

struct ZParams {
    int nx, ny, nz, W;
    const float2* dxs;   // alpha_x d_{x,i}
    const float2* dys;   // alpha_y d_{y,j}
    const float2* cz;    // h_z^2 k0^2(z_l) - 2(alpha_x + alpha_y + 1)
    float2 gz;           // gamma_z
    float zz;            // zeta_z
    // optional generated right-hand side: y[l][j][i] += sum_{t<4} P[t][l][j] Q[t][l][i]  (PFFT)
    const float2* P;
    const float2* Q;
};

__device__ inline float2 f2(float a, float b) { return make_float2(a, b); }

// a / b for the well-scaled pivots of these systems (|b| ~ 1e-3 .. 1e2): a conj(b) / |b|^2
__device__ inline float2 qdiv(float2 a, float2 b) {
    const float r = __frcp_rn(fmaf(b.x, b.x, b.y * b.y));
    return make_float2((a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r);
}
// 1 / b (one correctly rounded reciprocal; every division of an elimination step shares it)
__device__ inline float2 crcp(float2 b) {
    const float r = __frcp_rn(fmaf(b.x, b.x, b.y * b.y));
    return make_float2(b.x * r, -b.y * r);
}

// The steps of the factorised solve, every operation rounded as written (explicit fma/mul/add, so that no
// kernel contracts differently): the set-up factors, the forward and backward sweeps over stored factors
// and the sweeps that recompute the factors all produce the same bits.
// pivot step: m_l = 1 / (b_l - a_l c'_{l-1}) with b_l = s + cz_l (+ gamma_z at the ends), then c'_l = sup_l m_l
// (*dmag, when given: |Re| + |Im| of the pivot, for the tiny-pivot check of the set-up)
__device__ __forceinline__ float2 zpivot(float2 s, float2 czl, bool end, float2 gz, float a, float sup, float2& c,
                                         float* dmag = nullptr) {
    float bx = __fadd_rn(s.x, czl.x), by = __fadd_rn(s.y, czl.y);
    if (end) { bx = __fadd_rn(bx, gz.x); by = __fadd_rn(by, gz.y); }
    const float dx = __fmaf_rn(-c.x, a, bx), dy = __fmaf_rn(-c.y, a, by);
    if (dmag) *dmag = fabsf(dx) + fabsf(dy);
    // 1/|pivot|^2 by the hardware reciprocal (at most one ulp off, one instruction: the recurrence is the
    // critical path of every line), then m = conj(pivot) / |pivot|^2
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))));
    const float2 m = make_float2(__fmul_rn(dx, r), __fmul_rn(-dy, r));
    c = make_float2(__fmul_rn(m.x, sup), __fmul_rn(m.y, sup));
    return m;
}
// forward: d_l = (y_l - a_l d_{l-1}) m_l
__device__ __forceinline__ float2 zfwd(float2 y, float2 d, float a, float2 m) {
    const float tx = __fmaf_rn(-d.x, a, y.x), ty = __fmaf_rn(-d.y, a, y.y);
    return make_float2(__fmaf_rn(tx, m.x, __fmul_rn(-ty, m.y)), __fmaf_rn(tx, m.y, __fmul_rn(ty, m.x)));
}
// backward: x_l = d_l - sup_l (m_l x_{l+1})
__device__ __forceinline__ float2 zbwd(float2 d, float2 m, float2 x, float sup) {
    const float px = __fmaf_rn(m.x, x.x, __fmul_rn(-m.y, x.y)), py = __fmaf_rn(m.x, x.y, __fmul_rn(m.y, x.x));
    return make_float2(__fmaf_rn(-px, sup, d.x), __fmaf_rn(-py, sup, d.y));
}

template <int L, int MCH>
__global__ void __launch_bounds__(L * 32)
zsolve_kernel(ZParams p, const float2* in, float2* out, unsigned* status) {
    // per chunk and line: [0] g_s, [1] p_s, [2] q_s, [3] g_e, [4] p_e, [5] q_e; reused by the interface
    // solve for Y_c / X_c (slots 0 and 3) and Gamma_c (slots 1 and 2)
    __shared__ float2 sh[6][32][L];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int W = p.W, nz = p.nz;
    const int i = blockIdx.x * L + lane, j = blockIdx.y;
    const bool live = i < p.nx;
    // balanced chunks: every chunk has at least two rows when nz >= 2W (MCH >= 4 guarantees it)
    const int s = (int)(((long)w * nz) / W), e = (int)(((long)(w + 1) * nz) / W) - 1;
    const int len = e - s + 1;
    const size_t plane = (size_t)p.nx * p.ny;
    const size_t base = (size_t)j * p.nx + (live ? i : 0);
    float2 dxy = f2(0.f, 0.f);
    if (live) dxy = cadd(p.dxs[i], p.dys[j]);

    auto diag = [dxy, p, nz](int l) {
        float2 b = cadd(dxy, p.cz[l]);
        if (l == 0 || l == nz - 1) b = cadd(b, p.gz);
        return b;
    };
    auto sub = [p, nz](int l) { return l == 0 ? 0.f : (l == nz - 1 ? p.zz : 1.f); };
    auto sup = [p, nz](int l) { return l == nz - 1 ? 0.f : (l == 0 ? p.zz : 1.f); };

    float2 y[MCH], bd[MCH];
#pragma unroll
    for (int k = 0; k < MCH; ++k)
        y[k] = (in && live && k < len) ? in[base + (size_t)(s + k) * plane] : f2(0.f, 0.f);
    if (p.P && live) {
#pragma unroll
        for (int k = 0; k < MCH; ++k)
            if (k < len) {
                const int l = s + k;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    y[k] = cadd(y[k], cmul(p.P[((size_t)t * nz + l) * p.ny + j], p.Q[((size_t)t * nz + l) * p.nx + i]));
            }
    }
#pragma unroll
    for (int k = 0; k < MCH; ++k) bd[k] = (k < len) ? diag(s + k) : f2(1.f, 0.f);
    float minpiv = 1e30f;
    auto piv = [&](float2 d) { minpiv = fminf(minpiv, fabsf(d.x) + fabsf(d.y)); };

    // down elimination with x_{s-1} as parameter: x_e = d' + l' x_{s-1} - c' x_{e+1}
    float2 cp = f2(0.f, 0.f), dp = f2(0.f, 0.f), lp = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < MCH; ++k) {
        if (k < len) {
            const int l = s + k;
            const float a = sub(l);
            const float2 den = (k == 0) ? bd[k] : csub(bd[k], cscale(cp, a));
            piv(den);
            const float2 ri = crcp(den);
            dp = cmul((k == 0) ? y[k] : csub(y[k], cscale(dp, a)), ri);
            lp = (k == 0) ? cscale(ri, -a) : cmul(cscale(lp, -a), ri);
            cp = cscale(ri, sup(l));
        }
    }
    // up elimination with x_{e+1} as parameter: x_s = dh - ch x_{s-1} + rh x_{e+1}
    float2 ch = f2(0.f, 0.f), dh = f2(0.f, 0.f), rh = f2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < MCH; ++kk) {
        const int k = MCH - 1 - kk;   // reverse order, written as a forward loop so it unrolls
        if (k < len) {
            const int l = s + k;
            const float c = sup(l);
            const bool first = (k == len - 1);
            const float2 den = first ? bd[k] : csub(bd[k], cscale(ch, c));
            piv(den);
            const float2 ri = crcp(den);
            dh = cmul(first ? y[k] : csub(y[k], cscale(dh, c)), ri);
            rh = first ? cscale(ri, -c) : cmul(cscale(rh, -c), ri);
            ch = cscale(ri, sub(l));
        }
    }
    sh[0][w][lane] = dh;                       // g_s
    sh[1][w][lane] = cscale(ch, -1.f);         // p_s (coefficient of x_{s-1})
    sh[2][w][lane] = rh;                       // q_s (coefficient of x_{e+1})
    sh[3][w][lane] = dp;                       // g_e
    sh[4][w][lane] = lp;                       // p_e
    sh[5][w][lane] = cscale(cp, -1.f);         // q_e
    __syncthreads();

    // interface system: X_c = (x_s, x_e) of chunk c,  X_c + A_c X_{c-1} + C_c X_{c+1} = G_c with
    // A_c = [[0, -p_s], [0, -p_e]] and C_c = [[-q_s, 0], [-q_e, 0]].  Block LU, one thread per line:
    // B_c = I - A_c Gamma_{c-1}, Y_c = B_c^-1 (G_c - A_c Y_{c-1}), Gamma_c = B_c^-1 C_c (first column only).
    if (w == 0) {
        float2 G1 = f2(0.f, 0.f), Y1 = f2(0.f, 0.f);
        for (int c = 0; c < W; ++c) {
            const float2 ps = sh[1][c][lane], qs = sh[2][c][lane], pe = sh[4][c][lane], qe = sh[5][c][lane];
            const float2 b00 = cadd(f2(1.f, 0.f), cmul(ps, G1));
            const float2 b10 = cmul(pe, G1);                 // B_c = [[b00, 0], [b10, 1]]
            const float2 r0 = cadd(sh[0][c][lane], cmul(ps, Y1));
            const float2 r1 = cadd(sh[3][c][lane], cmul(pe, Y1));
            piv(b00);
            const float2 y0 = qdiv(r0, b00);
            const float2 y1 = csub(r1, cmul(b10, y0));
            const float2 g0 = qdiv(cscale(qs, -1.f), b00);
            const float2 g1 = csub(cscale(qe, -1.f), cmul(b10, g0));
            sh[0][c][lane] = y0; sh[3][c][lane] = y1;
            sh[1][c][lane] = g0; sh[2][c][lane] = g1;
            G1 = g1; Y1 = y1;
        }
        float2 nxt = f2(0.f, 0.f);   // X_{c+1}[0]
        for (int c = W - 1; c >= 0; --c) {
            const float2 x0 = csub(sh[0][c][lane], cmul(sh[1][c][lane], nxt));
            const float2 x1 = csub(sh[3][c][lane], cmul(sh[2][c][lane], nxt));
            sh[0][c][lane] = x0; sh[3][c][lane] = x1;
            nxt = x0;
        }
    }
    __syncthreads();

    // finish the chunk by a Thomas sweep with known x_{s-1} (Lv) and x_{e+1} (Rv)
    const float2 Lv = w > 0 ? sh[3][w - 1][lane] : f2(0.f, 0.f);
    const float2 Rv = w < W - 1 ? sh[0][w + 1][lane] : f2(0.f, 0.f);
    float2 cpk[MCH];
    float2 c_prev = f2(0.f, 0.f), d_prev = Lv;
#pragma unroll
    for (int k = 0; k < MCH; ++k) {
        cpk[k] = f2(0.f, 0.f);
        if (k < len) {
            const int l = s + k;
            const float a = sub(l);
            const float2 den = (k == 0) ? bd[k] : csub(bd[k], cscale(c_prev, a));
            float2 rhs = csub(y[k], cscale(d_prev, a));
            const bool last = (k == len - 1);
            if (last) rhs = csub(rhs, cscale(Rv, sup(l)));
            const float2 ri = crcp(den);
            cpk[k] = cscale(ri, last ? 0.f : sup(l));
            y[k] = cmul(rhs, ri);
            c_prev = cpk[k];
            d_prev = y[k];
        }
    }
    float2 xn = f2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < MCH; ++kk) {
        const int k = MCH - 1 - kk;
        if (k < len) {
            xn = csub(y[k], cmul(cpk[k], xn));
            if (live) out[base + (size_t)(s + k) * plane] = xn;
        }
    }
    if (live && !(minpiv > 1e-30f)) atomicOr(status, (unsigned)HELM_DEV_PIVOT);
}

// ---- factorised z-solve (EigT) -------------------------------------------------------------------
// The systems of a context never change, so their Thomas factorisation is computed once at set-up:
//   m_l = 1 / (b_l - a_l c'_{l-1}),   c'_l = sup_l m_l,   (a_l, sup_l the sub- and super-diagonal)
// and stored per point (complex64).  An application is then one thread per line: forward
// d_l = (y_l - a_l d_{l-1}) m_l written over the output, backward x_l = d_l - sup_l m_l x_{l+1}, i.e.
// one complex product per step and sweep, no divisions, no interface system.  The backward sweep
// re-reads d and m soon after the forward sweep wrote/read them, mostly from L2.  Lines of consecutive
// x are consecutive threads, so every step is a contiguous row access.
constexpr int ZU = 8;   // steps whose loads are issued together

__global__ void __launch_bounds__(128) zfactor_kernel(ZParams p, float2* __restrict__ m, unsigned* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= p.nx) return;
    const size_t plane = (size_t)p.nx * p.ny, base = (size_t)j * p.nx + i;
    const float2 dxy = make_float2(__fadd_rn(p.dxs[i].x, p.dys[j].x), __fadd_rn(p.dxs[i].y, p.dys[j].y));
    float2 cprev = f2(0.f, 0.f);
    float minpiv = 1e30f;
    for (int l = 0; l < p.nz; ++l) {
        const float a = l == 0 ? 0.f : (l == p.nz - 1 ? p.zz : 1.f);
        const float sup = l == p.nz - 1 ? 0.f : (l == 0 ? p.zz : 1.f);
        float dm;
        const float2 mi = zpivot(dxy, p.cz[l], l == 0 || l == p.nz - 1, p.gz, a, sup, cprev, &dm);
        minpiv = fminf(minpiv, dm);
        m[base + (size_t)l * plane] = mi;
    }
    if (!(minpiv > 1e-30f)) atomicOr(status, (unsigned)HELM_DEV_PIVOT);
}

__global__ void __launch_bounds__(128) zsolve_fact_kernel(int nx, int ny, int nz, float zz, const float2* __restrict__ m,
                                                         const float2* in, float2* out, const float2* __restrict__ P,
                                                         const float2* __restrict__ Q) {
    // blockIdx.y = (right-hand side of a batch group) * ny + j; the factors m are shared
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y % ny, vb = blockIdx.y / ny;
    if (i >= nx) return;
    const size_t plane = (size_t)nx * ny, base = (size_t)j * nx + i, voff = (size_t)vb * plane * nz;
    if (vb) {
        if (in) in += voff;
        out += voff;
    }
    float2 d = f2(0.f, 0.f);
    for (int l0 = 0; l0 < nz; l0 += ZU) {
        float2 yv[ZU], mv[ZU];
#pragma unroll
        for (int u = 0; u < ZU; ++u)
            if (l0 + u < nz) {
                yv[u] = in ? in[base + (size_t)(l0 + u) * plane] : f2(0.f, 0.f);
                mv[u] = m[base + (size_t)(l0 + u) * plane];
            }
        if (P) {
            // generated right-hand side: y[l][j][i] += sum_{t<4} P[t][l][j] Q[t][l][i]
#pragma unroll
            for (int u = 0; u < ZU; ++u) {
                const int l = l0 + u;
                if (l < nz) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        yv[u] = cadd(yv[u], cmul(P[((size_t)t * nz + l) * ny + j], Q[((size_t)t * nz + l) * nx + i]));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < ZU; ++u) {
            const int l = l0 + u;
            if (l < nz) {
                const float a = l == 0 ? 0.f : (l == nz - 1 ? zz : 1.f);
                d = zfwd(yv[u], d, a, mv[u]);
                out[base + (size_t)l * plane] = d;
            }
        }
    }
    float2 x = f2(0.f, 0.f);
    for (int l1 = nz; l1 > 0; l1 -= ZU) {
        float2 dv[ZU], mv[ZU];
#pragma unroll
        for (int u = 0; u < ZU; ++u) {
            const int l = l1 - 1 - u;
            if (l >= 0) {
                dv[u] = out[base + (size_t)l * plane];
                mv[u] = m[base + (size_t)l * plane];
            }
        }
#pragma unroll
        for (int u = 0; u < ZU; ++u) {
            const int l = l1 - 1 - u;
            if (l >= 0) {
                const float sup = l == nz - 1 ? 0.f : (l == 0 ? zz : 1.f);
                x = zbwd(dv[u], mv[u], x, sup);
                out[base + (size_t)l * plane] = x;
            }
        }
    }
}

// Factorised solve, L2-resident form (no generated right-hand side, even N_x).  The backward sweep reads
// d and m again; when every line runs at once those re-reads (16 B/pt) miss the L2, so here a persistent
// grid of a few 64-thread CTAs per SM keeps about 20k-40k lines in flight (their d and m stay in L2) and
// walks the rest in turn.  Each thread takes two adjacent lines (16-byte accesses) and streams its inputs
// through a private ring of ZB blocks of ZU steps in shared memory by cp.async (one group per block, no
// block barrier); a landed block is read into registers at once and its ZU dependent steps then run back
// to back, so the shared-memory latency is paid once per block rather than once per step.
constexpr int ZRT = 64, ZU2 = 8, ZB = 4;
constexpr size_t ZRING_BYTES = (size_t)ZB * ZU2 * 2 * ZRT * sizeof(float4);   // 64 KiB

__device__ __forceinline__ void zcp16(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void zcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void zwait_ring() { asm volatile("cp.async.wait_group %0;\n" ::"n"(ZB - 1) : "memory"); }
__device__ __forceinline__ void zwait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// nb > 1: nb right-hand side grids back to back (a batch group), sharing the factors m
__global__ void __launch_bounds__(ZRT) zsolve_ring_kernel(int nx, int ny, int nz, float zz,
                                                         const float4* __restrict__ m, const float4* in, float4* out,
                                                         int nb) {
    extern __shared__ float4 zring[];   // [ZB * ZU2][2][ZRT]
    const int tid = threadIdx.x;
    const int hx = nx / 2, npairs = hx * ny;
    const int nblk = (nz + ZU2 - 1) / ZU2;
    const size_t plane = (size_t)hx * ny;   // in float4 (two lines) units
    auto slot = [&](int st, int a) -> float4* { return &zring[((size_t)st * 2 + a) * ZRT + tid]; };
    for (int prb = blockIdx.x * ZRT + tid; prb < npairs * nb; prb += gridDim.x * ZRT) {
        const int pr = prb % npairs, vb = prb / npairs;
        const size_t off = (size_t)pr;   // pair pr = (j, i/2) is float4 pr of every plane
        const size_t voff = (size_t)vb * plane * nz;   // this right-hand side's grid (the factors are shared)
        // ---- forward: d_l = (y_l - a_l d_{l-1}) m_l, steps in increasing l
        auto fetch_f = [&](int b) {
            if (b < nblk) {
#pragma unroll
                for (int u = 0; u < ZU2; ++u) {
                    const int l = b * ZU2 + u;
                    if (l < nz) {
                        zcp16(slot((b % ZB) * ZU2 + u, 0), in + voff + off + (size_t)l * plane);
                        zcp16(slot((b % ZB) * ZU2 + u, 1), m + off + (size_t)l * plane);
                    }
                }
            }
            zcommit();
        };
        for (int b = 0; b < ZB - 1; ++b) fetch_f(b);
        float2 d0 = f2(0.f, 0.f), d1 = d0;
        for (int b = 0; b < nblk; ++b) {
            fetch_f(b + ZB - 1);
            zwait_ring();   // block b has landed
            float4 y[ZU2], mm[ZU2];
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                y[u] = *slot((b % ZB) * ZU2 + u, 0);
                mm[u] = *slot((b % ZB) * ZU2 + u, 1);
            }
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                const int l = b * ZU2 + u;
                if (l < nz) {
                    const float a = l == 0 ? 0.f : (l == nz - 1 ? zz : 1.f);
                    d0 = zfwd(f2(y[u].x, y[u].y), d0, a, f2(mm[u].x, mm[u].y));
                    d1 = zfwd(f2(y[u].z, y[u].w), d1, a, f2(mm[u].z, mm[u].w));
                    out[voff + off + (size_t)l * plane] = make_float4(d0.x, d0.y, d1.x, d1.y);
                }
            }
        }
        zwait_all();
        __threadfence_block();
        // ---- backward: x_l = d_l - s_l m_l x_{l+1}, steps in decreasing l (block b holds l = nz-1-(b ZU2 + u))
        auto fetch_b = [&](int b) {
            if (b < nblk) {
#pragma unroll
                for (int u = 0; u < ZU2; ++u) {
                    const int l = nz - 1 - (b * ZU2 + u);
                    if (l >= 0) {
                        zcp16(slot((b % ZB) * ZU2 + u, 0), out + voff + off + (size_t)l * plane);
                        zcp16(slot((b % ZB) * ZU2 + u, 1), m + off + (size_t)l * plane);
                    }
                }
            }
            zcommit();
        };
        for (int b = 0; b < ZB - 1; ++b) fetch_b(b);
        float2 x0 = f2(0.f, 0.f), x1 = x0;
        for (int b = 0; b < nblk; ++b) {
            fetch_b(b + ZB - 1);
            zwait_ring();
            float4 dv[ZU2], mm[ZU2];
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                dv[u] = *slot((b % ZB) * ZU2 + u, 0);
                mm[u] = *slot((b % ZB) * ZU2 + u, 1);
            }
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                const int l = nz - 1 - (b * ZU2 + u);
                if (l >= 0) {
                    const float sup = l == nz - 1 ? 0.f : (l == 0 ? zz : 1.f);
                    x0 = zbwd(f2(dv[u].x, dv[u].y), f2(mm[u].x, mm[u].y), x0, sup);
                    x1 = zbwd(f2(dv[u].z, dv[u].w), f2(mm[u].z, mm[u].w), x1, sup);
                    out[voff + off + (size_t)l * plane] = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
            }
        }
        zwait_all();
    }
}

// EigT form without the factor stream: the pivots depend only on the line's lateral shift
// s_ij = alpha_x d_{x,i} + alpha_y d_{y,j} and the plane, so the forward sweep recomputes them step by step
// (the same operations as zfactor_kernel, one reciprocal per step) and saves the recurrence's state
// c'_{l-1} at the start of every block of ZU2 steps to a small scratch (2 bytes per point, [block][pair]
// so that a warp's saves are one contiguous row); the backward sweep recomputes the ZU2 factors of a block
// forward from its checkpoint into registers and then runs the block backwards.  HBM sees y read, the
// forward values written over the output and read back (mostly from L2), and x written: the 8 bytes per
// point of factors and their L2 footprint are gone.  A grid is one thread per pair of lines (32k threads
// at 256^3, three to four 64-thread CTAs per SM), so latency is hidden by prefetch depth: a six-block ring
// per thread (48 steps ahead, 48 KiB per CTA), and each backward block's checkpoint is loaded one block
// ahead of its use.
constexpr int ZPB = 6;   // ring depth (blocks) of the pivot-recomputing kernel
constexpr size_t ZPIV_SMEM = (size_t)ZPB * ZU2 * ZRT * sizeof(float4);   // 48 KiB
__device__ __forceinline__ void zwait_piv() { asm volatile("cp.async.wait_group %0;\n" ::"n"(ZPB - 1) : "memory"); }

__device__ __forceinline__ void zcp8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// a pair of lines' complex values from / to four 16-bit values (memory order re0, im0, re1, im1), H = 1 BF16,
// 2 FP16 (clamped to the finite range); widening is exact
template <int H>
__device__ __forceinline__ float4 h4_to_f4(uint2 w) {
    if (H == 2) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xFFFF0000u), __uint_as_float(w.y << 16),
                       __uint_as_float(w.y & 0xFFFF0000u));
}
template <int H>
__device__ __forceinline__ uint32_t zpack16(float lo, float hi) {
    if (H == 2) {
        const __half2 v = __floats2half2_rn(fminf(fmaxf(lo, -65504.f), 65504.f), fminf(fmaxf(hi, -65504.f), 65504.f));
        return *reinterpret_cast<const uint32_t*>(&v);
    }
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// H (1 BF16, 2 FP16): y read and x written (times oscale) in 16 bits (uint2 per line pair), the forward
// values d kept in FP32 in dscr (a complex64-sized grid of the caller); H = 0: float4 in and out and
// dscr = out (d over the output).
template <int H>
__global__ void __launch_bounds__(ZRT, 4) zsolve_piv_kernel(int nx, int ny, int nz, float zz, float2 gz,
                                                           const float2* __restrict__ dxs,
                                                           const float2* __restrict__ dys,
                                                           const float2* __restrict__ cz, const void* inv, void* outv,
                                                           float4* dscr, float4* __restrict__ ck, int nb,
                                                           float oscale = 1.f, double* __restrict__ h16d = nullptr,
                                                           float gain = 1.f) {
    constexpr bool BF = H != 0;
    // FP16 chain with dynamic stage scales (h16d): the output scale from the bound of ||T2|| (h16d[1]),
    // recorded in h16d[5]; the squared norm of what is stored accumulates into h16d[2]
    float nacc = 0.f;
    if (BF && h16d) {
        const double n2 = h16d[1];
        float sc = 1.f;
        if (n2 > 0.0) {
            int e = 15 - (int)ceil(log2((double)gain * sqrt(n2)));
            e = e < -100 ? -100 : (e > 100 ? 100 : e);
            sc = ldexpf(1.f, e);
        }
        oscale *= sc;
        if (blockIdx.x == 0 && threadIdx.x == 0) h16d[5] = sc;
    }
    extern __shared__ float4 zsm[];   // [ZPB * ZU2][ZRT]
    const float4* in = reinterpret_cast<const float4*>(inv);
    const uint2* inb = reinterpret_cast<const uint2*>(inv);
    float4* out = BF ? dscr : reinterpret_cast<float4*>(outv);   // where d goes (and comes back from)
    uint2* outb = reinterpret_cast<uint2*>(outv);
    const int tid = threadIdx.x;
    const int hx = nx / 2, npairs = hx * ny, nall = npairs * nb;
    const int nblk = (nz + ZU2 - 1) / ZU2;
    const size_t plane = (size_t)hx * ny;   // in float4 (two lines) units
    auto slot = [&](int st) -> float4* { return &zsm[(size_t)st * ZRT + tid]; };
    for (int prb = blockIdx.x * ZRT + tid; prb < nall; prb += gridDim.x * ZRT) {
        const int pr = prb % npairs, vb = prb / npairs;
        const int j = pr / hx, i0 = 2 * (pr - j * hx);
        const float2 s0 = make_float2(__fadd_rn(dxs[i0].x, dys[j].x), __fadd_rn(dxs[i0].y, dys[j].y));
        const float2 s1 = make_float2(__fadd_rn(dxs[i0 + 1].x, dys[j].x), __fadd_rn(dxs[i0 + 1].y, dys[j].y));
        const size_t off = (size_t)pr, voff = (size_t)vb * plane * nz;
        // block blk of src (steps l = blk ZU2 + u) into ring position pos
        auto fetch = [&](const float4* src, int blk, int pos) {
            if (blk >= 0 && blk < nblk) {
#pragma unroll
                for (int u = 0; u < ZU2; ++u) {
                    const int l = blk * ZU2 + u;
                    if (l < nz) zcp16(slot((pos % ZPB) * ZU2 + u), src + voff + off + (size_t)l * plane);
                }
            }
            zcommit();
        };
        // the same for the BF16 input (8 bytes per step into the first half of a slot)
        auto fetch_in = [&](int blk, int pos) {
            if (!BF) { fetch(in, blk, pos); return; }
            if (blk >= 0 && blk < nblk) {
#pragma unroll
                for (int u = 0; u < ZU2; ++u) {
                    const int l = blk * ZU2 + u;
                    if (l < nz) zcp8(slot((pos % ZPB) * ZU2 + u), inb + voff + off + (size_t)l * plane);
                }
            }
            zcommit();
        };
        // one pivot step of both lines: m_l and the new c'_l from c'_{l-1}
        auto pivots = [&](int l, float2& c0, float2& c1, float2& m0, float2& m1) {
            const float a = l == 0 ? 0.f : (l == nz - 1 ? zz : 1.f);
            const float sup = l == nz - 1 ? 0.f : (l == 0 ? zz : 1.f);
            const float2 czl = cz[l];
            const bool end = l == 0 || l == nz - 1;
            m0 = zpivot(s0, czl, end, gz, a, sup, c0);
            m1 = zpivot(s1, czl, end, gz, a, sup, c1);
        };
        // ---- forward: d_l = (y_l - a_l d_{l-1}) m_l
        for (int b = 0; b < ZPB - 1; ++b) fetch_in(b, b);
        float2 d0 = f2(0.f, 0.f), d1 = d0, c0 = d0, c1 = d0;
        for (int b = 0; b < nblk; ++b) {
            fetch_in(b + ZPB - 1, b + ZPB - 1);
            zwait_piv();   // block b has landed
            ck[(size_t)b * nall + prb] = make_float4(c0.x, c0.y, c1.x, c1.y);
            float4 y[ZU2];
#pragma unroll
            for (int u = 0; u < ZU2; ++u)
                y[u] = BF ? h4_to_f4<H>(*reinterpret_cast<const uint2*>(slot((b % ZPB) * ZU2 + u)))
                          : *slot((b % ZPB) * ZU2 + u);
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                const int l = b * ZU2 + u;
                if (l < nz) {
                    const float a = l == 0 ? 0.f : (l == nz - 1 ? zz : 1.f);
                    float2 m0, m1;
                    pivots(l, c0, c1, m0, m1);
                    d0 = zfwd(f2(y[u].x, y[u].y), d0, a, m0);
                    d1 = zfwd(f2(y[u].z, y[u].w), d1, a, m1);
                    out[voff + off + (size_t)l * plane] = make_float4(d0.x, d0.y, d1.x, d1.y);
                }
            }
        }
        zwait_all();
        __threadfence_block();
        // ---- backward: x_l = d_l - sup_l m_l x_{l+1}, blocks in decreasing order
        for (int b = 0; b < ZPB - 1; ++b) fetch(out, nblk - 1 - b, b);
        float2 x0 = f2(0.f, 0.f), x1 = x0;
        float4 cnext = ck[(size_t)(nblk - 1) * nall + prb];
        for (int b = 0; b < nblk; ++b) {
            fetch(out, nblk - 1 - (b + ZPB - 1), b + ZPB - 1);
            const int blk = nblk - 1 - b;
            const float4 cv = cnext;
            if (blk > 0) cnext = ck[(size_t)(blk - 1) * nall + prb];   // the next block's checkpoint, early
            float2 cc0 = f2(cv.x, cv.y), cc1 = f2(cv.z, cv.w);
            float2 m0[ZU2], m1[ZU2];
#pragma unroll
            for (int u = 0; u < ZU2; ++u) {
                const int l = blk * ZU2 + u;
                m0[u] = m1[u] = f2(0.f, 0.f);
                if (l < nz) pivots(l, cc0, cc1, m0[u], m1[u]);
            }
            zwait_piv();
#pragma unroll
            for (int uu = 0; uu < ZU2; ++uu) {
                const int u = ZU2 - 1 - uu, l = blk * ZU2 + u;
                if (l < nz) {
                    const float4 dv = *slot((b % ZPB) * ZU2 + u);
                    const float sup = l == nz - 1 ? 0.f : (l == 0 ? zz : 1.f);
                    x0 = zbwd(f2(dv.x, dv.y), m0[u], x0, sup);
                    x1 = zbwd(f2(dv.z, dv.w), m1[u], x1, sup);
                    if (BF) {
                        const float a = oscale * x0.x, b2 = oscale * x0.y, c2 = oscale * x1.x, d2 = oscale * x1.y;
                        outb[voff + off + (size_t)l * plane] = make_uint2(zpack16<H>(a, b2), zpack16<H>(c2, d2));
                        nacc = fmaf(a, a, fmaf(b2, b2, fmaf(c2, c2, fmaf(d2, d2, nacc))));
                    }
                    else out[voff + off + (size_t)l * plane] = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
            }
        }
        zwait_all();
    }
    if (BF && h16d) {
        double d = (double)nacc;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(h16d + 2, d);
    }
}

}  // namespace

// Set-up: the Thomas factors of the z-systems with lateral eigenvalue shifts dxs_i + dys_j (one complex64
// per point) into *m (allocated here if NULL).
helm_status zsolve_factor_with(helm_ctx* c, const float2* dxs, const float2* dys, float2** m, cudaStream_t s) {
    if (!*m) {
        if (cudaMalloc(m, c->npts * sizeof(float2)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    }
    if (!c->zring_sms) {   // the ring kernel of the factorised solve: shared memory and grid size
        HELM_CUDA_TRY(cudaFuncSetAttribute(zsolve_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)ZRING_BYTES));
        HELM_CUDA_TRY(cudaDeviceGetAttribute(&c->zring_sms, cudaDevAttrMultiProcessorCount, c->device));
    }
    ZParams p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.dxs = dxs; p.dys = dys; p.cz = c->cz;
    p.P = nullptr; p.Q = nullptr;
    p.gz = make_float2((float)c->gam[2].x, (float)c->gam[2].y);
    p.zz = (float)c->zeta[2];
    dim3 grid((c->nx + 127) / 128, c->ny);
    zfactor_kernel<<<grid, 128, 0, s>>>(p, *m, c->status_d);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status zsolve_factor(helm_ctx* c, cudaStream_t s) { return zsolve_factor_with(c, c->dxs, c->dys, &c->zfac, s); }

// factorised solve with factors m, optional input (NULL = 0) and optional generated right-hand side
helm_status launch_zsolve_fact(helm_ctx* c, const float2* m, const float2* in, float2* out, const float2* P,
                               const float2* Q, cudaStream_t s, int nb) {
    prof_begin(c, s, PROF_ZSOLVE);
    if (!P && in && c->nx % 2 == 0 && c->tune_zring && c->zring_sms > 0) {
        const int sms = c->zring_sms;
        const int npairs = c->nx / 2 * c->ny * nb;
        const int need = (npairs + ZRT - 1) / ZRT;
        const int grid = need < sms * c->tune_zring ? need : sms * c->tune_zring;
        zsolve_ring_kernel<<<grid, ZRT, ZRING_BYTES, s>>>(c->nx, c->ny, c->nz, (float)c->zeta[2],
                                                         reinterpret_cast<const float4*>(m),
                                                         reinterpret_cast<const float4*>(in), reinterpret_cast<float4*>(out),
                                                         nb);
        prof_end(c, s);
        HELM_CUDA_TRY(cudaGetLastError());
        return HELM_OK;
    }
    dim3 grid((c->nx + 127) / 128, c->ny * nb);
    zsolve_fact_kernel<<<grid, 128, 0, s>>>(c->nx, c->ny, c->nz, (float)c->zeta[2], m, in, out, P, Q);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status launch_zsolve_gen(helm_ctx* c, const float2* in, float2* out, const float2* dxs, const float2* dys,
                              const float2* P, const float2* Q, cudaStream_t s) {
    ZParams p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
    p.dxs = dxs; p.dys = dys; p.cz = c->cz;
    p.P = P; p.Q = Q;
    p.gz = make_float2((float)c->gam[2].x, (float)c->gam[2].y);
    p.zz = (float)c->zeta[2];
    if (c->nz > 512) return HELM_ERR_UNSUPPORTED;
    prof_begin(c, s, PROF_ZSOLVE);
    if (c->nz <= 256) {
        p.W = (c->nz + 7) / 8;
        dim3 grid((c->nx + 15) / 16, c->ny), block(16, p.W);
        zsolve_kernel<16, 8><<<grid, block, 0, s>>>(p, in, out, c->status_d);
    } else {
        p.W = (c->nz + 15) / 16;
        dim3 grid((c->nx + 15) / 16, c->ny), block(16, p.W);
        zsolve_kernel<16, 16><<<grid, block, 0, s>>>(p, in, out, c->status_d);
    }
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

size_t zsolve_ck_bytes(const helm_ctx* c, int nb) {
    return (size_t)((c->nz + ZU2 - 1) / ZU2) * (size_t)(c->nx / 2) * c->ny * nb * sizeof(float4);
}

// the pivot checkpoints of nb right-hand sides per z-solve launch (device memory of the context)
helm_status zsolve_reserve(helm_ctx* c, int nb) {
    const size_t bytes = zsolve_ck_bytes(c, nb);
    if (bytes <= c->zck_bytes) return HELM_OK;
    cudaFree(c->zck);
    c->zck = nullptr;
    c->zck_bytes = 0;
    if (cudaMalloc(&c->zck, bytes) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    c->zck_bytes = bytes;
    return HELM_OK;
}

helm_status launch_zsolve(helm_ctx* c, const float2* in, float2* out, cudaStream_t s, int nb) {
    if (!c->zfac) {
        helm_status st;
        for (int v = 0; v < nb; ++v)
            if ((st = launch_zsolve_gen(c, in + (size_t)v * c->npts, out + (size_t)v * c->npts, c->dxs, c->dys, nullptr,
                                        nullptr, s)) != HELM_OK)
                return st;
        return HELM_OK;
    }
    if (in && c->nx % 2 == 0 && c->tune_zring && c->zring_sms > 0 && !c->zpiv_off) {
        // EigT: pivots recomputed from the shifts (the set-up factors' operations), checkpoints in a scratch
        // of the context (grown here outside stream capture; a capturing caller reserves it beforehand)
        // (c->zck_slot: the first checkpoint slot of this launch; concurrent solves of one context in a batch
        // plan each capture with their own slots)
        const int npairs = c->nx / 2 * c->ny * nb;
        const int slot = c->zck_slot;
        if (zsolve_ck_bytes(c, slot + nb) > c->zck_bytes) {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            HELM_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
            if (cap != cudaStreamCaptureStatusNone) return launch_zsolve_fact(c, c->zfac, in, out, nullptr, nullptr, s, nb);
            helm_status st;
            if ((st = zsolve_reserve(c, slot + nb)) != HELM_OK) return st;
        }
        if (!(c->zpiv_ready & 1)) {
            HELM_CUDA_TRY(cudaFuncSetAttribute(zsolve_piv_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)ZPIV_SMEM));
            c->zpiv_ready |= 1;
        }
        prof_begin(c, s, PROF_ZSOLVE);
        const int sms = c->zring_sms;
        const int need = (npairs + ZRT - 1) / ZRT;
        const int cap = sms * 2 * c->tune_zring;   // tune_zring 1..3: 2, 4 or 6 CTAs per SM (at most 4 resident)
        const int grid = need < cap ? need : cap;
        zsolve_piv_kernel<0><<<grid, ZRT, ZPIV_SMEM, s>>>(c->nx, c->ny, c->nz, (float)c->zeta[2],
                                                               make_float2((float)c->gam[2].x, (float)c->gam[2].y), c->dxs,
                                                               c->dys, c->cz, in, out, reinterpret_cast<float4*>(out),
                                                               reinterpret_cast<float4*>(c->zck) + (size_t)slot * zsolve_ck_bytes(c, 1) / sizeof(float4),
                                                               nb);
        prof_end(c, s);
        HELM_CUDA_TRY(cudaGetLastError());
        return HELM_OK;
    }
    return launch_zsolve_fact(c, c->zfac, in, out, nullptr, nullptr, s, nb);
}

// The z-solves of the 16-bit transform chain (HELM_PREC_BF16, HELM_PREC_FP16): the pivot-recomputing kernel
// with 16-bit y and x (in may equal out; x scaled by oscale) and the FP32 forward values in dscr (npts * nb
// complex64 of the caller).  No fallback: a launch under stream capture without reserved checkpoints
// returns HELM_ERR_UNSUPPORTED.
helm_status launch_zsolve_h16(helm_ctx* c, const void* in, void* out, float4* dscr, float oscale, cudaStream_t s, int nb,
                              double* h16d, float gain) {
    const int H = c->opt.precision == HELM_PREC_FP16 ? 2 : 1;
    if (c->nx % 2 != 0 || c->zring_sms <= 0) return HELM_ERR_UNSUPPORTED;
    const int slot = c->zck_slot;
    if (zsolve_ck_bytes(c, slot + nb) > c->zck_bytes) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        HELM_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
        if (cap != cudaStreamCaptureStatusNone) return HELM_ERR_UNSUPPORTED;
        helm_status st;
        if ((st = zsolve_reserve(c, slot + nb)) != HELM_OK) return st;
    }
    if (!(c->zpiv_ready & (2 << (H - 1)))) {
        if (H == 2)
            HELM_CUDA_TRY(cudaFuncSetAttribute(zsolve_piv_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZPIV_SMEM));
        else
            HELM_CUDA_TRY(cudaFuncSetAttribute(zsolve_piv_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZPIV_SMEM));
        c->zpiv_ready |= 2 << (H - 1);
    }
    prof_begin(c, s, PROF_ZSOLVE);
    const int npairs = c->nx / 2 * c->ny * nb;
    const int need = (npairs + ZRT - 1) / ZRT;
    const int cap = c->zring_sms * 2 * (c->tune_zring > 0 ? c->tune_zring : 1);
    const int grid = need < cap ? need : cap;
    float4* ck = reinterpret_cast<float4*>(c->zck) + (size_t)slot * zsolve_ck_bytes(c, 1) / sizeof(float4);
    const float2 gz = make_float2((float)c->gam[2].x, (float)c->gam[2].y);
    if (H == 2)
        zsolve_piv_kernel<2><<<grid, ZRT, ZPIV_SMEM, s>>>(c->nx, c->ny, c->nz, (float)c->zeta[2], gz, c->dxs, c->dys, c->cz,
                                                           in, out, dscr, ck, nb, oscale, h16d, gain);
    else
        zsolve_piv_kernel<1><<<grid, ZRT, ZPIV_SMEM, s>>>(c->nx, c->ny, c->nz, (float)c->zeta[2], gz, c->dxs, c->dys, c->cz,
                                                           in, out, dscr, ck, nb, oscale);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
