// Restarted right-preconditioned GMRES(m) and flexible GMRES on the device (Sec. 5: the paper uses
// right-preconditioned restarted GMRES after Saad [s]; the flexible form is Saad's Alg. 9.6).
//
// Per inner step j:  z_j = M^-1 v_j  ->  w = A z_j  ->  h_{i,j} = v_i^H w, w -= sum h_{i,j} v_i (classical
// Gram-Schmidt, optionally twice)  ->  h_{j+1,j} = ||w||, Givens rotation, residual estimate |g_{j+1}|.
// Krylov vectors are complex64; inner products are accumulated in FP64; H, the rotations and g are FP64
// on the device.  Normalisation is lazy: the stored vector is w and v_{j+1} = sigma_{j+1} w with
// sigma_{j+1} = 1/h_{j+1,j}; sigma is folded into the consumers (preconditioner input, inner products,
// updates), which saves one pass over the grid per step.
// The iterate x is complex128.  Each cycle ends with the FP64 true residual r = F - A x (Sec. 5.1 rel-res),
// which decides convergence and seeds the next cycle.
#include "common.cuh"
#include <cuda_fp16.h>
#include "dfloat.cuh"
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

int residual_ctas(const helm_ctx* c);

struct Ctrl {
    double beta0;   // ||F - A x0||
    double beta;    // ||F - A x|| at the last true residual
    double est;     // |g_{j+1}| / beta0
    double hnext;   // h_{j+1,j}
    double rmax;    // ||F - A x||_inf
    int flags;      // HELM_DEV_* bits
    int pad;
};

// Inner tolerance of a restart cycle (iterative refinement with a low-precision inner solve).  The Krylov
// vectors and the stencil are complex64, so a cycle lowers the true residual by at most about 1e-5
// relative to the residual it started from (the stencil's rounding, amplified by its cancellation at ~10
// points per wavelength), while the GMRES estimate keeps falling.  Each cycle therefore stops once its
// estimate, relative to the cycle's starting residual beta_k, reaches kInnerFloor, and the next cycle
// restarts from the double-float true residual.  kInnerFloor = 1e-4 rather than the floor itself: shorter
// cycles also keep the Gram-Schmidt work (which grows with the cycle's length) low; measured on the 20-bump
// and single-inclusion media from 100^3 to 400^3, 1e-4 gave the shortest solves of 1e-5 ... 1e-2.
// In terms of est = |g_{j+1}| / beta_0: stop when est <= max(rtol, kInnerFloor * beta_k / beta_0).
constexpr double kInnerFloor = 1e-4;
__host__ __device__ inline double inner_threshold(double rtol, double beta_k, double beta0, double floor = kInnerFloor) {
    const double f = beta0 > 0 ? floor * beta_k / beta0 : 0.0;
    return rtol > f ? rtol : f;
}
// The FP16 Krylov basis (HELM_PREC_FP16, flexible single solves) holds each basis vector to 2^-11 relative,
// so the Arnoldi relation itself is exact only to a few 1e-4 and a cycle cannot lower the residual by
// 1e-4 reliably; its cycles stop at 1e-3 (measured on the 20-bump medium: the FP16 basis then needs no more
// inner iterations than the complex64 one at 128^3, two more with 1e-4 cycles).
constexpr double kInnerFloorH16 = 1e-3;

struct KrylovWork {
    int m = 0, flexible = 0, NB = 0, nres = 0;
    int NBd = 0;             // CTAs of the inner-product kernel: one full wave of resident CTAs
    size_t npts = 0;
    size_t vs = 0;           // distance between consecutive basis vectors of V and Z (npts unless interleaved)
    int shared = 0;          // V, Z and sigma belong to a batch group (interleaved with its other lanes)
    float2* V = nullptr;     // (m+1) stored vectors
    float2* Z = nullptr;     // m preconditioned vectors (flexible) or one scratch vector
    double* sigma = nullptr; // [m+1]
    double2* H = nullptr;    // (m+1) x m, column-major
    double* cs = nullptr;    // [m]
    double2* sn = nullptr;   // [m]
    double2* g = nullptr;    // [m+1]
    double2* y = nullptr;    // [m]
    double2* part = nullptr; // [NB][m+1]
    double* rpart = nullptr; // [2*nres]
    float2* coef = nullptr;  // [m+1]
    Ctrl* ctrl_d = nullptr;
    Ctrl* ctrl_h = nullptr;  // pinned
    double2* xbuf = nullptr; // device copy of x when the caller passes host memory
    double2* bbuf = nullptr;
    float4* xdf = nullptr;   // the iterate in double-float (re.hi, im.hi, re.lo, im.lo)
    float4* Fdf = nullptr;   // the right-hand side in double-float
    unsigned* nzflag = nullptr;
    Ctrl* slots_h = nullptr;         // pinned [m]: the controls after each iteration of a cycle
    cudaEvent_t* ev_slot = nullptr;  // [m]: recorded after each slot's copy
    // FP16 basis: v_i = c16[i] V16_i, V16 (m+1) FP16 grids of 2 npts halves; w16s = s0 / ||w|| of the step
    uint16_t* V16 = nullptr;
    double* c16 = nullptr;           // [m+1]
    double* w16s = nullptr;          // [1]
    int db_ready = 0;                // shared-memory attribute of the staged inner-product kernel set
    // the Givens step of the FP16-basis solve on a side stream: ev_upd[j] after the update of step j (main
    // stream), ev_giv[j] after its Givens step (side stream), which the next step joins before the last pass
    // of its preconditioner
    cudaStream_t side = nullptr;
    cudaEvent_t* ev_upd = nullptr;
    cudaEvent_t* ev_giv = nullptr;
};

namespace {

constexpr int NT = 256;
constexpr int GRP = 8;
// smallest one-step reduction of the GMRES residual estimate assumed by the look-ahead of the solve loop
constexpr double kLookaheadDrop = 0.05;

// partial inner products conj(v_i) . w for i in [0, nv); part[blk * ld + i].
// Two points per 16-byte load, two loads of each vector in flight per thread; per-thread sums are
// compensated FP32 (Kahan), FP64 only across threads (GB300's FP64 rate made FP64 partial sums the
// limiter).  npts is even.
__device__ __forceinline__ void dots_body(const float2* __restrict__ V, size_t npts, int nv,
                                          const float2* __restrict__ w, double2* __restrict__ part, int ld, size_t vs) {
    __shared__ double2 red[NT / 32][GRP];
    const int tid = threadIdx.x;
    const size_t n4 = npts / 2;
    const size_t stride = (size_t)gridDim.x * NT;
    const float4* __restrict__ W4 = reinterpret_cast<const float4*>(w);
    for (int g0 = 0; g0 < nv; g0 += GRP) {
        const int ng = min(GRP, nv - g0);
        // compensated (Kahan) FP32 sums per thread; FP64 only for the cross-thread reduction
        float2 ks[GRP], kc[GRP];
#pragma unroll
        for (int q = 0; q < GRP; ++q) { ks[q] = make_float2(0, 0); kc[q] = make_float2(0, 0); }
        for (size_t id = blockIdx.x * (size_t)NT + tid; id < n4; id += 2 * stride) {
            const size_t id2 = id + stride;
            const bool two = id2 < n4;
            const float4 wa = W4[id];
            const float4 wb = two ? W4[id2] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < GRP; ++q)
                if (q < ng) {
                    const float4* __restrict__ V4 = reinterpret_cast<const float4*>(V + (size_t)(g0 + q) * vs);
                    const float4 va = V4[id];
                    const float4 vb = two ? V4[id2] : make_float4(0.f, 0.f, 0.f, 0.f);
                    float re = va.x * wa.x, im = va.x * wa.y;
                    re = fmaf(va.y, wa.y, re);
                    im = fmaf(-va.y, wa.x, im);
                    re = fmaf(va.z, wa.z, fmaf(va.w, wa.w, re));
                    im = fmaf(va.z, wa.w, fmaf(-va.w, wa.z, im));
                    re = fmaf(vb.x, wb.x, fmaf(vb.y, wb.y, re));
                    im = fmaf(vb.x, wb.y, fmaf(-vb.y, wb.x, im));
                    re = fmaf(vb.z, wb.z, fmaf(vb.w, wb.w, re));
                    im = fmaf(vb.z, wb.w, fmaf(-vb.w, wb.z, im));
                    float y = re - kc[q].x, t = ks[q].x + y;
                    kc[q].x = (t - ks[q].x) - y; ks[q].x = t;
                    y = im - kc[q].y; t = ks[q].y + y;
                    kc[q].y = (t - ks[q].y) - y; ks[q].y = t;
                }
        }
        double2 acc[GRP];
#pragma unroll
        for (int q = 0; q < GRP; ++q) {
            acc[q] = make_double2((double)ks[q].x - (double)kc[q].x, (double)ks[q].y - (double)kc[q].y);
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, o);
            }
        }
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q < GRP; ++q) red[tid >> 5][q] = acc[q];
        __syncthreads();
        if (tid < ng) {
            double2 s = make_double2(0, 0);
            for (int wi = 0; wi < NT / 32; ++wi) { s.x += red[wi][tid].x; s.y += red[wi][tid].y; }
            part[(size_t)blockIdx.x * ld + g0 + tid] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(NT) dots_kernel(const float2* __restrict__ V, size_t npts, int nv,
                                                 const float2* __restrict__ w, double2* __restrict__ part, int ld,
                                                 size_t vs) {
    dots_body(V, npts, nv, w, part, ld, vs);
}

// Software-pipelined variant: groups of G basis vectors, one 16-byte load per vector and thread per
// iteration, and the next iteration's loads issued before this iteration's compensated sums, so every
// warp keeps two iterations of loads in flight instead of waiting a full memory latency per iteration.
template <int G>
__device__ __forceinline__ void dots_pipe_body(const float2* __restrict__ V, size_t npts, int nv,
                                               const float2* __restrict__ w, double2* __restrict__ part, int ld,
                                               size_t vs) {
    __shared__ double2 red[NT / 32][G];
    const int tid = threadIdx.x;
    const size_t n4 = npts / 2;
    const size_t stride = (size_t)gridDim.x * NT;
    const float4* __restrict__ W4 = reinterpret_cast<const float4*>(w);
    for (int g0 = 0; g0 < nv; g0 += G) {
        const int ng = min(G, nv - g0);
        float2 ks[G], kc[G];
        const float4* __restrict__ V4[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            ks[q] = make_float2(0, 0);
            kc[q] = make_float2(0, 0);
            V4[q] = reinterpret_cast<const float4*>(V + (size_t)(g0 + (q < ng ? q : 0)) * vs);
        }
        size_t id = blockIdx.x * (size_t)NT + tid;
        float4 wa = make_float4(0.f, 0.f, 0.f, 0.f), va[G];
        if (id < n4) {
            wa = W4[id];
#pragma unroll
            for (int q = 0; q < G; ++q) va[q] = q < ng ? V4[q][id] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (; id < n4; id += stride) {
            const size_t nid = id + stride;
            float4 wb = make_float4(0.f, 0.f, 0.f, 0.f), vb[G];
#pragma unroll
            for (int q = 0; q < G; ++q) vb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nid < n4) {
                wb = W4[nid];
#pragma unroll
                for (int q = 0; q < G; ++q)
                    if (q < ng) vb[q] = V4[q][nid];
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const float4 a = va[q];
                float re = a.x * wa.x, im = a.x * wa.y;
                re = fmaf(a.y, wa.y, re);
                im = fmaf(-a.y, wa.x, im);
                re = fmaf(a.z, wa.z, fmaf(a.w, wa.w, re));
                im = fmaf(a.z, wa.w, fmaf(-a.w, wa.z, im));
                float y = re - kc[q].x, t = ks[q].x + y;
                kc[q].x = (t - ks[q].x) - y; ks[q].x = t;
                y = im - kc[q].y; t = ks[q].y + y;
                kc[q].y = (t - ks[q].y) - y; ks[q].y = t;
            }
            wa = wb;
#pragma unroll
            for (int q = 0; q < G; ++q) va[q] = vb[q];
        }
        double2 acc[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            acc[q] = make_double2((double)ks[q].x - (double)kc[q].x, (double)ks[q].y - (double)kc[q].y);
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, o);
            }
        }
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q < G; ++q) red[tid >> 5][q] = acc[q];
        __syncthreads();
        if (tid < ng) {
            double2 sum = make_double2(0, 0);
            for (int wi = 0; wi < NT / 32; ++wi) { sum.x += red[wi][tid].x; sum.y += red[wi][tid].y; }
            part[(size_t)blockIdx.x * ld + g0 + tid] = sum;
        }
        __syncthreads();
    }
}

template <int G>
__global__ void __launch_bounds__(NT) dots_pipe_kernel(const float2* __restrict__ V, size_t npts, int nv,
                                                      const float2* __restrict__ w, double2* __restrict__ part, int ld,
                                                      size_t vs) {
    dots_pipe_body<G>(V, npts, nv, w, part, ld, vs);
}

// one block per basis vector i: h_i = sigma_i * sum over blocks of the partial products, coef_i = sigma_i h_i
__device__ __forceinline__ void reduce_h_body(const double2* __restrict__ part, int NB, int ld, int nv,
                                              const double* __restrict__ sigma, double2* __restrict__ Hcol,
                                              float2* __restrict__ coef, int first_pass) {
    __shared__ double rx[32], ry[32];
    const int i = blockIdx.x;
    if (i >= nv) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double sx = 0, sy = 0;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) {
        const double2 v = part[(size_t)b * ld + i];
        sx += v.x;
        sy += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) { rx[wid] = sx; ry[wid] = sy; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    sx = 0;
    sy = 0;
    for (int w = 0; w < nw; ++w) { sx += rx[w]; sy += ry[w]; }
    const double sg = sigma[i];
    const double2 h = make_double2(sx * sg, sy * sg);
    Hcol[i] = first_pass ? h : cadd(Hcol[i], h);
    coef[i] = make_float2((float)(h.x * sg), (float)(h.y * sg));
}
__global__ void reduce_h_kernel(const double2* __restrict__ part, int NB, int ld, int nv, const double* __restrict__ sigma,
                                double2* __restrict__ Hcol, float2* __restrict__ coef, int first_pass) {
    reduce_h_body(part, NB, ld, nv, sigma, Hcol, coef, first_pass);
}

// w -= sum_i coef_i V_i (i < nv); per-block partial ||w||^2 in part[blk * ld].x.  Two points per
// 16-byte load; the basis loop is unrolled by four so that four vector loads are in flight.
__device__ __forceinline__ void update_body(const float2* __restrict__ V, size_t npts, int nv,
                                            const float2* __restrict__ coef, float2* __restrict__ w,
                                            double2* __restrict__ part, int ld, size_t vs) {
    __shared__ float2 cf[72];
    __shared__ double red[NT / 32];
    for (int i = threadIdx.x; i < nv; i += NT) cf[i] = coef[i];
    __syncthreads();
    float fs = 0.f, fc = 0.f;   // per-thread compensated FP32 sum of |w|^2 (FP64 only across threads)
    const size_t n4 = npts / 2;
    float4* W4 = reinterpret_cast<float4*>(w);
    for (size_t id = blockIdx.x * (size_t)NT + threadIdx.x; id < n4; id += (size_t)gridDim.x * NT) {
        float4 x = W4[id];
        int i = 0;
        for (; i + 4 <= nv; i += 4) {
            float4 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = reinterpret_cast<const float4*>(V + (size_t)(i + q) * vs)[id];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 c = cf[i + q];
                x.x -= c.x * v[q].x - c.y * v[q].y;
                x.y -= c.x * v[q].y + c.y * v[q].x;
                x.z -= c.x * v[q].z - c.y * v[q].w;
                x.w -= c.x * v[q].w + c.y * v[q].z;
            }
        }
        for (; i < nv; ++i) {
            const float4 v = reinterpret_cast<const float4*>(V + (size_t)i * vs)[id];
            const float2 c = cf[i];
            x.x -= c.x * v.x - c.y * v.y;
            x.y -= c.x * v.y + c.y * v.x;
            x.z -= c.x * v.z - c.y * v.w;
            x.w -= c.x * v.w + c.y * v.z;
        }
        W4[id] = x;
        kahan_add(fs, fc, fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, x.w * x.w))));
    }
    double acc = (double)fs - (double)fc;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int wi = 0; wi < NT / 32; ++wi) s += red[wi];
        part[(size_t)blockIdx.x * ld] = make_double2(s, 0.0);
    }
}
__global__ void __launch_bounds__(NT) update_kernel(const float2* __restrict__ V, size_t npts, int nv,
                                                   const float2* __restrict__ coef, float2* __restrict__ w,
                                                   double2* __restrict__ part, int ld, size_t vs) {
    update_body(V, npts, nv, coef, w, part, ld, vs);
}

// ---- FP16 Krylov basis (HELM_PREC_FP16, flexible single solves) ------------------------------------
// v_i = c16[i] V16_i with V16_i an FP16 grid (two complex points per 8-byte load); w stays complex64.
// Inner products conj(V16_i) . w for i < nv and ||w||^2 (slot nv of part) in one pass.  Packed f32x2
// arithmetic: with v = (vr, vi) and the broadcast pairs (wr, wr), (wi, wi) of the point (formed once per
// point for all G vectors), P += v (wr, wr) and Q += v (wi, wi) per vector, and at the end
// conj(v) w = (P.x + Q.y, Q.x - P.y): two FMA2 per vector and point.  Plain FP32 sums per thread (a basis
// held to 2^-11 needs no compensation), FP64 across threads.
__device__ __forceinline__ float2 h2f(uint32_t u) { return __half22float2(*reinterpret_cast<const __half2*>(&u)); }
template <int G>
__global__ void __launch_bounds__(NT) dots16_kernel(const uint16_t* __restrict__ V16, size_t npts, int nv,
                                                   const float2* __restrict__ w, double2* __restrict__ part, int ld) {
    __shared__ double2 red[NT / 32][G + 1];
    const int tid = threadIdx.x;
    const size_t n4 = npts / 2;
    const size_t stride = (size_t)gridDim.x * NT;
    const float4* __restrict__ W4 = reinterpret_cast<const float4*>(w);
    for (int g0 = 0; g0 < nv; g0 += G) {
        const int ng = min(G, nv - g0);
        const bool first = g0 == 0;
        float2 P[G], Q[G];
        float2 nn = make_float2(0.f, 0.f);   // ||w||^2 (first group)
        const uint2* __restrict__ V2[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            P[q] = make_float2(0.f, 0.f);
            Q[q] = make_float2(0.f, 0.f);
            V2[q] = reinterpret_cast<const uint2*>(V16 + (size_t)(g0 + (q < ng ? q : 0)) * 2 * npts);
        }
        size_t id = blockIdx.x * (size_t)NT + tid;
        float4 wa = make_float4(0.f, 0.f, 0.f, 0.f);
        uint2 va[G];
#pragma unroll
        for (int q = 0; q < G; ++q) va[q] = make_uint2(0u, 0u);
        if (id < n4) {
            wa = W4[id];
#pragma unroll
            for (int q = 0; q < G; ++q) if (q < ng) va[q] = V2[q][id];
        }
        for (; id < n4; id += stride) {
            const size_t nid = id + stride;
            float4 wb = make_float4(0.f, 0.f, 0.f, 0.f);
            uint2 vb[G];
#pragma unroll
            for (int q = 0; q < G; ++q) vb[q] = make_uint2(0u, 0u);
            if (nid < n4) {
                wb = W4[nid];
#pragma unroll
                for (int q = 0; q < G; ++q)
                    if (q < ng) vb[q] = V2[q][nid];
            }
            const float2 r0 = bc2(wa.x), i0 = bc2(wa.y), r1 = bc2(wa.z), i1 = bc2(wa.w);
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const float2 v0 = h2f(va[q].x), v1 = h2f(va[q].y);
                P[q] = fma2(v1, r1, fma2(v0, r0, P[q]));
                Q[q] = fma2(v1, i1, fma2(v0, i0, Q[q]));
            }
            if (first) nn = fma2(make_float2(wa.z, wa.w), make_float2(wa.z, wa.w), fma2(make_float2(wa.x, wa.y), make_float2(wa.x, wa.y), nn));
            wa = wb;
#pragma unroll
            for (int q = 0; q < G; ++q) va[q] = vb[q];
        }
        double2 acc[G + 1];
#pragma unroll
        for (int q = 0; q < G; ++q) acc[q] = make_double2((double)P[q].x + (double)Q[q].y, (double)Q[q].x - (double)P[q].y);
        acc[G] = make_double2((double)nn.x + (double)nn.y, 0.0);
#pragma unroll
        for (int q = 0; q <= G; ++q)
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, o);
            }
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q <= G; ++q) red[tid >> 5][q] = acc[q];
        __syncthreads();
        if (tid < ng || (first && tid == G)) {
            double2 sum = make_double2(0, 0);
            for (int wi = 0; wi < NT / 32; ++wi) { sum.x += red[wi][tid].x; sum.y += red[wi][tid].y; }
            part[(size_t)blockIdx.x * ld + (tid == G ? nv : g0 + tid)] = sum;
        }
        __syncthreads();
    }
}
// Staged form (nv + 1 <= 32): one CTA per SM walks chunks of T points; a producer warp copies w (8 B/pt) and
// the nv basis chunks (4 B/pt each) of a chunk into a three-stage shared-memory ring with bulk copies
// (cp.async.bulk, completion by mbarrier transaction count), so the bytes in flight per SM (up to three
// 64 KiB stages) do not depend on registers; eight consumer warps take the nv inner products and ||w||^2
// (item nv) by item (warp k: items k, k + 8, ...), two FMA2 per point and item as above, FP32 per chunk and
// FP64 across chunks.  Every wait is bounded by wlim (HELM_DEV_WAIT on expiry); the producer waits for the
// copies it issued before the CTA exits.
constexpr int DB_NS = 3, DB_CW = 8, DB_NT = (DB_CW + 1) * 32;
constexpr int DB_STAGE = 64 * 1024;
constexpr size_t DB_SMEM = (size_t)DB_NS * DB_STAGE;
constexpr long DB_DRAIN = 1L << 22;
__device__ __forceinline__ uint32_t db_su(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool db_wait(uint32_t bar, uint32_t parity, long limit) {
    for (long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void db_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__global__ void __launch_bounds__(DB_NT, 1) dots16b_kernel(const uint16_t* __restrict__ V16, size_t npts, int nv,
                                                          const float2* __restrict__ w, double2* __restrict__ part,
                                                          int ld, int T, unsigned* status, long wlim) {
    extern __shared__ __align__(128) unsigned char dbs[];
    __shared__ __align__(8) uint64_t full[DB_NS], empty[DB_NS];
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long nch = (long)((npts + T - 1) / T);
    const long mine = nch > blockIdx.x ? (nch - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // chunks of this CTA
    if (threadIdx.x == 0) {
        for (int q = 0; q < DB_NS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(db_su(&full[q])), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(db_su(&empty[q])), "r"(DB_CW) : "memory");
        }
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool ok = true;
    if (warp == DB_CW) {   // producer
        long issued = 0;
        if (lane == 0) {
            for (long k = 0; k < mine && ok; ++k) {
                const int q = (int)(k % DB_NS);
                if (k >= DB_NS) ok = db_wait(db_su(&empty[q]), (uint32_t)(((k / DB_NS) - 1) & 1), wlim);
                if (!ok) break;
                const size_t start = (size_t)(blockIdx.x + k * gridDim.x) * T;
                const uint32_t cnt = (uint32_t)min((size_t)T, npts - start);
                const uint32_t base = db_su(dbs + (size_t)q * DB_STAGE);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(db_su(&full[q])),
                             "r"(cnt * 8u + (uint32_t)nv * cnt * 4u) : "memory");
                db_bulk(base, w + start, cnt * 8u, db_su(&full[q]));
                for (int i = 0; i < nv; ++i)
                    db_bulk(base + (uint32_t)T * 8u + (uint32_t)i * T * 4u, V16 + (size_t)i * 2 * npts + 2 * start, cnt * 4u,
                            db_su(&full[q]));
                ++issued;
            }
            if (!ok) {
                atomicOr(status, (unsigned)HELM_DEV_WAIT);
                fail = 1;
            }
            // the copies in flight land before the CTA leaves (the consumers may have stopped waiting)
            for (long k = issued > DB_NS ? issued - DB_NS : 0; k < issued; ++k)
                db_wait(db_su(&full[k % DB_NS]), (uint32_t)((k / DB_NS) & 1), DB_DRAIN);
        }
    } else {               // consumers: items warp, warp + 8, ... (< nv + 1)
        double2 acc[4];
        for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
        for (long k = 0; k < mine && ok; ++k) {
            const int q = (int)(k % DB_NS);
            ok = __all_sync(0xffffffffu, db_wait(db_su(&full[q]), (uint32_t)((k / DB_NS) & 1), wlim));
            if (!ok) break;
            const size_t start = (size_t)(blockIdx.x + k * gridDim.x) * T;
            const int cnt = (int)min((size_t)T, npts - start);
            const float2* sw = reinterpret_cast<const float2*>(dbs + (size_t)q * DB_STAGE);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = warp + u * DB_CW;
                if (i > nv) break;
                float2 P = make_float2(0.f, 0.f), Q = P;
                if (i < nv) {
                    const uint32_t* sv = reinterpret_cast<const uint32_t*>(dbs + (size_t)q * DB_STAGE + (size_t)T * 8 +
                                                                           (size_t)i * T * 4);
                    for (int p = lane; p < cnt; p += 32) {
                        const float2 wv = sw[p], v = h2f(sv[p]);
                        P = fma2(v, bc2(wv.x), P);
                        Q = fma2(v, bc2(wv.y), Q);
                    }
                    acc[u].x += (double)P.x + (double)Q.y;
                    acc[u].y += (double)Q.x - (double)P.y;
                } else {
                    for (int p = lane; p < cnt; p += 32) {
                        const float2 wv = sw[p];
                        P = fma2(wv, wv, P);
                    }
                    acc[u].x += (double)P.x + (double)P.y;
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(db_su(&empty[q])) : "memory");
        }
        if (!ok && lane == 0) {
            atomicOr(status, (unsigned)HELM_DEV_WAIT);
            fail = 1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = warp + u * DB_CW;
            for (int o = 16; o > 0; o >>= 1) {
                acc[u].x += __shfl_down_sync(0xffffffffu, acc[u].x, o);
                acc[u].y += __shfl_down_sync(0xffffffffu, acc[u].y, o);
            }
            if (lane == 0 && i <= nv) part[(size_t)blockIdx.x * ld + i] = acc[u];
        }
    }
    __syncthreads();
}

// blocks i < nv: h_i = c16[i] sum_b part[b][i], coef_i = c16[i] h_i; block nv: w16s = s0 / ||w||
__global__ void reduce16_kernel(const double2* __restrict__ part, int NB, int ld, int nv, const double* __restrict__ c16,
                                double2* __restrict__ Hcol, float2* __restrict__ coef, float s0, double* __restrict__ w16s) {
    __shared__ double rx[32], ry[32];
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double sx = 0, sy = 0;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) {
        const double2 v = part[(size_t)b * ld + i];
        sx += v.x;
        sy += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) { rx[wid] = sx; ry[wid] = sy; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    sx = 0;
    sy = 0;
    for (int w = 0; w < nw; ++w) { sx += rx[w]; sy += ry[w]; }
    if (i == nv) {
        const double nr = sqrt(sx);
        w16s[0] = nr > 0.0 ? (double)s0 / nr : 0.0;
        return;
    }
    const double cg = c16[i];
    const double2 h = make_double2(sx * cg, sy * cg);
    Hcol[i] = h;
    coef[i] = make_float2((float)(h.x * cg), (float)(h.y * cg));
}
// V16_out = FP16(w16s (w - sum_i coef_i V16_i)) (clamped to the finite range; ||.||_F <= s0 since the
// projection does not lengthen w); per-block partial ||w - sum||^2 in part[blk * ld].x.  Packed form: with
// the broadcast pairs (cr, cr), (ci, ci) of each coefficient (staged in shared memory), T1 += v (cr, cr),
// T2 += v (ci, ci), and sum coef_i v_i = (T1.x - T2.y, T1.y + T2.x).
__global__ void __launch_bounds__(NT) update16_kernel(const uint16_t* __restrict__ V16, size_t npts, int nv,
                                                     const float2* __restrict__ coef, const float2* __restrict__ w,
                                                     uint16_t* __restrict__ Vout, const double* __restrict__ w16s,
                                                     double2* __restrict__ part, int ld) {
    __shared__ float4 cf[72];   // (cr, cr, ci, ci)
    __shared__ double red[NT / 32];
    for (int i = threadIdx.x; i < nv; i += NT) cf[i] = make_float4(coef[i].x, coef[i].x, coef[i].y, coef[i].y);
    __syncthreads();
    const float sc = (float)w16s[0];
    float2 nn = make_float2(0.f, 0.f);
    const size_t n4 = npts / 2;
    const float4* W4 = reinterpret_cast<const float4*>(w);
    uint2* O2 = reinterpret_cast<uint2*>(Vout);
    for (size_t id = blockIdx.x * (size_t)NT + threadIdx.x; id < n4; id += (size_t)gridDim.x * NT) {
        const float4 x = W4[id];
        float2 A0 = make_float2(0.f, 0.f), B0 = A0, A1 = A0, B1 = A0;   // T1, T2 of the two points
        int i = 0;
        for (; i + 4 <= nv; i += 4) {
            uint2 u[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) u[q] = reinterpret_cast<const uint2*>(V16 + (size_t)(i + q) * 2 * npts)[id];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 c = cf[i + q];
                const float2 v0 = h2f(u[q].x), v1 = h2f(u[q].y);
                A0 = fma2(v0, make_float2(c.x, c.y), A0);
                B0 = fma2(v0, make_float2(c.z, c.w), B0);
                A1 = fma2(v1, make_float2(c.x, c.y), A1);
                B1 = fma2(v1, make_float2(c.z, c.w), B1);
            }
        }
        for (; i < nv; ++i) {
            const uint2 u = reinterpret_cast<const uint2*>(V16 + (size_t)i * 2 * npts)[id];
            const float4 c = cf[i];
            const float2 v0 = h2f(u.x), v1 = h2f(u.y);
            A0 = fma2(v0, make_float2(c.x, c.y), A0);
            B0 = fma2(v0, make_float2(c.z, c.w), B0);
            A1 = fma2(v1, make_float2(c.x, c.y), A1);
            B1 = fma2(v1, make_float2(c.z, c.w), B1);
        }
        const float2 y0 = make_float2(x.x - (A0.x - B0.y), x.y - (A0.y + B0.x));
        const float2 y1 = make_float2(x.z - (A1.x - B1.y), x.w - (A1.y + B1.x));
        const __half2 a = __floats2half2_rn(fminf(fmaxf(sc * y0.x, -65504.f), 65504.f), fminf(fmaxf(sc * y0.y, -65504.f), 65504.f));
        const __half2 b = __floats2half2_rn(fminf(fmaxf(sc * y1.x, -65504.f), 65504.f), fminf(fmaxf(sc * y1.y, -65504.f), 65504.f));
        O2[id] = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
        nn = fma2(y1, y1, fma2(y0, y0, nn));
    }
    double acc = (double)nn.x + (double)nn.y;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        for (int wi = 0; wi < NT / 32; ++wi) sum += red[wi];
        part[(size_t)blockIdx.x * ld] = make_double2(sum, 0.0);
    }
}
// c16[j] = sigma[j] / w16s (v_j = sigma_j (w - sum) = c16[j] V16_j); j = 0 (a restart): c16[0] = 1 / s0
__global__ void c16_kernel(const double* __restrict__ sigma, int j, const double* __restrict__ w16s, double* c16, float s0) {
    if (threadIdx.x == 0) c16[j] = j == 0 ? 1.0 / (double)s0 : (w16s[0] > 0.0 ? sigma[j] / w16s[0] : 0.0);
}

__device__ inline void givens(double2 a, double2 b, double& c, double2& s) {
    const double ab = hypot(b.x, b.y);
    if (ab == 0.0) { c = 1.0; s = make_double2(0, 0); return; }
    const double aa = hypot(a.x, a.y);
    if (aa == 0.0) { c = 0.0; s = make_double2(b.x / ab, -b.y / ab); return; }
    const double t = hypot(aa, ab);
    c = aa / t;
    const double2 ph = make_double2(a.x / aa, a.y / aa);          // a/|a|
    s = cmul(ph, make_double2(b.x / t, -b.y / t));                // (a/|a|) conj(b)/t
}

// Finish column j: h_{j+1,j} from the partial norms, previous rotations, the new rotation, g, est.  The
// column and the previous rotations are staged in shared memory by the whole block; one thread then
// applies the rotations.
__device__ __forceinline__ void givens_body(const double2* __restrict__ part, int NB, int ld, int j, int m, double2* H,
                                            double* cs, double2* sn, double2* g, double* sigma, Ctrl* ctrl) {
    __shared__ double red[32];
    __shared__ double2 col[72], snv[72];
    __shared__ double csv[72];
    double2* hcol = H + (size_t)j * (m + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) { csv[i] = cs[i]; snv[i] = sn[i]; }
    for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = hcol[i];
    double s = 0;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) s += part[(size_t)b * ld].x;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const double hn = sqrt(tot);
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        const double2 t = cadd(cscale(a, csv[i]), cmul(snv[i], b));
        const double2 snc = make_double2(snv[i].x, -snv[i].y);
        col[i + 1] = csub(cscale(b, csv[i]), cmul(snc, a));
        col[i] = t;
    }
    double c;
    double2 sj;
    givens(col[j], col[j + 1], c, sj);
    cs[j] = c;
    sn[j] = sj;
    col[j] = cadd(cscale(col[j], c), cmul(sj, col[j + 1]));
    for (int i = 0; i <= j; ++i) hcol[i] = col[i];
    hcol[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    g[j + 1] = cscale(cmul(make_double2(sj.x, -sj.y), gj), -1.0);
    g[j] = cscale(gj, c);
    sigma[j + 1] = hn > 0 ? 1.0 / hn : 0.0;
    const double est = hypot(g[j + 1].x, g[j + 1].y) / ctrl->beta0;
    ctrl->est = est;
    ctrl->hnext = hn;
    if (!isfinite(hn) || !isfinite(est) || !isfinite(col[j].x) || !isfinite(col[j].y)) ctrl->flags |= HELM_DEV_NAN;
}
// (with the FP16 basis also c16[j+1] = sigma_{j+1} / w16s, the scale of V16_{j+1}: one thread after the body)
__global__ void givens_kernel(const double2* __restrict__ part, int NB, int ld, int j, int m, double2* H, double* cs,
                              double2* sn, double2* g, double* sigma, Ctrl* ctrl, const double* w16s = nullptr,
                              double* c16 = nullptr) {
    givens_body(part, NB, ld, j, m, H, cs, sn, g, sigma, ctrl);
    if (c16 && threadIdx.x == 0) {
        __threadfence_block();
        c16[j + 1] = w16s[0] > 0.0 ? sigma[j + 1] / w16s[0] : 0.0;
    }
}

// y = R^-1 g (k x k upper triangular part of the rotated H)
__global__ void lsq_kernel(const double2* __restrict__ H, const double2* __restrict__ g, int k, int m, double2* y,
                           Ctrl* ctrl, const int* __restrict__ kdev) {
    if (threadIdx.x != 0) return;
    if (kdev) k = *kdev;
    for (int i = k - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int q = i + 1; q < k; ++q) s = csub(s, cmul(H[(size_t)q * (m + 1) + i], y[q]));
        y[i] = cdiv(s, H[(size_t)i * (m + 1) + i]);
        if (!isfinite(y[i].x) || !isfinite(y[i].y)) ctrl->flags |= HELM_DEV_NAN;
    }
}

// flexible: x += sum_i y_i Z_i.  The cycle's correction is summed in FP32 (each y_i rounded to complex64), two
// points per 16-byte load, and added to the double-float iterate once per point.  Its rounding error, a few
// units of 2^-24 of the correction, perturbs the next true residual by about 1e-6 of the residual this cycle
// removed, far below the 1e-4 a cycle lowers it by; the next cycle starts from the exact (double-float)
// residual of the iterate, so the error is corrected like any other (iterative refinement).
__global__ void __launch_bounds__(NT) combine_flex_kernel(const float2* __restrict__ Z, size_t npts, int k,
                                                         const double2* __restrict__ y, float4* __restrict__ x,
                                                         const int* __restrict__ kdev, size_t vs) {
    __shared__ float2 ys[64];
    if (kdev) k = *kdev;
    for (int i = threadIdx.x; i < k; i += NT) ys[i] = make_float2((float)y[i].x, (float)y[i].y);
    __syncthreads();
    const size_t n2 = npts / 2;
    for (size_t id = blockIdx.x * (size_t)NT + threadIdx.x; id < n2; id += (size_t)gridDim.x * NT) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        int i = 0;
        auto term = [&](const float2 c, const float4 z) {
            a.x = fmaf(c.x, z.x, fmaf(-c.y, z.y, a.x));
            a.y = fmaf(c.x, z.y, fmaf(c.y, z.x, a.y));
            a.z = fmaf(c.x, z.z, fmaf(-c.y, z.w, a.z));
            a.w = fmaf(c.x, z.w, fmaf(c.y, z.z, a.w));
        };
        for (; i + 4 <= k; i += 4) {   // four loads in flight
            float4 zv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) zv[q] = reinterpret_cast<const float4*>(Z + (size_t)(i + q) * vs)[id];
#pragma unroll
            for (int q = 0; q < 4; ++q) term(ys[i + q], zv[q]);
        }
        for (; i < k; ++i) term(ys[i], reinterpret_cast<const float4*>(Z + (size_t)i * vs)[id]);
        x[2 * id] = cdf_to4(cdf_add(cdf_from4(x[2 * id]), cdf_from_f2(make_float2(a.x, a.y))));
        x[2 * id + 1] = cdf_to4(cdf_add(cdf_from4(x[2 * id + 1]), cdf_from_f2(make_float2(a.z, a.w))));
    }
}

// right-preconditioned: u = sum_i (y_i sigma_i) V_i  (complex64; u is a complex64 preconditioner input)
__global__ void __launch_bounds__(NT) combine_v_kernel(const float2* __restrict__ V, size_t npts, int k,
                                                      const double2* __restrict__ y, const double* __restrict__ sigma,
                                                      float2* __restrict__ u, const int* __restrict__ kdev, size_t vs) {
    __shared__ float2 ys[64];
    if (kdev) k = *kdev;
    for (int i = threadIdx.x; i < k; i += NT) {
        const double2 v = cscale(y[i], sigma[i]);
        ys[i] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    for (size_t id = blockIdx.x * (size_t)NT + threadIdx.x; id < npts; id += (size_t)gridDim.x * NT) {
        float2 a = make_float2(0.f, 0.f);
        for (int i = 0; i < k; ++i) a = cfma(ys[i], V[(size_t)i * vs + id], a);
        u[id] = a;
    }
}

// x += z in double-float
__global__ void add_kernel(const float2* __restrict__ z, float4* __restrict__ x, size_t npts) {
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < npts; id += (size_t)gridDim.x * blockDim.x) {
        const float2 v = z[id];
        x[id] = cdf_to4(cdf_add(cdf_from4(x[id]), cdf_from_f2(v)));
    }
}

// FP64 -> double-float; flags a nonzero entry of a (used to recognise x0 = 0)
// The conversions stream 32 bytes per point; four independent loads per thread keep enough bytes in flight.
__global__ void to_df_kernel(const double2* __restrict__ a, float4* __restrict__ b, size_t npts, unsigned* nz) {
    unsigned any = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t id0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id0 < npts; id0 += 4 * stride) {
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t id = id0 + u * stride;
            v[u] = id < npts ? a[id] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t id = id0 + u * stride;
            if (id < npts) {
                b[id] = split4_bits(v[u]);
                // nonzero test on the patterns (+-0 have only the sign bit)
                any |= ((((unsigned long long)__double_as_longlong(v[u].x)) << 1) |
                        (((unsigned long long)__double_as_longlong(v[u].y)) << 1)) != 0ull;
            }
        }
    }
    if (nz && __any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(nz, 1u);
}
__global__ void from_df_kernel(const float4* __restrict__ a, double2* __restrict__ b, size_t npts) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t id0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id0 < npts; id0 += 4 * stride) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t id = id0 + u * stride;
            v[u] = id < npts ? a[id] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t id = id0 + u * stride;
            if (id < npts) b[id] = df4_to_double2(v[u]);
        }
    }
}

// r = F (x = 0): complex64 copy of F with the residual partials of the stencil form
__global__ void __launch_bounds__(NT) residual_zero_kernel(const float4* __restrict__ F, float2* __restrict__ r,
                                                          size_t npts, double* __restrict__ part) {
    __shared__ double rs[NT / 32], rm[NT / 32];
    float fs = 0.f, fc = 0.f, fm = 0.f;   // per-thread compensated FP32 sum and max of |r|^2; FP64 across threads
    for (size_t id = blockIdx.x * (size_t)NT + threadIdx.x; id < npts; id += (size_t)gridDim.x * NT) {
        const float2 v = cdf_round(cdf_from4(F[id]));
        r[id] = v;
        const float a2 = fmaf(v.x, v.x, v.y * v.y);
        kahan_add(fs, fc, a2);
        fm = fmaxf(fm, a2);
    }
    double s = (double)fs - (double)fc, mx = (double)fm;
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = s; rm[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ss = 0, m = 0;
        for (int w = 0; w < NT / 32; ++w) { ss += rs[w]; m = fmax(m, rm[w]); }
        part[2 * blockIdx.x] = ss;
        part[2 * blockIdx.x + 1] = sqrt(m);
    }
}

// beta = ||r||_2, rmax = ||r||_inf from the residual partials; sigma_0 = 1/beta, g = (beta, 0, ...)
__global__ void resnorm_kernel(const double* __restrict__ rpart, int n, double* sigma, double2* g, int m, Ctrl* ctrl,
                               int first) {
    __shared__ double rs[32], rm[32];
    double s = 0, mx = 0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) { s += rpart[2 * b]; mx = fmax(mx, rpart[2 * b + 1]); }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = s; rm[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot = 0, mm = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tot += rs[w]; mm = fmax(mm, rm[w]); }
    const double beta = sqrt(tot);
    ctrl->beta = beta;
    ctrl->rmax = mm;
    if (first) { ctrl->beta0 = beta; ctrl->flags = 0; }
    if (!isfinite(beta)) ctrl->flags |= HELM_DEV_NAN;
    sigma[0] = beta > 0 ? 1.0 / beta : 0.0;
    g[0] = make_double2(beta, 0.0);
    for (int i = 1; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked, mapped host memory (cudaHostAlloc / registered), else NULL: kernels
// then read the caller's vector over the host link directly instead of staging it with a copy first.
void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void free_work(KrylovWork* k) {
    if (!k->shared) { cudaFree(k->V); cudaFree(k->Z); cudaFree(k->sigma); }
    cudaFree(k->H); cudaFree(k->cs); cudaFree(k->sn);
    cudaFree(k->g); cudaFree(k->y); cudaFree(k->part); cudaFree(k->rpart); cudaFree(k->coef); cudaFree(k->ctrl_d);
    cudaFreeHost(k->ctrl_h); cudaFree(k->xbuf); cudaFree(k->bbuf); cudaFree(k->xdf); cudaFree(k->Fdf);
    cudaFree(k->nzflag);
    cudaFree(k->V16); cudaFree(k->c16); cudaFree(k->w16s);
    cudaFreeHost(k->slots_h);
    if (k->ev_slot) {
        for (int j = 0; j < k->m; ++j)
            if (k->ev_slot[j]) cudaEventDestroy(k->ev_slot[j]);
        delete[] k->ev_slot;
    }
    for (cudaEvent_t* ev : {k->ev_upd, k->ev_giv})
        if (ev) {
            for (int j = 0; j < k->m; ++j)
                if (ev[j]) cudaEventDestroy(ev[j]);
            delete[] ev;
        }
    if (k->side) cudaStreamDestroy(k->side);
}

int dots_ctas(const helm_ctx* c);
int launch_dots(const helm_ctx* c, const float2* V, size_t npts, int nv, const float2* w, double2* part, int ld,
                int nbd, cudaStream_t s, size_t vs = 0);

// Krylov workspace of restart length m for the context's grid; NB = CTAs of the Arnoldi kernels.
// Vs, Zs, sigs (optional, all three or none): the lane's share of a batch group's interleaved basis (vector
// stride vs), preconditioned vectors and normalisation factors, which the group owns.
helm_status alloc_work(helm_ctx* c, KrylovWork* k, int m, int flex, int NB, float2* Vs = nullptr, float2* Zs = nullptr,
                       double* sigs = nullptr, size_t vs = 0) {
    k->m = m; k->flexible = flex; k->npts = c->npts; k->vs = vs ? vs : c->npts;
    k->NB = NB;
    k->NBd = dots_ctas(c);
    k->nres = residual_ctas(c);
    const size_t vb = c->npts * sizeof(float2);
    if (Vs) {
        k->shared = 1;
        k->V = Vs;
        k->Z = Zs;
        k->sigma = sigs;
    } else {
        if (cudaMalloc(&k->V, vb * (m + 1)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
        if (cudaMalloc(&k->Z, vb * (flex ? m : 1)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
        HELM_CUDA_TRY(cudaMalloc(&k->sigma, sizeof(double) * (m + 1)));
    }
    HELM_CUDA_TRY(cudaMalloc(&k->H, sizeof(double2) * (m + 1) * m));
    HELM_CUDA_TRY(cudaMalloc(&k->cs, sizeof(double) * m));
    HELM_CUDA_TRY(cudaMalloc(&k->sn, sizeof(double2) * m));
    HELM_CUDA_TRY(cudaMalloc(&k->g, sizeof(double2) * (m + 1)));
    HELM_CUDA_TRY(cudaMalloc(&k->y, sizeof(double2) * m));
    HELM_CUDA_TRY(cudaMalloc(&k->part, sizeof(double2) * (size_t)std::max(k->NB, k->NBd) * (m + 1)));
    HELM_CUDA_TRY(cudaMalloc(&k->rpart, sizeof(double) * 2 * k->nres));
    HELM_CUDA_TRY(cudaMalloc(&k->coef, sizeof(float2) * (m + 1)));
    HELM_CUDA_TRY(cudaMalloc(&k->ctrl_d, sizeof(Ctrl)));
    HELM_CUDA_TRY(cudaMallocHost(&k->ctrl_h, sizeof(Ctrl)));
    if (cudaMalloc(&k->xdf, c->npts * sizeof(float4)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    if (cudaMalloc(&k->Fdf, c->npts * sizeof(float4)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    HELM_CUDA_TRY(cudaMalloc(&k->nzflag, sizeof(unsigned)));
    HELM_CUDA_TRY(cudaMemset(k->H, 0, sizeof(double2) * (m + 1) * m));
    HELM_CUDA_TRY(cudaMemset(k->ctrl_d, 0, sizeof(Ctrl)));
    return HELM_OK;
}

// The inner-product kernels hold several compensated sums per thread (many registers, few CTAs per SM):
// a grid of exactly the resident CTAs avoids a partial second wave.  Variants (helm_autotune picks):
// 0 = groups of eight, two loads per vector per iteration; 1 = pipelined groups of four; 2 = pipelined
// groups of eight.
const void* dots_fn(int v) {
    if (v == 1) return (const void*)dots_pipe_kernel<4>;
    if (v == 2) return (const void*)dots_pipe_kernel<8>;
    return (const void*)dots_kernel;
}

int dots_ctas_for(const helm_ctx* c, int v) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dots_fn(v), NT, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 2;
    }
    return (sms > 0 ? sms : 148) * per;
}

int dots_ctas(const helm_ctx* c) {
    int m = 0;
    for (int v = 0; v < 3; ++v) m = std::max(m, dots_ctas_for(c, v));
    return m;   // partial buffers sized for any variant
}

// vs: distance between consecutive basis vectors (0 = npts, the single solve's contiguous basis)
int launch_dots(const helm_ctx* c, const float2* V, size_t npts, int nv, const float2* w, double2* part, int ld,
                int nbd, cudaStream_t s, size_t vs) {
    (void)nbd;
    if (!vs) vs = npts;
    // variant 2 takes the four-wide kernel for up to four vectors (fewer registers, more resident CTAs)
    const int v = (c->tune_dots == 2 && nv <= 4) ? 1 : c->tune_dots;
    const int nb = dots_ctas_for(c, v);
    if (v == 1) dots_pipe_kernel<4><<<nb, NT, 0, s>>>(V, npts, nv, w, part, ld, vs);
    else if (v == 2) dots_pipe_kernel<8><<<nb, NT, 0, s>>>(V, npts, nv, w, part, ld, vs);
    else dots_kernel<<<nb, NT, 0, s>>>(V, npts, nv, w, part, ld, vs);
    return nb;
}

int default_nb(const helm_ctx* c) {
    if (c->tune_nb > 0) return c->tune_nb;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    return 4 * (sms > 0 ? sms : 148);
}

helm_status ensure_work(helm_ctx* c) {
    const int m = c->opt.restart, flex = c->opt.flexible;
    KrylovWork* k = c->kw;
    if (k && k->m == m && k->flexible == flex && k->NB == default_nb(c)) return HELM_OK;
    krylov_free(c);
    k = new KrylovWork();
    c->kw = k;
    return alloc_work(c, k, m, flex, default_nb(c));
}

// control slots and events of the single-solve loop (batch lanes do not use them)
helm_status ensure_slots(KrylovWork* k) {
    if (k->slots_h) return HELM_OK;
    HELM_CUDA_TRY(cudaMallocHost(&k->slots_h, sizeof(Ctrl) * k->m));
    k->ev_slot = new cudaEvent_t[k->m]();
    for (int j = 0; j < k->m; ++j) HELM_CUDA_TRY(cudaEventCreateWithFlags(&k->ev_slot[j], cudaEventDisableTiming));
    return HELM_OK;
}

helm_status read_ctrl(KrylovWork* k, cudaStream_t s) {
    HELM_CUDA_TRY(cudaMemcpyAsync(k->ctrl_h, k->ctrl_d, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return HELM_OK;
}

helm_status true_residual(helm_ctx* c, bool xzero, int first, cudaStream_t s) {
    KrylovWork* k = c->kw;
    if (xzero) {
        prof_begin(c, s, PROF_OTHER);
        residual_zero_kernel<<<k->nres, NT, 0, s>>>(k->Fdf, k->V, c->npts, k->rpart);
        prof_end(c, s);
        HELM_CUDA_TRY(cudaGetLastError());
    } else {
        helm_status st = launch_residual(c, k->xdf, k->Fdf, k->V, k->rpart, s);
        if (st != HELM_OK) return st;
    }
    prof_begin(c, s, PROF_SMALL);
    resnorm_kernel<<<1, 256, 0, s>>>(k->rpart, k->nres, k->sigma, k->g, k->m, k->ctrl_d, first);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return read_ctrl(k, s);
}

}  // namespace

void krylov_free(helm_ctx* c) {
    KrylovWork* k = c->kw;
    if (!k) return;
    free_work(k);
    delete k;
    c->kw = nullptr;
}

helm_status gmres_run(helm_ctx* c, const double2* b_in, double2* x_in, helm_solve_info* info, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    helm_status st = ensure_work(c);
    if (st != HELM_OK) return st;
    KrylovWork* k = c->kw;
    if ((st = ensure_slots(k)) != HELM_OK) return st;
    const size_t npts = c->npts, vbytes = npts * sizeof(double2);
    const int m = c->opt.restart, flex = c->opt.flexible;
    // device memory is used in place; mapped page-locked host memory is read (b, x0) and written (x) by the
    // conversion kernels through its device address; other host memory is staged by copies
    const bool xdev = is_device_ptr(x_in), bdev = is_device_ptr(b_in);
    double2* const xmap = xdev ? nullptr : (double2*)mapped_host_ptr(x_in);
    const double2* const bmap = bdev ? nullptr : (const double2*)mapped_host_ptr(b_in);
    double2* x = xdev ? x_in : xmap;
    const double2* b = bdev ? b_in : bmap;
    if (!x) {
        if (!k->xbuf) HELM_CUDA_TRY(cudaMalloc(&k->xbuf, vbytes));
        HELM_CUDA_TRY(cudaMemcpyAsync(k->xbuf, x_in, vbytes, cudaMemcpyHostToDevice, s));
        x = k->xbuf;
    }
    if (!b) {
        if (!k->bbuf) HELM_CUDA_TRY(cudaMalloc(&k->bbuf, vbytes));
        HELM_CUDA_TRY(cudaMemcpyAsync(k->bbuf, b_in, vbytes, cudaMemcpyHostToDevice, s));
        b = k->bbuf;
    }
    HELM_CUDA_TRY(cudaMemsetAsync(c->status_d, 0, sizeof(unsigned), s));
    const int NB = k->NB, ld = m + 1;
    const int ublocks = NB;
    int its = 0, restarts = 0;
    int cyc[16] = {0};
    helm_status result = HELM_ERR_NOT_CONVERGED;
    // HELM_PREC_FP16, flexible, one Gram-Schmidt pass: the Krylov basis in FP16 (v_i = c16[i] V16_i), the
    // preconditioner reading it directly, the cycles ending at kInnerFloorH16
    const bool h16b = c->opt.precision == HELM_PREC_FP16 && flex && !c->opt.reorth && !c->net &&
                      c->opt.precond == HELM_PRECOND_EIGT && c->tmaps;
    const float s0 = c->h16s[0];
    if (h16b && !k->side) {
        HELM_CUDA_TRY(cudaStreamCreateWithFlags(&k->side, cudaStreamNonBlocking));
        k->ev_upd = new cudaEvent_t[m]();
        k->ev_giv = new cudaEvent_t[m]();
        for (int j = 0; j < m; ++j) {
            HELM_CUDA_TRY(cudaEventCreateWithFlags(&k->ev_upd[j], cudaEventDisableTiming));
            HELM_CUDA_TRY(cudaEventCreateWithFlags(&k->ev_giv[j], cudaEventDisableTiming));
        }
    }
    if (h16b && !k->V16) {
        if (cudaMalloc(&k->V16, (size_t)(m + 1) * npts * 2 * sizeof(uint16_t)) != cudaSuccess ||
            cudaMalloc(&k->c16, (m + 1) * sizeof(double)) != cudaSuccess || cudaMalloc(&k->w16s, sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(k->V16); cudaFree(k->c16); cudaFree(k->w16s);
            k->V16 = nullptr; k->c16 = nullptr; k->w16s = nullptr;
            return HELM_ERR_NOMEM;
        }
    }
    // internal double-float copies of b and x; x0 = 0 is recognised and then r0 = b without a matvec
    unsigned xnz = 0;
    HELM_CUDA_TRY(cudaMemsetAsync(k->nzflag, 0, sizeof(unsigned), s));
    to_df_kernel<<<NB, NT, 0, s>>>(b, k->Fdf, npts, nullptr);
    to_df_kernel<<<NB, NT, 0, s>>>(x, k->xdf, npts, k->nzflag);
    HELM_CUDA_TRY(cudaMemcpyAsync(&xnz, k->nzflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = true_residual(c, xnz == 0, 1, s)) != HELM_OK) return st;
    const double beta0 = k->ctrl_h->beta0;
    double est = 1.0;
    if (!(beta0 > 0)) {
        result = (k->ctrl_h->flags & HELM_DEV_NAN) ? HELM_ERR_NAN : HELM_OK;
    } else {
        for (;;) {
            if (k->ctrl_h->beta / beta0 <= c->opt.rtol) { result = HELM_OK; break; }
            if (k->ctrl_h->flags & HELM_DEV_NAN) { result = HELM_ERR_NAN; break; }
            if (its >= c->opt.max_iter) { result = HELM_ERR_NOT_CONVERGED; break; }
            int kk = 0, launched = 0;
            bool breakdown = false;
            // iteration j of the cycle; its control block is copied to slot j behind it
            auto enqueue = [&](int j) -> helm_status {
                float2* vj = k->V + (size_t)j * npts;
                float2* w = k->V + (size_t)(j + 1) * npts;
                float2* z = flex ? k->Z + (size_t)j * npts : k->Z;
                helm_status e;
                if (h16b) {
                    float2* wv = k->V + npts;   // complex64 scratch: A z_j, orthogonalised into V16_{j+1}
                    uint16_t* Vj = k->V16 + (size_t)j * 2 * npts;
                    c->h16_join = j > 0 ? k->ev_giv[j - 1] : nullptr;   // the last pass reads c16[j]
                    e = precond_h16_basis(c, Vj, z, k->c16, j, s);
                    c->h16_join = nullptr;
                    if (e != HELM_OK) return e;
                    if ((e = launch_stencil_f32(c, z, wv, nullptr, 0, s)) != HELM_OK) return e;
                    prof_begin(c, s, PROF_DOTS);
                    int nbd16 = k->NBd;
                    if (j + 2 <= 32 && c->zring_sms > 0 && c->zring_sms <= std::max(k->NB, k->NBd)) {
                        // staged form: T points per chunk so that one stage holds w and the j + 1 basis chunks
                        const int T = std::max(64, (int)(DB_STAGE / (8 + 4 * (j + 1))) / 64 * 64);
                        nbd16 = c->zring_sms;
                        if (!k->db_ready) {
                            HELM_CUDA_TRY(cudaFuncSetAttribute(dots16b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)DB_SMEM));
                            k->db_ready = 1;
                        }
                        dots16b_kernel<<<nbd16, DB_NT, DB_SMEM, s>>>(k->V16, npts, j + 1, wv, k->part, ld, T, c->status_d,
                                                                     (long)c->wait_limit);
                    } else {
                        dots16_kernel<8><<<k->NBd, NT, 0, s>>>(k->V16, npts, j + 1, wv, k->part, ld);
                    }
                    prof_end(c, s);
                    prof_begin(c, s, PROF_SMALL);
                    reduce16_kernel<<<j + 2, 128, 0, s>>>(k->part, nbd16, ld, j + 1, k->c16, k->H + (size_t)j * (m + 1),
                                                          k->coef, s0, k->w16s);
                    prof_end(c, s);
                    prof_begin(c, s, PROF_UPDATE);
                    update16_kernel<<<ublocks, NT, 0, s>>>(k->V16, npts, j + 1, k->coef, wv, Vj + 2 * npts, k->w16s,
                                                           k->part, ld);
                    prof_end(c, s);
                    // the Givens step on the side stream: the next step's first passes do not need it
                    HELM_CUDA_TRY(cudaEventRecord(k->ev_upd[j], s));
                    HELM_CUDA_TRY(cudaStreamWaitEvent(k->side, k->ev_upd[j], 0));
                    givens_kernel<<<1, 256, 0, k->side>>>(k->part, NB, ld, j, m, k->H, k->cs, k->sn, k->g, k->sigma,
                                                          k->ctrl_d, k->w16s, k->c16);
                    HELM_CUDA_TRY(cudaGetLastError());
                    HELM_CUDA_TRY(cudaMemcpyAsync(&k->slots_h[j], k->ctrl_d, sizeof(Ctrl), cudaMemcpyDeviceToHost, k->side));
                    HELM_CUDA_TRY(cudaEventRecord(k->ev_slot[j], k->side));
                    HELM_CUDA_TRY(cudaEventRecord(k->ev_giv[j], k->side));
                    return HELM_OK;
                }
                if ((e = precond_apply(c, vj, z, k->sigma, j, s)) != HELM_OK) return e;
                if ((e = launch_stencil_f32(c, z, w, nullptr, 0, s)) != HELM_OK) return e;
                const int passes = c->opt.reorth ? 2 : 1;
                for (int pass = 0; pass < passes; ++pass) {
                    prof_begin(c, s, PROF_DOTS);
                    const int nbd = launch_dots(c, k->V, npts, j + 1, w, k->part, ld, k->NBd, s);
                    prof_end(c, s);
                    prof_begin(c, s, PROF_SMALL);
                    reduce_h_kernel<<<j + 1, 128, 0, s>>>(k->part, nbd, ld, j + 1, k->sigma, k->H + (size_t)j * (m + 1),
                                                      k->coef, pass == 0);
                    prof_end(c, s);
                    prof_begin(c, s, PROF_UPDATE);
                    update_kernel<<<ublocks, NT, 0, s>>>(k->V, npts, j + 1, k->coef, w, k->part, ld, npts);
                    prof_end(c, s);
                }
                prof_begin(c, s, PROF_SMALL);
                givens_kernel<<<1, 256, 0, s>>>(k->part, NB, ld, j, m, k->H, k->cs, k->sn, k->g, k->sigma, k->ctrl_d);
                prof_end(c, s);
                HELM_CUDA_TRY(cudaGetLastError());
                HELM_CUDA_TRY(cudaMemcpyAsync(&k->slots_h[j], k->ctrl_d, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
                HELM_CUDA_TRY(cudaEventRecord(k->ev_slot[j], s));
                return HELM_OK;
            };
            // Look-ahead: while the last known estimate is far above rtol, iteration j+1 is enqueued before
            // the estimate of iteration j is read, so the device never waits for the host.  An iteration
            // enqueued beyond the end of the cycle leaves columns j+1.. of H and g[j+2] behind, which the
            // least-squares solve of the first kk columns does not read; the control block is restored.
            double est_prev = k->ctrl_h->beta / beta0;
            const double thr = inner_threshold(c->opt.rtol, k->ctrl_h->beta, beta0, h16b ? kInnerFloorH16 : kInnerFloor);
            if (h16b) {   // v_0 = r / beta into V16_0 (r is V_0 of the true residual), c16[0] = 1 / s0
                if ((st = to_h16_basis(c, k->V, k->V16, k->sigma, 0, s)) != HELM_OK) return st;
                c16_kernel<<<1, 32, 0, s>>>(k->sigma, 0, k->w16s, k->c16, s0);
                HELM_CUDA_TRY(cudaGetLastError());
            }
            for (int j = 0; j < m; ++j) {
                if (launched <= j) {
                    if ((st = enqueue(j)) != HELM_OK) {
                        if (k->side) cudaStreamSynchronize(k->side);
                        return st;
                    }
                    launched = j + 1;
                }
                if (j + 1 < m && its + 2 <= c->opt.max_iter && est_prev * kLookaheadDrop > thr) {
                    if ((st = enqueue(j + 1)) != HELM_OK) {
                        if (k->side) cudaStreamSynchronize(k->side);
                        return st;
                    }
                    launched = j + 2;
                }
                HELM_CUDA_TRY(cudaEventSynchronize(k->ev_slot[j]));
                const Ctrl& cj = k->slots_h[j];
                ++its;
                kk = j + 1;
                est = cj.est;
                est_prev = est;
                if (cj.flags & HELM_DEV_NAN) break;
                if (est <= thr || its >= c->opt.max_iter) break;
                if (!(cj.hnext > 0)) { breakdown = true; break; }
            }
            *k->ctrl_h = k->slots_h[kk - 1];
            if (h16b) HELM_CUDA_TRY(cudaStreamWaitEvent(s, k->ev_giv[launched - 1], 0));   // every Givens step of the cycle
            if (launched > kk)
                HELM_CUDA_TRY(cudaMemcpyAsync(k->ctrl_d, &k->slots_h[kk - 1], sizeof(Ctrl), cudaMemcpyHostToDevice, s));
            if (k->ctrl_h->flags & HELM_DEV_NAN) { result = HELM_ERR_NAN; break; }
            prof_begin(c, s, PROF_SMALL);
            lsq_kernel<<<1, 32, 0, s>>>(k->H, k->g, kk, m, k->y, k->ctrl_d, nullptr);
            prof_end(c, s);
            if (flex) {
                prof_begin(c, s, PROF_COMBINE);
                combine_flex_kernel<<<NB, NT, 0, s>>>(k->Z, npts, kk, k->y, k->xdf, nullptr, npts);
                prof_end(c, s);
            } else {
                float2* u = k->V + (size_t)kk * npts;   // V_kk is not needed by the update
                prof_begin(c, s, PROF_COMBINE);
                combine_v_kernel<<<NB, NT, 0, s>>>(k->V, npts, kk, k->y, k->sigma, u, nullptr, npts);
                prof_end(c, s);
                if ((st = precond_apply(c, u, u, nullptr, 0, s)) != HELM_OK) return st;
                prof_begin(c, s, PROF_COMBINE);
                add_kernel<<<NB, NT, 0, s>>>(u, k->xdf, npts);
                prof_end(c, s);
            }
            HELM_CUDA_TRY(cudaGetLastError());
            if (restarts < 16) cyc[restarts] = kk;
            ++restarts;
            if ((st = true_residual(c, false, 0, s)) != HELM_OK) return st;
            if (breakdown && k->ctrl_h->beta / beta0 > c->opt.rtol) { result = HELM_ERR_BREAKDOWN; break; }
        }
    }
    unsigned dstat = 0;
    from_df_kernel<<<NB, NT, 0, s>>>(k->xdf, x, npts);
    HELM_CUDA_TRY(cudaMemcpyAsync(&dstat, c->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    if (!xdev && !xmap) HELM_CUDA_TRY(cudaMemcpyAsync(x_in, x, vbytes, cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (result == HELM_OK && (dstat & HELM_DEV_PIVOT)) result = HELM_ERR_PIVOT;
    if (dstat & HELM_DEV_WAIT) result = HELM_ERR_ITER_LIMIT;
    if (info) {
        info->status = result;
        info->iterations = its;
        info->restarts = restarts;
        info->relres_true = beta0 > 0 ? k->ctrl_h->beta / beta0 : 0.0;
        info->relres_est = est;
        info->beta0 = beta0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < 16; ++i) info->cycle_its[i] = cyc[i];
    }
    return result;
}

// r = b - A x with the double-float residual kernel; |r|_2 and |r|_inf in FP64 (helm_residual).
helm_status residual_run(helm_ctx* c, const double2* b, const double2* x, float2* r, double* nrm2, double* nrmi,
                         cudaStream_t s) {
    helm_status st = ensure_work(c);
    if (st != HELM_OK) return st;
    KrylovWork* k = c->kw;
    const size_t npts = c->npts;
    to_df_kernel<<<k->NB, NT, 0, s>>>(b, k->Fdf, npts, nullptr);
    to_df_kernel<<<k->NB, NT, 0, s>>>(x, k->xdf, npts, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    if ((st = launch_residual(c, k->xdf, k->Fdf, r ? r : k->V, k->rpart, s)) != HELM_OK) return st;
    std::vector<double> h(2 * (size_t)k->nres);
    HELM_CUDA_TRY(cudaMemcpyAsync(h.data(), k->rpart, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    double t = 0, m = 0;
    for (int i = 0; i < k->nres; ++i) { t += h[2 * i]; m = m > h[2 * i + 1] ? m : h[2 * i + 1]; }
    if (nrm2) *nrm2 = sqrt(t);
    if (nrmi) *nrmi = m;
    return HELM_OK;
}

// ---- launch-shape autotuning ------------------------------------------------------------------
// The Arnoldi kernels (inner products, update, solution combine) are grid-stride loops whose CTA count
// trades latency hiding against the cost of the per-CTA partial sums; the best count depends on the
// grid size.  helm_autotune times the candidates on the context's own grid and keeps the fastest.

namespace {

struct TuneKey {
    int nx, ny, nz, order;
    bool operator<(const TuneKey& o) const {
        if (nx != o.nx) return nx < o.nx;
        if (ny != o.ny) return ny < o.ny;
        if (nz != o.nz) return nz < o.nz;
        return order < o.order;
    }
};
struct TuneVal {
    int nb, stencil, dots, tc, ypers, zring;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

extern "C" helm_status helm_autotune(helm_ctx* c, int* nb_out, int* variant_out, int* dots_out, void* stream) {
    if (!c) return HELM_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(TuneKey{c->nx, c->ny, c->nz, c->opt.order});
        if (it != g_tune_cache.end()) {
            c->tune_nb = it->second.nb;
            c->tune_stencil = std::min(it->second.stencil, stencil_variants(c) - 1);
            c->tune_dots = it->second.dots;
            c->tune_tc = it->second.tc;
            c->tune_ypers = it->second.ypers;
            c->tune_zring = it->second.zring;
            if (nb_out) *nb_out = c->tune_nb;
            if (variant_out) *variant_out = c->tune_stencil;
            if (dots_out) *dots_out = c->tune_dots;
            return HELM_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    HELM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (sms <= 0) sms = 148;
    const size_t npts = c->npts;
    const int nv = 8, ld = nv + 1;
    const int cand[] = {sms / 2, sms, 2 * sms, 4 * sms, 8 * sms};
    const int maxnb = (int)std::min<size_t>((npts / 2 + NT - 1) / NT, (size_t)16 * sms);
    float2* V = nullptr;
    double2* part = nullptr;
    float2* coef = nullptr;
    if (cudaMalloc(&V, npts * sizeof(float2) * (nv + 1)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    if (cudaMalloc(&part, sizeof(double2) * ld * 16 * (size_t)sms) != cudaSuccess ||
        cudaMalloc(&coef, sizeof(float2) * ld) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(V); cudaFree(part);
        return HELM_ERR_NOMEM;
    }
    cudaMemsetAsync(V, 0, npts * sizeof(float2) * (nv + 1), s);
    cudaMemsetAsync(coef, 0, sizeof(float2) * ld, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 4 * sms;
    float best_ms = 1e30f;
    float2* w = V + (size_t)nv * npts;
    for (int nb : cand) {
        nb = std::max(1, std::min(nb, maxnb));
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            dots_kernel<<<nb, NT, 0, s>>>(V, npts, nv, w, part, ld, npts);
            update_kernel<<<nb, NT, 0, s>>>(V, npts, nv, coef, w, part, ld, npts);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);   // the first run is a warm-up
        }
        if (tmin < best_ms * 0.97f) { best_ms = tmin; best = nb; }
    }
    // the matvec variant: time each on the context's grid (input and output in the scratch vectors)
    int best_st = 0;
    float best_st_ms = 1e30f;
    for (int v = 0; v < stencil_variants(c); ++v) {
        c->tune_stencil = v;
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch_stencil_f32(c, V, V + npts, nullptr, 0, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);
        }
        if (tmin < best_st_ms * 0.97f) { best_st_ms = tmin; best_st = v; }
    }
    c->tune_stencil = best_st;
    // the inner-product variant, on eight basis vectors
    int best_d = 0;
    float best_d_ms = 1e30f;
    for (int v = 0; v < 3; ++v) {
        c->tune_dots = v;
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch_dots(c, V, npts, nv, w, part, ld, 0, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);
        }
        if (tmin < best_d_ms * 0.97f) { best_d_ms = tmin; best_d = v; }
    }
    c->tune_dots = best_d;
    auto time_it = [&](auto&& launch) {
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);
        }
        return tmin;
    };
    // the tensor-core transform variants (persistent or one tile per CTA), timed on a whole preconditioner
    // application
    if (c->opt.precision == HELM_PREC_TF32 && c->tmaps && c->opt.precond != HELM_PRECOND_NONE) {
        int btc = c->tune_tc, byp = c->tune_ypers;
        float bms = 1e30f;
        for (int tc = 1; tc >= 0; --tc)
            for (int yp = 1; yp >= 0; --yp) {
                c->tune_tc = tc;
                c->tune_ypers = yp;
                const float ms = time_it([&] { precond_apply(c, V, V + npts, nullptr, 0, s); });
                if (ms < bms * 0.97f) { bms = ms; btc = tc; byp = yp; }
            }
        c->tune_tc = btc;
        c->tune_ypers = byp;
    }
    // the factorised z-solve: CTAs per SM of the L2-resident kernel (0 = one thread per line)
    if (c->zfac && c->opt.precond == HELM_PRECOND_EIGT && c->nx % 2 == 0) {
        int bz = c->tune_zring;
        float bms = 1e30f;
        for (int zr = 0; zr <= 3; ++zr) {
            c->tune_zring = zr;
            const float ms = time_it([&] { launch_zsolve(c, V, V + npts, s); });
            if (ms < bms * 0.97f) { bms = ms; bz = zr; }
        }
        c->tune_zring = bz;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(V); cudaFree(part); cudaFree(coef);
    HELM_CUDA_TRY(cudaGetLastError());
    c->tune_nb = best;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[TuneKey{c->nx, c->ny, c->nz, c->opt.order}] =
            TuneVal{best, best_st, best_d, c->tune_tc, c->tune_ypers, c->tune_zring};
    }
    if (nb_out) *nb_out = best;
    if (variant_out) *variant_out = best_st;
    if (dots_out) *dots_out = best_d;
    return HELM_OK;
}

// ---- batched solves ---------------------------------------------------------------------------
// Many problems (contexts of any size and options) times nrhs right-hand sides each, solved together:
// every (problem, right-hand side) pair is a lane with its own Krylov workspace and preconditioner
// scratch; the lanes of one problem form a group that shares the operator launches.  One restart cycle of
// every lane is one CUDA graph,
//   for each group (independent branches):  begin; IF(any lane runs it) iteration 0; ...; iteration m-1;
//                                            IF(cycle) end of each lane
// whose conditions are set on the device (convergence estimate, iteration limit, breakdown; a finished lane
// skips everything), so a launch costs the host one graph launch and one synchronisation per restart cycle
// for the whole batch.  The host relaunches the graph while any lane wants another cycle (a device flag per
// lane); there is no device-side loop, so a lane can never spin.

struct LaneCtl {
    int active, kk, its, restarts, brk, cycles, max_iter, m;
    double rtol;
    int cyc[16];
    int go;          // the lane runs its next iteration (read by its group)
};

namespace {

// would the lane run another cycle?  (the same test opens each cycle)
__device__ bool lane_wants_cycle(const Ctrl* ctrl, const LaneCtl* L) {
    if (!L->active) return false;
    if (!(ctrl->beta0 > 0)) return false;
    if (ctrl->beta / ctrl->beta0 <= L->rtol) return false;
    if (ctrl->flags & HELM_DEV_NAN) return false;
    if (L->its >= L->max_iter || L->brk || L->cycles > L->max_iter) return false;
    return true;
}

// end of iteration j of a lane that ran it: counts it and decides whether the lane runs iteration j+1
// (has_next = 0 after the last iteration of a cycle)
__device__ void lane_iter_step(const Ctrl* __restrict__ ctrl, LaneCtl* L, int j, int has_next) {
    L->its += 1;
    L->kk = j + 1;
    bool go = !(ctrl->flags & HELM_DEV_NAN) && ctrl->est > inner_threshold(L->rtol, ctrl->beta, ctrl->beta0) &&
              L->its < L->max_iter && j + 1 < L->m;
    if (!(ctrl->hnext > 0)) { go = false; L->brk = 1; }
    L->go = (go && has_next) ? 1 : 0;
}

// The per-lane device pointers of a batch group, indexed by lane.  The group's Arnoldi kernels take their
// lane from the grid (blockIdx.y, or blockIdx.x for the one-block-per-lane kernels) and return at once for a
// lane that does not run the current iteration (L->go = 0), so one launch serves all the group's lanes.
struct LaneDev {
    float2* V;        // the lane's v_0; its basis vectors are vs apart (interleaved with the group's other lanes)
    double2* part;
    double2* H;
    double* cs;
    double2* sn;
    double2* g;
    double* sigma;
    float2* coef;
    Ctrl* ctrl;
    LaneCtl* L;
};

// h = V^H w of every running lane (w = its v_{j+1} slot); VAR 0: dots_body, 4 or 8: dots_pipe_body<VAR>
template <int VAR>
__global__ void __launch_bounds__(NT) grp_dots_kernel(const LaneDev* __restrict__ lt, size_t npts, int nv, int j,
                                                     int ld, size_t vs) {
    const LaneDev& d = lt[blockIdx.y];
    if (!d.L->go) return;
    const float2* w = d.V + (size_t)(j + 1) * vs;
    if constexpr (VAR == 0) dots_body(d.V, npts, nv, w, d.part, ld, vs);
    else dots_pipe_body<VAR>(d.V, npts, nv, w, d.part, ld, vs);
}

__global__ void grp_reduce_h_kernel(const LaneDev* __restrict__ lt, int NB, int ld, int nv, int j, int m,
                                    int first_pass) {
    const LaneDev& d = lt[blockIdx.y];
    if (!d.L->go) return;
    reduce_h_body(d.part, NB, ld, nv, d.sigma, d.H + (size_t)j * (m + 1), d.coef, first_pass);
}

__global__ void __launch_bounds__(NT) grp_update_kernel(const LaneDev* __restrict__ lt, size_t npts, int nv, int j,
                                                       int ld, size_t vs) {
    const LaneDev& d = lt[blockIdx.y];
    if (!d.L->go) return;
    update_body(d.V, npts, nv, d.coef, d.V + (size_t)(j + 1) * vs, d.part, ld, vs);
}

__global__ void grp_givens_kernel(const LaneDev* __restrict__ lt, int NB, int ld, int j, int m) {
    const LaneDev& d = lt[blockIdx.x];
    if (!d.L->go) return;
    givens_body(d.part, NB, ld, j, m, d.H, d.cs, d.sn, d.g, d.sigma, d.ctrl);
}

// end of the group's iteration j: steps every lane that ran it and opens iteration j+1 (handle hnext) when
// any lane runs it
__global__ void grp_iter_end_kernel(const LaneDev* __restrict__ lt, int nb, int j, cudaGraphConditionalHandle hnext,
                                    int has_next) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int any = 0;
    for (int r = 0; r < nb; ++r) {
        LaneCtl* L = lt[r].L;
        if (!L->go) continue;
        lane_iter_step(lt[r].ctrl, L, j, has_next);
        any |= L->go;
    }
    if (has_next) cudaGraphSetConditional(hnext, any ? 1u : 0u);
}

// start of a restart cycle of the group: each lane decides whether it runs the cycle (more[r], its
// cycle-end handle hcyc[r]); the group's iteration 0 (handle h0) runs when any lane does
__global__ void grp_begin_kernel(const LaneDev* __restrict__ lt, int nb, int* more,
                                 const cudaGraphConditionalHandle* __restrict__ hcyc, cudaGraphConditionalHandle h0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int any = 0;
    for (int r = 0; r < nb; ++r) {
        LaneCtl* L = lt[r].L;
        const bool go = lane_wants_cycle(lt[r].ctrl, L);
        if (!go) L->active = 0;
        else L->cycles += 1;
        L->kk = 0;
        L->go = go ? 1 : 0;
        more[r] = go ? 1 : 0;
        cudaGraphSetConditional(hcyc[r], go ? 1u : 0u);
        any |= go;
    }
    cudaGraphSetConditional(h0, any ? 1u : 0u);
}

__global__ void lane_cycle_end_kernel(const Ctrl* __restrict__ ctrl, LaneCtl* L, int* more) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (L->restarts < 16) L->cyc[L->restarts] = L->kk;
    L->restarts += 1;
    *more = lane_wants_cycle(ctrl, L) ? 1 : 0;
}

struct Lane {
    helm_ctx* c = nullptr;
    double2* b = nullptr;
    double2* x = nullptr;
    KrylovWork w;
    float2* tmp = nullptr;
    LaneCtl* L_d = nullptr;
    int* more = nullptr;       // device flag: the lane wants another cycle
    LaneCtl L_h{};
    Ctrl ctrl_copy{};
    int index = 0;
};

size_t lane_bytes(const helm_ctx* c) {
    const int m = c->opt.restart;
    return c->npts * (sizeof(float2) * ((size_t)m + 1 + (c->opt.flexible ? m : 1) + 1) + 2 * sizeof(float4));
}

// the preconditioner of a lane, on the lane's own scratch vector (the context's is shared by all its lanes)
// (the lanes' cycle ends run as parallel branches: their z-solves take the stored-factor kernel, which
// needs no per-context scratch)
helm_status lane_precond(Lane& ln, const float2* r, float2* z, const double* sigma, int sidx, cudaStream_t s) {
    float2* save = ln.c->tmp;
    ln.c->tmp = ln.tmp;
    ln.c->zpiv_off = 1;
    helm_status st = precond_apply(ln.c, r, z, sigma, sidx, s);
    ln.c->zpiv_off = 0;
    ln.c->tmp = save;
    return st;
}

helm_status lane_cycle_end(Lane& ln, cudaStream_t s) {
    helm_ctx* c = ln.c;
    KrylovWork* k = &ln.w;
    const size_t npts = c->npts;
    const int m = k->m, NB = k->NB;
    const int* kk = &ln.L_d->kk;
    helm_status st;
    lsq_kernel<<<1, 32, 0, s>>>(k->H, k->g, 0, m, k->y, k->ctrl_d, kk);
    if (k->flexible) {
        combine_flex_kernel<<<NB, NT, 0, s>>>(k->Z, npts, 0, k->y, k->xdf, kk, k->vs);
    } else {
        combine_v_kernel<<<NB, NT, 0, s>>>(k->V, npts, 0, k->y, k->sigma, k->Z, kk, k->vs);
        if ((st = lane_precond(ln, k->Z, k->Z, nullptr, 0, s)) != HELM_OK) return st;
        add_kernel<<<NB, NT, 0, s>>>(k->Z, k->xdf, npts);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    if ((st = launch_residual(c, k->xdf, k->Fdf, k->V, k->rpart, s)) != HELM_OK) return st;
    resnorm_kernel<<<1, 256, 0, s>>>(k->rpart, k->nres, k->sigma, k->g, m, k->ctrl_d, 0);
    lane_cycle_end_kernel<<<1, 32, 0, s>>>(k->ctrl_d, ln.L_d, ln.more);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// Capture what `enqueue` launches on s into graph g after the nodes deps.
template <typename F>
helm_status capture_into(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaStream_t s, F enqueue) {
    HELM_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, deps, nullptr, nd, cudaStreamCaptureModeRelaxed));
    helm_status st = enqueue();
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &out);
    if (st != HELM_OK) return st;
    HELM_CUDA_TRY(e);
    return HELM_OK;
}

helm_status add_cond(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    const cudaError_t e = cudaGraphAddNode(node, g, deps, nullptr, nd, &p);
    if (e != cudaSuccess) {
        char what[96];
        snprintf(what, sizeof(what), "cudaGraphAddNode(conditional type %d, %zu deps)", (int)type, nd);
        return helm_fail_cuda(e, what);
    }
    *body = p.conditional.phGraph_out[0];
    return HELM_OK;
}

// A group: the consecutive lanes of one context (its right-hand sides) in a plan.  Their basis vectors,
// preconditioned vectors and normalisation factors are interleaved in group buffers (vector v_j of lane r
// at V + (j nb + r) npts), so that each step of iteration j runs once for the whole group: one x-pass GEMM over
// nb N_y N_z rows, one y-pass over nb N_z slices, one z-solve over nb N_x N_y lines, one matvec launch over nb
// grids (the context's coefficients read once per tile for all of them), and one launch of each Arnoldi
// kernel over all the lanes (a lane that has left the cycle returns at once).
struct Group {
    helm_ctx* c = nullptr;
    int first = 0, nb = 0;          // lanes first .. first + nb - 1 of the plan
    float2* V = nullptr;            // (m + 1) nb vectors
    float2* Z = nullptr;            // m nb (flexible) or nb vectors
    float2* tmp = nullptr;          // nb vectors: the group's preconditioner scratch (lane r's own: vector r)
    double* sigma = nullptr;        // nb (m + 1)
    LaneDev* lt = nullptr;          // device table of the lanes' pointers
    int slot = 0;                   // z-solve checkpoint slot of the group's first lane within its context
    cudaGraphConditionalHandle* hcyc = nullptr;   // device copy of the lanes' cycle-end handles
};

// The nodes of one group's restart cycle (every conditional node has its own handle, default 0 at each launch):
//   begin (each lane decides whether it runs the cycle)
//   -> IF(iteration 0) { M^-1 and A for all the group's vectors; Gram-Schmidt, norm and Givens rotation of
//      every running lane; end (opens iteration 1 if any lane runs it) } -> ... -> IF(iteration m-1) { ... }
//   -> IF(lane r cycle) { least squares, x update, true residual } for every lane r (branches).
helm_status build_group(cudaGraph_t G, Group& gr, std::vector<Lane>& lanes, int* more, cudaStream_t s) {
    helm_ctx* c = gr.c;
    const int nb = gr.nb, m = lanes[gr.first].w.m, flex = c->opt.flexible, ld = m + 1;
    const size_t npts = c->npts, vs = (size_t)nb * npts;
    const KrylovWork& k0 = lanes[gr.first].w;
    std::vector<cudaGraphConditionalHandle> hcyc(nb), hg(m);
    for (int r = 0; r < nb; ++r)
        HELM_CUDA_TRY(cudaGraphConditionalHandleCreate(&hcyc[r], G, 0, cudaGraphCondAssignDefault));
    for (int j = 0; j < m; ++j) HELM_CUDA_TRY(cudaGraphConditionalHandleCreate(&hg[j], G, 0, cudaGraphCondAssignDefault));
    HELM_CUDA_TRY(cudaMemcpy(gr.hcyc, hcyc.data(), sizeof(cudaGraphConditionalHandle) * nb, cudaMemcpyHostToDevice));
    helm_status st;
    cudaGraphNode_t prev;
    {
        const LaneDev* lt = gr.lt;
        int n = nb;
        const cudaGraphConditionalHandle* hc = gr.hcyc;
        cudaGraphConditionalHandle h0 = hg[0];
        void* args[] = {(void*)&lt, (void*)&n, (void*)&more, (void*)&hc, (void*)&h0};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)grp_begin_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
        HELM_CUDA_TRY(cudaGraphAddKernelNode(&prev, G, nullptr, 0, &kp));
    }
    const int passes = c->opt.reorth ? 2 : 1;
    for (int j = 0; j < m; ++j) {
        cudaGraphNode_t gnode;
        cudaGraph_t gb;
        if ((st = add_cond(G, &prev, 1, hg[j], cudaGraphCondTypeIf, &gnode, &gb)) != HELM_OK) return st;
        float2* vj = gr.V + (size_t)j * vs;
        float2* zj = flex ? gr.Z + (size_t)j * vs : gr.Z;
        float2* w = gr.V + (size_t)(j + 1) * vs;
        const int has_next = j + 1 < m ? 1 : 0;
        const cudaGraphConditionalHandle hn = has_next ? hg[j + 1] : hg[j];
        st = capture_into(gb, nullptr, 0, s, [&]() {
            float2* save = c->tmp;
            c->tmp = gr.tmp;
            c->zck_slot = gr.slot;
            helm_status e = precond_apply_nb(c, vj, zj, nb, gr.sigma, j, m + 1, s);
            c->zck_slot = 0;
            c->tmp = save;
            if (e != HELM_OK) return e;
            if ((e = launch_stencil_f32_nb(c, zj, w, nb, s)) != HELM_OK) return e;
            const int nv = j + 1;
            const int var = (c->tune_dots == 2 && nv <= 4) ? 1 : c->tune_dots;
            const int nbd = dots_ctas_for(c, var);
            for (int pass = 0; pass < passes; ++pass) {
                const dim3 gd(nbd, nb);
                if (var == 1) grp_dots_kernel<4><<<gd, NT, 0, s>>>(gr.lt, npts, nv, j, ld, vs);
                else if (var == 2) grp_dots_kernel<8><<<gd, NT, 0, s>>>(gr.lt, npts, nv, j, ld, vs);
                else grp_dots_kernel<0><<<gd, NT, 0, s>>>(gr.lt, npts, nv, j, ld, vs);
                grp_reduce_h_kernel<<<dim3(nv, nb), 128, 0, s>>>(gr.lt, nbd, ld, nv, j, m, pass == 0);
                grp_update_kernel<<<dim3(k0.NB, nb), NT, 0, s>>>(gr.lt, npts, nv, j, ld, vs);
            }
            grp_givens_kernel<<<nb, 256, 0, s>>>(gr.lt, k0.NB, ld, j, m);
            grp_iter_end_kernel<<<1, 32, 0, s>>>(gr.lt, nb, j, hn, has_next);
            HELM_CUDA_TRY(cudaGetLastError());
            return HELM_OK;
        });
        if (st != HELM_OK) return st;
        prev = gnode;
    }
    for (int r = 0; r < nb; ++r) {
        Lane& ln = lanes[gr.first + r];
        cudaGraphNode_t cnode;
        cudaGraph_t cb;
        if ((st = add_cond(G, &prev, 1, hcyc[r], cudaGraphCondTypeIf, &cnode, &cb)) != HELM_OK) return st;
        if ((st = capture_into(cb, nullptr, 0, s, [&]() { return lane_cycle_end(ln, s); })) != HELM_OK) return st;
    }
    return HELM_OK;
}

void free_lane(Lane& ln) {
    free_work(&ln.w);
    ln.w = KrylovWork();
    cudaFree(ln.L_d);
    ln.tmp = nullptr;   // a view of the group's scratch
    ln.L_d = nullptr;
    ln.more = nullptr;
}

void free_group(Group& g) {
    cudaFree(g.V);
    cudaFree(g.Z);
    cudaFree(g.tmp);
    cudaFree(g.sigma);
    cudaFree(g.lt);
    cudaFree(g.hcyc);
    g = Group();
}

}  // namespace

// A batch plan: the lanes' workspaces and the instantiated restart-cycle graph, reusable across runs.
struct helm_batch {
    std::vector<Lane> lanes;
    std::vector<Group> groups;
    std::vector<helm_ctx*> ctxs;
    int nprob = 0, nrhs = 0;
    int* flags = nullptr;
    cudaGraph_t G = nullptr;
    cudaGraphExec_t X = nullptr;
    cudaStream_t cs = nullptr;
};

namespace {

void plan_free(helm_batch* P) {
    if (P->X) cudaGraphExecDestroy(P->X);
    if (P->G) cudaGraphDestroy(P->G);
    if (P->cs) cudaStreamDestroy(P->cs);
    cudaFree(P->flags);
    for (Lane& ln : P->lanes) free_lane(ln);
    for (Group& g : P->groups) free_group(g);
    P->groups.clear();
    P->X = nullptr; P->G = nullptr; P->cs = nullptr; P->flags = nullptr;
}

// workspace of every group and lane, and the graph of one restart cycle of all lanes
helm_status plan_build(helm_batch* P) {
    helm_status st;
    // groups: runs of consecutive lanes of the same context.  Below kGroupMinPoints a problem's right-hand
    // sides run as independent single-lane groups instead: there the operators are latency-bound, and
    // independent chains keep more of the GPU busy than shared launches save (measured on the 64 x 4 batch
    // of 48^3 .. 160^3 problems).  Each lane has its own z-solve checkpoint slot within its context.
    constexpr size_t kGroupMinPoints = (size_t)160 * 160 * 160;
    std::vector<std::pair<helm_ctx*, int>> nlanes;   // lanes per context so far
    for (size_t i = 0; i < P->lanes.size();) {
        Group g;
        g.c = P->lanes[i].c;
        g.first = (int)i;
        if (g.c->npts >= kGroupMinPoints) {
            while (i < P->lanes.size() && P->lanes[i].c == g.c) ++i;
        } else {
            ++i;
        }
        g.nb = (int)i - g.first;
        size_t e = 0;
        while (e < nlanes.size() && nlanes[e].first != g.c) ++e;
        if (e == nlanes.size()) nlanes.push_back({g.c, 0});
        g.slot = nlanes[e].second;   // the context's lanes before this group
        nlanes[e].second += g.nb;
        P->groups.push_back(g);
    }
    for (Group& g : P->groups) {
        helm_ctx* c = g.c;
        const int m = c->opt.restart, flex = c->opt.flexible, nb = g.nb;
        const size_t vb = c->npts * sizeof(float2);
        auto A = [](void** p, size_t bytes) {
            if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
            return true;
        };
        if (!A((void**)&g.V, vb * (m + 1) * nb) || !A((void**)&g.Z, vb * (flex ? m : 1) * nb) ||
            !A((void**)&g.tmp, vb * nb) || !A((void**)&g.sigma, sizeof(double) * (m + 1) * nb) ||
            !A((void**)&g.lt, sizeof(LaneDev) * nb) || !A((void**)&g.hcyc, sizeof(cudaGraphConditionalHandle) * nb))
            return HELM_ERR_NOMEM;
        std::vector<LaneDev> lt(nb);
        for (int r = 0; r < nb; ++r) {
            Lane& ln = P->lanes[g.first + r];
            if ((st = alloc_work(c, &ln.w, m, flex, default_nb(c), g.V + (size_t)r * c->npts,
                                 g.Z + (size_t)r * c->npts, g.sigma + (size_t)r * (m + 1), (size_t)nb * c->npts)) !=
                HELM_OK)
                return st;
            ln.tmp = g.tmp + (size_t)r * c->npts;
            HELM_CUDA_TRY(cudaMalloc(&ln.L_d, sizeof(LaneCtl)));
            const KrylovWork& k = ln.w;
            lt[r] = LaneDev{k.V, k.part, k.H, k.cs, k.sn, k.g, k.sigma, k.coef, k.ctrl_d, ln.L_d};
        }
        HELM_CUDA_TRY(cudaMemcpy(g.lt, lt.data(), sizeof(LaneDev) * nb, cudaMemcpyHostToDevice));
        if ((st = zsolve_reserve(c, g.slot + nb)) != HELM_OK) return st;   // before capture
    }
    HELM_CUDA_TRY(cudaMalloc(&P->flags, sizeof(int) * P->lanes.size()));
    for (size_t i = 0; i < P->lanes.size(); ++i) P->lanes[i].more = P->flags + i;
    HELM_CUDA_TRY(cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking));
    HELM_CUDA_TRY(cudaGraphCreate(&P->G, 0));
    std::vector<int> prof_on(P->ctxs.size(), 0);
    for (size_t p = 0; p < P->ctxs.size(); ++p)
        if (P->ctxs[p]->prof) { prof_on[p] = P->ctxs[p]->prof->enabled; P->ctxs[p]->prof->enabled = 0; }  // no event nodes
    st = HELM_OK;
    for (size_t i = 0; st == HELM_OK && i < P->groups.size(); ++i)
        st = build_group(P->G, P->groups[i], P->lanes, P->flags + P->groups[i].first, P->cs);
    for (size_t p = 0; p < P->ctxs.size(); ++p)
        if (P->ctxs[p]->prof) P->ctxs[p]->prof->enabled = prof_on[p];
    if (st != HELM_OK) return st;
    const cudaError_t e = cudaGraphInstantiate(&P->X, P->G, 0);
    if (e != cudaSuccess) return helm_fail_cuda(e, "cudaGraphInstantiate");
    return HELM_OK;
}

// one solve of every lane from the current contents of b and x
helm_status plan_run(helm_batch* P, cudaStream_t s) {
    helm_status st;
    std::vector<Lane>& lanes = P->lanes;
    for (helm_ctx* c : P->ctxs) HELM_CUDA_TRY(cudaMemsetAsync(c->status_d, 0, sizeof(unsigned), s));
    for (Lane& ln : lanes) {
        HELM_CUDA_TRY(cudaMemsetAsync(ln.w.nzflag, 0, sizeof(unsigned), s));
        to_df_kernel<<<ln.w.NB, NT, 0, s>>>(ln.b, ln.w.Fdf, ln.c->npts, nullptr);
        to_df_kernel<<<ln.w.NB, NT, 0, s>>>(ln.x, ln.w.xdf, ln.c->npts, ln.w.nzflag);
        HELM_CUDA_TRY(cudaGetLastError());
    }
    std::vector<unsigned> nz(lanes.size(), 0);
    for (size_t i = 0; i < lanes.size(); ++i)
        HELM_CUDA_TRY(cudaMemcpyAsync(&nz[i], lanes[i].w.nzflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    // initial true residuals (r0 = b without a matvec when x0 = 0) and the lane controls
    for (size_t i = 0; i < lanes.size(); ++i) {
        Lane& ln = lanes[i];
        helm_ctx* c = ln.c;
        KrylovWork* k = &ln.w;
        if (nz[i]) {
            if ((st = launch_residual(c, k->xdf, k->Fdf, k->V, k->rpart, s)) != HELM_OK) return st;
        } else {
            residual_zero_kernel<<<k->nres, NT, 0, s>>>(k->Fdf, k->V, c->npts, k->rpart);
        }
        resnorm_kernel<<<1, 256, 0, s>>>(k->rpart, k->nres, k->sigma, k->g, k->m, k->ctrl_d, 1);
        LaneCtl L{};
        L.active = 1;
        L.max_iter = c->opt.max_iter;
        L.m = c->opt.restart;
        L.rtol = c->opt.rtol;
        ln.L_h = L;
        HELM_CUDA_TRY(cudaMemcpyAsync(ln.L_d, &ln.L_h, sizeof(LaneCtl), cudaMemcpyHostToDevice, s));
        HELM_CUDA_TRY(cudaGetLastError());
    }
    // one graph launch per restart cycle while any lane wants another (bounded by the largest iteration limit)
    int max_cycles = 1;
    for (Lane& ln : lanes) max_cycles = std::max(max_cycles, ln.c->opt.max_iter + 1);
    std::vector<int> more(lanes.size(), 1);
    cudaError_t e;
    for (int cyc = 0; cyc <= max_cycles; ++cyc) {
        if ((e = cudaGraphLaunch(P->X, s)) != cudaSuccess) return helm_fail_cuda(e, "cudaGraphLaunch");
        if ((e = cudaMemcpyAsync(more.data(), P->flags, sizeof(int) * lanes.size(), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return helm_fail_cuda(e, "batched restart cycle");
        bool any = false;
        for (int v : more) any = any || v;
        if (!any) break;
    }
    // solutions and controls back
    for (Lane& ln : lanes) {
        from_df_kernel<<<ln.w.NB, NT, 0, s>>>(ln.w.xdf, ln.x, ln.c->npts);
        HELM_CUDA_TRY(cudaMemcpyAsync(ln.w.ctrl_h, ln.w.ctrl_d, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaMemcpyAsync(&ln.L_h, ln.L_d, sizeof(LaneCtl), cudaMemcpyDeviceToHost, s));
    }
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    for (Lane& ln : lanes) ln.ctrl_copy = *ln.w.ctrl_h;
    return HELM_OK;
}

helm_status check_batch_args(helm_ctx* const* ctxs, int nprob, const void* const* b, void* const* x, int nrhs) {
    if (!ctxs || !b || !x || nprob < 1 || nrhs < 1) return HELM_ERR_ARG;
    for (int p = 0; p < nprob; ++p) {
        helm_ctx* c = ctxs[p];
        if (!c || !b[p] || !x[p]) return HELM_ERR_ARG;
        // the high-order closure's padded operands are one per context: lanes of a graph could race on them
        if (c->opt.precond == HELM_PRECOND_PFFT || c->opt.precond == HELM_PRECOND_FFT2 || c->net || c->ho)
            return HELM_ERR_UNSUPPORTED;
        // the 16-bit chains run in the lanes' group iterations only: their z-solves keep per-context state
        // (checkpoint slots, stage norms), which concurrent cycle-end preconditioners of non-flexible lanes
        // would share
        if ((c->opt.precision == HELM_PREC_BF16 || c->opt.precision == HELM_PREC_FP16) && !c->opt.flexible)
            return HELM_ERR_UNSUPPORTED;
        if (!is_device_ptr(b[p]) || !is_device_ptr(x[p])) return HELM_ERR_ARG;
        for (int q = 0; q < p; ++q)
            if (ctxs[q] == c) return HELM_ERR_ARG;   // each context once (its right-hand sides are its lanes)
    }
    return HELM_OK;
}

Lane make_lane(helm_ctx* c, const void* b, void* x, int r, int index) {
    Lane ln;
    ln.c = c;
    ln.b = (double2*)b + (size_t)r * c->npts;
    ln.x = (double2*)x + (size_t)r * c->npts;
    ln.index = index;
    return ln;
}

// per-lane status and info from the lane controls (same rules as helm_gmres_solve)
helm_status lane_info(const Lane& ln, unsigned dstat, double secs, helm_solve_info* inf) {
    const LaneCtl& L = ln.L_h;
    const double beta0 = ln.ctrl_copy.beta0, beta = ln.ctrl_copy.beta;
    helm_status stt;
    if (!(beta0 > 0)) stt = (ln.ctrl_copy.flags & HELM_DEV_NAN) ? HELM_ERR_NAN : HELM_OK;
    else if (beta / beta0 <= ln.c->opt.rtol) stt = HELM_OK;
    else if (ln.ctrl_copy.flags & HELM_DEV_NAN) stt = HELM_ERR_NAN;
    else if (L.brk) stt = HELM_ERR_BREAKDOWN;
    else stt = HELM_ERR_NOT_CONVERGED;
    if (stt == HELM_OK && (dstat & HELM_DEV_PIVOT)) stt = HELM_ERR_PIVOT;
    if (dstat & HELM_DEV_WAIT) stt = HELM_ERR_ITER_LIMIT;
    if (inf) {
        *inf = helm_solve_info{};
        inf->status = stt;
        inf->iterations = L.its;
        inf->restarts = L.restarts;
        inf->relres_true = beta0 > 0 ? beta / beta0 : 0.0;
        inf->relres_est = ln.ctrl_copy.est;
        inf->beta0 = beta0;
        inf->seconds = secs;
        for (int q = 0; q < 16; ++q) inf->cycle_its[q] = L.cyc[q];
    }
    return stt;
}

helm_status fill_infos(const std::vector<Lane>& lanes, const std::vector<helm_ctx*>& ctxs, int nrhs, double secs,
                       helm_solve_info* infos, cudaStream_t s) {
    std::vector<unsigned> dstat(ctxs.size(), 0);
    for (size_t p = 0; p < ctxs.size(); ++p)
        HELM_CUDA_TRY(cudaMemcpyAsync(&dstat[p], ctxs[p]->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    helm_status worst = HELM_OK;
    for (const Lane& ln : lanes) {
        const helm_status stt = lane_info(ln, dstat[ln.index / nrhs], secs, infos ? infos + ln.index : nullptr);
        if (worst == HELM_OK && stt != HELM_OK) worst = stt;
    }
    return worst;
}

}  // namespace

extern "C" helm_status helm_batch_create(helm_ctx* const* ctxs, int nprob, const void* const* b, void* const* x,
                                         int nrhs, void* stream, helm_batch** out) {
    if (!out) return HELM_ERR_ARG;
    *out = nullptr;
    helm_status st = check_batch_args(ctxs, nprob, b, x, nrhs);
    if (st != HELM_OK) return st;
    size_t need = 0;
    for (int p = 0; p < nprob; ++p) need += (size_t)nrhs * lane_bytes(ctxs[p]);
    size_t freeb = 0, totb = 0;
    HELM_CUDA_TRY(cudaMemGetInfo(&freeb, &totb));
    if (need > (size_t)(0.85 * (double)freeb)) return HELM_ERR_NOMEM;
    helm_batch* P = new helm_batch();
    P->nprob = nprob;
    P->nrhs = nrhs;
    for (int p = 0; p < nprob; ++p) {
        P->ctxs.push_back(ctxs[p]);
        for (int r = 0; r < nrhs; ++r) P->lanes.push_back(make_lane(ctxs[p], b[p], x[p], r, p * nrhs + r));
    }
    (void)stream;
    if ((st = plan_build(P)) != HELM_OK) {
        plan_free(P);
        delete P;
        return st;
    }
    *out = P;
    return HELM_OK;
}

extern "C" helm_status helm_batch_run(helm_batch* P, helm_solve_info* infos, void* stream) {
    if (!P) return HELM_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    helm_status st = plan_run(P, s);
    if (st != HELM_OK) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return fill_infos(P->lanes, P->ctxs, P->nrhs, secs, infos, s);
}

extern "C" void helm_batch_destroy(helm_batch* P) {
    if (!P) return;
    plan_free(P);
    delete P;
}

extern "C" helm_status helm_gmres_solve_batched(helm_ctx* const* ctxs, int nprob, const void* const* b, void* const* x,
                                                int nrhs, helm_solve_info* infos, void* stream) {
    helm_status st = check_batch_args(ctxs, nprob, b, x, nrhs);
    if (st != HELM_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Lane> all;
    for (int p = 0; p < nprob; ++p)
        for (int r = 0; r < nrhs; ++r) all.push_back(make_lane(ctxs[p], b[p], x[p], r, p * nrhs + r));
    // groups by workspace size, largest lanes first, each fitting in 60% of the free memory
    std::vector<size_t> order(all.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return all[a].c->npts > all[c].c->npts; });
    size_t freeb = 0, totb = 0;
    HELM_CUDA_TRY(cudaMemGetInfo(&freeb, &totb));
    const size_t budget = (size_t)(0.6 * (double)freeb);
    std::vector<Lane> done;
    size_t i = 0;
    while (i < order.size()) {
        helm_batch P;
        size_t used = 0;
        while (i < order.size() && (P.lanes.empty() || used + lane_bytes(all[order[i]].c) <= budget)) {
            used += lane_bytes(all[order[i]].c);
            P.lanes.push_back(all[order[i++]]);
        }
        for (Lane& ln : P.lanes)
            if (std::find(P.ctxs.begin(), P.ctxs.end(), ln.c) == P.ctxs.end()) P.ctxs.push_back(ln.c);
        st = plan_build(&P);
        if (st == HELM_OK) st = plan_run(&P, s);
        for (Lane& ln : P.lanes) {
            Lane d = ln;
            d.w = KrylovWork();
            d.tmp = nullptr; d.L_d = nullptr; d.more = nullptr;
            done.push_back(d);
        }
        plan_free(&P);
        if (st != HELM_OK) return st;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::vector<helm_ctx*> cv(ctxs, ctxs + nprob);
    return fill_infos(done, cv, nrhs, secs, infos, s);
}
