// Learned correction (an extension of the method, not in the paper): a small 3D U-Net N applied after
// the EigT preconditioner inside flexible GMRES,
//     c = s * N( v/RMS(v), M^-1 v/s, Re(k^2/k0^2) - 1 ),    s = RMS(M^-1 v),
//     z = M^-1 v + alpha c,   alpha = <A c, v - A M^-1 v> / <A c, A c>  (complex, minimises |v - A z|_2),
// trained on (residual, error) pairs of the solver's own solves.  The minimal-residual step makes plain
// EigT the fallback: |v - A z| <= |v - A M^-1 v| for any network output, alpha -> 0 for a useless one,
// and the correction is dropped (z = M^-1 v) when A c vanishes or any of the sums is not finite.
//
// Network (width c):  a1 = relu(conv(x, 5->c)), a2 = relu(conv(a1, c->c)), p = avgpool2(a2),
// b1 = relu(conv(p, c->2c)), b2 = relu(conv(b1, 2c->2c)), u = [upsample2(b2), a2],
// d1 = relu(conv(u, 3c->c)), y = conv(d1, c->2).  3x3x3 convolutions, zero padding, stride 1.
// Activations and weights are stored in BF16, every product is accumulated in FP32; training keeps FP32
// master weights, FP32 activation gradients and Adam moments.  Layout [B][C][Z][Y][X].
//
// Kernels: the 3x3x3 convolutions run on the tcgen05 tensor cores as implicit GEMMs (conv_tc.cu: forward
// and data gradient through flipped/transposed weights with the ReLU mask fused, weight gradient with the
// taps' accumulators in tensor memory) whenever a layer has at most 64 outputs (widths up to 32); wider
// layers take the direct kernels written here (a shared-memory halo tile per input channel, and the
// weight gradient as a tiled reduction with one atomic per CTA and tap).  Also here: pooling/upsampling and
// their adjoints, MSE, Adam, feature assembly and the correction step.
#include "common.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

typedef __nv_bfloat16 bf16;

struct helm_net {
    int c = 0;
    size_t nparam = 0;
    float *W = nullptr, *G = nullptr, *Mom = nullptr, *Vel = nullptr;   // fp32 master weights, grads, Adam
    bf16* Wb = nullptr;                                                 // bf16 copy
    size_t woff[6], boff[6];
    int co[6], ci[6];
    // activation workspace for B x Z x Y x X
    size_t cap = 0;   // inference capacity in (B * vol) points
    size_t gcap = 0;  // gradient-buffer capacity
    int B = 0, Z = 0, Y = 0, X = 0;
    bf16 *x = nullptr, *a1 = nullptr, *u = nullptr, *d1 = nullptr;      // full resolution (u holds [up(b2), a2])
    bf16 *p = nullptr, *b1 = nullptr, *b2 = nullptr;                    // half resolution
    float* y = nullptr;
    float *gA = nullptr, *gB = nullptr, *gU = nullptr, *gH1 = nullptr, *gH2 = nullptr;   // gradient buffers
    // statistics and reduction scratch (16 doubles): 0 sum|v|^2, 1 sum|M^-1 v|^2, 2 |alpha| of the last
    // correction, 3 corrections dropped, 4 corrections applied, 5 sum over applied corrections of
    // |v - A z|^2/|v - A M^-1 v|^2, 6-7 <Ac, rho>, 8 |Ac|^2, 9 |rho|^2, 15 scratch of helm_net_target
    double* stats = nullptr;
    // solver-side fields (complex64, one grid): v = sigma r, c, A M^-1 v, A c
    float2 *vbuf = nullptr, *cbuf = nullptr, *az0 = nullptr, *ac = nullptr;
    size_t fcap = 0;
    bf16* wscr = nullptr;          // weights arranged for the tensor-core convolutions (one layer at a time)
    unsigned* status = nullptr;    // device status word of the network's own calls (bounded waits)
};

// conv_tc.cu
bool conv_tc_supported(int Cin, int Cout);
bool wgrad_tc_supported(int Cin, int Cout);
size_t conv_tc_scratch_bytes(int Cin, int Cout);
helm_status conv_tc_prepare();
template <typename TIN, typename TOUT>
helm_status conv_tc(const TIN* in, int Cin, size_t in_bs, const __nv_bfloat16* w, int wmode, const float* bias,
                    TOUT* out, int Cout, size_t out_bs, int B, int Z, int Y, int X, int relu,
                    const __nv_bfloat16* mask, size_t mask_bs, __nv_bfloat16* wscr, unsigned* status, cudaStream_t s);
helm_status wgrad_tc(const __nv_bfloat16* in, int Cin, size_t in_bs, const float* g, int Cout, size_t g_bs, int B, int Z,
                     int Y, int X, float* gw, float* gb, unsigned* status, cudaStream_t s);

namespace {

constexpr int TXC = 8, TYC = 8, TZC = 4;      // output tile of the convolution (256 threads)
constexpr int COT = 8;                        // output channels per CTA

__device__ __forceinline__ float ld(const bf16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ void st(bf16* p, size_t i, float v) { p[i] = __float2bfloat16(v); }
__device__ __forceinline__ void st(float* p, size_t i, float v) { p[i] = v; }

// out[b][o][q] = act( bias[o] + sum_{i,t} W(o,i,t) in[b][i][q + off_t] ),  zero padding.
// W(o,i,t) = w[(o*Cin + i)*27 + t] (wmode 0) or w[(i*Cout + o)*27 + 26 - t] (wmode 1: data gradient).
// mask (optional): out *= (mask[b][o][q] > 0), for the ReLU of the layer whose gradient this is.
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) conv3_kernel(const TIN* __restrict__ in, int Cin, size_t in_bs,
                                                    const bf16* __restrict__ w, int wmode,
                                                    const float* __restrict__ bias, TOUT* __restrict__ out, int Cout,
                                                    size_t out_bs, int Z, int Y, int X, int relu,
                                                    const bf16* __restrict__ mask, size_t mask_bs) {
    __shared__ float tile[(TZC + 2) * (TYC + 2) * (TXC + 2)];
    __shared__ float wsm[COT * 27];
    const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tz = threadIdx.x >> 6;
    const int ntx = (X + TXC - 1) / TXC;
    const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
    const int x0 = bx * TXC, y0 = by * TYC, z0 = blockIdx.y * TZC;
    const int nco = (Cout + COT - 1) / COT;
    const int b = blockIdx.z / nco, o0 = (blockIdx.z % nco) * COT;
    const size_t vol = (size_t)Z * Y * X;
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    float acc[COT];
#pragma unroll
    for (int o = 0; o < COT; ++o) acc[o] = 0.f;
    const TIN* inb = in + (size_t)b * in_bs;
    for (int i = 0; i < Cin; ++i) {
        __syncthreads();
        const TIN* ch = inb + (size_t)i * vol;
        for (int q = threadIdx.x; q < (TZC + 2) * (TYC + 2) * (TXC + 2); q += 256) {
            const int lx = q % (TXC + 2), ly = (q / (TXC + 2)) % (TYC + 2), lz = q / ((TXC + 2) * (TYC + 2));
            const int X_ = x0 + lx - 1, Y_ = y0 + ly - 1, Z_ = z0 + lz - 1;
            float v = 0.f;
            if (X_ >= 0 && X_ < X && Y_ >= 0 && Y_ < Y && Z_ >= 0 && Z_ < Z) v = ld(ch, ((size_t)Z_ * Y + Y_) * X + X_);
            tile[q] = v;
        }
        for (int q = threadIdx.x; q < COT * 27; q += 256) {
            const int o = q / 27, t = q - o * 27;
            float v = 0.f;
            if (o0 + o < Cout)
                v = __bfloat162float(wmode ? w[((size_t)i * Cout + o0 + o) * 27 + 26 - t] : w[((size_t)(o0 + o) * Cin + i) * 27 + t]);
            wsm[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
            const float v = tile[((tz + dz) * (TYC + 2) + ty + dy) * (TXC + 2) + tx + dx];
#pragma unroll
            for (int o = 0; o < COT; ++o) acc[o] = fmaf(wsm[o * 27 + t], v, acc[o]);
        }
    }
    if (gx >= X || gy >= Y || gz >= Z) return;
    const size_t q = ((size_t)gz * Y + gy) * X + gx;
#pragma unroll
    for (int o = 0; o < COT; ++o) {
        if (o0 + o >= Cout) break;
        float v = acc[o] + (bias ? bias[o0 + o] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        if (mask && !(__bfloat162float(mask[(size_t)b * mask_bs + (size_t)(o0 + o) * vol + q]) > 0.f)) v = 0.f;
        st(out, (size_t)b * out_bs + (size_t)(o0 + o) * vol + q, v);
    }
}

// gw[o][i][t] += sum_{b,q} g[b][o][q] in[b][i][q + off_t];  gb[o] += sum g  (one atomic per CTA and tap)
__global__ void __launch_bounds__(256) conv3_wgrad_kernel(const bf16* __restrict__ in, int Cin, size_t in_bs,
                                                          const float* __restrict__ g, int Cout, size_t g_bs, int B,
                                                          int Z, int Y, int X, float* __restrict__ gw,
                                                          float* __restrict__ gb) {
    __shared__ float tile[(TZC + 2) * (TYC + 2) * (TXC + 2)];
    __shared__ float gt[COT][TZC * TYC * TXC];
    const int i = blockIdx.x;
    const int o0 = blockIdx.y * COT;
    const int ntx = (X + TXC - 1) / TXC, nty = (Y + TYC - 1) / TYC, ntz = (Z + TZC - 1) / TZC;
    const int ntiles = B * ntx * nty * ntz;
    const size_t vol = (size_t)Z * Y * X;
    // thread -> (o, t) pair; 8 x 27 = 216 active
    const int o = threadIdx.x / 27, t = threadIdx.x - o * 27;
    const bool act = threadIdx.x < COT * 27 && o0 + o < Cout;
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    float acc = 0.f, accb = 0.f;
    for (int tile_id = blockIdx.z; tile_id < ntiles; tile_id += gridDim.z) {
        int r = tile_id;
        const int bx = r % ntx; r /= ntx;
        const int by = r % nty; r /= nty;
        const int bz = r % ntz; r /= ntz;
        const int b = r;
        const int x0 = bx * TXC, y0 = by * TYC, z0 = bz * TZC;
        __syncthreads();
        const bf16* ch = in + (size_t)b * in_bs + (size_t)i * vol;
        for (int q = threadIdx.x; q < (TZC + 2) * (TYC + 2) * (TXC + 2); q += 256) {
            const int lx = q % (TXC + 2), ly = (q / (TXC + 2)) % (TYC + 2), lz = q / ((TXC + 2) * (TYC + 2));
            const int X_ = x0 + lx - 1, Y_ = y0 + ly - 1, Z_ = z0 + lz - 1;
            float v = 0.f;
            if (X_ >= 0 && X_ < X && Y_ >= 0 && Y_ < Y && Z_ >= 0 && Z_ < Z) v = ld(ch, ((size_t)Z_ * Y + Y_) * X + X_);
            tile[q] = v;
        }
        for (int q = threadIdx.x; q < COT * TZC * TYC * TXC; q += 256) {
            const int oo = q / (TZC * TYC * TXC), pp = q - oo * (TZC * TYC * TXC);
            const int lx = pp % TXC, ly = (pp / TXC) % TYC, lz = pp / (TXC * TYC);
            const int X_ = x0 + lx, Y_ = y0 + ly, Z_ = z0 + lz;
            float v = 0.f;
            if (o0 + oo < Cout && X_ < X && Y_ < Y && Z_ < Z)
                v = g[(size_t)b * g_bs + (size_t)(o0 + oo) * vol + ((size_t)Z_ * Y + Y_) * X + X_];
            gt[oo][pp] = v;
        }
        __syncthreads();
        if (act) {
            for (int pp = 0; pp < TZC * TYC * TXC; ++pp) {
                const int lx = pp % TXC, ly = (pp / TXC) % TYC, lz = pp / (TXC * TYC);
                const float gv = gt[o][pp];
                acc = fmaf(gv, tile[((lz + dz) * (TYC + 2) + ly + dy) * (TXC + 2) + lx + dx], acc);
                if (t == 0 && i == 0) accb += gv;
            }
        }
    }
    if (act) {
        atomicAdd(&gw[((size_t)(o0 + o) * Cin + i) * 27 + t], acc);
        if (t == 0 && i == 0) atomicAdd(&gb[o0 + o], accb);
    }
}

__global__ void avgpool2_kernel(const bf16* __restrict__ in, size_t in_bs, bf16* __restrict__ out, int C, int B,
                                int Z, int Y, int X) {
    const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
    const size_t n = (size_t)B * C * Zh * Yh * Xh;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        size_t r = id;
        const int x = r % Xh; r /= Xh;
        const int y = r % Yh; r /= Yh;
        const int z = r % Zh; r /= Zh;
        const int c = r % C; const int b = (int)(r / C);
        const bf16* s = in + (size_t)b * in_bs + (size_t)c * Z * Y * X;
        float acc = 0.f;
        for (int k = 0; k < 8; ++k)
            acc += ld(s, ((size_t)(2 * z + (k >> 2)) * Y + 2 * y + ((k >> 1) & 1)) * X + 2 * x + (k & 1));
        out[id] = __float2bfloat16(0.125f * acc);
    }
}

// out (full res, channels 0..C-1 of a [B][Cu] buffer) = upsample2(in): one thread per pair of output points
// (x even, x + 1) of a row, which share their source value; grid.x = (x block, y, z), grid.y = (b, c)
__global__ void upsample2_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, size_t out_bs, int C, int B,
                                 int Z, int Y, int X) {
    const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
    const int nxb = (Xh + blockDim.x - 1) / blockDim.x;
    int r = blockIdx.x;
    const int xh = (r % nxb) * blockDim.x + threadIdx.x;
    r /= nxb;
    const int y = r % Y, z = r / Y;
    if (xh >= Xh) return;
    const int c = blockIdx.y % C, b = blockIdx.y / C;
    const bf16 v = in[(((size_t)b * C + c) * Zh + z / 2) * ((size_t)Yh * Xh) + (size_t)(y / 2) * Xh + xh];
    __nv_bfloat162 two;
    two.x = v;
    two.y = v;
    bf16* o = out + (size_t)b * out_bs + (size_t)c * Z * Y * X + ((size_t)z * Y + y) * X + 2 * xh;
    *reinterpret_cast<__nv_bfloat162*>(o) = two;
}

// g_half[b][c] = mask(b2 > 0) * sum of the 8 children of gu[b][c] (adjoint of upsample2)
__global__ void upsample2_adj_kernel(const float* __restrict__ gu, size_t gu_bs, const bf16* __restrict__ mask,
                                     float* __restrict__ gh, int C, int B, int Z, int Y, int X) {
    const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
    const size_t n = (size_t)B * C * Zh * Yh * Xh;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        size_t r = id;
        const int x = r % Xh; r /= Xh;
        const int y = r % Yh; r /= Yh;
        const int z = r % Zh; r /= Zh;
        const int c = r % C; const int b = (int)(r / C);
        const float* s = gu + (size_t)b * gu_bs + (size_t)c * Z * Y * X;
        float acc = 0.f;
        for (int k = 0; k < 8; ++k)
            acc += s[((size_t)(2 * z + (k >> 2)) * Y + 2 * y + ((k >> 1) & 1)) * X + 2 * x + (k & 1)];
        gh[id] = (__bfloat162float(mask[id]) > 0.f) ? acc : 0.f;
    }
}

// ga2 = mask(a2 > 0) * (gu_a2 + upsample2(gp)/8)   (adjoint of avgpool2 added to the skip gradient)
__global__ void skip_grad_kernel(const float* __restrict__ gu_a2, size_t gu_bs, const float* __restrict__ gp,
                                 const bf16* __restrict__ a2, size_t a2_bs, float* __restrict__ ga2, int C, int B,
                                 int Z, int Y, int X) {
    const size_t vol = (size_t)Z * Y * X;
    const size_t n = (size_t)B * C * vol;
    const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        size_t r = id;
        const int x = r % X; r /= X;
        const int y = r % Y; r /= Y;
        const int z = r % Z; r /= Z;
        const int c = r % C; const int b = (int)(r / C);
        const size_t q = ((size_t)z * Y + y) * X + x;
        float v = gu_a2[(size_t)b * gu_bs + (size_t)c * vol + q] +
                  0.125f * gp[(((size_t)b * C + c) * Zh + z / 2) * Yh * Xh + (size_t)(y / 2) * Xh + x / 2];
        if (!(__bfloat162float(a2[(size_t)b * a2_bs + (size_t)c * vol + q]) > 0.f)) v = 0.f;
        ga2[id] = v;
    }
}

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g, size_t n,
                           double* __restrict__ loss) {
    __shared__ double red[8];
    double s = 0;
    const float inv = 1.f / (float)n;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float d = y[id] - t[id];
        g[id] = d * inv;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        atomicAdd(loss, 0.5 * tot / (double)n);
    }
}

__global__ void adam_kernel(float* W, const float* G, float* M, float* V, bf16* Wb, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= n) return;
    const float g = G[id];
    const float m = b1 * M[id] + (1.f - b1) * g;
    const float v = b2 * V[id] + (1.f - b2) * g * g;
    M[id] = m;
    V[id] = v;
    const float w = W[id] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    W[id] = w;
    Wb[id] = __float2bfloat16(w);
}

__global__ void to_bf16_kernel(const float* a, bf16* b, size_t n) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id < n) b[id] = __float2bfloat16(a[id]);
}

// acc[slot] += sum |v|^2 (FP64 partials)
__global__ void sumsq_kernel(const float2* __restrict__ v, size_t n, double* acc) {
    __shared__ double r[8];
    double s = 0;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float2 a = v[id];
        s += (double)a.x * a.x + (double)a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += r[w];
        atomicAdd(acc, t);
    }
}

// x[c0] = Re(v)/rms(v), x[c0+1] = Im(v)/rms(v)  (rms from the sum of squares in *acc); bf16 planes of n
__global__ void feat_pair_kernel(const float2* __restrict__ v, const double* __restrict__ acc, size_t n,
                                 bf16* __restrict__ x0, bf16* __restrict__ x1) {
    const float iv = acc[0] > 0 ? (float)(1.0 / sqrt(acc[0] / (double)n)) : 0.f;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float2 a = v[id];
        x0[id] = __float2bfloat16(a.x * iv);
        x1[id] = __float2bfloat16(a.y * iv);
    }
}

// x = Re(k^2)/k0^2 - 1
__global__ void feat_contrast_kernel(const float2* __restrict__ k2, float ik02, size_t n, bf16* __restrict__ x) {
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        x[id] = __float2bfloat16(k2[id].x * ik02 - 1.f);
}

// x0 = Re(r)/rms(r), x1 = Im(r)/rms(r) (bf16) and v = sigma[sidx] r (the vector M^-1 is applied to)
__global__ void feat_v_kernel(const float2* __restrict__ r, const double* __restrict__ acc, size_t n,
                              bf16* __restrict__ x0, bf16* __restrict__ x1, const double* __restrict__ sigma, int sidx,
                              float2* __restrict__ v) {
    const float iv = acc[0] > 0 ? (float)(1.0 / sqrt(acc[0] / (double)n)) : 0.f;
    const float sg = sigma ? (float)sigma[sidx] : 1.f;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float2 a = r[id];
        x0[id] = __float2bfloat16(a.x * iv);
        x1[id] = __float2bfloat16(a.y * iv);
        v[id] = make_float2(a.x * sg, a.y * sg);
    }
}

// c = s (y_re + i y_im), s = sqrt(acc[1]/n) = RMS(M^-1 v)
__global__ void make_c_kernel(const float* __restrict__ y, const double* __restrict__ acc, size_t n,
                              float2* __restrict__ c) {
    const float s = (float)sqrt(acc[1] / (double)n);
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        c[id] = make_float2(s * y[id], s * y[n + id]);
}

// rho = v - A z0:  acc[6..7] += <Ac, rho> = sum conj(Ac) rho,  acc[8] += |Ac|^2,  acc[9] += |rho|^2
__global__ void mr_dots_kernel(const float2* __restrict__ v, const float2* __restrict__ az0,
                               const float2* __restrict__ ac, size_t n, double* __restrict__ acc) {
    __shared__ double red[4][8];
    double pr = 0, pi = 0, q = 0, rr = 0;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float2 a = ac[id], b = v[id], z = az0[id];
        const double rx = (double)b.x - z.x, ry = (double)b.y - z.y;
        pr += (double)a.x * rx + (double)a.y * ry;
        pi += (double)a.x * ry - (double)a.y * rx;
        q += (double)a.x * a.x + (double)a.y * a.y;
        rr += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) {
        pr += __shfl_down_sync(0xffffffffu, pr, o);
        pi += __shfl_down_sync(0xffffffffu, pi, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
        rr += __shfl_down_sync(0xffffffffu, rr, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = pr; red[1][w] = pi; red[2][w] = q; red[3][w] = rr; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
        atomicAdd(&acc[6 + threadIdx.x], t);
    }
}

// z += alpha c with alpha = acc[6..7]/acc[8]; dropped when |Ac| = 0 or a sum is not finite
__global__ void mr_apply_kernel(const float2* __restrict__ c, double* __restrict__ acc, size_t n,
                                float2* __restrict__ z) {
    const double pr = acc[6], pi = acc[7], q = acc[8], rr = acc[9];
    const bool ok = q > 0 && isfinite(q) && isfinite(pr) && isfinite(pi) && isfinite(rr);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ok) {
            acc[2] = sqrt(pr * pr + pi * pi) / q;
            acc[4] += 1.0;
            acc[5] += rr > 0 ? fmax(0.0, rr - (pr * pr + pi * pi) / q) / rr : 1.0;
        } else {
            acc[2] = 0.0;
            acc[3] += 1.0;
        }
    }
    if (!ok) return;
    const float ar = (float)(pr / q), ai = (float)(pi / q);
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const float2 a = c[id];
        float2 b = z[id];
        b.x += ar * a.x - ai * a.y;
        b.y += ar * a.y + ai * a.x;
        z[id] = b;
    }
}

// t = (xs - xk - mv)/rms(mv): the training target of the network for v = b - A xk, whose exact
// preconditioned image is A^-1 v = xs - xk (xs the converged solution); complex128 xs, xk
__global__ void target_kernel(const double2* __restrict__ xs, const double2* __restrict__ xk,
                              const float2* __restrict__ mv, const double* __restrict__ acc, size_t n,
                              float* __restrict__ t) {
    const double is = acc[0] > 0 ? 1.0 / sqrt(acc[0] / (double)n) : 0.0;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const double2 a = xs[id], b = xk[id];
        const float2 m = mv[id];
        t[id] = (float)((a.x - b.x - (double)m.x) * is);
        t[n + id] = (float)((a.y - b.y - (double)m.y) * is);
    }
}

unsigned nblk(size_t n) { const size_t b = (n + 255) / 256; return (unsigned)(b > 4096 ? 4096 : b); }

// the convolution of a layer: tensor cores where the shape allows, else the direct kernel
template <typename TIN, typename TOUT>
void conv(helm_net* n, const TIN* in, int Cin, size_t in_bs, const bf16* w, int wmode, const float* bias, TOUT* out,
          int Cout, size_t out_bs, int B, int Z, int Y, int X, int relu, const bf16* mask, size_t mask_bs,
          unsigned* status, cudaStream_t s) {
    if (conv_tc_supported(Cin, Cout)) {
        conv_tc<TIN, TOUT>(in, Cin, in_bs, w, wmode, bias, out, Cout, out_bs, B, Z, Y, X, relu, mask, mask_bs, n->wscr,
                           status, s);
        return;
    }
    const int ntx = (X + TXC - 1) / TXC, nty = (Y + TYC - 1) / TYC, ntz = (Z + TZC - 1) / TZC;
    dim3 grid(ntx * nty, ntz, B * ((Cout + COT - 1) / COT));
    conv3_kernel<TIN, TOUT><<<grid, 256, 0, s>>>(in, Cin, in_bs, w, wmode, bias, out, Cout, out_bs, Z, Y, X, relu, mask,
                                                mask_bs);
}

void wgrad(helm_net* n, const bf16* in, int Cin, size_t in_bs, const float* g, int Cout, size_t g_bs, int B, int Z,
           int Y, int X, float* gw, float* gb, cudaStream_t s) {
    if (wgrad_tc_supported(Cin, Cout)) {
        wgrad_tc(in, Cin, in_bs, g, Cout, g_bs, B, Z, Y, X, gw, gb, n->status, s);
        return;
    }
    dim3 grid(Cin, (Cout + COT - 1) / COT, 16);
    conv3_wgrad_kernel<<<grid, 256, 0, s>>>(in, Cin, in_bs, g, Cout, g_bs, B, Z, Y, X, gw, gb);
}

void free_bufs(void** ps, int n) {
    for (int i = 0; i < n; ++i) {
        if (ps[i]) cudaFree(ps[i]);
    }
}

// inference workspace for B x Z x Y x X (grown on demand, never shrunk)
helm_status ensure_ws(helm_net* n, int B, int Z, int Y, int X) {
    if (B < 1 || Z < 2 || Y < 2 || X < 2 || Z % 2 || Y % 2 || X % 2) return HELM_ERR_ARG;
    const size_t pts = (size_t)B * Z * Y * X;
    n->B = B; n->Z = Z; n->Y = Y; n->X = X;
    if (pts <= n->cap) return HELM_OK;
    void* ps[] = {n->x, n->a1, n->u, n->d1, n->p, n->b1, n->b2, n->y};
    free_bufs(ps, 8);
    n->x = n->a1 = n->u = n->d1 = n->p = n->b1 = n->b2 = nullptr;
    n->y = nullptr;
    n->cap = 0;
    const size_t c = n->c, h = pts / 8;
    auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    const bool ok = A((void**)&n->x, 5 * pts * 2) && A((void**)&n->a1, c * pts * 2) && A((void**)&n->u, 3 * c * pts * 2) &&
                    A((void**)&n->d1, c * pts * 2) && A((void**)&n->p, c * h * 2) && A((void**)&n->b1, 2 * c * h * 2) &&
                    A((void**)&n->b2, 2 * c * h * 2) && A((void**)&n->y, 2 * pts * 4);
    if (!ok) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    n->cap = pts;
    return HELM_OK;
}

// gradient workspace for the current B x Z x Y x X (training only)
helm_status ensure_grad_ws(helm_net* n) {
    const size_t pts = (size_t)n->B * n->Z * n->Y * n->X;
    if (pts <= n->gcap) return HELM_OK;
    void* ps[] = {n->gA, n->gB, n->gU, n->gH1, n->gH2};
    free_bufs(ps, 5);
    n->gA = n->gB = n->gU = n->gH1 = n->gH2 = nullptr;
    n->gcap = 0;
    const size_t c = n->c, h = pts / 8;
    auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    const bool ok = A((void**)&n->gA, c * pts * 4) && A((void**)&n->gB, c * pts * 4) && A((void**)&n->gU, 3 * c * pts * 4) &&
                    A((void**)&n->gH1, 2 * c * h * 4) && A((void**)&n->gH2, 2 * c * h * 4);
    if (!ok) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    n->gcap = pts;
    return HELM_OK;
}

// forward of the workspace input n->x into n->y (bounded-wait failures OR-ed into *status)
void forward(helm_net* n, unsigned* status, cudaStream_t s) {
    const int c = n->c, B = n->B, Z = n->Z, Y = n->Y, X = n->X;
    const size_t vol = (size_t)Z * Y * X, hv = vol / 8;
    const bf16* W = n->Wb;
    const float* F = n->W;
    bf16* a2 = n->u + 2 * c * vol;   // skip channels live inside u
    conv<bf16, bf16>(n, n->x, 5, 5 * vol, W + n->woff[0], 0, F + n->boff[0], n->a1, c, c * vol, B, Z, Y, X, 1, nullptr, 0, status, s);
    conv<bf16, bf16>(n, n->a1, c, c * vol, W + n->woff[1], 0, F + n->boff[1], a2, c, 3 * c * vol, B, Z, Y, X, 1, nullptr, 0, status, s);
    avgpool2_kernel<<<nblk(B * c * hv), 256, 0, s>>>(a2, 3 * c * vol, n->p, c, B, Z, Y, X);
    conv<bf16, bf16>(n, n->p, c, c * hv, W + n->woff[2], 0, F + n->boff[2], n->b1, 2 * c, 2 * c * hv, B, Z / 2, Y / 2, X / 2, 1,
                     nullptr, 0, status, s);
    conv<bf16, bf16>(n, n->b1, 2 * c, 2 * c * hv, W + n->woff[3], 0, F + n->boff[3], n->b2, 2 * c, 2 * c * hv, B, Z / 2, Y / 2,
                     X / 2, 1, nullptr, 0, status, s);
    upsample2_kernel<<<dim3((unsigned)((X / 2 + 127) / 128 * Y * Z), (unsigned)(B * 2 * c)), 128, 0, s>>>(
        n->b2, n->u, 3 * c * vol, 2 * c, B, Z, Y, X);
    conv<bf16, bf16>(n, n->u, 3 * c, 3 * c * vol, W + n->woff[4], 0, F + n->boff[4], n->d1, c, c * vol, B, Z, Y, X, 1, nullptr,
                     0, status, s);
    conv<bf16, float>(n, n->d1, c, c * vol, W + n->woff[5], 0, F + n->boff[5], n->y, 2, 2 * vol, B, Z, Y, X, 0, nullptr, 0, status, s);
}

}  // namespace

helm_status ensure_field_ws(helm_net* n, size_t npts);

extern "C" {

size_t helm_net_num_params(const helm_net* n) { return n ? n->nparam : 0; }

helm_status helm_net_create(int width, unsigned long long seed, helm_net** out) {
    if (!out) return HELM_ERR_ARG;
    *out = nullptr;   // on every error return
    if (width < 1 || width > 64) return HELM_ERR_ARG;
    helm_net* n = new helm_net();
    n->c = width;
    const int c = width;
    const int co[6] = {c, c, 2 * c, 2 * c, c, 2}, ci[6] = {5, c, c, 2 * c, 3 * c, c};
    size_t off = 0;
    for (int l = 0; l < 6; ++l) {
        n->co[l] = co[l]; n->ci[l] = ci[l];
        n->woff[l] = off; off += (size_t)co[l] * ci[l] * 27;
        n->boff[l] = off; off += co[l];
    }
    n->nparam = off;
    std::vector<float> h(off, 0.f);
    unsigned long long st = seed * 2862933555777941757ull + 3037000493ull;
    auto rnd = [&]() {   // splitmix64 -> uniform (0,1)
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < 6; ++l) {
        const double std = sqrt(2.0 / (27.0 * ci[l])) * (l == 5 ? 0.1 : 1.0);
        for (size_t k = 0; k < (size_t)co[l] * ci[l] * 27; ++k) {
            const double u1 = rnd(), u2 = rnd();
            h[n->woff[l] + k] = (float)(std * sqrt(-2.0 * log(u1)) * cos(2 * M_PI * u2));
        }
    }
    size_t scr = 0;   // arranged weights of the largest layer, in either direction
    for (int l = 0; l < 6; ++l) {
        scr = std::max(scr, conv_tc_scratch_bytes(ci[l], co[l]));
        scr = std::max(scr, conv_tc_scratch_bytes(co[l], ci[l]));
    }
    bool ok = cudaMalloc(&n->W, off * 4) == cudaSuccess && cudaMalloc(&n->G, off * 4) == cudaSuccess &&
              cudaMalloc(&n->Mom, off * 4) == cudaSuccess && cudaMalloc(&n->Vel, off * 4) == cudaSuccess &&
              cudaMalloc(&n->Wb, off * 2) == cudaSuccess && cudaMalloc(&n->stats, 16 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&n->wscr, scr) == cudaSuccess && cudaMalloc(&n->status, sizeof(unsigned)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); helm_net_destroy(n); return HELM_ERR_NOMEM; }
    cudaMemcpy(n->W, h.data(), off * 4, cudaMemcpyHostToDevice);
    cudaMemset(n->G, 0, off * 4);
    cudaMemset(n->Mom, 0, off * 4);
    cudaMemset(n->Vel, 0, off * 4);
    cudaMemset(n->stats, 0, 16 * sizeof(double));
    cudaMemset(n->status, 0, sizeof(unsigned));
    if (conv_tc_prepare() != HELM_OK) { cudaGetLastError(); helm_net_destroy(n); return HELM_ERR_CUDA; }
    to_bf16_kernel<<<(unsigned)((off + 255) / 256), 256>>>(n->W, n->Wb, off);
    if (cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); helm_net_destroy(n); return HELM_ERR_CUDA; }
    *out = n;
    return HELM_OK;
}

void helm_net_destroy(helm_net* n) {
    if (!n) return;
    void* ps[] = {n->W, n->G, n->Mom, n->Vel, n->Wb, n->stats, n->x, n->a1, n->u, n->d1, n->p, n->b1, n->b2, n->y,
                  n->gA, n->gB, n->gU, n->gH1, n->gH2, n->vbuf, n->cbuf, n->az0, n->ac, n->wscr, n->status};
    for (void* p : ps) if (p) cudaFree(p);
    delete n;
}

helm_status helm_net_set_params(helm_net* n, const float* host, size_t count) {
    if (!n || !host || count != n->nparam) return HELM_ERR_ARG;
    HELM_CUDA_TRY(cudaMemcpy(n->W, host, count * 4, cudaMemcpyHostToDevice));
    to_bf16_kernel<<<(unsigned)((count + 255) / 256), 256>>>(n->W, n->Wb, count);
    HELM_CUDA_TRY(cudaDeviceSynchronize());
    return HELM_OK;
}

helm_status helm_net_get_params(helm_net* n, float* host, size_t count) {
    if (!n || !host || count != n->nparam) return HELM_ERR_ARG;
    HELM_CUDA_TRY(cudaMemcpy(host, n->W, count * 4, cudaMemcpyDeviceToHost));
    return HELM_OK;
}

helm_status helm_net_get_grads(helm_net* n, float* host, size_t count) {
    if (!n || !host || count != n->nparam) return HELM_ERR_ARG;
    HELM_CUDA_TRY(cudaMemcpy(host, n->G, count * 4, cudaMemcpyDeviceToHost));
    unsigned st = 0;
    HELM_CUDA_TRY(cudaMemcpy(&st, n->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & HELM_DEV_WAIT) return HELM_ERR_ITER_LIMIT;
    return HELM_OK;
}

helm_status helm_net_zero_grad(helm_net* n, void* stream) {
    if (!n) return HELM_ERR_ARG;
    HELM_CUDA_TRY(cudaMemsetAsync(n->G, 0, n->nparam * 4, (cudaStream_t)stream));
    return HELM_OK;
}

helm_status helm_net_forward(helm_net* n, const void* x, float* y, int B, int Z, int Y, int X, void* stream) {
    if (!n || !x || !y || B < 1) return HELM_ERR_ARG;
    helm_status st = ensure_ws(n, B, Z, Y, X);
    if (st != HELM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pts = (size_t)B * Z * Y * X;
    HELM_CUDA_TRY(cudaMemcpyAsync(n->x, x, 5 * pts * 2, cudaMemcpyDeviceToDevice, s));
    forward(n, n->status, s);
    HELM_CUDA_TRY(cudaMemcpyAsync(y, n->y, 2 * pts * 4, cudaMemcpyDeviceToDevice, s));
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_net_backward(helm_net* n, const float* gy, void* stream) {
    if (!n || !gy || !n->cap) return HELM_ERR_ARG;
    helm_status st = ensure_grad_ws(n);
    if (st != HELM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int c = n->c, B = n->B, Z = n->Z, Y = n->Y, X = n->X;
    const size_t vol = (size_t)Z * Y * X, hv = vol / 8;
    const bf16* W = n->Wb;
    float* G = n->G;
    const bf16* a2 = n->u + 2 * c * vol;
    // layer 6 (linear): d1 gradient with the ReLU mask of d1
    wgrad(n, n->d1, c, c * vol, gy, 2, 2 * vol, B, Z, Y, X, G + n->woff[5], G + n->boff[5], s);
    conv<float, float>(n, gy, 2, 2 * vol, W + n->woff[5], 1, nullptr, n->gB, c, c * vol, B, Z, Y, X, 0, n->d1, c * vol, n->status, s);
    // layer 5: u gradient (no mask: u mixes up(b2) and a2, masks applied below)
    wgrad(n, n->u, 3 * c, 3 * c * vol, n->gB, c, c * vol, B, Z, Y, X, G + n->woff[4], G + n->boff[4], s);
    conv<float, float>(n, n->gB, c, c * vol, W + n->woff[4], 1, nullptr, n->gU, 3 * c, 3 * c * vol, B, Z, Y, X, 0, nullptr, 0, n->status, s);
    // up branch: adjoint of upsample2 with the ReLU mask of b2
    upsample2_adj_kernel<<<nblk(B * 2 * c * hv), 256, 0, s>>>(n->gU, 3 * c * vol, n->b2, n->gH1, 2 * c, B, Z, Y, X);
    // layer 4: b1 gradient with mask(b1)
    wgrad(n, n->b1, 2 * c, 2 * c * hv, n->gH1, 2 * c, 2 * c * hv, B, Z / 2, Y / 2, X / 2, G + n->woff[3], G + n->boff[3], s);
    conv<float, float>(n, n->gH1, 2 * c, 2 * c * hv, W + n->woff[3], 1, nullptr, n->gH2, 2 * c, 2 * c * hv, B, Z / 2, Y / 2,
                       X / 2, 0, n->b1, 2 * c * hv, n->status, s);
    // layer 3: p gradient (no ReLU on p) into gH1 (c channels)
    wgrad(n, n->p, c, c * hv, n->gH2, 2 * c, 2 * c * hv, B, Z / 2, Y / 2, X / 2, G + n->woff[2], G + n->boff[2], s);
    conv<float, float>(n, n->gH2, 2 * c, 2 * c * hv, W + n->woff[2], 1, nullptr, n->gH1, c, c * hv, B, Z / 2, Y / 2, X / 2, 0,
                       nullptr, 0, n->status, s);
    // a2 gradient: skip part + adjoint of avgpool2, masked by a2
    skip_grad_kernel<<<nblk(B * c * vol), 256, 0, s>>>(n->gU + 2 * c * vol, 3 * c * vol, n->gH1, a2, 3 * c * vol, n->gA, c,
                                                       B, Z, Y, X);
    // layer 2: a1 gradient with mask(a1)
    wgrad(n, n->a1, c, c * vol, n->gA, c, c * vol, B, Z, Y, X, G + n->woff[1], G + n->boff[1], s);
    conv<float, float>(n, n->gA, c, c * vol, W + n->woff[1], 1, nullptr, n->gB, c, c * vol, B, Z, Y, X, 0, n->a1, c * vol, n->status, s);
    // layer 1
    wgrad(n, n->x, 5, 5 * vol, n->gB, c, c * vol, B, Z, Y, X, G + n->woff[0], G + n->boff[0], s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_net_adam(helm_net* n, float lr, float b1, float b2, float eps, int step, void* stream) {
    if (!n || step < 1) return HELM_ERR_ARG;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((n->nparam + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n->W, n->G, n->Mom, n->Vel, n->Wb,
                                                                                      n->nparam, lr, b1, b2, eps, c1, c2);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_net_mse(const float* y, const float* t, float* gy, size_t count, double* loss_dev, void* stream) {
    if (!y || !t || !gy || !loss_dev || !count) return HELM_ERR_ARG;
    mse_kernel<<<nblk(count), 256, 0, (cudaStream_t)stream>>>(y, t, gy, count, loss_dev);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_net_features(helm_ctx* c, helm_net* n, const void* v, const void* mv, void* x, void* stream) {
    if (!c || !n || !v || !mv || !x) return HELM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = c->npts;
    double* acc = n->stats;
    bf16* X = (bf16*)x;
    HELM_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
    sumsq_kernel<<<nblk(N), 256, 0, s>>>((const float2*)v, N, acc);
    sumsq_kernel<<<nblk(N), 256, 0, s>>>((const float2*)mv, N, acc + 1);
    feat_pair_kernel<<<nblk(N), 256, 0, s>>>((const float2*)v, acc, N, X, X + N);
    feat_pair_kernel<<<nblk(N), 256, 0, s>>>((const float2*)mv, acc + 1, N, X + 2 * N, X + 3 * N);
    feat_contrast_kernel<<<nblk(N), 256, 0, s>>>(c->k2_f, (float)(1.0 / (c->k0 * c->k0)), N, X + 4 * N);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_net_target(helm_ctx* c, helm_net* n, const void* xs, const void* xk, const void* mv, float* t,
                            void* stream) {
    if (!c || !n || !xs || !xk || !mv || !t) return HELM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = c->npts;
    double* acc = n->stats + 15;
    HELM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double), s));
    sumsq_kernel<<<nblk(N), 256, 0, s>>>((const float2*)mv, N, acc);
    target_kernel<<<nblk(N), 256, 0, s>>>((const double2*)xs, (const double2*)xk, (const float2*)mv, acc, N, t);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status helm_attach_net(helm_ctx* c, helm_net* n) {
    if (!c) return HELM_ERR_ARG;
    if (n) {
        if (!c->opt.flexible || c->nx % 2 || c->ny % 2 || c->nz % 2) return HELM_ERR_ARG;
        helm_status st = ensure_ws(n, 1, c->nz, c->ny, c->nx);
        if (st != HELM_OK) return st;
        if ((st = ensure_field_ws(n, c->npts)) != HELM_OK) return st;
    }
    c->net = n;
    return HELM_OK;
}

helm_status helm_net_stats(helm_net* n, double* host6) {
    if (!n || !host6) return HELM_ERR_ARG;
    HELM_CUDA_TRY(cudaMemcpy(host6, n->stats, 6 * sizeof(double), cudaMemcpyDeviceToHost));
    return HELM_OK;
}

}  // extern "C"

// solver-side field buffers for npts points
helm_status ensure_field_ws(helm_net* n, size_t npts) {
    if (npts <= n->fcap) return HELM_OK;
    void* ps[] = {n->vbuf, n->cbuf, n->az0, n->ac};
    free_bufs(ps, 4);
    n->vbuf = n->cbuf = n->az0 = n->ac = nullptr;
    n->fcap = 0;
    const size_t b = npts * sizeof(float2);
    const bool ok = cudaMalloc(&n->vbuf, b) == cudaSuccess && cudaMalloc(&n->cbuf, b) == cudaSuccess &&
                    cudaMalloc(&n->az0, b) == cudaSuccess && cudaMalloc(&n->ac, b) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    n->fcap = npts;
    return HELM_OK;
}

// Before M^-1: the per-call sums are reset, the r features written and v = sigma[sidx] r kept (r may be
// overwritten by M^-1 afterwards).
helm_status learned_pre(helm_ctx* c, const float2* r, const double* sigma, int sidx, cudaStream_t s) {
    helm_net* n = c->net;
    helm_status st = ensure_ws(n, 1, c->nz, c->ny, c->nx);
    if (st != HELM_OK) return st;
    if ((st = ensure_field_ws(n, c->npts)) != HELM_OK) return st;
    const size_t N = c->npts;
    double* acc = n->stats;
    prof_begin(c, s, PROF_LEARNED);
    HELM_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
    HELM_CUDA_TRY(cudaMemsetAsync(acc + 6, 0, 4 * sizeof(double), s));
    sumsq_kernel<<<nblk(N), 256, 0, s>>>(r, N, acc);
    feat_v_kernel<<<nblk(N), 256, 0, s>>>(r, acc, N, n->x, n->x + N, sigma, sidx, n->vbuf);
    feat_contrast_kernel<<<nblk(N), 256, 0, s>>>(c->k2_f, (float)(1.0 / (c->k0 * c->k0)), N, n->x + 4 * N);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// After M^-1 (z = z0 = M^-1 v): c = s N(features), then the minimal-residual step z = z0 + alpha c.
helm_status learned_post(helm_ctx* c, float2* z, cudaStream_t s) {
    helm_net* n = c->net;
    const size_t N = c->npts;
    double* acc = n->stats;
    helm_status st;
    prof_begin(c, s, PROF_LEARNED);
    sumsq_kernel<<<nblk(N), 256, 0, s>>>(z, N, acc + 1);
    feat_pair_kernel<<<nblk(N), 256, 0, s>>>(z, acc + 1, N, n->x + 2 * N, n->x + 3 * N);
    forward(n, c->status_d, s);
    make_c_kernel<<<nblk(N), 256, 0, s>>>(n->y, acc, N, n->cbuf);
    prof_end(c, s);
    if ((st = launch_stencil_f32_cls(c, z, n->az0, nullptr, 0, PROF_LEARNED, s)) != HELM_OK) return st;
    if ((st = launch_stencil_f32_cls(c, n->cbuf, n->ac, nullptr, 0, PROF_LEARNED, s)) != HELM_OK) return st;
    prof_begin(c, s, PROF_LEARNED);
    mr_dots_kernel<<<nblk(N), 256, 0, s>>>(n->vbuf, n->az0, n->ac, N, acc);
    mr_apply_kernel<<<nblk(N), 256, 0, s>>>(n->cbuf, acc, N, z);
    prof_end(c, s);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
