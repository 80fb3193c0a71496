// 3x3x3 convolutions of the learned correction on the tcgen05 tensor cores (BF16 operands, FP32 accumulation
// in tensor memory), as implicit GEMMs.  An extension of the method (the paper has no network); the
// network, its layout ([B][C][Z][Y][X], x fastest) and the direct SIMT kernels it replaces live in
// learned.cu.
//
// Forward (and data gradient, which is the same convolution with flipped, transposed weights):
//   out[o][p] = act(bias[o] + sum_{t, i} W(o, i, t) in[i][p + off_t]),  zero padding.
//   A CTA computes CT_TY rows of CT_TX = 128 points along x: per row one accumulator of M = 128 points by
//   N = Cout (padded to a multiple of 16) in tensor memory.  The K dimension runs over 16-channel chunks
//   and the 27 taps.  For a chunk, the CTA stages the input halo slab (3 planes x (CT_TY + 2) rows x 130
//   points x 16 channels) in shared memory as 16-byte cells of 8 channels, laid out [channel group][z][y][x]
//   so that consecutive x are consecutive cells.  That layout is the canonical K-major, no-swizzle operand
//   layout (8 rows of 16 bytes per core matrix), and a tap's shifted view of the slab is the same layout
//   at another start address: the 27 taps read one slab, nothing is copied per tap.  The weights of the
//   chunk (27 taps x N x 16, pre-arranged by arrange_w_kernel) arrive by one bulk copy.  Two stages.
//   Warps 0-7 gather the slab (8-point vector loads of the channel-first input, a register transpose into
//   the cells, BF16, zeros outside the grid); warps 0-3 then run the epilogue (bias, ReLU, optional mask,
//   channel-first stores); warp 8 allocates tensor memory and one lane issues the MMAs (M = 128, N = Np,
//   K = 16 each).
// Weight gradient:  gW[o][i][t] = sum_p g[o][p] in[i][p + off_t].
//   A CTA owns one 16-channel chunk of i and walks a share of the 128-point row tiles.  Per tile: A = the
//   gradient rows (M = 128 output channels, padded, K = 128 points, K-major cells of 8 points) and B = the
//   same input slab, read as an MN-major operand (N = 16 channels, K = points; the tap's shift is again a
//   start address).  27 accumulators of 128 x 16 live in tensor memory for the CTA's whole share and are
//   added to gW (FP32 atomics) at the end.
// Every mbarrier wait is bounded; an expired wait raises HELM_DEV_WAIT, the CTA waits (bounded) for its bulk
// copies and MMAs in flight, frees its tensor memory and exits.
#include "common.cuh"
#include <cuda_bf16.h>
#include <algorithm>

typedef __nv_bfloat16 bf16;

namespace {

constexpr int CT_TX = 128;                         // output points per row (MMA M)
constexpr int CT_SX = CT_TX + 2;                   // slab points per row (one halo point each side)
constexpr int CT_NPMAX = 64;                       // largest padded output-channel count
constexpr long CT_WAIT = 1L << 22;                 // bound of every mbarrier wait (polls)
constexpr int CT_PW = 8;                           // producer warps (gather); warps 0-3 also run the epilogue
constexpr int CT_THREADS = (CT_PW + 1) * 32;       // + one warp for tensor memory and the MMAs
constexpr int CT_MW = CT_PW;                       // the MMA warp

template <int TY>
struct CtLayout {
    static constexpr int SY = TY + 2;
    static constexpr int CELLS = 2 * 3 * SY * CT_SX;            // 16-byte cells of one 16-channel chunk
    static constexpr int SLAB = CELLS * 16;
    static constexpr int CG = 3 * SY * CT_SX * 16;              // bytes between the two channel groups
};
// forward: two rows per CTA; a stage is the slab and the chunk's weights (27 x 2 x Np x 16 bytes); two stages
// when there are several channel chunks, one (and so more CTAs per SM) when there is one
constexpr int FW_TY = 2;
constexpr int FW_WMAX = 27 * 2 * CT_NPMAX * 16;                 // 55,296 bytes
constexpr int FW_SMEM = 2 * (CtLayout<FW_TY>::SLAB + FW_WMAX) + 128;   // the largest request
__host__ __device__ constexpr int fw_stage_bytes(int Np) { return CtLayout<FW_TY>::SLAB + 27 * 2 * Np * 16; }
// weight gradient: one row per tile; a stage is the slab and the gradient tile (16 x 128 cells)
constexpr int WG_G = 16 * 128 * 16;                             // 32,768
constexpr int WG_STAGE = CtLayout<1>::SLAB + WG_G;              // 70,208
constexpr int WG_NS = 3;
constexpr int WG_SMEM = WG_NS * WG_STAGE + 128;

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, long limit) {
    for (long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(b), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion on bar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}
// shared-memory matrix descriptor, no swizzle: start, LBO (the stride between 8-element groups along K) and
// SBO (along M or N) in bytes, multiples of 16; a core matrix is 8 rows of 16 contiguous bytes
__device__ __forceinline__ uint64_t ndesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor, kind::f16 with BF16 A and B, FP32 D; a_mn/b_mn = 1 for MN-major operands
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                     "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float ldf(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ void stf(bf16* p, size_t i, float v) { p[i] = __float2bfloat16(v); }
__device__ __forceinline__ void stf(float* p, size_t i, float v) { p[i] = v; }
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// 8 consecutive values of one row (x = xb .. xb + 7) as four packed BF16 pairs: one 16-byte (BF16) or two
// 16-byte (FP32) loads inside the row when aligned (rows of a multiple of 8 points), else per point, zeros
// outside 0 .. X - 1
__device__ __forceinline__ uint4 load8(const bf16* __restrict__ row, int xb, int X, bool vec) {
    if (vec && xb >= 0 && xb + 8 <= X) return *reinterpret_cast<const uint4*>(row + xb);
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (xb + k >= 0 && xb + k < X) ? __bfloat162float(row[xb + k]) : 0.f;
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}
__device__ __forceinline__ uint4 load8(const float* __restrict__ row, int xb, int X, bool vec) {
    if (vec && xb >= 0 && xb + 8 <= X) {
        const float4 a = *reinterpret_cast<const float4*>(row + xb), b = *reinterpret_cast<const float4*>(row + xb + 4);
        return make_uint4(pack2(a.x, a.y), pack2(a.z, a.w), pack2(b.x, b.y), pack2(b.z, b.w));
    }
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (xb + k >= 0 && xb + k < X) ? row[xb + k] : 0.f;
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}
__device__ __forceinline__ uint32_t u4w(const uint4& q, int i) { return i == 0 ? q.x : (i == 1 ? q.y : (i == 2 ? q.z : q.w)); }

// Fill the slab of one 16-channel chunk (channels c0 .. c0 + 15) for output rows y0 .. y0 + TY - 1 of plane
// z: cell q = ((cg * 3 + dz) * SY + yr) * 130 + xi holds channels c0 + 8 cg .. + 7 of the input point
// (z + dz - 1, y0 + yr - 1, x0 + xi - 1); zero outside the grid and beyond Cin.  A work item is one row of
// the slab and one group of 8 points x = x0 - 8 + 8 g (g = 0 .. 17, aligned when x0 is): it loads the 8
// channels' rows of those points (8-point vector loads) and writes the 8 cells, a transpose of the
// channel-first input into the channel-contiguous cells done on packed BF16 pairs (byte permutes).
template <int TY, typename TIN>
__device__ __forceinline__ void fill_slab(unsigned char* slab, const TIN* __restrict__ in, int Cin, int c0, int z,
                                          int y0, int x0, int Z, int Y, int X, int t, int nthreads) {
    typedef CtLayout<TY> L;
    constexpr int NG = (CT_SX + 14) / 8;   // 18 groups cover x0 - 8 .. x0 + 135 (the slab is x0 - 1 .. x0 + 128)
    const size_t vol = (size_t)Z * Y * X;
    const bool vec = (X % 8) == 0;
    for (int it = t; it < 2 * 3 * L::SY * NG; it += nthreads) {
        const int g = it % NG;
        int r = it / NG;
        const int yr = r % L::SY;
        r /= L::SY;
        const int dz = r % 3, cg = r / 3;
        const int gz = z + dz - 1, gy = y0 + yr - 1, xb = x0 - 8 + 8 * g;
        const bool rowok = gz >= 0 && gz < Z && gy >= 0 && gy < Y;
        const size_t roff = rowok ? ((size_t)gz * Y + gy) * X : 0;
        uint4 row[8];   // channel j: the 8 points as BF16 pairs
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ch = c0 + 8 * cg + j;
            row[j] = (rowok && ch < Cin) ? load8(in + (size_t)ch * vol + roff, xb, X, vec) : make_uint4(0u, 0u, 0u, 0u);
        }
        unsigned char* rowp = slab + (size_t)(((cg * 3 + dz) * L::SY + yr) * CT_SX) * 16;
        // Store slot k writes the cell of point k ^ sw (sw = g mod 8).  A thread's 8 cells are 128 contiguous
        // bytes and neighbouring threads take neighbouring groups, so with the same order everywhere all the
        // 16-byte stores of one warp instruction would hit the same four banks; rotated, they spread over all
        // 32.  The rotation is applied to the loaded words (point pair k >> 1 is word k >> 1 of each row) and
        // to the half selector (point parity), so every register index stays static.
        const int sw = g & 7;
        if (sw & 2)
#pragma unroll
            for (int j = 0; j < 8; ++j) row[j] = make_uint4(row[j].y, row[j].x, row[j].w, row[j].z);
        if (sw & 4)
#pragma unroll
            for (int j = 0; j < 8; ++j) row[j] = make_uint4(row[j].z, row[j].w, row[j].x, row[j].y);
        const uint32_t sel_even = (sw & 1) ? 0x7632u : 0x5410u, sel_odd = (sw & 1) ? 0x5410u : 0x7632u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int xi = 8 * g - 7 + (k ^ sw);   // slab index of the point xb + (k ^ sw)
            if (xi >= 0 && xi < CT_SX) {
                // cell word m = (channel 2m, channel 2m + 1) at the point: the low (even point) or high halves
                const uint32_t sel = (k & 1) ? sel_odd : sel_even;
                uint32_t w[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) w[m] = __byte_perm(u4w(row[2 * m], k >> 1), u4w(row[2 * m + 1], k >> 1), sel);
                *reinterpret_cast<uint4*>(rowp + (size_t)xi * 16) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// ---- forward / data gradient ------------------------------------------------------------------------------
// wt: arranged weights [nkc][27][2][Np][8] (bf16); mask (optional): out *= (mask > 0)
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(CT_THREADS, 3)
conv_tc_kernel(const TIN* __restrict__ in, int Cin, size_t in_bs, const bf16* __restrict__ wt, int Np,
               const float* __restrict__ bias, TOUT* __restrict__ out, int Cout, size_t out_bs, int Z, int Y, int X,
               int relu, const bf16* __restrict__ mask, size_t mask_bs, int nst, unsigned* status) {
    typedef CtLayout<FW_TY> L;
    extern __shared__ __align__(128) unsigned char csm[];
    unsigned char* base = (unsigned char*)(((uintptr_t)csm + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) uint64_t full[2], wfull[2], empty[2], accf, drainb;
    __shared__ uint32_t tslot;
    __shared__ int fail_any;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntx = (X + CT_TX - 1) / CT_TX, nty = (Y + FW_TY - 1) / FW_TY;
    int tile = blockIdx.x;
    const int xt = tile % ntx;
    tile /= ntx;
    const int yt = tile % nty;
    tile /= nty;
    const int z = tile % Z, b = tile / Z;
    const int x0 = xt * CT_TX, y0 = yt * FW_TY;
    const int nkc = (Cin + 15) / 16;
    const uint32_t wbytes = 27u * 2u * (uint32_t)Np * 16u;
    const size_t stage = (size_t)fw_stage_bytes(Np);   // a multiple of 16
    const uint32_t ncols = FW_TY * Np <= 32 ? 32 : (FW_TY * Np <= 64 ? 64 : 128);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            bar_init(s32(&full[s]), CT_PW);
            bar_init(s32(&wfull[s]), 1);
            bar_init(s32(&empty[s]), 1);
        }
        bar_init(s32(&accf), 1);
        bar_init(s32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == CT_MW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&tslot)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int issued = 0;   // chunks whose weight copy thread 0 issued
    const TIN* inb = in + (size_t)b * in_bs;
    if (warp < CT_PW) {
        for (int kc = 0; kc < nkc && ok; ++kc) {
            const int s = kc % nst, u = kc / nst;
            if (u >= 1) ok = __all_sync(0xffffffffu, bar_wait(s32(&empty[s]), (uint32_t)((u - 1) & 1), CT_WAIT));
            if (!ok) break;
            unsigned char* st = base + (size_t)s * stage;
            if (threadIdx.x == 0) {
                bar_expect(s32(&wfull[s]), wbytes);
                bulk_g2s(s32(st + L::SLAB), wt + (size_t)kc * 27 * 2 * Np * 8, wbytes, s32(&wfull[s]));
                ++issued;
            }
            fill_slab<FW_TY>(st, inb, Cin, 16 * kc, z, y0, x0, Z, Y, X, threadIdx.x, CT_PW * 32);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the MMAs read the slab (async proxy)
            __syncwarp();
            if (lane == 0) bar_arrive(s32(&full[s]));
        }
        // epilogue (warps 0-3): this warp's 32 accumulator lanes are the points x0 + 32 (warp) + lane
        if (ok && warp < 4) ok = __all_sync(0xffffffffu, bar_wait(s32(&accf), 0, CT_WAIT));
        if (ok && warp < 4) {
            tc_after();
            const size_t vol = (size_t)Z * Y * X;
            const int x = x0 + 32 * warp + lane;
            for (int r = 0; r < FW_TY; ++r) {
                const int y = y0 + r;
                const size_t q = ((size_t)z * Y + y) * X + x;
                for (int cb = 0; cb < Np; cb += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * Np + cb), v);
                    if (x < X && y < Y) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int o = cb + j;
                            if (o < Cout) {
                                float a = v[j] + (bias ? bias[o] : 0.f);
                                if (relu) a = fmaxf(a, 0.f);
                                if (mask && !(__bfloat162float(mask[(size_t)b * mask_bs + (size_t)o * vol + q]) > 0.f))
                                    a = 0.f;
                                stf(out, (size_t)b * out_bs + (size_t)o * vol + q, a);
                            }
                        }
                    }
                }
            }
        }
    } else if (lane == 0) {
        const uint32_t idesc = idesc_bf16(128, Np, 0, 0);
        for (int kc = 0; kc < nkc && ok; ++kc) {
            const int s = kc % nst, u = kc / nst;
            ok = bar_wait(s32(&full[s]), (uint32_t)(u & 1), CT_WAIT) && bar_wait(s32(&wfull[s]), (uint32_t)(u & 1), CT_WAIT);
            if (!ok) break;
            tc_after();
            const uint32_t slab = s32(base + (size_t)s * stage), wsm = slab + L::SLAB;
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                // B: tap t's weights [2 channel groups][Np][8]: next channel group (K) Np*16 bytes, next 8 outputs 128
                const uint64_t bd = ndesc(wsm + (uint32_t)t * 2u * (uint32_t)Np * 16u, (uint32_t)Np * 16u, 128u);
#pragma unroll
                for (int r = 0; r < FW_TY; ++r) {
                    // A: the tap's view of the slab; next channel group (K) L::CG bytes, next 8 points (M) 128
                    const uint32_t a0 = slab + (uint32_t)(((dz * L::SY + r + dy) * CT_SX + dx) * 16);
                    mma_bf16(tmem + (uint32_t)(r * Np), ndesc(a0, (uint32_t)L::CG, 128u), bd, idesc, (kc | t) ? 1u : 0u);
                }
            }
            mma_commit(s32(&empty[s]));
        }
        if (ok) mma_commit(s32(&accf));
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && lane == 0) {
        if (warp == 0) {
            // the weight copies of the last (at most nst) issued chunks may still be in flight
            for (int kc = issued > nst ? issued - nst : 0; kc < issued; ++kc)
                bar_wait(s32(&wfull[kc % nst]), (uint32_t)((kc / nst) & 1), CT_WAIT);
        } else if (warp == CT_MW) {
            mma_commit(s32(&drainb));
            bar_wait(s32(&drainb), 0, CT_WAIT);
        }
    }
    tc_before();
    __syncthreads();
    if (warp == CT_MW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---- weight gradient ---------------------------------------------------------------------------------
// gw[o][i][t] += sum_{b, p} g[b][o][p] in[b][i][p + off_t] for the 16 input channels of chunk blockIdx.x;
// Cout <= 128.  Tiles: (b, z, y, 128-point x block), CTA y takes tiles blockIdx.y, + gridDim.y, ...
template <typename TG>
__global__ void __launch_bounds__(CT_THREADS, 1)
wgrad_tc_kernel(const bf16* __restrict__ in, int Cin, size_t in_bs, const TG* __restrict__ g, int Cout, size_t g_bs,
                int B, int Z, int Y, int X, float* __restrict__ gw, unsigned* status) {
    typedef CtLayout<1> L;
    extern __shared__ __align__(128) unsigned char csm[];
    unsigned char* base = (unsigned char*)(((uintptr_t)csm + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) uint64_t full[WG_NS], empty[WG_NS], accf, drainb;
    __shared__ uint32_t tslot;
    __shared__ int fail_any;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kc = blockIdx.x;
    const int ntx = (X + CT_TX - 1) / CT_TX;
    const int ntiles = B * Z * Y * ntx;
    const size_t vol = (size_t)Z * Y * X;
    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_NS; ++s) { bar_init(s32(&full[s]), CT_PW); bar_init(s32(&empty[s]), 1); }
        bar_init(s32(&accf), 1);
        bar_init(s32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == CT_MW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&tslot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int nt = 0;   // tiles this CTA processed
    if (warp < CT_PW) {
        for (int tile = blockIdx.y; tile < ntiles && ok; tile += gridDim.y, ++nt) {
            int r = tile;
            const int xt = r % ntx;
            r /= ntx;
            const int y = r % Y;
            r /= Y;
            const int z = r % Z, bb = r / Z;
            const int x0 = xt * CT_TX;
            const int s = nt % WG_NS, u = nt / WG_NS;
            if (u >= 1) ok = __all_sync(0xffffffffu, bar_wait(s32(&empty[s]), (uint32_t)((u - 1) & 1), CT_WAIT));
            if (!ok) break;
            unsigned char* st = base + (size_t)s * WG_STAGE;
            fill_slab<1>(st, in + (size_t)bb * in_bs, Cin, 16 * kc, z, y, x0, Z, Y, X, threadIdx.x, CT_PW * 32);
            // gradient cells: cell (kq, o) = g[o][z][y][x0 + 8 kq .. + 7], layout [kq][o][8]; zero beyond Cout, X
            unsigned char* gs = st + L::SLAB;
            const TG* gb = g + (size_t)bb * g_bs + ((size_t)z * Y + y) * X;
            const bool vec = (X % 8) == 0;
            for (int q = threadIdx.x; q < 16 * 128; q += CT_PW * 32) {
                const int o = q % 128, kq = q / 128;
                *reinterpret_cast<uint4*>(gs + (size_t)q * 16) =
                    o < Cout ? load8(gb + (size_t)o * vol, x0 + 8 * kq, X, vec) : make_uint4(0u, 0u, 0u, 0u);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(s32(&full[s]));
        }
        if (ok && warp < 4) ok = __all_sync(0xffffffffu, bar_wait(s32(&accf), 0, CT_WAIT));
        if (ok && nt > 0 && warp < 4) {
            tc_after();
            const int o = 32 * warp + lane;
            for (int t = 0; t < 27; ++t) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * t), v);
                if (o < Cout) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int i = 16 * kc + j;
                        if (i < Cin) atomicAdd(&gw[((size_t)o * Cin + i) * 27 + t], v[j]);
                    }
                }
            }
        }
    } else if (lane == 0) {
        // A (gradient, K-major): next 8 points (K) 2048 bytes, next 8 outputs (M) 128; B (slab, MN-major): next
        // 8 points (K) 128 bytes, next channel group (N) L::CG.  Without swizzling the leading-byte offset is the
        // K stride and the stride-byte offset the M/N stride for either major-ness.
        const uint32_t idesc = idesc_bf16(128, 16, 0, 1);
        int n = 0;
        for (int tile = blockIdx.y; tile < ntiles && ok; tile += gridDim.y, ++n) {
            const int s = n % WG_NS, u = n / WG_NS;
            ok = bar_wait(s32(&full[s]), (uint32_t)(u & 1), CT_WAIT);
            if (!ok) break;
            tc_after();
            const uint32_t slab = s32(base + (size_t)s * WG_STAGE), gsm = slab + L::SLAB;
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const uint64_t ad = ndesc(gsm + (uint32_t)(2 * kk) * 2048u, 2048u, 128u);
                    const uint64_t bd = ndesc(slab + (uint32_t)(((dz * L::SY + dy) * CT_SX + 16 * kk + dx) * 16), 128u,
                                              (uint32_t)L::CG);
                    mma_bf16(tmem + (uint32_t)(16 * t), ad, bd, idesc, (n | kk) ? 1u : 0u);
                }
            }
            mma_commit(s32(&empty[s]));
        }
        if (ok) mma_commit(s32(&accf));
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && warp == CT_MW && lane == 0) {
        mma_commit(s32(&drainb));
        bar_wait(s32(&drainb), 0, CT_WAIT);
    }
    tc_before();
    __syncthreads();
    if (warp == CT_MW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// arranged[kc][t][cg][o][j] = W(o0 + o, 16 kc + 8 cg + j, t) for the output slice o0 .. o0 + Np - 1, zero beyond
// Cout / Cin; W(o, i, t) = w[(o Cin + i) 27 + t] (wmode 0) or w[(i Cout + o) 27 + 26 - t] (wmode 1: the data
// gradient's flipped, transposed weights)
__global__ void arrange_w_kernel(const bf16* __restrict__ w, int Cin, int Cout, int o0, int wmode, int Np, int nkc,
                                 bf16* __restrict__ dst) {
    const size_t n = (size_t)nkc * 27 * 2 * Np * 8;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        size_t r = id;
        const int j = (int)(r % 8);
        r /= 8;
        const int o = (int)(r % Np);
        r /= Np;
        const int cg = (int)(r % 2);
        r /= 2;
        const int t = (int)(r % 27);
        const int kc = (int)(r / 27);
        const int i = 16 * kc + 8 * cg + j, oo = o0 + o;
        bf16 v = __float2bfloat16(0.f);
        if (oo < Cout && i < Cin)
            v = wmode ? w[((size_t)i * Cout + oo) * 27 + 26 - t] : w[((size_t)oo * Cin + i) * 27 + t];
        dst[id] = v;
    }
}

// gb[o] += sum_{b, p} g[b][o][p]
template <typename TG>
__global__ void bias_grad_kernel(const TG* __restrict__ g, int Cout, size_t g_bs, int B, size_t vol, float* gb) {
    __shared__ float red[8];
    const int o = blockIdx.x;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (size_t q = blockIdx.y * (size_t)blockDim.x + threadIdx.x; q < vol; q += (size_t)gridDim.y * blockDim.x)
            s += ldf(g, (size_t)b * g_bs + (size_t)o * vol + q);
    for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(&gb[o], t);
    }
}

int g_conv_sms = 0;

}  // namespace

// shapes the tensor-core convolutions take (outputs in slices of at most 64 for the forward kernel; the
// weight gradient holds up to 128 outputs in its accumulator rows)
bool conv_tc_supported(int Cin, int Cout) { return Cin >= 1 && Cout >= 1; }
bool wgrad_tc_supported(int Cin, int Cout) { return Cin >= 1 && Cout >= 1 && Cout <= 128; }
size_t conv_tc_scratch_bytes(int Cin, int Cout) {
    const int Np = std::min((Cout + 15) / 16 * 16, CT_NPMAX), nkc = (Cin + 15) / 16;
    return (size_t)nkc * 27 * 2 * Np * 8 * sizeof(bf16);
}

helm_status conv_tc_prepare() {
    HELM_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<bf16, bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    HELM_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<bf16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    HELM_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    HELM_CUDA_TRY(cudaFuncSetAttribute(wgrad_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM));
    int dev = 0;
    HELM_CUDA_TRY(cudaGetDevice(&dev));
    HELM_CUDA_TRY(cudaDeviceGetAttribute(&g_conv_sms, cudaDevAttrMultiProcessorCount, dev));
    return HELM_OK;
}

// out = act(conv(in, W) + bias) with the tensor cores; wscr holds conv_tc_scratch_bytes(Cin, Cout)
template <typename TIN, typename TOUT>
helm_status conv_tc(const TIN* in, int Cin, size_t in_bs, const bf16* w, int wmode, const float* bias, TOUT* out,
                    int Cout, size_t out_bs, int B, int Z, int Y, int X, int relu, const bf16* mask, size_t mask_bs,
                    bf16* wscr, unsigned* status, cudaStream_t s) {
    const int nkc = (Cin + 15) / 16;
    const size_t vol = (size_t)Z * Y * X;
    const int ntx = (X + CT_TX - 1) / CT_TX, nty = (Y + FW_TY - 1) / FW_TY;
    const long tiles = (long)B * Z * nty * ntx;
    // output slices of at most 64 channels (one accumulator width each); the launches follow one another on s
    for (int o0 = 0; o0 < Cout; o0 += CT_NPMAX) {
        const int Co = std::min(Cout - o0, CT_NPMAX), Np = (Co + 15) / 16 * 16;
        const size_t na = (size_t)nkc * 27 * 2 * Np * 8;
        arrange_w_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(w, Cin, Cout, o0, wmode, Np, nkc, wscr);
        // one stage: a CTA's chunks follow one another, and the two to three CTAs an SM holds overlap each
        // other's gathers, MMAs and epilogues instead
        const int nst = 1;
        const size_t smem = (size_t)nst * fw_stage_bytes(Np) + 128;
        conv_tc_kernel<TIN, TOUT><<<(unsigned)tiles, CT_THREADS, smem, s>>>(
            in, Cin, in_bs, wscr, Np, bias ? bias + o0 : nullptr, out + (size_t)o0 * vol, Co, out_bs, Z, Y, X, relu,
            mask ? mask + (size_t)o0 * vol : nullptr, mask_bs, nst, status);
        HELM_CUDA_TRY(cudaGetLastError());
    }
    return HELM_OK;
}
template helm_status conv_tc<bf16, bf16>(const bf16*, int, size_t, const bf16*, int, const float*, bf16*, int, size_t,
                                         int, int, int, int, int, const bf16*, size_t, bf16*, unsigned*, cudaStream_t);
template helm_status conv_tc<bf16, float>(const bf16*, int, size_t, const bf16*, int, const float*, float*, int, size_t,
                                          int, int, int, int, int, const bf16*, size_t, bf16*, unsigned*, cudaStream_t);
template helm_status conv_tc<float, float>(const float*, int, size_t, const bf16*, int, const float*, float*, int,
                                           size_t, int, int, int, int, int, const bf16*, size_t, bf16*, unsigned*,
                                           cudaStream_t);

// gw += d loss/d W and gb += d loss/d bias for the gradient g of the layer output (FP32, [B][Cout][vol])
helm_status wgrad_tc(const bf16* in, int Cin, size_t in_bs, const float* g, int Cout, size_t g_bs, int B, int Z, int Y,
                     int X, float* gw, float* gb, unsigned* status, cudaStream_t s) {
    const int nkc = (Cin + 15) / 16;
    const int ntx = (X + CT_TX - 1) / CT_TX;
    const long ntiles = (long)B * Z * Y * ntx;
    const int sms = g_conv_sms > 0 ? g_conv_sms : 148;
    long per = (2L * sms + nkc - 1) / nkc;   // CTAs per chunk: about two waves over the SMs in all
    if (per > ntiles) per = ntiles;
    if (per < 1) per = 1;
    wgrad_tc_kernel<float><<<dim3((unsigned)nkc, (unsigned)per), CT_THREADS, WG_SMEM, s>>>(in, Cin, in_bs, g, Cout, g_bs, B, Z,
                                                                                      Y, X, gw, status);
    const size_t vol = (size_t)Z * Y * X;
    bias_grad_kernel<float><<<dim3((unsigned)Cout, 64), 256, 0, s>>>(g, Cout, g_bs, B, vol, gb);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}
