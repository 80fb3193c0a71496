// EigT steps 2 and 4 (Sec. 4.1, Eq. EIG_SOLVER) on the 5th-generation tensor cores (tcgen05, sm_103a):
// the dense complex contractions Ybar_l = V_y^-1 Y_l V_x^-T and U_l = V_y Ubar_l V_x^T with TF32 operands
// and FP32 accumulation in tensor memory.
//
// x-pass (right multiply, contraction over x):  every row r = (l, j) of the grid is a complex vector of
//   length N_x.  In the interleaved (re, im) layout the row is a real vector of length 2 N_x, and the
//   complex product with W becomes one real GEMM  Out[r] = Row[r] B^T  with the real embedding
//     B[2n][2k] = Re W_kn,  B[2n][2k+1] = -Im W_kn,  B[2n+1][2k] = Im W_kn,  B[2n+1][2k+1] = Re W_kn.
//   A = the grid viewed as (N_y N_z) x 2N_x (K-major, straight from HBM by TMA), B = 2N_x x 2N_x (K-major).
// y-pass (left multiply per slice, contraction over y):  Out_l = W Y_l with Y_l viewed as N_y x 2N_x real
//   (N contiguous, "MN-major", staged with the 32-byte-chunk 128-byte swizzle).  Two accumulators P = Re(W) Y_l and Q = Im(W) Y_l share every B tile; the
//   epilogue forms Out_re = P_re - Q_im, Out_im = P_im + Q_re.
//
// Kernel structure (one 128 x 128 output tile per CTA, 192 threads, two CTAs per SM):
//   warp 0      TMA producer: cp.async.bulk.tensor tiles (128-byte swizzle) into a STAGES-deep ring,
//               completion tracked by mbarrier transaction counts
//   warp 1      allocates tensor memory; one lane issues tcgen05.mma (M=128, N=128, K=8) and commits
//               each stage back to the producer
//   warps 2-5   epilogue: tcgen05.ld of the accumulator lanes they own, scale, vectorised stores
// Every mbarrier wait is bounded by the context's wait limit (a kernel argument); on expiry the CTA raises
// HELM_DEV_WAIT and skips its remaining work.  Before it frees its tensor memory and exits, it drains what
// it still has in flight under a separate fixed bound: the producer waits for the TMA loads it issued, the
// MMA thread commits once more and waits for its MMAs.  No cluster multicast is used.
#include "common.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

constexpr int BM = 128, BN = 128, BK = 32;      // BK fp32 elements = 128 bytes = one swizzle row
constexpr int TILE = BM * BK * 4;               // 16 KiB: a 128-row tile of one K block
constexpr int XSTAGES = 3, YSTAGES = 2;
constexpr int XEPI_LD = 20;                                  // x-pass staging row: 16 floats + 4 pad
constexpr int XEPI_BYTES = 4 * 32 * XEPI_LD * 4;             // four epilogue warps x 32 rows
constexpr int YEPI_LD = 36;                                  // y-pass staging row: 32 floats + 4 pad
constexpr long DRAIN_LIMIT = 1L << 22;          // bound of the drain waits after an expired wait

struct TcState {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    // operand sets: 0/1 EigT forward/inverse (V^-1, V), 2/3 PFFT sine transforms forward/inverse (S^T, S)
    float* Bx[4] = {nullptr, nullptr, nullptr, nullptr};   // x-pass real-embedded operands, [2N][2N]
    float* Wy[4] = {nullptr, nullptr, nullptr, nullptr};   // y-pass operands, [2][N_y][ldw] (re, im planes)
    float* Bxl[4] = {nullptr, nullptr, nullptr, nullptr};  // 3xTF32: remainders of Bx and Wy
    float* Wyl[4] = {nullptr, nullptr, nullptr, nullptr};
    int ldw = 0;
    int split = 0;             // HELM_PREC_TF32X3
    CUtensorMap mapBx[4];
    CUtensorMap mapBx256[4];   // the same operands in 256-row boxes (256-wide x-pass tiles)
    CUtensorMap mapWy[4];
    CUtensorMap mapBxl[4], mapBx256l[4], mapWyl[4];
    // HELM_PREC_BF16 / HELM_PREC_FP16: the EigT operand sets 0/1 rounded to that type (h16 = 1 BF16, 2 FP16;
    // row stride ldwb of the y-pass planes)
    int h16 = 0;
    int ldwb = 0;
    uint16_t* Bxb[2] = {nullptr, nullptr};
    uint16_t* Wyb[2] = {nullptr, nullptr};
    CUtensorMap mapBxb[2], mapBxb256[2], mapWyb[2];
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long limit) {
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
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
// UMMA shared-memory descriptor, version 1.  Layout 2 = 128-byte swizzle of 16-byte chunks (K-major
// operands here); layout 1 = 128-byte swizzle of 32-byte chunks, the form 32-bit (TF32) MN-major operands
// take, whose swizzle atom is 4 rows x 128 bytes (TMA: CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout = 2) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}
// instruction descriptor, kind::tf32: D = F32, A = B = TF32, majors, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// instruction descriptor, kind::f16: D = F32 (1), A = B = BF16 (1) or F16 (0), majors, N >> 3, M >> 4
// (H: 1 = BF16, 2 = FP16 operands)
__host__ __device__ constexpr uint32_t idesc_h16(int H, int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | ((H == 1 ? 1u : 0u) << 7) | ((H == 1 ? 1u : 0u) << 10) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16kind(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
template <int H>
__device__ __forceinline__ void mma_op(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (H) mma_f16kind(d, a, b, idesc, acc);   // kind::f16; the operand type is in idesc
    else mma_tf32(d, a, b, idesc, acc);
}
// two floats rounded to nearest even BF16 (H = 1) or FP16 (H = 2, clamped to the finite range), packed low
// half first (memory order)
// FP16 chain: the power-of-two scale 2^e with gain sqrt(nsq) 2^e <= 2^15 (nsq the squared Frobenius norm of the
// stage's input, gain the stage operator's norm bound), 1 for an all-zero input
__device__ __forceinline__ float stage_scale(double gain, double nsq) {
    if (!(nsq > 0.0)) return 1.f;
    int e = 15 - (int)ceil(log2(gain * sqrt(nsq)));
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    return ldexpf(1.f, e);
}
template <int H>
__device__ __forceinline__ uint32_t pack16(float lo, float hi) {
    if (H == 2) {
        const __half2 v = __floats2half2_rn(fminf(fmaxf(lo, -65504.f), 65504.f), fminf(fmaxf(hi, -65504.f), 65504.f));
        return *reinterpret_cast<const uint32_t*>(&v);
    }
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TMEM_LD32(taddr, r)                                                                                          \
    asm volatile(                                                                                                    \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19," \
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                                     \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),            \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),      \
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),    \
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])     \
        : "r"(taddr))
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Drain after an expired wait: the producer thread waits, under the fixed drain bound, for the TMA loads
// of the last `ns` pipeline iterations it issued (one per stage, so every barrier phase is unambiguous);
// the MMA thread commits once more and waits for that commit, which completes after all its MMAs.
__device__ __forceinline__ void drain_tma(const uint64_t* full, int ns, long issued) {
    for (long it = issued > ns ? issued - ns : 0; it < issued; ++it)
        mbar_wait(su32(&full[it % ns]), (uint32_t)((it / ns) & 1), DRAIN_LIMIT);
}
__device__ __forceinline__ void drain_mma(uint64_t* bar) {
    mma_commit(su32(bar));
    mbar_wait(su32(bar), 0, DRAIN_LIMIT);
}

// ---- three-product split TF32 ("3xTF32") -----------------------------------------------------------
// a = hi + lo with hi = a rounded to TF32 (10 explicit mantissa bits, round to nearest) and lo = a - hi
// (exact in FP32, below 2^-11 |a|); a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b, the dropped lo_a lo_b and the
// tensor core's truncation of lo to TF32 are below 2^-21 of the product.  The bases are split once at
// set-up; the streamed grid tile is split in shared memory by four converter warps, element by element,
// so the swizzled layout TMA wrote stays valid for both halves.
__device__ __forceinline__ float tf32_rna(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return __uint_as_float(r);
}
// one 16 KiB data tile (4096 floats) by 128 threads: hi in place, lo into the parallel tile
__device__ __forceinline__ void split_tile(float4* hi, float4* lo, int t) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = t + 128 * i;
        const float4 v = hi[k];
        const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
        hi[k] = h;
        lo[k] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
    // the MMAs read both tiles through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- x-pass: Out[M][N2] = alpha * A[M][K2] B[N2][K2]^T -------------------------------------------
__global__ void __launch_bounds__(192, 1)
xpass_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float* __restrict__ out,
                int M, int N2, int K2, float alpha, const double* __restrict__ alpha_dev, int aidx, int rows_per,
                int astride, unsigned* status,
                long wlim) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[XSTAGES], empty[XSTAGES], accf, drainb;
    __shared__ int fail_any;
    __shared__ uint32_t tslot;
    const uint32_t raw = su32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int nk = (K2 + BK - 1) / BK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < XSTAGES; ++s) { mbar_init(su32(&full[s]), 1); mbar_init(su32(&empty[s]), 1); }
        mbar_init(su32(&accf), 1);
        mbar_init(su32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    long issued = 0;   // pipeline iterations whose TMA loads the producer issued
    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % XSTAGES;
                const uint32_t ph = (kb / XSTAGES) & 1;
                if (kb >= XSTAGES) ok = mbar_wait(su32(&empty[s]), ph ^ 1, wlim);
                if (!ok) break;
                const uint32_t sa = base + s * 2 * TILE, sb = sa + TILE;
                mbar_expect_tx(su32(&full[s]), 2 * TILE);
                tma_2d(sa, &tmA, su32(&full[s]), kb * BK, m0);
                tma_2d(sb, &tmB, su32(&full[s]), kb * BK, n0);
                ++issued;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(BM, BN, 0, 0);
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % XSTAGES;
                const uint32_t ph = (kb / XSTAGES) & 1;
                ok = mbar_wait(su32(&full[s]), ph, wlim);
                if (!ok) break;
                fence_after();
                const uint32_t sa = base + s * 2 * TILE, sb = sa + TILE;
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk)
                    mma_tf32(tmem, sdesc(sa + kk * 32, 16, 1024), sdesc(sb + kk * 32, 16, 1024), idesc,
                             (kb | kk) ? 1u : 0u);
                mma_commit(su32(&empty[s]));
            }
            mma_commit(su32(&accf));
        }
    } else {
        ok = mbar_wait(su32(&accf), 0, wlim);
        ok = __all_sync(0xffffffffu, ok);
        fence_after();
        const int q = warp & 3;
        const int row = m0 + 32 * q + lane;
        // rows of the b-th vector of a batch scale by alpha_dev[aidx + b astride] (b = row / rows_per)
        const float al = alpha * (alpha_dev ? (float)alpha_dev[aidx + (min(row, M - 1) / rows_per) * astride] : 1.f);
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, r);
                tmem_wait_ld();
                const int col = n0 + c;
                if (row < M && col < N2) {
                    float* dst = out + (size_t)row * N2 + col;
                    if (col + 32 <= N2) {
#pragma unroll
                        for (int v = 0; v < 32; v += 4)
                            *reinterpret_cast<float4*>(dst + v) =
                                make_float4(al * __uint_as_float(r[v]), al * __uint_as_float(r[v + 1]),
                                            al * __uint_as_float(r[v + 2]), al * __uint_as_float(r[v + 3]));
                    } else {
#pragma unroll
                        for (int v = 0; v < 32; ++v)
                            if (col + v < N2) dst[v] = al * __uint_as_float(r[v]);
                    }
                }
            }
        }
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && lane == 0) {
        if (warp == 0) drain_tma(full, XSTAGES, issued);
        else if (warp == 1) drain_mma(&drainb);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---- y-pass: Out_l[ny][N2] = W Y_l, W = Wr + i Wi -------------------------------------------------
__global__ void __launch_bounds__(192, 1)
ypass_tc_kernel(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmY, float* __restrict__ out,
                int ny, int N2, unsigned* status, long wlim) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[YSTAGES], empty[YSTAGES], accf, drainb;
    __shared__ int fail_any;
    __shared__ uint32_t tslot;
    const uint32_t raw = su32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, l = blockIdx.z;
    const int nk = (ny + BK - 1) / BK;
    constexpr int STAGE = 3 * TILE;   // Wr tile, Wi tile, B tile (4 boxes of 32 K-rows x 128 bytes)
    if (threadIdx.x == 0) {
        for (int s = 0; s < YSTAGES; ++s) { mbar_init(su32(&full[s]), 1); mbar_init(su32(&empty[s]), 1); }
        mbar_init(su32(&accf), 1);
        mbar_init(su32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    long issued = 0;   // pipeline iterations whose TMA loads the producer issued
    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % YSTAGES;
                const uint32_t ph = (kb / YSTAGES) & 1;
                if (kb >= YSTAGES) ok = mbar_wait(su32(&empty[s]), ph ^ 1, wlim);
                if (!ok) break;
                const uint32_t sw = base + s * STAGE, sb = sw + 2 * TILE;
                mbar_expect_tx(su32(&full[s]), STAGE);
                tma_3d(sw, &tmW, su32(&full[s]), kb * BK, m0, 0);
                tma_3d(sw + TILE, &tmW, su32(&full[s]), kb * BK, m0, 1);
#pragma unroll
                for (int b = 0; b < BN / 32; ++b) tma_3d(sb + b * 4096, &tmY, su32(&full[s]), n0 + 32 * b, kb * BK, l);
                ++issued;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(BM, BN, 0, 1);
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % YSTAGES;
                const uint32_t ph = (kb / YSTAGES) & 1;
                ok = mbar_wait(su32(&full[s]), ph, wlim);
                if (!ok) break;
                fence_after();
                const uint32_t sw = base + s * STAGE, sb = sw + 2 * TILE;
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    // MN-major: LBO = next 32-column chunk (4 KiB), SBO = next 4-row K group (512 B)
                    const uint64_t bd = sdesc(sb + kk * 1024, 4096, 512, 1);
                    const uint32_t acc = (kb | kk) ? 1u : 0u;
                    mma_tf32(tmem, sdesc(sw + kk * 32, 16, 1024), bd, idesc, acc);
                    mma_tf32(tmem + BN, sdesc(sw + TILE + kk * 32, 16, 1024), bd, idesc, acc);
                }
                mma_commit(su32(&empty[s]));
            }
            mma_commit(su32(&accf));
        }
    } else {
        ok = mbar_wait(su32(&accf), 0, wlim);
        ok = __all_sync(0xffffffffu, ok);
        fence_after();
        const int q = warp & 3;
        // every MMA has completed, so the pipeline stages are free: each warp stages its 32 rows of a
        // 32-column chunk there (stride YEPI_LD floats) and stores full 128-byte row segments
        float* stg = reinterpret_cast<float*>(dsm + (base - raw)) + q * 32 * YEPI_LD;
        const int rbase = m0 + 32 * q;
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t p[32], qq[32];
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, p);
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(BN + c), qq);
                tmem_wait_ld();
#pragma unroll
                for (int v = 0; v < 32; v += 4)
                    *reinterpret_cast<float4*>(stg + lane * YEPI_LD + v) =
                        make_float4(__uint_as_float(p[v]) - __uint_as_float(qq[v + 1]),
                                    __uint_as_float(p[v + 1]) + __uint_as_float(qq[v]),
                                    __uint_as_float(p[v + 2]) - __uint_as_float(qq[v + 3]),
                                    __uint_as_float(p[v + 3]) + __uint_as_float(qq[v + 2]));
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3), cc = 4 * (lane & 7);
                    const int grow = rbase + rr, gcol = n0 + c + cc;
                    const float4 v = *reinterpret_cast<const float4*>(stg + rr * YEPI_LD + cc);
                    if (grow < ny && gcol < N2) {
                        float* dst = out + ((size_t)l * ny + grow) * N2 + gcol;
                        if (gcol + 4 <= N2) *reinterpret_cast<float4*>(dst) = v;
                        else {
                            dst[0] = v.x;
                            if (gcol + 1 < N2) dst[1] = v.y;
                            if (gcol + 2 < N2) dst[2] = v.z;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && lane == 0) {
        if (warp == 0) drain_tma(full, YSTAGES, issued);
        else if (warp == 1) drain_mma(&drainb);
    }
    fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
}

// stage counts of the persistent x-pass: 128-wide tiles two CTAs per SM, 256-wide tiles one CTA per SM
// (2 x 256 accumulator columns fill the tensor memory); 1024 bytes of slack align the ring
// the split (3xTF32) form holds the data tile, its remainder and both halves of the basis tile per stage
template <int BNT, bool SPLIT = false>
struct PersX {
    static constexpr int STAGES = SPLIT ? (BNT == 256 ? 2 : 3) : (BNT == 256 ? 4 : XSTAGES);
    static constexpr int STAGE_BYTES = (SPLIT ? 2 : 1) * (BM * BK * 4 + BNT * BK * 4);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + XEPI_BYTES + 1024;
};

// ---- persistent x-pass: one CTA walks many output tiles, the accumulator is double-buffered in tensor
// memory so that the epilogue of tile t overlaps the loads and MMAs of tile t+1 (the y-pass, whose two
// accumulators per tile would need all 512 columns for double buffering, keeps one tile per CTA) --------
// Barriers: full/empty per shared-memory stage (the stage counter runs across tiles), accf[b] (MMA ->
// epilogue: accumulator buffer b holds a finished tile), acce[b] (epilogue -> MMA: buffer b drained; four
// arrivals, one per epilogue warp).  Tiles are ordered N-fastest so that consecutive tiles of a CTA share
// their A rows in L2.
// SPLIT: 3xTF32 with tmBl the remainder of the basis; 320 threads, warps 6-9 split the data tiles.
// Stage layout: [A | B] (TF32), [A hi | A lo | B hi | B lo] (SPLIT).
// H: 16-bit operands, 1 = BF16, 2 = FP16 (kind::f16; a 128-byte swizzle row holds 64 of them, so a stage
// carries twice the K depth of the TF32 form in the same bytes); OBF: the output rounded to that type
// (row-major pairs).
template <int BNT, bool SPLIT, int H = 0, bool OBF = false>
__global__ void __launch_bounds__(SPLIT ? 320 : 192, 1)
xpass_tc_pers_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmBl, void* __restrict__ outv, int M, int N2, int K2,
                     float alpha, const double* __restrict__ alpha_dev, int aidx, int rows_per, int astride,
                     unsigned* status, long wlim, const double* __restrict__ alpha_dev2 = nullptr,
                     double* __restrict__ nsq_out = nullptr) {
    extern __shared__ uint8_t dsm[];
    constexpr int NS = PersX<BNT, SPLIT>::STAGES, BTILE = BNT * BK * 4, STAGE = PersX<BNT, SPLIT>::STAGE_BYTES;
    constexpr int KE = H ? 2 * BK : BK;    // K elements per stage (128 bytes per operand row)
    float* out = reinterpret_cast<float*>(outv);
    constexpr int AOFF_LO = TILE, BOFF = SPLIT ? 2 * TILE : TILE, BOFF_LO = BOFF + BTILE;
    __shared__ __align__(8) uint64_t full[NS], empty[NS], conv[NS], accf[2], acce[2], drainb;
    __shared__ int fail_any;
    __shared__ uint32_t tslot;
    const uint32_t raw = su32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K2 + KE - 1) / KE;
    const int ntn = (N2 + BNT - 1) / BNT, ntm = (M + BM - 1) / BM, ntiles = ntn * ntm;
    float* epi = reinterpret_cast<float*>(dsm + (base - raw) + NS * STAGE);   // epilogue staging rows
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(su32(&full[s]), 1);
            mbar_init(su32(&empty[s]), 1);
            mbar_init(su32(&conv[s]), 4);
        }
        for (int b = 0; b < 2; ++b) { mbar_init(su32(&accf[b]), 1); mbar_init(su32(&acce[b]), 4); }
        mbar_init(su32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(2 * BNT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    long issued = 0;   // pipeline iterations whose TMA loads the producer issued
    if (warp == 0) {
        if (lane == 0) {
            long it = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int n0 = (t % ntn) * BNT, m0 = (t / ntn) * BM;
                for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                    const int s = (int)(it % NS);
                    const uint32_t ph = (uint32_t)((it / NS) & 1);
                    if (it >= NS) ok = mbar_wait(su32(&empty[s]), ph ^ 1, wlim);
                    if (!ok) break;
                    const uint32_t sa = base + s * STAGE, sb = sa + BOFF;
                    mbar_expect_tx(su32(&full[s]), SPLIT ? TILE + 2 * BTILE : STAGE);
                    tma_2d(sa, &tmA, su32(&full[s]), kb * KE, m0);
                    tma_2d(sb, &tmB, su32(&full[s]), kb * KE, n0);
                    if (SPLIT) tma_2d(sa + BOFF_LO, &tmBl, su32(&full[s]), kb * KE, n0);
                    ++issued;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = H ? idesc_h16(H, BM, BNT, 0, 0) : idesc_tf32(BM, BNT, 0, 0);
            long it = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
                const int b = lt & 1;
                if (lt >= 2) ok = mbar_wait(su32(&acce[b]), (uint32_t)(((lt >> 1) - 1) & 1), wlim);
                if (!ok) break;
                fence_after();
                const uint32_t acc_t = tmem + (uint32_t)(b * BNT);
                for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                    const int s = (int)(it % NS);
                    const uint32_t ph = (uint32_t)((it / NS) & 1);
                    ok = mbar_wait(su32(SPLIT ? &conv[s] : &full[s]), ph, wlim);
                    if (!ok) break;
                    fence_after();
                    const uint32_t sa = base + s * STAGE, sb = sa + BOFF;
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t ad = sdesc(sa + kk * 32, 16, 1024), bd = sdesc(sb + kk * 32, 16, 1024);
                        if (SPLIT) {
                            // small products first: lo_a hi_b + hi_a lo_b + hi_a hi_b
                            mma_tf32(acc_t, sdesc(sa + AOFF_LO + kk * 32, 16, 1024), bd, idesc, (kb | kk) ? 1u : 0u);
                            mma_tf32(acc_t, ad, sdesc(sa + BOFF_LO + kk * 32, 16, 1024), idesc, 1u);
                            mma_tf32(acc_t, ad, bd, idesc, 1u);
                        } else {
                            mma_op<H>(acc_t, ad, bd, idesc, (kb | kk) ? 1u : 0u);
                        }
                    }
                    mma_commit(su32(&empty[s]));
                }
                if (ok) mma_commit(su32(&accf[b]));
            }
        }
    } else if (!SPLIT || warp < 6) {
        const int q = warp & 3;
        int lt = 0;
        float nacc = 0.f;   // squared norm of what this thread stored (OBF, nsq_out)
        const float al2 = alpha_dev2 ? (float)alpha_dev2[0] : 1.f;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            const int n0 = (t % ntn) * BNT, m0 = (t / ntn) * BM;
            // this thread's accumulator row; rows of the v-th vector of a batch scale by alpha_dev[aidx + v astride]
            const int arow = min(m0 + 32 * q + lane, M - 1);
            const float al = alpha * al2 * (alpha_dev ? (float)alpha_dev[aidx + (arow / rows_per) * astride] : 1.f);
            ok = __all_sync(0xffffffffu, mbar_wait(su32(&accf[b]), (uint32_t)((lt >> 1) & 1), wlim));
            if (!ok) break;
            fence_after();
            // each thread holds one row of the accumulator; 16-column halves go through this warp's staging
            // rows (stride XEPI_LD floats, conflict-free both ways) so that the stores are 64-byte row segments
            float* stg = epi + q * 32 * XEPI_LD;
            const int rbase = m0 + 32 * q;
#pragma unroll 1
            for (int c = 0; c < BNT; c += 32) {
                uint32_t r[32];
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BNT + c), r);
                tmem_wait_ld();
                if (OBF) {
                    // the thread's 32 columns as 16 16-bit pairs (64 bytes) into its staging row, then 16-byte
                    // pieces of four rows per instruction: 64-byte row segments in global memory
                    uint32_t* su = reinterpret_cast<uint32_t*>(stg);
                    if (nsq_out && m0 + 32 * q + lane < M)
#pragma unroll
                        for (int v = 0; v < 32; ++v) {
                            const float x = al * __uint_as_float(r[v]);
                            if (n0 + c + v < N2) nacc = fmaf(x, x, nacc);
                        }
#pragma unroll
                    for (int v = 0; v < 16; v += 4)
                        *reinterpret_cast<uint4*>(su + lane * XEPI_LD + v) =
                            make_uint4(pack16<H>(al * __uint_as_float(r[2 * v]), al * __uint_as_float(r[2 * v + 1])),
                                       pack16<H>(al * __uint_as_float(r[2 * v + 2]), al * __uint_as_float(r[2 * v + 3])),
                                       pack16<H>(al * __uint_as_float(r[2 * v + 4]), al * __uint_as_float(r[2 * v + 5])),
                                       pack16<H>(al * __uint_as_float(r[2 * v + 6]), al * __uint_as_float(r[2 * v + 7])));
                    __syncwarp();
                    uint16_t* ob = reinterpret_cast<uint16_t*>(outv);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = 8 * i + (lane >> 2), cc = 4 * (lane & 3);
                        const int grow = rbase + rr, gcol = n0 + c + 2 * cc;
                        const uint4 v = *reinterpret_cast<const uint4*>(su + rr * XEPI_LD + cc);
                        if (grow < M && gcol < N2) {
                            uint16_t* dst = ob + (size_t)grow * N2 + gcol;
                            if (gcol + 8 <= N2) *reinterpret_cast<uint4*>(dst) = v;
                            else {
                                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                                for (int e = 0; e < 4 && gcol + 2 * e < N2; ++e) reinterpret_cast<uint32_t*>(dst)[e] = w[e];
                            }
                        }
                    }
                    __syncwarp();
                    continue;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int v = 0; v < 16; v += 4)
                        *reinterpret_cast<float4*>(stg + lane * XEPI_LD + v) =
                            make_float4(al * __uint_as_float(r[16 * h + v]), al * __uint_as_float(r[16 * h + v + 1]),
                                        al * __uint_as_float(r[16 * h + v + 2]), al * __uint_as_float(r[16 * h + v + 3]));
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = 8 * i + (lane >> 2), cc = 4 * (lane & 3);
                        const int grow = rbase + rr, gcol = n0 + c + 16 * h + cc;
                        const float4 v = *reinterpret_cast<const float4*>(stg + rr * XEPI_LD + cc);
                        if (grow < M && gcol < N2) {
                            float* dst = out + (size_t)grow * N2 + gcol;
                            if (gcol + 4 <= N2) *reinterpret_cast<float4*>(dst) = v;
                            else {
                                dst[0] = v.x;
                                if (gcol + 1 < N2) dst[1] = v.y;
                                if (gcol + 2 < N2) dst[2] = v.z;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(su32(&acce[b]));
        }
        if (nsq_out) {
            double d = (double)nacc;
            for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
            if (lane == 0) atomicAdd(nsq_out, d);
        }
    } else {
        // converter warps (SPLIT): split each data tile once its TMA loads have landed, then release the
        // stage to the MMA thread (one arrival per warp)
        const int ct = threadIdx.x - 192;
        long it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
            for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                const int s = (int)(it % NS);
                ok = __all_sync(0xffffffffu, mbar_wait(su32(&full[s]), (uint32_t)((it / NS) & 1), wlim));
                if (!ok) break;
                float4* a = reinterpret_cast<float4*>(dsm + (base - raw) + (size_t)s * STAGE);
                split_tile(a, a + AOFF_LO / 16, ct);
                __syncwarp();
                if (lane == 0) mbar_arrive(su32(&conv[s]));
            }
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && lane == 0) {
        if (warp == 0) drain_tma(full, NS, issued);
        else if (warp == 1) drain_mma(&drainb);
    }
    fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BNT) : "memory");
}

// ---- persistent y-pass: the accumulator pair (P, Q) of a tile is double-buffered in tensor memory
// (2 x 2 x 128 columns), so the epilogue of tile t overlaps the loads and MMAs of tile t+1; one CTA per
// SM.  Tiles are ordered (slice, column block, row block) with the row block fastest, so that the two row
// blocks of a data tile run at the same time on neighbouring CTAs and share it in L2.  Barriers as in the
// persistent x-pass.
// pipeline stages and shared memory; the split (3xTF32) form adds the remainders of W and of the data tile
template <bool SPLIT>
struct PersY {
    static constexpr int STAGES = SPLIT ? 2 : 4;
    static constexpr int STAGE_BYTES = (SPLIT ? 6 : 3) * TILE;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 4 * 32 * YEPI_LD * 4 + 1024;
};

// SPLIT: 3xTF32 with tmWl the remainder of W; 320 threads, warps 6-9 split the data tiles.
// Stage layout: [Wr | Wi | D] (TF32), [Wr hi | Wi hi | D hi | Wr lo | Wi lo | D lo] (SPLIT); D is 4 boxes of
// 32 K-rows x 128 bytes.
// H: 16-bit operands and output (1 = BF16, 2 = FP16), the output scaled by alpha.  W (K-major) as in the
// TF32 form with 64 K elements per 128-byte row;
// the data tile is two boxes of 64 columns x 64 K-rows in the ordinary 128-byte swizzle (16-byte chunks),
// the canonical MN-major layout of 16-bit operands: LBO = the next 64-column chunk (8 KiB), SBO = the next
// 8-row K group (1 KiB), 2 KiB per MMA K-step of 16.
template <bool SPLIT, int H = 0>
__global__ void __launch_bounds__(SPLIT ? 320 : 192, 1)
ypass_tc_pers_kernel(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmY,
                     const __grid_constant__ CUtensorMap tmWl, void* __restrict__ outv, int ny, int N2, int nz,
                     unsigned* status, long wlim, float alpha = 1.f, double* __restrict__ h16d = nullptr,
                     float gain = 1.f, int role = 0) {
    extern __shared__ uint8_t dsm[];
    constexpr int YPS = PersY<SPLIT>::STAGES, STAGE = PersY<SPLIT>::STAGE_BYTES;
    constexpr int WLO = 3 * TILE, DLO = 5 * TILE;
    constexpr int KE = H ? 2 * BK : BK;
    float* out = reinterpret_cast<float*>(outv);
    __shared__ __align__(8) uint64_t full[YPS], empty[YPS], conv[YPS], accf[2], acce[2], drainb;
    __shared__ int fail_any;
    __shared__ uint32_t tslot;
    const uint32_t raw = su32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (ny + KE - 1) / KE;
    const int ntm = (ny + BM - 1) / BM, ntn = (N2 + BN - 1) / BN, ntiles = ntm * ntn * nz;
    float* epi = reinterpret_cast<float*>(dsm + (base - raw) + YPS * STAGE);   // epilogue staging rows
    if (threadIdx.x == 0) {
        for (int s = 0; s < YPS; ++s) {
            mbar_init(su32(&full[s]), 1);
            mbar_init(su32(&empty[s]), 1);
            mbar_init(su32(&conv[s]), 4);
        }
        for (int b = 0; b < 2; ++b) { mbar_init(su32(&accf[b]), 1); mbar_init(su32(&acce[b]), 4); }
        mbar_init(su32(&drainb), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(4 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    long issued = 0;   // pipeline iterations whose TMA loads the producer issued
    if (warp == 0) {
        if (lane == 0) {
            long it = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int mb = t % ntm, nb = (t / ntm) % ntn, l = t / (ntm * ntn);
                const int m0 = mb * BM, n0 = nb * BN;
                for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                    const int s = (int)(it % YPS);
                    const uint32_t ph = (uint32_t)((it / YPS) & 1);
                    if (it >= YPS) ok = mbar_wait(su32(&empty[s]), ph ^ 1, wlim);
                    if (!ok) break;
                    const uint32_t sw = base + s * STAGE, sb = sw + 2 * TILE;
                    mbar_expect_tx(su32(&full[s]), SPLIT ? 5 * TILE : STAGE);
                    tma_3d(sw, &tmW, su32(&full[s]), kb * KE, m0, 0);
                    tma_3d(sw + TILE, &tmW, su32(&full[s]), kb * KE, m0, 1);
                    if (SPLIT) {
                        tma_3d(sw + WLO, &tmWl, su32(&full[s]), kb * BK, m0, 0);
                        tma_3d(sw + WLO + TILE, &tmWl, su32(&full[s]), kb * BK, m0, 1);
                    }
                    if (H) {
#pragma unroll
                        for (int q = 0; q < BN / 64; ++q) tma_3d(sb + q * 8192, &tmY, su32(&full[s]), n0 + 64 * q, kb * KE, l);
                    } else {
#pragma unroll
                        for (int q = 0; q < BN / 32; ++q) tma_3d(sb + q * 4096, &tmY, su32(&full[s]), n0 + 32 * q, kb * BK, l);
                    }
                    ++issued;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = H ? idesc_h16(H, BM, BN, 0, 1) : idesc_tf32(BM, BN, 0, 1);
            long it = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
                const int b = lt & 1;
                if (lt >= 2) ok = mbar_wait(su32(&acce[b]), (uint32_t)(((lt >> 1) - 1) & 1), wlim);
                if (!ok) break;
                fence_after();
                const uint32_t accP = tmem + (uint32_t)(b * 2 * BN), accQ = accP + BN;
                for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                    const int s = (int)(it % YPS);
                    const uint32_t ph = (uint32_t)((it / YPS) & 1);
                    ok = mbar_wait(su32(SPLIT ? &conv[s] : &full[s]), ph, wlim);
                    if (!ok) break;
                    fence_after();
                    const uint32_t sw = base + s * STAGE, sb = sw + 2 * TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        // MN-major: LBO = next 32-column chunk (4 KiB), SBO = next 4-row K group (512 B)
                        // (BF16: next 64-column chunk 8 KiB, next 8-row group 1 KiB, layout 2)
                        const uint64_t bd = H ? sdesc(sb + kk * 2048, 8192, 1024, 2) : sdesc(sb + kk * 1024, 4096, 512, 1);
                        const uint64_t wr = sdesc(sw + kk * 32, 16, 1024), wi = sdesc(sw + TILE + kk * 32, 16, 1024);
                        const uint32_t acc = (kb | kk) ? 1u : 0u;
                        if (SPLIT) {
                            // small products first: hi_W lo_D + lo_W hi_D + hi_W hi_D
                            const uint64_t bl = sdesc(sw + DLO + kk * 1024, 4096, 512, 1);
                            mma_tf32(accP, wr, bl, idesc, acc);
                            mma_tf32(accQ, wi, bl, idesc, acc);
                            mma_tf32(accP, sdesc(sw + WLO + kk * 32, 16, 1024), bd, idesc, 1u);
                            mma_tf32(accQ, sdesc(sw + WLO + TILE + kk * 32, 16, 1024), bd, idesc, 1u);
                            mma_tf32(accP, wr, bd, idesc, 1u);
                            mma_tf32(accQ, wi, bd, idesc, 1u);
                        } else {
                            mma_op<H>(accP, wr, bd, idesc, acc);
                            mma_op<H>(accQ, wi, bd, idesc, acc);
                        }
                    }
                    mma_commit(su32(&empty[s]));
                }
                if (ok) mma_commit(su32(&accf[b]));
            }
        }
    } else if (!SPLIT || warp < 6) {
        const int q = warp & 3;
        float* stg = epi + q * 32 * YEPI_LD;
        int lt = 0;
        // FP16 chain with dynamic stage scales (h16d): role 0 (forward) scales by the bound of ||T1|| (h16d[0]),
        // records it in h16d[4] and accumulates its own output's squared norm into h16d[1]; role 1 (inverse)
        // scales by that of ||T3|| (h16d[2]), records h16d[6] and the undo factor 1/(s2 s3 s4) in h16d[7]
        float nacc = 0.f;
        if (h16d) {
            const float sc = stage_scale((double)gain, h16d[role == 0 ? 0 : 2]);
            if (blockIdx.x == 0 && threadIdx.x == 64) {
                h16d[role == 0 ? 4 : 6] = sc;
                if (role == 1) h16d[7] = 1.0 / (h16d[4] * h16d[5] * (double)sc);
            }
            alpha *= sc;
        }
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            const int mb = t % ntm, nb = (t / ntm) % ntn, l = t / (ntm * ntn);
            const int m0 = mb * BM, n0 = nb * BN;
            ok = __all_sync(0xffffffffu, mbar_wait(su32(&accf[b]), (uint32_t)((lt >> 1) & 1), wlim));
            if (!ok) break;
            fence_after();
            const int rbase = m0 + 32 * q;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t p[32], qq[32];
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * BN + c), p);
                TMEM_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * BN + BN + c), qq);
                tmem_wait_ld();
                if (H) {
                    // 16 complex values (re = P_re - Q_im, im = P_im + Q_re) as 16-bit pairs: 64 bytes per row
                    uint32_t* su = reinterpret_cast<uint32_t*>(stg);
#pragma unroll
                    for (int v = 0; v < 16; v += 4) {
                        uint32_t w[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int k = 2 * (v + e);
                            const float re = alpha * (__uint_as_float(p[k]) - __uint_as_float(qq[k + 1]));
                            const float im = alpha * (__uint_as_float(p[k + 1]) + __uint_as_float(qq[k]));
                            w[e] = pack16<H>(re, im);
                            if (h16d && role == 0 && rbase + lane < ny && n0 + c + k < N2) nacc = fmaf(re, re, fmaf(im, im, nacc));
                        }
                        *reinterpret_cast<uint4*>(su + lane * XEPI_LD + v) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    __syncwarp();
                    uint16_t* ob = reinterpret_cast<uint16_t*>(outv);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = 8 * i + (lane >> 2), cc = 4 * (lane & 3);
                        const int grow = rbase + rr, gcol = n0 + c + 2 * cc;
                        const uint4 v = *reinterpret_cast<const uint4*>(su + rr * XEPI_LD + cc);
                        if (grow < ny && gcol < N2) {
                            uint16_t* dst = ob + ((size_t)l * ny + grow) * N2 + gcol;
                            if (gcol + 8 <= N2) *reinterpret_cast<uint4*>(dst) = v;
                            else {
                                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                                for (int e = 0; e < 4 && gcol + 2 * e < N2; ++e) reinterpret_cast<uint32_t*>(dst)[e] = w[e];
                            }
                        }
                    }
                    __syncwarp();
                    continue;
                }
#pragma unroll
                for (int v = 0; v < 32; v += 4)
                    *reinterpret_cast<float4*>(stg + lane * YEPI_LD + v) =
                        make_float4(__uint_as_float(p[v]) - __uint_as_float(qq[v + 1]),
                                    __uint_as_float(p[v + 1]) + __uint_as_float(qq[v]),
                                    __uint_as_float(p[v + 2]) - __uint_as_float(qq[v + 3]),
                                    __uint_as_float(p[v + 3]) + __uint_as_float(qq[v + 2]));
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3), cc = 4 * (lane & 7);
                    const int grow = rbase + rr, gcol = n0 + c + cc;
                    const float4 v = *reinterpret_cast<const float4*>(stg + rr * YEPI_LD + cc);
                    if (grow < ny && gcol < N2) {
                        float* dst = out + ((size_t)l * ny + grow) * N2 + gcol;
                        if (gcol + 4 <= N2) *reinterpret_cast<float4*>(dst) = v;
                        else {
                            dst[0] = v.x;
                            if (gcol + 1 < N2) dst[1] = v.y;
                            if (gcol + 2 < N2) dst[2] = v.z;
                        }
                    }
                }
                __syncwarp();
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(su32(&acce[b]));
        }
        if (h16d && role == 0) {
            double d = (double)nacc;
            for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
            if (lane == 0) atomicAdd(h16d + 1, d);
        }
    } else {
        // converter warps (SPLIT): split each data tile once its TMA loads have landed
        const int ct = threadIdx.x - 192;
        long it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
            for (int kb = 0; kb < nk && ok; ++kb, ++it) {
                const int s = (int)(it % YPS);
                ok = __all_sync(0xffffffffu, mbar_wait(su32(&full[s]), (uint32_t)((it / YPS) & 1), wlim));
                if (!ok) break;
                unsigned char* st = dsm + (base - raw) + (size_t)s * STAGE;
                split_tile(reinterpret_cast<float4*>(st + 2 * TILE), reinterpret_cast<float4*>(st + DLO), ct);
                __syncwarp();
                if (lane == 0) mbar_arrive(su32(&conv[s]));
            }
    }
    if (!ok) {
        atomicOr(status, (unsigned)HELM_DEV_WAIT);
        fail_any = 1;
    }
    __syncthreads();
    if (fail_any && lane == 0) {
        if (warp == 0) drain_tma(full, YPS, issued);
        else if (warp == 1) drain_mma(&drainb);
    }
    fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * BN) : "memory");
}

// ---- operand preparation (set-up) ----------------------------------------------------------------
// v rounded to TF32 (hi) and, when lo is wanted, the TF32 rounding of the remainder v - hi
__device__ __forceinline__ float to_tf32(double v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)v));
    return __uint_as_float(r);
}
__device__ __forceinline__ void put_split(float* hi, float* lo, size_t i, double v) {
    const float h = to_tf32(v);
    hi[i] = h;
    if (lo) lo[i] = to_tf32(v - (double)h);
}

// B[2n][2k] from W_kn = src[n][k] (src row-major N x N complex128); Bl (may be NULL) the remainders
__global__ void embed_x_kernel(int N, const double2* __restrict__ src, float* __restrict__ B, float* __restrict__ Bl) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * N) return;
    const int n = (int)(id / N), k = (int)(id % N);
    const double2 w = src[(size_t)n * N + k];
    const size_t L2 = 2 * (size_t)N;
    put_split(B, Bl, (2 * n) * L2 + 2 * k, w.x);
    put_split(B, Bl, (2 * n) * L2 + 2 * k + 1, -w.y);
    put_split(B, Bl, (2 * n + 1) * L2 + 2 * k, w.y);
    put_split(B, Bl, (2 * n + 1) * L2 + 2 * k + 1, w.x);
}

// W planes: re at [0][j'][j], im at [1][j'][j], row stride ldw (zero padded); Wl (may be NULL) the remainders
__global__ void split_y_kernel(int N, int ldw, const double2* __restrict__ src, float* __restrict__ W,
                               float* __restrict__ Wl) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * ldw) return;
    const int r = (int)(id / ldw), k = (int)(id % ldw);
    const double2 w = k < N ? src[(size_t)r * N + k] : make_double2(0.0, 0.0);
    put_split(W, Wl, (size_t)r * ldw + k, w.x);
    put_split(W, Wl, (size_t)N * ldw + (size_t)r * ldw + k, w.y);
}

// 16-bit (round to nearest even from FP64) copies of an operand set: the same layouts as the TF32 ones
template <int H>
__device__ __forceinline__ uint16_t h16_bits(double v) {
    if (H == 2) return __half_as_ushort(__double2half(v));
    return __bfloat16_as_ushort(__double2bfloat16(v));
}
template <int H>
__global__ void embed_x_h16_kernel(int N, const double2* __restrict__ src, uint16_t* __restrict__ B) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * N) return;
    const int n = (int)(id / N), k = (int)(id % N);
    const double2 w = src[(size_t)n * N + k];
    const size_t L2 = 2 * (size_t)N;
    B[(2 * n) * L2 + 2 * k] = h16_bits<H>(w.x);
    B[(2 * n) * L2 + 2 * k + 1] = h16_bits<H>(-w.y);
    B[(2 * n + 1) * L2 + 2 * k] = h16_bits<H>(w.y);
    B[(2 * n + 1) * L2 + 2 * k + 1] = h16_bits<H>(w.x);
}
template <int H>
__global__ void split_y_h16_kernel(int N, int ldw, const double2* __restrict__ src, uint16_t* __restrict__ W) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)N * ldw) return;
    const int r = (int)(id / ldw), k = (int)(id % ldw);
    const double2 w = k < N ? src[(size_t)r * N + k] : make_double2(0.0, 0.0);
    W[(size_t)r * ldw + k] = h16_bits<H>(w.x);
    W[(size_t)N * ldw + (size_t)r * ldw + k] = h16_bits<H>(w.y);
}

helm_status encode(TcState* t, CUtensorMap* map, int rank, void* ptr, const cuuint64_t* dims, const cuuint64_t* strides,
                   const cuuint32_t* box, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B,
                   CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32) {
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = t->encode(map, dt, rank, ptr, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HELM_OK : HELM_ERR_CUDA;
}

size_t xsmem() { return (size_t)XSTAGES * 2 * TILE + 1024; }
size_t ysmem() { return (size_t)YSTAGES * 3 * TILE + 1024; }
int g_sms = 0;

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// the x-pass and y-pass operands of set i from FP64 sources (x: W_kn = srcx[n][k]; y: srcy)
helm_status tc_fill_set(TcState* t, int nx, int ny, int i, const double2* srcx, const double2* srcy, cudaStream_t s) {
    const size_t nb = (size_t)4 * nx * nx, nw = (size_t)2 * ny * t->ldw;
    if (cudaMalloc(&t->Bx[i], nb * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    if (cudaMalloc(&t->Wy[i], nw * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    if (t->split) {
        if (cudaMalloc(&t->Bxl[i], nb * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
        if (cudaMalloc(&t->Wyl[i], nw * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
    }
    embed_x_kernel<<<(unsigned)((nx * (size_t)nx + 255) / 256), 256, 0, s>>>(nx, srcx, t->Bx[i], t->Bxl[i]);
    split_y_kernel<<<(unsigned)((ny * (size_t)t->ldw + 255) / 256), 256, 0, s>>>(ny, t->ldw, srcy, t->Wy[i], t->Wyl[i]);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

}  // namespace

helm_status tc_encode_set(TcState* t, int nx, int ny, int i);

helm_status tc_prepare(helm_ctx* c, cudaStream_t s) {
    if (c->nx % 2 != 0) return HELM_ERR_UNSUPPORTED;
    const int h16 = c->opt.precision == HELM_PREC_BF16 ? 1 : c->opt.precision == HELM_PREC_FP16 ? 2 : 0;
    if (c->opt.precision != HELM_PREC_TF32 && c->opt.precision != HELM_PREC_TF32X3 && !h16) return HELM_ERR_UNSUPPORTED;
    if (h16 && c->nx % 4 != 0) return HELM_ERR_UNSUPPORTED;
    TcState* t = new TcState();
    c->tmaps = t;
    t->split = c->opt.precision == HELM_PREC_TF32X3;
    t->h16 = h16;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&t->encode, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !t->encode) {
        cudaGetLastError();
        return HELM_ERR_CUDA;
    }
    const int nx = c->nx, ny = c->ny;
    t->ldw = (ny + 3) / 4 * 4;
    helm_status st;
    // forward: W_kn = Vxi[n][k], V_y^-1; inverse: W_kn = Vx[n][k], V_y
    if ((st = tc_fill_set(t, nx, ny, 0, c->Vxi, c->Vyi, s)) != HELM_OK) return st;
    if ((st = tc_fill_set(t, nx, ny, 1, c->Vx, c->Vy, s)) != HELM_OK) return st;
    for (int i = 0; i < 2; ++i)
        if (tc_encode_set(t, nx, ny, i) != HELM_OK) return HELM_ERR_CUDA;
    if (t->h16 == 1) {   // BF16 has FP32's range: no stage scales
        for (int k = 0; k < 5; ++k) c->h16s[k] = 1.f;
        c->h16s[5] = (float)(c->h[2] * c->h[2]);
    }
    if (t->h16 == 2) {   // FP16: power-of-two stage scales from the set-up bounds, and the norm scratch
        helm_status sst = h16_scales(c, s);
        if (sst != HELM_OK) return sst;
        if (cudaMalloc(&c->h16n, (2 + 1024) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->h16d, 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return HELM_ERR_NOMEM;
        }
        HELM_CUDA_TRY(cudaMemsetAsync(c->h16d, 0, 8 * sizeof(double), s));
    }
    if (t->h16) {
        // the EigT sets in 16 bits (the TF32 sets above serve helm_precond_step and the PFFT passes)
        t->ldwb = (ny + 7) / 8 * 8;
        const size_t nb = (size_t)4 * nx * nx, nw = (size_t)2 * ny * t->ldwb;
        const double2* sx[2] = {c->Vxi, c->Vx};
        const double2* sy[2] = {c->Vyi, c->Vy};
        for (int i = 0; i < 2; ++i) {
            if (cudaMalloc(&t->Bxb[i], nb * sizeof(uint16_t)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
            if (cudaMalloc(&t->Wyb[i], nw * sizeof(uint16_t)) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_NOMEM; }
            const unsigned gx = (unsigned)((nx * (size_t)nx + 255) / 256), gy = (unsigned)((ny * (size_t)t->ldwb + 255) / 256);
            if (h16 == 2) {
                embed_x_h16_kernel<2><<<gx, 256, 0, s>>>(nx, sx[i], t->Bxb[i]);
                split_y_h16_kernel<2><<<gy, 256, 0, s>>>(ny, t->ldwb, sy[i], t->Wyb[i]);
            } else {
                embed_x_h16_kernel<1><<<gx, 256, 0, s>>>(nx, sx[i], t->Bxb[i]);
                split_y_h16_kernel<1><<<gy, 256, 0, s>>>(ny, t->ldwb, sy[i], t->Wyb[i]);
            }
            HELM_CUDA_TRY(cudaGetLastError());
            const cuuint64_t d[2] = {(cuuint64_t)2 * nx, (cuuint64_t)2 * nx};
            const cuuint64_t st[1] = {(cuuint64_t)2 * nx * sizeof(uint16_t)};
            const cuuint32_t box[2] = {2 * BK, BN}, box256[2] = {2 * BK, 256};
            const cuuint64_t dw[3] = {(cuuint64_t)ny, (cuuint64_t)ny, 2};
            const cuuint64_t sw[2] = {(cuuint64_t)t->ldwb * sizeof(uint16_t), (cuuint64_t)t->ldwb * ny * sizeof(uint16_t)};
            const cuuint32_t bw[3] = {2 * BK, BM, 1};
            const CUtensorMapDataType bt = h16 == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
            if (encode(t, &t->mapBxb[i], 2, t->Bxb[i], d, st, box, CU_TENSOR_MAP_SWIZZLE_128B, bt) != HELM_OK) return HELM_ERR_CUDA;
            if ((2 * nx) % 256 == 0 &&
                encode(t, &t->mapBxb256[i], 2, t->Bxb[i], d, st, box256, CU_TENSOR_MAP_SWIZZLE_128B, bt) != HELM_OK)
                return HELM_ERR_CUDA;
            if (encode(t, &t->mapWyb[i], 3, t->Wyb[i], dw, sw, bw, CU_TENSOR_MAP_SWIZZLE_128B, bt) != HELM_OK) return HELM_ERR_CUDA;
        }
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, false, 1, true>, PersX<128, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, false, 1, true>, PersX<256, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, false, 1, false>, PersX<128, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, false, 1, false>, PersX<256, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, false, 2, true>, PersX<128, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, false, 2, true>, PersX<256, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, false, 2, false>, PersX<128, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, false, 2, false>, PersX<256, false>::SMEM));
        HELM_CUDA_TRY(smem_attr(ypass_tc_pers_kernel<false, 1>, PersY<false>::SMEM));
        HELM_CUDA_TRY(smem_attr(ypass_tc_pers_kernel<false, 2>, PersY<false>::SMEM));
    }
    HELM_CUDA_TRY(smem_attr(xpass_tc_kernel, xsmem()));
    HELM_CUDA_TRY(smem_attr(ypass_tc_kernel, ysmem()));
    HELM_CUDA_TRY(smem_attr(ypass_tc_pers_kernel<false>, PersY<false>::SMEM));
    HELM_CUDA_TRY(smem_attr(ypass_tc_pers_kernel<true>, PersY<true>::SMEM));
    HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, false>, PersX<128, false>::SMEM));
    HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, false>, PersX<256, false>::SMEM));
    HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<128, true>, PersX<128, true>::SMEM));
    HELM_CUDA_TRY(smem_attr(xpass_tc_pers_kernel<256, true>, PersX<256, true>::SMEM));
    HELM_CUDA_TRY(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, c->device));
    return HELM_OK;
}

// TMA descriptors of operand set i (its matrices already written)
helm_status tc_encode_set(TcState* t, int nx, int ny, int i) {
    const cuuint64_t d[2] = {(cuuint64_t)2 * nx, (cuuint64_t)2 * nx};
    const cuuint64_t st[1] = {(cuuint64_t)2 * nx * sizeof(float)};
    const cuuint32_t box[2] = {BK, BN};
    const cuuint64_t dw[3] = {(cuuint64_t)ny, (cuuint64_t)ny, 2};
    const cuuint64_t sw[2] = {(cuuint64_t)t->ldw * sizeof(float), (cuuint64_t)t->ldw * ny * sizeof(float)};
    const cuuint32_t bw[3] = {BK, BM, 1};
    const cuuint32_t box256[2] = {BK, 256};
    for (int h = 0; h < (t->split ? 2 : 1); ++h) {
        float* bx = h ? t->Bxl[i] : t->Bx[i];
        float* wy = h ? t->Wyl[i] : t->Wy[i];
        if (encode(t, h ? &t->mapBxl[i] : &t->mapBx[i], 2, bx, d, st, box) != HELM_OK) return HELM_ERR_CUDA;
        if ((2 * nx) % 256 == 0)   // the only grids that take 256-wide tiles
            if (encode(t, h ? &t->mapBx256l[i] : &t->mapBx256[i], 2, bx, d, st, box256) != HELM_OK) return HELM_ERR_CUDA;
        if (encode(t, h ? &t->mapWyl[i] : &t->mapWy[i], 3, wy, dw, sw, bw) != HELM_OK) return HELM_ERR_CUDA;
    }
    return HELM_OK;
}

// PFFT on the tensor cores: operand sets 2 (forward: rows times S_x, S_y^T times slices) and 3 (inverse:
// rows times S_x^T, S_y times slices) from the FP64 sine bases S[l][j] (row-major, real).
helm_status tc_prepare_sine(helm_ctx* c, const double2* Sx, const double2* Sy, const double2* SxT, const double2* SyT,
                            cudaStream_t s) {
    TcState* t = (TcState*)c->tmaps;
    if (!t) return HELM_ERR_UNSUPPORTED;
    const int nx = c->nx, ny = c->ny;
    helm_status st;
    // x-pass computes row . src^T: forward wants row . S_x (src = S_x^T), inverse row . S_x^T (src = S_x);
    // y-pass computes src . slice: forward S_y^T, inverse S_y
    if ((st = tc_fill_set(t, nx, ny, 2, SxT, SyT, s)) != HELM_OK) return st;
    if ((st = tc_fill_set(t, nx, ny, 3, Sx, Sy, s)) != HELM_OK) return st;
    for (int i = 2; i < 4; ++i)
        if (tc_encode_set(t, nx, ny, i) != HELM_OK) return HELM_ERR_CUDA;
    return HELM_OK;
}

helm_status tc_xpass(helm_ctx* c, int inverse, const float2* in, float2* out, float alpha, const double* alpha_dev,
                     int aidx, cudaStream_t s, int nb, int astride) {
    TcState* t = (TcState*)c->tmaps;
    if (!t) return HELM_ERR_UNSUPPORTED;
    // nb vectors of the grid back to back: one GEMM over nb N_y N_z rows
    const int rp = c->ny * c->nz, as = astride;
    const int M = rp * nb, N2 = 2 * c->nx;
    CUtensorMap mapA;
    const cuuint64_t d[2] = {(cuuint64_t)N2, (cuuint64_t)M};
    const cuuint64_t st[1] = {(cuuint64_t)N2 * sizeof(float)};
    const cuuint32_t box[2] = {BK, BM};
    if (encode(t, &mapA, 2, (void*)in, d, st, box) != HELM_OK) return HELM_ERR_CUDA;
    dim3 grid((N2 + BN - 1) / BN, (M + BM - 1) / BM);
    const long wl = (long)c->wait_limit;
    float* o = (float*)out;
    if (t->split && g_sms > 0) {
        // 3xTF32: persistent kernels only
        if (N2 % 256 == 0) {
            const int ntiles = (N2 / 256) * (int)grid.y;
            const int pg = ntiles < g_sms ? ntiles : g_sms;
            xpass_tc_pers_kernel<256, true><<<pg, 320, PersX<256, true>::SMEM, s>>>(
                mapA, t->mapBx256[inverse], t->mapBx256l[inverse], o, M, N2, N2, alpha, alpha_dev, aidx, rp, as, c->status_d, wl);
        } else {
            const int ntiles = (int)(grid.x * grid.y);
            const int pg = ntiles < g_sms ? ntiles : g_sms;
            xpass_tc_pers_kernel<128, true><<<pg, 320, PersX<128, true>::SMEM, s>>>(
                mapA, t->mapBx[inverse], t->mapBxl[inverse], o, M, N2, N2, alpha, alpha_dev, aidx, rp, as, c->status_d, wl);
        }
    } else if (c->tune_tc == 1 && g_sms > 0) {
        if (N2 % 256 == 0) {
            // 256-wide tiles, one CTA per SM
            const int ntiles = (N2 / 256) * (int)grid.y;
            const int pg = ntiles < g_sms ? ntiles : g_sms;
            xpass_tc_pers_kernel<256, false><<<pg, 192, PersX<256, false>::SMEM, s>>>(
                mapA, t->mapBx256[inverse], t->mapBx256[inverse], o, M, N2, N2, alpha, alpha_dev, aidx, rp, as, c->status_d, wl);
        } else {
            const int ntiles = (int)(grid.x * grid.y);
            const int pg = ntiles < 2 * g_sms ? ntiles : 2 * g_sms;
            xpass_tc_pers_kernel<128, false><<<pg, 192, PersX<128, false>::SMEM, s>>>(
                mapA, t->mapBx[inverse], t->mapBx[inverse], o, M, N2, N2, alpha, alpha_dev, aidx, rp, as, c->status_d, wl);
        }
    } else {
        xpass_tc_kernel<<<grid, 192, xsmem(), s>>>(mapA, t->mapBx[inverse], o, M, N2, N2, alpha, alpha_dev, aidx, rp, as,
                                                    c->status_d, wl);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

helm_status tc_ypass(helm_ctx* c, int inverse, const float2* in, float2* out, cudaStream_t s, int nb) {
    TcState* t = (TcState*)c->tmaps;
    if (!t) return HELM_ERR_UNSUPPORTED;
    const int ny = c->ny, N2 = 2 * c->nx, nzb = c->nz * nb;   // nb vectors: nb N_z slices
    CUtensorMap mapY;
    const cuuint64_t d[3] = {(cuuint64_t)N2, (cuuint64_t)ny, (cuuint64_t)nzb};
    const cuuint64_t st[2] = {(cuuint64_t)N2 * sizeof(float), (cuuint64_t)N2 * ny * sizeof(float)};
    const cuuint32_t box[3] = {32, BK, 1};
    if (encode(t, &mapY, 3, (void*)in, d, st, box, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B) != HELM_OK) return HELM_ERR_CUDA;
    dim3 grid((N2 + BN - 1) / BN, (ny + BM - 1) / BM, nzb);
    const long wl = (long)c->wait_limit;
    const int ntiles = (int)(grid.x * grid.y * grid.z);
    const int pg = g_sms > 0 && ntiles > g_sms ? g_sms : ntiles;
    if (t->split && g_sms > 0) {
        ypass_tc_pers_kernel<true><<<pg, 320, PersY<true>::SMEM, s>>>(t->mapWy[inverse], mapY, t->mapWyl[inverse],
                                                                     (float*)out, ny, N2, nzb, c->status_d, wl);
    } else if (c->tune_ypers && g_sms > 0) {
        ypass_tc_pers_kernel<false><<<pg, 192, PersY<false>::SMEM, s>>>(t->mapWy[inverse], mapY, t->mapWy[inverse],
                                                                       (float*)out, ny, N2, nzb, c->status_d, wl);
    } else {
        ypass_tc_kernel<<<grid, 192, ysmem(), s>>>(t->mapWy[inverse], mapY, (float*)out, ny, N2, c->status_d, wl);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// 16-bit transform chain (HELM_PREC_BF16, HELM_PREC_FP16): x-pass from a 16-bit grid (N_y N_z nb rows of
// 2 N_x) to a 16-bit or, when out_h16 is 0, an FP32 (complex64) grid, scaled as tc_xpass
template <int H, bool OBF>
void xpass_h16_launch(TcState* t, helm_ctx* c, int inverse, const CUtensorMap& mapA, void* out, int M, int N2,
                      float alpha, const double* alpha_dev, int aidx, int rp, int astride, cudaStream_t s,
                      const double* alpha_dev2, double* nsq_out) {
    const long wl = (long)c->wait_limit;
    const int mt = (M + BM - 1) / BM;
    if (N2 % 256 == 0) {
        const int ntiles = (N2 / 256) * mt, pg = ntiles < g_sms ? ntiles : g_sms;
        xpass_tc_pers_kernel<256, false, H, OBF><<<pg, 192, PersX<256, false>::SMEM, s>>>(
            mapA, t->mapBxb256[inverse], t->mapBxb256[inverse], out, M, N2, N2, alpha, alpha_dev, aidx, rp, astride,
            c->status_d, wl, alpha_dev2, nsq_out);
    } else {
        const int ntiles = ((N2 + BN - 1) / BN) * mt, pg = ntiles < 2 * g_sms ? ntiles : 2 * g_sms;
        xpass_tc_pers_kernel<128, false, H, OBF><<<pg, 192, PersX<128, false>::SMEM, s>>>(
            mapA, t->mapBxb[inverse], t->mapBxb[inverse], out, M, N2, N2, alpha, alpha_dev, aidx, rp, astride,
            c->status_d, wl, alpha_dev2, nsq_out);
    }
}

helm_status tc_xpass_h16(helm_ctx* c, int inverse, const void* in, void* out, int out_h16, float alpha,
                         const double* alpha_dev, int aidx, cudaStream_t s, int nb, int astride,
                         const double* alpha_dev2, double* nsq_out) {
    TcState* t = (TcState*)c->tmaps;
    if (!t || !t->h16 || g_sms <= 0) return HELM_ERR_UNSUPPORTED;
    const int rp = c->ny * c->nz;
    const int M = rp * nb, N2 = 2 * c->nx;
    CUtensorMap mapA;
    const cuuint64_t d[2] = {(cuuint64_t)N2, (cuuint64_t)M};
    const cuuint64_t st[1] = {(cuuint64_t)N2 * sizeof(uint16_t)};
    const cuuint32_t box[2] = {2 * BK, BM};
    const CUtensorMapDataType dt = t->h16 == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (encode(t, &mapA, 2, (void*)in, d, st, box, CU_TENSOR_MAP_SWIZZLE_128B, dt) != HELM_OK) return HELM_ERR_CUDA;
    if (t->h16 == 2) {
        if (out_h16) xpass_h16_launch<2, true>(t, c, inverse, mapA, out, M, N2, alpha, alpha_dev, aidx, rp, astride, s, alpha_dev2, nsq_out);
        else xpass_h16_launch<2, false>(t, c, inverse, mapA, out, M, N2, alpha, alpha_dev, aidx, rp, astride, s, alpha_dev2, nsq_out);
    } else {
        if (out_h16) xpass_h16_launch<1, true>(t, c, inverse, mapA, out, M, N2, alpha, alpha_dev, aidx, rp, astride, s, alpha_dev2, nsq_out);
        else xpass_h16_launch<1, false>(t, c, inverse, mapA, out, M, N2, alpha, alpha_dev, aidx, rp, astride, s, alpha_dev2, nsq_out);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// y-pass of the 16-bit chain: 16-bit slices in, 16-bit slices out (scaled by alpha)
helm_status tc_ypass_h16(helm_ctx* c, int inverse, const void* in, void* out, float alpha, cudaStream_t s, int nb,
                         double* h16d, float gain) {
    TcState* t = (TcState*)c->tmaps;
    if (!t || !t->h16 || g_sms <= 0) return HELM_ERR_UNSUPPORTED;
    const int ny = c->ny, N2 = 2 * c->nx, nzb = c->nz * nb;
    CUtensorMap mapY;
    const cuuint64_t d[3] = {(cuuint64_t)N2, (cuuint64_t)ny, (cuuint64_t)nzb};
    const cuuint64_t st[2] = {(cuuint64_t)N2 * sizeof(uint16_t), (cuuint64_t)N2 * ny * sizeof(uint16_t)};
    const cuuint32_t box[3] = {64, 2 * BK, 1};
    const CUtensorMapDataType dt = t->h16 == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (encode(t, &mapY, 3, (void*)in, d, st, box, CU_TENSOR_MAP_SWIZZLE_128B, dt) != HELM_OK) return HELM_ERR_CUDA;
    const long wl = (long)c->wait_limit;
    const int ntiles = ((N2 + BN - 1) / BN) * ((ny + BM - 1) / BM) * nzb;
    const int pg = ntiles > g_sms ? g_sms : ntiles;
    if (t->h16 == 2)
        ypass_tc_pers_kernel<false, 2><<<pg, 192, PersY<false>::SMEM, s>>>(t->mapWyb[inverse], mapY, t->mapWyb[inverse],
                                                                          out, ny, N2, nzb, c->status_d, wl, alpha, h16d,
                                                                          gain, inverse);
    else
        ypass_tc_pers_kernel<false, 1><<<pg, 192, PersY<false>::SMEM, s>>>(t->mapWyb[inverse], mapY, t->mapWyb[inverse],
                                                                          out, ny, N2, nzb, c->status_d, wl, alpha);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

void tc_release(helm_ctx* c) {
    TcState* t = (TcState*)c->tmaps;
    if (!t) return;
    for (int i = 0; i < 2; ++i) {
        cudaFree(t->Bxb[i]);
        cudaFree(t->Wyb[i]);
    }
    for (int i = 0; i < 4; ++i) {
        cudaFree(t->Bx[i]);
        cudaFree(t->Wy[i]);
        cudaFree(t->Bxl[i]);
        cudaFree(t->Wyl[i]);
    }
    delete t;
    c->tmaps = nullptr;
}
