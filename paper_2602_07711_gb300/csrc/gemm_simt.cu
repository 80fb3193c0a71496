// Complex64 GEMM on the CUDA cores (FFMA): the eigenvector transforms of EigT steps 2 and 4
// (Sec. 4.1, Eq. EIG_SOLVER) in the plain complex64 mode.
//   C[b] = alpha * A[b] B[b],  A: M x K, B: K x N, C: M x N, row-major, batch strides sA/sB/sC.
// x-pass (right multiply by V_x^-T or V_x^T):  A = the grid viewed as (N_y N_z) x N_x rows, B = operand.
// y-pass (left multiply by V_y^-1 or V_y):      A = operand (sA = 0), B = slice l, batch = N_z.
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 complex accumulators per thread, K staged in
// shared memory 16 at a time; thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j, so shared
// memory reads are broadcasts (A) or conflict-free 128-byte rows (B) and global stores coalesce.
#include "common.cuh"

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256)
cgemm_kernel(int M, int N, int K, const float2* __restrict__ A, long lda, long sA, const float2* __restrict__ B,
             long ldb, long sB, float2* __restrict__ C, long ldc, long sC, float alpha, const double* alpha_dev, int aidx,
             int rows_per, int astride) {
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: 64 rows x 16 k -> 1024 values, 4 per thread; consecutive threads take consecutive k
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int r = e >> 4, kk = e & 15;
            const int gr = m0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[(long)gr * lda + gk] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int kk = e >> 6, cidx = e & 63;
            const int gk = k0 + kk, gc = n0 + cidx;
            Bs[kk][cidx] = (gk < K && gc < N) ? B[(long)gk * ldb + gc] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = m0 + ty + 16 * i;
        if (gr >= M) continue;
        float al = alpha;
        if (alpha_dev) al *= (float)alpha_dev[aidx + (rows_per > 0 ? (gr / rows_per) * astride : 0)];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = n0 + tx + 16 * j;
            if (gc < N) C[(long)gr * ldc + gc] = make_float2(al * acc[i][j].x, al * acc[i][j].y);
        }
    }
}
}  // namespace

void launch_cgemm_simt(int M, int N, int K, const float2* A, long lda, long sA, const float2* B, long ldb, long sB,
                       float2* C, long ldc, long sC, int batch, float alpha, const double* alpha_dev, int aidx,
                       cudaStream_t s, int rows_per, int astride) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    cgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha, alpha_dev, aidx, rows_per,
                                      astride);
}
