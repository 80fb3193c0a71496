// helm_residual_noalloc: the true residual r = b - A x (double-float arithmetic) for callers that must
// not allocate device memory while they run, e.g. an application whose memory pool owns the whole device
// after warm-up, or a runtime that forbids cudaMalloc/cudaFree (both synchronise the device) between its
// steps.  The helm_residual entry point keeps its double-float copies of b and x and its per-CTA partial
// sums in workspace it allocates on first use; this variant keeps them in one file-scope device array
// instead.  Like helm_residual it copies the two norms to host memory and synchronises the stream.
#include "common.cuh"
#include "dfloat.cuh"

int residual_ctas(const helm_ctx* c);

namespace {
constexpr size_t NA_MAX_POINTS_ = (size_t)1 << 21;
constexpr size_t NA_SCRATCH_BYTES = 2 * NA_MAX_POINTS_ * 16 + (size_t)2 * 65536 * 8 + 256;
}  // namespace

// The scratch: double-float b, double-float x, residual partials, two result words (65 MiB + 256 B).
// Every GPU that loads the library holds it until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_scratch[NA_SCRATCH_BYTES];

namespace {

constexpr size_t NA_MAX_POINTS = (size_t)1 << 21;   // 2,097,152 points (128^3)
constexpr int NA_MAX_CTAS = 65536;                  // residual CTAs (one partial pair each)
constexpr size_t NA_DF_BYTES = NA_MAX_POINTS * sizeof(float4);
constexpr size_t NA_PART_BYTES = (size_t)2 * NA_MAX_CTAS * sizeof(double);
static_assert(2 * NA_DF_BYTES + NA_PART_BYTES + 256 == NA_SCRATCH_BYTES, "scratch layout");

// Host side: the device address of g_scratch per device, looked up once per device with that device
// current.  (The name g_scratch in host code is only a host-side stand-in, not a device address.)
constexpr int NA_MAX_DEVICES = 64;
void* g_scratch_dev[NA_MAX_DEVICES] = {nullptr};

__global__ void na_to_df_kernel(const double2* __restrict__ a, float4* __restrict__ b, size_t n) {
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        b[id] = split4_bits(a[id]);
    }
}

// out[0] = sqrt(sum part[2i]), out[1] = max part[2i+1]
__global__ void na_reduce_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double rs[32], rm[32];
    double s = 0, m = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { s += part[2 * i]; m = fmax(m, part[2 * i + 1]); }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = s; rm[threadIdx.x >> 5] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0, tm = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ts += rs[w]; tm = fmax(tm, rm[w]); }
        out[0] = sqrt(ts);
        out[1] = tm;
    }
}

bool na_dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" helm_status helm_residual_noalloc(helm_ctx* c, const void* b, const void* x, void* r, double* nrm2,
                                             double* nrmi, void* stream) {
    if (!c || !b || !x || !r) return HELM_ERR_ARG;
    if (c->npts > NA_MAX_POINTS) return HELM_ERR_ARG;
    const int nres = residual_ctas(c);
    if (nres > NA_MAX_CTAS) return HELM_ERR_ARG;
    if (!na_dev_ptr(b) || !na_dev_ptr(x) || !na_dev_ptr(r)) return HELM_ERR_ARG;
    int dev = 0;
    HELM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return HELM_ERR_ARG;
    if (!g_scratch_dev[dev]) {
        // first call on this device: look up the array's device address (the device is current)
        void* p = nullptr;
        HELM_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
        g_scratch_dev[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_scratch_dev[dev];
    float4* Fdf = (float4*)base;
    float4* xdf = (float4*)(base + NA_DF_BYTES);
    double* part = (double*)(base + 2 * NA_DF_BYTES);
    double* res = (double*)(base + 2 * NA_DF_BYTES + NA_PART_BYTES);
    cudaStream_t s = (cudaStream_t)stream;
    // every region the kernels read is fully written by this call before it is read
    na_to_df_kernel<<<512, 256, 0, s>>>((const double2*)b, Fdf, c->npts);
    na_to_df_kernel<<<512, 256, 0, s>>>((const double2*)x, xdf, c->npts);
    HELM_CUDA_TRY(cudaGetLastError());
    helm_status st = launch_residual(c, xdf, Fdf, (float2*)r, part, s);
    if (st != HELM_OK) return st;
    na_reduce_kernel<<<1, 256, 0, s>>>(part, nres, res);
    HELM_CUDA_TRY(cudaGetLastError());
    double h[2] = {0.0, 0.0};
    HELM_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (nrm2) *nrm2 = h[0];
    if (nrmi) *nrmi = h[1];
    return HELM_OK;
}
