// Tensor-core (tcgen05) eigenvector transforms: not built yet.
#include "common.cuh"

helm_status tc_prepare(helm_ctx* c, cudaStream_t s) { (void)c; (void)s; return HELM_ERR_UNSUPPORTED; }
helm_status tc_xpass(helm_ctx* c, int inverse, const float2* in, float2* out, float alpha, const double* alpha_dev,
                     int aidx, cudaStream_t s) {
    (void)c; (void)inverse; (void)in; (void)out; (void)alpha; (void)alpha_dev; (void)aidx; (void)s;
    return HELM_ERR_UNSUPPORTED;
}
helm_status tc_ypass(helm_ctx* c, int inverse, const float2* in, float2* out, cudaStream_t s) {
    (void)c; (void)inverse; (void)in; (void)out; (void)s;
    return HELM_ERR_UNSUPPORTED;
}
void tc_release(helm_ctx* c) { (void)c; }
