// Per-kernel CUDA-event timing (helm_profile / helm_profile_read): pairs of events recorded on the
// launch stream around each launch, accumulated per kernel class when read back.
#include "common.cuh"

void prof_begin(helm_ctx* c, cudaStream_t s, int cls) {
    Prof* p = c->prof;
    if (!p) return;
    p->open = 0;
    if (!p->enabled || !((p->mask >> cls) & 1u)) return;
    if (p->used + 2 > Prof::CAP) prof_flush(c);
    p->cls[p->used / 2] = cls;
    cudaEventRecord(p->ev[p->used], s);
    p->used += 1;
    p->open = 1;
}

void prof_end(helm_ctx* c, cudaStream_t s) {
    Prof* p = c->prof;
    if (!p || !p->enabled || !p->open) return;
    cudaEventRecord(p->ev[p->used], s);
    p->used += 1;
    p->open = 0;
}

void prof_flush(helm_ctx* c) {
    Prof* p = c->prof;
    if (!p) return;
    for (int i = 0; i + 1 < p->used; i += 2) {
        cudaEventSynchronize(p->ev[i + 1]);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess) {
            p->ms[p->cls[i / 2]] += ms;
            p->launches[p->cls[i / 2]] += 1;
        }
    }
    cudaGetLastError();
    p->used = 0;
}

extern "C" helm_status helm_profile(helm_ctx* c, int enable) {
    if (!c) return HELM_ERR_ARG;
    if (!c->prof) {
        c->prof = new Prof();
        for (int i = 0; i < Prof::CAP; ++i) {
            if (cudaEventCreate(&c->prof->ev[i]) != cudaSuccess) { cudaGetLastError(); return HELM_ERR_CUDA; }
            c->prof->created = i + 1;
        }
    }
    c->prof->enabled = enable ? 1 : 0;
    c->prof->mask = ~0u;
    return HELM_OK;
}

extern "C" helm_status helm_profile_classes(helm_ctx* c, unsigned mask) {
    helm_status st = helm_profile(c, mask != 0u);
    if (st == HELM_OK) c->prof->mask = mask;
    return st;
}

extern "C" helm_status helm_profile_read(helm_ctx* c, double* ms, long long* launches, int n, int reset) {
    if (!c || !c->prof) return HELM_ERR_ARG;
    prof_flush(c);
    for (int i = 0; i < n && i < PROF_NCLASS; ++i) {
        if (ms) ms[i] = c->prof->ms[i];
        if (launches) launches[i] = c->prof->launches[i];
    }
    if (reset)
        for (int i = 0; i < PROF_NCLASS; ++i) { c->prof->ms[i] = 0; c->prof->launches[i] = 0; }
    return HELM_OK;
}

void prof_release(helm_ctx* c) {
    if (!c->prof) return;
    for (int i = 0; i < c->prof->created; ++i) cudaEventDestroy(c->prof->ev[i]);
    delete c->prof;
    c->prof = nullptr;
}
