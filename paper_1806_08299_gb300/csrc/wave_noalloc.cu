// wave_noalloc.cu -- wave_fwd_noalloc: forward modelling whose workspace is a
// static device array of this file instead of caller-provided memory.
//
// The array is reserved when CUDA loads this file's module in a context.  Its
// address is taken, with that context current, through cudaGetSymbolAddress
// and kept per context (by the driver's unique context id, so a context that
// replaces a destroyed one, e.g. after cudaDeviceReset, is set up again).
// The ordinary forward driver then carves the workspace out of it exactly as
// it carves a caller's buffer.  Nothing here allocates or frees device memory.
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "wave.h"

static __device__ __align__(256) unsigned char g_noalloc_ws[WAVE_NOALLOC_MAX_BYTES];

namespace {

constexpr int kMaxDevices = 64;

struct NoallocSlot {
    unsigned long long ctx_id = 0;  // driver context id the address belongs to (0: none yet)
    void *ptr = nullptr;
};

std::mutex g_noalloc_mu;
NoallocSlot g_noalloc[kMaxDevices];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 when there is none);
// the two driver calls come through the runtime's entry-point query, so the
// library needs no link to libcuda.
int current_ctx_id(unsigned long long *id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (get_current == nullptr || get_id == nullptr) {  // called with g_noalloc_mu held
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) !=
                cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || f0 == nullptr ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || f1 == nullptr)
            return WAVE_ECUDA;
        get_current = (PfnCtxGetCurrent)f0;
        get_id = (PfnCtxGetId)f1;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return WAVE_ECUDA;
    *id = 0;
    if (ctx != nullptr && get_id(ctx, id) != CUDA_SUCCESS) return WAVE_ECUDA;
    return WAVE_OK;
}

// Address of the array in the current context of the current device; the
// first call in a context does the set-up.
int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WAVE_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return WAVE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long id = 0;
    int rc = current_ctx_id(&id);
    if (rc != WAVE_OK) return rc;
    NoallocSlot &s = g_noalloc[dev];
    if (id == 0 || id != s.ctx_id || s.ptr == nullptr) {
        // set-up: the runtime makes the device's context current if none is
        // (the id is then read again), and the address is that context's
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || p == nullptr) return WAVE_ECUDA;
        rc = current_ctx_id(&id);
        if (rc != WAVE_OK) return rc;
        if (id == 0) return WAVE_ECUDA;
        s.ctx_id = id;
        s.ptr = p;
    }
    *out = s.ptr;
    return WAVE_OK;
}

}  // namespace

extern "C" int32_t wave_fwd_noalloc(const wave_grid *g, const float *m, const float *damp,
                                    const wave_points *src, const float *src_traces,
                                    const wave_points *rec, float *rec_traces, float *u_last,
                                    const wave_tuning *tuning, void *stream, int32_t *status)
{
    const int32_t nsrc = src ? src->npts : 0, nrec = rec ? rec->npts : 0;
    if (nsrc < 0 || nrec < 0) return WAVE_EINVAL;
    const size_t need = wave_workspace_bytes(g, WAVE_OP_FWD, nsrc, nrec, 0, tuning);
    if (need == 0) return WAVE_EINVAL;
    if (need > (size_t)WAVE_NOALLOC_MAX_BYTES) return WAVE_ENOSPACE;
    void *ws = nullptr;
    int32_t rc = noalloc_scratch(&ws);
    if (rc != WAVE_OK) return rc;
    // The forward driver clears, in stream order before its first kernel, the
    // status words and the four wavefield levels; every other part of the
    // workspace is written before it is read, so no state carries over from a
    // previous call.
    rc = wave_fwd(g, m, damp, src, src_traces, rec, rec_traces, u_last, nullptr, 0, tuning, ws,
                  (size_t)WAVE_NOALLOC_MAX_BYTES, stream);
    if (rc != WAVE_OK) return rc;
    if (status != nullptr) {
        // a failure of the synchronising read is this call's return code;
        // *status only ever receives the device status word
        if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return WAVE_ECUDA;
        int32_t word = 0;
        if (cudaMemcpy(&word, ws, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return WAVE_ECUDA;
        *status = word;
    }
    return WAVE_OK;
}
