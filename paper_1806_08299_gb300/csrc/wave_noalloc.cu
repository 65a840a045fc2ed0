// wave_noalloc.cu -- wave_fwd_noalloc: forward modelling whose workspace is a
// static device array of this file instead of caller-provided memory.
//
// The array is reserved when CUDA loads this file's module on a device.  Its
// address is taken once per device, with that device current, through
// cudaGetSymbolAddress, and the ordinary forward driver then carves the
// workspace out of it exactly as it carves a caller's buffer.  Nothing here
// allocates or frees device memory.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "wave.h"

static __device__ __align__(256) unsigned char g_noalloc_ws[WAVE_NOALLOC_MAX_BYTES];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];  // address of g_noalloc_ws per device, once set up

// Address of the array on the current device; the first call on a device
// does the set-up.
int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WAVE_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return WAVE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || p == nullptr) return WAVE_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
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
    if (status != nullptr) *status = wave_status(ws, stream);
    return WAVE_OK;
}
