// batch.cu -- batched shots over windows of one global model (the
// wave_*_batched entry points of include/wave.h).
//
// Shot i runs on slot i mod C (C = concurrency): a library-owned stream and a
// slot of the caller's workspace holding the window of m and damp, the
// single-shot workspace, and for the gradient the checkpoints, the window
// gradient and a global-size accumulator.  The slot streams wait for the
// caller's stream at the start and the caller's stream waits for them at the
// end, so the call is ordered on `stream` like any other entry point.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "wave.h"

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kHead = 256;  // batch status word, then padding
constexpr int kMaxConc = 16;
constexpr int kMaxDevices = 64;

size_t al(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, 152LL * 32));
}

// w[x][y][z] = g[ox + x][oy + y][oz + z] (window of a global [.][NY][NZ] array)
__global__ void window_copy_kernel(const float *__restrict__ g, int NY, int NZ, int ox, int oy,
                                   int oz, int nx, int ny, int nz, float *__restrict__ w)
{
    const long long n = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nz);
        const long long xy = p / nz;
        const int y = (int)(xy % ny);
        const int x = (int)(xy / ny);
        w[p] = g[((long long)(ox + x) * NY + (oy + y)) * NZ + (oz + z)];
    }
}

// acc[ox + x][oy + y][oz + z] += w[x][y][z]
__global__ void window_add_kernel(const float *__restrict__ w, int nx, int ny, int nz, int NY, int NZ,
                                  int ox, int oy, int oz, float *__restrict__ acc)
{
    const long long n = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nz);
        const long long xy = p / nz;
        const int y = (int)(xy % ny);
        const int x = (int)(xy / ny);
        const long long q = ((long long)(ox + x) * NY + (oy + y)) * NZ + (oz + z);
        acc[q] = __fadd_rn(acc[q], w[p]);
    }
}

// out = a (first) or out + a
__global__ void accumulate_kernel(const float *__restrict__ a, long long n, int first,
                                  float *__restrict__ out)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        out[p] = first ? a[p] : __fadd_rn(out[p], a[p]);
}

// the most severe (most negative) status of a shot goes into the batch word
__global__ void status_merge_kernel(const int *shot_status, int *batch_status)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicMin(batch_status, *shot_status);
}

std::mutex g_pool_mu;
cudaStream_t g_pool[kMaxDevices][kMaxConc];

int pool_streams(int conc, cudaStream_t *out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WAVE_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return WAVE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int i = 0; i < conc; ++i) {
        if (g_pool[dev][i] == nullptr &&
            cudaStreamCreateWithFlags(&g_pool[dev][i], cudaStreamNonBlocking) != cudaSuccess) {
            g_pool[dev][i] = nullptr;
            return WAVE_ECUDA;
        }
        out[i] = g_pool[dev][i];
    }
    return WAVE_OK;
}

// The window of shot s as a grid of its own.
int shot_grid(const wave_grid *G, const wave_shot &s, wave_grid *out)
{
    *out = *G;
    for (int a = 0; a < 3; ++a) {
        if (s.origin[a] < 0 || s.n[a] < G->space_order + 1 ||
            (long long)s.origin[a] + s.n[a] > G->n[a])
            return WAVE_EINVAL;
        out->n[a] = s.n[a];
    }
    if (s.src.npts < 0 || s.rec.npts < 0) return WAVE_EINVAL;
    return WAVE_OK;
}

struct SlotLayout {
    size_t win = 0;    // bytes of one window field (largest shot)
    size_t ws = 0;     // single-shot workspace (largest shot)
    size_t ckpt = 0;   // checkpoints (gradient only)
    size_t glob = 0;   // global accumulator (gradient only)
    size_t slot = 0;   // bytes per slot
    size_t total = 0;  // whole batch workspace
};

int layout(const wave_grid *G, int nshots, const wave_shot *shots, int k, int conc, SlotLayout *L)
{
    if (G == nullptr || nshots < 1 || shots == nullptr || k < 0 || conc < 1 || conc > kMaxConc)
        return WAVE_EINVAL;
    const size_t glob_n = (size_t)G->n[0] * G->n[1] * G->n[2];
    if (wave_workspace_bytes(G, WAVE_OP_FWD, 0, 0, 0, nullptr) == 0) return WAVE_EINVAL;
    for (int i = 0; i < nshots; ++i) {
        wave_grid g;
        if (shot_grid(G, shots[i], &g)) return WAVE_EINVAL;
        const size_t n = (size_t)g.n[0] * g.n[1] * g.n[2];
        L->win = std::max(L->win, al(sizeof(float) * n));
        const int ns = shots[i].src.npts, nr = shots[i].rec.npts;
        size_t ws;
        if (k == 0) {
            ws = wave_workspace_bytes(&g, WAVE_OP_FWD, ns, nr, 0, nullptr);
        } else {
            ws = std::max(wave_workspace_bytes(&g, WAVE_OP_FWD, ns, 0, 0, nullptr),
                          wave_workspace_bytes(&g, WAVE_OP_GRAD, ns, nr, k, nullptr));
            L->ckpt = std::max(L->ckpt, al(wave_ckpt_bytes(&g, k)));
        }
        if (ws == 0) return WAVE_EINVAL;
        L->ws = std::max(L->ws, al(ws));
    }
    if (k > 0) L->glob = al(sizeof(float) * glob_n);
    // m and damp windows, workspace; gradient: checkpoints, window gradient, accumulator
    L->slot = 2 * L->win + L->ws + (k > 0 ? L->ckpt + L->win + L->glob : 0);
    L->total = kHead + (size_t)conc * L->slot;
    return WAVE_OK;
}

wave_tuning batch_tuning(const wave_tuning *t)
{
    wave_tuning u;
    std::memset(&u, 0, sizeof(u));
    if (t != nullptr) u = *t;
    if (u.time_tile == 0) {
        u.time_tile = 1;
        u.tile_y = 0;
        u.tile_x = 0;
        u.vec = 0;
    }
    u.flags &= ~(WAVE_TIME_SWEEPS | WAVE_AUTOTUNE_SHAPE);
    return u;
}

// Fork the slot streams off `stream`, and join them back.
struct ForkJoin {
    cudaStream_t main;
    cudaStream_t *slots;
    int n;
    int begin()
    {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return WAVE_ECUDA;
        int rc = cudaEventRecord(e, main) == cudaSuccess ? WAVE_OK : WAVE_ECUDA;
        for (int i = 0; i < n && rc == WAVE_OK; ++i)
            if (cudaStreamWaitEvent(slots[i], e, 0) != cudaSuccess) rc = WAVE_ECUDA;
        cudaEventDestroy(e);
        return rc;
    }
    int end()
    {
        int rc = WAVE_OK;
        for (int i = 0; i < n; ++i) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return WAVE_ECUDA;
            if (cudaEventRecord(e, slots[i]) != cudaSuccess || cudaStreamWaitEvent(main, e, 0) != cudaSuccess)
                rc = WAVE_ECUDA;
            cudaEventDestroy(e);
        }
        return rc;
    }
};

int conc_of(int concurrency) { return concurrency == 0 ? 4 : concurrency; }

}  // namespace

extern "C" {

size_t wave_batch_workspace_bytes(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                                  int32_t ckpt_every, int32_t concurrency)
{
    SlotLayout L;
    if (ckpt_every < 0 || layout(g, nshots, shots, ckpt_every, conc_of(concurrency), &L)) return 0;
    return L.total;
}

int32_t wave_fwd_batched(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                         const float *m, const float *damp, const float *src_traces,
                         float *rec_traces, int32_t concurrency, const wave_tuning *tuning,
                         void *ws, size_t ws_bytes, void *stream_)
{
    const int conc = conc_of(concurrency);
    SlotLayout L;
    int rc = layout(g, nshots, shots, 0, conc, &L);
    if (rc) return rc;
    if (!m || !damp || !ws || (uintptr_t)ws % kAlign) return WAVE_EINVAL;
    if (ws_bytes < L.total) return WAVE_ENOSPACE;
    long long nsrc_all = 0, nrec_all = 0;
    for (int i = 0; i < nshots; ++i) {
        nsrc_all += shots[i].src.npts;
        nrec_all += shots[i].rec.npts;
    }
    if ((nsrc_all > 0 && !src_traces) || (nrec_all > 0 && !rec_traces)) return WAVE_EINVAL;
    const int used = std::min(conc, (int)nshots);
    cudaStream_t slots[kMaxConc];
    if ((rc = pool_streams(used, slots))) return rc;
    cudaStream_t stream = (cudaStream_t)stream_;
    char *base = (char *)ws;
    int *bstatus = (int *)base;
    if (cudaMemsetAsync(bstatus, 0, sizeof(int), stream) != cudaSuccess) return WAVE_ECUDA;
    ForkJoin fj{stream, slots, used};
    if ((rc = fj.begin())) return rc;
    const wave_tuning tune = batch_tuning(tuning);
    long long so = 0, ro = 0;  // trace column offsets of the shot (in units of nt rows)
    for (int i = 0; i < nshots && rc == WAVE_OK; ++i) {
        const wave_shot &s = shots[i];
        wave_grid gw;
        shot_grid(g, s, &gw);
        const int k = i % used;
        cudaStream_t st = slots[k];
        char *slot = base + kHead + (size_t)k * L.slot;
        float *mw = (float *)slot, *dw = (float *)(slot + L.win);
        void *sws = slot + 2 * L.win;
        const long long n = (long long)gw.n[0] * gw.n[1] * gw.n[2];
        window_copy_kernel<<<grid_for(n), 256, 0, st>>>(m, g->n[1], g->n[2], s.origin[0], s.origin[1],
                                                        s.origin[2], gw.n[0], gw.n[1], gw.n[2], mw);
        window_copy_kernel<<<grid_for(n), 256, 0, st>>>(damp, g->n[1], g->n[2], s.origin[0], s.origin[1],
                                                        s.origin[2], gw.n[0], gw.n[1], gw.n[2], dw);
        if (cudaGetLastError() != cudaSuccess) rc = WAVE_ECUDA;
        if (rc == WAVE_OK)
            rc = wave_fwd(&gw, mw, dw, &s.src, s.src.npts ? src_traces + so * g->nt : nullptr, &s.rec,
                          s.rec.npts ? rec_traces + ro * g->nt : nullptr, nullptr, nullptr, 0, &tune, sws,
                          L.ws, st);
        if (rc == WAVE_OK) {
            status_merge_kernel<<<1, 32, 0, st>>>((const int *)sws, bstatus);
            if (cudaGetLastError() != cudaSuccess) rc = WAVE_ECUDA;
        }
        so += s.src.npts;
        ro += s.rec.npts;
    }
    const int rj = fj.end();
    return rc ? rc : rj;
}

int32_t wave_grad_batched(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                          const float *m, const float *damp, const float *src_traces,
                          const float *rec_resid, int32_t ckpt_every, float *grad,
                          int32_t concurrency, const wave_tuning *tuning, void *ws,
                          size_t ws_bytes, void *stream_)
{
    const int conc = conc_of(concurrency);
    if (ckpt_every < 1) return WAVE_EINVAL;
    SlotLayout L;
    int rc = layout(g, nshots, shots, ckpt_every, conc, &L);
    if (rc) return rc;
    if (!m || !damp || !grad || !ws || (uintptr_t)ws % kAlign) return WAVE_EINVAL;
    if (ws_bytes < L.total) return WAVE_ENOSPACE;
    long long nsrc_all = 0, nrec_all = 0;
    for (int i = 0; i < nshots; ++i) {
        nsrc_all += shots[i].src.npts;
        nrec_all += shots[i].rec.npts;
    }
    if ((nsrc_all > 0 && !src_traces) || (nrec_all > 0 && !rec_resid)) return WAVE_EINVAL;
    const int used = std::min(conc, (int)nshots);
    cudaStream_t slots[kMaxConc];
    if ((rc = pool_streams(used, slots))) return rc;
    cudaStream_t stream = (cudaStream_t)stream_;
    char *base = (char *)ws;
    int *bstatus = (int *)base;
    const long long nglob = (long long)g->n[0] * g->n[1] * g->n[2];
    if (cudaMemsetAsync(bstatus, 0, sizeof(int), stream) != cudaSuccess) return WAVE_ECUDA;
    ForkJoin fj{stream, slots, used};
    if ((rc = fj.begin())) return rc;
    const wave_tuning tune = batch_tuning(tuning);
    auto slot_ptr = [&](int k) { return base + kHead + (size_t)k * L.slot; };
    for (int k = 0; k < used && rc == WAVE_OK; ++k) {
        float *acc = (float *)(slot_ptr(k) + 2 * L.win + L.ws + L.ckpt + L.win);
        if (cudaMemsetAsync(acc, 0, sizeof(float) * nglob, slots[k]) != cudaSuccess) rc = WAVE_ECUDA;
    }
    long long so = 0, ro = 0;
    for (int i = 0; i < nshots && rc == WAVE_OK; ++i) {
        const wave_shot &s = shots[i];
        wave_grid gw;
        shot_grid(g, s, &gw);
        const int k = i % used;
        cudaStream_t st = slots[k];
        char *slot = slot_ptr(k);
        float *mw = (float *)slot, *dw = (float *)(slot + L.win);
        void *sws = slot + 2 * L.win;
        float *ck = (float *)(slot + 2 * L.win + L.ws);
        float *gwin = (float *)(slot + 2 * L.win + L.ws + L.ckpt);
        float *acc = (float *)(slot + 2 * L.win + L.ws + L.ckpt + L.win);
        const long long n = (long long)gw.n[0] * gw.n[1] * gw.n[2];
        window_copy_kernel<<<grid_for(n), 256, 0, st>>>(m, g->n[1], g->n[2], s.origin[0], s.origin[1],
                                                        s.origin[2], gw.n[0], gw.n[1], gw.n[2], mw);
        window_copy_kernel<<<grid_for(n), 256, 0, st>>>(damp, g->n[1], g->n[2], s.origin[0], s.origin[1],
                                                        s.origin[2], gw.n[0], gw.n[1], gw.n[2], dw);
        if (cudaGetLastError() != cudaSuccess) rc = WAVE_ECUDA;
        const float *q = s.src.npts ? src_traces + so * g->nt : nullptr;
        // forward with checkpoints (no receivers needed), then the gradient
        if (rc == WAVE_OK)
            rc = wave_fwd(&gw, mw, dw, &s.src, q, nullptr, nullptr, nullptr, ck, ckpt_every, &tune, sws,
                          L.ws, st);
        if (rc == WAVE_OK) {
            status_merge_kernel<<<1, 32, 0, st>>>((const int *)sws, bstatus);
            rc = wave_grad(&gw, mw, dw, &s.src, q, &s.rec, s.rec.npts ? rec_resid + ro * g->nt : nullptr,
                           ck, ckpt_every, gwin, &tune, sws, L.ws, st);
        }
        if (rc == WAVE_OK) {
            status_merge_kernel<<<1, 32, 0, st>>>((const int *)sws, bstatus);
            window_add_kernel<<<grid_for(n), 256, 0, st>>>(gwin, gw.n[0], gw.n[1], gw.n[2], g->n[1],
                                                           g->n[2], s.origin[0], s.origin[1], s.origin[2],
                                                           acc);
            if (cudaGetLastError() != cudaSuccess) rc = WAVE_ECUDA;
        }
        so += s.src.npts;
        ro += s.rec.npts;
    }
    const int rj = fj.end();
    if (rc) return rc;
    if (rj) return rj;
    // slots summed in slot order on the caller's stream
    for (int k = 0; k < used; ++k) {
        const float *acc = (const float *)(slot_ptr(k) + 2 * L.win + L.ws + L.ckpt + L.win);
        accumulate_kernel<<<grid_for(nglob), 256, 0, stream>>>(acc, nglob, k == 0, grad);
    }
    return cudaGetLastError() == cudaSuccess ? WAVE_OK : WAVE_ECUDA;
}

}  // extern "C"
