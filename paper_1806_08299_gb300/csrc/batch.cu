// batch.cu -- batched shots over windows of one global model (the
// wave_*_batched entry points of include/wave.h).
//
// Shots run in groups of C (C = concurrency).  Shot i uses slot i mod C of
// the caller's workspace: the window of m and damp, the single-shot
// workspace and, for the gradient, the checkpoints and the window gradient.
//
//  * Lockstep (the default plan, or a plan of a batched kernel): the shots
//    of a group advance together, one launch of a batched kernel per time
//    step (or per T steps of the stage-specialised one) for all of them, on
//    the caller's stream (host runtime, wave_api.cu).
//  * Otherwise each shot runs wave_fwd / wave_grad on its slot's
//    library-owned stream; the slot streams wait for the caller's stream at
//    the start and the caller's stream waits for them at the end.
//
// Either way the window gradients are added into the global gradient in shot
// order, so both give the same, deterministic result.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "wave.h"
#include "wave_internal.h"

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
    size_t table = 0;  // per-shot launch arguments of a lockstep group
    size_t slot = 0;   // bytes per slot
    size_t total = 0;  // whole batch workspace
};

int layout(const wave_grid *G, int nshots, const wave_shot *shots, int k, int conc, SlotLayout *L)
{
    if (G == nullptr || nshots < 1 || shots == nullptr || k < 0 || conc < 1 || conc > kMaxConc)
        return WAVE_EINVAL;
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
    for (int g0 = 0; g0 < nshots; g0 += conc)
        L->table = std::max(L->table, al(wt::lockstep_table_bytes(G, std::min(conc, nshots - g0), shots + g0, k)));
    // m and damp windows, workspace; gradient: checkpoints and the window gradient
    L->slot = 2 * L->win + L->ws + (k > 0 ? L->ckpt + L->win : 0);
    L->total = kHead + L->table + (size_t)conc * L->slot;
    return WAVE_OK;
}

wave_tuning batch_tuning(const wave_tuning *t)
{
    wave_tuning u;
    std::memset(&u, 0, sizeof(u));
    if (t != nullptr) u = *t;
    if (u.time_tile == 0) {  // the lockstep engine times its forward kernel
        u.tile_y = 0;
        u.tile_x = 0;
        u.vec = 0;
        u.tile_z = 0;
        u.rows = 0;
        u.kernel = 0;
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

// Everything one batched call needs to address its shots.
struct Batch {
    const wave_grid *g;
    int nshots;
    const wave_shot *shots;
    SlotLayout L;
    char *base;
    std::vector<long long> so, ro;  // trace column offset of each shot (units of nt rows)

    char *slot(int k) const { return base + kHead + L.table + (size_t)k * L.slot; }
    void *table() const { return base + kHead; }
    int *status() const { return (int *)base; }
    wt::ShotSlot shot_slot(int i, int k, const float *src_traces, float *rec_traces, const float *resid) const
    {
        char *sl = slot(k);
        wt::ShotSlot x;
        x.shot = &shots[i];
        x.mw = (float *)sl;
        x.dw = (float *)(sl + L.win);
        x.ws = sl + 2 * L.win;
        x.ws_bytes = L.ws;
        x.ckpt = L.ckpt ? (float *)(sl + 2 * L.win + L.ws) : nullptr;
        x.gwin = L.ckpt ? (float *)(sl + 2 * L.win + L.ws + L.ckpt) : nullptr;
        x.q = shots[i].src.npts ? src_traces + so[i] * g->nt : nullptr;
        x.rec_out = (rec_traces && shots[i].rec.npts) ? rec_traces + ro[i] * g->nt : nullptr;
        x.resid = (resid && shots[i].rec.npts) ? resid + ro[i] * g->nt : nullptr;
        return x;
    }
};

int batch_setup(const wave_grid *g, int nshots, const wave_shot *shots, int k, int conc, void *ws,
                size_t ws_bytes, Batch *b)
{
    b->g = g;
    b->nshots = nshots;
    b->shots = shots;
    int rc = layout(g, nshots, shots, k, conc, &b->L);
    if (rc) return rc;
    if (ws == nullptr || (uintptr_t)ws % kAlign) return WAVE_EINVAL;
    if (ws_bytes < b->L.total) return WAVE_ENOSPACE;
    b->base = (char *)ws;
    b->so.assign(nshots, 0);
    b->ro.assign(nshots, 0);
    for (int i = 1; i < nshots; ++i) {
        b->so[i] = b->so[i - 1] + shots[i - 1].src.npts;
        b->ro[i] = b->ro[i - 1] + shots[i - 1].rec.npts;
    }
    return WAVE_OK;
}

int copy_windows(const Batch &b, const wt::ShotSlot &x, const float *m, const float *damp, cudaStream_t st)
{
    const wave_shot &s = *x.shot;
    const long long n = (long long)s.n[0] * s.n[1] * s.n[2];
    window_copy_kernel<<<grid_for(n), 256, 0, st>>>(m, b.g->n[1], b.g->n[2], s.origin[0], s.origin[1],
                                                    s.origin[2], s.n[0], s.n[1], s.n[2], x.mw);
    window_copy_kernel<<<grid_for(n), 256, 0, st>>>(damp, b.g->n[1], b.g->n[2], s.origin[0], s.origin[1],
                                                    s.origin[2], s.n[0], s.n[1], s.n[2], x.dw);
    return cudaGetLastError() == cudaSuccess ? WAVE_OK : WAVE_ECUDA;
}

int add_window(const Batch &b, const wt::ShotSlot &x, float *grad, cudaStream_t st)
{
    const wave_shot &s = *x.shot;
    const long long n = (long long)s.n[0] * s.n[1] * s.n[2];
    window_add_kernel<<<grid_for(n), 256, 0, st>>>(x.gwin, s.n[0], s.n[1], s.n[2], b.g->n[1], b.g->n[2],
                                                   s.origin[0], s.origin[1], s.origin[2], grad);
    return cudaGetLastError() == cudaSuccess ? WAVE_OK : WAVE_ECUDA;
}

int merge_status(const Batch &b, const wt::ShotSlot &x, cudaStream_t st)
{
    status_merge_kernel<<<1, 32, 0, st>>>((const int *)x.ws, b.status());
    return cudaGetLastError() == cudaSuccess ? WAVE_OK : WAVE_ECUDA;
}

// Both entry points: lockstep groups on `stream` when the plan has a batched
// kernel, else shots on slot streams.  k = 0: forward; k >= 1: gradient.
int run_batch(const wave_grid *g, int nshots, const wave_shot *shots, const float *m, const float *damp,
              const float *src_traces, float *rec_traces, const float *rec_resid, int k, float *grad,
              int concurrency, const wave_tuning *tuning, void *ws, size_t ws_bytes, cudaStream_t stream)
{
    const int conc = conc_of(concurrency);
    Batch b;
    int rc = batch_setup(g, nshots, shots, k, conc, ws, ws_bytes, &b);
    if (rc) return rc;
    if (!m || !damp || (k > 0 && !grad)) return WAVE_EINVAL;
    long long nsrc_all = 0, nrec_all = 0;
    for (int i = 0; i < nshots; ++i) {
        nsrc_all += shots[i].src.npts;
        nrec_all += shots[i].rec.npts;
    }
    if (nsrc_all > 0 && !src_traces) return WAVE_EINVAL;
    if (nrec_all > 0 && ((k == 0 && !rec_traces) || (k > 0 && !rec_resid))) return WAVE_EINVAL;
    const wave_tuning tune = batch_tuning(tuning);
    if (cudaMemsetAsync(b.status(), 0, sizeof(int), stream) != cudaSuccess) return WAVE_ECUDA;
    if (k > 0 && cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)g->n[0] * g->n[1] * g->n[2], stream) !=
                     cudaSuccess)
        return WAVE_ECUDA;
    const int used = std::min(conc, nshots);

    if (wt::lockstep_supported(g, &tune, k)) {
        for (int g0 = 0; g0 < nshots && rc == WAVE_OK; g0 += used) {
            const int n = std::min(used, nshots - g0);
            std::vector<wt::ShotSlot> sl(n);
            for (int i = 0; i < n && rc == WAVE_OK; ++i) {
                sl[i] = b.shot_slot(g0 + i, i, src_traces, rec_traces, rec_resid);
                rc = copy_windows(b, sl[i], m, damp, stream);
            }
            if (rc == WAVE_OK) rc = wt::lockstep_group(g, n, sl.data(), k, &tune, b.table(), b.L.table, stream);
            for (int i = 0; i < n && rc == WAVE_OK; ++i) {
                rc = merge_status(b, sl[i], stream);
                if (rc == WAVE_OK && k > 0) rc = add_window(b, sl[i], grad, stream);  // shot order
            }
        }
        return rc;
    }

    cudaStream_t slots[kMaxConc];
    if ((rc = pool_streams(used, slots))) return rc;
    ForkJoin fj{stream, slots, used};
    if ((rc = fj.begin())) return rc;
    // window gradients go into grad in shot order: shot i's add waits for shot i-1's
    cudaEvent_t added = nullptr;
    for (int i = 0; i < nshots && rc == WAVE_OK; ++i) {
        const int kslot = i % used;
        cudaStream_t st = slots[kslot];
        const wt::ShotSlot x = b.shot_slot(i, kslot, src_traces, rec_traces, rec_resid);
        wave_grid gw;
        shot_grid(g, shots[i], &gw);
        rc = copy_windows(b, x, m, damp, st);
        if (rc == WAVE_OK && k == 0)
            rc = wave_fwd(&gw, x.mw, x.dw, &shots[i].src, x.q, &shots[i].rec, x.rec_out, nullptr, nullptr, 0,
                          &tune, x.ws, x.ws_bytes, st);
        if (rc == WAVE_OK && k > 0) {
            // forward with checkpoints (no receivers needed), then the gradient
            rc = wave_fwd(&gw, x.mw, x.dw, &shots[i].src, x.q, nullptr, nullptr, nullptr, x.ckpt, k, &tune, x.ws,
                          x.ws_bytes, st);
            if (rc == WAVE_OK) rc = merge_status(b, x, st);
            if (rc == WAVE_OK)
                rc = wave_grad(&gw, x.mw, x.dw, &shots[i].src, x.q, &shots[i].rec, x.resid, x.ckpt, k, x.gwin,
                               &tune, x.ws, x.ws_bytes, st);
        }
        if (rc == WAVE_OK) rc = merge_status(b, x, st);
        if (rc == WAVE_OK && k > 0) {
            if (added != nullptr && cudaStreamWaitEvent(st, added, 0) != cudaSuccess) rc = WAVE_ECUDA;
            if (rc == WAVE_OK) rc = add_window(b, x, grad, st);
            if (added != nullptr) cudaEventDestroy(added);
            added = nullptr;
            if (rc == WAVE_OK && (cudaEventCreateWithFlags(&added, cudaEventDisableTiming) != cudaSuccess ||
                                  cudaEventRecord(added, st) != cudaSuccess))
                rc = WAVE_ECUDA;
        }
    }
    if (added != nullptr) cudaEventDestroy(added);
    const int rj = fj.end();
    return rc ? rc : rj;
}

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
                         void *ws, size_t ws_bytes, void *stream)
{
    try {
        return run_batch(g, nshots, shots, m, damp, src_traces, rec_traces, nullptr, 0, nullptr, concurrency,
                         tuning, ws, ws_bytes, (cudaStream_t)stream);
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_describe_batch_plan(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                                 int32_t ckpt_every, int32_t concurrency, const wave_tuning *tuning,
                                 int32_t *out)
{
    SlotLayout L;
    if (out == nullptr || ckpt_every < 0 || layout(g, nshots, shots, ckpt_every, conc_of(concurrency), &L))
        return WAVE_EINVAL;
    try {
        const wave_tuning tune = batch_tuning(tuning);
        return wt::lockstep_describe(g, std::min(conc_of(concurrency), (int)nshots), shots, ckpt_every, &tune,
                                     out);
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_grad_batched(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                          const float *m, const float *damp, const float *src_traces,
                          const float *rec_resid, int32_t ckpt_every, float *grad,
                          int32_t concurrency, const wave_tuning *tuning, void *ws,
                          size_t ws_bytes, void *stream)
{
    if (ckpt_every < 1) return WAVE_EINVAL;
    try {
        return run_batch(g, nshots, shots, m, damp, src_traces, nullptr, rec_resid, ckpt_every, grad,
                         concurrency, tuning, ws, ws_bytes, (cudaStream_t)stream);
    } catch (...) {
        return WAVE_EINVAL;
    }
}

}  // extern "C"
