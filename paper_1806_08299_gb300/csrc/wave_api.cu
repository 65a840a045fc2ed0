// wave_api.cu -- host runtime behind the C ABI in include/wave.h.
//
// Argument checks, stencil coefficients, sparse point tables, workspace
// layout, launch sequencing (time tiles, checkpoints, recompute segments),
// the autotuner and the device status word.  All device memory comes from
// the caller's workspace; nothing here allocates on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "wave.h"
#include "wave_internal.h"

namespace {

using wt::PointTable;
using wt::Stencil;
using wt::SweepArgs;
using wt::SweepVariant;

constexpr size_t kAlign = 256;
constexpr int kStatusWords = 64;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

#define CK(call)                                         \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return WAVE_ECUDA;        \
    } while (0)

struct Dims {
    int nx, ny, nz, nzp;
    long long npad;  // nx * ny * nzp
    long long n;     // nx * ny * nz
};

int check_grid(const wave_grid *g, Dims *d)
{
    if (g == nullptr) return WAVE_EINVAL;
    const int so = g->space_order;
    if (so < 2 || so > 16 || so % 2) return WAVE_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < so + 1 || g->n[a] > (1 << 20)) return WAVE_EINVAL;
        if (!(g->h[a] > 0.f) || !std::isfinite(g->h[a])) return WAVE_EINVAL;
    }
    if (!(g->dt > 0.f) || !std::isfinite(g->dt) || g->nt < 1) return WAVE_EINVAL;
    d->nx = g->n[0];
    d->ny = g->n[1];
    d->nz = g->n[2];
    d->nzp = (g->n[2] + 7) / 8 * 8;  // rows of whole 8-point (32-byte) groups
    d->npad = (long long)d->nx * d->ny * d->nzp;
    d->n = (long long)d->nx * d->ny * d->nz;
    if (d->npad > (1LL << 36)) return WAVE_EINVAL;
    if ((long long)d->ny * d->nzp >= (1LL << 31)) return WAVE_EINVAL;  // one x-plane < 2^31 points
    return WAVE_OK;
}

// TMA descriptor of a padded [nx][ny][nzp] float32 array with a (bz, by, 1)
// box; out-of-bounds elements read as zero.  cuTensorMapEncodeTiled comes from
// the driver through the runtime's entry-point query (no link to libcuda).
int encode_map(CUtensorMap *map, const float *base, const Dims &d, int bz, int by)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (fn == nullptr) {
            cudaDriverEntryPointQueryResult q;
            void *f = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                                 &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess || f == nullptr)
                return WAVE_ECUDA;
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
        }
    }
    const cuuint64_t dims[3] = {(cuuint64_t)d.nzp, (cuuint64_t)d.ny, (cuuint64_t)d.nx};
    const cuuint64_t strides[2] = {(cuuint64_t)d.nzp * 4, (cuuint64_t)d.ny * d.nzp * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bz, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? WAVE_OK : WAVE_ECUDA;
}

// A second-difference store [rows][nx][ny][nzp] as one tensor of rows * nx
// planes (row r, plane x = plane r * nx + x), box bz x by x 1.
int encode_rows_map(CUtensorMap *map, const float *base, const Dims &d, long long rows, int bz, int by)
{
    if (rows < 1 || (long long)d.nx * rows > 0x7fffffffLL) return WAVE_EINVAL;
    Dims dr = d;
    dr.nx = (int)(d.nx * rows);
    return encode_map(map, base, dr, bz, by);
}

// c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!) by the product form
// (r!)^2/((r-k)!(r+k)!) = prod_{j=1..k} (r-k+j)/(r+j), exact to double rounding.
void fd_coeffs(int so, double *c)
{
    const int r = so / 2;
    double sum = 0.0;
    for (int k = 1; k <= r; ++k) {
        double ratio = 1.0;
        for (int j = 1; j <= k; ++j) ratio *= (double)(r - k + j) / (double)(r + j);
        const double ck = ((k % 2) ? 2.0 : -2.0) * ratio / ((double)k * k);
        c[k] = ck;
        sum += ck;
    }
    c[0] = -2.0 * sum;
}

double symbol_at_pi(int so)
{
    double c[wt::kMaxR + 1];
    fd_coeffs(so, c);
    double s = c[0];
    for (int k = 1; k <= so / 2; ++k) s += 2.0 * ((k % 2) ? -c[k] : c[k]);
    return std::fabs(s);
}

Stencil make_stencil(const wave_grid *g)
{
    double c[wt::kMaxR + 1];
    fd_coeffs(g->space_order, c);
    Stencil st;
    std::memset(&st, 0, sizeof(st));
    const double ih[3] = {1.0 / ((double)g->h[0] * g->h[0]), 1.0 / ((double)g->h[1] * g->h[1]),
                          1.0 / ((double)g->h[2] * g->h[2])};
    auto both = [](double v) { return make_float2((float)v, (float)v); };
    st.cc = both((c[0] * ih[0] + c[0] * ih[1]) + c[0] * ih[2]);
    for (int k = 1; k <= g->space_order / 2; ++k) {
        st.cx[k] = both(c[k] * ih[0]);
        st.cy[k] = both(c[k] * ih[1]);
        st.cz[k] = both(c[k] * ih[2]);
    }
    return st;
}

// ---------------------------------------------------------------------------
// Sparse point tables
// ---------------------------------------------------------------------------

struct HostTable {
    std::vector<int> plane_start;  // nx + 1
    std::vector<int4> pts;         // sorted (x, y, z) -> (y, z, begin, end)
    std::vector<int> item;
    std::vector<float> w;          // injection weights per item
    std::vector<float> wts;        // record: [npts][8] interpolation weights
};

// Trilinear corners and weights of one point; corner c = 4 dx + 2 dy + dz,
// cell = floor(x/h) clamped to [0, n-2].  Returns false if outside the grid.
bool trilinear(const Dims &d, const float *h, const float *xyz, long long corner[8],
               float w[8], int cx[8], int cy[8], int cz[8])
{
    const int n[3] = {d.nx, d.ny, d.nz};
    int cell[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        const double s = (double)xyz[a] / (double)h[a];
        if (!std::isfinite(s) || s < -1e-4 || s > (double)(n[a] - 1) + 1e-4) return false;
        int i = (int)std::floor(s);
        if (i < 0) i = 0;
        if (i > n[a] - 2) i = n[a] - 2;
        cell[a] = i;
        f[a] = s - (double)i;
    }
    for (int c = 0; c < 8; ++c) {
        const int dx = (c >> 2) & 1, dy = (c >> 1) & 1, dz = c & 1;
        const double wx = dx ? f[0] : 1.0 - f[0];
        const double wy = dy ? f[1] : 1.0 - f[1];
        const double wz = dz ? f[2] : 1.0 - f[2];
        cx[c] = cell[0] + dx;
        cy[c] = cell[1] + dy;
        cz[c] = cell[2] + dz;
        corner[c] = ((long long)cx[c] * d.ny + cy[c]) * d.nz + cz[c];
        w[c] = (float)(wx * wy * wz);
    }
    return true;
}

// Build a table of unique grid points touched by `pts`.  For injection
// (record == false) each unique point lists (point index, weight) in
// ascending point order; for recording it lists the corner slots 8 r + c.
int build_table(const Dims &d, const float *h, const wave_points *p, bool record, HostTable *t)
{
    const int np = p ? p->npts : 0;
    t->plane_start.assign(d.nx + 1, 0);
    t->pts.clear();
    t->item.clear();
    t->w.clear();
    t->wts.assign((size_t)8 * np, 0.f);
    if (np == 0) return WAVE_OK;
    if (p->xyz == nullptr) return WAVE_EINVAL;
    struct Entry {
        int x, y, z, idx;
        float w;
    };
    std::vector<Entry> ent;
    ent.reserve((size_t)8 * np);
    for (int i = 0; i < np; ++i) {
        long long corner[8];
        float w[8];
        int cx[8], cy[8], cz[8];
        if (!trilinear(d, h, p->xyz + 3 * i, corner, w, cx, cy, cz)) return WAVE_EINVAL;
        for (int c = 0; c < 8; ++c) {
            ent.push_back({cx[c], cy[c], cz[c], record ? 8 * i + c : i, w[c]});
            t->wts[(size_t)8 * i + c] = w[c];
        }
    }
    // stable sort keeps ascending point index among equal grid points
    std::stable_sort(ent.begin(), ent.end(), [](const Entry &a, const Entry &b) {
        return std::tie(a.x, a.y, a.z) < std::tie(b.x, b.y, b.z);
    });
    for (size_t i = 0; i < ent.size();) {
        size_t j = i;
        const int begin = (int)t->item.size();
        while (j < ent.size() && ent[j].x == ent[i].x && ent[j].y == ent[i].y && ent[j].z == ent[i].z) {
            t->item.push_back(ent[j].idx);
            t->w.push_back(ent[j].w);
            ++j;
        }
        t->pts.push_back(make_int4(ent[i].y, ent[i].z, begin, (int)t->item.size()));
        t->plane_start[ent[i].x + 1]++;
        i = j;
    }
    for (int x = 0; x < d.nx; ++x) t->plane_start[x + 1] += t->plane_start[x];
    return WAVE_OK;
}

// Device copy of a table inside the workspace.
struct DevTable {
    int *plane_start = nullptr;
    int4 *pts = nullptr;
    int *item = nullptr;
    float *w = nullptr;
    float *wts = nullptr;
    int npts = 0;
    float *f = nullptr;      // injection tables: room for the summed entry values [rows][8 npts]
    long long fstride = 0;
    bool fready = false;     // f holds this call's sums (sum_table)
    PointTable view() const
    {
        return PointTable{npts ? plane_start : nullptr, pts, item, w, fready ? f : nullptr, fstride};
    }
};

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------

struct Carver {
    char *base;
    size_t off = 0, cap;
    bool dry;
    Carver(void *b, size_t c, bool d) : base((char *)b), cap(c), dry(d) {}
    template <class T>
    T *take(size_t count)
    {
        const size_t bytes = align_up(sizeof(T) * std::max<size_t>(count, 1));
        T *p = dry ? nullptr : (T *)(base + off);
        off += bytes;
        return p;
    }
};

// rows > 0: an injection table, with room for the summed value of each
// entry at each of `rows` trace rows
void carve_table(Carver &c, const Dims &d, int np, DevTable *t, int rows = 0)
{
    t->plane_start = c.take<int>(d.nx + 1);
    t->pts = c.take<int4>((size_t)8 * np);
    t->item = c.take<int>((size_t)8 * np);
    t->w = c.take<float>((size_t)8 * np);
    t->wts = c.take<float>((size_t)8 * np);
    t->npts = np;
    if (rows > 0 && np > 0) {
        t->fstride = 8LL * np;
        t->f = c.take<float>((size_t)rows * 8 * np);
    }
}

int upload_table(const HostTable &h, const DevTable &t, cudaStream_t s)
{
    if (t.npts == 0) return WAVE_OK;
    CK(cudaMemcpyAsync(t.plane_start, h.plane_start.data(), sizeof(int) * h.plane_start.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(t.pts, h.pts.data(), sizeof(int4) * h.pts.size(), cudaMemcpyHostToDevice, s));
    if (!h.item.empty()) {
        CK(cudaMemcpyAsync(t.item, h.item.data(), sizeof(int) * h.item.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(t.w, h.w.data(), sizeof(float) * h.w.size(), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync(t.wts, h.wts.data(), sizeof(float) * h.wts.size(), cudaMemcpyHostToDevice, s));
    return WAVE_OK;
}

// The value each entry of injection table t injects at every trace row of
// the call (traces q [rows][nq]), summed once here so that the sweeps read
// one value per entry and plane instead of its items, weights and traces.
int sum_table(const HostTable &h, DevTable &t, const float *q, int nq, int rows, cudaStream_t s)
{
    t.fready = false;
    if (t.npts == 0 || t.f == nullptr || q == nullptr || rows <= 0 || h.pts.empty()) return WAVE_OK;
    CK(wt::launch_inj_sum(t.pts, t.item, t.w, q, nq, (int)h.pts.size(), rows, t.fstride, t.f, s));
    t.fready = true;
    return WAVE_OK;
}

struct Layout {
    int *status = nullptr;
    float *cB = nullptr, *cC = nullptr, *cE = nullptr;
    float *U[4] = {nullptr, nullptr, nullptr, nullptr};
    float *V[4] = {nullptr, nullptr, nullptr, nullptr};
    float *G = nullptr;
    float *store = nullptr;
    float *slots = nullptr;  // revolve: nslots states of two levels
    DevTable inj, rec, inj2;
    float *corner = nullptr;
    int *order = nullptr;    // launch order of the sweep's blocks (order_cap entries)
    int *order_b = nullptr;  // GRAD, REVOLVE, BORN: a second order buffer (the other jobs of the call)
    int *order_c = nullptr;  // REVOLVE: a third
    long long order_cap = 0;
    size_t bytes = 0;
};

// op FWD: inj = sources, rec = receivers, corner [nt][8 nrec]
// op ADJ: inj = receivers, rec = sources, corner [nt][8 nsrc]
// op GRAD: inj = sources (recompute), inj2 = receivers (adjoint), V, G, store [k]
// op REVOLVE: as GRAD with one store row, then ckpt_every (= nslots) states
// op BORN: E, U (background), V (perturbation), G = the Born coefficient P,
//          one store row (the background's D), inj = sources, rec = receivers
//          (recording the perturbation), corner [nt][8 nrec]
Layout carve(void *ws, size_t cap, bool dry, const Dims &d, int op, int nsrc, int nrec, int nt,
             int ckpt_every)
{
    Carver c(ws, cap, dry);
    Layout L;
    const bool grad = op == WAVE_OP_GRAD || op == WAVE_OP_REVOLVE;
    L.status = c.take<int>(kStatusWords);
    L.cB = c.take<float>(d.npad);
    L.cC = c.take<float>(d.npad);
    if (grad || op == WAVE_OP_BORN) L.cE = c.take<float>(d.npad);
    for (int i = 0; i < 4; ++i) L.U[i] = c.take<float>(d.npad);
    if (op == WAVE_OP_BORN) {
        for (int i = 0; i < 4; ++i) L.V[i] = c.take<float>(d.npad);
        L.G = c.take<float>(d.npad);
        L.store = c.take<float>(d.npad);
        carve_table(c, d, nsrc, &L.inj, nt);
        carve_table(c, d, nrec, &L.rec);
        L.corner = c.take<float>((size_t)nt * 8 * std::max(nrec, 0));
    } else if (grad) {
        for (int i = 0; i < 4; ++i) L.V[i] = c.take<float>(d.npad);
        L.G = c.take<float>(d.npad);
        const int rows = op == WAVE_OP_REVOLVE ? 1 : std::max(1, std::min(ckpt_every, nt));
        L.store = c.take<float>((size_t)d.npad * (size_t)rows);
        if (op == WAVE_OP_REVOLVE) L.slots = c.take<float>((size_t)d.npad * 2 * (size_t)std::max(0, ckpt_every));
        carve_table(c, d, nsrc, &L.inj, nt);
        carve_table(c, d, nrec, &L.inj2, nt);
    } else {
        const int ni = op == WAVE_OP_FWD ? nsrc : nrec;
        const int nr = op == WAVE_OP_FWD ? nrec : nsrc;
        carve_table(c, d, ni, &L.inj, nt);
        carve_table(c, d, nr, &L.rec);
        L.corner = c.take<float>((size_t)nt * 8 * std::max(nr, 0));
    }
    if (nsrc + nrec > 0) {
        // as many blocks as the smallest compiled tile (32 x 8) with one-plane
        // x-chunks can make
        L.order_cap = (long long)((d.nzp + 31) / 32) * ((d.ny + 7) / 8) * d.nx;
        L.order = c.take<int>((size_t)L.order_cap);
        if (op == WAVE_OP_GRAD || op == WAVE_OP_REVOLVE || op == WAVE_OP_BORN)
            L.order_b = c.take<int>((size_t)L.order_cap);
        if (op == WAVE_OP_REVOLVE) L.order_c = c.take<int>((size_t)L.order_cap);
    }
    L.bytes = c.off;
    return L;
}

// ---------------------------------------------------------------------------
// Variants, plans and the autotuner
// ---------------------------------------------------------------------------

int variants_for(int R, const SweepVariant **out)
{
    switch (R) {
    case 1: return wt::sweep_variants_r1(out);
    case 2: return wt::sweep_variants_r2(out);
    case 3: return wt::sweep_variants_r3(out);
    case 4: return wt::sweep_variants_r4(out);
    case 5: return wt::sweep_variants_r5(out);
    case 6: return wt::sweep_variants_r6(out);
    case 7: return wt::sweep_variants_r7(out);
    case 8: return wt::sweep_variants_r8(out);
    default: *out = nullptr; return 0;
    }
}

int sm_count()
{
    static const int n = [] {  // thread-safe one-time initialisation
        int dev = 0, c = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
            c = 152;
        return c;
    }();
    return n;
}

struct Plan {
    const SweepVariant *v = nullptr;
    int chunk = 0;
    bool chunk_given = false;  // the caller's tile_x, kept for every variant of the run
};

int tiles(int n, int b) { return (n + b - 1) / b; }

// Dynamic shared memory of a launch: rings, barriers and the per-plane
// sparse slices of an x-chunk.
size_t launch_smem(const SweepVariant *v, int chunk)
{
    return v->smem + wt::sweep_table_bytes(chunk, v->R * v->T) + 16;
}

// Largest x-chunk whose sparse slices still fit the per-block limit.
int max_chunk(const SweepVariant *v)
{
    const long long room = (227LL * 1024 - 16 - (long long)v->smem - 15) / 10 - 3LL * v->R * v->T - 2;
    return (int)std::max(16LL, std::min(room, 1LL << 20));
}

// Resident blocks per SM of variant v at `chunk` (cached per device).
int occupancy(const SweepVariant *v, int chunk)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, size_t>, int> cache;
    const size_t smem = launch_smem(v, chunk);
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, v->func, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    wt::allow_max_dynamic_smem(v->func);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&occ, v->func, v->threads, smem,
                                                               cudaOccupancyDefault) != cudaSuccess ||
        occ < 1)
        occ = 1;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = occ;
    return occ;
}

// Default x-chunk.  Blocks (column tile x chunk) run in about ceil(blocks /
// slots) waves of resident blocks.  A chunk of c planes streams c + 2RT
// planes; its first 2R planes only fill the queue (no arithmetic, no
// coefficient loads), counted at half a plane each, plus a few planes' worth
// for the block's set-up.
int default_chunk(const Dims &d, const SweepVariant *v)
{
    const long long cols = (long long)tiles(d.nzp, v->BZ) * tiles(d.ny, v->BY);
    const int RT = v->R * v->T;
    int best = std::min(d.nx, max_chunk(v));
    double best_cost = 1e300;
    for (int nch = 1; nch <= 64; ++nch) {
        const int chunk = tiles(d.nx, nch);
        if (chunk > max_chunk(v)) continue;
        if (nch > 1 && chunk < 2 * RT) break;
        const long long blocks = cols * tiles(d.nx, chunk);
        const long long slots = (long long)sm_count() * occupancy(v, chunk);
        const long long rounds = (blocks + slots - 1) / slots;
        const double cost = (double)rounds * (chunk + 2.0 * RT - v->R + 4.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = chunk;
        }
    }
    return best;
}

// Rows per thread of a variant (sweep.cuh variants: one).
int rows_of(const SweepVariant *v) { return v->VY > 0 ? v->VY : 1; }

// The gradient-mode variant (XB = mode) of shape v (same kernel family,
// tile, rows and, for the stage-specialised sweep, prefetch), or nullptr.
int mode_variants_for(int R, const SweepVariant **out)
{
    switch (R) {
    case 1: return wt::sweep_mode_variants_r1(out);
    case 2: return wt::sweep_mode_variants_r2(out);
    case 3: return wt::sweep_mode_variants_r3(out);
    case 4: return wt::sweep_mode_variants_r4(out);
    case 5: return wt::sweep_mode_variants_r5(out);
    case 6: return wt::sweep_mode_variants_r6(out);
    case 7: return wt::sweep_mode_variants_r7(out);
    case 8: return wt::sweep_mode_variants_r8(out);
    default: *out = nullptr; return 0;
    }
}

// The two-step Adams-Bashforth variant (mode 4) of radius R and depth T.
const SweepVariant *ab2_variant(int R, int T)
{
    const SweepVariant *vs = nullptr;
    const int nv = mode_variants_for(R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].XB == 4 && vs[i].T == T) return &vs[i];
    return nullptr;
}

// The fused Born variant (mode 5: background and perturbation in one
// sweep) of radius R, or nullptr.
const SweepVariant *born_fused_variant(int R)
{
    const SweepVariant *vs = nullptr;
    const int nv = mode_variants_for(R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].XB == 5) return &vs[i];
    return nullptr;
}

// The variant of the Born perturbation sweep (mode 3) of radius R.
const SweepVariant *born_variant(int R)
{
    const SweepVariant *vs = nullptr;
    const int nv = mode_variants_for(R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].XB == 3) return &vs[i];
    return nullptr;
}

const SweepVariant *mode_variant(const SweepVariant *v, int mode)
{
    const SweepVariant *vs = nullptr;
    const int nv = mode_variants_for(v->R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].T == v->T && vs[i].V == v->V && vs[i].BZ == v->BZ && vs[i].BY == v->BY && vs[i].XB == mode &&
            vs[i].kind == v->kind && rows_of(&vs[i]) == rows_of(v) && (v->kind == 0 || vs[i].P == v->P))
            return &vs[i];
    if (v->kind == 1)  // another shape of the same family and depth
        for (int i = 0; i < nv; ++i)
            if (vs[i].T == v->T && vs[i].XB == mode && vs[i].kind == 1) return &vs[i];
    return nullptr;
}

// Whether variant v is of the kernel family `kernel` names (wave_tuning.kernel:
// 0 any, 1 the sweep of sweep.cuh, 2 the stage-specialised sweep).
bool kernel_matches(const SweepVariant *v, int kernel) { return kernel == 0 || kernel == v->kind + 1; }

// Pick the variant for radius R with time tile T (and tile_y / vec if given).
// The first compiled variant of radius R and depth T with the given shape
// (0 = any value of that field).
const SweepVariant *find_variant(int R, int T, int tile_y, int vec, int tile_z = 0, int kernel = 0,
                                 int rows = 0)
{
    const SweepVariant *vs;
    const int nv = variants_for(R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].T == T && (tile_y == 0 || vs[i].BY == tile_y) && (vec == 0 || vs[i].V == vec) &&
            (tile_z == 0 || vs[i].BZ == tile_z) && kernel_matches(&vs[i], kernel) &&
            (rows == 0 || rows_of(&vs[i]) == rows))
            return &vs[i];
    return nullptr;
}

// Largest-T variant of radius R with T <= limit (T = 1 always exists), of
// kernel family `kind` where one exists (any family otherwise; -1: any).
const SweepVariant *fallback_variant(int R, int limit, int kind = -1)
{
    const SweepVariant *vs;
    const int nv = variants_for(R, &vs);
    const SweepVariant *best = nullptr;
    for (int i = 0; i < nv; ++i) {
        if (vs[i].T > limit) continue;
        const bool better = best == nullptr || vs[i].T > best->T ||
                            (vs[i].T == best->T && kind >= 0 && vs[i].kind == kind && best->kind != kind);
        if (better) best = &vs[i];
    }
    return best;
}

struct TuneKey {
    int nx, ny, nz, so, dev, T;  // T = 0: any depth
    bool operator<(const TuneKey &o) const
    {
        return std::tie(nx, ny, nz, so, dev, T) < std::tie(o.nx, o.ny, o.nz, o.so, o.dev, o.T);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, Plan> g_tune_cache;

bool tune_log()
{
    const char *e = std::getenv("WAVE_AUTOTUNE_LOG");
    return e != nullptr && e[0] != '\0' && e[0] != '0';
}

// Optional plan cache file (env WAVE_TUNE_CACHE = path): one plan per line,
//   nx ny nz space_order T_requested  ->  T tile_y vec chunk [tile_z [kernel rows]]
// Lines naming variants that are not compiled in, or of another format, are
// ignored; a line without tile_z takes the first variant of that shape, and a
// line without kernel and rows the first of either kernel family.

bool cache_lookup_file(const TuneKey &k, Plan *out)
{
    const char *path = std::getenv("WAVE_TUNE_CACHE");
    if (path == nullptr || !path[0]) return false;
    FILE *f = std::fopen(path, "r");
    if (f == nullptr) return false;
    int nx, ny, nz, so, tr, T, by, vec, chunk, bz, kern, rows;
    bool found = false;
    char line[256];
    while (std::fgets(line, sizeof(line), f) != nullptr) {
        bz = kern = rows = 0;
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d", &nx, &ny, &nz, &so, &tr, &T,
                                    &by, &vec, &chunk, &bz, &kern, &rows);
        if (got != 9 && got != 10 && got != 12) continue;
        if (nx == k.nx && ny == k.ny && nz == k.nz && so == k.so && tr == k.T) {
            const SweepVariant *v = find_variant(so / 2, T, by, vec, bz, kern, rows);
            if (v != nullptr && chunk > 0) {
                out->v = v;
                out->chunk = chunk;
                found = true;  // the last matching line wins
            }
        }
    }
    std::fclose(f);
    return found;
}

void cache_store_file(const TuneKey &k, const Plan &p)
{
    const char *path = std::getenv("WAVE_TUNE_CACHE");
    if (path == nullptr || !path[0]) return;
    FILE *f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d\n", k.nx, k.ny, k.nz, k.so, k.T, p.v->T, p.v->BY,
                 p.v->V, p.chunk, p.v->BZ, p.v->kind + 1, rows_of(p.v));
    std::fclose(f);
}

TuneKey tune_key(const Dims &d, int so, int T)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return TuneKey{d.nx, d.ny, d.nz, so, dev, T};
}

// ---------------------------------------------------------------------------
// The sweep driver
// ---------------------------------------------------------------------------

// What one run of consecutive steps injects, records and stores.  Every row
// index is "base + dir * j" for local step j of the run (j = 0 first).
struct State;  // a wavefield's four buffers and which hold levels n and n-1 (below)

// The heavy-first launch order a job's order buffer holds: the launch shape
// it was computed for.  A caller that runs one job in many short run_steps
// calls (one step each) keeps one of these per job and order buffer, so that
// the order is computed and uploaded once, not per call (an upload from
// pageable host memory first waits for the stream to drain).
struct OrderCache {
    const SweepVariant *v = nullptr;
    int chunk = 0;
    bool ordered = false;
};

struct Job {
    Dims d;
    Stencil st;
    const float *cB, *cC, *cE;
    int *status = nullptr;
    int withhold = 0;
    PointTable inj{};
    const float *q = nullptr;
    int nq = 0, q_base = 0, q_dir = 1;
    PointTable rec{};
    float *corner = nullptr;
    int nslot = 0, c_base = 0, c_dir = 1;
    float *dstore = nullptr;
    long long d_base = 0;
    int d_dir = 1;
    const float *dload = nullptr;
    long long l_base = 0;
    int l_dir = 1;
    long long l_rows = 1;  // rows of the store dload points at
    float *gacc = nullptr;
    const float *born = nullptr;  // Born perturbation sweep: the coefficient P = -dm / dt^2 (padded)
    int ab2 = 0;                  // two-step Adams-Bashforth heat: its depth (1 or 2); 0: not that scheme
    State *s2 = nullptr;          // fused Born (with born): the perturbation field's state, advanced with s
    // host copies of the injection / record tables and the device buffer for
    // the heavy-first launch order (nullptr: natural order)
    const HostTable *hinj = nullptr, *hrec = nullptr;
    int *order = nullptr;
    long long order_cap = 0;
    OrderCache *ocache = nullptr;  // kept across run_steps calls (the order buffer is this job's alone)
};

// Events around the sweep launches of the last timed call on this thread.
struct SweepProf {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int launches = 0, steps = 0;
    bool valid = false, active = false;
};
thread_local SweepProf g_prof;

int prof_begin(const wave_tuning *t, cudaStream_t s)
{
    g_prof.active = t != nullptr && (t->flags & WAVE_TIME_SWEEPS);
    if (!g_prof.active) return WAVE_OK;
    if (g_prof.e0 == nullptr) {
        CK(cudaEventCreate(&g_prof.e0));
        CK(cudaEventCreate(&g_prof.e1));
    }
    g_prof.launches = 0;
    g_prof.steps = 0;
    g_prof.valid = false;
    CK(cudaEventRecord(g_prof.e0, s));
    return WAVE_OK;
}

int prof_end(cudaStream_t s)
{
    if (!g_prof.active) return WAVE_OK;
    CK(cudaEventRecord(g_prof.e1, s));
    g_prof.valid = true;
    g_prof.active = false;
    return WAVE_OK;
}

// Four buffers; (a, b) index levels n and n-1.
struct State {
    float *buf[4];
    int a = 0, b = 1;
};

// Arguments and TMA descriptors of the launch that advances state `s` of
// `job` by variant v from local step j (rows of the step-dependent tables are
// those of step j), with x-chunk `chunk`.  *nblocks receives the grid size.
int build_launch(const Job &job, const State &s, int j, const SweepVariant *v, int chunk, SweepArgs *ap,
                 wt::SweepMaps *mp, wt::TMaps *tm, long long *nblocks)
{
    const Dims &d = job.d;
    SweepArgs &a = *ap;
    std::memset(&a, 0, sizeof(a));
    std::memset(mp, 0, sizeof(*mp));
    std::memset(tm, 0, sizeof(*tm));
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nzp;
    a.sx = (int)((long long)d.ny * d.nzp);
    a.npad = d.npad;
    a.status = job.status;
    int rc = WAVE_OK;
    if (v->kind == 1) {
        // stage-specialised sweep: stage-1 boxes, its centre box, and the
        // output-tile boxes of stage 2
        rc = encode_map(&tm->uc, s.buf[s.a], d, v->WC, v->HC);
        if (!rc) rc = encode_map(&tm->uf, s.buf[s.a], d, v->W1, v->H1);
        if (!rc) rc = encode_map(&tm->um, s.buf[s.b], d, v->W1, v->H1);
        if (!rc) rc = encode_map(&tm->B, job.cB, d, v->W1, v->H1);
        if (!rc) rc = encode_map(&tm->C, job.cC, d, v->W1, v->H1);
        if (!rc && v->T == 2) rc = encode_map(&tm->u2, s.buf[s.a], d, v->BZ, v->BY);
        if (!rc && v->T == 2) rc = encode_map(&tm->B2, job.cB, d, v->BZ, v->BY);
        if (!rc && v->T == 2) rc = encode_map(&tm->C2, job.cC, d, v->BZ, v->BY);
        // gradient modes (XB = MODE): E, or this launch's D rows and G
        if (!rc && v->XB == 1) {
            rc = encode_map(&tm->x0, job.cE, d, v->W1, v->H1);
            if (!rc && v->T == 2) rc = encode_map(&tm->y0, job.cE, d, v->BZ, v->BY);
        }
        // the D rows: the whole store, the launch's rows chosen by l_row0
        if (!rc && v->XB == 2) {
            if (v->T == 1) {
                rc = encode_rows_map(&tm->x0, job.dload, d, job.l_rows, v->W1, v->H1);
                if (!rc) rc = encode_map(&tm->x1, job.gacc, d, v->W1, v->H1);
            } else {
                rc = encode_rows_map(&tm->y0, job.dload, d, job.l_rows, v->BZ, v->BY);
                if (!rc) rc = encode_rows_map(&tm->y1, job.dload, d, job.l_rows, v->BZ, v->BY);
                if (!rc) rc = encode_map(&tm->y2, job.gacc, d, v->BZ, v->BY);
            }
        }
        if (!rc && v->XB == 3) {
            rc = encode_rows_map(&tm->x0, job.dload, d, job.l_rows, v->W1, v->H1);
            if (!rc) rc = encode_map(&tm->x1, job.born, d, v->W1, v->H1);
        }
        // fused Born: E and P, and the perturbation field's centre box and levels
        if (!rc && v->XB == 5) {
            if (job.s2 == nullptr) return WAVE_EINVAL;
            const State &s2 = *job.s2;
            rc = encode_map(&tm->x0, job.cE, d, v->W1, v->H1);
            if (!rc) rc = encode_map(&tm->x1, job.born, d, v->W1, v->H1);
            if (!rc) rc = encode_map(&tm->y0, s2.buf[s2.a], d, v->WC, v->HC);
            if (!rc) rc = encode_map(&tm->y1, s2.buf[s2.a], d, v->W1, v->H1);
            if (!rc) rc = encode_map(&tm->y2, s2.buf[s2.b], d, v->W1, v->H1);
        }
        if (rc) return rc;
    } else {
        rc = encode_map(&mp->u, s.buf[s.a], d, v->PW, v->H0);
        if (!rc) rc = encode_map(&mp->um, s.buf[s.b], d, v->W0, v->HK);
        if (!rc) rc = encode_map(&mp->B, job.cB, d, v->W0, v->HK);
        if (!rc) rc = encode_map(&mp->C, job.cC, d, v->W0, v->HK);
    }
    if (!rc && v->kind == 0 && v->T == 1) rc = encode_map(&mp->uk, s.buf[s.a], d, v->W0, v->HK);
    // the extra boxes of sweep.cuh's gradient modes (the stage-specialised
    // sweep reads its gradient-mode arrays with plain loads)
    if (!rc && v->kind == 0 && v->XB == 1) rc = encode_map(&mp->x0, job.cE, d, v->W0, v->HK);
    if (!rc && v->kind == 0 && v->XB == 2) {
        const long long row = job.l_base + (long long)job.l_dir * j;  // this step's D row
        rc = encode_map(&mp->x0, job.dload + row * d.npad, d, v->W0, v->HK);
        if (!rc) rc = encode_map(&mp->x1, job.gacc, d, v->W0, v->HK);
    }
    if (rc) return rc;
    int spare[2], ns = 0;
    for (int i = 0; i < 4; ++i)
        if (i != s.a && i != s.b) spare[ns++] = i;
    if (v->T == 1 && !(v->kind == 1 && v->XB == 4)) {
        a.out_hi = s.buf[s.b];
        if (v->kind == 1 && v->XB == 5) a.out_lo = job.s2->buf[job.s2->b];  // in place, as the background
    } else {
        // T >= 2, and the two-step Adams-Bashforth sweep at any depth: the new
        // level and the new rate (the old ones are still read by neighbours)
        a.out_hi = s.buf[spare[0]];
        a.out_lo = s.buf[spare[1]];
    }
    a.cE = job.cE;
    a.inj = job.inj;
    // the sweeps read injection values only from the call's sums (sum_table)
    if (a.inj.plane_start != nullptr && a.inj.f == nullptr) return WAVE_EINVAL;
    a.q = job.q;
    a.nq = job.nq;
    a.q_row0 = job.q_base + job.q_dir * j;
    a.q_dir = job.q_dir;
    a.rec = job.rec;
    a.corner = job.corner;
    a.nslot = job.nslot;
    a.c_row0 = job.c_base + job.c_dir * j;
    a.c_dir = job.c_dir;
    a.dstore = job.dstore;
    a.d_row0 = job.d_base + (long long)job.d_dir * j;
    a.d_dir = job.d_dir;
    a.dload = job.dload;
    a.l_row0 = job.l_base + (long long)job.l_dir * j;
    a.l_dir = job.l_dir;
    a.gacc = job.gacc;
    // the two-step Adams-Bashforth weights of stage 1: an Euler step first
    a.ab1 = job.ab2 != 0 && job.q_base + j == 0 ? 1.f : 1.5f;
    a.ab0 = job.ab2 != 0 && job.q_base + j == 0 ? 0.f : -0.5f;
    a.withhold = job.withhold;
    a.chunk = chunk;
    a.tiles_z = tiles(d.nzp, v->BZ);
    a.tiles_y = tiles(d.ny, v->BY);
    *nblocks = (long long)a.tiles_z * a.tiles_y * tiles(d.nx, chunk);
    return *nblocks > 0x7fffffffLL ? WAVE_EINVAL : WAVE_OK;
}

// The state after one launch of depth T: T = 1 writes level n+1 where n-1
// was; T >= 2 writes the two spare buffers.
void advance_state(State &s, int T)
{
    if (T == 1) {
        std::swap(s.a, s.b);
    } else {
        int spare[2], ns = 0;
        for (int i = 0; i < 4; ++i)
            if (i != s.a && i != s.b) spare[ns++] = i;
        s.a = spare[0];
        s.b = spare[1];
    }
}

long long floor_div(long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Mark the tiles of variant v with x-chunk `chunk` whose sweep handles a point
// of table t: the kernel's own per-block relevance tests, on the host.  An
// injection table (record false) concerns a block's whole layout
// [gy0, gy0 + H0) x [gz0 + ZL, gz0 + ZR), a record table its own tile
// [gy0 + RT, +BY) x [gz0 + A0, +BZ), over the planes [X0 - 2RT, X1 + RT + 2)
// the block scans.  Returns whether any tile was marked.
bool mark_heavy(const Dims &d, const SweepVariant *v, int chunk, const HostTable *t, bool record,
                std::vector<char> &heavy)
{
    if (t == nullptr || t->pts.empty()) return false;
    const int R = v->R, RT = v->R * v->T, BZ = v->BZ, BY = v->BY;
    const int A0 = (RT + 3) / 4 * 4, H0 = BY + 2 * RT;
    const int ZL = (A0 - (v->T - 1) * R) / 4 * 4, ZR = (A0 + BZ + (v->T - 1) * R + 3) / 4 * 4;
    const int tz = tiles(d.nzp, BZ), ty = tiles(d.ny, BY), tx = tiles(d.nx, chunk);
    heavy.resize((size_t)tz * ty * tx, 0);
    // y and z ranges relative to (tile origin - RT, tile origin - A0):
    // sweep.cuh injects over its layout [0, H0) x [ZL, ZR); the
    // stage-specialised sweep over its stage-1 region (the tile widened by
    // (T-1)R rows and (T-1)RP columns); both record over the tile itself
    int ylo = record ? RT : 0, yhi = record ? RT + BY : H0;
    int zlo = record ? A0 : ZL, zhi = record ? A0 + BZ : ZR;
    if (v->kind == 1 && !record) {
        const int RP = (R + 3) / 4 * 4;
        ylo = RT - (v->T - 1) * R;
        yhi = ylo + v->H1;
        zlo = A0 - (v->T - 1) * RP;
        zhi = zlo + v->W1;
    }
    bool any = false;
    for (int x = 0; x < d.nx; ++x) {
        for (int e = t->plane_start[x]; e < t->plane_start[x + 1]; ++e) {
            const long long y = t->pts[e].x, z = t->pts[e].y;
            const long long x0 = std::max(0LL, floor_div(x - RT - 2, chunk) - 1);
            const long long x1 = std::min<long long>(tx - 1, floor_div(x + 2 * RT, chunk));
            const long long y0 = std::max(0LL, floor_div(y + RT - yhi, BY));
            const long long y1 = std::min<long long>(ty - 1, floor_div(y + RT - ylo, BY));
            const long long z0 = std::max(0LL, floor_div(z + A0 - zhi, BZ));
            const long long z1 = std::min<long long>(tz - 1, floor_div(z + A0 - zlo, BZ));
            for (long long txi = x0; txi <= x1; ++txi) {
                const long long X0 = txi * chunk, X1 = std::min<long long>(X0 + chunk, d.nx);
                if (x < X0 - 2 * RT || x >= X1 + RT + 2) continue;
                for (long long tyi = y0; tyi <= y1; ++tyi) {
                    const long long gy0 = tyi * BY - RT;
                    if (y < gy0 + ylo || y >= gy0 + yhi) continue;
                    for (long long tzi = z0; tzi <= z1; ++tzi) {
                        const long long gz0 = tzi * BZ - A0;
                        if (z < gz0 + zlo || z >= gz0 + zhi) continue;
                        heavy[(size_t)(tzi + tz * (tyi + ty * txi))] = 1;
                        any = true;
                    }
                }
            }
        }
    }
    return any;
}

// Launch order of the blocks of variant v with x-chunk `chunk`: the tiles
// that handle a point of the injection or record table first, then the rest,
// each group in natural order, so that the blocks with the extra sparse work
// run in the first waves.  Empty when no tile is heavy.
void heavy_first_order(const Dims &d, const SweepVariant *v, int chunk, const HostTable *inj,
                       const HostTable *rec, std::vector<int> *order)
{
    order->clear();
    std::vector<char> heavy;
    const bool a = mark_heavy(d, v, chunk, inj, false, heavy);
    const bool b = mark_heavy(d, v, chunk, rec, true, heavy);
    if (!a && !b) return;
    order->reserve(heavy.size());
    for (size_t t = 0; t < heavy.size(); ++t)
        if (heavy[t]) order->push_back((int)t);
    for (size_t t = 0; t < heavy.size(); ++t)
        if (!heavy[t]) order->push_back((int)t);
}

// Advance `st` by nsteps.  When ckpt != nullptr, state c = (u^{ck}, u^{ck-1})
// is copied to ckpt + c * 2 * npad at every step count j0 + j that is a
// multiple of ckpt_every (j counts from the run start, j0 = global offset).
int run_steps(const Job &job, State &s, int nsteps, const Plan &plan, cudaStream_t stream,
              float *ckpt = nullptr, int ckpt_every = 0, int j0 = 0)
{
    const Dims &d = job.d;
    const int R = plan.v->R;
    OrderCache own;  // launch shape the order buffer holds
    OrderCache &oc = job.ocache != nullptr ? *job.ocache : own;
    int j = 0;
    while (j <= nsteps) {
        if (ckpt != nullptr && (j0 + j) % ckpt_every == 0 && j < nsteps) {
            float *dst = ckpt + (size_t)((j0 + j) / ckpt_every) * 2 * d.npad;
            CK(cudaMemcpyAsync(dst, s.buf[s.a], sizeof(float) * d.npad, cudaMemcpyDeviceToDevice, stream));
            CK(cudaMemcpyAsync(dst + d.npad, s.buf[s.b], sizeof(float) * d.npad,
                               cudaMemcpyDeviceToDevice, stream));
        }
        if (j == nsteps) break;
        int limit = nsteps - j;
        if (ckpt != nullptr) limit = std::min(limit, ckpt_every - (j0 + j) % ckpt_every);
        const SweepVariant *v = plan.v->T <= limit ? plan.v : fallback_variant(R, limit, plan.v->kind);
        if (v == nullptr) return WAVE_EUNSUPPORTED;
        int chunk =
            std::min((v == plan.v && plan.chunk > 0) ? plan.chunk : default_chunk(d, v), max_chunk(v));
        // gradient sweeps: the mode variant of the same untiled shape, if compiled,
        // streams their extra inputs (E, or D and G) through TMA
        const int mode = job.ab2 != 0 ? 4
                         : job.gacc != nullptr ? 2
                         : job.dstore != nullptr ? 1
                         : job.born != nullptr ? (job.s2 != nullptr ? 5 : 3) : 0;
        if (mode == 5) {
            v = born_fused_variant(R);
            if (v == nullptr) return WAVE_EUNSUPPORTED;
            chunk = std::min(default_chunk(d, v), max_chunk(v));
        } else if (mode == 4) {
            // the Adams-Bashforth heat sweep: the first step (the Euler start)
            // and a last odd step run untiled
            const int Tw = (j == 0 || limit < 2) ? 1 : job.ab2;
            v = ab2_variant(R, Tw);
            if (v == nullptr) v = ab2_variant(R, 1);
            if (v == nullptr) return WAVE_EUNSUPPORTED;
            chunk = std::min(plan.chunk_given && v->T == plan.v->T ? plan.chunk : default_chunk(d, v), max_chunk(v));
        } else if (mode == 3) {
            // the Born perturbation sweep has one untiled variant per radius
            v = born_variant(R);
            if (v == nullptr) return WAVE_EUNSUPPORTED;
            chunk = std::min(default_chunk(d, v), max_chunk(v));
        } else if (mode > 0 && v->kind == 1) {
            // a stage-specialised shape runs its gradient-mode variant where one
            // is compiled; otherwise the untiled default of sweep.cuh (whose
            // gradient-mode variants stream the extra arrays through TMA, and
            // whose wavefield is bitwise the same) runs the gradient sweeps
            const SweepVariant *mv = mode_variant(v, mode);
            v = mv != nullptr ? mv : find_variant(R, 1, 0, 0, 0, 1);
            if (v == nullptr) return WAVE_EUNSUPPORTED;
            chunk = std::min(plan.chunk_given ? chunk : default_chunk(d, v), max_chunk(v));
        }
        if (mode > 0 && v->kind == 0 && v->T == 1) {
            const SweepVariant *mv = mode_variant(v, mode);
            if (mv != nullptr) {
                // the plan's chunk was chosen for the plain variant, whose
                // blocks per SM can differ: size the mode variant's own grid
                v = mv;
                chunk = std::min(plan.chunk_given ? chunk : default_chunk(d, mv), max_chunk(mv));
            }
        }
        SweepArgs a;
        wt::SweepMaps maps;
        wt::TMaps tmaps;
        long long nblocks = 0;
        int rc = build_launch(job, s, j, v, chunk, &a, &maps, &tmaps, &nblocks);
        if (rc) return rc;
        if (job.order != nullptr && (v != oc.v || chunk != oc.chunk)) {
            oc.v = v;
            oc.chunk = chunk;
            std::vector<int> ord;
            heavy_first_order(d, v, chunk, job.hinj, job.hrec, &ord);
            oc.ordered = !ord.empty() && (long long)ord.size() == nblocks && nblocks <= job.order_cap;
            if (oc.ordered)
                CK(cudaMemcpyAsync(job.order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice,
                                   stream));
        }
        a.order = oc.ordered ? job.order : nullptr;
        if (v->kind == 1)
            CK(v->launch_t((int)nblocks, stream, a, job.st, tmaps));
        else
            CK(v->launch((int)nblocks, stream, a, job.st, maps));
        if (g_prof.active) {
            g_prof.launches++;
            g_prof.steps += v->T;
        }
        advance_state(s, mode == 4 ? 2 : v->T);  // Adams-Bashforth: new level and rate in the spares
        if (mode == 5) advance_state(*job.s2, 1);
        j += v->T;
    }
    return WAVE_OK;
}

// Device figures the runtime bound of a plan uses: theoretical memory
// bandwidth (bytes/s), shared-memory (LSU data pipe) bandwidth at 128 bytes per
// clock per SM at the maximum SM clock (bytes/s), and the L2 size (bytes).
struct DevicePeaks {
    double hbm = 0.0, lsu = 0.0, l2 = 0.0;
};

DevicePeaks device_peaks()
{
    static std::mutex mu;
    static std::map<int, DevicePeaks> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int mem_khz = 0, bus_bits = 0, sm_khz = 0, l2 = 0;
    DevicePeaks p;
    if (cudaDeviceGetAttribute(&mem_khz, cudaDevAttrMemoryClockRate, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&bus_bits, cudaDevAttrGlobalMemoryBusWidth, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sm_khz, cudaDevAttrClockRate, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess) {
        p.hbm = 2.0 * mem_khz * 1e3 * bus_bits / 8.0;  // double data rate
        p.lsu = (double)sm_count() * 128.0 * sm_khz * 1e3;
        p.l2 = l2;
    }
    cache[dev] = p;
    return p;
}

// Bytes one point-update of stage s (1-based, of depth T) moves through the
// SM's LSU data pipe -- the shared-memory and global loads and stores of the
// kernel's code, per point -- for variant v.  TMA copies into shared memory
// do not pass through that pipe.
double lsu_bytes_per_point(const SweepVariant *v, int s)
{
    const int R = v->R, RP = (R + 3) / 4 * 4;
    if (v->kind == 1) {
        // per thread and plane (VY rows x 4 points): the queue feed, the z
        // halos, 2R rows of y-neighbours, level n-1 (or n), B and C, and the
        // plane's output (T = 1: stored; T = 2 stage 1: into ring 1, whose
        // stage-2 feed read is the stage-2 feed above; stage 2: two levels)
        const double VY = v->VY;
        const double out = v->T == 1 ? 16.0 * VY : (s == 1 ? 16.0 * VY : 32.0 * VY);
        return (16.0 * VY + 8.0 * RP * VY + 32.0 * R + 48.0 * VY + out) / (4.0 * VY);
    }
    // sweep.cuh, V points per thread: the feed (stage 1) or the exchanged
    // centre plane, the z window, 2R rows of y-neighbours, B and C, level n-1
    // (stage 1), and the stored or exchanged output
    const double V = v->V;
    return 4.0 + (V + 2.0 * RP) * 4.0 / V + 8.0 * R + 8.0 + (s == 1 ? 4.0 : 0.0) + 4.0;
}

// Lower bound on the milliseconds of one time step of plan (v, chunk) on grid
// d, assuming perfect scheduling: the paper's proposal for pruning the
// auto-tuner's search space (Sec. 6.3.3).  The larger of
//  * DRAM: the compulsory bytes (20 per point-update untiled, 24/T for depth T)
//    at the theoretical memory bandwidth, counted only when the fields are
//    larger than L2 (otherwise they may be served by it);
//  * LSU: lsu_bytes_per_point for every point each stage computes -- the
//    tile and the halo its stage recomputes, over the planes of each x-chunk
//    plus the chunk margins that stage computes, and the tiles overhanging
//    the grid -- at the LSU data-pipe bandwidth.
// hbm, lsu > 0 override the device figures (bytes/s); l2 < 0 ignores L2.
double plan_bound_ms(const Dims &d, const SweepVariant *v, int chunk, double hbm, double lsu, double l2)
{
    const double N = (double)d.npad;
    const int T = v->T, R = v->R, RP = (R + 3) / 4 * 4;
    const double tz = tiles(d.nzp, v->BZ), ty = tiles(d.ny, v->BY), tx = tiles(d.nx, chunk);
    double lsu_bytes = 0.0;
    for (int s = 1; s <= T; ++s) {
        double rows, cols;  // the region stage s computes per tile and plane
        if (v->kind == 1) {
            rows = v->BY + 2.0 * (T - s) * R;
            cols = v->BZ + 2.0 * (T - s) * RP;
        } else {
            rows = v->BY + 2.0 * (T - s) * R;
            cols = v->BZ + 2.0 * (T - s) * R;
        }
        const double planes = d.nx + tx * 2.0 * (T - s) * R;
        lsu_bytes += tz * ty * planes * rows * cols * lsu_bytes_per_point(v, s);
    }
    const double dram_bytes = N * (T == 1 ? 20.0 : 24.0);
    const bool over_l2 = l2 < 0 || 5.0 * 4.0 * N > 2.0 * l2;
    const double t_dram = over_l2 && hbm > 0 ? dram_bytes / hbm : 0.0;
    const double t_lsu = lsu > 0 ? lsu_bytes / lsu : 0.0;
    return 1e3 * std::max(t_dram, t_lsu) / T;
}

// Counts of the last autotuner run on this host thread.
struct TuneStats {
    int candidates = 0, pruned = 0;
};
thread_local TuneStats g_tune_stats;

bool tune_prune()
{
    const char *e = std::getenv("WAVE_TUNE_NOPRUNE");
    return e == nullptr || e[0] == '\0' || e[0] == '0';
}

// Time candidate plans on the real coefficients (zero wavefield, no sparse
// points) and cache the fastest: the paper's auto-tuner extended to the time
// tile (Sec. 4.4, Sec. 5.2.2), here over (T, tile, x-chunk).  Candidates are
// timed in two passes over the whole list (a warm-up launch before the first)
// and each keeps its better pass, so that no candidate's result rests on one
// run taken in one GPU state; candidates within a few percent of each other
// are otherwise decided by noise.
int autotune(const Dims &d, const Stencil &st, const float *cB, const float *cC, float *const U[4],
             int *status, int R, int T_only, cudaStream_t stream, Plan *out)
{
    const SweepVariant *vs;
    const int nv = variants_for(R, &vs);
    std::vector<Plan> cands;
    for (int i = 0; i < nv; ++i) {
        const SweepVariant *v = &vs[i];
        if (T_only > 0 && v->T != T_only) continue;
        std::vector<int> chunks = {default_chunk(d, v)};
        for (int c : {d.nx, (d.nx + 1) / 2, (d.nx + 3) / 4, 128, 64})
            if (c >= 4 * v->R * v->T && c <= d.nx &&
                std::find(chunks.begin(), chunks.end(), c) == chunks.end())
                chunks.push_back(c);
        for (int chunk : chunks) {
            Plan p;
            p.v = v;
            p.chunk = chunk;
            cands.push_back(p);
        }
    }
    if (cands.empty()) return WAVE_EUNSUPPORTED;
    // Candidates are timed in order of their runtime bound, lowest first; one
    // whose bound exceeds the best time measured so far cannot win and is
    // not timed (WAVE_TUNE_NOPRUNE=1 times every candidate).
    const DevicePeaks pk = device_peaks();
    std::vector<double> bound(cands.size());
    std::vector<size_t> order(cands.size());
    for (size_t c = 0; c < cands.size(); ++c) {
        bound[c] = plan_bound_ms(d, cands[c].v, cands[c].chunk, pk.hbm, pk.lsu, pk.l2);
        order[c] = c;
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return bound[a] < bound[b]; });
    const bool prune = tune_prune();
    std::vector<char> skip(cands.size(), 0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<float> best(cands.size(), 1e30f);
    float best_all = 1e30f;
    int rc = WAVE_OK;
    for (int pass = 0; pass < 2 && rc == WAVE_OK; ++pass) {
        for (size_t oi = 0; oi < cands.size() && rc == WAVE_OK; ++oi) {
            const size_t c = order[oi];
            if (pass == 0 && prune && bound[c] > (double)best_all) skip[c] = 1;
            if (skip[c]) continue;
            const Plan &p = cands[c];
            Job job;
            job.d = d;
            job.st = st;
            job.cB = cB;
            job.cC = cC;
            job.cE = nullptr;
            job.status = status;
            State s;
            for (int k = 0; k < 4; ++k) s.buf[k] = U[k];
            const int steps = std::max(12, 12 * p.v->T);
            if (pass == 0 && (rc = run_steps(job, s, p.v->T, p, stream))) break;  // warm-up
            if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = WAVE_ECUDA; break; }
            if ((rc = run_steps(job, s, steps, p, stream))) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = WAVE_ECUDA;
                break;
            }
            best[c] = std::min(best[c], ms / steps);
            best_all = std::min(best_all, best[c]);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    g_tune_stats.candidates = (int)cands.size();
    g_tune_stats.pruned = (int)std::count(skip.begin(), skip.end(), 1);
    size_t bi = order[0];
    for (size_t c = 0; c < cands.size(); ++c)
        if (!skip[c]) {
            bi = c;
            break;
        }
    for (size_t c = 0; c < cands.size(); ++c) {
        if (skip[c]) {
            if (tune_log())
                std::fprintf(stderr, "wave autotune: kernel=%d T=%d tile=%dx%d vec=%d rows=%d P=%d chunk=%d: "
                             "bound %.4f ms/step, not timed\n", cands[c].v->kind + 1, cands[c].v->T,
                             cands[c].v->BZ, cands[c].v->BY, cands[c].v->V, rows_of(cands[c].v), cands[c].v->P,
                             cands[c].chunk, bound[c]);
            continue;
        }
        if (tune_log())
            std::fprintf(stderr, "wave autotune: kernel=%d T=%d tile=%dx%d vec=%d rows=%d P=%d chunk=%d: %.4f ms/step "
                         "(bound %.4f)\n", cands[c].v->kind + 1, cands[c].v->T, cands[c].v->BZ, cands[c].v->BY,
                         cands[c].v->V, rows_of(cands[c].v), cands[c].v->P, cands[c].chunk, best[c], bound[c]);
        // a later candidate must be clearly faster: timings within 1 % are
        // ties, and ties keep the earlier one (the default variant and chunk
        // come first), so run-to-run noise does not flip the plan
        if (best[c] < 0.99f * best[bi]) bi = c;
    }
    *out = cands[bi];
    return WAVE_OK;
}

// Plan for this call: explicit tuning, or the cached / freshly tuned one.
// `may_tune` is false for dry queries (wave_describe_plan).
int resolve_plan(const Dims &d, const wave_grid *g, const wave_tuning *t, bool may_tune,
                 const Stencil *st, const float *cB, const float *cC, float *const U[4], int *status,
                 cudaStream_t stream, Plan *out)
{
    const int R = g->space_order / 2;
    const int T = t ? t->time_tile : 0;
    if (T < 0 || (t && (t->tile_x < 0 || t->tile_y < 0 || t->vec < 0 || t->kernel < 0 || t->kernel > 2 ||
                        t->rows < 0)))
        return WAVE_EINVAL;
    const bool shape_tune = T > 0 && t && (t->flags & WAVE_AUTOTUNE_SHAPE);
    if (shape_tune && fallback_variant(R, T) == nullptr) return WAVE_EUNSUPPORTED;
    if (T > 0 && !shape_tune) {
        const SweepVariant *v = find_variant(R, T, t ? t->tile_y : 0, t ? t->vec : 0, t ? t->tile_z : 0,
                                             t ? t->kernel : 0, t ? t->rows : 0);
        if (v == nullptr) return WAVE_EUNSUPPORTED;
        out->v = v;
        out->chunk = (t && t->tile_x > 0) ? std::min(t->tile_x, d.nx) : default_chunk(d, v);
        out->chunk_given = t && t->tile_x > 0;
        return WAVE_OK;
    }
    const TuneKey key = tune_key(d, g->space_order, T);
    // wave_autotune_stats describes the autotuner run of the last call that
    // resolved a plan this way; a plan from a cache leaves none
    if (may_tune) g_tune_stats = TuneStats();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            return WAVE_OK;
        }
        Plan fp;
        if (cache_lookup_file(key, &fp)) {
            g_tune_cache[key] = fp;
            *out = fp;
            return WAVE_OK;
        }
    }
    if (!may_tune) {
        out->v = shape_tune ? find_variant(R, T, 0, 0) : fallback_variant(R, 1);
        if (out->v == nullptr) return WAVE_EUNSUPPORTED;
        out->chunk = default_chunk(d, out->v);
        return WAVE_OK;
    }
    Plan p;
    const int rc = autotune(d, *st, cB, cC, U, status, R, T, stream, &p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = p;
    cache_store_file(key, p);
    *out = p;
    return WAVE_OK;
}

// The shapes that run the gradient sweeps of wave_grad: the recompute sweep
// storing second differences (mode 1) and the adjoint sweep with the imaging
// condition (mode 2), chosen each on its own.  Which is fastest depends on
// the grid and on the phase -- the shared-warp untiled sweep streams E, D and
// G through TMA with three or four blocks per SM, the stage-specialised
// shapes save DRAM bytes but hold fewer warps, the imaging condition loads
// and stores more per point than the recompute, and a block that injects
// many points waits on their table and trace loads every plane -- so the
// candidates are timed once per (grid, forward plan, source and receiver
// counts) on the workspace's scratch state with the call's own sources and
// receivers, a few steps of each phase, and the fastest of each phase kept.
// The candidates: the untiled default of sweep.cuh (its own mode variants),
// and, when the forward plan is stage-specialised, every compiled
// stage-specialised mode variant of the plan's depth or untiled.  Every
// candidate gives the same bits.
struct GradKey {
    int nx, ny, nz, so, dev, nsrc, nrec, rows;
    const SweepVariant *v;
    bool operator<(const GradKey &o) const
    {
        return std::tie(nx, ny, nz, so, dev, nsrc, nrec, rows, v) <
               std::tie(o.nx, o.ny, o.nz, o.so, o.dev, o.nsrc, o.nrec, o.rows, o.v);
    }
};
std::mutex g_grad_mu;
std::map<GradKey, std::pair<Plan, Plan>> g_grad_cache;

int grad_plan(const Dims &d, const wave_grid *g, const Plan &fwd, const Stencil &st, const float *cB,
              const float *cC, const float *cE, float *const U[4], float *store, int store_rows, float *G,
              int *status, const PointTable &src, const float *src_traces, int nsrc, const PointTable &rec,
              const float *rec_resid, int nrec, const HostTable *hsrc, const HostTable *hrec, int *order,
              long long order_cap, cudaStream_t stream, Plan *rout, Plan *aout)
{
    const int R = g->space_order / 2;
    int dev = 0;
    cudaGetDevice(&dev);
    Plan p0;  // the untiled default of sweep.cuh: its own mode variants
    p0.v = find_variant(R, 1, 0, 0, 0, 1);
    if (p0.v == nullptr) return WAVE_EUNSUPPORTED;
    p0.chunk = default_chunk(d, p0.v);
    std::vector<Plan> cands[2];  // [0] recompute (mode 1), [1] adjoint (mode 2)
    for (int k = 0; k < 2; ++k) {
        cands[k].push_back(p0);
        if (fwd.v->kind != 1) continue;
        const SweepVariant *vs = nullptr;
        const int nv = mode_variants_for(R, &vs);
        for (int i = 0; i < nv; ++i) {
            const SweepVariant *v = &vs[i];
            if (v->kind != 1 || v->XB != k + 1 || (v->T != 1 && v->T != fwd.v->T)) continue;
            Plan p;
            p.v = v;  // a mode variant runs itself in its own mode (mode_variant)
            p.chunk = fwd.chunk_given ? fwd.chunk : default_chunk(d, v);
            p.chunk_given = fwd.chunk_given;
            cands[k].push_back(p);
            // and half the x-chunk: twice the blocks, so that blocks that
            // inject on every plane (a receiver line along x) run first and
            // overlap a later wave instead of setting the step time
            const int half = p.chunk / 2;
            if (!fwd.chunk_given && half >= 4 * v->R * v->T && half >= 16) {
                p.chunk = half;
                p.chunk_given = true;
                cands[k].push_back(p);
            }
        }
    }
    // test hook: WAVE_GRAD_PIN="i,j" runs recompute candidate i and adjoint
    // candidate j of the lists above, untimed and uncached
    if (const char *pin = std::getenv("WAVE_GRAD_PIN")) {
        int i = -1, j = -1;
        if (std::sscanf(pin, "%d,%d", &i, &j) != 2 || i < 0 || j < 0 || i >= (int)cands[0].size() ||
            j >= (int)cands[1].size())
            return WAVE_EUNSUPPORTED;
        *rout = cands[0][i];
        *aout = cands[1][j];
        return WAVE_OK;
    }
    const GradKey key{d.nx, d.ny, d.nz, g->space_order, dev, nsrc, nrec, store_rows, fwd.v};
    {
        std::lock_guard<std::mutex> lk(g_grad_mu);
        auto it = g_grad_cache.find(key);
        if (it != g_grad_cache.end()) {
            *rout = it->second.first;
            *aout = it->second.second;
            return WAVE_OK;
        }
    }
    Plan best[2] = {cands[0][0], cands[1][0]};
    if (cands[0].size() > 1 || cands[1].size() > 1) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best_ms[2] = {1e30f, 1e30f};
        int rc = WAVE_OK;
        const int steps = std::min(16, store_rows);  // rows of the second-difference store
        for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(U[k], 0, sizeof(float) * d.npad, stream));
        CK(cudaMemsetAsync(store, 0, sizeof(float) * d.npad * (size_t)steps, stream));
        // recompute (second differences into store rows 0..steps-1) and
        // adjoint (imaging condition from those rows into G), on zero fields,
        // each candidate run twice back to back and its second run timed
        Job rj;
        rj.d = d;
        rj.st = st;
        rj.cB = cB;
        rj.cC = cC;
        rj.cE = cE;
        rj.status = status;
        rj.dstore = store;
        rj.inj = src;
        rj.q = src_traces;
        rj.nq = nsrc;
        Job aj = rj;
        aj.dstore = nullptr;
        aj.cE = nullptr;
        aj.inj = rec;
        aj.q = rec_resid;
        aj.nq = nrec;
        aj.q_base = steps - 1;
        aj.q_dir = -1;
        aj.dload = store;
        aj.l_rows = store_rows;
        aj.l_base = steps - 1;
        aj.l_dir = -1;
        aj.gacc = G;
        // the heavy-first launch order of the call's own sweeps
        rj.hinj = hsrc;
        aj.hinj = hrec;
        rj.order = aj.order = order;
        rj.order_cap = aj.order_cap = order_cap;
        for (int k = 0; k < 2 && rc == WAVE_OK; ++k) {
            for (const Plan &p : cands[k]) {
                // an untimed run (which also uploads the candidate's launch
                // order), then the timed one
                OrderCache oc;
                Job j = k == 0 ? rj : aj;
                j.ocache = &oc;
                float ms = 0.f;
                for (int pass = 0; pass < 2 && rc == WAVE_OK; ++pass) {
                    State s;
                    for (int i = 0; i < 4; ++i) s.buf[i] = U[i];
                    if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = WAVE_ECUDA; break; }
                    if ((rc = run_steps(j, s, steps, p, stream))) break;
                    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = WAVE_ECUDA;
                        break;
                    }
                }
                if (rc) break;
                if (ms < 0.99f * best_ms[k]) {  // ties keep the earlier candidate
                    best_ms[k] = ms;
                    best[k] = p;
                }
                if (tune_log())
                    std::fprintf(stderr,
                                 "wave gradient %s sweeps: kernel=%d T=%d tile=%dx%d rows=%d chunk=%d: %.4f ms for "
                                 "%d steps\n",
                                 k == 0 ? "recompute" : "adjoint", p.v->kind + 1, p.v->T, p.v->BZ, p.v->BY,
                                 rows_of(p.v), p.chunk, ms, steps);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_grad_mu);
    g_grad_cache[key] = std::make_pair(best[0], best[1]);
    *rout = best[0];
    *aout = best[1];
    return WAVE_OK;
}

int prep_model(const Dims &d, const wave_grid *g, const wave_tuning *t, const float *m,
               const float *damp, const Layout &L, cudaStream_t stream)
{
    const bool allow = t && (t->flags & WAVE_ALLOW_UNSTABLE);
    double stot = 0.0;
    for (int a = 0; a < 3; ++a) stot += symbol_at_pi(g->space_order) / ((double)g->h[a] * g->h[a]);
    const float stab = allow ? 0.f : (float)((double)g->dt * g->dt * stot);
    CK(cudaMemsetAsync(L.status, 0, sizeof(int) * kStatusWords, stream));
    CK(wt::launch_prep(m, damp, d.nx, d.ny, d.nz, d.nzp, g->dt, stab, L.cB, L.cC, L.cE, L.status,
                       stream));
    return WAVE_OK;
}

int check_points(const wave_points *p, bool need_data_ptr, const void *data)
{
    if (p == nullptr) return WAVE_OK;
    if (p->npts < 0) return WAVE_EINVAL;
    if (p->npts > 0 && (p->xyz == nullptr || (need_data_ptr && data == nullptr))) return WAVE_EINVAL;
    return WAVE_OK;
}

int npts_of(const wave_points *p) { return p ? p->npts : 0; }

// ---------------------------------------------------------------------------
// Batched shots in lockstep: one launch of the batched kernel per time step
// advances every shot of a group
// ---------------------------------------------------------------------------

const wt::MultiVariant *multi_variant(int R)
{
    const wt::MultiVariant *mv = nullptr;
    switch (R) {
    case 1: wt::sweep_multi_variant_r1(&mv); break;
    case 2: wt::sweep_multi_variant_r2(&mv); break;
    case 3: wt::sweep_multi_variant_r3(&mv); break;
    case 4: wt::sweep_multi_variant_r4(&mv); break;
    case 5: wt::sweep_multi_variant_r5(&mv); break;
    case 6: wt::sweep_multi_variant_r6(&mv); break;
    case 7: wt::sweep_multi_variant_r7(&mv); break;
    case 8: wt::sweep_multi_variant_r8(&mv); break;
    default: break;
    }
    return mv;
}

int tmulti_variants(int R, const wt::TMultiVariant **out)
{
    switch (R) {
    case 1: return wt::sweep_tmulti_variants_r1(out);
    case 2: return wt::sweep_tmulti_variants_r2(out);
    case 3: return wt::sweep_tmulti_variants_r3(out);
    case 4: return wt::sweep_tmulti_variants_r4(out);
    case 5: return wt::sweep_tmulti_variants_r5(out);
    case 6: return wt::sweep_tmulti_variants_r6(out);
    case 7: return wt::sweep_tmulti_variants_r7(out);
    case 8: return wt::sweep_tmulti_variants_r8(out);
    default: *out = nullptr; return 0;
    }
}

// The single-shot variant (kind 1) of a batched stage-specialised variant's
// shape and mode: its geometry and launch arguments.
const SweepVariant *tmulti_shape(const wt::TMultiVariant *tm)
{
    if (tm->mode == 0) return find_variant(tm->R, tm->T, tm->BY, tm->V, tm->BZ, 2, tm->VY);
    const SweepVariant *vs = nullptr;
    const int nv = mode_variants_for(tm->R, &vs);
    for (int i = 0; i < nv; ++i)
        if (vs[i].kind == 1 && vs[i].XB == tm->mode && vs[i].T == tm->T && vs[i].BY == tm->BY &&
            vs[i].BZ == tm->BZ && vs[i].V == tm->V && rows_of(&vs[i]) == tm->VY)
            return &vs[i];
    return nullptr;
}

// The kernel of a lockstep phase: the batched kernel of sweep.cuh (tm ==
// nullptr) or a batched stage-specialised variant tm with its single-shot
// shape tv.  `map` names the block map it launches with: 0 that of sweep.cuh's
// kernel, 1 the forward phases' stage-specialised shape, 2 the gradient
// phases' one.
struct LockKernel {
    const wt::TMultiVariant *tm = nullptr;
    const SweepVariant *tv = nullptr;
    int map = 0;
    int T() const { return tm != nullptr ? tm->T : 1; }
};

// The gradient phases' kernels: recompute (mode 1) and adjoint with the
// imaging condition (mode 2), of one shape.
struct LockGrad {
    LockKernel rec, adj;
};

constexpr int kLockMaps = 3;

struct LockShot {
    Dims d;
    wave_grid g;
    Layout L;
    HostTable ti, tr;
    Job job;        // job of the current phase
    State s;        // forward / recompute state
    State adj;      // adjoint state (gradient)
    int chunk[kLockMaps] = {0, 0, 0};            // x-chunk of each block map's kernel
    long long nblocks[kLockMaps] = {0, 0, 0};    // its blocks per launch
};

// Bytes of one phase's per-shot records (either batched kernel's form).
size_t lock_row_bytes(int nshots)
{
    return align_up(std::max(sizeof(wt::ShotSweep), sizeof(wt::ShotTSweep)) * (size_t)nshots);
}

// An upper bound on the blocks one launch of any batched kernel gives the
// group: every variant has BZ >= 24, BY >= 8 and an x-chunk of at least one
// plane.
long long lock_block_bound(int n, const wave_shot *shots)
{
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        const long long nzp = (shots[i].n[2] + 7) / 8 * 8;
        total += ((nzp + 23) / 24) * ((shots[i].n[1] + 7) / 8) * (long long)shots[i].n[0];
    }
    return total;
}

// Table of a lockstep group: three block maps (launch block -> (shot, tile)),
// each with room for `bound` blocks, then one row of per-shot records per
// phase.
size_t lock_map_bytes(long long bound) { return align_up(sizeof(int2) * (size_t)bound); }

size_t lock_table_bytes(int nshots, long long bound, int nphases)
{
    return kLockMaps * lock_map_bytes(bound) + (size_t)nphases * lock_row_bytes(nshots);
}

int lock_phases(int nt, int ckpt_every)
{
    return ckpt_every > 0 ? 1 + 2 * ((nt + ckpt_every - 1) / ckpt_every) : 1;
}

// Held while a host thread captures on the library's capture stream: the
// stream is shared by every thread of the process.
std::mutex g_capture_mu;

// The library's stream for capturing lockstep graphs on the current device.
int capture_stream(cudaStream_t *out)
{
    constexpr int kMaxDev = 64;
    static cudaStream_t streams[kMaxDev] = {};
    static std::mutex mu;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return WAVE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (streams[dev] == nullptr) CK(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    *out = streams[dev];
    return WAVE_OK;
}

struct LockTable {
    std::vector<char> rows;                  // one row of per-shot records per phase, row_bytes each
    std::vector<int2> map[kLockMaps];        // launch block -> (shot, tile), per kernel shape
    int2 *dev_map[kLockMaps] = {nullptr, nullptr, nullptr};
    char *dev_rows = nullptr;
    size_t row_bytes = 0;
    int nphases = 0;
};

// Checkpoint copies of every shot at local step j of a phase of depth T.
template <class StateOf>
int lock_ckpt(std::vector<LockShot> &ls, StateOf st_of, int j, int T, float *const *ckpts, int ckpt_every,
              cudaStream_t stream)
{
    for (size_t i = 0; i < ls.size(); ++i) {
        State sj = st_of((int)i);
        if ((j / T) & 1) advance_state(sj, T);
        float *dst = ckpts[i] + (size_t)(j / ckpt_every) * 2 * ls[i].d.npad;
        CK(cudaMemcpyAsync(dst, sj.buf[sj.a], sizeof(float) * ls[i].d.npad, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(dst + ls[i].d.npad, sj.buf[sj.b], sizeof(float) * ls[i].d.npad,
                           cudaMemcpyDeviceToDevice, stream));
    }
    return WAVE_OK;
}

// Enqueue `nsteps` steps of every shot on `stream`: shot i advances its state
// `st_of(i)` with job `ls[i].job` from local step 0, one launch of kernel k
// per T steps (nsteps and ckpt_every are multiples of T).  At every multiple
// of ckpt_every (ckpts != nullptr) its state (u^n, u^{n-1}) is copied to
// ckpts[i] first, as run_steps does.  The per-shot arguments of both buffer
// parities become the next phase row of `tab`.
template <class StateOf>
int lock_phase(std::vector<LockShot> &ls, StateOf st_of, int nsteps, const wt::MultiVariant *mv,
               const SweepVariant *v, const LockKernel &k, const Stencil &st, LockTable &tab,
               float *const *ckpts, int ckpt_every, cudaStream_t stream)
{
    const int n = (int)ls.size();
    const int ph = tab.nphases++;
    const bool staged = k.tm != nullptr;
    const int T = k.T();
    const int mp = staged ? k.map : 0;
    const size_t r0 = tab.rows.size();
    tab.rows.resize(r0 + tab.row_bytes, 0);
    int max_chunk_all = 0;
    for (int i = 0; i < n; ++i) {
        for (int p = 0; p < 2; ++p) {
            State sp = st_of(i);
            if (p == 1) advance_state(sp, T);
            long long nb = 0;
            int rc;
            if (staged) {
                wt::ShotTSweep *row = reinterpret_cast<wt::ShotTSweep *>(tab.rows.data() + r0) + i;
                wt::SweepMaps unused;
                rc = build_launch(ls[i].job, sp, 0, k.tv, ls[i].chunk[mp], &row->a[p], &unused, &row->mp[p], &nb);
            } else {
                wt::ShotSweep *row = reinterpret_cast<wt::ShotSweep *>(tab.rows.data() + r0) + i;
                wt::TMaps unused;
                rc = build_launch(ls[i].job, sp, 0, v, ls[i].chunk[mp], &row->a[p], &row->mp[p], &unused, &nb);
            }
            if (!rc && nb != ls[i].nblocks[mp]) rc = WAVE_EINVAL;
            if (rc) return rc;
        }
        max_chunk_all = std::max(max_chunk_all, ls[i].chunk[mp]);
    }
    const char *drow = tab.dev_rows + (size_t)ph * tab.row_bytes;
    const size_t smem = (staged ? k.tm->smem : mv->smem) +
                        wt::sweep_table_bytes(max_chunk_all, staged ? k.tm->R * T : mv->R * mv->T) + 16;
    for (int j = 0; j < nsteps; j += T) {
        if (ckpts != nullptr && j % ckpt_every == 0) {
            const int rc = lock_ckpt(ls, st_of, j, T, ckpts, ckpt_every, stream);
            if (rc) return rc;
        }
        if (staged)
            CK(k.tm->launch((int)tab.map[mp].size(), smem, stream, (const wt::ShotTSweep *)drow, tab.dev_map[mp],
                            st, (j / T) & 1, j));
        else
            CK(mv->launch((int)tab.map[0].size(), smem, stream, (const wt::ShotSweep *)drow, tab.dev_map[0], st,
                          j & 1, j));
    }
    if ((nsteps / T) & 1)
        for (int i = 0; i < n; ++i) advance_state(st_of(i), T);
    return WAVE_OK;
}

// Ends a stream capture however the enqueueing went; owns the graph.
struct Capture {
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    bool open = false;
    int begin(cudaStream_t st)
    {
        s = st;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        open = true;
        return WAVE_OK;
    }
    int end()
    {
        open = false;
        CK(cudaStreamEndCapture(s, &graph));
        return graph != nullptr ? WAVE_OK : WAVE_ECUDA;
    }
    ~Capture()
    {
        if (open) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g != nullptr) cudaGraphDestroy(g);
            cudaGetLastError();  // the failed capture's error is reported through the return code
        }
        if (graph != nullptr) cudaGraphDestroy(graph);
    }
};

// The forward job of shot x from step 0: sources, and receivers recorded
// unless the group computes a gradient.
void forward_job(LockShot &x, const wt::ShotSlot &slot, const Stencil &st, bool grad)
{
    Job &j = x.job;
    j = Job();
    j.d = x.d;
    j.st = st;
    j.cB = x.L.cB;
    j.cC = x.L.cC;
    j.status = x.L.status;
    j.inj = x.L.inj.view();
    j.q = slot.q;
    j.nq = slot.shot->src.npts;
    if (!grad) {
        j.rec = x.L.rec.view();
        j.corner = x.L.corner;
        j.nslot = 8 * slot.shot->rec.npts;
    }
}

// The recompute job of shot x over the segment from step s0: second
// differences into store rows 0.. (as wave_grad).
void recompute_job(LockShot &x, const wt::ShotSlot &slot, const Stencil &st, int s0)
{
    Job &rj = x.job;
    rj = Job();
    rj.d = x.d;
    rj.st = st;
    rj.cB = x.L.cB;
    rj.cC = x.L.cC;
    rj.status = x.L.status;
    rj.cE = x.L.cE;
    rj.inj = x.L.inj.view();
    rj.q = slot.q;
    rj.nq = slot.shot->src.npts;
    rj.q_base = s0;
    rj.q_dir = 1;
    rj.dstore = x.L.store;
    rj.d_base = 0;
    rj.d_dir = 1;
}

// The adjoint job of shot x over the segment [s0, s0 + len), newest step
// first, with the imaging condition from store rows len-1 .. 0 (as wave_grad).
void adjoint_job(LockShot &x, const wt::ShotSlot &slot, const Stencil &st, int s0, int len, int rows)
{
    Job &aj = x.job;
    aj = Job();
    aj.d = x.d;
    aj.st = st;
    aj.cB = x.L.cB;
    aj.cC = x.L.cC;
    aj.status = x.L.status;
    aj.inj = x.L.inj2.view();
    aj.q = slot.resid;
    aj.nq = slot.shot->rec.npts;
    aj.q_base = s0 + len - 1;
    aj.q_dir = -1;
    aj.dload = x.L.store;
    aj.l_rows = rows;
    aj.l_base = len - 1;
    aj.l_dir = -1;
    aj.gacc = x.L.G;
}

// The gradient's time loops of a lockstep group on `stream`: forward with
// checkpoints (kernel fw), then per segment (last first) the recompute with
// stored second differences and the adjoint with the imaging condition
// (kernels gr), as wave_grad does for one shot; window gradients (scaled by
// -1/dt^2) into slots[i].gwin.
int lock_grad(std::vector<LockShot> &ls, const wt::ShotSlot *slots, int ckpt_every, const wt::MultiVariant *mv,
              const SweepVariant *v, const LockKernel &fw, const LockGrad &gr, const Stencil &st, LockTable &tab,
              cudaStream_t stream, float dt)
{
    const int n = (int)ls.size();
    const int nt = ls[0].g.nt;
    const int rows = std::max(1, std::min(ckpt_every, nt));
    auto fwd_state = [&](int i) -> State & { return ls[i].s; };
    auto adj_state = [&](int i) -> State & { return ls[i].adj; };
    std::vector<float *> ck(n);
    for (int i = 0; i < n; ++i) ck[i] = slots[i].ckpt;
    int rc = lock_phase(ls, fwd_state, nt, mv, v, fw, st, tab, ck.data(), ckpt_every, stream);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        LockShot &x = ls[i];
        CK(cudaMemsetAsync(x.L.G, 0, sizeof(float) * x.d.npad, stream));
        for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(x.L.V[k], 0, sizeof(float) * x.d.npad, stream));
        x.adj = State();
        for (int k = 0; k < 4; ++k) x.adj.buf[k] = x.L.V[k];
    }
    const int nseg = (nt + ckpt_every - 1) / ckpt_every;
    for (int c = nseg - 1; c >= 0; --c) {
        const int s0 = c * ckpt_every;
        const int len = std::min(ckpt_every, nt - s0);
        for (int i = 0; i < n; ++i) {
            LockShot &x = ls[i];
            const float *cp = slots[i].ckpt + (size_t)c * 2 * x.d.npad;
            x.s = State();
            for (int k = 0; k < 4; ++k) x.s.buf[k] = x.L.U[k];
            CK(cudaMemcpyAsync(x.s.buf[0], cp, sizeof(float) * x.d.npad, cudaMemcpyDeviceToDevice, stream));
            CK(cudaMemcpyAsync(x.s.buf[1], cp + x.d.npad, sizeof(float) * x.d.npad, cudaMemcpyDeviceToDevice,
                               stream));
            recompute_job(x, slots[i], st, s0);
        }
        if ((rc = lock_phase(ls, fwd_state, len, mv, v, gr.rec, st, tab, nullptr, 0, stream))) return rc;
        for (int i = 0; i < n; ++i) adjoint_job(ls[i], slots[i], st, s0, len, rows);
        if ((rc = lock_phase(ls, adj_state, len, mv, v, gr.adj, st, tab, nullptr, 0, stream))) return rc;
    }
    const float scale = (float)(-1.0 / ((double)dt * (double)dt));
    for (int i = 0; i < n; ++i)
        CK(wt::launch_unpad(ls[i].L.G, ls[i].d.nx, ls[i].d.ny, ls[i].d.nz, ls[i].d.nzp, scale, slots[i].gwin,
                            stream));
    return WAVE_OK;
}

// Whether the batched stage-specialised variant tm (of depth T) can run a
// group's phases: T must divide nt and the checkpoint interval, so that every
// phase (forward, and each segment's recompute and adjoint) is a whole
// number of launches.
bool tmulti_fits(const wt::TMultiVariant *tm, int nt, int ckpt_every)
{
    return tm != nullptr && tmulti_shape(tm) != nullptr && nt % tm->T == 0 &&
           (ckpt_every <= 0 || ckpt_every % tm->T == 0);
}

// The forward-mode batched stage-specialised variant a tuning names (kernel
// 2, depth time_tile, tile_y / tile_z / rows / vec if given), or nullptr.
const wt::TMultiVariant *tmulti_named(int R, const wave_tuning *t)
{
    const wt::TMultiVariant *tms = nullptr;
    const int nv = tmulti_variants(R, &tms);
    for (int i = 0; i < nv; ++i)
        if (tms[i].mode == 0 && tms[i].T == t->time_tile && (t->tile_y == 0 || tms[i].BY == t->tile_y) &&
            (t->tile_z == 0 || tms[i].BZ == t->tile_z) && (t->rows == 0 || tms[i].VY == t->rows) &&
            (t->vec == 0 || tms[i].V == t->vec))
            return &tms[i];
    return nullptr;
}

// The mode-2 partner (same shape) of the mode-1 batched variant tms[i1], or -1.
int tmulti_partner(const wt::TMultiVariant *tms, int ntm, int i1)
{
    for (int i = 0; i < ntm; ++i)
        if (tms[i].mode == 2 && tms[i].T == tms[i1].T && tms[i].BZ == tms[i1].BZ && tms[i].BY == tms[i1].BY &&
            tms[i].V == tms[i1].V && tms[i].VY == tms[i1].VY)
            return i;
    return -1;
}

// The gradient kernels of choice c: -1 sweep.cuh's batched kernel, else the
// mode-1 batched variant tms[c] and its mode-2 partner (map 2).
LockGrad lock_grad_kernels(const wt::TMultiVariant *tms, int ntm, int c)
{
    LockGrad g;
    if (c < 0) return g;
    const int c2 = tmulti_partner(tms, ntm, c);
    if (c2 < 0) return g;
    g.rec.tm = &tms[c];
    g.rec.tv = tmulti_shape(g.rec.tm);
    g.rec.map = 2;
    g.adj.tm = &tms[c2];
    g.adj.tv = tmulti_shape(g.adj.tm);
    g.adj.map = 2;
    if (g.rec.tv == nullptr || g.adj.tv == nullptr) return LockGrad();
    return g;
}

// Kernel choices of autotuned survey groups, per (device, order, group shape,
// nt, checkpoint interval): forward (index into the radius's batched
// stage-specialised variants, or -1 for sweep.cuh's batched kernel) and
// gradient phases (the mode-1 variant, or -1).
struct LockKey {
    int dev, so, n;
    long long pts;
    int mx, my, mz, nt, ck;
    bool operator<(const LockKey &o) const
    {
        return std::tie(dev, so, n, pts, mx, my, mz, nt, ck) <
               std::tie(o.dev, o.so, o.n, o.pts, o.mx, o.my, o.mz, o.nt, o.ck);
    }
};
std::mutex g_lock_mu;
std::map<LockKey, std::pair<int, int>> g_lock_cache;

// The key of a group of n shots of grid G (their windows' extents).
int lock_key(const wave_grid *G, int n, const wave_shot *shots, int ckpt_every, LockKey *key)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    *key = LockKey{dev, G->space_order, n, 0, 0, 0, 0, G->nt, ckpt_every};
    for (int i = 0; i < n; ++i) {
        wave_grid g = *G;
        for (int a = 0; a < 3; ++a) g.n[a] = shots[i].n[a];
        Dims d;
        const int rc = check_grid(&g, &d);
        if (rc) return rc;
        key->pts += d.npad;
        key->mx = std::max(key->mx, d.nx);
        key->my = std::max(key->my, d.ny);
        key->mz = std::max(key->mz, d.nz);
    }
    return WAVE_OK;
}

}  // namespace

namespace wt {

int lockstep_group(const wave_grid *G, int n, const ShotSlot *slots, int ckpt_every,
                   const wave_tuning *tuning, void *table, size_t table_bytes, cudaStream_t stream)
{
    try {
        const int R = G->space_order / 2;
        const MultiVariant *mv = multi_variant(R);
        if (mv == nullptr || tuning == nullptr) return WAVE_EUNSUPPORTED;
        // the batched kernel of sweep.cuh runs its default untiled shape
        const SweepVariant *v = find_variant(R, 1, mv->BY, mv->V, mv->BZ, 1);
        if (v == nullptr || v->P != mv->P) return WAVE_EUNSUPPORTED;
        const bool grad = ckpt_every > 0;
        const int nt = G->nt;
        const int rows = grad ? std::max(1, std::min(ckpt_every, nt)) : 0;
        const wt::TMultiVariant *tms = nullptr;
        const int ntm = tmulti_variants(R, &tms);
        // kernels: named by the tuning, or timed below (time_tile 0)
        LockKernel fw;
        LockGrad gr;
        const bool tune = tuning->time_tile == 0;
        if (!tune && tuning->kernel == 2) {
            fw.tm = tmulti_named(R, tuning);
            if (!tmulti_fits(fw.tm, nt, ckpt_every)) return WAVE_EUNSUPPORTED;
            fw.tv = tmulti_shape(fw.tm);
            fw.map = 1;
            // the gradient phases on the first mode shape of the same depth
            for (int c = 0; c < ntm && grad && gr.rec.tm == nullptr; ++c)
                if (tms[c].mode == 1 && tms[c].T == fw.tm->T && tmulti_fits(&tms[c], nt, ckpt_every))
                    gr = lock_grad_kernels(tms, ntm, c);
        } else if (!tune && (tuning->time_tile != 1 || (tuning->tile_y && tuning->tile_y != v->BY) ||
                             (tuning->vec && tuning->vec != v->V) || (tuning->tile_z && tuning->tile_z != v->BZ))) {
            return WAVE_EUNSUPPORTED;
        }
        std::vector<LockShot> ls(n);
        Stencil st;
        // per-shot setup on `stream`: model coefficients, zero levels, point tables
        for (int i = 0; i < n; ++i) {
            LockShot &x = ls[i];
            const wave_shot &sh = *slots[i].shot;
            x.g = *G;
            for (int a = 0; a < 3; ++a) x.g.n[a] = sh.n[a];
            int rc = check_grid(&x.g, &x.d);
            if (rc) return rc;
            const int ns = sh.src.npts, nr = sh.rec.npts;
            x.L = carve(slots[i].ws, slots[i].ws_bytes, false, x.d, grad ? WAVE_OP_GRAD : WAVE_OP_FWD, ns, nr, nt,
                        grad ? ckpt_every : 0);
            if (x.L.bytes > slots[i].ws_bytes) return WAVE_ENOSPACE;
            if (build_table(x.d, x.g.h, &sh.src, false, &x.ti) ||
                build_table(x.d, x.g.h, &sh.rec, !grad, &x.tr))
                return WAVE_EINVAL;
            st = make_stencil(&x.g);
            if ((rc = prep_model(x.d, &x.g, tuning, slots[i].mw, slots[i].dw, x.L, stream))) return rc;
            for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(x.L.U[k], 0, sizeof(float) * x.d.npad, stream));
            if ((rc = upload_table(x.ti, x.L.inj, stream))) return rc;
            if ((rc = upload_table(x.tr, grad ? x.L.inj2 : x.L.rec, stream))) return rc;
            if ((rc = sum_table(x.ti, x.L.inj, slots[i].q, ns, nt, stream))) return rc;
            if (grad && (rc = sum_table(x.tr, x.L.inj2, slots[i].resid, nr, nt, stream))) return rc;
            for (int k = 0; k < 4; ++k) x.s.buf[k] = x.L.U[k];
            forward_job(x, slots[i], st, grad);
        }
        CK(wt::allow_max_dynamic_smem(mv->func));
        const int nphases = lock_phases(nt, ckpt_every);
        std::vector<wave_shot> gs(n);
        for (int i = 0; i < n; ++i) gs[i] = *slots[i].shot;
        const long long bound = lock_block_bound(n, gs.data());
        if (bound > 0x7fffffffLL || lock_table_bytes(n, bound, nphases) > table_bytes) return WAVE_ENOSPACE;
        LockTable tab;
        tab.row_bytes = lock_row_bytes(n);
        for (int k = 0; k < kLockMaps; ++k) tab.dev_map[k] = (int2 *)((char *)table + k * lock_map_bytes(bound));
        tab.dev_rows = (char *)table + kLockMaps * lock_map_bytes(bound);

        // x-chunks and the block map of a kernel: the tiles of every shot that
        // handle a source or receiver point (in any phase) first, then the rest
        auto set_map = [&](const LockKernel &k) -> int {
            const int mp = k.tm != nullptr ? k.map : 0;
            const SweepVariant *sv = k.tm != nullptr ? k.tv : v;
            std::vector<std::vector<char>> heavy(n);
            long long tot = 0;
            for (int i = 0; i < n; ++i) {
                LockShot &x = ls[i];
                const bool own_chunk = tuning->tile_x > 0 && !tune && (mp == 0 ? fw.tm == nullptr : mp == 1);
                x.chunk[mp] = std::min(own_chunk ? std::min(tuning->tile_x, x.d.nx) : default_chunk(x.d, sv),
                                       max_chunk(sv));
                x.nblocks[mp] = (long long)tiles(x.d.nzp, sv->BZ) * tiles(x.d.ny, sv->BY) * tiles(x.d.nx, x.chunk[mp]);
                tot += x.nblocks[mp];
                mark_heavy(x.d, sv, x.chunk[mp], &x.ti, false, heavy[i]);
                mark_heavy(x.d, sv, x.chunk[mp], &x.tr, !grad, heavy[i]);
                heavy[i].resize((size_t)x.nblocks[mp], 0);
            }
            if (tot > bound) return WAVE_ENOSPACE;
            std::vector<int2> &out = tab.map[mp];
            out.clear();
            for (int pass = 1; pass >= 0; --pass)
                for (int i = 0; i < n; ++i)
                    for (long long t = 0; t < ls[i].nblocks[mp]; ++t)
                        if (heavy[i][(size_t)t] == pass) out.push_back(make_int2(i, (int)t));
            if (k.tm != nullptr) CK(wt::allow_max_dynamic_smem(k.tm->func));
            return WAVE_OK;
        };
        auto upload_map = [&](int mp) -> int {
            CK(cudaMemcpyAsync(tab.dev_map[mp], tab.map[mp].data(), sizeof(int2) * tab.map[mp].size(),
                               cudaMemcpyHostToDevice, stream));
            return WAVE_OK;
        };
        int rc = set_map(LockKernel());
        if (rc) return rc;

        if (tune) {
            // Time the group's own shots on every candidate kernel, a few steps
            // from zeroed levels, best of two passes, per step; ties keep the
            // earlier (sweep.cuh's batched kernel first).  The forward phases
            // and, for the gradient, the recompute + adjoint phases are timed
            // separately; the choice is cached per group shape.
            LockKey key;
            if ((rc = lock_key(G, n, gs.data(), ckpt_every, &key))) return rc;
            std::pair<int, int> choice(-2, -2);
            {
                std::lock_guard<std::mutex> lk(g_lock_mu);
                auto it = g_lock_cache.find(key);
                if (it != g_lock_cache.end()) choice = it->second;
            }
            if (choice.first == -2) {
                cudaEvent_t e0, e1;
                CK(cudaEventCreate(&e0));
                CK(cudaEventCreate(&e1));
                auto st_fwd = [&](int i) -> State & { return ls[i].s; };
                auto st_adj = [&](int i) -> State & { return ls[i].adj; };
                // run `fn` (which enqueues launches) between events: ms, or < 0 on failure
                auto timed = [&](auto fn) -> float {
                    float ms = -1.f;
                    if (cudaEventRecord(e0, stream) != cudaSuccess) return -1.f;
                    if (fn() != WAVE_OK) return -1.f;
                    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                        return -1.f;
                    return ms;
                };
                // a phase's rows built on the host and uploaded before its launches
                auto run_phase = [&](auto st_of, int steps, const LockKernel &k) -> int {
                    LockTable tt;
                    tt.row_bytes = tab.row_bytes;
                    for (int m = 0; m < kLockMaps; ++m) {
                        tt.map[m] = tab.map[m];
                        tt.dev_map[m] = tab.dev_map[m];
                    }
                    tt.dev_rows = tab.dev_rows;
                    int r = lock_phase(ls, st_of, 0, mv, v, k, st, tt, nullptr, 0, stream);  // the row only
                    if (r) return r;
                    CK(cudaMemcpyAsync(tt.dev_rows, tt.rows.data(), tt.row_bytes, cudaMemcpyHostToDevice, stream));
                    tt.rows.clear();
                    tt.nphases = 0;
                    return lock_phase(ls, st_of, steps, mv, v, k, st, tt, nullptr, 0, stream);
                };
                int best_f = -1, best_g = -1;
                float tbest_f = 1e30f, tbest_g = 1e30f;
                std::vector<int> cf = {-1};
                for (int c = 0; c < ntm; ++c)
                    if (tms[c].mode == 0 && tmulti_fits(&tms[c], nt, ckpt_every)) cf.push_back(c);
                std::vector<int> cg = {-1};
                for (int c = 0; c < ntm && grad; ++c)
                    if (tms[c].mode == 1 && tmulti_fits(&tms[c], nt, ckpt_every) &&
                        lock_grad_kernels(tms, ntm, c).rec.tm != nullptr)
                        cg.push_back(c);
                for (int pass = 0; pass < 2 && rc == WAVE_OK; ++pass) {
                    for (size_t ci = 0; ci < cf.size() && rc == WAVE_OK; ++ci) {
                        LockKernel k;
                        if (cf[ci] >= 0) {
                            k.tm = &tms[cf[ci]];
                            k.tv = tmulti_shape(k.tm);
                            k.map = 1;
                            if ((rc = set_map(k)) || (rc = upload_map(1))) break;
                        } else if ((rc = upload_map(0))) {
                            break;
                        }
                        const int steps = std::min(8, nt);  // a multiple of every candidate's depth
                        for (int i = 0; i < n; ++i) forward_job(ls[i], slots[i], st, grad);
                        const float ms = timed([&] { return run_phase(st_fwd, steps, k); });
                        if (ms < 0.f) { rc = WAVE_ECUDA; break; }
                        if (tune_log() && pass == 1)
                            std::fprintf(stderr, "wave survey group: forward kernel=%d T=%d: %.4f ms for %d steps\n",
                                         k.tm ? 2 : 1, k.T(), ms, steps);
                        if (pass == 1 && ms / steps < 0.99f * tbest_f) {
                            tbest_f = ms / steps;
                            best_f = cf[ci];
                        }
                    }
                    for (size_t ci = 0; ci < cg.size() && rc == WAVE_OK && grad; ++ci) {
                        const LockGrad g = lock_grad_kernels(tms, ntm, cg[ci]);
                        const int T = g.rec.T();
                        const int steps = std::min(8, rows) / T * T;
                        if (steps < 1) continue;
                        if (g.rec.tm != nullptr) {
                            if ((rc = set_map(g.rec)) || (rc = upload_map(2))) break;
                        } else if ((rc = upload_map(0))) {
                            break;
                        }
                        for (int i = 0; i < n; ++i) {
                            ls[i].adj = State();
                            for (int k = 0; k < 4; ++k) ls[i].adj.buf[k] = ls[i].L.V[k];
                        }
                        const float ms = timed([&] {
                            for (int i = 0; i < n; ++i) recompute_job(ls[i], slots[i], st, 0);
                            int r = run_phase(st_fwd, steps, g.rec);
                            if (r) return r;
                            for (int i = 0; i < n; ++i) adjoint_job(ls[i], slots[i], st, 0, steps, rows);
                            return run_phase(st_adj, steps, g.adj);
                        });
                        if (ms < 0.f) { rc = WAVE_ECUDA; break; }
                        if (tune_log() && pass == 1)
                            std::fprintf(stderr,
                                         "wave survey group: gradient kernel=%d T=%d: %.4f ms for %d + %d steps\n",
                                         g.rec.tm ? 2 : 1, T, ms, steps, steps);
                        if (pass == 1 && ms / steps < 0.99f * tbest_g) {
                            tbest_g = ms / steps;
                            best_g = cg[ci];
                        }
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (rc) return rc;
                choice = std::make_pair(best_f, best_g);
                std::lock_guard<std::mutex> lk(g_lock_mu);
                g_lock_cache[key] = choice;
            }
            if (choice.first >= 0) {
                fw.tm = &tms[choice.first];
                fw.tv = tmulti_shape(fw.tm);
                fw.map = 1;
            }
            if (grad && choice.second >= 0) gr = lock_grad_kernels(tms, ntm, choice.second);
            // the timed launches left the levels (and the adjoint's) dirty: start
            // from zero again, with the forward job of every shot
            for (int i = 0; i < n; ++i) {
                LockShot &x = ls[i];
                x.s = State();
                x.adj = State();
                for (int k = 0; k < 4; ++k) {
                    x.s.buf[k] = x.L.U[k];
                    CK(cudaMemsetAsync(x.L.U[k], 0, sizeof(float) * x.d.npad, stream));
                }
                forward_job(x, slots[i], st, grad);
            }
        }
        if (fw.tm != nullptr && (rc = set_map(fw))) return rc;
        if (gr.rec.tm != nullptr && (rc = set_map(gr.rec))) return rc;
        tab.rows.reserve((size_t)nphases * tab.row_bytes);

        // The time loops go into one CUDA graph, captured on the library's
        // stream and launched on `stream` after the tables are uploaded.
        cudaStream_t cs;
        if ((rc = capture_stream(&cs))) return rc;
        std::lock_guard<std::mutex> capture_lock(g_capture_mu);  // released after `cap` ends
        Capture cap;
        if ((rc = cap.begin(cs))) return rc;
        auto fwd_state = [&](int i) -> State & { return ls[i].s; };
        if (!grad) {
            rc = lock_phase(ls, fwd_state, nt, mv, v, fw, st, tab, nullptr, 0, cs);
            for (int i = 0; i < n && rc == WAVE_OK; ++i)
                if (slots[i].shot->rec.npts > 0 && slots[i].rec_out != nullptr &&
                    wt::launch_gather(ls[i].L.corner, ls[i].L.rec.wts, nt, slots[i].shot->rec.npts, 1,
                                      slots[i].rec_out, cs) != cudaSuccess)
                    rc = WAVE_ECUDA;
        } else {
            rc = lock_grad(ls, slots, ckpt_every, mv, v, fw, gr, st, tab, cs, G->dt);
        }
        if (rc) return rc;
        if ((rc = cap.end())) return rc;
        if (tab.nphases != nphases || tab.rows.size() != (size_t)nphases * tab.row_bytes) return WAVE_EINVAL;
        cudaGraphExec_t exec = nullptr;
        CK(cudaGraphInstantiate(&exec, cap.graph, 0));
        rc = WAVE_OK;
        for (int k = 0; k < kLockMaps && rc == WAVE_OK; ++k)
            if (!tab.map[k].empty() &&
                cudaMemcpyAsync(tab.dev_map[k], tab.map[k].data(), sizeof(int2) * tab.map[k].size(),
                                cudaMemcpyHostToDevice, stream) != cudaSuccess)
                rc = WAVE_ECUDA;
        if (rc == WAVE_OK && cudaMemcpyAsync(tab.dev_rows, tab.rows.data(), tab.rows.size(), cudaMemcpyHostToDevice,
                                             stream) != cudaSuccess)
            rc = WAVE_ECUDA;
        if (rc == WAVE_OK && cudaGraphLaunch(exec, stream) != cudaSuccess) rc = WAVE_ECUDA;
        cudaGraphExecDestroy(exec);  // freed once the launch completes
        return rc;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

bool lockstep_supported(const wave_grid *G, const wave_tuning *tuning, int ckpt_every)
{
    if (G == nullptr || tuning == nullptr) return false;
    const int R = G->space_order / 2;
    const MultiVariant *mv = multi_variant(R);
    if (mv == nullptr) return false;
    if (tuning->time_tile == 0) return true;  // the forward kernel is timed; sweep.cuh's always fits
    if (tuning->kernel == 2) return tmulti_fits(tmulti_named(R, tuning), G->nt, ckpt_every);
    const SweepVariant *v = find_variant(R, 1, tuning->tile_y, tuning->vec, tuning->tile_z, 1);
    return tuning->time_tile == 1 && v != nullptr && v->V == mv->V && v->BZ == mv->BZ && v->BY == mv->BY &&
           v->P == mv->P;
}

int lockstep_describe(const wave_grid *G, int n, const wave_shot *shots, int ckpt_every,
                      const wave_tuning *tuning, int32_t *out)
{
    const int R = G->space_order / 2;
    const MultiVariant *mv = multi_variant(R);
    for (int k = 0; k < 11; ++k) out[k] = 0;
    if (!lockstep_supported(G, tuning, ckpt_every)) return WAVE_OK;  // per-shot streams
    out[8] = 1;
    const wt::TMultiVariant *tms = nullptr;
    const int ntm = tmulti_variants(R, &tms);
    const wt::TMultiVariant *tm = nullptr;
    LockGrad gr;
    if (tuning->time_tile == 0) {
        LockKey key;
        const int rc = lock_key(G, n, shots, ckpt_every, &key);
        if (rc) return rc;
        std::lock_guard<std::mutex> lk(g_lock_mu);
        auto it = g_lock_cache.find(key);
        if (it == g_lock_cache.end()) return WAVE_OK;  // not timed yet: out[0] = 0
        if (it->second.first >= 0) tm = &tms[it->second.first];
        if (ckpt_every > 0 && it->second.second >= 0) gr = lock_grad_kernels(tms, ntm, it->second.second);
    } else if (tuning->kernel == 2) {
        tm = tmulti_named(R, tuning);
        for (int c = 0; c < ntm && ckpt_every > 0 && tm != nullptr && gr.rec.tm == nullptr; ++c)
            if (tms[c].mode == 1 && tms[c].T == tm->T && tmulti_fits(&tms[c], G->nt, ckpt_every))
                gr = lock_grad_kernels(tms, ntm, c);
    }
    if (tm != nullptr) {
        const int v[8] = {tm->T, tm->BY, 0, tm->BZ, tm->V, tm->P, WAVE_KERNEL_STAGED, tm->VY};
        for (int k = 0; k < 8; ++k) out[k] = v[k];
    } else {
        const int v[8] = {1, mv->BY, 0, mv->BZ, mv->V, mv->P, WAVE_KERNEL_SHARED, 1};
        for (int k = 0; k < 8; ++k) out[k] = v[k];
    }
    if (ckpt_every > 0) {
        out[9] = gr.rec.tm != nullptr ? WAVE_KERNEL_STAGED : WAVE_KERNEL_SHARED;
        out[10] = gr.rec.T();
    }
    return WAVE_OK;
}

size_t lockstep_table_bytes(const wave_grid *G, int n, const wave_shot *shots, int ckpt_every)
{
    return lock_table_bytes(n, lock_block_bound(n, shots), lock_phases(G->nt, ckpt_every));
}

cudaError_t allow_max_dynamic_smem(const void *func)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, func})) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    done[{dev, func}] = true;
    return cudaSuccess;
}

}  // namespace wt

// ===========================================================================
// C ABI
// ===========================================================================

namespace {

// ---------------------------------------------------------------------------
// Binomial checkpointing (revolve): A. Griewank, "Achieving logarithmic growth
// of temporal and spatial complexity in reverse automatic differentiation",
// Optim. Methods Softw. 1 (1992); A. Griewank and A. Walther, "Algorithm 799:
// revolve", ACM TOMS 26 (2000).  The paper uses uniform checkpoints; this
// schedule reverses nt steps with a fixed number of stored states and the
// fewest recomputed forward steps.
// ---------------------------------------------------------------------------

enum RevKind { REV_ADVANCE = 0, REV_TAKESHOT = 1, REV_RESTORE = 2, REV_YOUTURN = 3 };
// ADVANCE a b: forward from the current state (step a) to step b
// TAKESHOT a k: store the current state (step a) in slot k
// RESTORE a k: make the state of step a in slot k current (k = -1: the zero
//              initial state, step 0)
// YOUTURN a: from the current state (step a) one forward step that stores
//            D^a, then the adjoint step of time index a
struct RevAction {
    int kind, a, b;
};

// C(n, k) saturated at cap (the partial products C(n-k+i, i) grow with i).
long long binom_sat(long long n, long long k, long long cap)
{
    if (k < 0 || k > n) return 0;
    k = std::min(k, n - k);
    unsigned __int128 c = 1;
    for (long long i = 1; i <= k; ++i) {
        c = c * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
        if (c > (unsigned __int128)cap) return cap;
    }
    return (long long)c;
}

// Forward steps (besides the one of each reversed step) that reverse l steps
// from a held start state with s free slots: with c = s + 1 stored states
// and r the least integer with C(c + r, c) >= l, the minimum is
// r l - C(c + r, r - 1) (Griewank 1992); s = 0 recomputes from the start.
long long rev_cost(long long l, long long s)
{
    if (l <= 1) return 0;
    if (s == 0) return l * (l - 1) / 2;
    long long r = 0;
    while (binom_sat(s + 1 + r, s + 1, l) < l) ++r;
    return r * l - binom_sat(s + 1 + r, r - 1, (long long)1 << 60);
}

struct RevGen {
    int nslots;
    int cur = 0;  // step of the current state (-1: none); the run starts at the zero state
    std::vector<RevAction> out;

    void ensure(int a, int slot)
    {
        if (cur != a) {
            out.push_back({REV_RESTORE, a, slot});
            cur = a;
        }
    }
    // reverse steps [a, b) given the state of step a in `slot` (or current),
    // s slots free (slots nslots - s .. nslots - 1)
    void reverse(int a, int b, int s, int slot)
    {
        const int l = b - a;
        if (l <= 0) return;
        if (l == 1) {
            ensure(a, slot);
            out.push_back({REV_YOUTURN, a, 0});
            cur = a + 1;
            return;
        }
        if (s == 0) {
            for (int k = b - 1; k >= a; --k) {
                ensure(a, slot);
                if (k > a) out.push_back({REV_ADVANCE, a, k});
                out.push_back({REV_YOUTURN, k, 0});
                cur = k + 1;
            }
            return;
        }
        // first stored state at a + m: m + cost(m, s) + cost(l - m, s - 1)
        // is least; the smallest such m
        long long best = -1;
        int m = 1;
        for (int j = 1; j < l; ++j) {
            const long long c = j + rev_cost(j, s) + rev_cost(l - j, s - 1);
            if (best < 0 || c < best) {
                best = c;
                m = j;
            }
        }
        ensure(a, slot);
        out.push_back({REV_ADVANCE, a, a + m});
        const int k = nslots - s;
        out.push_back({REV_TAKESHOT, a + m, k});
        cur = a + m;
        reverse(a + m, b, s - 1, k);
        reverse(a, a + m, s, slot);
    }
};

std::vector<RevAction> revolve_schedule(int nt, int nslots)
{
    RevGen g;
    g.nslots = nslots;
    g.reverse(0, nt, nslots, -1);
    return g.out;
}

}  // namespace

extern "C" {

int32_t wave_version(void) { return 100; }

const char *wave_strerror(int32_t code)
{
    switch (code) {
    case WAVE_OK: return "ok";
    case WAVE_EINVAL: return "invalid argument";
    case WAVE_EUNSTABLE: return "dt above the stability limit";
    case WAVE_ECUDA: return "CUDA runtime error";
    case WAVE_ETIMEOUT: return "device wait timed out";
    case WAVE_ENOSPACE: return "workspace too small";
    case WAVE_EUNSUPPORTED: return "tiling not compiled into this library";
    default: return "unknown error";
    }
}

int32_t wave_fd_coefficients(int32_t space_order, double *c_out)
{
    if (space_order < 2 || space_order > 16 || space_order % 2 || c_out == nullptr) return WAVE_EINVAL;
    fd_coeffs(space_order, c_out);
    return WAVE_OK;
}

double wave_cfl_dt(int32_t space_order, const float *h, float v_max)
{
    if (space_order < 2 || space_order > 16 || space_order % 2 || h == nullptr || !(v_max > 0.f))
        return -1.0;
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!(h[a] > 0.f)) return -1.0;
        s += symbol_at_pi(space_order) / ((double)h[a] * h[a]);
    }
    return 2.0 / ((double)v_max * std::sqrt(s));
}

size_t wave_workspace_bytes(const wave_grid *g, int32_t op, int32_t nsrc, int32_t nrec,
                            int32_t ckpt_every, const wave_tuning *tuning)
{
    (void)tuning;
    Dims d;
    if (check_grid(g, &d) || nsrc < 0 || nrec < 0 || op < WAVE_OP_FWD || op > WAVE_OP_BORN) return 0;
    if (op == WAVE_OP_GRAD && ckpt_every < 1) return 0;
    if (op == WAVE_OP_REVOLVE && (ckpt_every < 0 || ckpt_every > g->nt)) return 0;
    return carve(nullptr, 0, true, d, op, nsrc, nrec, g->nt, ckpt_every).bytes;
}

size_t wave_ckpt_bytes(const wave_grid *g, int32_t ckpt_every)
{
    Dims d;
    if (check_grid(g, &d) || ckpt_every < 1) return 0;
    const size_t nseg = (size_t)((g->nt + ckpt_every - 1) / ckpt_every);
    return nseg * 2 * sizeof(float) * (size_t)d.npad;
}

int32_t wave_fwd(const wave_grid *g, const float *m, const float *damp, const wave_points *src,
                 const float *src_traces, const wave_points *rec, float *rec_traces, float *u_last,
                 float *ckpt, int32_t ckpt_every, const wave_tuning *tuning, void *ws,
                 size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!m || !damp || !ws) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, false, nullptr)) return WAVE_EINVAL;
        if (ckpt != nullptr && ckpt_every < 1) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_FWD, nsrc, nrec, g->nt, ckpt_every);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ti, tr;
        if (build_table(d, g->h, src, false, &ti) || build_table(d, g->h, rec, true, &tr))
            return WAVE_EINVAL;
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        if ((rc = prep_model(d, g, tuning, m, damp, L, stream))) return rc;
        Plan plan;
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &plan))) return rc;
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
        if ((rc = upload_table(ti, L.inj, stream)) || (rc = upload_table(tr, L.rec, stream))) return rc;
        if ((rc = sum_table(ti, L.inj, src_traces, nsrc, g->nt, stream))) return rc;
        Job job;
        job.d = d;
        job.st = st;
        job.cB = L.cB;
        job.cC = L.cC;
        job.status = L.status;
        job.cE = nullptr;
        job.inj = L.inj.view();
        job.q = src_traces;
        job.nq = nsrc;
        job.rec = L.rec.view();
        job.corner = L.corner;
        job.nslot = 8 * nrec;
        job.withhold = (tuning && (tuning->flags & WAVE_TEST_WITHHOLD)) ? 1 : 0;
        job.hinj = &ti;
        job.hrec = &tr;
        job.order = L.order;
        job.order_cap = L.order_cap;
        State s;
        for (int i = 0; i < 4; ++i) s.buf[i] = L.U[i];
        if ((rc = prof_begin(tuning, stream))) return rc;
        if ((rc = run_steps(job, s, g->nt, plan, stream, ckpt, ckpt_every, 0))) return rc;
        if ((rc = prof_end(stream))) return rc;
        if (nrec > 0 && rec_traces != nullptr)
            CK(wt::launch_gather(L.corner, L.rec.wts, g->nt, nrec, 1, rec_traces, stream));
        if (u_last != nullptr) {
            CK(wt::launch_unpad(s.buf[s.a], d.nx, d.ny, d.nz, d.nzp, 1.f, u_last, stream));
            CK(wt::launch_unpad(s.buf[s.b], d.nx, d.ny, d.nz, d.nzp, 1.f, u_last + d.n, stream));
        }
        return WAVE_OK;
    } catch (const std::bad_alloc &) {
        return WAVE_EINVAL;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_adj(const wave_grid *g, const float *m, const float *damp, const wave_points *rec,
                 const float *rec_resid, const wave_points *src, float *src_adj, float *v_last,
                 const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!m || !damp || !ws) return WAVE_EINVAL;
        if (check_points(rec, true, rec_resid) || check_points(src, false, nullptr)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_ADJ, nsrc, nrec, g->nt, 0);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ti, tr;
        if (build_table(d, g->h, rec, false, &ti) || build_table(d, g->h, src, true, &tr))
            return WAVE_EINVAL;
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        if ((rc = prep_model(d, g, tuning, m, damp, L, stream))) return rc;
        Plan plan;
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &plan))) return rc;
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
        if ((rc = upload_table(ti, L.inj, stream)) || (rc = upload_table(tr, L.rec, stream))) return rc;
        if ((rc = sum_table(ti, L.inj, rec_resid, nrec, g->nt, stream))) return rc;
        // reversed step j produces nu^{nt-j}: it injects res^{nt-1-j} and records
        // dJ/dq^{nt-1-j}
        Job job;
        job.d = d;
        job.st = st;
        job.cB = L.cB;
        job.cC = L.cC;
        job.status = L.status;
        job.inj = L.inj.view();
        job.q = rec_resid;
        job.nq = nrec;
        job.q_base = g->nt - 1;
        job.q_dir = -1;
        job.rec = L.rec.view();
        job.corner = L.corner;
        job.nslot = 8 * nsrc;
        job.c_base = g->nt - 1;
        job.c_dir = -1;
        job.hinj = &ti;
        job.hrec = &tr;
        job.order = L.order;
        job.order_cap = L.order_cap;
        State s;
        for (int i = 0; i < 4; ++i) s.buf[i] = L.U[i];
        if ((rc = prof_begin(tuning, stream))) return rc;
        if ((rc = run_steps(job, s, g->nt, plan, stream))) return rc;
        if ((rc = prof_end(stream))) return rc;
        if (nsrc > 0 && src_adj != nullptr)
            CK(wt::launch_gather(L.corner, L.rec.wts, g->nt, nsrc, 1, src_adj, stream));
        if (v_last != nullptr) {
            CK(wt::launch_unpad(s.buf[s.a], d.nx, d.ny, d.nz, d.nzp, 1.f, v_last, stream));
            CK(wt::launch_unpad(s.buf[s.b], d.nx, d.ny, d.nz, d.nzp, 1.f, v_last + d.n, stream));
        }
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_grad(const wave_grid *g, const float *m, const float *damp, const wave_points *src,
                  const float *src_traces, const wave_points *rec, const float *rec_resid,
                  const float *ckpt, int32_t ckpt_every, float *grad, const wave_tuning *tuning,
                  void *ws, size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!m || !damp || !ws || !ckpt || !grad || ckpt_every < 1) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, true, rec_resid)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        const int nt = g->nt;
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_GRAD, nsrc, nrec, nt, ckpt_every);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ts, tr;
        if (build_table(d, g->h, src, false, &ts) || build_table(d, g->h, rec, false, &tr))
            return WAVE_EINVAL;
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        if ((rc = prep_model(d, g, tuning, m, damp, L, stream))) return rc;
        Plan fplan;
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &fplan))) return rc;
        // the sweeps below run in the gradient modes, on the shapes chosen for them
        const int store_rows = std::max(1, std::min(ckpt_every, nt));
        if ((rc = upload_table(ts, L.inj, stream)) || (rc = upload_table(tr, L.inj2, stream))) return rc;
        if ((rc = sum_table(ts, L.inj, src_traces, nsrc, nt, stream)) ||
            (rc = sum_table(tr, L.inj2, rec_resid, nrec, nt, stream)))
            return rc;
        Plan rplan, aplan;
        if ((rc = grad_plan(d, g, fplan, st, L.cB, L.cC, L.cE, L.U, L.store, store_rows, L.G, L.status,
                            L.inj.view(), src_traces, nsrc, L.inj2.view(), rec_resid, nrec, &ts, &tr, L.order,
                            L.order_cap, stream, &rplan, &aplan)))
            return rc;
        CK(cudaMemsetAsync(L.G, 0, sizeof(float) * d.npad, stream));
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.V[i], 0, sizeof(float) * d.npad, stream));
        State adj;
        for (int i = 0; i < 4; ++i) adj.buf[i] = L.V[i];
        // the recompute and adjoint jobs keep their launch orders across
        // segments, each in its own buffer
        OrderCache ocr, oca;
        const int nseg = (nt + ckpt_every - 1) / ckpt_every;
        if ((rc = prof_begin(tuning, stream))) return rc;
        for (int c = nseg - 1; c >= 0; --c) {
            const int s0 = c * ckpt_every;
            const int len = std::min(ckpt_every, nt - s0);
            // 1) recompute u over [s0, s0+len) from checkpoint c, storing
            //    D^n = u^{n+1} - 2u^n + u^{n-1} in store[n - s0]
            State fw;
            for (int i = 0; i < 4; ++i) fw.buf[i] = L.U[i];
            const float *cp = ckpt + (size_t)c * 2 * d.npad;
            CK(cudaMemcpyAsync(fw.buf[0], cp, sizeof(float) * d.npad, cudaMemcpyDeviceToDevice, stream));
            CK(cudaMemcpyAsync(fw.buf[1], cp + d.npad, sizeof(float) * d.npad, cudaMemcpyDeviceToDevice,
                               stream));
            fw.a = 0;
            fw.b = 1;
            Job rj;
            rj.d = d;
            rj.st = st;
            rj.cB = L.cB;
            rj.cC = L.cC;
            rj.status = L.status;
            rj.cE = L.cE;
            rj.inj = L.inj.view();
            rj.q = src_traces;
            rj.nq = nsrc;
            rj.q_base = s0;
            rj.q_dir = 1;
            rj.dstore = L.store;
            rj.d_base = 0;
            rj.d_dir = 1;
            rj.hinj = &ts;
            rj.order = L.order;
            rj.order_cap = L.order_cap;
            rj.ocache = &ocr;
            if ((rc = run_steps(rj, fw, len, rplan, stream))) return rc;
            // 2) adjoint over the segment, newest step first: reversed step
            //    for n = s0+len-1 .. s0 produces nu^{n+1}, injects res^n and
            //    accumulates G += nu^{n+1} D^n
            Job aj;
            aj.d = d;
            aj.st = st;
            aj.cB = L.cB;
            aj.cC = L.cC;
            aj.status = L.status;
            aj.inj = L.inj2.view();
            aj.q = rec_resid;
            aj.nq = nrec;
            aj.q_base = s0 + len - 1;
            aj.q_dir = -1;
            aj.dload = L.store;
            aj.l_rows = store_rows;
            aj.l_base = len - 1;
            aj.l_dir = -1;
            aj.gacc = L.G;
            aj.hinj = &tr;
            aj.order = L.order_b;
            aj.order_cap = L.order_cap;
            aj.ocache = &oca;
            if ((rc = run_steps(aj, adj, len, aplan, stream))) return rc;
        }
        if ((rc = prof_end(stream))) return rc;
        const float scale = (float)(-1.0 / ((double)g->dt * (double)g->dt));
        CK(wt::launch_unpad(L.G, d.nx, d.ny, d.nz, d.nzp, scale, grad, stream));
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_born(const wave_grid *g, const float *m, const float *damp, const float *dm,
                  const wave_points *src, const float *src_traces, const wave_points *rec, float *rec_traces,
                  float *du_last, const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!m || !damp || !dm || !ws) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, true, rec_traces)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        const int nt = g->nt;
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_BORN, nsrc, nrec, nt, 0);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ts, tr;
        if (build_table(d, g->h, src, false, &ts) || build_table(d, g->h, rec, true, &tr)) return WAVE_EINVAL;
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        // B, C and E of the background model; P = -dm / dt^2
        if ((rc = prep_model(d, g, tuning, m, damp, L, stream))) return rc;
        CK(wt::launch_pad(dm, d.nx, d.ny, d.nz, d.nzp, L.G, stream,
                          (float)(-1.0 / ((double)g->dt * (double)g->dt))));
        Plan plan;
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &plan))) return rc;
        if ((rc = upload_table(ts, L.inj, stream)) || (rc = upload_table(tr, L.rec, stream))) return rc;
        if ((rc = sum_table(ts, L.inj, src_traces, nsrc, nt, stream))) return rc;
        for (int i = 0; i < 4; ++i) {
            CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
            CK(cudaMemsetAsync(L.V[i], 0, sizeof(float) * d.npad, stream));
        }
        State bg, pt;
        for (int i = 0; i < 4; ++i) {
            bg.buf[i] = L.U[i];
            pt.buf[i] = L.V[i];
        }
        // step n: the background sweep stores D^n = u^{n+1} - 2u^n + u^{n-1}
        // (sources included), then the perturbation sweep takes C P D^n and
        // records the receivers from du^{n+1}
        Job bj;
        bj.d = d;
        bj.st = st;
        bj.cB = L.cB;
        bj.cC = L.cC;
        bj.cE = L.cE;
        bj.status = L.status;
        bj.inj = L.inj.view();
        bj.q = src_traces;
        bj.nq = nsrc;
        bj.dstore = L.store;
        bj.d_base = 0;
        bj.d_dir = 0;
        bj.hinj = &ts;
        bj.order = L.order;
        bj.order_cap = L.order_cap;
        Job pj;
        pj.d = d;
        pj.st = st;
        pj.cB = L.cB;
        pj.cC = L.cC;
        pj.status = L.status;
        pj.rec = L.rec.view();
        pj.corner = L.corner;
        pj.nslot = 8 * nrec;
        pj.dload = L.store;
        pj.l_rows = 1;
        pj.l_base = 0;
        pj.l_dir = 0;
        pj.born = L.G;
        pj.hrec = &tr;
        pj.order = L.order_b;
        pj.order_cap = L.order_cap;
        OrderCache ocb, ocp;  // each job's launch order, computed once for its many one-step calls
        bj.ocache = &ocb;
        pj.ocache = &ocp;
        if ((rc = prof_begin(tuning, stream))) return rc;
        const bool two = tuning != nullptr && (tuning->flags & WAVE_BORN_TWO_SWEEPS);
        if (!two && born_fused_variant(g->space_order / 2) != nullptr) {
            // one fused sweep per step: the background (sources, D in
            // registers) and the perturbation (receivers) together
            Job fj;
            fj.d = d;
            fj.st = st;
            fj.cB = L.cB;
            fj.cC = L.cC;
            fj.cE = L.cE;
            fj.status = L.status;
            fj.inj = L.inj.view();
            fj.q = src_traces;
            fj.nq = nsrc;
            fj.rec = L.rec.view();
            fj.corner = L.corner;
            fj.nslot = 8 * nrec;
            fj.born = L.G;
            fj.s2 = &pt;
            fj.hinj = &ts;
            fj.hrec = &tr;
            fj.order = L.order;
            fj.order_cap = L.order_cap;
            if ((rc = run_steps(fj, bg, nt, plan, stream))) return rc;
        } else {
            for (int n = 0; n < nt; ++n) {
                bj.q_base = n;
                if ((rc = run_steps(bj, bg, 1, plan, stream))) return rc;
                pj.c_base = n;
                if ((rc = run_steps(pj, pt, 1, plan, stream))) return rc;
            }
        }
        if ((rc = prof_end(stream))) return rc;
        if (nrec > 0) CK(wt::launch_gather(L.corner, L.rec.wts, nt, nrec, 1, rec_traces, stream));
        if (du_last != nullptr) {
            CK(wt::launch_unpad(pt.buf[pt.a], d.nx, d.ny, d.nz, d.nzp, 1.f, du_last, stream));
            CK(wt::launch_unpad(pt.buf[pt.b], d.nx, d.ny, d.nz, d.nzp, 1.f, du_last + (size_t)d.nx * d.ny * d.nz,
                                stream));
        }
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int64_t wave_revolve_forward_steps(int32_t nt, int32_t nslots)
{
    if (nt < 1 || nslots < 0 || nslots > nt) return -1;
    try {
        long long n = 0;
        for (const RevAction &x : revolve_schedule(nt, nslots)) {
            if (x.kind == REV_ADVANCE) n += x.b - x.a;
            if (x.kind == REV_YOUTURN) n += 1;
        }
        return n;
    } catch (...) {
        return -1;
    }
}

int32_t wave_revolve_schedule(int32_t nt, int32_t nslots, int32_t *actions, int32_t cap)
{
    if (nt < 1 || nslots < 0 || nslots > nt || cap < 0 || (cap > 0 && actions == nullptr)) return WAVE_EINVAL;
    try {
        const std::vector<RevAction> v = revolve_schedule(nt, nslots);
        for (int i = 0; i < (int)v.size() && i < cap; ++i) {
            actions[3 * i] = v[i].kind;
            actions[3 * i + 1] = v[i].a;
            actions[3 * i + 2] = v[i].b;
        }
        return (int32_t)v.size();
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_grad_revolve(const wave_grid *g, const float *m, const float *damp, const wave_points *src,
                          const float *src_traces, const wave_points *rec, const float *rec_resid,
                          int32_t nslots, float *grad, const wave_tuning *tuning, void *ws, size_t ws_bytes,
                          void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        const int nt = g->nt;
        if (!m || !damp || !ws || !grad || nslots < 0 || nslots > nt) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, true, rec_resid)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_REVOLVE, nsrc, nrec, nt, nslots);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ts, tr;
        if (build_table(d, g->h, src, false, &ts) || build_table(d, g->h, rec, false, &tr))
            return WAVE_EINVAL;
        const std::vector<RevAction> sched = revolve_schedule(nt, nslots);
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        if ((rc = prep_model(d, g, tuning, m, damp, L, stream))) return rc;
        // forward advances on the forward plan, the reversed steps on the
        // family the gradient modes run fastest on (as wave_grad)
        Plan fplan, rplan, aplan;
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &fplan))) return rc;
        if ((rc = upload_table(ts, L.inj, stream)) || (rc = upload_table(tr, L.inj2, stream))) return rc;
        if ((rc = sum_table(ts, L.inj, src_traces, nsrc, nt, stream)) ||
            (rc = sum_table(tr, L.inj2, rec_resid, nrec, nt, stream)))
            return rc;
        if ((rc = grad_plan(d, g, fplan, st, L.cB, L.cC, L.cE, L.U, L.store, 1, L.G, L.status, L.inj.view(),
                            src_traces, nsrc, L.inj2.view(), rec_resid, nrec, &ts, &tr, L.order, L.order_cap,
                            stream, &rplan, &aplan)))
            return rc;
        CK(cudaMemsetAsync(L.G, 0, sizeof(float) * d.npad, stream));
        for (int i = 0; i < 4; ++i) CK(cudaMemsetAsync(L.V[i], 0, sizeof(float) * d.npad, stream));
        for (int i = 0; i < 2; ++i) CK(cudaMemsetAsync(L.U[i], 0, sizeof(float) * d.npad, stream));
        State fw, adj;
        for (int i = 0; i < 4; ++i) {
            fw.buf[i] = L.U[i];
            adj.buf[i] = L.V[i];
        }
        const size_t lvl = sizeof(float) * d.npad;
        // the three jobs of the schedule, each with its own launch-order
        // buffer kept across its many short calls
        Job fj;  // forward advance
        fj.d = d;
        fj.st = st;
        fj.cB = L.cB;
        fj.cC = L.cC;
        fj.status = L.status;
        fj.inj = L.inj.view();
        fj.q = src_traces;
        fj.nq = nsrc;
        fj.q_dir = 1;
        fj.hinj = &ts;
        fj.order = L.order;
        fj.order_cap = L.order_cap;
        Job rj = fj;  // one recompute step from u^a storing D^a
        rj.cE = L.cE;
        rj.dstore = L.store;
        rj.d_base = 0;
        rj.d_dir = 1;
        rj.order = L.order_b;
        Job aj;  // the adjoint step of time index a: nu^{a+1}, res^a, G += nu^{a+1} D^a
        aj.d = d;
        aj.st = st;
        aj.cB = L.cB;
        aj.cC = L.cC;
        aj.status = L.status;
        aj.inj = L.inj2.view();
        aj.q = rec_resid;
        aj.nq = nrec;
        aj.q_dir = -1;
        aj.dload = L.store;
        aj.l_rows = 1;
        aj.l_base = 0;
        aj.l_dir = -1;
        aj.gacc = L.G;
        aj.hinj = &tr;
        aj.order = L.order_c;
        aj.order_cap = L.order_cap;
        OrderCache ocf, ocr, oca;
        fj.ocache = &ocf;
        rj.ocache = &ocr;
        aj.ocache = &oca;
        if ((rc = prof_begin(tuning, stream))) return rc;
        for (const RevAction &x : sched) {
            if (x.kind == REV_RESTORE) {
                fw.a = 0;
                fw.b = 1;
                if (x.b < 0) {  // the zero state of step 0
                    CK(cudaMemsetAsync(L.U[0], 0, lvl, stream));
                    CK(cudaMemsetAsync(L.U[1], 0, lvl, stream));
                } else {
                    const float *sp = L.slots + (size_t)x.b * 2 * d.npad;
                    CK(cudaMemcpyAsync(L.U[0], sp, lvl, cudaMemcpyDeviceToDevice, stream));
                    CK(cudaMemcpyAsync(L.U[1], sp + d.npad, lvl, cudaMemcpyDeviceToDevice, stream));
                }
            } else if (x.kind == REV_TAKESHOT) {
                float *sp = L.slots + (size_t)x.b * 2 * d.npad;
                CK(cudaMemcpyAsync(sp, fw.buf[fw.a], lvl, cudaMemcpyDeviceToDevice, stream));
                CK(cudaMemcpyAsync(sp + d.npad, fw.buf[fw.b], lvl, cudaMemcpyDeviceToDevice, stream));
            } else if (x.kind == REV_ADVANCE) {
                fj.q_base = x.a;
                if ((rc = run_steps(fj, fw, x.b - x.a, fplan, stream))) return rc;
            } else {
                rj.q_base = x.a;
                if ((rc = run_steps(rj, fw, 1, rplan, stream))) return rc;
                aj.q_base = x.a;
                if ((rc = run_steps(aj, adj, 1, aplan, stream))) return rc;
            }
        }
        if ((rc = prof_end(stream))) return rc;
        const float scale = (float)(-1.0 / ((double)g->dt * (double)g->dt));
        CK(wt::launch_unpad(L.G, d.nx, d.ny, d.nz, d.nzp, scale, grad, stream));
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_heat(const wave_grid *g, const float *kappa, const float *u0, const wave_points *src,
                  const float *src_traces, const wave_points *rec, float *rec_traces, float *u_out,
                  const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!u0 || !u_out || !ws) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, false, nullptr)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_FWD, nsrc, nrec, g->nt, 0);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ti, tr;
        if (build_table(d, g->h, src, false, &ti) || build_table(d, g->h, rec, true, &tr))
            return WAVE_EINVAL;
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        // B = 0, C = dt kappa; stability dt kappa |L| <= 2 (|L| at the Nyquist corner)
        const bool allow = tuning && (tuning->flags & WAVE_ALLOW_UNSTABLE);
        double stot = 0.0;
        for (int a = 0; a < 3; ++a) stot += symbol_at_pi(g->space_order) / ((double)g->h[a] * g->h[a]);
        CK(cudaMemsetAsync(L.status, 0, sizeof(int) * kStatusWords, stream));
        CK(wt::launch_heat_prep(kappa, d.nx, d.ny, d.nz, d.nzp, g->dt, allow ? 0.f : (float)(g->dt * stot),
                                L.cB, L.cC, L.status, stream));
        Plan plan;
        if ((rc = resolve_plan(d, g, tuning, true, &st, L.cB, L.cC, L.U, L.status, stream, &plan))) return rc;
        // level 0 = u0; level -1 is never weighted (B = 0) but must be finite
        // (the other two buffers are written before they are read)
        CK(cudaMemsetAsync(L.U[1], 0, sizeof(float) * d.npad, stream));
        CK(wt::launch_pad(u0, d.nx, d.ny, d.nz, d.nzp, L.U[0], stream));
        if ((rc = upload_table(ti, L.inj, stream)) || (rc = upload_table(tr, L.rec, stream))) return rc;
        if ((rc = sum_table(ti, L.inj, src_traces, nsrc, g->nt, stream))) return rc;
        Job job;
        job.d = d;
        job.st = st;
        job.cB = L.cB;
        job.cC = L.cC;
        job.status = L.status;
        job.cE = nullptr;
        job.inj = L.inj.view();
        job.q = src_traces;
        job.nq = nsrc;
        job.rec = L.rec.view();
        job.corner = L.corner;
        job.nslot = 8 * nrec;
        job.hinj = &ti;
        job.hrec = &tr;
        job.order = L.order;
        job.order_cap = L.order_cap;
        State s;
        for (int i = 0; i < 4; ++i) s.buf[i] = L.U[i];
        if ((rc = prof_begin(tuning, stream))) return rc;
        if ((rc = run_steps(job, s, g->nt, plan, stream))) return rc;
        if ((rc = prof_end(stream))) return rc;
        if (nrec > 0 && rec_traces != nullptr)
            CK(wt::launch_gather(L.corner, L.rec.wts, g->nt, nrec, 1, rec_traces, stream));
        CK(wt::launch_unpad(s.buf[s.a], d.nx, d.ny, d.nz, d.nzp, 1.f, u_out, stream));
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_heat_ab2(const wave_grid *g, const float *kappa, const float *u0, const wave_points *src,
                      const float *src_traces, const wave_points *rec, float *rec_traces, float *u_out,
                      const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream_)
{
    try {
        Dims d;
        int rc = check_grid(g, &d);
        if (rc) return rc;
        if (!u0 || !u_out || !ws) return WAVE_EINVAL;
        if (check_points(src, true, src_traces) || check_points(rec, false, nullptr)) return WAVE_EINVAL;
        if ((uintptr_t)ws % kAlign) return WAVE_EINVAL;
        const int nsrc = npts_of(src), nrec = npts_of(rec);
        const int R = g->space_order / 2;
        Layout L = carve(ws, ws_bytes, false, d, WAVE_OP_FWD, nsrc, nrec, g->nt, 0);
        if (L.bytes > ws_bytes) return WAVE_ENOSPACE;
        HostTable ti, tr;
        if (build_table(d, g->h, src, false, &ti) || build_table(d, g->h, rec, true, &tr)) return WAVE_EINVAL;
        // depth 2 where compiled, else 1; tuning->time_tile 1 asks for the
        // untiled sweep
        const int want = tuning != nullptr && tuning->time_tile == 1 ? 1 : 2;
        const int T = (want == 2 && ab2_variant(R, 2) != nullptr) ? 2 : 1;
        Plan plan;
        plan.v = ab2_variant(R, T);
        if (plan.v == nullptr) return WAVE_EUNSUPPORTED;
        plan.chunk_given = tuning != nullptr && tuning->tile_x > 0;
        plan.chunk = std::min(plan.chunk_given ? std::min(tuning->tile_x, d.nx) : default_chunk(d, plan.v),
                              max_chunk(plan.v));
        cudaStream_t stream = (cudaStream_t)stream_;
        const Stencil st = make_stencil(g);
        // B = 0, C = dt kappa; the two-step scheme is stable while
        // dt kappa |L| <= 1 (the check takes 2 dt |L| against 2)
        const bool allow = tuning && (tuning->flags & WAVE_ALLOW_UNSTABLE);
        double stot = 0.0;
        for (int a = 0; a < 3; ++a) stot += symbol_at_pi(g->space_order) / ((double)g->h[a] * g->h[a]);
        CK(cudaMemsetAsync(L.status, 0, sizeof(int) * kStatusWords, stream));
        CK(wt::launch_heat_prep(kappa, d.nx, d.ny, d.nz, d.nzp, g->dt, allow ? 0.f : (float)(2.0 * g->dt * stot),
                                L.cB, L.cC, L.status, stream));
        // level 0 = u0 in U[0]; the rate F^{-1} (weight 0 in the Euler start,
        // but read) = 0 in U[2]
        CK(wt::launch_pad(u0, d.nx, d.ny, d.nz, d.nzp, L.U[0], stream));
        CK(cudaMemsetAsync(L.U[2], 0, sizeof(float) * d.npad, stream));
        if ((rc = upload_table(ti, L.inj, stream)) || (rc = upload_table(tr, L.rec, stream))) return rc;
        if ((rc = sum_table(ti, L.inj, src_traces, nsrc, g->nt, stream))) return rc;
        Job job;
        job.d = d;
        job.st = st;
        job.cB = L.cB;
        job.cC = L.cC;
        job.status = L.status;
        job.cE = nullptr;
        job.inj = L.inj.view();
        job.q = src_traces;
        job.nq = nsrc;
        job.rec = L.rec.view();
        job.corner = L.corner;
        job.nslot = 8 * nrec;
        job.hinj = &ti;
        job.hrec = &tr;
        job.order = L.order;
        job.order_cap = L.order_cap;
        job.ab2 = T;
        State s;
        for (int i = 0; i < 4; ++i) s.buf[i] = L.U[i];
        s.a = 0;
        s.b = 2;
        if ((rc = prof_begin(tuning, stream))) return rc;
        if ((rc = run_steps(job, s, g->nt, plan, stream))) return rc;
        if ((rc = prof_end(stream))) return rc;
        if (nrec > 0 && rec_traces != nullptr)
            CK(wt::launch_gather(L.corner, L.rec.wts, g->nt, nrec, 1, rec_traces, stream));
        CK(wt::launch_unpad(s.buf[s.a], d.nx, d.ny, d.nz, d.nzp, 1.f, u_out, stream));
        return WAVE_OK;
    } catch (...) {
        return WAVE_EINVAL;
    }
}

int32_t wave_status(const void *ws, void *stream_)
{
    if (ws == nullptr) return WAVE_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return WAVE_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WAVE_ECUDA;
    return st;
}

int32_t wave_sweep_stats(float *ms, int32_t *launches, int32_t *steps)
{
    if (!g_prof.valid || ms == nullptr) return WAVE_EINVAL;
    if (cudaEventSynchronize(g_prof.e1) != cudaSuccess) return WAVE_ECUDA;
    if (cudaEventElapsedTime(ms, g_prof.e0, g_prof.e1) != cudaSuccess) return WAVE_ECUDA;
    if (launches) *launches = g_prof.launches;
    if (steps) *steps = g_prof.steps;
    return WAVE_OK;
}

int32_t wave_list_variants(int32_t space_order, int32_t *out, int32_t max)
{
    if (space_order < 2 || space_order > 16 || space_order % 2 || max < 0 || (max > 0 && !out))
        return WAVE_EINVAL;
    const SweepVariant *vs;
    const int nv = variants_for(space_order / 2, &vs);
    for (int i = 0; i < nv && i < max; ++i) {
        int32_t *o = out + 8 * i;
        o[0] = vs[i].T;
        o[1] = vs[i].BY;
        o[2] = vs[i].BZ;
        o[3] = vs[i].V;
        o[4] = vs[i].P;
        o[5] = vs[i].threads;
        o[6] = vs[i].kind + 1;
        o[7] = rows_of(&vs[i]);
    }
    return nv;
}

int32_t wave_autotune_stats(int32_t *candidates, int32_t *pruned)
{
    if (candidates == nullptr || pruned == nullptr) return WAVE_EINVAL;
    if (g_tune_stats.candidates == 0) return WAVE_EINVAL;
    *candidates = g_tune_stats.candidates;
    *pruned = g_tune_stats.pruned;
    return WAVE_OK;
}

int32_t wave_plan_bound(const wave_grid *g, const wave_tuning *tuning, double hbm_gbs, double lsu_gbs,
                        double l2_bytes, double *ms)
{
    Dims d;
    int rc = check_grid(g, &d);
    if (rc) return rc;
    if (ms == nullptr || tuning == nullptr || tuning->time_tile < 1) return WAVE_EINVAL;
    Plan p;
    float *U[4] = {nullptr, nullptr, nullptr, nullptr};
    if ((rc = resolve_plan(d, g, tuning, false, nullptr, nullptr, nullptr, U, nullptr, nullptr, &p))) return rc;
    double hbm = hbm_gbs * 1e9, lsu = lsu_gbs * 1e9, l2 = l2_bytes;
    if (hbm_gbs <= 0.0 || lsu_gbs <= 0.0 || l2_bytes == 0.0) {
        const DevicePeaks pk = device_peaks();
        if (hbm_gbs <= 0.0) hbm = pk.hbm;
        if (lsu_gbs <= 0.0) lsu = pk.lsu;
        if (l2_bytes == 0.0) l2 = pk.l2;
    }
    if (hbm <= 0.0 || lsu <= 0.0) return WAVE_ECUDA;
    *ms = plan_bound_ms(d, p.v, p.chunk, hbm, lsu, l2);
    return WAVE_OK;
}

int32_t wave_describe_grad_plan(const wave_grid *g, const wave_tuning *tuning, int32_t nsrc, int32_t nrec,
                                int32_t ckpt_every, int32_t *out)
{
    Dims d;
    int rc = check_grid(g, &d);
    if (rc) return rc;
    if (out == nullptr || nsrc < 0 || nrec < 0 || ckpt_every < 1) return WAVE_EINVAL;
    Plan fwd;
    float *U[4] = {nullptr, nullptr, nullptr, nullptr};
    if ((rc = resolve_plan(d, g, tuning, false, nullptr, nullptr, nullptr, U, nullptr, nullptr, &fwd))) return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    const int rows = std::max(1, std::min((int)ckpt_every, g->nt));
    const GradKey key{d.nx, d.ny, d.nz, g->space_order, dev, nsrc, nrec, rows, fwd.v};
    std::pair<Plan, Plan> pp;
    {
        std::lock_guard<std::mutex> lk(g_grad_mu);
        auto it = g_grad_cache.find(key);
        if (it == g_grad_cache.end()) return WAVE_EUNSUPPORTED;
        pp = it->second;
    }
    const Plan *ps[2] = {&pp.first, &pp.second};
    for (int k = 0; k < 2; ++k) {
        const Plan &p = *ps[k];
        int32_t *o = out + 8 * k;
        o[0] = p.v->T;
        o[1] = p.v->BY;
        o[2] = p.chunk > 0 ? p.chunk : default_chunk(d, p.v);
        o[3] = p.v->BZ;
        o[4] = p.v->V;
        o[5] = p.v->P;
        o[6] = p.v->kind + 1;
        o[7] = rows_of(p.v);
    }
    return WAVE_OK;
}

int32_t wave_describe_plan(const wave_grid *g, const wave_tuning *tuning, int32_t *out)
{
    Dims d;
    int rc = check_grid(g, &d);
    if (rc) return rc;
    if (out == nullptr) return WAVE_EINVAL;
    Plan p;
    float *U[4] = {nullptr, nullptr, nullptr, nullptr};
    if ((rc = resolve_plan(d, g, tuning, false, nullptr, nullptr, nullptr, U, nullptr, nullptr, &p))) return rc;
    out[0] = p.v->T;
    out[1] = p.v->BY;
    out[2] = p.chunk;
    out[3] = p.v->BZ;
    out[4] = p.v->V;
    out[5] = p.v->P;
    out[6] = p.v->kind + 1;
    out[7] = rows_of(p.v);
    return WAVE_OK;
}

}  // extern "C"
