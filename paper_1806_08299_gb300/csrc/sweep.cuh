// sweep.cuh -- the time-tiled leapfrog sweep for sm_103a.
//
// One launch advances the wavefield by T time steps (T = 1 is the untiled
// sweep).  It realises the paper's time tiling (Sec. 4.1 skewing, Sec. 4.2
// time tiles with min/max bounding) for a GPU:
//
//  * Each block owns an output tile of BZ (z) x BY (y) columns and an x-chunk
//    [X0, X1) of `chunk` planes, and streams along x.  In iteration i, plane
//    c0 = X0 - RT + i of level n enters, and stage s (1..T) computes level
//    n+s on plane c0 - s*R: the skew by the stencil radius R per time step of
//    Sec. 4.1, the minimum legal factor (Sec. 2.3.2.1).  Every x-dependence
//    of a stage is then already computed, and T time levels are live on chip
//    at once (the time buffer of Sec. 5.2.1).  Stage s starts at iteration
//    2sR, when its x-queue holds the chunk's own planes, so it computes
//    exactly the planes [X0 - (T-s)R, X1 + (T-s)R) that later stages and
//    stores need; the first 2R iterations load no ring-K data.  Block
//    indices run z-tile fastest, then y-tile, then chunk, so blocks resident
//    together stream neighbouring columns over the same x-range and share
//    their overlapping halos through L2.
//  * Point arithmetic runs on pairs of z points with the paired FP32
//    instructions of sm_100-class GPUs (__ffma2_rn and friends), each lane
//    rounded as its scalar counterpart.
//  * In y and z, neighbouring blocks read overlapping halos of width R*T and
//    recompute the shrinking halo of each stage, so blocks never wait on one
//    another.
//  * Staging (Blackwell TMA, warp specialised): a producer warp issues
//    cp.async.bulk.tensor loads up to P iterations ahead into two
//    shared-memory rings; "full" mbarriers (transaction counts) tell the
//    consumer threads a slot has landed and "empty" mbarriers (one arrival per
//    consumer thread) tell the producer a slot may be refilled, so consumer
//    warps are never held in lock step by the loads.  Ring U holds the
//    R+1+P most recent level-n planes with their y/z halos; stage 1 reads its
//    y and z neighbours there and its x neighbours from registers.  Ring K
//    holds, per iteration, level n-1 and the per-point
//    coefficients B, C of stage 1's plane; stage s reads the B, C that stage 1
//    read (s-1)R iterations earlier, so ring K is (T-1)R+1+P iterations deep.
//    The untiled sweep (T = 1) of radius R >= 3 keeps no ring U.  Each ring-K slot of it also
//    takes the centre plane c0 - R with its halo and, separately, the
//    level-n plane c0 in the K-box shape for the x-queue.  That plane comes
//    twice from L2 instead of staying R iterations in shared memory, so a
//    block needs 1+P slots instead of R+1+P planes, which at high orders
//    lets more blocks share an SM.
//    TMA fills everything outside
//    the grid with zeros; with B = C = 0 there, points outside the grid are
//    computed as exactly 0.  This plays the role of the paper's min/max bounds
//    (Sec. 4.2.2) without branches.
//  * Every stage keeps a register queue of the 2R+1 x-planes of its input
//    level per thread (V consecutive z points per thread).  Stages s >= 2
//    exchange their centre plane through shared memory for the y and z
//    neighbours (double buffered, one named barrier among the consumer threads
//    per plane); stage 1 reads them from ring U (T = 1: from the ring-K slot).
//  * Sources are injected and receiver corners recorded inside the sweep (the
//    imperfectly nested source/receiver loops the paper leaves open,
//    Sec. 4.5.1 and Sec. 6.3.1).
//  * Every mbarrier wait is bounded by %globaltimer; on expiry the thread
//    records WAVE_ETIMEOUT in the status word and raises a block-wide abort
//    flag; every thread leaves its loop at its next check, and the producer
//    waits (bounded) for its copies in flight before the block exits.
//
// Bit-exactness: every point update is the same sequence of IEEE-rounded
// operations (explicit __fmaf_rn / __fadd_rn / __fsub_rn / __fmul_rn, so no
// contraction choice is left to the compiler), whatever T, tile shape or
// launch split.  Tiled and untiled sweeps therefore agree bitwise, the GPU
// analogue of the paper's verification rule (Sec. 4.3, Sec. 5.4.3).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wt {

constexpr int kMaxR = 8;
constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded waits: 2 s

// Per-axis stencil coefficients c_k / h_a^2 in FP32, each stored twice (x
// and y of a float2) for the paired FP32 instructions; cc is the centre
// weight (c_0/hx^2 + c_0/hy^2) + c_0/hz^2 rounded once on the host.
struct Stencil {
    float2 cc;
    float2 cx[kMaxR + 1];
    float2 cy[kMaxR + 1];
    float2 cz[kMaxR + 1];
};

// Sparse points of one kind, sorted by (x, y, z).  plane_start[x] ..
// plane_start[x+1] index `pts`; each pt = (y, z, item_begin, item_end).
// Injection items: (source index, weight); record items: corner slot.
// Per-plane point tables, sorted by (x, y, z), each grid point once:
// pts = (y, z, begin, end) of its items in item (and w): the point index of
// an injection, the corner slot of a record.
struct PointTable {
    const int *plane_start;  // [nx + 1] or nullptr (no points)
    const int4 *pts;
    const int *item;
    const float *w;
    // injection tables: the value each entry injects at every trace row,
    // f[row * fstride + e] = sum over its items (ascending) of w q[row][item],
    // summed once per call before the sweeps (which read only f, pts and
    // plane_start; item and w serve that sum)
    const float *f;
    long long fstride;
};

struct SweepArgs {
    int nx, ny, nz;          // nz: padded z extent, a multiple of 8
    int sx;                  // ny * nz (< 2^31, checked on the host)
    long long npad;          // nx * ny * nz
    float *out_hi;           // level n+T (T == 1: may alias level n-1, updated in place)
    float *out_lo;           // level n+T-1 (T >= 2)
    const float *cE;         // per point -2 eta/(m+eta) (second-difference mode)
    PointTable inj;          // injection points
    const float *q;          // traces [rows][nq]
    int nq, q_row0, q_dir;   // stage s uses trace row q_row0 + q_dir*(s-1)
    PointTable rec;          // receiver corners
    float *corner;           // [rows][nslot]
    int nslot, c_row0, c_dir;
    float *dstore;           // second differences: row d_row0 + d_dir*(s-1) (or nullptr)
    long long d_row0;
    int d_dir;
    const float *dload;      // imaging condition: g += level * D[row] (or nullptr)
    long long l_row0;
    int l_dir;
    float *gacc;
    float ab1, ab0;          // two-step Adams-Bashforth weights of stage 1 (3/2, -1/2; 1, 0 to start)
    int withhold;            // test hook: the producer issues nothing (waits run out)
    int chunk;               // x planes per block
    int tiles_z, tiles_y;    // column tiles of the grid
    int *status;             // device status word (atomicMin of WAVE_E* codes)
    const int *order;        // launch order: block b sweeps tile order[b] (nullptr: tile b)
};

// TMA descriptors of the arrays the sweep reads (all [nx][ny][nz] float32):
//   u    : level n, box (PW, H0, 1)
//   um   : level n-1, box (W0, H0 - 2R, 1)
//   B, C : coefficients, box (W0, H0 - 2R, 1)
//   x0, x1 : the gradient sweeps' extra inputs (XB >= 1, same box as B):
//          second-difference mode x0 = E; imaging-condition mode x0 = this
//          step's stored D row, x1 = the gradient accumulator G
struct SweepMaps {
    CUtensorMap u, um, B, C, x0, x1;
    CUtensorMap uk;  // level n with the K-box shape: the x-queue feed of T == 1
};

// Shared memory of the per-plane sparse slices for an x-chunk of `chunk`
// planes at time-tile radius rt = R*T: plane_start slices of the injection
// and record tables (int each) and two relevance flags (byte each) per plane
// visited.
__host__ __device__ constexpr size_t sweep_table_bytes(int chunk, int rt)
{
    return (10 * (size_t)(chunk + 3 * rt + 2) + 15) / 16 * 16;
}

// XB: extra ring-K boxes of the gradient sweeps (0 = none: forward and
// adjoint; 1 = E, second-difference mode; 2 = D and G, imaging-condition
// mode), loaded by TMA with the other inputs instead of by the consumers.
template <int R, int T, int V, int BZ, int BY, int P, int MB, int XB = 0>
struct SweepShape {
    static constexpr int RT = R * T;
    static constexpr int A0 = ((RT + 3) / 4) * 4;   // z halo, keeps 16-byte alignment
    static constexpr int W0 = BZ + 2 * A0;          // layout width (z points)
    static constexpr int H0 = BY + 2 * RT;          // layout rows (y)
    // Consumer threads cover only what stage 1 computes: rows [R, H0 - R) and
    // the columns [ZL, ZR) of stage 1's z-range, V points per thread.
    static constexpr int ZL = (A0 - (T - 1) * R) / 4 * 4;
    static constexpr int ZR = (A0 + BZ + (T - 1) * R + 3) / 4 * 4;
    static constexpr int LZ = (ZR - ZL) / V;        // threads per row
    static constexpr int HT = H0 - 2 * R;           // thread rows
    static constexpr int NT = LZ * HT;              // consumer threads per block
    static constexpr int NTB = NT + 32;             // + one producer warp
    static constexpr int RP = ((R + 3) / 4) * 4;    // z pad of ring-U rows / centre planes
    static constexpr int PW = W0 + 2 * RP;          // ring-U / centre-plane pitch
    static constexpr int HK = H0 - 2 * R;           // rows of ring-K boxes (from row R)
    // T == 1 with R >= 3 keeps no ring U: each ring-K slot also holds the
    // centre plane c0 - R with its halo (for the y and z neighbours) and the
    // level-n plane c0 that enters the x-queue, so no slot has to outlive its
    // iteration (for R <= 2 the R+1+P planes of ring U are the smaller store)
    static constexpr bool SPLIT = T == 1 && R >= 3;
    static constexpr int DU = SPLIT ? 0 : R + 1 + P;  // ring-U depth (planes)
    static constexpr int DK = (T - 1) * R + 1 + P;  // ring-K depth (iterations)
    static constexpr int DF = P + 1;                // iterations in flight (full barriers)
    static constexpr unsigned UBOX = PW * H0 * 4;   // bytes of one U box
    static constexpr unsigned KBOX = W0 * HK * 4;   // bytes of one K box (um, B or C)
    static constexpr unsigned USLOT = (UBOX + 127) / 128 * 128;
    static constexpr unsigned KBOXP = (KBOX + 127) / 128 * 128;
    // byte offsets in a ring-K slot: [centre U box (T == 1)] u^{n-1}, B, C,
    // [x0, x1], [level-n feed box (T == 1)]
    static constexpr unsigned K_U = 0;
    static constexpr unsigned K_UM = SPLIT ? USLOT : 0;
    static constexpr unsigned K_B = K_UM + KBOXP;
    static constexpr unsigned K_C = K_UM + 2 * KBOXP;
    static constexpr unsigned K_X0 = K_UM + 3 * KBOXP;
    static constexpr unsigned K_X1 = K_UM + 4 * KBOXP;
    static constexpr unsigned K_F = K_UM + (3 + XB) * KBOXP;
    static constexpr unsigned KSLOT = SPLIT ? K_F + KBOXP : (3 + XB) * KBOXP;
    // bytes landing per iteration: from iteration 2R on, and before (fill)
    static constexpr unsigned TXB = UBOX + (3 + XB) * KBOX + (SPLIT ? KBOX : 0);
    static constexpr unsigned TX0 = SPLIT ? KBOX : UBOX;
    static constexpr int PLANE = PW * H0;           // centre plane (floats), stages >= 2
    static constexpr size_t OFF_K = (size_t)DU * USLOT;
    static constexpr size_t OFF_S = OFF_K + (size_t)DK * KSLOT;
    static constexpr size_t OFF_BAR = OFF_S + sizeof(float) * 2 * (T - 1) * PLANE;
    static constexpr size_t OFF_P = OFF_BAR + 8 * (2 * DF + DU + DK) + 16;
    static constexpr size_t SMEM = OFF_P;           // + per-plane sparse slices (smem_bytes)
    static size_t smem_bytes(int chunk) { return OFF_P + sweep_table_bytes(chunk, RT) + 16; }
    // blocks per SM the variant is compiled for (__launch_bounds__ minimum):
    // bounds the registers per thread; must also fit shared memory
    static constexpr int MINB = MB;
    static_assert(MB >= 1 && (size_t)MB * (SMEM + 4096) <= 228 * 1024 && MB * NTB <= 2048,
                  "blocks per SM do not fit shared memory or thread slots");
    static_assert(V == 2 || V == 4 || V == 8, "V must be 2, 4 or 8");
    static_assert(XB >= 0 && XB <= 2 && (XB == 0 || T == 1), "extra boxes only for untiled sweeps");
    // a thread's V points start at a multiple of V (rows are padded to a
    // multiple of 8), so they never straddle the end of a row
    static_assert(V < 8 || ((A0 - ZL) % 8 == 0 && BZ % 8 == 0), "V = 8 needs 8-aligned thread columns");
    static_assert(BZ % 4 == 0, "BZ must keep 16-byte alignment");
    static_assert(NT % 32 == 0, "consumer threads must fill whole warps (named barrier)");
    static_assert(NTB <= 1024, "too many threads per block");
    static_assert(R >= 1 && R <= kMaxR, "radius out of range");
    static_assert(PW <= 256 && H0 <= 256, "TMA box dimension above 256");
    static_assert(TXB < (1u << 20), "mbarrier tx count");
    static_assert(SMEM <= 220 * 1024, "shared memory above the per-block limit");
};

// ---------------------------------------------------------------------------
// PTX helpers (TMA, mbarrier)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Barrier 1 over the consumer threads only (the producer warp is not part of
// it); returns the OR of `flag` over them, so every consumer takes the same
// decision.
__device__ __forceinline__ bool consumer_sync_any(int nthreads, bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`; false if it did not complete within kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

// Acquire a TMA descriptor held in global memory (written by a host copy)
// for the tensormap proxy; the calling thread may then load through it.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// Ask for the box of `map` at (c0, c1, c2) to be brought into L2 (no shared
// memory, no barrier): a later tma_load_3d of it then waits for L2, not HBM.
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"((uint64_t)map),
                 "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

// V consecutive floats as V/2 pairs (shared or global memory; 16-byte
// aligned for V >= 4, 8-byte for V = 2).
template <int V>
__device__ __forceinline__ void ld2(float2 *d, const float *p)
{
    if constexpr (V >= 4) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(p)[i];
            d[2 * i] = make_float2(t.x, t.y);
            d[2 * i + 1] = make_float2(t.z, t.w);
        }
    } else {
        d[0] = *reinterpret_cast<const float2 *>(p);
    }
}

template <int V>
__device__ __forceinline__ void ldg2(float2 *d, const float *p)
{
    if constexpr (V >= 4) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
            d[2 * i] = make_float2(t.x, t.y);
            d[2 * i + 1] = make_float2(t.z, t.w);
        }
    } else {
        d[0] = __ldg(reinterpret_cast<const float2 *>(p));
    }
}

template <int V>
__device__ __forceinline__ void st2(float *p, const float2 *s)
{
    if constexpr (V >= 4) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(s[2 * i].x, s[2 * i].y, s[2 * i + 1].x, s[2 * i + 1].y);
    } else {
        *reinterpret_cast<float2 *>(p) = s[0];
    }
}

// u - w of a pair, exactly as two IEEE subtractions (negation is exact).
__device__ __forceinline__ float2 fsub2_rn(float2 u, float2 w)
{
    return __fadd2_rn(u, make_float2(-w.x, -w.y));
}

// The sweep of block `blk` of one problem: the body of the single-problem
// kernel and of the batched kernel below.
template <int R, int T, int V, int BZ, int BY, int P, int MB, int XB>
__device__ __forceinline__ void sweep_block(const SweepArgs &a, const Stencil &st, const SweepMaps &mp,
                                            const int blk)
{
    using S = SweepShape<R, T, V, BZ, BY, P, MB, XB>;
    constexpr int QL = 2 * R + 1;
    constexpr int ZW = V + 2 * S::RP;  // z window per thread (floats)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ringU = reinterpret_cast<float *>(smem_raw);
    unsigned char *ringK = smem_raw + S::OFF_K;
    float *splane = reinterpret_cast<float *>(smem_raw + S::OFF_S);  // [T-1][2][PLANE]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + S::OFF_BAR);  // per iteration in flight
    uint64_t *empF = full + S::DF;   // consumers have waited on full[] (one per iteration in flight)
    uint64_t *empU = empF + S::DF;   // per ring-U slot: released by all consumers
    uint64_t *empK = empU + S::DU;   // per ring-K slot: released by all consumers
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empK + S::DK);

    if (blockDim.x != S::NTB) {  // launched with the wrong shape: report, do nothing
        if (threadIdx.x == 0 && blk == 0) atomicMin(a.status, -1 /* WAVE_EINVAL */);
        return;
    }
    // Programmatic dependent launch: once every block of this launch has
    // started, the next launch on the stream may start its blocks, which run
    // their prologue (sparse-table scan, barrier set-up) and then wait below
    // for this launch to complete before touching any field.  Without the
    // launch attribute both instructions do nothing.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tid = threadIdx.x;
    const int col = S::ZL + (tid % S::LZ) * V;  // layout column of this thread's V points
    const int row = R + tid / S::LZ;            // layout row
    // blocks that hold sparse points come first in the launch order, so their
    // extra work overlaps the later waves instead of trailing the last one
    int b = a.order != nullptr ? __ldg(a.order + blk) : blk;
    const int tzi = b % a.tiles_z;
    b /= a.tiles_z;
    const int tyi = b % a.tiles_y;
    const int txi = b / a.tiles_y;
    const int X0 = txi * a.chunk;
    const int X1 = min(X0 + a.chunk, a.nx);
    const int gz0 = tzi * BZ - S::A0;  // global z of layout column 0
    const int gy0 = tyi * BY - S::RT;  // global y of layout row 0
    const int gz = gz0 + col;
    const int gy = gy0 + row;
    const bool in_yz = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const bool inner = in_yz && row >= S::RT && row < S::RT + BY && col >= S::A0 && col < S::A0 + BZ;
    const long long yz = in_yz ? (long long)gy * a.nz + gz : 0;
    const int ownU = row * S::PW + S::RP + col;        // in a U box / centre plane
    const int ownK = (row - R) * S::W0 + col;          // in a K box
    const int niter = (X1 - X0) + 2 * S::RT;
    const int c00 = X0 - S::RT;                        // plane of level n at iteration 0

    // Sparse tables of the planes this block visits, [X0 - 2RT, X1 + RT]:
    // plane_start slices (clamped, so planes outside the grid hold 0 points)
    // and a per-plane flag telling whether any point of that plane lies in
    // this block's layout, so that other blocks never touch the tables.
    const int pbase = X0 - 2 * S::RT;
    const int plen = (X1 - X0) + 3 * S::RT + 2;
    int *pinj = reinterpret_cast<int *>(smem_raw + S::OFF_P);
    int *prec = pinj + plen;
    unsigned char *finj = reinterpret_cast<unsigned char *>(prec + plen);
    unsigned char *frec = finj + plen;
    int my_inj = 0, my_rec = 0;  // this thread found a relevant point in some plane
    for (int k = tid; k < plen; k += S::NTB) {
        const int cp = min(max(pbase + k, 0), a.nx);
        const int ci = min(max(pbase + k + 1, 0), a.nx);
        int fi = 0, fr = 0;
        if (a.inj.plane_start != nullptr) {
            const int e0 = a.inj.plane_start[cp], e1 = a.inj.plane_start[ci];
            pinj[k] = e0;
            for (int eb = e0; eb < e1 && !fi; eb += 4) {
                int4 pt4[4];  // four table points per round trip
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    pt4[u] = eb + u < e1 ? __ldg(a.inj.pts + eb + u) : make_int4(-(1 << 30), -(1 << 30), 0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 pt = pt4[u];
                    fi |= pt.x >= gy0 && pt.x < gy0 + S::H0 && pt.y >= gz0 + S::ZL && pt.y < gz0 + S::ZR;
                }
            }
        } else {
            pinj[k] = 0;
        }
        if (a.rec.plane_start != nullptr) {
            const int e0 = a.rec.plane_start[cp], e1 = a.rec.plane_start[ci];
            prec[k] = e0;
            // four table points per round trip (a plane often holds a few)
            for (int eb = e0; eb < e1 && !fr; eb += 4) {
                int4 pt4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    pt4[u] = eb + u < e1 ? __ldg(a.rec.pts + eb + u) : make_int4(-(1 << 30), -(1 << 30), 0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 pt = pt4[u];
                    fr |= pt.x >= gy0 + S::RT && pt.x < gy0 + S::RT + BY && pt.y >= gz0 + S::A0 &&
                          pt.y < gz0 + S::A0 + BZ;
                }
            }
        } else {
            prec[k] = 0;
        }
        finj[k] = (unsigned char)fi;
        frec[k] = (unsigned char)fr;
        my_inj |= fi;
        my_rec |= fr;
    }
    for (int k = tid; k < 2 * (T - 1) * S::PLANE; k += S::NTB) splane[k] = 0.f;
    if (tid == 0) {
        for (int k = 0; k < S::DF; ++k) mbar_init(full + k, 1);
        // release barriers count consumer warps: lane 0 arrives for its warp
        for (int k = 0; k < S::DF + S::DU + S::DK; ++k) mbar_init(empF + k, S::NT / 32);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // whether any plane of this block holds a relevant point at all: most
    // blocks hold none and then never read the per-plane flags
    const bool any_inj = __syncthreads_or(my_inj) != 0;
    const bool any_rec = __syncthreads_or(my_rec) != 0;
    // the previous launch on the stream (the previous time step) has completed
    // and its writes are visible; every field access below comes after this
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (tid >= S::NT) {
        // ------------------------------ producer warp ------------------------------
        if (tid == S::NT && !a.withhold) {
            int ju = 0, jk = 0, jf = 0;  // slot of iteration j in ring U / ring K / full barriers
            int ru = 0, rk = 0, rf = 0;  // round of the slot: iteration j is its (r+1)-th use
            int j = 0;
            for (; j < niter; ++j) {
                if (*abort_flag) break;
                // Before its (r+1)-th use a slot must have been released r times:
                // empF -- every consumer has waited on the phase of full[jf] that
                // this iteration re-arms, so at most DF iterations are ever in
                // flight; empU / empK -- every consumer is done reading the slot.
                bool ok = true;
                if (rf > 0) ok = mbar_wait_bounded(empF + jf, (uint32_t)((rf - 1) & 1));
                if constexpr (!S::SPLIT)
                    if (ok && ru > 0) ok = mbar_wait_bounded(empU + ju, (uint32_t)((ru - 1) & 1));
                if (ok && rk > 0) ok = mbar_wait_bounded(empK + jk, (uint32_t)((rk - 1) & 1));
                if (!ok) {
                    *abort_flag = 1;
                    atomicMin(a.status, -4 /* WAVE_ETIMEOUT */);
                    break;
                }
                const int c0 = c00 + j;
                uint64_t *bf = full + jf;
                // (u^{n-1}, B, C) of plane c0 - R are first read by stage 1 at
                // iteration 2R: the ring-K slots of earlier iterations stay unused
                const bool kload = j >= 2 * R;
                unsigned char *kslot = ringK + (size_t)jk * S::KSLOT;
                mbar_expect_tx(bf, kload ? S::TXB : S::TX0);
                if constexpr (S::SPLIT) {
                    // level n of plane c0 for the x-queue (rows of the threads
                    // only), and from 2R on the centre plane c0 - R with halo
                    tma_load_3d(kslot + S::K_F, &mp.uk, gz0, gy0 + R, c0, bf);
                    if (kload) tma_load_3d(kslot + S::K_U, &mp.u, gz0 - S::RP, gy0, c0 - R, bf);
                } else {
                    tma_load_3d(ringU + (size_t)ju * (S::USLOT / 4), &mp.u, gz0 - S::RP, gy0, c0, bf);
                }
                if (kload) {
                    tma_load_3d(kslot + S::K_UM, &mp.um, gz0, gy0 + R, c0 - R, bf);
                    tma_load_3d(kslot + S::K_B, &mp.B, gz0, gy0 + R, c0 - R, bf);
                    tma_load_3d(kslot + S::K_C, &mp.C, gz0, gy0 + R, c0 - R, bf);
                    if constexpr (XB >= 1) tma_load_3d(kslot + S::K_X0, &mp.x0, gz0, gy0 + R, c0 - R, bf);
                    if constexpr (XB >= 2) tma_load_3d(kslot + S::K_X1, &mp.x1, gz0, gy0 + R, c0 - R, bf);
                }
                if constexpr (!S::SPLIT)
                    if (++ju == S::DU) { ju = 0; ++ru; }
                if (++jk == S::DK) { jk = 0; ++rk; }
                if (++jf == S::DF) { jf = 0; ++rf; }
            }
            // make sure no copy into this block's shared memory is still in
            // flight (only the last DF issued iterations can be)
            for (int i = (j > S::DF ? j - S::DF : 0); i < j; ++i)
                mbar_wait_bounded(full + i % S::DF, (uint32_t)((i / S::DF) & 1));
        }
        return;
    }

    // ------------------------------ consumer threads ------------------------------
    // Register queues, one per stage: q[s-1] holds level n+s-1 (stage s's
    // input) on the 2R+1 planes around stage s's centre, oldest first
    // (q[.][R] is the centre).  A push shifts the queue by one register pair
    // per entry: a few moves per plane, but one copy of the loop body, whose
    // instruction footprint a (2R+1)-fold unroll for compile-time rotation
    // would multiply.
    constexpr int V2 = V / 2;  // point pairs per thread: arithmetic in paired FP32
    float2 q[T][QL][V2];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int k = 0; k < QL; ++k)
#pragma unroll
            for (int j = 0; j < V2; ++j) q[s][k][j] = make_float2(0.f, 0.f);

    const bool lane0 = (tid & 31) == 0;
    int su = 0, sk = 0, sf = 0;  // ring slots of the current iteration
    uint32_t pf = 0;             // parity of the current full barrier phase
    int cur = 0;
    bool stop = false;
#pragma unroll 1
    for (int it = 0; it < niter && !stop; ++it) {
        {
            // T == 1 has no per-plane consumer barrier: every 8 planes each
            // warp checks, at a warp-uniform point, whether a wait anywhere in
            // the block ran out (its own expired waits stop it at once)
            if (T == 1 && (it & 7) == 0 && __any_sync(0xffffffffu, *abort_flag != 0)) {
                stop = true;
                break;
            }
            const int c0 = c00 + it;
            const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(full + sf, pf));
            if (!got) {
                if (lane0) {
                    *abort_flag = 1;
                    atomicMin(a.status, -4 /* WAVE_ETIMEOUT */);
                }
                if (T == 1) {  // T > 1: decided at the consumer barrier
                    stop = true;
                    break;
                }
            }
            if (lane0) mbar_arrive(empF + sf);  // this warp is past this phase of full[sf]
            // level n of plane c0 enters stage 1's queue (replacing its oldest)
            #pragma unroll
            for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                for (int j = 0; j < V2; ++j) q[0][k][j] = q[0][k + 1][j];
            const unsigned char *kslot = ringK + (size_t)sk * S::KSLOT;
            int suc = 0;  // ring-U slot of plane c0 - R (T > 1)
            if constexpr (S::SPLIT) {
                ld2<V>(q[0][QL - 1], reinterpret_cast<const float *>(kslot + S::K_F) + ownK);
            } else {
                ld2<V>(q[0][QL - 1], ringU + (size_t)su * (S::USLOT / 4) + ownU);
                suc = su - R < 0 ? su - R + S::DU : su - R;
            }

#pragma unroll
            for (int s = 1; s <= T; ++s) {
                float2(&qs)[QL][V2] = q[s - 1];
                const int cs = c0 - s * R;  // plane computed by stage s
                // rows this stage computes, and only once the item's own planes
                // fill its x-queue (local iteration 2sR on); earlier iterations
                // would only produce planes no later stage or store reads
                // (T = 1: every thread row is a stage-1 row)
                const bool rowok = (T == 1 || (row >= s * R && row < S::H0 - s * R)) && it >= 2 * s * R;
                const long long pidx = (long long)cs * a.sx + yz;  // 32 x 32 -> 64-bit product
                float2 un[V2], dd[V2];
#pragma unroll
                for (int j = 0; j < V2; ++j) { un[j] = make_float2(0.f, 0.f); dd[j] = un[j]; }
                const int kk = sk - (s - 1) * R;
                const unsigned char *ks = ringK + (size_t)(kk < 0 ? kk + S::DK : kk) * S::KSLOT;
                if (rowok) {
                    float2 cBv[V2], cCv[V2], up[V2], lap[V2];
                    ld2<V>(cBv, reinterpret_cast<const float *>(ks + S::K_B) + ownK);
                    ld2<V>(cCv, reinterpret_cast<const float *>(ks + S::K_C) + ownK);
                    // centre plane of stage s: ring U (s = 1) or the exchanged plane
                    const float *Pc = s == 1 ? (S::SPLIT ? reinterpret_cast<const float *>(ks + S::K_U)
                                                         : ringU + (size_t)suc * (S::USLOT / 4))
                                             : splane + ((s - 2) * 2 + cur) * S::PLANE;
                    // z window of the thread: pairs at even offsets (zz) and at odd
                    // offsets (zo = (z[2i+1], z[2i+2])); own points start at RP
                    float2 zz[ZW / 2], zo[ZW / 2 - 1];
#pragma unroll
                    for (int j = 0; j < ZW / V; ++j) ld2<V>(zz + j * V2, Pc + ownU - S::RP + j * V);
#pragma unroll
                    for (int i = 0; i < ZW / 2 - 1; ++i) zo[i] = make_float2(zz[i].y, zz[i + 1].x);
                    const int qc = R;  // centre
                    // R >= 3: three independent accumulation chains (centre and x,
                    // y, z), summed at the end, L u = (lx + ly) + lz, for latency;
                    // R <= 2: one chain, in the order centre, then per k x, y, z
                    float2 ly[V2], lz[V2];
#pragma unroll
                    for (int k = 1; k <= R; ++k) {
                        float2 yp[V2], ym[V2];
                        ld2<V>(yp, Pc + ownU + k * S::PW);
                        ld2<V>(ym, Pc + ownU - k * S::PW);
                        const int qp = R + k, qm = R - k;
#pragma unroll
                        for (int j = 0; j < V2; ++j) {
                            const int op = S::RP + 2 * j + k, om = S::RP + 2 * j - k;
                            const float2 zp = (op & 1) ? zo[(op - 1) >> 1] : zz[op >> 1];
                            const float2 zm = (om & 1) ? zo[(om - 1) >> 1] : zz[om >> 1];
                            const float2 sx = __fadd2_rn(qs[qp][j], qs[qm][j]);
                            const float2 sy = __fadd2_rn(yp[j], ym[j]);
                            const float2 sz = __fadd2_rn(zp, zm);
                            if (R <= 2) {
                                if (k == 1) lap[j] = __fmul2_rn(st.cc, qs[qc][j]);
                                lap[j] = __ffma2_rn(st.cx[k], sx, lap[j]);
                                lap[j] = __ffma2_rn(st.cy[k], sy, lap[j]);
                                lap[j] = __ffma2_rn(st.cz[k], sz, lap[j]);
                            } else if (k == 1) {
                                lap[j] = __ffma2_rn(st.cx[1], sx, __fmul2_rn(st.cc, qs[qc][j]));
                                ly[j] = __fmul2_rn(st.cy[1], sy);
                                lz[j] = __fmul2_rn(st.cz[1], sz);
                            } else {
                                lap[j] = __ffma2_rn(st.cx[k], sx, lap[j]);
                                ly[j] = __ffma2_rn(st.cy[k], sy, ly[j]);
                                lz[j] = __ffma2_rn(st.cz[k], sz, lz[j]);
                            }
                        }
                    }
                    if constexpr (R > 2) {
#pragma unroll
                        for (int j = 0; j < V2; ++j) lap[j] = __fadd2_rn(__fadd2_rn(lap[j], ly[j]), lz[j]);
                    }
                    if (s == 1) {
                        ld2<V>(up, reinterpret_cast<const float *>(kslot + S::K_UM) + ownK);  // level n-1
                    } else {
                        // level n+s-2 on plane cs: oldest of stage s-1's queue
#pragma unroll
                        for (int j = 0; j < V2; ++j) up[j] = q[s > 1 ? s - 2 : 0][0][j];
                    }
                    float2 du[V2];  // u^n - u^{n-1}
#pragma unroll
                    for (int j = 0; j < V2; ++j) {
                        const float2 u0 = qs[qc][j];
                        du[j] = fsub2_rn(u0, up[j]);
                        un[j] = __ffma2_rn(cCv[j], lap[j], __ffma2_rn(cBv[j], du[j], u0));
                    }
                    const bool plane_in = cs >= 0 && cs < a.nx;
                    if (a.dstore != nullptr && in_yz && plane_in) {
                        // u^{n+1} - 2u^n + u^{n-1} = E (u^n - u^{n-1}) + C (L u^n + f^n)
                        float2 e[V2];
                        if constexpr (XB == 1)
                            ld2<V>(e, reinterpret_cast<const float *>(ks + S::K_X0) + ownK);
                        else
                            ldg2<V>(e, a.cE + pidx);
#pragma unroll
                        for (int j = 0; j < V2; ++j)
                            dd[j] = __ffma2_rn(cCv[j], lap[j], __fmul2_rn(e[j], du[j]));
                    }
                    // point sources: f = sum_s w q_s (ascending source order), u += C f
                    if (any_inj && finj[cs - pbase] && in_yz) {
                        const int e0 = pinj[cs - pbase], e1 = pinj[cs - pbase + 1];
                        // each grid point appears at most once in the table, but up
                        // to V table points can fall in this thread's V z-points
                        float fv[V];
                        unsigned hits = 0u;
#pragma unroll
                        for (int j = 0; j < V; ++j) fv[j] = 0.f;
                        // the value each entry injects at this trace row, summed
                        // once per call (inj.f), loaded beside the entries
                        const float *frow = a.inj.f + (long long)(a.q_row0 + a.q_dir * (s - 1)) * a.inj.fstride;
                        for (int eb = e0; eb < e1; eb += 4) {
                            // four table points ((y, z), the first half of each
                            // record) and their values per round trip
                            int2 pt4[4];
                            float f4[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                pt4[u] = eb + u < e1 ? __ldg(reinterpret_cast<const int2 *>(a.inj.pts + eb + u))
                                                     : make_int2(-1, -1);
                                f4[u] = eb + u < e1 ? __ldg(frow + eb + u) : 0.f;
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int2 pt = pt4[u];
                                if (pt.x != gy || pt.y < gz || pt.y >= gz + V) continue;
                                const float f = f4[u];
                                const int jj = pt.y - gz;
#pragma unroll
                                for (int j = 0; j < V; ++j) fv[j] = jj == j ? f : fv[j];
                                hits |= 1u << jj;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < V; ++j)
                            if (hits & (1u << j)) {
                                float &uj = (j & 1) ? un[j >> 1].y : un[j >> 1].x;
                                float &dj = (j & 1) ? dd[j >> 1].y : dd[j >> 1].x;
                                const float cj = (j & 1) ? cCv[j >> 1].y : cCv[j >> 1].x;
                                uj = __fmaf_rn(cj, fv[j], uj);
                                dj = __fmaf_rn(cj, fv[j], dj);
                            }
                    }
                }
                const bool own_pt = inner && cs >= X0 && cs < X1;
                if (own_pt) {
                    // stages that store their level (s >= T-1) record after the sweep
                    if (s < T - 1 && any_rec && frec[cs - pbase]) {
                        const int e0 = prec[cs - pbase], e1 = prec[cs - pbase + 1];
                        for (int eb = e0; eb < e1; eb += 4) {
                            int4 pt4[4];  // four table points per round trip
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                pt4[u] = eb + u < e1 ? __ldg(a.rec.pts + eb + u) : make_int4(-1, -1, 0, 0);
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int4 pt = pt4[u];
                                if (pt.x != gy || pt.y < gz || pt.y >= gz + V) continue;
                                const int jj = pt.y - gz;
                                float v = un[0].x;
#pragma unroll
                                for (int j = 1; j < V; ++j) v = jj == j ? ((j & 1) ? un[j >> 1].y : un[j >> 1].x) : v;
                                const long long crow = (long long)(a.c_row0 + a.c_dir * (s - 1)) * a.nslot;
                                // corner slots two at a time (read-only loads ahead of the stores)
                                int itm = pt.z;
                                for (; itm + 1 < pt.w; itm += 2) {
                                    const int s0 = __ldg(a.rec.item + itm), s1 = __ldg(a.rec.item + itm + 1);
                                    a.corner[crow + s0] = v;
                                    a.corner[crow + s1] = v;
                                }
                                if (itm < pt.w) a.corner[crow + __ldg(a.rec.item + itm)] = v;
                            }
                        }
                    }
                    if (s == T) st2<V>(a.out_hi + pidx, un);
                    if (T >= 2 && s == T - 1) st2<V>(a.out_lo + pidx, un);
                    if (a.dstore != nullptr)
                        st2<V>(a.dstore + (a.d_row0 + (long long)a.d_dir * (s - 1)) * a.npad + pidx, dd);
                    if (a.gacc != nullptr) {
                        float2 dl[V2], g[V2];
                        if constexpr (XB == 2) {
                            ld2<V>(dl, reinterpret_cast<const float *>(ks + S::K_X0) + ownK);
                            ld2<V>(g, reinterpret_cast<const float *>(ks + S::K_X1) + ownK);
                        } else {
                            ldg2<V>(dl, a.dload + (a.l_row0 + (long long)a.l_dir * (s - 1)) * a.npad + pidx);
                            ld2<V>(g, a.gacc + pidx);
                        }
#pragma unroll
                        for (int j = 0; j < V2; ++j) g[j] = __ffma2_rn(un[j], dl[j], g[j]);
                        st2<V>(a.gacc + pidx, g);
                    }
                }
                if (s < T) {
                    // level n+s of plane cs enters stage s+1's queue (dropping its oldest)
                    float2(&qn)[QL][V2] = q[s < T ? s : 0];
#pragma unroll
                    for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                        for (int j = 0; j < V2; ++j) qn[k][j] = qn[k + 1][j];
#pragma unroll
                    for (int j = 0; j < V2; ++j) qn[QL - 1][j] = un[j];
                }
            }

            // release the ring slots read for the last time: U slot of plane
            // c0 - R (iteration it - R), K slot read by stage T (iteration it -
            // (T-1)R).  Slots of iterations before 0 were never filled.
            __syncwarp();
            if (lane0) {
                if constexpr (!S::SPLIT)
                    if (it >= R) mbar_arrive(empU + suc);
                if (it >= (T - 1) * R) {
                    const int kk = sk - (T - 1) * R;
                    mbar_arrive(empK + (kk < 0 ? kk + S::DK : kk));
                }
            }
            if constexpr (T > 1) {
                // centres of stages >= 2 for the next iteration (position R+1)
#pragma unroll
                for (int s = 2; s <= T; ++s)
                    st2<V>(splane + ((s - 2) * 2 + (cur ^ 1)) * S::PLANE + ownU, q[s - 1][R + 1]);
                const bool halt = consumer_sync_any(S::NT, *abort_flag != 0);
                cur ^= 1;
                if (halt) {
                    stop = true;
                    break;
                }
            }
            if constexpr (!S::SPLIT)
                if (++su == S::DU) su = 0;
            if (++sk == S::DK) sk = 0;
            if (++sf == S::DF) { sf = 0; pf ^= 1u; }
        }
    }

    // Receiver corners of the stored levels (stage T: out_hi, stage T-1:
    // out_lo), once the block's own points are written: the consumer threads
    // share out the record entries of the block's own planes, so the few
    // blocks holding receivers do not pay a chain of table loads per plane.
    if (any_rec) {  // block-uniform; every consumer thread has left the loop
        asm volatile("bar.sync 1, %0;" ::"r"(S::NT) : "memory");
        const int k0 = X0 - pbase, k1 = X1 - pbase;  // own planes in the plane slices
        const int E0 = prec[k0], E1 = prec[k1];      // their table entries, contiguous
        for (int e = E0 + tid; e < E1; e += S::NT) {
            int lo = k0, hi = k1 - 1;  // plane of entry e: last k with prec[k] <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prec[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int4 pt = __ldg(a.rec.pts + e);
            if (pt.x < gy0 + S::RT || pt.x >= gy0 + S::RT + BY || pt.y < gz0 + S::A0 || pt.y >= gz0 + S::A0 + BZ)
                continue;
            const long long pix = (long long)(pbase + lo) * a.sx + (long long)pt.x * a.nz + pt.y;
#pragma unroll
            for (int st = (T > 1 ? T - 1 : 1); st <= T; ++st) {
                const float v = (st == T ? a.out_hi : a.out_lo)[pix];  // written by this block
                const long long crow = (long long)(a.c_row0 + a.c_dir * (st - 1)) * a.nslot;
                for (int itm = pt.z; itm < pt.w; ++itm) a.corner[crow + __ldg(a.rec.item + itm)] = v;
            }
        }
    }
}

// One problem per launch: arguments and TMA descriptors in parameter space.
template <int R, int T, int V, int BZ, int BY, int P, int MB, int XB = 0>
__global__ void __launch_bounds__(SweepShape<R, T, V, BZ, BY, P, MB, XB>::NTB, MB)
sweep_kernel(const __grid_constant__ SweepArgs a, const __grid_constant__ Stencil st,
             const __grid_constant__ SweepMaps mp)
{
    sweep_block<R, T, V, BZ, BY, P, MB, XB>(a, st, mp, blockIdx.x);
}

// One shot of a batched launch, in device memory: its arguments and TMA
// descriptors for both parities of its ping-pong buffers (the row fields of
// the arguments hold the rows of step 0).
struct ShotSweep {  // 128-byte aligned, as its tensor maps
    SweepMaps mp[2];
    SweepArgs a[2];
};

// Every shot of a batch advanced by one launch: block i sweeps tile
// block_map[i].y of shot block_map[i].x (tiles holding sparse points of any
// shot first), the launch is time step `step` of all shots, and `parity`
// selects their buffers.  The shots share the stencil (grid spacing and space
// order), nt and dt.
template <int R, int T, int V, int BZ, int BY, int P, int MB>
__global__ void __launch_bounds__(SweepShape<R, T, V, BZ, BY, P, MB>::NTB, MB)
sweep_multi_kernel(const ShotSweep *__restrict__ shots, const int2 *__restrict__ block_map,
                   const __grid_constant__ Stencil st, int parity, int step)
{
    using S = SweepShape<R, T, V, BZ, BY, P, MB>;
    const int2 bm = block_map[blockIdx.x];
    const ShotSweep &sh = shots[bm.x];
    if (threadIdx.x == S::NT) {
        // the producer thread's TMA reads these descriptors from global
        // memory, which a host copy may have rewritten since a launch that
        // read the same addresses: acquire them for the tensormap proxy first
        const SweepMaps &m = sh.mp[parity];
        tensormap_acquire(&m.u);
        tensormap_acquire(&m.um);
        tensormap_acquire(&m.B);
        tensormap_acquire(&m.C);
        tensormap_acquire(&m.uk);
    }
    SweepArgs la = sh.a[parity];
    la.q_row0 += la.q_dir * step;
    la.c_row0 += la.c_dir * step;
    la.d_row0 += (long long)la.d_dir * step;
    la.l_row0 += (long long)la.l_dir * step;
    la.order = nullptr;
    sweep_block<R, T, V, BZ, BY, P, MB, 0>(la, st, sh.mp[parity], bm.y);
}

}  // namespace wt
