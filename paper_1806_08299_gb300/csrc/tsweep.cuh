// tsweep.cuh -- the stage-specialised sweep for sm_103a: one launch advances
// the wavefield by T = 1 or T = 2 time steps, each time step on its own
// group of warps.
//
// This is the paper's time tiling (Sec. 4.1 skewing by the stencil radius,
// Sec. 4.2 time tiles) laid out for a GPU block, with the stages of a tile
// given to different warps instead of one loop nest:
//
//  * A block owns an output tile of BZ (z) x BY (y) columns and an x-chunk
//    [X0, X1) of planes, and streams along x.  In iteration i the level-n
//    plane c0 = X0 - RT + i enters; stage s computes level n+s on plane
//    c0 - sR (the skew by R per time step).  Stage 1 starts at iteration 2R,
//    once its x-queue holds the planes c0 - 2R .. c0; stage 2 at 4R.
//  * Stage 1 (warps [0, N1)) computes level n+1 over the tile widened by R
//    rows and RP columns on each side (T = 2) -- the halo stage 2 reads --
//    or over the tile itself (T = 1, writing level n+1 to global memory).
//    Its inputs arrive through TMA in ring A: the level-n plane c0 for the
//    x-queue, the centre plane c0 - R with the y/z halo of the stencil, and
//    level n-1, B and C on plane c0 - R.
//  * Stage 2 (warps [N1, N1 + N2), T = 2) computes level n+2 over the tile.
//    Stage 1 hands it each plane of level n+1 through ring 1 in shared
//    memory; stage 2 pushes it into its own x-queue and reads the y/z
//    neighbours of its centre plane c0 - 2R, written R iterations earlier,
//    from the same ring.  Level n, B and C of plane c0 - 2R come through TMA
//    in ring B (from L2: ring A loaded them R iterations before).  Stage 2
//    writes levels n+2 and n+1 of the tile.
//  * A producer warp issues the TMA loads: lane 0 fills ring A, lane 1 ring
//    B, each up to P iterations ahead.  Every hand-off is an mbarrier
//    ("full" with transaction counts from the producer or one arrival per
//    stage-1 warp; "empty" with one arrival per consuming warp), so the two
//    stages and the producer run decoupled: stage 1 may run up to D1 - R
//    iterations ahead of stage 2.
//  * Each thread holds VY rows x V z-points.  The x-neighbours come from a
//    register queue of 2R+1 planes, the y-neighbours from shared memory
//    (rows of the thread's own VY rows from the queue centre), the
//    z-neighbours from a window whose middle V points are again the queue
//    centre and whose halos of RP points come from shared memory.  Point
//    pairs at odd z offsets are summed by two scalar additions into a fresh
//    register pair rather than regrouped by moves.
//  * TMA fills everything outside the grid with zeros, and B = C = 0 there,
//    so points outside the grid compute to exactly 0 without branches (the
//    paper's min/max bounds, Sec. 4.2.2).
//  * Every mbarrier wait is bounded by %globaltimer; on expiry the warp
//    records WAVE_ETIMEOUT in the status word, raises the block's abort
//    flag and leaves its loop; the warps waiting on it run out in turn, and
//    the producer waits (bounded) for its copies in flight before exiting.
//
// Bit-exactness: every point update is the sequence of IEEE-rounded
// operations of sweep.cuh (same chains, same order), so this kernel, the
// sweep of sweep.cuh, every T and every tile agree bit for bit (Sec. 4.3,
// Sec. 5.4.3).
#pragma once
#include "sweep.cuh"

namespace wt {

// TMA descriptors of the stage-specialised sweep (all [nx][ny][nzp] float32).
struct TMaps {
    CUtensorMap uc;         // level n, centre box (WC x HC) of stage 1
    CUtensorMap uf, um;     // level n and n-1 over the stage-1 region (W1 x H1)
    CUtensorMap B, C;       // coefficients over the stage-1 region
    CUtensorMap u2, B2, C2; // level n and coefficients over the output tile (BZ x BY), T = 2
    // gradient modes: stage-1 boxes x0, x1 (W1 x H1), stage-2 boxes y0..y2 (BZ x BY):
    //   MODE 1: x0 = E; y0 = E (T = 2)
    //   MODE 2: T = 1: x0 = D row l_row0, x1 = G;  T = 2: y0, y1 = D rows l_row0,
    //           l_row0 + l_dir, y2 = G
    //   MODE 3: T = 1: x0 = D row l_row0, x1 = P (Born source coefficient)
    //   MODE 4 (two-step Adams-Bashforth heat): um is the rate F^{n-1}; B and
    //           the stage-2 boxes u2, B2 are not loaded
    //   MODE 5 (fused Born, T = 1): x0 = E, x1 = P; the perturbation field's
    //           centre box y0 (WC x HC), its level n y1 and n-1 y2 (W1 x H1)
    // The D maps cover the whole store [rows][nx][ny][nzp] as one tensor of
    // rows * nx planes: row r, plane x is plane r * nx + x.  Every D box lies
    // in [X0, X1) in x, so none reaches into a neighbouring row, and one map
    // serves every step (the batched kernel reads it from a per-shot table).
    CUtensorMap x0, x1, y0, y1, y2;
};

// Threads per row group of a stage whose rows hold lz threads: lz rounded up
// to whole 8-lane phases of a 16-byte shared-memory access when that adds no
// warp, else lz.  A phase that straddles two rows meets the far end of the
// other row in the same banks (rows 64 + 8 floats wide: a two-way conflict on
// a quarter of the phases); with whole phases per row every access of a
// phase is 32 consecutive floats.
constexpr int tstage_row_threads(int lz, int ly)
{
    return ((lz + 7) / 8 * 8 * ly + 31) / 32 == (lz * ly + 31) / 32 ? (lz + 7) / 8 * 8 : lz;
}

// Place thread t of a stage on its grid of ly row groups of lzp thread slots,
// lz of them real: act tells whether it owns points; a slot past lz in its row
// repeats column c - 8 of the same row (in a bank group its phase does not
// use), a thread past the grid repeats thread 0.
__device__ __forceinline__ void tstage_place(int t, int lz, int lzp, int ly, bool &act, int &row, int &col)
{
    const bool in = t < lzp * ly;
    if (!in) t = 0;
    row = t / lzp;
    col = t - row * lzp;
    act = in && col < lz;
    if (col >= lz) col -= 8;
}

template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE = 0>
struct TShape {
    static constexpr int RT = R * T;
    static constexpr int RP = (R + 3) / 4 * 4;            // z halo of one stencil, 16-byte aligned
    static constexpr int H1 = BY + 2 * (T - 1) * R;       // stage-1 rows
    static constexpr int W1 = BZ + 2 * (T - 1) * RP;      // stage-1 columns (ring-1 pitch)
    static constexpr int HC = H1 + 2 * R;                 // centre box rows
    static constexpr int WC = W1 + 2 * RP;                // centre box columns (pitch)
    static constexpr int LZ1 = W1 / V, LY1 = H1 / VY;     // stage-1 thread grid
    static constexpr int LZ1P = tstage_row_threads(LZ1, LY1);
    static constexpr int N1 = (LZ1P * LY1 + 31) / 32 * 32;
    static constexpr int LZ2 = BZ / V, LY2 = BY / VY;     // stage-2 thread grid
    static constexpr int LZ2P = tstage_row_threads(LZ2, LY2);
    static constexpr int N2 = T == 2 ? (LZ2P * LY2 + 31) / 32 * 32 : 0;
    // MB = 0: one block per SM whose consumer warps take over the registers
    // of a producer warpgroup (setmaxnreg).  Each quarter of an SM has its
    // own 16K registers for every fourth warp, so a block of 8 consumer
    // warps and a producer warp is capped at 168 registers per thread; with
    // the producer widened to a warpgroup (one warp of it works) that gives
    // up all but PREG, the consumers run with CREG.
    static constexpr bool RSPLIT = MB == 0;
    static constexpr int MINB = RSPLIT ? 1 : MB;          // __launch_bounds__ minimum
    static constexpr int NP = RSPLIT ? 128 : 32;          // producer threads
    static constexpr int NTB = N1 + N2 + NP;
    static constexpr int LREG_ = (65536 / NTB) / 8 * 8;
    static constexpr int LREG = LREG_ > 255 ? 255 : LREG_;  // registers per thread at launch
    static constexpr int PREG = 40;
    static constexpr int CREG_ = ((LREG * NTB - PREG * NP) / (N1 + N2)) / 8 * 8;
    static constexpr int CREG = CREG_ > 232 ? 232 : CREG_;
    // L2 prefetch distance in iterations (0: none).  With one slot of
    // lookahead (P = 1) a ring-A load is issued about one iteration before
    // its use, which does not cover HBM latency, so its inputs are first
    // brought into L2 a few iterations ahead: fewer as an iteration gets
    // longer with the radius (measured on the 512^3 depth-2 tiles, GPts/s at
    // distances 1 / 2 / 3 / 4: so 2 481 / 498 / 503 / 492, so 4 451 / 460 /
    // 452 / 449, so 8 372 / 368 / 364 / 366); with P >= 2 the ring itself
    // covers the latency and the extra requests only cost.
    static constexpr int LP = P == 1 ? (R == 1 ? 3 : R == 2 ? 2 : 1) : 0;
    static constexpr int DA = P + 1;                      // ring A slots
    static constexpr int DB = T == 2 ? P + 1 : 0;         // ring B slots
    static constexpr int D1 = T == 2 ? R + 3 : 0;         // ring 1 planes
    static constexpr bool AB = MODE == 4;                 // two-step Adams-Bashforth (heat)
    static constexpr bool FB = MODE == 5;                 // fused Born: background and perturbation
    static constexpr unsigned CBOX = WC * HC * 4, FBOX = W1 * H1 * 4, SBOX = BZ * BY * 4;
    static constexpr unsigned CBOXP = (CBOX + 127) / 128 * 128;
    static constexpr unsigned FBOXP = (FBOX + 127) / 128 * 128;
    static constexpr unsigned SBOXP = (SBOX + 127) / 128 * 128;
    // extra boxes of the gradient modes per ring-A / ring-B slot
    static constexpr int XA =
        (MODE == 0 || MODE == 4) ? 0 : (T == 1 ? (MODE >= 3 ? 2 : MODE) : (MODE == 1 ? 1 : 0));
    static constexpr int XBB = T == 2 ? (MODE == 1 ? 1 : (MODE == 2 ? 3 : 0)) : 0;
    // ring A slot: centre box, level n (queue feed), level n-1, B, C, [x0, x1]
    // (AB: the rate F^{n-1} in the level n-1 box, no B box)
    // (FB: then the perturbation's centre box, level n and level n-1)
    static constexpr unsigned A_C = 0, A_F = CBOXP, A_UM = A_F + FBOXP, A_B = AB ? A_UM : A_UM + FBOXP,
                              A_CC = A_B + FBOXP, A_X0 = A_CC + FBOXP, A_X1 = A_X0 + FBOXP,
                              A_C2 = A_X0 + XA * FBOXP, A_F2 = A_C2 + CBOXP, A_UM2 = A_F2 + FBOXP,
                              ASLOT = FB ? A_UM2 + FBOXP : A_X0 + XA * FBOXP;
    // ring B slot: level n, B, C over the output tile, [y0, y1, y2] (AB: C only)
    static constexpr unsigned B_UM = 0, B_B = AB ? 0 : SBOXP, B_C = AB ? 0 : 2 * SBOXP, B_Y0 = 3 * SBOXP,
                              B_Y1 = 4 * SBOXP, B_Y2 = 5 * SBOXP, BSLOT = AB ? SBOXP : (3 + XBB) * SBOXP;
    // ring 1 slot: level n+1 over the stage-1 region (AB: then the rate F^n)
    static constexpr unsigned R1SLOT = (AB ? 2 : 1) * FBOXP;
    static constexpr size_t OFF_B = (size_t)DA * ASLOT;
    static constexpr size_t OFF_1 = OFF_B + (size_t)DB * BSLOT;
    static constexpr size_t OFF_BAR = OFF_1 + (size_t)D1 * R1SLOT;
    static constexpr size_t OFF_P = OFF_BAR + 8 * (2 * DA + 2 * DB + 2 * D1) + 16;
    static constexpr size_t SMEM = OFF_P;                 // + per-plane sparse slices
    static size_t smem_bytes(int chunk) { return OFF_P + sweep_table_bytes(chunk, RT) + 16; }
    static constexpr unsigned TXA = CBOX + ((AB ? 3 : 4) + XA) * FBOX + (FB ? CBOX + 2 * FBOX : 0);  // bytes of a
                                                             // ring-A slot from iteration 2R on
    static constexpr unsigned TXF = (FB ? 2 : 1) * FBOX;     // before (queue fill only)
    static constexpr unsigned TXB = (AB ? 1 : 3 + XBB) * SBOX;
    static_assert(T == 1 || T == 2, "stage-specialised sweep: T = 1 or 2");
    static_assert(V == 4, "four z points per thread (two pairs)");
    static_assert(VY == 1 || VY == 2, "one or two rows per thread");
    static_assert(BZ % 4 == 0 && BY % VY == 0 && H1 % VY == 0, "tile must split into thread blocks");
    static_assert((LZ1P == LZ1 || LZ1 >= 8) && (LZ2P == LZ2 || LZ2 >= 8), "padded rows repeat column c - 8");
    static_assert(R >= 1 && R <= kMaxR, "radius out of range");
    static_assert(WC <= 256 && HC <= 256, "TMA box dimension above 256");
    static_assert(TXA < (1u << 20), "mbarrier tx count");
    static_assert(NTB <= 1024, "too many threads per block");
    static_assert(SMEM <= 215 * 1024, "shared memory above the per-block limit");
    static_assert(MB >= 0 && (size_t)MINB * (SMEM + 4096) <= 228 * 1024 && MINB * NTB <= 2048,
                  "blocks per SM do not fit shared memory or thread slots");
    // the split: warpgroup-aligned roles, the consumers' registers within the
    // block's launch allocation and, per SM quarter, within its 16K
    static_assert(!RSPLIT || ((N1 + N2) % 128 == 0 && CREG >= LREG &&
                              (long long)CREG * (N1 + N2) + (long long)PREG * NP <= (long long)LREG * NTB &&
                              ((N1 + N2) / 128 * CREG + PREG) * 32 <= 16384),
                  "register split does not fit");
    static_assert(MODE >= 0 && MODE <= 5 && ((MODE != 3 && MODE != 5) || T == 1),
                  "mode: 0 plain, 1 second differences, 2 imaging condition, 3 Born source (T = 1), "
                  "4 two-step Adams-Bashforth, 5 fused Born (T = 1)");
};

// Level n+1 of a thread's VY x V points (VY rows, V/2 pairs each) from the
// x-queue q of level n (q[R] = the centre plane at the thread's own points),
// the centre plane pc (shared memory at the thread's first point, pitch PC
// floats) and level n-1, B, C (shared memory at the first point, pitch PK).
// cC receives C for the source injection.  The operations and their order
// are those of sweep_block in sweep.cuh: R <= 2 one chain (centre, then per
// k the x, y, z pair sums); R >= 3 three chains (centre + x), y, z summed as
// (x + y) + z; then u^{n+1} = u^n + B (u^n - u^{n-1}) + C L u^n.
// DD: also the second difference u^{n+1} - 2u^n + u^{n-1} = E (u^n - u^{n-1})
// + C L u^n into dd (before sources), from the caller's e = E, as sweep_block's
// second-difference mode computes it.
template <int R, int V, int VY, int PC, int PK, bool DD = false, bool AB = false>
__device__ __forceinline__ void tstage_update(float2 (&un)[VY][V / 2], float2 (&cC)[VY][V / 2],
                                              const float2 (&q)[2 * R + 1][VY][V / 2], const float *pc,
                                              const float *pum, const float *pB, const float *pCc,
                                              const Stencil &st, const float2 (*e)[V / 2] = nullptr,
                                              float2 (*dd)[V / 2] = nullptr)
{
    constexpr int V2 = V / 2;
    constexpr int RP = (R + 3) / 4 * 4;
    constexpr int ZW = V + 2 * RP;  // z window of a row: halo, own points (queue centre), halo
    float2 lap[VY][V2], ly[VY][V2], lz[VY][V2];
    // z windows, as scalars: w[v][RP .. RP + V) are the row's own points
    float w[VY][ZW];
#pragma unroll
    for (int v = 0; v < VY; ++v) {
#pragma unroll
        for (int i = 0; i < RP / 4; ++i) {
            const float4 l = reinterpret_cast<const float4 *>(pc + v * PC - RP)[i];
            const float4 r = reinterpret_cast<const float4 *>(pc + v * PC + V)[i];
            w[v][4 * i] = l.x; w[v][4 * i + 1] = l.y; w[v][4 * i + 2] = l.z; w[v][4 * i + 3] = l.w;
            w[v][RP + V + 4 * i] = r.x; w[v][RP + V + 4 * i + 1] = r.y;
            w[v][RP + V + 4 * i + 2] = r.z; w[v][RP + V + 4 * i + 3] = r.w;
        }
#pragma unroll
        for (int j = 0; j < V2; ++j) {
            w[v][RP + 2 * j] = q[R][v][j].x;
            w[v][RP + 2 * j + 1] = q[R][v][j].y;
        }
    }
#pragma unroll
    for (int k = 1; k <= R; ++k) {
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            // rows v + k and v - k: the thread's own rows from the queue
            // centre, the others from shared memory (a row shared by two own
            // rows is loaded once: the loads repeat the same address)
            const int dp = v + k, dm = v - k;
            float2 yp[V2], ym[V2];
            if (dp < VY) {
#pragma unroll
                for (int j = 0; j < V2; ++j) yp[j] = q[R][dp < VY ? dp : 0][j];
            } else {
                ld2<V>(yp, pc + dp * PC);
            }
            if (dm >= 0) {
#pragma unroll
                for (int j = 0; j < V2; ++j) ym[j] = q[R][dm >= 0 ? dm : 0][j];
            } else {
                ld2<V>(ym, pc + dm * PC);
            }
#pragma unroll
            for (int j = 0; j < V2; ++j) {
                const float2 u0 = q[R][v][j];
                const float2 sx = __fadd2_rn(q[R + k][v][j], q[R - k][v][j]);
                const float2 sy = __fadd2_rn(yp[j], ym[j]);
                const int a = RP + 2 * j + k, b = RP + 2 * j - k;
                float2 sz;
                if ((k & 1) == 0) {
                    sz = __fadd2_rn(make_float2(w[v][a], w[v][a + 1]), make_float2(w[v][b], w[v][b + 1]));
                } else {
                    sz.x = __fadd_rn(w[v][a], w[v][b]);
                    sz.y = __fadd_rn(w[v][a + 1], w[v][b + 1]);
                }
                if (R <= 2) {
                    if (k == 1) lap[v][j] = __fmul2_rn(st.cc, u0);
                    lap[v][j] = __ffma2_rn(st.cx[k], sx, lap[v][j]);
                    lap[v][j] = __ffma2_rn(st.cy[k], sy, lap[v][j]);
                    lap[v][j] = __ffma2_rn(st.cz[k], sz, lap[v][j]);
                } else if (k == 1) {
                    lap[v][j] = __ffma2_rn(st.cx[1], sx, __fmul2_rn(st.cc, u0));
                    ly[v][j] = __fmul2_rn(st.cy[1], sy);
                    lz[v][j] = __fmul2_rn(st.cz[1], sz);
                } else {
                    lap[v][j] = __ffma2_rn(st.cx[k], sx, lap[v][j]);
                    ly[v][j] = __ffma2_rn(st.cy[k], sy, ly[v][j]);
                    lz[v][j] = __ffma2_rn(st.cz[k], sz, lz[v][j]);
                }
            }
        }
    }
    if constexpr (AB) {
        // the rate's Laplacian only: un = L u^n (the caller adds f and forms
        // the two-step update)
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            ld2<V>(cC[v], pCc + v * PK);
#pragma unroll
            for (int j = 0; j < V2; ++j) {
                if constexpr (R > 2) lap[v][j] = __fadd2_rn(__fadd2_rn(lap[v][j], ly[v][j]), lz[v][j]);
                un[v][j] = lap[v][j];
            }
        }
        return;
    }
#pragma unroll
    for (int v = 0; v < VY; ++v) {
        float2 cB[V2], up[V2];
        ld2<V>(cB, pB + v * PK);
        ld2<V>(cC[v], pCc + v * PK);
        ld2<V>(up, pum + v * PK);
#pragma unroll
        for (int j = 0; j < V2; ++j) {
            if constexpr (R > 2) lap[v][j] = __fadd2_rn(__fadd2_rn(lap[v][j], ly[v][j]), lz[v][j]);
            const float2 u0 = q[R][v][j];
            const float2 du = fsub2_rn(u0, up[j]);
            un[v][j] = __ffma2_rn(cC[v][j], lap[v][j], __ffma2_rn(cB[j], du, u0));
            if constexpr (DD) dd[v][j] = __ffma2_rn(cC[v][j], lap[v][j], __fmul2_rn(e[v][j], du));
        }
    }
}

// The two-step Adams-Bashforth update of a thread's points from the rate
// F^n (in un on entry, sources included), F^{n-1} (fm) and the level u^n
// (the queue centre u0): u^{n+1} = u^n + C (w1 F^n + w0 F^{n-1}).  On return
// un holds u^{n+1} and fn the rate F^n.
template <int V, int VY>
__device__ __forceinline__ void ab2_finish(float2 (&un)[VY][V / 2], float2 (&fn)[VY][V / 2],
                                           const float2 (&cC)[VY][V / 2], const float2 (&fm)[VY][V / 2],
                                           const float2 (&u0)[VY][V / 2], float w1, float w0)
{
    const float2 a1 = make_float2(w1, w1), a0 = make_float2(w0, w0);
#pragma unroll
    for (int v = 0; v < VY; ++v)
#pragma unroll
        for (int j = 0; j < V / 2; ++j) {
            fn[v][j] = un[v][j];
            const float2 rate = __ffma2_rn(a1, fn[v][j], __fmul2_rn(a0, fm[v][j]));
            un[v][j] = __ffma2_rn(cC[v][j], rate, u0[v][j]);
        }
}

// Point sources of plane cs on a thread's VY x V points at global row gy
// (first row) and column gz: u += C f, f = sum of w q_s in ascending source
// order (the injection of sweep_block).  The warp scans the plane's table
// entries together: each lane loads one entry, a ballot keeps those inside the
// warp's rows [wy0, wy1) and columns [wz0, wz1), and every lane tests only
// those against its own points, so warps without a point of the plane pay one
// load and one vote per 32 entries.  Called by whole warps (block-uniform
// condition).  Each grid point appears once in the table, so the order in
// which its entry is met does not matter; its items are summed in order.
template <int V, int VY, bool DD = false>
__device__ __forceinline__ void tstage_inject(float2 (&un)[VY][V / 2], const float2 (&cC)[VY][V / 2],
                                              const SweepArgs &a, int e0, int e1, int gy, int gz, int qrow,
                                              int wy0, int wy1, int wz0, int wz1,
                                              float2 (*dd)[V / 2] = nullptr)
{
    // the value each entry injects at this trace row, summed once per call
    // (inj.f), loaded beside the entries: one round trip per 32 entries
    const float *frow = a.inj.f + (long long)qrow * a.inj.fstride;
    const int lane = threadIdx.x & 31;
    float fv[VY][V];
    unsigned hits[VY];
#pragma unroll
    for (int v = 0; v < VY; ++v) {
        hits[v] = 0u;
#pragma unroll
        for (int j = 0; j < V; ++j) fv[v][j] = 0.f;
    }
    for (int eb = e0; eb < e1; eb += 32) {
        // the entry's (y, z) only: the first half of its table record
        const int2 mine = eb + lane < e1 ? __ldg(reinterpret_cast<const int2 *>(a.inj.pts + eb + lane))
                                         : make_int2(-1, -1);
        const float fmine = eb + lane < e1 ? __ldg(frow + eb + lane) : 0.f;
        const bool rel = mine.x >= wy0 && mine.x < wy1 && mine.y >= wz0 && mine.y < wz1;
        unsigned m = __ballot_sync(0xffffffffu, rel);
        while (m != 0u) {
            const int l = __ffs(m) - 1;
            m &= m - 1u;
            int2 pt;
            pt.x = __shfl_sync(0xffffffffu, mine.x, l);
            pt.y = __shfl_sync(0xffffffffu, mine.y, l);
            const float f = __shfl_sync(0xffffffffu, fmine, l);
            const int v = pt.x - gy, jj = pt.y - gz;
            if (v < 0 || v >= VY || jj < 0 || jj >= V) continue;
#pragma unroll
            for (int vv = 0; vv < VY; ++vv)
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (vv == v && j == jj) fv[vv][j] = f;
            hits[v < VY ? v : 0] |= 1u << jj;
        }
    }
#pragma unroll
    for (int v = 0; v < VY; ++v)
#pragma unroll
        for (int j = 0; j < V; ++j)
            if (hits[v] & (1u << j)) {
                float &uj = (j & 1) ? un[v][j >> 1].y : un[v][j >> 1].x;
                const float cj = (j & 1) ? cC[v][j >> 1].y : cC[v][j >> 1].x;
                uj = __fmaf_rn(cj, fv[v][j], uj);
                if constexpr (DD) {
                    float &dj = (j & 1) ? dd[v][j >> 1].y : dd[v][j >> 1].x;
                    dj = __fmaf_rn(cj, fv[v][j], dj);
                }
            }
}

// Receiver corners of one plane from the values `val` of a thread's VY x V
// points at global row gy and column gz, into corner row crow (entries
// [e0, e1) of the plane's record table; warp-cooperative like
// tstage_inject, called by whole warps; lanes with act false own no point).
// The depth-2 Adams-Bashforth sweep records level n+1 this way, because it
// does not store that level.
template <int V, int VY>
__device__ __forceinline__ void tstage_record(const float2 (&val)[VY][V / 2], const SweepArgs &a, int e0, int e1,
                                              int gy, int gz, bool act, long long crow, int wy0, int wy1, int wz0,
                                              int wz1)
{
    const int lane = threadIdx.x & 31;
    for (int eb = e0; eb < e1; eb += 32) {
        const int4 mine = eb + lane < e1 ? __ldg(a.rec.pts + eb + lane) : make_int4(-1, -1, 0, 0);
        const bool rel = mine.x >= wy0 && mine.x < wy1 && mine.y >= wz0 && mine.y < wz1;
        unsigned m = __ballot_sync(0xffffffffu, rel);
        while (m != 0u) {
            const int l = __ffs(m) - 1;
            m &= m - 1u;
            const int px = __shfl_sync(0xffffffffu, mine.x, l), py = __shfl_sync(0xffffffffu, mine.y, l);
            const int pz = __shfl_sync(0xffffffffu, mine.z, l), pw = __shfl_sync(0xffffffffu, mine.w, l);
            const int v = px - gy, jj = py - gz;
            if (!act || v < 0 || v >= VY || jj < 0 || jj >= V) continue;
            float x = 0.f;
#pragma unroll
            for (int vv = 0; vv < VY; ++vv)
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (vv == v && j == jj) x = (j & 1) ? val[vv][j >> 1].y : val[vv][j >> 1].x;
            for (int itm = pz; itm < pw; ++itm) a.corner[crow + __ldg(a.rec.item + itm)] = x;
        }
    }
}

// The rows [y0, y1) and columns [z0, z1) that the lanes of the calling warp
// cover with their VY x V points at (gy, gz) (whole warp).
template <int V, int VY>
__device__ __forceinline__ void warp_extent(int gy, int gz, int &y0, int &y1, int &z0, int &z1)
{
    y0 = gy;
    y1 = gy + VY;
    z0 = gz;
    z1 = gz + V;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        z0 = min(z0, __shfl_xor_sync(0xffffffffu, z0, o));
        z1 = max(z1, __shfl_xor_sync(0xffffffffu, z1, o));
    }
}

__device__ __forceinline__ void tstage_abort(volatile int *abort_flag, int *status)
{
    *abort_flag = 1;
    atomicMin(status, -4 /* WAVE_ETIMEOUT */);
}

// MODE 0: forward / adjoint.  MODE 1 (the recompute sweep of the gradient):
// each stage also stores the second difference D of its level at its own
// points into row d_row0 + d_dir (s-1) of dstore, from E (cE) read with plain
// loads.  MODE 2 (the adjoint sweep with the imaging condition): the
// accumulator gacc at each own point takes g += level(n+s) D[l_row0 + l_dir
// (s-1)] for s = 1..T in that order; with T = 2 stage 2 does both, its queue
// centre being level n+1 of its own points.  MODE 3 (the perturbation sweep
// of Born modelling, T = 1): the new level takes the dense source C P D of
// the background's second difference D (row l_row0 of dload) with the
// per-point coefficient P = -dm / dt^2, as u^{n+1} + C (P D).  MODE 4 (the
// two-step Adams-Bashforth heat operator): level n-1 is replaced by the rate
// F^{n-1} = L u^{n-1} + f^{n-1}; each stage forms F = L u + f and
// u + C (3/2 F - 1/2 F_prev) (stage 1 with the launch's weights ab1, ab0,
// which start the scheme with an Euler step), hands F to stage 2 beside its
// level through ring 1, and the last stage stores the new level (out_hi)
// and its rate (out_lo).  MODE 5 (fused Born, T = 1): MODE 1 and MODE 3 in
// one pass, the background level n+1 to out_hi (its D kept in registers)
// and the perturbation's to out_lo; the receivers record the perturbation.
template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE>
__device__ __forceinline__ void tsweep_block(const SweepArgs &a, const Stencil &st, const TMaps &mp,
                                             const int blk)
{
    using S = TShape<R, T, V, VY, BZ, BY, P, MB, MODE>;
    constexpr int QL = 2 * R + 1, V2 = V / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *ringA = smem_raw;
    unsigned char *ringB = smem_raw + S::OFF_B;
    float *ring1 = reinterpret_cast<float *>(smem_raw + S::OFF_1);
    uint64_t *fullA = reinterpret_cast<uint64_t *>(smem_raw + S::OFF_BAR);
    uint64_t *emptyA = fullA + S::DA;
    uint64_t *fullB = emptyA + S::DA;
    uint64_t *emptyB = fullB + S::DB;
    uint64_t *full1 = emptyB + S::DB;
    uint64_t *empty1 = full1 + S::D1;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty1 + S::D1);

    if (blockDim.x != S::NTB) {  // launched with the wrong shape: report, do nothing
        if (threadIdx.x == 0 && blk == 0) atomicMin(a.status, -1 /* WAVE_EINVAL */);
        return;
    }
    // programmatic dependent launch (see sweep_block)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tid = threadIdx.x;
    int b = a.order != nullptr ? __ldg(a.order + blk) : blk;
    const int tzi = b % a.tiles_z;
    b /= a.tiles_z;
    const int tyi = b % a.tiles_y;
    const int txi = b / a.tiles_y;
    const int X0 = txi * a.chunk;
    const int X1 = min(X0 + a.chunk, a.nx);
    const int ty0 = tyi * BY, tz0 = tzi * BZ;      // output tile origin
    const int gy0 = ty0 - (T - 1) * R;             // stage-1 region origin
    const int gz0 = tz0 - (T - 1) * S::RP;
    const int niter = (X1 - X0) + 2 * S::RT;
    const int c00 = X0 - S::RT;                    // level-n plane of iteration 0

    // Sparse tables of the planes this block visits, [X0 - 2RT, X1 + RT]
    // (as in sweep_block): injection relevant over the stage-1 region,
    // records over the output tile.
    const int pbase = X0 - 2 * S::RT;
    const int plen = (X1 - X0) + 3 * S::RT + 2;
    int *pinj = reinterpret_cast<int *>(smem_raw + S::OFF_P);
    int *prec = pinj + plen;
    unsigned char *finj = reinterpret_cast<unsigned char *>(prec + plen);
    unsigned char *frec = finj + plen;
    int my_inj = 0, my_rec = 0;
    for (int k = tid; k < plen; k += S::NTB) {
        const int cp = min(max(pbase + k, 0), a.nx);
        const int ci = min(max(pbase + k + 1, 0), a.nx);
        int fi = 0, fr = 0;
        if (a.inj.plane_start != nullptr) {
            const int e0 = a.inj.plane_start[cp], e1 = a.inj.plane_start[ci];
            pinj[k] = e0;
            for (int eb = e0; eb < e1 && !fi; eb += 4) {
                int4 pt4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    pt4[u] = eb + u < e1 ? __ldg(a.inj.pts + eb + u) : make_int4(-(1 << 30), -(1 << 30), 0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 pt = pt4[u];
                    fi |= pt.x >= gy0 && pt.x < gy0 + S::H1 && pt.y >= gz0 && pt.y < gz0 + S::W1;
                }
            }
        } else {
            pinj[k] = 0;
        }
        if (a.rec.plane_start != nullptr) {
            const int e0 = a.rec.plane_start[cp], e1 = a.rec.plane_start[ci];
            prec[k] = e0;
            for (int eb = e0; eb < e1 && !fr; eb += 4) {
                int4 pt4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    pt4[u] = eb + u < e1 ? __ldg(a.rec.pts + eb + u) : make_int4(-(1 << 30), -(1 << 30), 0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 pt = pt4[u];
                    fr |= pt.x >= ty0 && pt.x < ty0 + BY && pt.y >= tz0 && pt.y < tz0 + BZ;
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
    if (tid == 0) {
        for (int k = 0; k < S::DA; ++k) {
            mbar_init(fullA + k, 1);
            mbar_init(emptyA + k, S::N1 / 32);
        }
        for (int k = 0; k < S::DB; ++k) {
            mbar_init(fullB + k, 1);
            mbar_init(emptyB + k, S::N2 / 32);
        }
        for (int k = 0; k < S::D1; ++k) {
            mbar_init(full1 + k, S::N1 / 32);
            mbar_init(empty1 + k, S::N2 / 32);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool any_inj = __syncthreads_or(my_inj) != 0;
    const bool any_rec = __syncthreads_or(my_rec) != 0;
    // the previous launch on the stream has completed; every field access
    // below comes after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const bool lane0 = (tid & 31) == 0;
    constexpr unsigned FULL = 0xffffffffu;

    if (tid >= S::N1 + S::N2) {
        // ------------------------------ producer warp ------------------------------
        if constexpr (S::RSPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(S::PREG));
        const int lane = tid - (S::N1 + S::N2);  // lanes 0 and 1 of the first producer warp work
        if (a.withhold) return;
        // plane offsets of this launch's D rows in the store tensor (MODE 2, 3)
        const int xrow = (T == 1 && (MODE == 2 || MODE == 3)) ? (int)(a.l_row0 * a.nx) : 0;
        const int yrow0 = (T == 2 && MODE == 2) ? (int)(a.l_row0 * a.nx) : 0;
        const int yrow1 = (T == 2 && MODE == 2) ? (int)((a.l_row0 + a.l_dir) * a.nx) : 0;
        if (lane == 0) {
            // ring A: the stage-1 inputs of iteration i
            int i = 0, s = 0, r = 0;
            for (; i < niter; ++i) {
                if (*abort_flag) break;
                if (r > 0 && !mbar_wait_bounded(emptyA + s, (uint32_t)((r - 1) & 1))) {
                    tstage_abort(abort_flag, a.status);
                    break;
                }
                const int c0 = c00 + i;
                unsigned char *sl = ringA + (size_t)s * S::ASLOT;
                const bool full_slot = i >= 2 * R;
                mbar_expect_tx(fullA + s, full_slot ? S::TXA : S::TXF);
                tma_load_3d(sl + S::A_F, &mp.uf, gz0, gy0, c0, fullA + s);
                if constexpr (S::FB) tma_load_3d(sl + S::A_F2, &mp.y1, gz0, gy0, c0, fullA + s);
                if (full_slot) {
                    tma_load_3d(sl + S::A_C, &mp.uc, gz0 - S::RP, gy0 - R, c0 - R, fullA + s);
                    tma_load_3d(sl + S::A_UM, &mp.um, gz0, gy0, c0 - R, fullA + s);
                    if constexpr (!S::AB) tma_load_3d(sl + S::A_B, &mp.B, gz0, gy0, c0 - R, fullA + s);
                    tma_load_3d(sl + S::A_CC, &mp.C, gz0, gy0, c0 - R, fullA + s);
                    if constexpr (S::XA >= 1) tma_load_3d(sl + S::A_X0, &mp.x0, gz0, gy0, c0 - R + xrow, fullA + s);
                    if constexpr (S::XA >= 2) tma_load_3d(sl + S::A_X1, &mp.x1, gz0, gy0, c0 - R, fullA + s);
                    if constexpr (S::FB) {
                        tma_load_3d(sl + S::A_C2, &mp.y0, gz0 - S::RP, gy0 - R, c0 - R, fullA + s);
                        tma_load_3d(sl + S::A_UM2, &mp.y2, gz0, gy0, c0 - R, fullA + s);
                    }
                }
                // bring the first-touch inputs of iteration i + LP into L2, so
                // that its loads above wait for L2 rather than HBM (the centre
                // box is the level-n plane that entered as feed R iterations
                // before it is used, and ring B re-reads planes ring A loaded)
                if (S::LP > 0 && i + S::LP < niter) {
                    tma_prefetch_3d(&mp.uf, gz0, gy0, c0 + S::LP);
                    if (i + S::LP >= 2 * R) {
                        tma_prefetch_3d(&mp.um, gz0, gy0, c0 + S::LP - R);
                        if constexpr (!S::AB) tma_prefetch_3d(&mp.B, gz0, gy0, c0 + S::LP - R);
                        tma_prefetch_3d(&mp.C, gz0, gy0, c0 + S::LP - R);
                        if constexpr (S::XA >= 1) tma_prefetch_3d(&mp.x0, gz0, gy0, c0 + S::LP - R + xrow);
                        if constexpr (S::XA >= 2) tma_prefetch_3d(&mp.x1, gz0, gy0, c0 + S::LP - R);
                    }
                }
                if (++s == S::DA) { s = 0; ++r; }
            }
            // no copy into this block's shared memory may still be in flight
            for (int k = (i > S::DA ? i - S::DA : 0); k < i; ++k)
                mbar_wait_bounded(fullA + k % S::DA, (uint32_t)((k / S::DA) & 1));
        } else if (T == 2 && lane == 1) {
            // ring B: level n, B, C over the tile for stage 2 (plane X0 + j)
            const int nj = niter - 4 * R;
            int j = 0, s = 0, r = 0;
            for (; j < nj; ++j) {
                if (*abort_flag) break;
                if (r > 0 && !mbar_wait_bounded(emptyB + s, (uint32_t)((r - 1) & 1))) {
                    tstage_abort(abort_flag, a.status);
                    break;
                }
                unsigned char *sl = ringB + (size_t)s * S::BSLOT;
                mbar_expect_tx(fullB + s, S::TXB);
                if constexpr (!S::AB) {
                    tma_load_3d(sl + S::B_UM, &mp.u2, tz0, ty0, X0 + j, fullB + s);
                    tma_load_3d(sl + S::B_B, &mp.B2, tz0, ty0, X0 + j, fullB + s);
                }
                tma_load_3d(sl + S::B_C, &mp.C2, tz0, ty0, X0 + j, fullB + s);
                if constexpr (S::XBB >= 1) tma_load_3d(sl + S::B_Y0, &mp.y0, tz0, ty0, X0 + j + yrow0, fullB + s);
                if constexpr (S::XBB >= 2) tma_load_3d(sl + S::B_Y1, &mp.y1, tz0, ty0, X0 + j + yrow1, fullB + s);
                if constexpr (S::XBB >= 3) tma_load_3d(sl + S::B_Y2, &mp.y2, tz0, ty0, X0 + j, fullB + s);
                // the gradient-mode arrays are first read here: into L2 ahead
                if constexpr (S::XBB >= 1) {
                    constexpr int LB = S::DB + 3;
                    if (j + LB < nj) {
                        tma_prefetch_3d(&mp.y0, tz0, ty0, X0 + j + LB + yrow0);
                        if constexpr (S::XBB >= 2) tma_prefetch_3d(&mp.y1, tz0, ty0, X0 + j + LB + yrow1);
                        if constexpr (S::XBB >= 3) tma_prefetch_3d(&mp.y2, tz0, ty0, X0 + j + LB);
                    }
                }
                if (++s == S::DB) { s = 0; ++r; }
            }
            if constexpr (T == 2)
                for (int k = (j > S::DB ? j - S::DB : 0); k < j; ++k)
                    mbar_wait_bounded(fullB + k % S::DB, (uint32_t)((k / S::DB) & 1));
        }
        return;
    }

    if constexpr (S::RSPLIT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(S::CREG));
    if (tid < S::N1) {
        // ------------------------------ stage 1 ------------------------------
        bool act;
        int ry, cz;
        tstage_place(tid, S::LZ1, S::LZ1P, S::LY1, act, ry, cz);
        ry *= VY;
        cz *= V;
        const int offF = ry * S::W1 + cz;                 // in stage-1 boxes and ring-1 planes
        const int offC = (ry + R) * S::WC + cz + S::RP;   // in the centre box
        const int gy = gy0 + ry, gz = gz0 + cz;
        int wy0, wy1, wz0, wz1;  // the warp's rows and columns (injection scan)
        warp_extent<V, VY>(gy, gz, wy0, wy1, wz0, wz1);
        float2 q[QL][VY][V2];
        float2 qb[S::FB ? QL : 1][VY][V2];  // FB: the perturbation's x-queue
#pragma unroll
        for (int k = 0; k < QL; ++k)
#pragma unroll
            for (int v = 0; v < VY; ++v)
#pragma unroll
                for (int j = 0; j < V2; ++j) q[k][v][j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < (S::FB ? QL : 1); ++k)
#pragma unroll
            for (int v = 0; v < VY; ++v)
#pragma unroll
                for (int j = 0; j < V2; ++j) qb[k][v][j] = make_float2(0.f, 0.f);
        // T = 1: stage 1 writes level n+1 of its own points (planes [X0, X1)),
        // and with AB the rate F^n beside it (FB: the perturbation's level)
        float *outp = nullptr, *outf = nullptr;
        bool sok[VY];
        if constexpr (T == 1) {
            outp = a.out_hi + ((long long)X0 * a.sx + (long long)gy * a.nz + gz);
            if constexpr (S::AB || S::FB) outf = a.out_lo + ((long long)X0 * a.sx + (long long)gy * a.nz + gz);
#pragma unroll
            for (int v = 0; v < VY; ++v) sok[v] = act && gy + v < a.ny && gz < a.nz;
        }
        int sa = 0;
        uint32_t pa = 0;
        int s1 = 0, r1 = 0;  // ring-1 slot of the next stage-1 plane, and its round
        // unrolled by three: the x-queue shift of each copy becomes register
        // renaming, and only the shift by three at the loop edge moves values
#pragma unroll 3
        for (int i = 0; i < niter; ++i) {
            if (!__all_sync(FULL, mbar_wait_bounded(fullA + sa, pa))) {
                if (lane0) tstage_abort(abort_flag, a.status);
                break;
            }
            const float *sl = reinterpret_cast<const float *>(ringA + (size_t)sa * S::ASLOT);
            // level n of plane c0 enters the x-queue (replacing its oldest)
#pragma unroll
            for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                for (int v = 0; v < VY; ++v)
#pragma unroll
                    for (int j = 0; j < V2; ++j) q[k][v][j] = q[k + 1][v][j];
#pragma unroll
            for (int v = 0; v < VY; ++v) ld2<V>(q[QL - 1][v], sl + S::A_F / 4 + offF + v * S::W1);
            if constexpr (S::FB) {
#pragma unroll
                for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                    for (int v = 0; v < VY; ++v)
#pragma unroll
                        for (int j = 0; j < V2; ++j) qb[k][v][j] = qb[k + 1][v][j];
#pragma unroll
                for (int v = 0; v < VY; ++v) ld2<V>(qb[QL - 1][v], sl + S::A_F2 / 4 + offF + v * S::W1);
            }
            if (i >= 2 * R) {
                float2 un[VY][V2], cC[VY][V2];
                const int cs = c00 + i - R;  // plane of level n+1
                // gradient modes: the points of this plane the stage owns (T = 1:
                // the tile; T = 2: the tile inside the stage-1 region, stage 1's
                // second differences only), their index and E or D, G
                constexpr bool DD1 = MODE == 1 || MODE == 5;  // FB: the background's D, in registers
                bool own[VY];
                long long pix = 0;
                float2 ex[VY][V2], dd[VY][V2];
                if constexpr (S::XA >= 1) {
                    // E (MODE 1) or this step's D row (MODE 2 and 3, T = 1) from the slot
                    pix = (long long)cs * a.sx + (long long)gy * a.nz + gz;
#pragma unroll
                    for (int v = 0; v < VY; ++v) {
                        own[v] = act && cs >= X0 && cs < X1 && gy + v >= ty0 && gy + v < ty0 + BY &&
                                 gy + v < a.ny && gz >= tz0 && gz < tz0 + BZ && gz < a.nz;
                        ld2<V>(ex[v], sl + S::A_X0 / 4 + offF + v * S::W1);
                    }
                }
                tstage_update<R, V, VY, S::WC, S::W1, DD1, S::AB>(un, cC, q, sl + S::A_C / 4 + offC,
                                                                  sl + S::A_UM / 4 + offF, sl + S::A_B / 4 + offF,
                                                                  sl + S::A_CC / 4 + offF, st, ex, dd);
                float2 fn[VY][V2];  // AB: the rate F^n
                if constexpr (S::AB) {
                    // F^n = L u^n + f^n, then u^{n+1} = u^n + C (w1 F^n + w0 F^{n-1})
                    if (any_inj && finj[cs - pbase]) {
                        float2 one[VY][V2];
#pragma unroll
                        for (int v = 0; v < VY; ++v)
#pragma unroll
                            for (int j = 0; j < V2; ++j) one[v][j] = make_float2(1.f, 1.f);
                        tstage_inject<V, VY>(un, one, a, pinj[cs - pbase], pinj[cs - pbase + 1], gy, gz, a.q_row0,
                                             wy0, wy1, wz0, wz1);
                    }
                    float2 fm[VY][V2];
#pragma unroll
                    for (int v = 0; v < VY; ++v) ld2<V>(fm[v], sl + S::A_UM / 4 + offF + v * S::W1);
                    ab2_finish<V, VY>(un, fn, cC, fm, q[R], a.ab1, a.ab0);
                } else if (any_inj && finj[cs - pbase]) {
                    tstage_inject<V, VY, DD1>(un, cC, a, pinj[cs - pbase], pinj[cs - pbase + 1], gy, gz,
                                              a.q_row0, wy0, wy1, wz0, wz1, dd);
                }
                if constexpr (MODE == 1) {
#pragma unroll
                    for (int v = 0; v < VY; ++v)
                        if (own[v]) st2<V>(a.dstore + a.d_row0 * a.npad + pix + (long long)v * a.nz, dd[v]);
                }
                if constexpr (MODE == 2 && T == 1) {
#pragma unroll
                    for (int v = 0; v < VY; ++v)
                        if (own[v]) {
                            float2 g[V2];
                            ld2<V>(g, sl + S::A_X1 / 4 + offF + v * S::W1);
#pragma unroll
                            for (int j = 0; j < V2; ++j) g[j] = __ffma2_rn(un[v][j], ex[v][j], g[j]);
                            st2<V>(a.gacc + pix + (long long)v * a.nz, g);
                        }
                }
                if constexpr (MODE == 3) {
#pragma unroll
                    for (int v = 0; v < VY; ++v) {
                        float2 pb[V2];
                        ld2<V>(pb, sl + S::A_X1 / 4 + offF + v * S::W1);
#pragma unroll
                        for (int j = 0; j < V2; ++j)
                            un[v][j] = __ffma2_rn(cC[v][j], __fmul2_rn(pb[j], ex[v][j]), un[v][j]);
                    }
                }
                float2 vn[VY][V2];  // FB: the perturbation's new level
                if constexpr (S::FB) {
                    // the perturbation sweep of MODE 3 on this plane, with the
                    // background's D from registers instead of a stored row
                    float2 cC2[VY][V2];
                    tstage_update<R, V, VY, S::WC, S::W1>(vn, cC2, qb, sl + S::A_C2 / 4 + offC,
                                                          sl + S::A_UM2 / 4 + offF, sl + S::A_B / 4 + offF,
                                                          sl + S::A_CC / 4 + offF, st);
#pragma unroll
                    for (int v = 0; v < VY; ++v) {
                        float2 pb[V2];
                        ld2<V>(pb, sl + S::A_X1 / 4 + offF + v * S::W1);
#pragma unroll
                        for (int j = 0; j < V2; ++j)
                            vn[v][j] = __ffma2_rn(cC2[v][j], __fmul2_rn(pb[j], dd[v][j]), vn[v][j]);
                    }
                }
                if constexpr (T == 1) {
#pragma unroll
                    for (int v = 0; v < VY; ++v)
                        if (sok[v]) {
                            st2<V>(outp + (long long)v * a.nz, un[v]);
                            if constexpr (S::AB) st2<V>(outf + (long long)v * a.nz, fn[v]);
                            if constexpr (S::FB) st2<V>(outf + (long long)v * a.nz, vn[v]);
                        }
                    outp += a.sx;
                    if constexpr (S::AB || S::FB) outf += a.sx;
                } else {
                    // hand the plane to stage 2 through ring 1
                    if (r1 > 0 && !__all_sync(FULL, mbar_wait_bounded(empty1 + s1, (uint32_t)((r1 - 1) & 1)))) {
                        if (lane0) tstage_abort(abort_flag, a.status);
                        break;
                    }
                    if (act) {
#pragma unroll
                        for (int v = 0; v < VY; ++v) {
                            st2<V>(ring1 + (size_t)s1 * (S::R1SLOT / 4) + offF + v * S::W1, un[v]);
                            if constexpr (S::AB)
                                st2<V>(ring1 + (size_t)s1 * (S::R1SLOT / 4) + S::FBOXP / 4 + offF + v * S::W1, fn[v]);
                        }
                    }
                    __syncwarp();
                    if (lane0) mbar_arrive(full1 + s1);
                    if (++s1 == S::D1) { s1 = 0; ++r1; }
                }
            }
            __syncwarp();
            if (lane0) mbar_arrive(emptyA + sa);
            if (++sa == S::DA) { sa = 0; pa ^= 1u; }
        }
    }

    if constexpr (T == 2) {
        if (tid >= S::N1) {
            // ------------------------------ stage 2 ------------------------------
            bool act;
            int ry, cz;
            tstage_place(tid - S::N1, S::LZ2, S::LZ2P, S::LY2, act, ry, cz);
            ry *= VY;
            cz *= V;
            const int off1 = (ry + R) * S::W1 + cz + S::RP;  // in ring-1 planes
            const int offS = ry * BZ + cz;                   // in ring-B boxes
            const int gy = ty0 + ry, gz = tz0 + cz;
            int wy0, wy1, wz0, wz1;
            warp_extent<V, VY>(gy, gz, wy0, wy1, wz0, wz1);
            bool sok[VY];
#pragma unroll
            for (int v = 0; v < VY; ++v) sok[v] = act && gy + v < a.ny && gz < a.nz;
            const long long o0 = (long long)X0 * a.sx + (long long)gy * a.nz + gz;
            float *oh = a.out_hi + o0, *ol = a.out_lo + o0;
            float2 q[QL][VY][V2];
#pragma unroll
            for (int k = 0; k < QL; ++k)
#pragma unroll
                for (int v = 0; v < VY; ++v)
#pragma unroll
                    for (int j = 0; j < V2; ++j) q[k][v][j] = make_float2(0.f, 0.f);
            int s1 = 0;            // ring-1 slot of the plane stage 1 produced this iteration
            uint32_t p1 = 0;
            int sc = 0;            // ring-1 slot of the centre plane (produced R iterations earlier)
            int sb = 0;
            uint32_t pb = 0;
#pragma unroll 3  // as stage 1
            for (int i = 2 * R; i < niter; ++i) {
                if (!__all_sync(FULL, mbar_wait_bounded(full1 + s1, p1))) {
                    if (lane0) tstage_abort(abort_flag, a.status);
                    break;
                }
                const float *rp = ring1 + (size_t)s1 * (S::R1SLOT / 4);
#pragma unroll
                for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                    for (int v = 0; v < VY; ++v)
#pragma unroll
                        for (int j = 0; j < V2; ++j) q[k][v][j] = q[k + 1][v][j];
#pragma unroll
                for (int v = 0; v < VY; ++v) ld2<V>(q[QL - 1][v], rp + off1 + v * S::W1);
                if (i >= 4 * R) {
                    if (!__all_sync(FULL, mbar_wait_bounded(fullB + sb, pb))) {
                        if (lane0) tstage_abort(abort_flag, a.status);
                        break;
                    }
                    const float *bp = reinterpret_cast<const float *>(ringB + (size_t)sb * S::BSLOT);
                    float2 un[VY][V2], cC[VY][V2];
                    constexpr bool DD1 = MODE == 1;
                    const long long pix = (long long)(c00 + i - 2 * R) * a.sx + (long long)gy * a.nz + gz;
                    float2 ex[VY][V2], dd[VY][V2], d0[VY][V2];
                    if constexpr (MODE != 0) {
                        // E (MODE 1) or the two D rows (MODE 2) from the ring-B slot
#pragma unroll
                        for (int v = 0; v < VY; ++v) {
                            if constexpr (MODE == 1) {
                                ld2<V>(ex[v], bp + S::B_Y0 / 4 + offS + v * BZ);
                            } else {
                                ld2<V>(d0[v], bp + S::B_Y0 / 4 + offS + v * BZ);
                                ld2<V>(ex[v], bp + S::B_Y1 / 4 + offS + v * BZ);
                            }
                        }
                    }
                    tstage_update<R, V, VY, S::W1, BZ, DD1, S::AB>(un, cC, q,
                                                                   ring1 + (size_t)sc * (S::R1SLOT / 4) + off1,
                                                                   bp + S::B_UM / 4 + offS, bp + S::B_B / 4 + offS,
                                                                   bp + S::B_C / 4 + offS, st, ex, dd);
                    const int cs = c00 + i - 2 * R;  // plane of level n+2, in [X0, X1)
                    float2 fn[VY][V2];  // AB: the rate F^{n+1}
                    if constexpr (S::AB) {
                        if (any_inj && finj[cs - pbase]) {
                            float2 one[VY][V2];
#pragma unroll
                            for (int v = 0; v < VY; ++v)
#pragma unroll
                                for (int j = 0; j < V2; ++j) one[v][j] = make_float2(1.f, 1.f);
                            tstage_inject<V, VY>(un, one, a, pinj[cs - pbase], pinj[cs - pbase + 1], gy, gz,
                                                 a.q_row0 + a.q_dir, wy0, wy1, wz0, wz1);
                        }
                        // F^n of the own points: stage 1's rate, in the same ring-1 slot
                        float2 fm[VY][V2];
#pragma unroll
                        for (int v = 0; v < VY; ++v)
                            ld2<V>(fm[v], ring1 + (size_t)sc * (S::R1SLOT / 4) + S::FBOXP / 4 + off1 + v * S::W1);
                        ab2_finish<V, VY>(un, fn, cC, fm, q[R], 1.5f, -0.5f);
                        // level n+1 is not stored: its receivers are recorded
                        // here, from the queue centre (this stage's own points)
                        if (any_rec && frec[cs - pbase])
                            tstage_record<V, VY>(q[R], a, prec[cs - pbase], prec[cs - pbase + 1], gy, gz, act,
                                                 (long long)a.c_row0 * a.nslot, wy0, wy1, wz0, wz1);
                    } else if (any_inj && finj[cs - pbase]) {
                        tstage_inject<V, VY, DD1>(un, cC, a, pinj[cs - pbase], pinj[cs - pbase + 1], gy, gz,
                                                  a.q_row0 + a.q_dir, wy0, wy1, wz0, wz1, dd);
                    }
#pragma unroll
                    for (int v = 0; v < VY; ++v)
                        if (sok[v]) {
                            st2<V>(oh + (long long)v * a.nz, un[v]);
                            // level n+1, or with AB the rate F^{n+1} (level n+1
                            // is not kept; its receivers were recorded above)
                            if constexpr (S::AB)
                                st2<V>(ol + (long long)v * a.nz, fn[v]);
                            else
                                st2<V>(ol + (long long)v * a.nz, q[R][v]);
                            if constexpr (MODE == 1)
                                st2<V>(a.dstore + (a.d_row0 + a.d_dir) * a.npad + pix + (long long)v * a.nz, dd[v]);
                            if constexpr (MODE == 2) {
                                // g += nu^{n+1} D[row 0] (stage 1's level: this
                                // queue's centre), then g += nu^{n+2} D[row 1]
                                float2 g[V2];
                                ld2<V>(g, bp + S::B_Y2 / 4 + offS + v * BZ);
#pragma unroll
                                for (int j = 0; j < V2; ++j) {
                                    g[j] = __ffma2_rn(q[R][v][j], d0[v][j], g[j]);
                                    g[j] = __ffma2_rn(un[v][j], ex[v][j], g[j]);
                                }
                                st2<V>(a.gacc + pix + (long long)v * a.nz, g);
                            }
                        }
                    oh += a.sx;
                    ol += a.sx;
                    __syncwarp();
                    if (lane0) mbar_arrive(emptyB + sb);
                    if (++sb == S::DB) { sb = 0; pb ^= 1u; }
                }
                if (i >= 3 * R) {
                    // the plane produced R iterations ago is read for the last time
                    __syncwarp();
                    if (lane0) mbar_arrive(empty1 + sc);
                    if (++sc == S::D1) sc = 0;
                }
                if (++s1 == S::D1) { s1 = 0; p1 ^= 1u; }
            }
        }
    }

    // Receiver corners of the stored levels (T: out_hi, T-1: out_lo; AB: T
    // only), once the block's own points are written, shared out over the
    // threads of the last stage (see sweep_block).
    constexpr int NL = T == 2 ? S::N2 : S::N1;  // threads of the last stage
    const int tl = T == 2 ? tid - S::N1 : tid;
    if (any_rec && tl >= 0 && tl < NL) {
        asm volatile("bar.sync 1, %0;" ::"r"(NL) : "memory");
        const int k0 = X0 - pbase, k1 = X1 - pbase;
        const int E0 = prec[k0], E1 = prec[k1];
        for (int e = E0 + tl; e < E1; e += NL) {
            int lo = k0, hi = k1 - 1;  // plane of entry e: last k with prec[k] <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prec[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int4 pt = __ldg(a.rec.pts + e);
            if (pt.x < ty0 || pt.x >= ty0 + BY || pt.y < tz0 || pt.y >= tz0 + BZ) continue;
            const long long pix = (long long)(pbase + lo) * a.sx + (long long)pt.x * a.nz + pt.y;
#pragma unroll
            for (int sg = (T > 1 && !S::AB ? T - 1 : T); sg <= T; ++sg) {
                // written by this block (FB: the perturbation's level)
                const float v = (sg == T && !S::FB ? a.out_hi : a.out_lo)[pix];
                const long long crow = (long long)(a.c_row0 + a.c_dir * (sg - 1)) * a.nslot;
                for (int itm = pt.z; itm < pt.w; ++itm) a.corner[crow + __ldg(a.rec.item + itm)] = v;
            }
        }
    }
}

// MB: resident blocks per SM the variant is compiled for (the
// __launch_bounds__ minimum, which caps the registers per thread); 0: one
// block per SM with the registers split between producer and consumers.
template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE = 0>
__global__ void __launch_bounds__(TShape<R, T, V, VY, BZ, BY, P, MB, MODE>::NTB,
                                  TShape<R, T, V, VY, BZ, BY, P, MB, MODE>::MINB)
tsweep_kernel(const __grid_constant__ SweepArgs a, const __grid_constant__ Stencil st,
              const __grid_constant__ TMaps mp)
{
    tsweep_block<R, T, V, VY, BZ, BY, P, MB, MODE>(a, st, mp, blockIdx.x);
}

}  // namespace wt

namespace wt {

// One shot of a batched launch of the stage-specialised sweep, in device
// memory: its arguments and TMA descriptors for both parities of its buffer
// rotation (the row fields of the arguments hold the rows of step 0).
struct ShotTSweep {  // 128-byte aligned, as its tensor maps
    TMaps mp[2];
    SweepArgs a[2];
};

// Every shot of a batch advanced by one launch (T time steps): block i sweeps
// tile block_map[i].y of shot block_map[i].x, the launch starts at time step
// `step` of every shot, and `parity` selects their buffers.  MODE as
// tsweep_block: forward and adjoint sweeps (0), and the gradient's recompute
// (1) and imaging-condition (2) sweeps, whose D rows advance with `step`.
template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE>
__global__ void __launch_bounds__(TShape<R, T, V, VY, BZ, BY, P, MB, MODE>::NTB,
                                  TShape<R, T, V, VY, BZ, BY, P, MB, MODE>::MINB)
tsweep_multi_kernel(const ShotTSweep *__restrict__ shots, const int2 *__restrict__ block_map,
                    const __grid_constant__ Stencil st, int parity, int step)
{
    using S = TShape<R, T, V, VY, BZ, BY, P, MB, MODE>;
    const int2 bm = block_map[blockIdx.x];
    const ShotTSweep &sh = shots[bm.x];
    const int pl = (int)threadIdx.x - (S::N1 + S::N2);  // producer lane
    // the producer lanes' TMA reads these descriptors from global memory,
    // which a host copy may have rewritten since a launch that read the same
    // addresses: each lane acquires the ones it loads through
    const TMaps &m = sh.mp[parity];
    if (pl == 0) {
        tensormap_acquire(&m.uc);
        tensormap_acquire(&m.uf);
        tensormap_acquire(&m.um);
        tensormap_acquire(&m.B);
        tensormap_acquire(&m.C);
        if constexpr (S::XA >= 1) tensormap_acquire(&m.x0);
        if constexpr (S::XA >= 2) tensormap_acquire(&m.x1);
    } else if (T == 2 && pl == 1) {
        tensormap_acquire(&m.u2);
        tensormap_acquire(&m.B2);
        tensormap_acquire(&m.C2);
        if constexpr (S::XBB >= 1) tensormap_acquire(&m.y0);
        if constexpr (S::XBB >= 2) tensormap_acquire(&m.y1);
        if constexpr (S::XBB >= 3) tensormap_acquire(&m.y2);
    }
    SweepArgs la = sh.a[parity];
    la.q_row0 += la.q_dir * step;
    la.c_row0 += la.c_dir * step;
    la.d_row0 += (long long)la.d_dir * step;
    la.l_row0 += (long long)la.l_dir * step;
    la.order = nullptr;
    tsweep_block<R, T, V, VY, BZ, BY, P, MB, MODE>(la, st, m, bm.y);
}

}  // namespace wt
