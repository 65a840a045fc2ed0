// sweep.cuh -- the time-tiled leapfrog sweep for sm_103a.
//
// One launch advances the wavefield by T time steps (T = 1 is the untiled
// sweep).  It realises the paper's time tiling (Sec. 4.1 skewing, Sec. 4.2
// time tiles with min/max bounding) for a GPU:
//
//  * Each block owns an output tile of BZ (z) x BY (y) columns and an x-chunk
//    of `chunk` planes, and streams along x.  Stage s (1..T) computes level
//    n+s on plane c_0 - s*R, where c_0 is the plane of level n loaded in the
//    same iteration: the skew by the stencil radius R per time step of
//    Sec. 4.1, the minimum legal factor (Sec. 2.3.2.1).  The x-dependences
//    of a stage are thereby always already computed, and T time levels are
//    live on chip at once (the time buffer of Sec. 5.2.1).
//  * In y and z, neighbouring blocks read overlapping halos of width R*T and
//    recompute the shrinking halo of each stage, so blocks never wait on one
//    another.  Points outside the grid read as 0 and, because the per-point
//    coefficients B, C are 0 there, are computed as exactly 0: this plays the
//    role of the paper's min/max bounds (Sec. 4.2.2) without branches.
//  * Per thread: one column of V consecutive z points; for every stage a
//    register queue of the 2R+1 x-planes it needs; the centre plane of every
//    stage goes through shared memory (double buffered, one barrier per
//    plane) for the y and z neighbours.
//  * Sources are injected and receiver corners recorded inside the sweep (the
//    imperfectly nested source/receiver loops the paper leaves open,
//    Sec. 4.5.1 and Sec. 6.3.1).
//
// Bit-exactness: every point update is the same sequence of IEEE-rounded
// operations (explicit __fmaf_rn / __fadd_rn / __fsub_rn / __fmul_rn, so no
// contraction choice is left to the compiler), whatever T, tile shape or
// launch split.  Tiled and untiled sweeps therefore agree bitwise, the GPU
// analogue of the paper's verification rule (Sec. 4.3, Sec. 5.4.3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wt {

constexpr int kMaxR = 8;

// Per-axis stencil coefficients c_k / h_a^2 in FP32; cc is the centre
// weight (c_0/hx^2 + c_0/hy^2) + c_0/hz^2 rounded once on the host.
struct Stencil {
    float cc;
    float cx[kMaxR + 1];
    float cy[kMaxR + 1];
    float cz[kMaxR + 1];
};

// Sparse points of one kind, sorted by (x, y, z).  plane_start[x] ..
// plane_start[x+1] index `pts`; each pt = (y, z, item_begin, item_end).
// Injection items: (source index, weight); record items: corner slot.
struct PointTable {
    const int *plane_start;  // [nx + 1] or nullptr (no points)
    const int4 *pts;
    const int *item;
    const float *w;
};

struct SweepArgs {
    int nx, ny, nz;          // nz: padded z extent, a multiple of 4
    long long sx;            // ny * nz
    long long npad;          // nx * ny * nz
    const float *u;          // level n
    const float *um;         // level n-1
    float *out_hi;           // level n+T (T == 1: may alias um, updated in place)
    float *out_lo;           // level n+T-1 (T >= 2)
    const float *cB;         // per point (m-eta)/(m+eta)
    const float *cC;         // per point dt^2/(m+eta)
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
    int chunk;               // x planes per block
    int tiles_z, tiles_y;
};

template <int R, int T, int V, int BZ, int BY>
struct SweepShape {
    static constexpr int RT = R * T;
    static constexpr int A0 = ((RT + 3) / 4) * 4;  // z halo, keeps 16-byte alignment
    static constexpr int W0 = BZ + 2 * A0;         // layout width (z points)
    static constexpr int LZ = W0 / V;              // threads per layout row
    static constexpr int H0 = BY + 2 * RT;         // layout rows (y)
    static constexpr int NT = LZ * H0;             // threads per block
    static constexpr int RP = ((R + V - 1) / V) * V;
    static constexpr int PW = W0 + 2 * RP;         // shared row pitch (floats)
    static constexpr int PLANE = PW * H0;
    static constexpr size_t SMEM = sizeof(float) * 2 * T * PLANE;
    static_assert(BZ % 4 == 0, "BZ must keep 16-byte alignment");
    static_assert(W0 % V == 0, "layout width must be a multiple of V");
    static_assert(NT <= 1024, "too many threads per block");
    static_assert(R >= 1 && R <= kMaxR, "radius out of range");
};

template <int V>
__device__ __forceinline__ void ld_vec(float (&d)[V], const float *p)
{
    if constexpr (V == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        d[0] = t.x; d[1] = t.y;
    } else {
        d[0] = *p;
    }
}

template <int V>
__device__ __forceinline__ void ldg_vec(float (&d)[V], const float *p)
{
    if constexpr (V == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        d[0] = t.x; d[1] = t.y;
    } else {
        d[0] = __ldg(p);
    }
}

template <int V>
__device__ __forceinline__ void st_vec(float *p, const float (&s)[V])
{
    if constexpr (V == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(s[0], s[1], s[2], s[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(s[0], s[1]);
    } else {
        *p = s[0];
    }
}

template <int R, int T, int V, int BZ, int BY>
__global__ void __launch_bounds__(SweepShape<R, T, V, BZ, BY>::NT, 1)
sweep_kernel(const SweepArgs a, const Stencil st)
{
    using S = SweepShape<R, T, V, BZ, BY>;
    constexpr int QL = 2 * R + 1;
    constexpr int ZW = V + 2 * S::RP;  // z window per thread (floats)
    extern __shared__ __align__(16) float smem[];  // [T][2][PLANE]

    const int tid = threadIdx.x;
    const int lane = tid % S::LZ;
    const int row = tid / S::LZ;
    int b = blockIdx.x;
    const int tzi = b % a.tiles_z;
    b /= a.tiles_z;
    const int tyi = b % a.tiles_y;
    const int txi = b / a.tiles_y;
    const int X0 = txi * a.chunk;
    const int X1 = min(X0 + a.chunk, a.nx);
    const int gz = tzi * BZ - S::A0 + lane * V;
    const int gy = tyi * BY - S::RT + row;
    const bool in_yz = gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const bool inner = in_yz && row >= S::RT && row < S::RT + BY &&
                       lane * V >= S::A0 && lane * V < S::A0 + BZ;
    const bool row1 = row >= R && row < S::H0 - R;  // rows stage 1 computes
    const long long yz = in_yz ? (long long)gy * a.nz + gz : 0;
    const int own = row * S::PW + S::RP + lane * V;

    for (int i = tid; i < 2 * T * S::PLANE; i += S::NT) smem[i] = 0.f;

    float q[T][QL][V];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int k = 0; k < QL; ++k)
#pragma unroll
            for (int j = 0; j < V; ++j) q[s][k][j] = 0.f;

    const int niter = (X1 - X0) + 2 * S::RT;
    int c0 = X0 - S::RT;  // plane of level n entering the pipeline this iteration
    float pre_u[V], pre_um[V], um_cur[V];
#pragma unroll
    for (int j = 0; j < V; ++j) { pre_u[j] = 0.f; pre_um[j] = 0.f; }
    if (in_yz && c0 >= 0 && c0 < a.nx) ld_vec<V>(pre_u, a.u + (long long)c0 * a.sx + yz);
    if (in_yz && row1 && c0 - R >= 0 && c0 - R < a.nx)
        ld_vec<V>(pre_um, a.um + (long long)(c0 - R) * a.sx + yz);
    __syncthreads();

    int cur = 0;
    for (int it = 0; it < niter; ++it, ++c0) {
        // level n of plane c0 enters stage 1's queue
#pragma unroll
        for (int k = 0; k < QL - 1; ++k)
#pragma unroll
            for (int j = 0; j < V; ++j) q[0][k][j] = q[0][k + 1][j];
#pragma unroll
        for (int j = 0; j < V; ++j) { q[0][QL - 1][j] = pre_u[j]; um_cur[j] = pre_um[j]; }
        {
            const int cn = c0 + 1, cm = c0 + 1 - R;
#pragma unroll
            for (int j = 0; j < V; ++j) { pre_u[j] = 0.f; pre_um[j] = 0.f; }
            if (in_yz && cn >= 0 && cn < a.nx) ld_vec<V>(pre_u, a.u + (long long)cn * a.sx + yz);
            if (in_yz && row1 && cm >= 0 && cm < a.nx)
                ld_vec<V>(pre_um, a.um + (long long)cm * a.sx + yz);
        }

#pragma unroll
        for (int s = 1; s <= T; ++s) {
            const int cs = c0 - s * R;  // plane computed by stage s
            const bool rowok = row >= s * R && row < S::H0 - s * R;
            const bool plane_in = cs >= 0 && cs < a.nx;
            const long long pidx = (long long)cs * a.sx + yz;
            float un[V], dd[V];
#pragma unroll
            for (int j = 0; j < V; ++j) { un[j] = 0.f; dd[j] = 0.f; }
            float lap[V], cBv[V], cCv[V];
#pragma unroll
            for (int j = 0; j < V; ++j) { lap[j] = 0.f; cBv[j] = 0.f; cCv[j] = 0.f; }
            if (rowok) {
                const float *P = smem + ((s - 1) * 2 + cur) * S::PLANE;
                float zz[ZW / V][V];
#pragma unroll
                for (int j = 0; j < ZW / V; ++j) ld_vec<V>(zz[j], P + own - S::RP + j * V);
#pragma unroll
                for (int j = 0; j < V; ++j) lap[j] = __fmul_rn(st.cc, q[s - 1][R][j]);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    float yp[V], ym[V];
                    ld_vec<V>(yp, P + own + k * S::PW);
                    ld_vec<V>(ym, P + own - k * S::PW);
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        lap[j] = __fmaf_rn(st.cx[k], __fadd_rn(q[s - 1][R + k][j], q[s - 1][R - k][j]), lap[j]);
                        lap[j] = __fmaf_rn(st.cy[k], __fadd_rn(yp[j], ym[j]), lap[j]);
                        lap[j] = __fmaf_rn(st.cz[k],
                                           __fadd_rn(zz[(S::RP + j + k) / V][(S::RP + j + k) % V],
                                                     zz[(S::RP + j - k) / V][(S::RP + j - k) % V]),
                                           lap[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < V; ++j) { cBv[j] = 0.f; cCv[j] = 0.f; }
                if (in_yz && plane_in) {
                    ldg_vec<V>(cBv, a.cB + pidx);
                    ldg_vec<V>(cCv, a.cC + pidx);
                }
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const float u0 = q[s - 1][R][j];
                    const float up = (s == 1) ? um_cur[j] : q[s > 1 ? s - 2 : 0][0][j];
                    un[j] = __fmaf_rn(cCv[j], lap[j], __fmaf_rn(cBv[j], __fsub_rn(u0, up), u0));
                }
                if (a.dstore != nullptr && in_yz && plane_in) {
                    // u^{n+1} - 2u^n + u^{n-1} = E (u^n - u^{n-1}) + C (L u^n + f^n)
                    float e[V];
                    ldg_vec<V>(e, a.cE + pidx);
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        const float u0 = q[s - 1][R][j];
                        const float up = (s == 1) ? um_cur[j] : q[s > 1 ? s - 2 : 0][0][j];
                        dd[j] = __fmaf_rn(cCv[j], lap[j], __fmul_rn(e[j], __fsub_rn(u0, up)));
                    }
                }
                // point sources: f = sum_s w q_s (ascending source order), u += C f
                if (a.inj.plane_start != nullptr && in_yz && plane_in) {
                    // each grid point appears at most once in the table
                    const int e0 = a.inj.plane_start[cs], e1 = a.inj.plane_start[cs + 1];
                    float fv = 0.f;
                    int hit = -1;
                    for (int e = e0; e < e1; ++e) {
                        const int4 pt = a.inj.pts[e];
                        if (pt.x == gy && pt.y >= gz && pt.y < gz + V) {
                            const long long qrow = (long long)(a.q_row0 + a.q_dir * (s - 1)) * a.nq;
                            float f = 0.f;
                            for (int itm = pt.z; itm < pt.w; ++itm)
                                f = __fmaf_rn(a.inj.w[itm], a.q[qrow + a.inj.item[itm]], f);
                            fv = f;
                            hit = pt.y - gz;
                        }
                    }
                    if (hit >= 0) {
#pragma unroll
                        for (int j = 0; j < V; ++j)
                            if (hit == j) {
                                un[j] = __fmaf_rn(cCv[j], fv, un[j]);
                                dd[j] = __fmaf_rn(cCv[j], fv, dd[j]);
                            }
                    }
                }
            }
            const bool own_pt = inner && cs >= X0 && cs < X1;
            if (own_pt) {
                if (a.rec.plane_start != nullptr) {
                    const int e0 = a.rec.plane_start[cs], e1 = a.rec.plane_start[cs + 1];
                    for (int e = e0; e < e1; ++e) {
                        const int4 pt = a.rec.pts[e];
                        if (pt.x == gy && pt.y >= gz && pt.y < gz + V) {
                            float v = 0.f;
#pragma unroll
                            for (int j = 0; j < V; ++j)
                                if (pt.y - gz == j) v = un[j];
                            const long long crow = (long long)(a.c_row0 + a.c_dir * (s - 1)) * a.nslot;
                            for (int itm = pt.z; itm < pt.w; ++itm) a.corner[crow + a.rec.item[itm]] = v;
                        }
                    }
                }
                if (s == T) st_vec<V>(a.out_hi + pidx, un);
                if (T >= 2 && s == T - 1) st_vec<V>(a.out_lo + pidx, un);
                if (a.dstore != nullptr)
                    st_vec<V>(a.dstore + (a.d_row0 + (long long)a.d_dir * (s - 1)) * a.npad + pidx, dd);
                if (a.gacc != nullptr) {
                    float dl[V], g[V];
                    ldg_vec<V>(dl, a.dload + (a.l_row0 + (long long)a.l_dir * (s - 1)) * a.npad + pidx);
                    ld_vec<V>(g, a.gacc + pidx);
#pragma unroll
                    for (int j = 0; j < V; ++j) g[j] = __fmaf_rn(un[j], dl[j], g[j]);
                    st_vec<V>(a.gacc + pidx, g);
                }
            }
            if (s < T) {
#pragma unroll
                for (int k = 0; k < QL - 1; ++k)
#pragma unroll
                    for (int j = 0; j < V; ++j) q[s][k][j] = q[s][k + 1][j];
#pragma unroll
                for (int j = 0; j < V; ++j) q[s][QL - 1][j] = un[j];
            }
        }

        // centres of the next iteration (plane c_s + 1 of each stage's input)
#pragma unroll
        for (int s = 0; s < T; ++s)
            st_vec<V>(smem + (s * 2 + (cur ^ 1)) * S::PLANE + own, q[s][R + 1]);
        __syncthreads();
        cur ^= 1;
    }
}

}  // namespace wt
