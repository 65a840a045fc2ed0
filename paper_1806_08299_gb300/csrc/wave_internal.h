// wave_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sweep.cuh"
#include "tsweep.cuh"
#include "wave.h"

namespace wt {

// One compiled sweep variant, its layout and its launcher.  kind 0 is the
// sweep of sweep.cuh (all stages on the same warps; launch, maps SweepMaps),
// kind 1 the stage-specialised sweep of tsweep.cuh (launch_t, maps TMaps).
struct SweepVariant {
    int R, T, V, BZ, BY, P, threads;  // threads: consumers + the producer warp
    int W0, H0, PW, HK;  // kind 0: layout width/rows, ring-U pitch, ring-K rows
    size_t smem;         // shared memory without the plane_start slices
    cudaError_t (*launch)(int nblocks, cudaStream_t stream, const SweepArgs &a, const Stencil &st,
                          const SweepMaps &m);
    const void *func;
    int XB;    // extra ring-K boxes of a gradient-mode variant (0: forward and adjoint)
    int kind;  // 0: sweep.cuh, 1: tsweep.cuh
    int VY;    // rows per thread (kind 1; kind 0: 1)
    int W1, H1, WC, HC;  // kind 1: stage-1 region and centre box (columns, rows)
    cudaError_t (*launch_t)(int nblocks, cudaStream_t stream, const SweepArgs &a, const Stencil &st,
                            const TMaps &m);
};

// Variants of radius r (defined in sweep_r<r>.cu).
int sweep_variants_r1(const SweepVariant **out);
int sweep_variants_r2(const SweepVariant **out);
int sweep_variants_r3(const SweepVariant **out);
int sweep_variants_r4(const SweepVariant **out);
int sweep_variants_r5(const SweepVariant **out);
int sweep_variants_r6(const SweepVariant **out);
int sweep_variants_r7(const SweepVariant **out);
int sweep_variants_r8(const SweepVariant **out);

// Batched variants: the batched kernel for a shape of radius r, one per
// radius (the default untiled shape).
struct MultiVariant {
    int R, T, V, BZ, BY, P, threads;
    size_t smem;  // shared memory without the plane_start slices
    cudaError_t (*launch)(int nblocks, size_t smem, cudaStream_t stream, const ShotSweep *shots,
                          const int2 *block_map, const Stencil &st, int parity, int step);
    const void *func;
};
int sweep_multi_variant_r1(const MultiVariant **out);
int sweep_multi_variant_r2(const MultiVariant **out);
int sweep_multi_variant_r3(const MultiVariant **out);
int sweep_multi_variant_r4(const MultiVariant **out);
int sweep_multi_variant_r5(const MultiVariant **out);
int sweep_multi_variant_r6(const MultiVariant **out);
int sweep_multi_variant_r7(const MultiVariant **out);
int sweep_multi_variant_r8(const MultiVariant **out);

// Batched variants of the stage-specialised sweep (the sweeps of a lockstep
// group: forward with mode 0, the gradient's recompute with mode 1 and its
// imaging-condition adjoint with mode 2), per radius; each has the
// single-shot variant of the same shape and mode (kind 1) for its geometry.
struct TMultiVariant {
    int R, T, V, VY, BZ, BY, P, mode, threads;
    size_t smem;  // shared memory without the plane_start slices
    cudaError_t (*launch)(int nblocks, size_t smem, cudaStream_t stream, const ShotTSweep *shots,
                          const int2 *block_map, const Stencil &st, int parity, int step);
    const void *func;
};
int sweep_tmulti_variants_r1(const TMultiVariant **out);
int sweep_tmulti_variants_r2(const TMultiVariant **out);
int sweep_tmulti_variants_r3(const TMultiVariant **out);
int sweep_tmulti_variants_r4(const TMultiVariant **out);
int sweep_tmulti_variants_r5(const TMultiVariant **out);
int sweep_tmulti_variants_r6(const TMultiVariant **out);
int sweep_tmulti_variants_r7(const TMultiVariant **out);
int sweep_tmulti_variants_r8(const TMultiVariant **out);

// One shot of a batched call: its device memory and its slices of the traces.
struct ShotSlot {
    const wave_shot *shot;
    float *mw, *dw;     // the shot's window of m and damp (unpadded)
    void *ws;           // single-shot workspace (WAVE_OP_FWD or WAVE_OP_GRAD layout)
    size_t ws_bytes;
    float *ckpt;        // checkpoints (gradient) or nullptr
    float *gwin;        // window gradient out, unpadded and scaled (gradient) or nullptr
    const float *q;     // source traces [nt][nsrc_s] or nullptr
    float *rec_out;     // receiver traces out [nt][nrec_s] (forward) or nullptr
    const float *resid; // residual [nt][nrec_s] (gradient) or nullptr
};

// Whether wave_*_batched can run with `tuning` (time_tile 0: the batch's
// forward kernel is chosen by timing) on a batched kernel; ckpt_every as for
// lockstep_group.
bool lockstep_supported(const wave_grid *g, const wave_tuning *tuning, int ckpt_every);
// The kernels of a lockstep group of the n shots: forward (out[0..7] in the
// form of wave_describe_plan, out[8] = 1; all 0 when the group runs per shot,
// out[0] = 0 while an autotuned choice is not made yet) and, for the
// gradient, the recompute and adjoint phases' family and depth (out[9, 10]).
int lockstep_describe(const wave_grid *g, int n, const wave_shot *shots, int ckpt_every,
                      const wave_tuning *tuning, int32_t *out);

// Run a group of shots in lockstep (host runtime, wave_api.cu): the window of
// m and damp is already in each slot (in stream order); every time step is one
// launch of the batched kernel for all shots, and the time loops are one CUDA
// graph launched on `stream`.  Forward (ckpt_every == 0): traces into
// rec_out.  Gradient (ckpt_every >= 1): forward with checkpoints, then per
// segment the recompute and the adjoint with the imaging condition; window
// gradients into gwin.  `table` (table_bytes, from lockstep_table_bytes with
// the same ckpt_every) holds the per-shot launch arguments of every phase.
int lockstep_group(const wave_grid *g, int n, const ShotSlot *slots, int ckpt_every,
                   const wave_tuning *tuning, void *table, size_t table_bytes, cudaStream_t stream);
size_t lockstep_table_bytes(const wave_grid *g, int n, const wave_shot *shots, int ckpt_every);

// Gradient-mode variants (XB = 1, 2) of radius r; radii without any return 0.
int sweep_mode_variants_r1(const SweepVariant **out);
int sweep_mode_variants_r2(const SweepVariant **out);
int sweep_mode_variants_r3(const SweepVariant **out);
int sweep_mode_variants_r4(const SweepVariant **out);
int sweep_mode_variants_r5(const SweepVariant **out);
int sweep_mode_variants_r6(const SweepVariant **out);
int sweep_mode_variants_r7(const SweepVariant **out);
int sweep_mode_variants_r8(const SweepVariant **out);

// Auxiliary kernels (aux_kernels.cu).  Status codes are written to status[0]
// with atomicMin, so the most severe (most negative) error wins.
cudaError_t launch_prep(const float *m, const float *damp, int nx, int ny, int nz, int nzp,
                        float dt, float stab_lhs, float *cB, float *cC, float *cE, int *status,
                        cudaStream_t s);
cudaError_t launch_heat_prep(const float *kappa, int nx, int ny, int nz, int nzp, float dt, float stab,
                             float *cB, float *cC, int *status, cudaStream_t s);
cudaError_t launch_pad(const float *src, int nx, int ny, int nz, int nzp, float *dst,
                       cudaStream_t s, float scale = 1.f);
cudaError_t launch_unpad(const float *src, int nx, int ny, int nz, int nzp, float scale,
                         float *dst, cudaStream_t s);
cudaError_t launch_gather(const float *corner, const float *w, int rows, int npts, int row_dir,
                          float *out, cudaStream_t s);
// F[r][e] (row stride fstride) = the ascending sum of w q[r][item] over the
// items of injection entry e, for rows [0, rows) of traces q [rows][nq].
cudaError_t launch_inj_sum(const int4 *pts, const int *item, const float *w, const float *q, int nq, int ne,
                           int rows, long long fstride, float *F, cudaStream_t s);

// Raise the dynamic shared-memory limit of kernel `func` on the current
// device to the device's opt-in maximum, once per (device, kernel); it is
// never lowered, so occupancy queries and launches of any chunk size agree
// (wave_api.cu).
cudaError_t allow_max_dynamic_smem(const void *func);

template <int R, int T, int V, int BZ, int BY, int P, int MB, int XB = 0>
cudaError_t launch_sweep(int nblocks, cudaStream_t stream, const SweepArgs &a, const Stencil &st,
                         const SweepMaps &m)
{
    using S = SweepShape<R, T, V, BZ, BY, P, MB, XB>;
    const size_t smem = S::smem_bytes(a.chunk);
    cudaError_t e = allow_max_dynamic_smem((const void *)sweep_kernel<R, T, V, BZ, BY, P, MB, XB>);
    if (e != cudaSuccess) return e;
    // programmatic dependent launch: the sweep may start while the previous
    // kernel on the stream finishes (the kernel waits for it before any field
    // access, see sweep.cuh)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)S::NTB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sweep_kernel<R, T, V, BZ, BY, P, MB, XB>, a, st, m);
}

// A register-split shape (MB = 0) relies on its kernel being compiled with
// the launch register count the split assumes; with fewer, the consumers'
// setmaxnreg.inc would wait for registers the block does not hold.  Checked
// once per kernel before its first launch.
template <class S>
cudaError_t check_regsplit(const void *func)
{
    if constexpr (!S::RSPLIT) {
        return cudaSuccess;
    } else {
        static std::atomic<int> state{0};  // 0: not checked, 1: fits, 2: does not
        int s = state.load();
        if (s == 0) {
            cudaFuncAttributes fa;
            const cudaError_t e = cudaFuncGetAttributes(&fa, func);
            if (e != cudaSuccess) return e;
            s = (long long)fa.numRegs * S::NTB >=
                        (long long)S::CREG * (S::N1 + S::N2) + (long long)S::PREG * S::NP
                    ? 1
                    : 2;
            state.store(s);
        }
        return s == 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
    }
}

template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE = 0>
cudaError_t launch_tsweep(int nblocks, cudaStream_t stream, const SweepArgs &a, const Stencil &st,
                          const TMaps &m)
{
    using S = TShape<R, T, V, VY, BZ, BY, P, MB, MODE>;
    const size_t smem = S::smem_bytes(a.chunk);
    cudaError_t e = allow_max_dynamic_smem((const void *)tsweep_kernel<R, T, V, VY, BZ, BY, P, MB, MODE>);
    if (e == cudaSuccess) e = check_regsplit<S>((const void *)tsweep_kernel<R, T, V, VY, BZ, BY, P, MB, MODE>);
    if (e != cudaSuccess) return e;
    // programmatic dependent launch, as launch_sweep
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)S::NTB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tsweep_kernel<R, T, V, VY, BZ, BY, P, MB, MODE>, a, st, m);
}

template <int R, int T, int V, int VY, int BZ, int BY, int P, int MB, int MODE>
cudaError_t launch_tsweep_multi(int nblocks, size_t smem, cudaStream_t stream, const ShotTSweep *shots,
                                const int2 *block_map, const Stencil &st, int parity, int step)
{
    const void *func = (const void *)tsweep_multi_kernel<R, T, V, VY, BZ, BY, P, MB, MODE>;
    cudaError_t e = allow_max_dynamic_smem(func);
    if (e == cudaSuccess) e = check_regsplit<TShape<R, T, V, VY, BZ, BY, P, MB, MODE>>(func);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)TShape<R, T, V, VY, BZ, BY, P, MB, MODE>::NTB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tsweep_multi_kernel<R, T, V, VY, BZ, BY, P, MB, MODE>, shots, block_map,
                              st, parity, step);
}

template <int R, int T, int V, int BZ, int BY, int P, int MB>
cudaError_t launch_sweep_multi(int nblocks, size_t smem, cudaStream_t stream, const ShotSweep *shots,
                               const int2 *block_map, const Stencil &st, int parity, int step)
{
    using S = SweepShape<R, T, V, BZ, BY, P, MB>;
    cudaError_t e = allow_max_dynamic_smem((const void *)sweep_multi_kernel<R, T, V, BZ, BY, P, MB>);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)S::NTB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sweep_multi_kernel<R, T, V, BZ, BY, P, MB>, shots, block_map, st,
                              parity, step);
}

}  // namespace wt

#define WAVE_VARIANT_ENTRY(R_, T_, V_, BZ_, BY_, P_, MB_)                                         \
    {R_, T_, V_, BZ_, BY_, P_, wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::NTB,                \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::W0,                                          \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::H0,                                          \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::PW,                                          \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::HK,                                          \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::SMEM,                                        \
     &wt::launch_sweep<R_, T_, V_, BZ_, BY_, P_, MB_>,                                           \
     (const void *)&wt::sweep_kernel<R_, T_, V_, BZ_, BY_, P_, MB_>, 0},

#define WAVE_MODE_VARIANT_ENTRY(R_, T_, V_, BZ_, BY_, P_, MB_, XB_)                               \
    {R_, T_, V_, BZ_, BY_, P_, wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::NTB,           \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::W0,                                     \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::H0,                                     \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::PW,                                     \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::HK,                                     \
     wt::SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>::SMEM,                                   \
     &wt::launch_sweep<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>,                                      \
     (const void *)&wt::sweep_kernel<R_, T_, V_, BZ_, BY_, P_, MB_, XB_>, XB_},

#define WAVE_TMODE_ENTRY(R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_)                                 \
    {R_, T_, V_, BZ_, BY_, P_, wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::NTB, 0, 0, 0, 0, \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::SMEM, nullptr,                            \
     (const void *)&wt::tsweep_kernel<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>, M_, 1, VY_,         \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::W1,                                       \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::H1,                                       \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::WC,                                       \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::HC,                                       \
     &wt::launch_tsweep<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>},
#define WAVE_TVARIANT_ENTRY(R_, T_, V_, VY_, BZ_, BY_, P_, MB_) \
    WAVE_TMODE_ENTRY(R_, T_, V_, VY_, BZ_, BY_, P_, MB_, 0)

#define WAVE_DEFINE_MULTI(R_, T_, V_, BZ_, BY_, P_, MB_)                                         \
    namespace wt {                                                                                \
    static const MultiVariant kMulti_r##R_ = {                                                    \
        R_, T_, V_, BZ_, BY_, P_, SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::NTB,                  \
        SweepShape<R_, T_, V_, BZ_, BY_, P_, MB_>::SMEM, &launch_sweep_multi<R_, T_, V_, BZ_, BY_, P_, MB_>, \
        (const void *)&sweep_multi_kernel<R_, T_, V_, BZ_, BY_, P_, MB_>};                         \
    int sweep_multi_variant_r##R_(const MultiVariant **out)                                       \
    {                                                                                             \
        *out = &kMulti_r##R_;                                                                     \
        return 1;                                                                                 \
    }                                                                                             \
    }

#define WAVE_TMULTI_ENTRY(R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_)                                 \
    {R_, T_, V_, VY_, BZ_, BY_, P_, M_, wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::NTB,   \
     wt::TShape<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>::SMEM,                                     \
     &wt::launch_tsweep_multi<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>,                             \
     (const void *)&wt::tsweep_multi_kernel<R_, T_, V_, VY_, BZ_, BY_, P_, MB_, M_>},

// the list may be empty: a zero sentinel keeps the array non-empty
#define WAVE_DEFINE_TMULTI(r_)                                                                    \
    namespace wt {                                                                                \
    static const TMultiVariant kTMulti_r##r_[] = {WAVE_TMULTI_VARIANTS_R##r_(WAVE_TMULTI_ENTRY)   \
                                                  {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr, nullptr}}; \
    int sweep_tmulti_variants_r##r_(const TMultiVariant **out)                                    \
    {                                                                                             \
        *out = kTMulti_r##r_;                                                                     \
        return (int)(sizeof(kTMulti_r##r_) / sizeof(kTMulti_r##r_[0])) - 1;                       \
    }                                                                                             \
    }

#define WAVE_DEFINE_MODES(r_)                                                                     \
    namespace wt {                                                                                \
    static const SweepVariant kModeVariants_r##r_[] = {                                           \
        WAVE_SWEEP_MODE_VARIANTS_R##r_(WAVE_MODE_VARIANT_ENTRY)                                    \
            WAVE_TSWEEP_MODE_VARIANTS_R##r_(WAVE_TMODE_ENTRY)};                                     \
    int sweep_mode_variants_r##r_(const SweepVariant **out)                                       \
    {                                                                                             \
        *out = kModeVariants_r##r_;                                                               \
        return (int)(sizeof(kModeVariants_r##r_) / sizeof(kModeVariants_r##r_[0]));               \
    }                                                                                             \
    }

#define WAVE_DEFINE_RADIUS(r_)                                                                    \
    namespace wt {                                                                                \
    static const SweepVariant kVariants_r##r_[] = {WAVE_SWEEP_VARIANTS_R##r_(WAVE_VARIANT_ENTRY) \
                                                   WAVE_TSWEEP_VARIANTS_R##r_(WAVE_TVARIANT_ENTRY)}; \
    int sweep_variants_r##r_(const SweepVariant **out)                                            \
    {                                                                                             \
        *out = kVariants_r##r_;                                                                   \
        return (int)(sizeof(kVariants_r##r_) / sizeof(kVariants_r##r_[0]));                       \
    }                                                                                             \
    }
