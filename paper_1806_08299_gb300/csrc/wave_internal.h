// wave_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sweep.cuh"

namespace wt {

// One compiled sweep variant, its layout and its launcher.
struct SweepVariant {
    int R, T, V, BZ, BY, P, threads;  // threads: consumers + the producer warp
    int W0, H0, PW, HK;  // layout width/rows, ring-U pitch, ring-K rows
    size_t smem;         // shared memory without the plane_start slices
    cudaError_t (*launch)(int nblocks, cudaStream_t stream, const SweepArgs &a, const Stencil &st,
                          const SweepMaps &m);
    const void *func;
    int XB;  // extra ring-K boxes of a gradient-mode variant (0: forward and adjoint)
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

// Gradient-mode variants (XB = 1, 2) of radius r; radii without any return 0.
int sweep_mode_variants_r2(const SweepVariant **out);
int sweep_mode_variants_r4(const SweepVariant **out);

// Auxiliary kernels (aux_kernels.cu).  Status codes are written to status[0]
// with atomicMin, so the most severe (most negative) error wins.
cudaError_t launch_prep(const float *m, const float *damp, int nx, int ny, int nz, int nzp,
                        float dt, float stab_lhs, float *cB, float *cC, float *cE, int *status,
                        cudaStream_t s);
cudaError_t launch_pad(const float *src, int nx, int ny, int nz, int nzp, float *dst,
                       cudaStream_t s);
cudaError_t launch_unpad(const float *src, int nx, int ny, int nz, int nzp, float scale,
                         float *dst, cudaStream_t s);
cudaError_t launch_gather(const float *corner, const float *w, int rows, int npts, int row_dir,
                          float *out, cudaStream_t s);

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

#define WAVE_DEFINE_MODES(r_)                                                                     \
    namespace wt {                                                                                \
    static const SweepVariant kModeVariants_r##r_[] = {                                           \
        WAVE_SWEEP_MODE_VARIANTS_R##r_(WAVE_MODE_VARIANT_ENTRY)};                                 \
    int sweep_mode_variants_r##r_(const SweepVariant **out)                                       \
    {                                                                                             \
        *out = kModeVariants_r##r_;                                                               \
        return (int)(sizeof(kModeVariants_r##r_) / sizeof(kModeVariants_r##r_[0]));               \
    }                                                                                             \
    }

#define WAVE_DEFINE_RADIUS(r_)                                                                    \
    namespace wt {                                                                                \
    static const SweepVariant kVariants_r##r_[] = {WAVE_SWEEP_VARIANTS_R##r_(WAVE_VARIANT_ENTRY)}; \
    int sweep_variants_r##r_(const SweepVariant **out)                                            \
    {                                                                                             \
        *out = kVariants_r##r_;                                                                   \
        return (int)(sizeof(kVariants_r##r_) / sizeof(kVariants_r##r_[0]));                       \
    }                                                                                             \
    }
