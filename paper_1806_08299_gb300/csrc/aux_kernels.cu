// aux_kernels.cu -- per-call preparation and epilogue kernels.
#include <cuda_runtime.h>

#include "wave_internal.h"

namespace wt {

// Model preparation.  From m and damp ([nx][ny][nz], caller layout) it writes
// the per-point coefficients of the update
//   u^{n+1} = u^n + B (u^n - u^{n-1}) + C (L u^n + f^n)
//   B = (m - eta)/(m + eta), C = dt^2/(m + eta), E = -2 eta/(m + eta) = B - 1,
//   eta = damp dt / 2,
// in the z-padded layout [nx][ny][nzp]; the padding (z >= nz) gets B = C = E = 0
// so padded points stay exactly 0.  Points with m <= 0 (or NaN) or damp < 0
// record WAVE_EINVAL; points whose local undamped von Neumann condition
// dt^2 S / m <= 4 fails record WAVE_EUNSTABLE (stab_lhs = dt^2 S, or 0 to skip).
__global__ void prep_kernel(const float *__restrict__ m, const float *__restrict__ damp, int nx,
                            int ny, int nz, int nzp, float dt, float stab_lhs,
                            float *__restrict__ cB, float *__restrict__ cC,
                            float *__restrict__ cE, int *status)
{
    const long long npad = (long long)nx * ny * nzp;
    const float half_dt = 0.5f * dt;
    const float dt2 = __fmul_rn(dt, dt);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npad;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nzp);
        const long long xy = p / nzp;
        float b = 0.f, c = 0.f, e = 0.f;
        if (z < nz) {
            const long long src = xy * nz + z;
            const float mm = m[src], dd = damp[src];
            if (!(mm > 0.f) || !(dd >= 0.f)) {
                atomicMin(status, -1 /* WAVE_EINVAL */);
            } else {
                if (stab_lhs > 0.f && stab_lhs > 4.f * mm) atomicMin(status, -2 /* WAVE_EUNSTABLE */);
                const float eta = __fmul_rn(dd, half_dt);
                const float den = __fadd_rn(mm, eta);
                b = __fdiv_rn(__fsub_rn(mm, eta), den);
                c = __fdiv_rn(dt2, den);
                e = __fdiv_rn(-2.f * eta, den);
            }
        }
        cB[p] = b;
        cC[p] = c;
        if (cE != nullptr) cE[p] = e;
    }
}

// dst = scale src in the z-padded layout, 0 in the padding (scale 1 copies
// the values exactly)
__global__ void pad_kernel(const float *__restrict__ src, int nx, int ny, int nz, int nzp, float scale,
                           float *__restrict__ dst)
{
    const long long npad = (long long)nx * ny * nzp;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npad;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nzp);
        const long long xy = p / nzp;
        dst[p] = z < nz ? __fmul_rn(scale, src[xy * nz + z]) : 0.f;
    }
}

__global__ void unpad_kernel(const float *__restrict__ src, int nx, int ny, int nz, int nzp,
                             float scale, float *__restrict__ dst)
{
    const long long n = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nz);
        const long long xy = p / nz;
        const float v = src[xy * nzp + z];
        dst[p] = scale == 1.f ? v : __fmul_rn(v, scale);
    }
}

// Receiver interpolation from recorded corner values:
//   out[row][r] = sum_{c=0..7} w[r][c] * corner[row'][8r + c]   (c ascending)
// where row' = row (row_dir = +1) or rows-1-row (row_dir = -1, adjoint runs).
__global__ void gather_kernel(const float *__restrict__ corner, const float *__restrict__ w,
                              int rows, int npts, int row_dir, float *__restrict__ out)
{
    const long long total = (long long)rows * npts;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i % npts);
        const int row = (int)(i / npts);
        const int src_row = row_dir > 0 ? row : rows - 1 - row;
        const float *cv = corner + (long long)src_row * 8 * npts + 8LL * r;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc = __fmaf_rn(w[8 * r + c], cv[c], acc);
        out[i] = acc;
    }
}

// Per-entry injection values of every trace row of a call:
//   F[r][e] = sum over the entry's items i (ascending) of w[i] q[r][item[i]]
// the sum the sweep forms when it reaches the entry's plane (the same fused
// multiply-adds in the same order, so the same bits), formed once per call
// instead, so that the sweep's plane loop reads one value per entry.
__global__ void inj_sum_kernel(const int4 *__restrict__ pts, const int *__restrict__ item,
                               const float *__restrict__ w, const float *__restrict__ q, int nq, int ne,
                               int rows, long long fstride, float *__restrict__ F)
{
    const long long total = (long long)rows * ne;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ne);
        const int e = (int)(i - (long long)r * ne);
        const int4 pt = pts[e];
        const float *qr = q + (long long)r * nq;
        float f = 0.f;
        for (int k = pt.z; k < pt.w; ++k) f = __fmaf_rn(w[k], qr[item[k]], f);
        F[(long long)r * fstride + e] = f;
    }
}

static int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

// Heat (Laplace) operator, Sec. 5.7: u^{n+1} = u^n + dt kappa (L u^n + f^n) is
// the leapfrog update with B = 0 and C = dt kappa (kappa = 1 when null).
// Explicit Euler is stable while dt kappa |L| <= 2: stab = dt |L| (0 skips).
__global__ void heat_prep_kernel(const float *__restrict__ kappa, int nx, int ny, int nz, int nzp,
                                 float dt, float stab, float *__restrict__ cB, float *__restrict__ cC,
                                 int *status)
{
    const long long npad = (long long)nx * ny * nzp;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npad;
         p += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(p % nzp);
        const long long xy = p / nzp;
        float c = 0.f;
        if (z < nz) {
            const float k = kappa != nullptr ? kappa[xy * nz + z] : 1.f;
            if (!(k >= 0.f) || !(k < 3.0e38f)) {
                atomicMin(status, -1 /* WAVE_EINVAL */);
            } else {
                if (stab > 0.f && __fmul_rn(k, stab) > 2.f) atomicMin(status, -2 /* WAVE_EUNSTABLE */);
                c = __fmul_rn(dt, k);
            }
        }
        cB[p] = 0.f;
        cC[p] = c;
    }
}

cudaError_t launch_heat_prep(const float *kappa, int nx, int ny, int nz, int nzp, float dt, float stab,
                             float *cB, float *cC, int *status, cudaStream_t s)
{
    heat_prep_kernel<<<grid_for((long long)nx * ny * nzp), 256, 0, s>>>(kappa, nx, ny, nz, nzp, dt, stab,
                                                                       cB, cC, status);
    return cudaGetLastError();
}

cudaError_t launch_prep(const float *m, const float *damp, int nx, int ny, int nz, int nzp,
                        float dt, float stab_lhs, float *cB, float *cC, float *cE, int *status,
                        cudaStream_t s)
{
    prep_kernel<<<grid_for((long long)nx * ny * nzp), 256, 0, s>>>(m, damp, nx, ny, nz, nzp, dt,
                                                                  stab_lhs, cB, cC, cE, status);
    return cudaGetLastError();
}

cudaError_t launch_pad(const float *src, int nx, int ny, int nz, int nzp, float *dst,
                       cudaStream_t s, float scale)
{
    pad_kernel<<<grid_for((long long)nx * ny * nzp), 256, 0, s>>>(src, nx, ny, nz, nzp, scale, dst);
    return cudaGetLastError();
}

cudaError_t launch_unpad(const float *src, int nx, int ny, int nz, int nzp, float scale,
                         float *dst, cudaStream_t s)
{
    unpad_kernel<<<grid_for((long long)nx * ny * nz), 256, 0, s>>>(src, nx, ny, nz, nzp, scale,
                                                                  dst);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *corner, const float *w, int rows, int npts, int row_dir,
                          float *out, cudaStream_t s)
{
    if (rows <= 0 || npts <= 0) return cudaSuccess;
    gather_kernel<<<grid_for((long long)rows * npts), 256, 0, s>>>(corner, w, rows, npts, row_dir,
                                                                   out);
    return cudaGetLastError();
}

cudaError_t launch_inj_sum(const int4 *pts, const int *item, const float *w, const float *q, int nq, int ne,
                           int rows, long long fstride, float *F, cudaStream_t s)
{
    if (rows <= 0 || ne <= 0) return cudaSuccess;
    inj_sum_kernel<<<grid_for((long long)rows * ne), 256, 0, s>>>(pts, item, w, q, nq, ne, rows, fstride, F);
    return cudaGetLastError();
}

}  // namespace wt
