// Double-float outer loop of mixed-precision defect correction: the kernels
// over the bodies of df_bodies.cuh, and their launchers.
//
// On GB300 the FP64 pipe runs at about 1/70 of the FP32 rate, so the ~70 FP32
// instructions per node of the double-float residual cost far less than the
// ~10 FP64 ones they replace.  The residual is exact up to about 1e-14 of
// |A||P|, far below what the 1e-10 stopping test needs; it is then rounded
// to FP32, the right-hand side of the FP32 V-cycles.
#include "device_util.cuh"
#include "df_bodies.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

template <bool D3>
__global__ void df_residual_kernel(Geom g, const PlaneCoefDF* __restrict__ cdf, const float* __restrict__ hi,
                                   const float* __restrict__ lo, const float* __restrict__ fh,
                                   const float* __restrict__ fl, float* __restrict__ r32,
                                   double* __restrict__ partial) {
    df_residual_body<D3>(g, cdf, hi, lo, fh, fl, r32, partial, blockIdx, gridDim);
}

__global__ void df_correct_kernel(Geom g, int d3, const float* __restrict__ e, float* __restrict__ hi,
                                  float* __restrict__ lo) {
    df_correct_body(g, d3, e, hi, lo, blockIdx, gridDim);
}

__global__ void df_split_kernel(Geom g, int d3, const double* __restrict__ f, float* __restrict__ hi,
                                float* __restrict__ lo) {
    df_split_body(g, d3, f, hi, lo, blockIdx, gridDim);
}

__global__ void df_to_double_kernel(size_t n, const float* __restrict__ hi, const float* __restrict__ lo,
                                    double* __restrict__ P) {
    df_to_double_body(n, hi, lo, P, blockIdx, gridDim);
}

__global__ void df_coef_kernel(int nz, const PlaneCoef<double>* __restrict__ c, PlaneCoefDF* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    auto split = [](double x, float& h, float& l) {
        h = float(x);
        l = float(x - double(h));
    };
    PlaneCoefDF d;
    split(c[k].cx, d.cxh, d.cxl);
    split(c[k].cy, d.cyh, d.cyl);
    split(c[k].cz, d.czh, d.czl);
    split(c[k].d, d.dh, d.dl);
    out[k] = d;
}

__global__ void df_copy_plane_kernel(Geom g2, const float* __restrict__ hi2, const float* __restrict__ lo2, Geom g3,
                                     float* __restrict__ hi3, float* __restrict__ lo3) {
    df_copy_plane_body(g2, hi2, lo2, g3, hi3, lo3, blockIdx);
}

}  // namespace

void launch_df_coef(const Geom& g, const PlaneCoef<double>* coef, PlaneCoefDF* cdf, cudaStream_t st) {
    df_coef_kernel<<<(g.nz + 127) / 128, 128, 0, st>>>(g.nz, coef, cdf);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_df_split(const Geom& g, int dim, const double* f, float* hi, float* lo, cudaStream_t st) {
    const int d3 = dim == 3;
    df_split_kernel<<<df_grid(g, d3, 0), dim3(DF_BX, DF_BY), 0, st>>>(g, d3, f, hi, lo);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

int launch_df_residual(const Geom& g, int dim, const PlaneCoefDF* cdf, const float* hi, const float* lo,
                       const float* fh, const float* fl, float* r32, double* partial, int max_blocks, cudaStream_t st) {
    const int d3 = dim == 3;
    const dim3 grid = df_residual_grid(g, d3, max_blocks);
    if (d3) df_residual_kernel<true><<<grid, dim3(DF_BX, DF_BY), 0, st>>>(g, cdf, hi, lo, fh, fl, r32, partial);
    else df_residual_kernel<false><<<grid, dim3(DF_BX, DF_BY), 0, st>>>(g, cdf, hi, lo, fh, fl, r32, partial);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    return int(grid.x * grid.y * grid.z);
}

void launch_df_correct(const Geom& g, int dim, const float* e, float* hi, float* lo, cudaStream_t st) {
    const int d3 = dim == 3;
    df_correct_kernel<<<df_grid(g, d3, 0), dim3(DF_BX, DF_BY), 0, st>>>(g, d3, e, hi, lo);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_df_to_double(const Geom& g, const float* hi, const float* lo, double* P, cudaStream_t st) {
    df_to_double_kernel<<<DF_TO_DOUBLE_BLOCKS, DF_TO_DOUBLE_THREADS, 0, st>>>(g.n, hi, lo, P);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_df_copy_plane(const Geom& g2, const float* hi2, const float* lo2, const Geom& g3, float* hi3, float* lo3,
                          cudaStream_t st) {
    const dim3 grid = df_plane_grid(g2);
    df_copy_plane_kernel<<<grid, dim3(DF_BX, DF_BY), 0, st>>>(g2, hi2, lo2, g3, hi3, lo3);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
