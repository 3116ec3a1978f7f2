// Zebra z-line Gauss-Seidel pass: kernels over the bodies in line_body.cuh
// (FP64 levels: one thread per column; FP32 levels: the partitioned column
// solve, 32 columns x S segments per block).
#include "device_util.cuh"
#include "line_body.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

template <typename T, int U>
__global__ void __launch_bounds__(LX* LY) zline_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef,
                                                       T* __restrict__ u, const T* __restrict__ f,
                                                       T* __restrict__ w, int colour, int hx) {
    zline_body<T, U>(g, coef, u, f, w, colour, hx, blockIdx);
}

// SY warps per block at most: 8 (levels of up to 191 interior planes) or 32
template <int SY>
__global__ void __launch_bounds__(32 * SY) zline_part_kernel(Geom g, const PlaneCoef<float>* __restrict__ coef,
                                                          float* __restrict__ u, const float* __restrict__ f,
                                                          int colour, int hx) {
    zline_part_body(g, coef, u, f, colour, hx, blockIdx);
}

}  // namespace

template <typename T>
void launch_zline(const Geom& g, const PlaneCoef<T>* coef, T* u, const T* f, T* scratch, cudaStream_t st) {
    if (g.nx < 3 || g.ny < 3 || g.nz < 3) return;
    if (g.nz > MAXZ) throw Error(MHS_ERR_INVALID_ARG, "z-line smoother: at most 1026 planes");
    const int hx = zline_hx(g);
    if constexpr (sizeof(T) == 4) {
        const int n = g.nz - 2, S = zpart_segments(n);
        const size_t smem = zpart_smem(n, S);   // up to 172 KB (1024 planes, 32 segments)
        static bool attr = false;
        if (!attr) {
            MHS_CUDA(cudaFuncSetAttribute(zline_part_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            MHS_CUDA(cudaFuncSetAttribute(zline_part_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            attr = true;
        }
        const dim3 grid = zline_part_grid(g);
        for (int colour = 0; colour < 2; ++colour) {
            if (S <= 8) zline_part_kernel<8><<<grid, dim3(32, S), smem, st>>>(g, coef, u, f, colour, hx);
            else zline_part_kernel<32><<<grid, dim3(32, S), smem, st>>>(g, coef, u, f, colour, hx);
            count_launches(1);
        }
        (void)scratch;
    } else {
        const dim3 grid = zline_grid(g);
        constexpr int U = ZLINE_U<T>;
        for (int colour = 0; colour < 2; ++colour) {
            zline_kernel<T, U><<<grid, dim3(LX, LY), 0, st>>>(g, coef, u, f, scratch, colour, hx);
            count_launches(1);
        }
    }
    MHS_CUDA(cudaGetLastError());
}

template void launch_zline<float>(const Geom&, const PlaneCoef<float>*, float*, const float*, float*, cudaStream_t);
template void launch_zline<double>(const Geom&, const PlaneCoef<double>*, double*, const double*, double*,
                                   cudaStream_t);

}  // namespace mhs
