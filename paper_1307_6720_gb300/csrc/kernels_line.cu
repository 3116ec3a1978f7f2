// Zebra z-line Gauss-Seidel pass: kernels over the body in line_body.cuh.
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

}  // namespace

template <typename T>
void launch_zline(const Geom& g, const PlaneCoef<T>* coef, T* u, const T* f, T* scratch, cudaStream_t st) {
    if (g.nx < 3 || g.ny < 3 || g.nz < 3) return;
    if (g.nz > MAXZ) throw Error(MHS_ERR_INVALID_ARG, "z-line smoother: at most 1026 planes");
    const int hx = zline_hx(g);
    const dim3 grid = zline_grid(g);
    constexpr int U = ZLINE_U<T>;
    for (int colour = 0; colour < 2; ++colour) {
        zline_kernel<T, U><<<grid, dim3(LX, LY), 0, st>>>(g, coef, u, f, scratch, colour, hx);
        count_launches(1);
    }
    MHS_CUDA(cudaGetLastError());
}

template void launch_zline<float>(const Geom&, const PlaneCoef<float>*, float*, const float*, float*, cudaStream_t);
template void launch_zline<double>(const Geom&, const PlaneCoef<double>*, double*, const double*, double*,
                                   cudaStream_t);

}  // namespace mhs
