// Device-side convergence control and the one-CTA multigrid sub-cycle: the
// kernels over the bodies of sub_body.cuh, and their launchers.
#include <cmath>

#include "device_util.cuh"
#include "mhs_internal.h"
#include "solver.h"
#include "sub_body.cuh"

namespace mhs {

namespace {

__global__ void bnorm_kernel(const double* __restrict__ partial, int n, SolveCtl* ctl) {
    bnorm_body(partial, n, ctl);
}

__global__ void check_kernel(const double* __restrict__ partial, int n, SolveCtl* ctl, int first,
                             cudaGraphConditionalHandle handle, int use_handle) {
    const int cont = check_body(partial, n, ctl, first);
    if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(handle, cont);
}

template <typename T, bool D3>
__global__ void __launch_bounds__(SX * SY) subcycle_kernel(const SubParams<T> p) {
    subcycle_body<T, D3>(p);
}

}  // namespace

void launch_bnorm(const double* partial, int n, SolveCtl* ctl, cudaStream_t st) {
    bnorm_kernel<<<1, 1024, 0, st>>>(partial, n, ctl);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_check(const double* partial, int n, SolveCtl* ctl, int first, cudaGraphConditionalHandle handle,
                  int use_handle, cudaStream_t st) {
    check_kernel<<<1, 1024, 0, st>>>(partial, n, ctl, first, handle, use_handle);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

size_t subcycle_smem_limit() { return 220 * 1024; }

void subcycle_prepare() {
    const int lim = int(subcycle_smem_limit());
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
}

template <typename T>
void launch_subcycle(const SubParams<T>& p, cudaStream_t st) {
    const dim3 blk(SX, p.rows);
    if (p.dim == 3) subcycle_kernel<T, true><<<1, blk, p.smem_bytes, st>>>(p);
    else subcycle_kernel<T, false><<<1, blk, p.smem_bytes, st>>>(p);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template void launch_subcycle<double>(const SubParams<double>&, cudaStream_t);
template void launch_subcycle<float>(const SubParams<float>&, cudaStream_t);

}  // namespace mhs
