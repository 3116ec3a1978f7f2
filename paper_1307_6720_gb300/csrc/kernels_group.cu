// Grouped kernels: one launch runs one multigrid operation for every item of
// a table (an instance and one of its levels), over the same per-block
// bodies as the solo kernels.  Block b of the launch belongs to the item
// with the largest first-block offset <= b (binary search) and takes the
// local block index b - first within that item's own grid, so each instance
// is decomposed exactly as in its solo launch.  A whole block leaves early
// when its item is gated off (instance converged, sweep count reached, or
// outside the current full-multigrid step); the test is uniform over the
// block, so the bodies' barriers stay matched.
#include <algorithm>

#include "device_util.cuh"
#include "df_bodies.cuh"
#include "group.h"
#include "line_body.cuh"
#include "mg_bodies.cuh"
#include "sub_body.cuh"

namespace mhs {

namespace {

struct GBlock {
    const GItem* it;
    dim3 b, gd;
};

// item of this block, and whether it runs
__device__ __forceinline__ bool locate(const GItem* __restrict__ items, int n, int gate, int sweep, int fmg_step,
                                       GBlock& out) {
    int lo = 0, hi = n - 1;
    const int blk = int(blockIdx.x);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= blk) lo = mid;
        else hi = mid - 1;
    }
    const GItem& it = items[lo];
    if (gate == G_ACTIVE && !it.ctl->cont) return false;
    if (sweep >= 0 && sweep >= it.ia[0]) return false;
    if (fmg_step >= 0 && it.ia[1] < fmg_step) return false;
    const int lb = blk - it.first;
    out.it = &it;
    out.b = dim3(lb % it.gx, (lb / it.gx) % it.gy, lb / (it.gx * it.gy));
    out.gd = dim3(it.gx, it.gy, it.gz);
    return true;
}

template <typename T, bool D3>
__global__ void g_colour_kernel(const GItem* items, int n, int colour, int sweep, int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, sweep, fmg_step, k)) return;
    const GItem& it = *k.it;
    if constexpr (sizeof(T) == 4 && D3) {
        if (use_v4(it.g)) {   // the quad form the solo launch uses on such levels
            colour_body_v4(it.g, static_cast<const PlaneCoef<float>*>(it.coef), static_cast<float*>(it.p[0]),
                           static_cast<const float*>(it.p[1]), colour, k.b, k.gd);
            return;
        }
    }
    colour_body<T, D3>(it.g, static_cast<const PlaneCoef<T>*>(it.coef), static_cast<T*>(it.p[0]),
                       static_cast<const T*>(it.p[1]), colour, k.b, k.gd);
}

template <typename T, int U>
__global__ void __launch_bounds__(LX* LY) g_zline_kernel(const GItem* items, int n, int colour, int sweep,
                                                         int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, sweep, fmg_step, k)) return;
    const GItem& it = *k.it;
    zline_body<T, U>(it.g, static_cast<const PlaneCoef<T>*>(it.coef), static_cast<T*>(it.p[0]),
                     static_cast<const T*>(it.p[1]), static_cast<T*>(it.p[2]), colour, zline_hx(it.g), k.b);
}

// FP32 levels: the partitioned column solve; the block has as many warps as
// the most segments among the launch's items
template <int SY>
__global__ void __launch_bounds__(32 * SY) g_zline_part_kernel(const GItem* items, int n, int colour,
                                                                               int sweep, int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, sweep, fmg_step, k)) return;
    const GItem& it = *k.it;
    zline_part_body(it.g, static_cast<const PlaneCoef<float>*>(it.coef), static_cast<float*>(it.p[0]),
                    static_cast<const float*>(it.p[1]), colour, zline_hx(it.g), k.b);
}

template <typename T, bool D3, bool NORM>
__global__ void g_residual_kernel(const GItem* items, int n, int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, fmg_step, k)) return;
    const GItem& it = *k.it;
    if constexpr (sizeof(T) == 4 && D3 && !NORM) {
        if (use_v4(it.g)) {
            residual_body_v4(it.g, static_cast<const PlaneCoef<float>*>(it.coef), static_cast<const float*>(it.p[0]),
                             static_cast<const float*>(it.p[1]), static_cast<float*>(it.p[2]), k.b, k.gd);
            return;
        }
    }
    if (it.ia[2]) {   // right after a red-black sweep: red nodes only (as the solo launch)
        residual_red_body<T, D3, NORM>(it.g, static_cast<const PlaneCoef<T>*>(it.coef),
                                       static_cast<const T*>(it.p[0]), static_cast<const T*>(it.p[1]),
                                       static_cast<T*>(it.p[2]), static_cast<double*>(it.p[3]), k.b, k.gd);
        return;
    }
    residual_body<T, D3, NORM>(it.g, static_cast<const PlaneCoef<T>*>(it.coef), static_cast<const T*>(it.p[0]),
                               static_cast<const T*>(it.p[1]), static_cast<T*>(it.p[2]),
                               static_cast<double*>(it.p[3]), k.b, k.gd);
}

template <typename T, bool D3>
__global__ void __launch_bounds__(RR_THREADS) g_resid_restrict_kernel(const GItem* items, int n, int fmg_step,
                                                                     int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, fmg_step, k)) return;
    const GItem& it = *k.it;
    resid_restrict_body<T, D3>(it.g, it.g2, static_cast<const PlaneCoef<T>*>(it.coef), static_cast<const T*>(it.p[0]),
                               static_cast<const T*>(it.p[1]), static_cast<T*>(it.p[2]), static_cast<T*>(it.p[3]), k.b,
                               k.gd);
}

// rotated: the restriction of a rotated FP64 cycle (red residual flag in
// ia[3]) rather than of a V-cycle level after its own residual (ia[2])
template <typename T, bool D3>
__global__ void g_restrict_kernel(const GItem* items, int n, int fmg_step, int gate, int rotated) {
    GBlock k;
    if (!locate(items, n, gate, -1, fmg_step, k)) return;
    const GItem& it = *k.it;
    restrict_body<T, D3>(it.g, it.g2, static_cast<const T*>(it.p[0]), static_cast<T*>(it.p[1]),
                         static_cast<T*>(it.p[2]), k.b, k.gd, (rotated ? it.ia[3] : it.ia[2]) != 0);
}

template <typename T, bool D3>
__global__ void g_prolong_kernel(const GItem* items, int n, int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, fmg_step, k)) return;
    const GItem& it = *k.it;
    prolong_body<T, D3>(it.g, it.g2, static_cast<const T*>(it.p[0]), static_cast<T*>(it.p[1]), k.b, k.gd);
}

// one block per instance: ia[2] = index of its first SubParams (start level
// = its cut-off ia[3]); a V-cycle from `start` begins the sub-cycle at
// max(start, cut-off)
template <typename T, bool D3>
__global__ void __launch_bounds__(SX * SY) g_subcycle_kernel(const GItem* items, int n, const SubParams<T>* params,
                                                             int start, int fmg_step, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, fmg_step, k)) return;
    const GItem& it = *k.it;
    const int s = start > it.ia[3] ? start : it.ia[3];
    subcycle_body<T, D3>(params[it.ia[2] + s - it.ia[3]]);
}

// zero ia[0] 32-bit words at p[0]
__global__ void g_zero_kernel(const GItem* items, int n, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, -1, k)) return;
    const GItem& it = *k.it;
    unsigned* a = static_cast<unsigned*>(it.p[0]);
    const size_t words = size_t(unsigned(it.ia[0]));
    for (size_t o = k.b.x * size_t(blockDim.x) + threadIdx.x; o < words; o += size_t(k.gd.x) * blockDim.x) a[o] = 0u;
}

__global__ void g_lower_rhs_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    lower_rhs_body(k.it->g, static_cast<const double*>(k.it->p[0]), static_cast<double*>(k.it->p[1]), k.b);
}

__global__ void g_copy_plane_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    copy_plane_body(k.it->g, static_cast<const double*>(k.it->p[0]), k.it->g2, static_cast<double*>(k.it->p[1]),
                    k.b);
}

__global__ void g_lift_norm_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    lift_norm_body(k.it->g, static_cast<const PlaneCoef<double>*>(k.it->coef), static_cast<const double*>(k.it->p[0]),
                   static_cast<double*>(k.it->p[1]), k.b, k.gd);
}

__global__ void g_df_split_kernel(const GItem* items, int n, int d3) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    df_split_body(k.it->g, d3, static_cast<const double*>(k.it->p[0]), static_cast<float*>(k.it->p[1]),
                  static_cast<float*>(k.it->p[2]), k.b, k.gd);
}

__global__ void g_df_copy_plane_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    const GItem& it = *k.it;
    df_copy_plane_body(it.g, static_cast<const float*>(it.p[0]), static_cast<const float*>(it.p[1]), it.g2,
                       static_cast<float*>(it.p[2]), static_cast<float*>(it.p[3]), k.b);
}

template <bool D3>
__global__ void g_df_residual_kernel(const GItem* items, int n, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, -1, k)) return;
    const GItem& it = *k.it;
    df_residual_body<D3>(it.g, static_cast<const PlaneCoefDF*>(it.coef), static_cast<const float*>(it.p[0]),
                         static_cast<const float*>(it.p[1]), static_cast<const float*>(it.p[2]),
                         static_cast<const float*>(it.p[3]), static_cast<float*>(it.p[4]),
                         static_cast<double*>(it.p[5]), k.b, k.gd);
}

__global__ void g_df_correct_kernel(const GItem* items, int n, int d3, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, -1, k)) return;
    df_correct_body(k.it->g, d3, static_cast<const float*>(k.it->p[0]), static_cast<float*>(k.it->p[1]),
                    static_cast<float*>(k.it->p[2]), k.b, k.gd);
}

__global__ void g_df_to_double_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    df_to_double_body(k.it->g.n, static_cast<const float*>(k.it->p[0]), static_cast<const float*>(k.it->p[1]),
                      static_cast<double*>(k.it->p[2]), k.b, k.gd);
}

__global__ void g_bnorm_kernel(const GItem* items, int n) {
    GBlock k;
    if (!locate(items, n, G_ALL, -1, -1, k)) return;
    bnorm_body(static_cast<const double*>(k.it->p[0]), k.it->ia[0], k.it->ctl);
}

__global__ void g_check_kernel(const GItem* items, int n, int first, int gate) {
    GBlock k;
    if (!locate(items, n, gate, -1, -1, k)) return;
    check_body(static_cast<const double*>(k.it->p[0]), k.it->ia[0], k.it->ctl, first);
}

// OR of the instances' continuation flags: the condition of the group's while node
__global__ void g_any_kernel(SolveCtl* const* ctls, int n, cudaGraphConditionalHandle handle, int use_handle,
                             int* any_out) {
    int a = 0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) a |= ctls[q]->cont;
    a = __syncthreads_or(a);
    if (threadIdx.x == 0) {
        if (any_out) *any_out = a;
        if (use_handle) cudaGraphSetConditional(handle, a ? 1u : 0u);
    }
}

__global__ void g_gather_ctl_kernel(SolveCtl* const* ctls, int n, SolveCtl* out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) out[q] = *ctls[q];
}

inline void after_launch() {
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

const dim3 kMG(MG_BX, MG_BY), kDF(DF_BX, DF_BY), kLine(LX, LY);

}  // namespace

template <typename T>
void glaunch_colour(const GTable& t, int d3, int colour, int sweep, int fmg_step, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_colour_kernel<T, true><<<t.blocks, kMG, 0, st>>>(t.items, t.n, colour, sweep, fmg_step, gate);
    else g_colour_kernel<T, false><<<t.blocks, kMG, 0, st>>>(t.items, t.n, colour, sweep, fmg_step, gate);
    after_launch();
}

template <typename T>
void glaunch_zline(const GTable& t, int colour, int sweep, int fmg_step, int gate, cudaStream_t st) {
    if (!t.n) return;
    if constexpr (sizeof(T) == 4) {
        static bool attr = false;
        if (!attr) {
            MHS_CUDA(cudaFuncSetAttribute(g_zline_part_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            MHS_CUDA(cudaFuncSetAttribute(g_zline_part_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            attr = true;
        }
        const dim3 blk(32, t.ty);
        if (t.ty <= 8) g_zline_part_kernel<8><<<t.blocks, blk, t.smem, st>>>(t.items, t.n, colour, sweep, fmg_step, gate);
        else g_zline_part_kernel<32><<<t.blocks, blk, t.smem, st>>>(t.items, t.n, colour, sweep, fmg_step, gate);
    } else {
        g_zline_kernel<T, ZLINE_U<T>><<<t.blocks, kLine, 0, st>>>(t.items, t.n, colour, sweep, fmg_step, gate);
    }
    after_launch();
}

template <typename T>
void glaunch_residual(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_residual_kernel<T, true, false><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate);
    else g_residual_kernel<T, false, false><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate);
    after_launch();
}

template <typename T>
void glaunch_residual_norm(const GTable& t, int d3, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_residual_kernel<T, true, true><<<t.blocks, kMG, 0, st>>>(t.items, t.n, -1, gate);
    else g_residual_kernel<T, false, true><<<t.blocks, kMG, 0, st>>>(t.items, t.n, -1, gate);
    after_launch();
}

template <typename T>
void glaunch_restrict(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st, int rotated) {
    if (!t.n) return;
    if (d3) g_restrict_kernel<T, true><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate, rotated);
    else g_restrict_kernel<T, false><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate, rotated);
    after_launch();
}

template <typename T>
void glaunch_resid_restrict(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_resid_restrict_kernel<T, true><<<t.blocks, RR_THREADS, 0, st>>>(t.items, t.n, fmg_step, gate);
    else g_resid_restrict_kernel<T, false><<<t.blocks, RR_THREADS, 0, st>>>(t.items, t.n, fmg_step, gate);
    after_launch();
}

template <typename T>
void glaunch_prolong(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_prolong_kernel<T, true><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate);
    else g_prolong_kernel<T, false><<<t.blocks, kMG, 0, st>>>(t.items, t.n, fmg_step, gate);
    after_launch();
}

template <typename T>
void glaunch_subcycle(const GTable& t, const SubParams<T>* params, int d3, int start, int fmg_step, int gate,
                      size_t smem, int rows, cudaStream_t st) {
    if (!t.n) return;
    const dim3 blk(SX, rows);
    if (d3) g_subcycle_kernel<T, true><<<t.blocks, blk, smem, st>>>(t.items, t.n, params, start, fmg_step, gate);
    else g_subcycle_kernel<T, false><<<t.blocks, blk, smem, st>>>(t.items, t.n, params, start, fmg_step, gate);
    after_launch();
}

void gsubcycle_prepare() {
    const int lim = int(subcycle_smem_limit());
    MHS_CUDA(cudaFuncSetAttribute(g_subcycle_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(g_subcycle_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(g_subcycle_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(g_subcycle_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
}

void glaunch_zero(const GTable& t, int gate, cudaStream_t st) {
    if (!t.n) return;
    g_zero_kernel<<<t.blocks, 256, 0, st>>>(t.items, t.n, gate);
    after_launch();
}

void glaunch_lower_rhs(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_lower_rhs_kernel<<<t.blocks, kMG, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_copy_plane(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_copy_plane_kernel<<<t.blocks, kMG, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_lift_norm(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_lift_norm_kernel<<<t.blocks, kMG, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_df_split(const GTable& t, int d3, cudaStream_t st) {
    if (!t.n) return;
    g_df_split_kernel<<<t.blocks, kDF, 0, st>>>(t.items, t.n, d3);
    after_launch();
}

void glaunch_df_copy_plane(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_df_copy_plane_kernel<<<t.blocks, kDF, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_df_residual(const GTable& t, int d3, int gate, cudaStream_t st) {
    if (!t.n) return;
    if (d3) g_df_residual_kernel<true><<<t.blocks, kDF, 0, st>>>(t.items, t.n, gate);
    else g_df_residual_kernel<false><<<t.blocks, kDF, 0, st>>>(t.items, t.n, gate);
    after_launch();
}

void glaunch_df_correct(const GTable& t, int d3, int gate, cudaStream_t st) {
    if (!t.n) return;
    g_df_correct_kernel<<<t.blocks, kDF, 0, st>>>(t.items, t.n, d3, gate);
    after_launch();
}

void glaunch_df_to_double(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_df_to_double_kernel<<<t.blocks, DF_TO_DOUBLE_THREADS, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_bnorm(const GTable& t, cudaStream_t st) {
    if (!t.n) return;
    g_bnorm_kernel<<<t.blocks, 1024, 0, st>>>(t.items, t.n);
    after_launch();
}

void glaunch_check(const GTable& t, int first, int gate, cudaStream_t st) {
    if (!t.n) return;
    g_check_kernel<<<t.blocks, 1024, 0, st>>>(t.items, t.n, first, gate);
    after_launch();
}

void glaunch_any(SolveCtl* const* ctls, int n, cudaGraphConditionalHandle handle, int use_handle, int* any_out,
                 cudaStream_t st) {
    g_any_kernel<<<1, 256, 0, st>>>(ctls, n, handle, use_handle, any_out);
    after_launch();
}

void glaunch_gather_ctl(SolveCtl* const* ctls, int n, SolveCtl* out, cudaStream_t st) {
    if (n <= 0) return;
    g_gather_ctl_kernel<<<(n + 255) / 256, 256, 0, st>>>(ctls, n, out);
    after_launch();
}

#define MHS_GINST(T)                                                                                          \
    template void glaunch_colour<T>(const GTable&, int, int, int, int, int, cudaStream_t);                    \
    template void glaunch_zline<T>(const GTable&, int, int, int, int, cudaStream_t);                          \
    template void glaunch_residual<T>(const GTable&, int, int, int, cudaStream_t);                            \
    template void glaunch_residual_norm<T>(const GTable&, int, int, cudaStream_t);                            \
    template void glaunch_restrict<T>(const GTable&, int, int, int, cudaStream_t, int);                            \
    template void glaunch_resid_restrict<T>(const GTable&, int, int, int, cudaStream_t);                      \
    template void glaunch_prolong<T>(const GTable&, int, int, int, cudaStream_t);                             \
    template void glaunch_subcycle<T>(const GTable&, const SubParams<T>*, int, int, int, int, size_t, int, cudaStream_t);
MHS_GINST(double)
MHS_GINST(float)
#undef MHS_GINST

}  // namespace mhs
