// Separable solve of one level with the sine transforms of each plane fused
// into one kernel: the coarse-grid solves of the V-cycles (and any other
// single-level separable solve whose planes fit the shared memory of a
// thread-block cluster).
//
// The staged separable solve (kernels_sep.cu) runs one launch per transform
// pass (x, y, mode solves, inverse y, inverse x) with the transformed data
// round-tripping through global memory; on the small levels of a coarse-grid
// solve (65^3, 65^2 nodes) every pass is a few microseconds of latency.  Here
// a cluster of C CTAs owns one plane: CTA r transforms its rows (x lines)
// into its shared memory, the cluster synchronises, and each CTA then reads
// its columns (y lines) straight from the other CTAs' shared memory
// (distributed shared memory) and transforms them; the way back is the
// mirror image.  The lower-boundary problem (one plane) is solved in one
// launch: x transforms, y transforms, the division by the mode eigenvalues,
// inverse y and inverse x.  A 3D level takes three launches: forward x and y
// per plane into the transformed array t[k][m][n], the tridiagonal mode
// solves along z (the staged solve's kernel), inverse y and x per plane.
//
// Every line is transformed by the building blocks of dst_body.cuh with the
// pairing of the staged transforms (lines 2q and 2q + 1 share an FFT), every
// scale and division is the staged solve's operation, so the results equal
// the staged solve's bit for bit (grouped solves, which launch the staged
// passes, stay bitwise equal to solo solves).
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "dst_body.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace cg = cooperative_groups;

namespace mhs {

namespace {

template <typename T>
struct PlaneSepArgs {
    int nxi = 0, nyi = 0;              // interior nodes of a plane (x lines have nxi elements, y lines nyi)
    int Lx = 0, Ly = 0, bx = 0, by = 0;   // transform lengths (nxi + 1, nyi + 1) and log2 of their FFT lengths
    int pr = 0, pc = 0;                // row pairs and column pairs per CTA
    int PSx = 0, PSy = 0, ldr = 0, ldc = 0;
    int zsz = 0, obsz = 0;             // complex elements of the FFT area, elements of the result area
    const T* f = nullptr;              // interior element (i, j) of plane k at f + k f_plane + j f_line + i
    long long f_plane = 0, f_line = 0;
    T* out = nullptr;                  // same layout
    long long out_plane = 0, out_line = 0;
    T* t = nullptr;                    // transformed data, element n of y line m of plane k at t + k t_plane + m nyi + n
    long long t_plane = 0;
    const void* twx = nullptr;
    const void* twy = nullptr;
    const T* mux = nullptr;            // 2D: mode eigenvalues and 1/h^2 factors of the division
    const T* muy = nullptr;
    T cf = T(0), cs = T(0);
    T scale = T(1);
    int accumulate = 0;
};

enum { PLANE_SOLVE2D = 0, PLANE_FORWARD = 1, PLANE_INVERSE = 2 };

// grid (C, planes), cluster (C, 1, 1): CTA rank r of the cluster of plane k
template <typename T, int MODE>
__global__ void __launch_bounds__(256) sep_plane_kernel(PlaneSepArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char plane_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = int(cl.block_rank());
    const int k = blockIdx.y;
    C* twx = reinterpret_cast<C*>(plane_smem);
    C* twy = twx + a.Lx;
    C* z = twy + a.Ly;
    T* ob = reinterpret_cast<T*>(z + a.zsz);
    T* rowb = ob + a.obsz;                                  // this CTA's rows: rowb[jl * ldr + m]
    T* colb = rowb + size_t(2 * a.pr) * a.ldr;              // this CTA's columns: colb[ml * ldc + j]
    const int j0 = rank * 2 * a.pr, nlr = max(0, min(2 * a.pr, a.nyi - j0));
    const int m0 = rank * 2 * a.pc, nlc = max(0, min(2 * a.pc, a.nxi - m0));
    const C* gx = static_cast<const C*>(a.twx);
    const C* gy = static_cast<const C*>(a.twy);
    for (int e = threadIdx.x; e < a.Lx; e += blockDim.x) twx[e] = gx[e];
    for (int e = threadIdx.x; e < a.Ly; e += blockDim.x) twy[e] = gy[e];
    const int rows_per = 2 * a.pr, cols_per = 2 * a.pc;

    // rows of plane k transformed along x (input f), results into rowb
    auto forward_x = [&]() {
        dst_zero<T>(z, a.pr, a.PSx, a.Lx, nlr);
        __syncthreads();
        const T* src = a.f + k * a.f_plane + (long long)j0 * a.f_line;
        const long long fl = a.f_line;
        dst_load<T>(z, a.PSx, nlr, a.Lx, a.bx, twx, [&](int l, int i) { return src[(long long)l * fl + i]; });
        __syncthreads();
        dst_fft<T>(z, twx, a.pr, a.PSx, a.bx, a.Lx);
        dst_post<T>(z, a.PSx, nlr, a.Lx, ob);
        __syncthreads();
        for (int e = threadIdx.x; e < nlr * a.nxi; e += blockDim.x) {
            const int l = e / a.nxi, m = e - l * a.nxi;
            rowb[l * a.ldr + m] = dst_result(T(1), ob[l * a.Lx + m], false, T(0));
        }
    };
    // columns transformed along y from ld(l, n), results into ob
    auto along_y = [&](auto ld, bool remote) {
        dst_zero<T>(z, a.pc, a.PSy, a.Ly, nlc);
        __syncthreads();
        dst_load<T>(z, a.PSy, nlc, a.Ly, a.by, twy, ld);
        __syncthreads();
        // the last read of other CTAs' shared memory: none of them may exit before it
        if (remote) cl.sync();
        dst_fft<T>(z, twy, a.pc, a.PSy, a.by, a.Ly);
        dst_post<T>(z, a.PSy, nlc, a.Ly, ob);
        __syncthreads();
    };
    // the cluster's columns of the row transforms (distributed shared memory)
    auto from_rows = [&](int l, int j) {
        const int owner = j / rows_per;
        const T* rb = cl.map_shared_rank(rowb, owner);
        return rb[(j - owner * rows_per) * a.ldr + m0 + l];
    };
    // ob -> colb (the inverse y results, scale 1)
    auto to_cols = [&]() {
        for (int e = threadIdx.x; e < nlc * a.nyi; e += blockDim.x) {
            const int l = e / a.nyi, j = e - l * a.nyi;
            colb[l * a.ldc + j] = dst_result(T(1), ob[l * a.Ly + j], false, T(0));
        }
    };
    // rows transformed back along x from the cluster's columns, into out
    auto inverse_x = [&]() {
        dst_zero<T>(z, a.pr, a.PSx, a.Lx, nlr);
        __syncthreads();
        dst_load<T>(z, a.PSx, nlr, a.Lx, a.bx, twx, [&](int l, int m) {
            const int owner = m / cols_per;
            const T* cb = cl.map_shared_rank(colb, owner);
            return cb[(m - owner * cols_per) * a.ldc + j0 + l];
        });
        __syncthreads();
        cl.sync();   // every remote read done before any CTA of the cluster exits
        dst_fft<T>(z, twx, a.pr, a.PSx, a.bx, a.Lx);
        dst_post<T>(z, a.PSx, nlr, a.Lx, ob);
        __syncthreads();
        T* dst = a.out + k * a.out_plane + (long long)j0 * a.out_line;
        const bool acc = a.accumulate != 0;
        for (int e = threadIdx.x; e < nlr * a.nxi; e += blockDim.x) {
            const int l = e / a.nxi, i = e - l * a.nxi;
            T* o = dst + (long long)l * a.out_line + i;
            *o = dst_result(a.scale, ob[l * a.Lx + i], acc, acc ? *o : T(0));
        }
    };

    if constexpr (MODE == PLANE_SOLVE2D) {
        forward_x();
        cl.sync();
        along_y(from_rows, false);
        // division by the mode eigenvalue, then the inverse y transform of the same columns
        for (int e = threadIdx.x; e < nlc * a.nyi; e += blockDim.x) {
            const int l = e / a.nyi, n = e - l * a.nyi;
            ob[l * a.Ly + n] = mode_divide(ob[l * a.Ly + n], a.cf, a.muy[n], a.cs, a.mux[m0 + l]);
        }
        __syncthreads();
        along_y([&](int l, int n) { return ob[l * a.Ly + n]; }, false);
        to_cols();
        cl.sync();   // also: every CTA has finished reading the others' rows
        inverse_x();
    } else if constexpr (MODE == PLANE_FORWARD) {
        forward_x();
        cl.sync();
        along_y(from_rows, true);
        T* dst = a.t + k * a.t_plane + (long long)m0 * a.nyi;
        for (int e = threadIdx.x; e < nlc * a.nyi; e += blockDim.x) {
            const int l = e / a.nyi, n = e - l * a.nyi;
            dst[(long long)l * a.nyi + n] = dst_result(T(1), ob[l * a.Ly + n], false, T(0));
        }
    } else {
        const T* src = a.t + k * a.t_plane + (long long)m0 * a.nyi;
        const int ny = a.nyi;
        along_y([&](int l, int n) { return src[(long long)l * ny + n]; }, false);
        to_cols();
        cl.sync();
        inverse_x();
    }
}

constexpr int PLANE_THREADS = 256;
constexpr size_t PLANE_SMEM_MAX = 227 * 1024;

template <typename T>
size_t plane_smem(const PlaneSepArgs<T>& a) {
    using C = typename Cplx<T>::type;
    return size_t(a.Lx + a.Ly + a.zsz) * sizeof(C) +
           (size_t(a.obsz) + size_t(2 * a.pr) * a.ldr + size_t(2 * a.pc) * a.ldc) * sizeof(T);
}

template <typename T>
void fill_shape(PlaneSepArgs<T>& a, int csize) {
    const int pairs_r = (a.nyi + 1) / 2, pairs_c = (a.nxi + 1) / 2;
    a.pr = (pairs_r + csize - 1) / csize;
    a.pc = (pairs_c + csize - 1) / csize;
    a.PSx = pair_stride(fft_length<T>(a.Lx));
    a.PSy = pair_stride(fft_length<T>(a.Ly));
    a.ldr = a.nxi | 1;
    a.ldc = a.nyi | 1;
    a.zsz = std::max(a.pr * a.PSx, a.pc * a.PSy);
    a.obsz = std::max(2 * a.pr * a.Lx, 2 * a.pc * a.Ly);
}

template <typename T, int MODE>
void* kernel_of() { return reinterpret_cast<void*>(&sep_plane_kernel<T, MODE>); }

// clusters of this shape and shared memory can run on the device (queried once per configuration)
template <typename T, int MODE>
bool cluster_fits(int csize, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, bool> known;
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find({csize, smem});
    if (it != known.end()) return it->second;
    bool ok = false;
    const void* fn = kernel_of<T, MODE>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(PLANE_SMEM_MAX)) == cudaSuccess &&
        (csize <= 8 || cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = csize;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3(csize, 1, 1);
        cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) == cudaSuccess && clusters > 0;
    }
    (void)cudaGetLastError();
    known[{csize, smem}] = ok;
    return ok;
}

template <typename T, int MODE>
void launch_plane(const PlaneSepArgs<T>& a, int csize, int planes, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = csize;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(csize, planes, 1);
    cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    MHS_CUDA(cudaLaunchKernelEx(&cfg, sep_plane_kernel<T, MODE>, a));
    count_launches(1);
}

}  // namespace

// Cluster size for a level: the largest power of two up to 16 with at
// least one row pair and one column pair per CTA whose clusters, one per
// plane, fit about one wave of the 152 SMs, doubled while a CTA's share of
// the plane does not fit shared memory, then halved until the configuration
// is launchable.  0: the plane kernels do not apply (slow transforms, or
// planes too large for the shared memory of 16 CTAs).
template <typename T>
int plane_cluster_size(const Geom& g, int dim) {
    const int nxi = g.nx - 2, nyi = g.ny - 2, planes = dim == 3 ? g.nz - 2 : 1;
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (nxi < 1 || nyi < 1 || planes < 1 || !pow2(g.nx - 1) || !pow2(g.ny - 1)) return 0;
    const int pairs = std::min((nxi + 1) / 2, (nyi + 1) / 2);
    auto smem_of = [&](int c) {
        PlaneSepArgs<T> a;
        a.nxi = nxi;
        a.nyi = nyi;
        a.Lx = g.nx - 1;
        a.Ly = g.ny - 1;
        fill_shape(a, c);
        return plane_smem(a);
    };
    int c = 1;
    while (c * 2 <= 16 && c * 2 <= pairs && c * 2 * planes <= 152) c *= 2;
    while (smem_of(c) > PLANE_SMEM_MAX && c * 2 <= 16 && c * 2 <= pairs) c *= 2;
    for (; c >= 1; c /= 2) {
        const size_t smem = smem_of(c);
        if (smem > PLANE_SMEM_MAX) return 0;   // smaller clusters need more per CTA
        const bool ok = dim == 3 ? cluster_fits<T, PLANE_FORWARD>(c, smem) && cluster_fits<T, PLANE_INVERSE>(c, smem)
                                 : cluster_fits<T, PLANE_SOLVE2D>(c, smem);
        if (ok) return c;
    }
    return 0;
}

// A e = f on level g by the plane kernels (see the file comment): f and out
// pitched level arrays (interior read / written, out added to with
// accumulate), t dense scratch of the interior size (3D).  Returns false
// when the level does not qualify; nothing is launched then.
template <typename T>
bool plane_level_solve(const Geom& g, int dim, const SepTables& tab, const T* f, T* t, T* out, bool accumulate,
                       const SepStage<T>* mode_solve, cudaStream_t st) {
    if (!tab.twx || !tab.twy) return false;
    const int c = plane_cluster_size<T>(g, dim);
    if (c == 0) return false;
    const int nxi = g.nx - 2, nyi = g.ny - 2, planes = dim == 3 ? g.nz - 2 : 1;
    auto ilog2 = [](int v) {
        int b = 0;
        while ((1 << b) < v) ++b;
        return b;
    };
    PlaneSepArgs<T> a;
    a.nxi = nxi;
    a.nyi = nyi;
    a.Lx = g.nx - 1;
    a.Ly = g.ny - 1;
    a.bx = ilog2(fft_length<T>(a.Lx));
    a.by = ilog2(fft_length<T>(a.Ly));
    fill_shape(a, c);
    const long long off = dim == 3 ? (long long)g.plane + g.px + 1 : (long long)g.px + 1;
    const long long sA = dim == 3 ? (long long)g.plane : 0;
    a.f = f + off;
    a.f_plane = sA;
    a.f_line = g.px;
    a.out = out + off;
    a.out_plane = sA;
    a.out_line = g.px;
    a.t = t;
    a.t_plane = (long long)nxi * nyi;
    a.twx = tab.twx;
    a.twy = tab.twy;
    a.mux = static_cast<const T*>(tab.mux);
    a.muy = static_cast<const T*>(tab.muy);
    a.cf = T(1.0 / (g.hy * g.hy));
    a.cs = T(1.0 / (g.hx * g.hx));
    a.scale = T((2.0 / (g.nx - 1)) * (2.0 / (g.ny - 1)));
    a.accumulate = accumulate ? 1 : 0;
    const size_t smem = plane_smem(a);
    if (dim == 2) {
        launch_plane<T, PLANE_SOLVE2D>(a, c, 1, smem, st);
        return true;
    }
    launch_plane<T, PLANE_FORWARD>(a, c, planes, smem, st);
    launch_sep_stage<T>(*mode_solve, st);
    launch_plane<T, PLANE_INVERSE>(a, c, planes, smem, st);
    return true;
}

template int plane_cluster_size<double>(const Geom&, int);
template int plane_cluster_size<float>(const Geom&, int);
template bool plane_level_solve<double>(const Geom&, int, const SepTables&, const double*, double*, double*, bool,
                                        const SepStage<double>*, cudaStream_t);
template bool plane_level_solve<float>(const Geom&, int, const SepTables&, const float*, float*, float*, bool,
                                       const SepStage<float>*, cudaStream_t);

}  // namespace mhs
