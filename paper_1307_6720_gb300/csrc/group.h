// Grouped launches: one kernel launch performs one multigrid operation for
// many independent instances (uneven grids), each instance with the block
// decomposition of its own solo launch, so that a grouped solve is bitwise
// identical to solving every instance alone.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "mhs_internal.h"

namespace mhs {

// One (instance, level) of a grouped launch.  Pointers and integers are
// interpreted by the operation (see the launchers in kernels_group.cu).
struct GItem {
    int q;                 // instance index within the group
    int first;             // first block of the item in the grouped grid
    int gx, gy, gz;        // the item's own grid (the solo launch's)
    Geom g, g2;            // level, and its partner (coarse or fine level, or the 3D level of a plane copy)
    const void* coef;      // PlaneCoef<T> / PlaneCoefDF of the level
    void* p[6];            // arrays
    int ia[4];             // integers: sweep count, FMG top level, partial count, ...
    SolveCtl* ctl;         // the instance's control block of the current problem
};

// gate of a grouped launch: run every item, or only items whose instance still iterates
enum GGate { G_ALL = 0, G_ACTIVE = 1 };

// Device table of items with its total block count.
struct GTable {
    GItem* items = nullptr;   // device
    int n = 0;                // items
    int blocks = 0;           // sum of the items' grid sizes
    int ty = 0;               // FP32 z-line passes: warps per block (most segments of the items' columns)
    unsigned smem = 0;        // and their dynamic shared memory (the largest item's)
};

// launchers (kernels_group.cu); `sweep` gates smoothing items by ia[0] > sweep,
// `fmg_step` (>= 0) gates items by ia[1] >= fmg_step (the instance's FMG top level)
template <typename T>
void glaunch_colour(const GTable& t, int d3, int colour, int sweep, int fmg_step, int gate, cudaStream_t st);
template <typename T>
void glaunch_zline(const GTable& t, int colour, int sweep, int fmg_step, int gate, cudaStream_t st);
template <typename T>
void glaunch_residual(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st);
template <typename T>
void glaunch_residual_norm(const GTable& t, int d3, int gate, cudaStream_t st);
template <typename T>
void glaunch_restrict(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st, int rotated = 0);
// residual and restriction in one pass (FP32 levels; items: p = u, f, coarse
// f, coarse u)
template <typename T>
void glaunch_resid_restrict(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st);
template <typename T>
void glaunch_prolong(const GTable& t, int d3, int fmg_step, int gate, cudaStream_t st);
template <typename T>
void glaunch_subcycle(const GTable& t, const SubParams<T>* params, int d3, int start, int fmg_step, int gate,
                      size_t smem, int rows, cudaStream_t st);
void glaunch_zero(const GTable& t, int gate, cudaStream_t st);
void glaunch_lower_rhs(const GTable& t, cudaStream_t st);
void glaunch_copy_plane(const GTable& t, cudaStream_t st);
void glaunch_lift_norm(const GTable& t, cudaStream_t st);
void glaunch_df_split(const GTable& t, int d3, cudaStream_t st);
void glaunch_df_copy_plane(const GTable& t, cudaStream_t st);
void glaunch_df_residual(const GTable& t, int d3, int gate, cudaStream_t st);
void glaunch_df_correct(const GTable& t, int d3, int gate, cudaStream_t st);
void glaunch_df_to_double(const GTable& t, cudaStream_t st);
void glaunch_bnorm(const GTable& t, cudaStream_t st);
void glaunch_check(const GTable& t, int first, int gate, cudaStream_t st);
void glaunch_any(SolveCtl* const* ctls, int n, cudaGraphConditionalHandle handle, int use_handle, int* any_out,
                 cudaStream_t st);
void glaunch_gather_ctl(SolveCtl* const* ctls, int n, SolveCtl* out, cudaStream_t st);
void gsubcycle_prepare();

// One instance's stage of a separable coarse-grid solve in a grouped launch
// (the stage's arguments and its solo grid; `top` gates full-multigrid steps
// like GItem::ia[1]).
template <typename T>
struct GSepItem {
    int first;          // first block of the item in the grouped grid
    int gx, gy, gz;     // the stage's own grid
    SolveCtl* ctl;      // the instance's control block
    int top;            // the instance's full-multigrid top level
    SepStage<T> st;
};
template <typename T>
struct GSepTable {
    GSepItem<T>* items = nullptr;   // device
    int n = 0, blocks = 0, threads = 0, kind = SEP_DST;
    size_t smem = 0;                // largest dynamic shared memory of the items
};
template <typename T>
void glaunch_sep(const GSepTable<T>& t, int fmg_step, int gate, cudaStream_t st);   // kernels_sep.cu
template <typename T>
void glaunch_dst(const GSepTable<T>& t, int fmg_step, int gate, cudaStream_t st);   // kernels_dst.cu

#ifdef __CUDACC__
// item of this block of a grouped launch (binary search over first-block
// offsets), its local block index in lb; nullptr when the item is gated off
template <typename I>
__device__ __forceinline__ const I* glocate(const I* __restrict__ items, int n, int gate, int fmg_step, int& lb) {
    int lo = 0, hi = n - 1;
    const int blk = int(blockIdx.x);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= blk) lo = mid;
        else hi = mid - 1;
    }
    const I& it = items[lo];
    if (gate == G_ACTIVE && !it.ctl->cont) return nullptr;
    if (fmg_step >= 0 && it.top < fmg_step) return nullptr;
    lb = blk - it.first;
    return &it;
}
#endif

// tables of one problem (lower boundary or interior) of a group
struct GDim {
    int dim = 3;
    int L = 0;                                   // most levels of any instance
    int max_nu1 = 0, max_nu2 = 0, max_top = -1;  // largest sweep counts and FMG top level
    // per level l (items of the instances for which l is a global level)
    std::vector<GTable> pre_pt, post_pt, pre_ln, post_ln, res, restr, resr, prol;   // resr: the fused pass (FP32)
    // full multigrid: restriction of the residual and prolongation of the
    // coarse solution, per level, for the instances using it
    std::vector<GTable> fmg_restr, fmg_prol;
    GTable sub, sub8;                            // sub-cycle: one item per instance (32 or 8 rows of threads)
    GTable subz, subz8;                          // the same for instances whose sub-cycle starts at level 0
    // separable coarse-grid solves of the instances that end their cycles in one:
    // one table per (stage, kind), in launch order, in the cycle precision
    std::vector<GSepTable<float>> exact32;
    std::vector<GSepTable<double>> exact64;
    void* params = nullptr;                      // SubParams<T>[], device
    size_t sub_smem = 0;
    // once per solve
    GTable zero_u, lower_rhs, zero_hi, zero_lo, split, copy_u, copy_t, df_copy, lift, bnorm, check1;
    // the first test; cycle end (every instance), and after the full-multigrid cycle (instances using it)
    GTable res_norm0, res_norm, check, fmg_res_norm, fmg_check;
    // mixed mode
    GTable zero_e, correct, fmg_zero_e, fmg_correct, to_double;
};

// One part of a group: instances solved by one graph (one launch per
// operation and level for all of them).
struct GPart {
    std::vector<mhs_ctx*> hs;
    int mode = MHS_MIXED;
    // a part of one instance runs that instance's own solve (its captured
    // graph, or the host-driven sequence when eager) on the part's launch
    // stream: the grouped launches would serve no second instance
    bool solo = false;
    cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> allocs;
    GDim d2, d3;
    SolveCtl** ctls = nullptr;          // device: [2n] = n lower-boundary then n interior control blocks
    SolveCtl* gathered = nullptr;       // device copy of the 2n control blocks after a solve
    SolveCtl* gathered_host = nullptr;  // pinned
    cudaGraphExec_t exec = nullptr;
    long long n_fixed = 0, n_cycle2 = 0, n_cycle3 = 0;   // kernel launches of the graph's sections
    bool eager = false;                 // host-driven launches instead of the graph
    double tol = 0.0;                   // tolerance of the solve in flight
    cudaStream_t launch_stream = nullptr;   // stream of the solve in flight
    int* any_dev = nullptr;             // OR of the continuation flags (eager loop)
    int* any_host = nullptr;            // pinned
};

}  // namespace mhs

// A group: its instances split into parts whose working sets fit the L2
// cache, the parts launched round-robin on a few streams.
struct mhs_group {
    std::vector<mhs::GPart*> parts;
    std::vector<std::vector<int>> members;   // instance indices of each part
    std::vector<cudaStream_t> streams;       // launch streams
    int n = 0;
    bool eager = false;
};
