// Driver entry points used by the C-ABI layer.
#pragma once

#include <cmath>
#include <vector>

#include "mhs_internal.h"

namespace mhs {

// xi(z) of Sect. 3.2 on the host (the device copy is xi_of in kernels_mg.cu)
inline double xi_host(const mhs_xi_params& x, double z) {
    switch (x.kind) {
    case MHS_XI_EXP: return x.a * std::exp(-x.kappa * z);
    case MHS_XI_EXP_SIN: return (x.a + x.b * std::sin(x.omega * z)) * std::exp(-x.kappa * z);
    default: return 0.0;
    }
}

// Autotuner (tune.cu): anisotropy class of a handle's interior operator,
// floor(log2(max_k  weakest horizontal spacing^2 / ((1 - xi_k) h_z^2))), at least 0
int aniso_class(const mhs_ctx* c);
void autotune(mhs_ctx* c, double tol, int mode, int repeats, mhs_tune_result* out);
// z-line smoothing on the interior levels: forced by MHS_FLAG_ZLINE, excluded by
// MHS_FLAG_POINT, otherwise chosen when the anisotropy class is 5 or more
inline bool use_zline(const mhs_ctx* c) {
    if (c->opts.flags & MHS_FLAG_ZLINE) return true;
    if (c->opts.flags & MHS_FLAG_POINT) return false;
    return c->aniso >= 5;
}
bool tune_lookup(const mhs_ctx* c, int mode, mhs_solver_opts* o);
void tune_clear();

// grouped solves (group.cu)
mhs_group* group_create(mhs_ctx** hs, int n, int mode, size_t part_bytes, int nstreams);
void group_destroy(mhs_group* G);
void group_set_eager(mhs_group* G, bool eager);
mhs_status group_solve(mhs_group* G, double tol, mhs_solve_info* infos, mhs_status* statuses);
size_t cycle_bytes(const mhs_ctx* c, int mode);

// slots of NormScratch::result
constexpr int NORM_B_SLOT = 0;        // ||b||^2 of the current solve
constexpr int NORM_RES_SLOT = 1;      // ||f - A u||^2 after the latest cycle
constexpr int NORM_SCRATCH_SLOT = 2;  // residual norms inside V-cycles (unused by the driver)
constexpr int NORM_HOOK_SLOT = 3;     // level-hook residuals

void create(mhs_ctx* c);
void destroy(mhs_ctx* c);
void compute_coefficients(mhs_ctx* c);
void invalidate_graphs(mhs_ctx* c);
void choose_cuts(mhs_ctx* c);
mhs_status solve(mhs_ctx* c, double tol, int mode, mhs_solve_info* info);
void solve_begin(mhs_ctx* c, double tol, int mode);
mhs_status solve_end(mhs_ctx* c, double tol, int mode, mhs_solve_info* info);
mhs_status batch_solve(mhs_ctx** hs, int n, double tol, int mode, mhs_solve_info* infos, mhs_status* statuses);
template <typename T>
void vcycle(mhs_ctx* c, Hierarchy& H, int l);
template <typename T>
void smooth_hook(mhs_ctx* c, Hierarchy& H, int l);   // one sweep as the V-cycle runs it
double read_norm2(mhs_ctx* c, int slot);
void ensure_field_buffers(mhs_ctx* c);
void ensure_post_buffers(mhs_ctx* c);
// separable solver (kernels_sep.cu)
bool sep_level_ok(const Geom& g);   // sine transforms fast (nx - 1, ny - 1 powers of two) or short (nx, ny <= 66)
template <typename T>
void sep_tables(mhs_ctx* c, Hierarchy& H, int l);   // build level l's tables once (allocates: not while capturing)
template <typename T>
void sep_exact(mhs_ctx* c, Hierarchy& H, int l);    // u = A^{-1} f on level l (interior; r, t scratch)
void sep_refresh(mhs_ctx* c, Hierarchy& H);         // recompute the pivots of every built table (new coefficients)
template <typename T>
void sep_exact_plan(mhs_ctx* c, Hierarchy& H, int l, std::vector<SepStage<T>>& stages);   // sep_exact's launches
void sep_prepare(mhs_ctx* c, int mode);             // finest-level tables of both hierarchies for a solve mode
void sep_solve(mhs_ctx* c, Hierarchy& H);           // mixed mode: FP32 e = A^{-1} f on the finest level
bool sep_fp64_available(const mhs_ctx* c);          // FP64 direct solves: sep_level_ok of the finest grid
void sep_correct64(mhs_ctx* c, Hierarchy& H);       // FP64 mode: P += A^{-1} r on the finest level
void ensure_staging(mhs_ctx* c);
// device bytes of a handle for a grid (upper bound used for admission) and
// the bytes a handle holds (every allocation it made, plus field buffers not
// yet allocated)
size_t handle_bytes_estimate(int nx, int ny, int nz, double Lx, double Ly, double Lz);
size_t handle_bytes_held(const mhs_ctx* c);

// FP64 cycles of the finest level with the test after the pre-smoothing (level 0 above the sub-cycle cut-off)
bool rotated_cycles(const mhs_ctx* c, const Hierarchy& H);
// residuals right after red-black point sweeps, computed on red nodes only (FP64): a V-cycle level after its
// pre-smoothing, the test of a rotated cycle, the test after the full-multigrid first cycle
bool red_residual_level(const mhs_ctx* c, const Hierarchy& H);
bool red_residual_cycle(const mhs_ctx* c, const Hierarchy& H);
bool red_residual_fmg(const mhs_ctx* c, const Hierarchy& H);
bool red_residual_rotated(const mhs_ctx* c, const Hierarchy& H);

// conversions between the FP64 staging buffer and FP32 level arrays (kernels_mg.cu)
void launch_d2f(const double* src, float* dst, size_t n, cudaStream_t st);
void launch_pack(const double* src, double* dst, int nx, int px, size_t rows, cudaStream_t st);   // pitched -> dense
void launch_f2d(const float* src, double* dst, size_t n, cudaStream_t st);

}  // namespace mhs
