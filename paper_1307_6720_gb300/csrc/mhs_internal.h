// Internal declarations of libmhs (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mhs.h"

namespace mhs {

// Error carrying an mhs_status across internal C++ layers; caught at the ABI.
struct Error : std::runtime_error {
    mhs_status status;
    Error(mhs_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

void cuda_check(cudaError_t e, const char* what, const char* file, int line);

// Process-wide count of kernels this library has launched (mhs_kernel_launches).
void count_launches(long long n);
long long launches();
#define MHS_CUDA(call) ::mhs::cuda_check((call), #call, __FILE__, __LINE__)

__host__ __device__ inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Per-plane coefficients of the interior operator of eq. (scalar_pot) on one
// level: (A u)_ijk = cx_k (u_E + u_W) + cy_k (u_N + u_S) + cz (u_U + u_D) + d_k u_ijk,
// cx_k = (1 - xi(z_k))/hx^2, cy_k = (1 - xi(z_k))/hy^2, cz = 1/hz^2,
// d_k = -2 (cx_k + cy_k + cz) + alpha^2; inv_d = 1/d_k.
// For the lower-boundary operator of eq. (lower_bound): one plane with
// xi = 0, cz = 0, alpha = 0.
// ax = cx/d, ay = cy/d, az = cz/d let a Gauss-Seidel update be written as
// u = f/d - ax (u_E + u_W) - ay (u_N + u_S) - az (u_U + u_D).
template <typename T>
struct PlaneCoef {
    T cx, cy, cz, d, inv_d, ax, ay, az;
    // forward-elimination factors of the tridiagonal column systems solved by
    // the z-line smoother (the same for every column of the level):
    // lm = 1 / pivot_k, lsup = cz * lm, pivot_1 = d_1, pivot_k = d_k - cz lsup_{k-1}
    T lm, lsup;
    // alpha^2 - 2 cz, formed in FP64 before rounding: the part of the diagonal
    // that the separable solver's mode systems keep after the horizontal terms
    // are diagonalised (it would cancel against them if taken from d)
    T base;
    // partitioned column solve of the FP32 z-line smoother (line_body.cuh):
    // on a plane inside a segment, the segment's own elimination factors
    // (zlm = 1 / local pivot, zsup = cz zlm) and the segment solution's
    // responses zg, zh to unit values at its lower and upper interface planes;
    // on an interface plane, the factors of the interface system (zlm = 1 /
    // pivot, zsup = eliminated super-diagonal, zg = sub-diagonal, zh = 0)
    T zlm, zsup, zg, zh;
};

// Geometry of one level.  Device arrays are pitched: element (i,j,k) at
// i + px*(j + ny*k) with px = nx rounded up to a multiple of 4 elements, so
// every row starts on a 16-byte boundary for float and 32 bytes for double.
struct Geom {
    int nx = 0, ny = 0, nz = 0;   // nz = 1 for the lower-boundary plane
    int px = 0;                   // row pitch in elements
    size_t plane = 0;             // px * ny
    size_t n = 0;                 // plane * nz (allocated elements)
    double hx = 0, hy = 0, hz = 0;
    size_t interior() const { return size_t(nx - 2) * (ny - 2) * (nz > 1 ? nz - 2 : 1); }
};

Geom make_geom(int nx, int ny, int nz, double Lx, double Ly, double Lz);

// Arrays of one level for one precision.
template <typename T>
struct LevelArrays {
    T* u = nullptr;               // iterate (finest interior level: P, with Dirichlet data on the boundary)
    T* f = nullptr;               // right-hand side
    T* r = nullptr;               // residual
    T* t = nullptr;               // second iterate buffer for out-of-place sweeps (same boundary values as u)
    PlaneCoef<T>* coef = nullptr; // nz entries (device)
};

// Per-plane coefficients of the finest level as double-float pairs
// (value = hi + lo, each an FP32 word) for the FP32-only outer residual of
// mixed mode.
struct PlaneCoefDF {
    float cxh, cxl, cyh, cyl, czh, czl, dh, dl;
};

// Finest-level state of mixed mode: the outer iterate P = hi + lo and the
// right-hand side f = fh + fl as double-float pairs (FP32 words).
struct DFState {
    float *hi = nullptr, *lo = nullptr, *fh = nullptr, *fl = nullptr;
    PlaneCoefDF* coef = nullptr;
};

// Tables of the separable solver on one level (device, owned by the
// context's allocation list): the mode eigenvalues -4 sin^2(pi m / (2 (n - 1)))
// of the x and y second differences, either the FFT twiddles (nx - 1 and
// ny - 1 powers of two) or the dense sine matrices (short rows), and for 3D
// levels the elimination factors of every mode's tridiagonal system along z
// (inverse pivots and eliminated super-diagonals, in the layout of the
// transformed data), which depend on alpha and xi but not on the right-hand
// side.  Element type: double for sep64, float for sep32.
struct SepTables {
    void *mux = nullptr, *muy = nullptr;
    void *twx = nullptr, *twy = nullptr;
    void *sx = nullptr, *sy = nullptr;
    void *inv = nullptr, *sup = nullptr;
    bool ready = false;
};

struct Hierarchy {
    int dim = 3;                          // 3: interior, 2: lower boundary plane
    std::vector<Geom> g;                  // level geometries, 0 = finest
    std::vector<LevelArrays<double>> d;   // FP64 arrays
    std::vector<LevelArrays<float>> s;    // FP32 arrays
    int cut64 = 0, cut32 = 0;             // first level handled by the one-CTA sub-cycle (per precision)
    // level whose system the V-cycles of each precision solve exactly by the separable
    // solver: the chosen level when the cycle reaches it before the sub-cycle cut-off, else -1
    int exact64 = -1, exact32 = -1;
    std::vector<SepTables> sep64, sep32;  // separable-solver tables per level (built on demand)
    DFState df;                           // finest-level double-float state (mixed mode)
    // TMA plane maps of the FP32 arrays u, t, f per level (3D levels; see kernels_tma.cu)
    std::vector<CUtensorMap> tm_u, tm_t, tm_f;   // index 2 l + (tiles of 16 rows)
    int nlev() const { return int(g.size()); }
};

// Device-side control block of one iterative solve (lower-boundary or
// interior): the convergence test runs on the device so that the whole
// solve can be one CUDA graph with a conditional while node.
struct SolveCtl {
    double tol;        // stop when rel < tol
    double bnorm;      // ||b||_2 of the lifted right-hand side
    double rel0, rel;  // relative residual at the start / after the latest cycle
    int max_cycles;
    int cycles;
    int status;        // MHS_OK or MHS_ERR_NONFINITE
    int cont;          // 1 while another cycle is needed
    int bodies;        // cycles run by a while body (the full-multigrid cycle of the prologue is not one)
};

// One level of a multigrid sub-hierarchy solved inside a single CTA.
template <typename T>
struct SubLevel {
    Geom g;
    const PlaneCoef<T>* coef;
    int off_u, off_f;    // element offsets of u and f in dynamic shared memory
};

constexpr int MAX_SUB_LEVELS = 12;

template <typename T>
struct SubParams {
    int nlev, dim, nu1, nu2;
    int rows;            // the CTA is 32 x rows threads (8 for small sub-hierarchies, 32 otherwise)
    int line;            // 1: zebra z-line smoothing on 3D levels, 0: red-black point smoothing
    SubLevel<T> L[MAX_SUB_LEVELS];
    T* u_g;              // iterate of the top level in global memory (in/out)
    const T* f_g;        // right-hand side of the top level in global memory
    size_t smem_bytes;
};

// Device scratch for norms: per-block partial sums and the final values.
struct NormScratch {
    double* partial = nullptr;   // max_blocks entries
    double* result = nullptr;    // a few doubles (norm^2 slots)
    double* host = nullptr;      // pinned mirror of result
    int max_blocks = 0;
};

// Optional per-operation device timing with CUDA events on the handle's
// stream (off by default; enabled through mhs_set_kernel_timing).  Each
// timed operation adds its algorithmic bytes and flops so that achieved
// bandwidth and arithmetic rates can be formed from measured durations.
struct KernelTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;   // 2 events per record
    std::vector<int> kind;           // operation kind per record
    std::vector<char> fine;          // record belongs to the finest interior level
    std::vector<double> bytes, flops;
    size_t used = 0;
    double ms[MHS_KT_COUNT] = {};
    long long count[MHS_KT_COUNT] = {};
    double alg_bytes[MHS_KT_COUNT] = {};
    double alg_flops[MHS_KT_COUNT] = {};
    double ms0[MHS_KT_COUNT] = {};              // the same totals restricted to the finest interior level
    long long count0[MHS_KT_COUNT] = {};
    double alg_bytes0[MHS_KT_COUNT] = {};
    double alg_flops0[MHS_KT_COUNT] = {};

    // start a record; returns its index or -1 when disabled
    int begin(int k, double b, double f, cudaStream_t st, bool finest = false);
    void end(int rec, cudaStream_t st);
    void collect();   // synchronises on the recorded events and folds them into the totals
    void reset();
    void destroy();
};

struct TimedScope {
    KernelTimer& t;
    cudaStream_t st;
    int rec;
    TimedScope(KernelTimer& timer, int k, double b, double f, cudaStream_t s, bool finest = false)
        : t(timer), st(s), rec(timer.begin(k, b, f, s, finest)) {}
    ~TimedScope() { t.end(rec, st); }
};

}  // namespace mhs

namespace mhs {
// Everything a captured solve depends on besides device memory: the options
// and the choices derived from them and from the problem.
struct GraphKey {
    int v[12];
    bool operator==(const GraphKey& o) const {
        for (int q = 0; q < 12; ++q)
            if (v[q] != o.v[q]) return false;
        return true;
    }
};
struct CachedGraph {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    long long count[4] = {};    // kernels per graph section (see build_graph)
    unsigned long long used = 0;
};
}  // namespace mhs

struct mhs_ctx {
    int nx, ny, nz;
    double Lx, Ly, Lz, alpha;
    mhs_xi_params xi;
    mhs_atmos_params atm;
    mhs_solver_opts opts;
    int aniso = 0;                 // anisotropy class of the interior operator (set with the coefficients)
    cudaStream_t stream = nullptr;
    mhs::Hierarchy h3, h2;
    mhs::NormScratch ns;
    double* bz = nullptr;          // lower-boundary field [ny x px] (device, pitched)
    double* prof = nullptr;        // per fine plane: xi, dxi, p_b, rho_b and folded constants (8*nz doubles, device)
    int* flag = nullptr;           // device flags (non-finite input detection)
    int* flag_host = nullptr;      // pinned mirror
    double* staging = nullptr;     // FP64 staging buffer of the finest size (level hooks, lazily allocated)
    double* fld[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // pitched Bx, By, Bz, p, rho
    double* post[5] = {nullptr, nullptr, nullptr, nullptr, nullptr}; // pitched jx, jy, jz, |j|, |B| (on first use)
    bool have_bz = false, have_solution = false;
    bool f_zero_finest = true;     // the finest interior right-hand side is identically zero (no hook wrote it)
    std::vector<void*> allocations;
    size_t dev_bytes = 0;          // bytes of every device allocation the handle holds (server budget)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    mhs::KernelTimer timer;
    mhs::SolveCtl* ctl = nullptr;       // device control blocks [0] lower boundary, [1] interior
    mhs::SolveCtl* ctl_host = nullptr;  // pinned mirror
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;  // private streams for graph capture
    // captured solves per precision mode, one per option set (see graph_key in solver.cu), so that
    // switching between option sets (e.g. the autotuner's per-class choices in a server) replays
    // instead of recapturing; least recently used evicted beyond a few
    std::vector<mhs::CachedGraph> graphs[2];
    unsigned long long graph_clock = 0;
    long long launched_count[4] = {};                          // kernels per section of the launched graph
    bool use_graphs = true;
    bool pending_graph = false;                                 // the enqueued solve is a graph launch
    cudaStream_t bstream = nullptr;                             // stream of this handle inside batched solves
};

namespace mhs {

// ---- kernels (kernels_mg.cu) ----
template <typename T>
void launch_coef(const Geom& g, int dim, double alpha, const mhs_xi_params& xi, PlaneCoef<T>* coef,
                 cudaStream_t st);
void launch_profiles(const Geom& g, const mhs_xi_params& xi, const mhs_atmos_params& atm, double* prof,
                     cudaStream_t st);
template <typename T>
void launch_fill(T* a, size_t n, T v, cudaStream_t st);
template <typename T>
void launch_smooth(const Geom& g, int dim, const PlaneCoef<T>* coef, T* u, const T* f, cudaStream_t st, int tile = 1);
// residual r = f - A u; with partial != nullptr also per-block partial sums
// of r^2; returns the number of partials written.  red: u comes straight out
// of a red-black sweep, so the black nodes' residual is zero to rounding; they
// are stored as 0 and only the red nodes are computed (half the work)
template <typename T>
int launch_residual(const Geom& g, int dim, const PlaneCoef<T>* coef, const T* u, const T* f, T* r,
                    double* partial, int max_blocks, cudaStream_t st, bool red = false);
// finish partial sums into *out (fixed order)
void launch_norm_finish(const double* partial, int n, double* out, cudaStream_t st);
template <typename T>
void launch_restrict(const Geom& gf, const Geom& gc, int dim, const T* rf, T* fc, T* uc_zero, cudaStream_t st,
                     bool red = false);   // red: rf is zero at black nodes (restrict_body)
template <typename T>
void launch_prolong(const Geom& gc, const Geom& gf, int dim, const T* uc, T* uf, cudaStream_t st);
// residual of u and its full-weighting restriction to fc in one launch (the
// residual is not stored), uc zeroed
template <typename T>
void launch_resid_restrict(const Geom& gf, const Geom& gc, int dim, const PlaneCoef<T>* coef, const T* u, const T* f,
                           T* fc, T* uc, cudaStream_t st);
template <typename T>
void launch_coarse(const Geom& g, int dim, const PlaneCoef<T>* coef, T* u, const T* f, cudaStream_t st);
// lower-boundary right-hand side f = -B_z at interior nodes (FP64 and FP32 copies)
void launch_lower_rhs(const Geom& g, const double* bz, double* f64, cudaStream_t st);
template <typename T>
void launch_zero_interior(const Geom& g, int dim, T* u, cudaStream_t st);
// dst = src on the six boundary faces of a 3D level
template <typename T>
void launch_copy_faces(const Geom& g, const T* src, T* dst, cudaStream_t st);
void launch_copy_plane(const Geom& g2, const double* src2d, const Geom& g3, double* dst3d, cudaStream_t st);
void launch_count_nonfinite(const Geom& g, const double* bz, int* flag, cudaStream_t st);
// norm^2 of the lifted right-hand side of the interior problem: cz * P[k=0] on plane k=1
int launch_lift_norm(const Geom& g3, const PlaneCoef<double>* coef, const double* u, double* partial,
                     cudaStream_t st);

// ---- fused out-of-place red-black sweep (kernels_sweep.cu) ----
template <typename T>
void launch_sweep(const Geom& g, const PlaneCoef<T>* coef, const T* uin, const T* f, T* uout, cudaStream_t st);

// ---- discrete sine transforms of lines (kernels_dst.cu) ----
// lines of N = L - 1 elements, L a power of two: element i of line l of plane p
// at in + p in_plane + l in_line + i; result element m at
// out + p out_plane + l out_line + m out_elem (out_elem = 1: lines; else transposed, out_line = 1)
template <typename T>
struct DstArgs {
    int L = 0, log2n = 0, lines = 0, planes = 0, pairs = 0;   // L = N (power of two), log2n = log2 L
    const T* in = nullptr;
    long long in_plane = 0, in_line = 0;
    T* out = nullptr;
    long long out_plane = 0, out_line = 0, out_elem = 1;
    T scale = T(1);
    int accumulate = 0;         // 1: out += result instead of out = result
    const void* tw = nullptr;   // complex twiddles e^{-2 pi i q / (2L)}, q < L
};
template <typename T>
void* make_twiddles(int L, size_t* bytes = nullptr);

// ---- stages of one separable solve (kernels_sep.cu, kernels_dst.cu) ----
// C_b = scale A_b B_b (+ C_b with accumulate), b < batch, row-major with
// leading dimensions and batch strides (0: shared by the batch)
template <typename T>
struct GemmArgs {
    int M = 0, N = 0, K = 0;
    const T* A = nullptr;
    long long lda = 0, sA = 0;
    const T* B = nullptr;
    long long ldb = 0, sB = 0;
    T* C = nullptr;
    long long ldc = 0, sC = 0;
    T scale = T(1);
    int accumulate = 0;
};
// mode systems on transformed data t[k][slow][fast] (k < nzi; nzi = 1: the
// lower-boundary division by cf mu_fast + cs mu_slow)
template <typename T>
struct ModeArgs {
    int nfast = 0, nslow = 0, nzi = 0;
    const PlaneCoef<T>* coef = nullptr;
    const T* inv = nullptr;     // elimination factors (3D)
    const T* sup = nullptr;
    T* t = nullptr;
    const T* mufast = nullptr;  // mode eigenvalues (2D)
    const T* muslow = nullptr;
    T cf = T(0), cs = T(0);
};
enum SepKind { SEP_DST = 0, SEP_GEMM = 1, SEP_SCAN = 2, SEP_THOMAS = 3, SEP_DIVIDE = 4 };
// one kernel launch of a separable solve with its launch shape
template <typename T>
struct SepStage {
    int kind = SEP_DST;
    dim3 grid;
    int threads = 0;
    size_t smem = 0;
    DstArgs<T> dst;
    GemmArgs<T> gemm;
    ModeArgs<T> mode;
};
// launch shape of a sine-transform stage (sets a.pairs)
template <typename T>
void dst_shape(DstArgs<T>& a, dim3& grid, int& threads, size_t& smem);
template <typename T>
void launch_dst_stage(const SepStage<T>& s, cudaStream_t st);
// any stage of a separable solve (transform, dense product, mode solves)
template <typename T>
void launch_sep_stage(const SepStage<T>& s, cudaStream_t st);
// separable solve of one level with per-plane transforms in thread-block
// clusters (kernels_sepplane.cu); false (nothing launched) when the level does
// not qualify.  mode_solve: the 3D mode-solve stage on t.
template <typename T>
bool plane_level_solve(const Geom& g, int dim, const SepTables& tab, const T* f, T* t, T* out, bool accumulate,
                       const SepStage<T>* mode_solve, cudaStream_t st);
template <typename T>
int plane_cluster_size(const Geom& g, int dim);

// ---- zebra z-line Gauss-Seidel sweep, both colours (kernels_line.cu); scratch holds g.n elements ----
template <typename T>
void launch_zline(const Geom& g, const PlaneCoef<T>* coef, T* u, const T* f, T* scratch, cudaStream_t st);

// ---- post-processing (kernels_post.cu) ----
void launch_current(const Geom& g, double mu0, const double* Bx, const double* By, const double* Bz, double* jx,
                    double* jy, double* jz, double* jmag, double* bmag, cudaStream_t st);
void launch_trace(int nx, int ny, int nz, double Lx, double Ly, double Lz, size_t px, size_t plane, const double* Bx,
                  const double* By, const double* Bz, const double* seeds, int n, double ds, int max_steps,
                  double dir, double* points, int* lengths, cudaStream_t st);

// ---- TMA-staged fused sweep for FP32 levels (kernels_tma.cu) ----
void make_plane_map(CUtensorMap* map, const Geom& g, const float* base, int rows);
void launch_sweep_tma(const Geom& g, int rows, const CUtensorMap& tm_in, const CUtensorMap& tm_f,
                      const PlaneCoef<float>* coef, float* uout, int* err, cudaStream_t st);

// ---- control and sub-cycle (kernels_ctl.cu) ----
void launch_bnorm(const double* partial, int n, SolveCtl* ctl, cudaStream_t st);
void launch_check(const double* partial, int n, SolveCtl* ctl, int first, cudaGraphConditionalHandle handle,
                  int use_handle, cudaStream_t st);
size_t subcycle_smem_limit();
// rows of 32 threads of the sub-cycle CTA of a hierarchy cut at a level with
// `interior` interior nodes: small coarse problems pay mostly for block-wide
// barriers, which are cheaper with fewer warps
inline int subcycle_rows(size_t interior) { return interior <= 2048 ? 8 : 32; }
void subcycle_prepare();
template <typename T>
void launch_subcycle(const SubParams<T>& p, cudaStream_t st);

// ---- double-float outer loop of mixed mode (kernels_df.cu) ----
void launch_df_coef(const Geom& g, const PlaneCoef<double>* coef, PlaneCoefDF* cdf, cudaStream_t st);
// (fh, fl) <- f (double) at interior nodes (f == nullptr: zero)
void launch_df_split(const Geom& g, int dim, const double* f, float* hi, float* lo, cudaStream_t st);
// r32 = fh + fl - A (hi + lo) rounded to FP32, with per-block partial sums of r32^2; returns the partial count
int launch_df_residual(const Geom& g, int dim, const PlaneCoefDF* cdf, const float* hi, const float* lo,
                       const float* fh, const float* fl, float* r32, double* partial, int max_blocks, cudaStream_t st);
// (hi, lo) += e at interior nodes
void launch_df_correct(const Geom& g, int dim, const float* e, float* hi, float* lo, cudaStream_t st);
// P = hi + lo (double) at every node
void launch_df_to_double(const Geom& g, const float* hi, const float* lo, double* P, cudaStream_t st);
// plane k = 0 of a 3D double-float pair from a 2D pair
void launch_df_copy_plane(const Geom& g2, const float* hi2, const float* lo2, const Geom& g3, float* hi3, float* lo3,
                          cudaStream_t st);

// ---- fields (kernels_fields.cu) ----
void launch_fields(const Geom& g, double alpha, const mhs_atmos_params& atm, const double* prof,
                   const double* P, double* Bx, double* By, double* Bz, double* p, double* rho, int bz_mode,
                   cudaStream_t st);

}  // namespace mhs
