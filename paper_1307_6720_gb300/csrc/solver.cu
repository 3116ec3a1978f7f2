// Host-side multigrid driver: hierarchy construction, V-cycles, the FP64
// and the FP32-in-FP64 (defect correction) solves of Sect. 2.2 steps 2-3, and
// field recovery (steps 4-5).  Every arithmetic step runs in the kernels of
// kernels_mg.cu / kernels_fields.cu; this file only sequences launches.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
    if (e != cudaSuccess) {
        char buf[512];
        std::snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
        throw Error(MHS_ERR_CUDA, buf);
    }
}

Geom make_geom(int nx, int ny, int nz, double Lx, double Ly, double Lz) {
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.px = int(round_up(size_t(nx), 4));
    g.plane = size_t(g.px) * ny;
    g.n = g.plane * nz;
    g.hx = Lx / (nx - 1);
    g.hy = Ly / (ny - 1);
    g.hz = nz > 1 ? Lz / (nz - 1) : 0.0;
    return g;
}

static bool coarsenable(int n) { return n >= 5 && (n - 1) % 2 == 0; }

static void* dev_alloc(mhs_ctx* c, size_t bytes) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error(MHS_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->allocations.push_back(p);
    c->dev_bytes += round_up(bytes ? bytes : 16, 256);
    MHS_CUDA(cudaMemsetAsync(p, 0, bytes ? bytes : 16, c->stream));
    return p;
}

// Smallest level count handled by the one-CTA sub-cycle: the sub-hierarchy
// from level l down must fit in shared memory (u and f per level) and the
// level must be small enough that one SM sweeps it quickly (FP64 runs at a
// small fraction of the FP32 rate on one SM, so its cut-off is lower).
static int choose_cut(const Hierarchy& H, size_t elem, size_t max_interior) {
    int cut = H.nlev() - 1;
    for (int l = H.nlev() - 1; l >= 0; --l) {
        size_t bytes = 0;
        const size_t coef = elem == 8 ? sizeof(PlaneCoef<double>) : sizeof(PlaneCoef<float>);
        for (int m = l; m < H.nlev(); ++m) bytes += 2 * round_up(H.g[m].n, 4) * elem + H.g[m].nz * coef;
        // the sub-cycle decodes node indices with float reciprocals (exact for rows of <= 1024 nodes)
        if (bytes > subcycle_smem_limit() || H.g[l].interior() > max_interior || H.g[l].nx - 2 > 1024 ||
            H.g[l].ny - 2 > 1024)
            break;
        cut = l;
    }
    return cut;
}

static void build_hierarchy(mhs_ctx* c, Hierarchy& H, int dim) {
    H.dim = dim;
    int nx = c->nx, ny = c->ny, nz = dim == 3 ? c->nz : 1;
    for (;;) {
        H.g.push_back(make_geom(nx, ny, nz, c->Lx, c->Ly, c->Lz));
        const bool can = coarsenable(nx) && coarsenable(ny) && (dim == 2 || coarsenable(nz));
        if (!can || H.g.size() == size_t(MAX_SUB_LEVELS)) break;
        nx = (nx - 1) / 2 + 1;
        ny = (ny - 1) / 2 + 1;
        if (dim == 3) nz = (nz - 1) / 2 + 1;
    }
    const Geom& gc = H.g.back();
    if (2 * gc.n * sizeof(double) > subcycle_smem_limit() || gc.nx - 2 > 1024 || gc.ny - 2 > 1024)
        throw Error(MHS_ERR_INVALID_ARG,
                    "coarsest multigrid level too large (" + std::to_string(gc.nx) + "x" + std::to_string(gc.ny) +
                        "x" + std::to_string(gc.nz) + "); use node counts of the form 2^k m + 1 with small m");
    for (const Geom& g : H.g) {
        LevelArrays<double> d;
        LevelArrays<float> s;
        d.u = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.f = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.r = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.t = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.coef = static_cast<PlaneCoef<double>*>(dev_alloc(c, g.nz * sizeof(PlaneCoef<double>)));
        s.u = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.f = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.r = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.t = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.coef = static_cast<PlaneCoef<float>*>(dev_alloc(c, g.nz * sizeof(PlaneCoef<float>)));
        H.d.push_back(d);
        H.s.push_back(s);
    }
    if (dim == 3) {
        H.tm_u.resize(2 * H.g.size());
        H.tm_t.resize(2 * H.g.size());
        H.tm_f.resize(2 * H.g.size());
        for (size_t l = 0; l < H.g.size(); ++l)
            for (int r = 0; r < 2; ++r) {   // tiles of 8 and of 16 rows
                make_plane_map(&H.tm_u[2 * l + r], H.g[l], H.s[l].u, 8 << r);
                make_plane_map(&H.tm_t[2 * l + r], H.g[l], H.s[l].t, 8 << r);
                make_plane_map(&H.tm_f[2 * l + r], H.g[l], H.s[l].f, 8 << r);
            }
    }
    const Geom& g0 = H.g[0];
    H.df.hi = static_cast<float*>(dev_alloc(c, g0.n * sizeof(float)));
    H.df.lo = static_cast<float*>(dev_alloc(c, g0.n * sizeof(float)));
    H.df.fh = static_cast<float*>(dev_alloc(c, g0.n * sizeof(float)));
    H.df.fl = static_cast<float*>(dev_alloc(c, g0.n * sizeof(float)));
    H.df.coef = static_cast<PlaneCoefDF*>(dev_alloc(c, g0.nz * sizeof(PlaneCoefDF)));
}

// Coarse-grid solve of the V-cycles by the separable solver: the first level
// below the finest with at most sep_coarse interior nodes whose transforms
// are available; -1 when none qualifies or the option is off.
static int choose_exact(const Hierarchy& H, int sep_coarse) {
    if (sep_coarse <= 0) return -1;
    for (int l = 1; l < H.nlev(); ++l)
        if (H.g[l].interior() <= size_t(sep_coarse) && sep_level_ok(H.g[l])) return l;
    return -1;
}

void choose_cuts(mhs_ctx* c) {
    for (Hierarchy* H : {&c->h3, &c->h2}) {
        H->cut64 = choose_cut(*H, sizeof(double), size_t(c->opts.cut64));
        H->cut32 = choose_cut(*H, sizeof(float), size_t(c->opts.cut32));
        const int e = choose_exact(*H, c->opts.sep_coarse);
        H->exact64 = e >= 1 && e <= H->cut64 ? e : -1;
        H->exact32 = e >= 1 && e <= H->cut32 ? e : -1;
        // tables now: graph capture must not allocate
        if (H->exact64 >= 0) sep_tables<double>(c, *H, H->exact64);
        if (H->exact32 >= 0) sep_tables<float>(c, *H, H->exact32);
    }
}

void compute_coefficients(mhs_ctx* c) {
    for (Hierarchy* H : {&c->h3, &c->h2}) {
        for (int l = 0; l < H->nlev(); ++l) {
            launch_coef<double>(H->g[l], H->dim, c->alpha, c->xi, H->d[l].coef, c->stream);
            launch_coef<float>(H->g[l], H->dim, c->alpha, c->xi, H->s[l].coef, c->stream);
        }
        launch_df_coef(H->g[0], H->d[0].coef, H->df.coef, c->stream);
    }
    launch_profiles(c->h3.g[0], c->xi, c->atm, c->prof, c->stream);
    // separable-solver pivots follow alpha and xi (tables live in device memory, so
    // captured graphs stay valid)
    for (Hierarchy* H : {&c->h3, &c->h2}) sep_refresh(c, *H);
    // the smoother may follow the anisotropy class; the graph key holds the choice,
    // so a captured solve is rebuilt only when the choice changes
    c->aniso = aniso_class(c);
}

void create(mhs_ctx* c) {
    MHS_CUDA(cudaEventCreate(&c->ev0));
    MHS_CUDA(cudaEventCreate(&c->ev1));
    MHS_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    MHS_CUDA(cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking));
    subcycle_prepare();
    build_hierarchy(c, c->h3, 3);
    build_hierarchy(c, c->h2, 2);
    c->ns.max_blocks = 65536;
    c->ns.partial = static_cast<double*>(dev_alloc(c, c->ns.max_blocks * sizeof(double)));
    c->ns.result = static_cast<double*>(dev_alloc(c, 16 * sizeof(double)));
    MHS_CUDA(cudaMallocHost(&c->ns.host, 16 * sizeof(double)));
    c->flag = static_cast<int*>(dev_alloc(c, 16 * sizeof(int)));
    MHS_CUDA(cudaMallocHost(&c->flag_host, 16 * sizeof(int)));
    c->ctl = static_cast<SolveCtl*>(dev_alloc(c, 2 * sizeof(SolveCtl)));
    MHS_CUDA(cudaMallocHost(&c->ctl_host, 2 * sizeof(SolveCtl)));
    c->bz = static_cast<double*>(dev_alloc(c, c->h2.g[0].n * sizeof(double)));
    c->prof = static_cast<double*>(dev_alloc(c, 8 * size_t(c->nz) * sizeof(double)));
    compute_coefficients(c);
    choose_cuts(c);   // after the coefficients: separable tables derive their pivots from them
    MHS_CUDA(cudaStreamSynchronize(c->stream));
}

void invalidate_graphs(mhs_ctx* c) {
    for (int m = 0; m < 2; ++m) {
        for (CachedGraph& e : c->graphs[m])
            if (e.exec) cudaGraphExecDestroy(e.exec);
        c->graphs[m].clear();
    }
}

void destroy(mhs_ctx* c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    invalidate_graphs(c);
    for (void* p : c->allocations) cudaFree(p);
    c->allocations.clear();
    if (c->ns.host) cudaFreeHost(c->ns.host);
    if (c->flag_host) cudaFreeHost(c->flag_host);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    if (c->staging) cudaFree(c->staging);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->bstream) cudaStreamDestroy(c->bstream);
    c->timer.destroy();
}

// ------------------------------- V-cycle ---------------------------------

template <typename T>
static LevelArrays<T>& arrays(Hierarchy& H, int l);
template <>
LevelArrays<double>& arrays<double>(Hierarchy& H, int l) { return H.d[l]; }
template <>
LevelArrays<float>& arrays<float>(Hierarchy& H, int l) { return H.s[l]; }

template <typename T>
static int cut_of(const Hierarchy& H) { return sizeof(T) == 8 ? H.cut64 : H.cut32; }
template <typename T>
static int exact_of(const Hierarchy& H) { return sizeof(T) == 8 ? H.exact64 : H.exact32; }

// V-cycle from level l down; levels at or below the cut-off run in one CTA.
template <typename T>
void subcycle(mhs_ctx* c, Hierarchy& H, int l) {
    SubParams<T> p{};
    p.nlev = H.nlev() - l;
    p.dim = H.dim;
    p.nu1 = c->opts.nu1;
    p.nu2 = c->opts.nu2;
    p.line = H.dim == 3 && use_zline(c) ? 1 : 0;
    // thread count from the cut-off level (not from l), so that every entry
    // into this hierarchy's sub-cycle uses the same CTA shape
    p.rows = subcycle_rows(H.g[std::min(cut_of<T>(H), H.nlev() - 1)].interior());
    size_t off = 0;
    for (int m = 0; m < p.nlev; ++m) {
        const Geom& g = H.g[l + m];
        p.L[m].g = g;
        p.L[m].coef = arrays<T>(H, l + m).coef;
        p.L[m].off_u = int(off);
        off += round_up(g.n, 4);
        p.L[m].off_f = int(off);
        off += round_up(g.n, 4);
    }
    p.u_g = arrays<T>(H, l).u;
    p.f_g = arrays<T>(H, l).f;
    size_t ncoef = 0;
    for (int m = 0; m < p.nlev; ++m) ncoef += size_t(H.g[l + m].nz);
    p.smem_bytes = round_up(ncoef * sizeof(PlaneCoef<T>), 16) + off * sizeof(T);
    if (p.smem_bytes > subcycle_smem_limit()) throw Error(MHS_ERR_INVALID_ARG, "sub-cycle does not fit shared memory");
    const bool dbl = sizeof(T) == 8;
    TimedScope t(c->timer, dbl ? MHS_KT_COARSE64 : MHS_KT_COARSE32, 2.0 * H.g[l].n * sizeof(T), 0.0, c->stream);
    launch_subcycle<T>(p, c->stream);
}

// n smoothing sweeps on level l.  With z-line smoothing (use_zline), 3D
// levels run zebra z-line sweeps (in place, the level's r as scratch).  Otherwise red-black
// sweeps: 3D levels use the fused out-of-place sweep (FP32 levels of at least
// fused_min interior nodes, FP64 with MHS_FLAG_FUSED_SWEEP64), alternating
// between u and its twin t; the rest the two colour passes in place.
template <typename T>
static void smooth_n(mhs_ctx* c, Hierarchy& H, int l, const T* f, int n, bool fine, double bytes, double flops) {
    LevelArrays<T>& A = arrays<T>(H, l);
    const Geom& g = H.g[l];
    const bool dbl = sizeof(T) == 8;
    if (H.dim == 3 && use_zline(c)) {
        for (int q = 0; q < n; ++q) {
            TimedScope t(c->timer, dbl ? MHS_KT_SMOOTH64 : MHS_KT_SMOOTH32, bytes, flops, c->stream, fine);
            launch_zline<T>(g, A.coef, A.u, f, A.r, c->stream);
        }
        return;
    }
    const bool fused = H.dim == 3 && A.t &&
                       (dbl ? (c->opts.flags & MHS_FLAG_FUSED_SWEEP64) != 0
                            : g.interior() >= size_t(c->opts.fused_min));
    // FP32 3D levels stage their planes by TMA (maps of u, t and f built at creation)
    const bool tma = fused && !dbl && !H.tm_u.empty() && !(c->opts.flags & MHS_FLAG_NO_TMA) &&
                     f == reinterpret_cast<const T*>(H.s[l].f);
    for (int q = 0; q < n; ++q) {
        TimedScope t(c->timer, dbl ? MHS_KT_SMOOTH64 : MHS_KT_SMOOTH32, bytes, flops, c->stream, fine);
        const bool even = (q & 1) == 0;
        if (tma) {
            const int rows = c->opts.tma_rows, m = 2 * l + (rows == 16 ? 1 : 0);
            launch_sweep_tma(g, rows, even ? H.tm_u[m] : H.tm_t[m], H.tm_f[m], H.s[l].coef,
                             even ? H.s[l].t : H.s[l].u, c->flag + 1, c->stream);
        } else if (fused) {
            launch_sweep<T>(g, A.coef, even ? A.u : A.t, f, even ? A.t : A.u, c->stream);
        } else {
            launch_smooth<T>(g, H.dim, A.coef, A.u, f, c->stream, c->opts.tile);
        }
    }
    if (fused && (n & 1)) MHS_CUDA(cudaMemcpyAsync(A.u, A.t, g.n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
}

// Per-level accounting and right-hand side of the V-cycle's operations on
// level l: f vanishes on the finest FP64 interior level (the Dirichlet data
// sits in u); algorithmic flops per node: the update u = f/d - ax(E+W) -
// ay(N+S) [- az(U+D)] takes 2 (3) additions, 2 (3) multiplications, 2 (3)
// subtractions and, with f, one more multiplication and subtraction; the
// residual f - A u adds the centre term (a multiplication and an addition).
template <typename T>
struct LevelOps {
    const T* f;
    double s, N, fs, upd_flops, res_flops;
    bool fine;
    LevelOps(mhs_ctx* c, Hierarchy& H, int l) {
        const bool dbl = sizeof(T) == 8;
        const Geom& g = H.g[l];
        s = sizeof(T);
        N = double(g.interior());
        const bool f_zero = dbl && l == 0 && H.dim == 3 && c->f_zero_finest;
        fs = f_zero ? 0.0 : s;
        f = f_zero ? nullptr : arrays<T>(H, l).f;
        upd_flops = H.dim == 3 ? (f_zero ? 8.0 : 10.0) : 7.0;
        res_flops = H.dim == 3 ? (f_zero ? 10.0 : 11.0) : 8.0;
        fine = H.dim == 3 && l == 0;
    }
};

// the coarse-grid correction of level l from its residual: restriction of
// the residual in A.r (unless the fused pass of FP32 levels has already
// restricted it; red: A.r is a residual taken on red nodes only), the coarser
// cycle, interpolation added to u
template <typename T>
static void coarse_correction(mhs_ctx* c, Hierarchy& H, int l, const LevelOps<T>& o, bool restricted,
                              bool red = false) {
    cudaStream_t st = c->stream;
    const bool dbl = sizeof(T) == 8;
    LevelArrays<T>& A = arrays<T>(H, l);
    LevelArrays<T>& C = arrays<T>(H, l + 1);
    const double N = o.N, s = o.s, Nc = double(H.g[l + 1].interior());
    if (!restricted) {
        TimedScope t(c->timer, dbl ? MHS_KT_RESTRICT64 : MHS_KT_RESTRICT32, (N + 2 * Nc) * s,
                     Nc * (H.dim == 3 ? 54.0 : 18.0), st, o.fine);
        launch_restrict<T>(H.g[l], H.g[l + 1], H.dim, A.r, C.f, C.u, st, red);
    }
    vcycle<T>(c, H, l + 1);
    {
        TimedScope t(c->timer, dbl ? MHS_KT_PROLONG64 : MHS_KT_PROLONG32, (2 * N + Nc) * s, 4.0 * N, st, o.fine);
        launch_prolong<T>(H.g[l + 1], H.g[l], H.dim, C.u, A.u, st);
    }
}

// Residuals taken right after red-black point sweeps (FP64 cycles; the FP32
// residuals of mixed mode stay full): red nodes computed, black nodes 0, as
// the black nodes, updated last, satisfy their own rows to rounding.  The
// solo solve and grouped solves take the same choices from these.
static bool point_smoothing(const mhs_ctx* c, const Hierarchy& H) { return H.dim == 2 || !use_zline(c); }

// a V-cycle level's residual after its pre-smoothing
bool red_residual_level(const mhs_ctx* c, const Hierarchy& H) { return point_smoothing(c, H) && c->opts.nu1 >= 1; }

template <typename T>
void vcycle(mhs_ctx* c, Hierarchy& H, int l) {
    cudaStream_t st = c->stream;
    if (l == exact_of<T>(H)) {
        // coarse-grid solve: A u = f exactly (u's interior overwritten; the
        // correction's boundary values are zero on coarse levels)
        const Geom& g = H.g[l];
        TimedScope t(c->timer, sizeof(T) == 8 ? MHS_KT_COARSE64 : MHS_KT_COARSE32, 2.0 * g.interior() * sizeof(T),
                     0.0, st);
        sep_exact<T>(c, H, l);
        return;
    }
    if (l >= cut_of<T>(H)) {
        subcycle<T>(c, H, l);
        return;
    }
    LevelArrays<T>& A = arrays<T>(H, l);
    const Geom& g = H.g[l];
    const bool dbl = sizeof(T) == 8;
    const LevelOps<T> o(c, H, l);
    const double sweep_bytes = o.N * (2 * o.s + o.fs);
    smooth_n<T>(c, H, l, o.f, c->opts.nu1, o.fine, sweep_bytes, o.N * o.upd_flops);
    if (!dbl) {
        // FP32 levels (bandwidth-bound): residual and restriction in one pass, the residual not
        // stored (u and f read, the coarse right-hand side and iterate written; flops of the
        // residual and of the 27-point (9-point) weighting per coarse node)
        LevelArrays<T>& C = arrays<T>(H, l + 1);
        const double Nc = double(H.g[l + 1].interior());
        TimedScope t(c->timer, MHS_KT_RESID32, o.N * (o.s + o.fs) + 2 * Nc * o.s,
                     o.N * o.res_flops + Nc * (H.dim == 3 ? 54.0 : 18.0), st, o.fine);
        launch_resid_restrict<T>(g, H.g[l + 1], H.dim, A.coef, A.u, o.f, C.f, C.u, st);
    } else {
        // FP64 levels (bound by the FP64 pipe, which the fused pass would not relieve): the
        // residual on red nodes after the sweep, then the restriction
        TimedScope t(c->timer, MHS_KT_RESID64, sweep_bytes, o.N * o.res_flops, st, o.fine);
        launch_residual<T>(g, H.dim, A.coef, A.u, o.f, A.r, nullptr, 0, st, red_residual_level(c, H));
    }
    coarse_correction<T>(c, H, l, o, !dbl, dbl && red_residual_level(c, H));
    smooth_n<T>(c, H, l, o.f, c->opts.nu2, o.fine, sweep_bytes, o.N * o.upd_flops);
}

// FP64 cycles of the finest level with the convergence test after the
// pre-smoothing: the coarse-grid correction of the residual of the latest
// test (in A.r), post-smoothing, then the next cycle's pre-smoothing; the
// residual of that iterate (with norm partials) serves both the test and the
// next restriction, so a cycle computes one finest-level residual instead of
// two.  Levels of nu1 + nu2 sweeps per cycle as in vcycle; the solve returns
// the iterate whose residual passed the test.  Needs level 0 above the
// sub-cycle cut-off.
bool rotated_cycles(const mhs_ctx* c, const Hierarchy& H) {
    (void)c;
    return H.cut64 >= 1 && H.nlev() > 1;
}

// the convergence test of a rotated cycle (after the pre-smoothing, or the
// post-smoothing when nu1 = 0), unless the step is a separable direct solve
bool red_residual_cycle(const mhs_ctx* c, const Hierarchy& H) {
    return rotated_cycles(c, H) && point_smoothing(c, H) && c->opts.nu1 + c->opts.nu2 >= 1 &&
           !((c->opts.flags & MHS_FLAG_SEPARABLE) && sep_fp64_available(c));
}

// the test after the full-multigrid first cycle (after level 0's post-smoothing)
bool red_residual_fmg(const mhs_ctx* c, const Hierarchy& H) {
    return rotated_cycles(c, H) && point_smoothing(c, H) && c->opts.nu2 >= 1;
}

// the residual that a rotated cycle restricts (that of the latest test: the
// full-multigrid cycle's for the first cycle, a rotated cycle's after it) is
// taken on red nodes whichever test it comes from; without the full-multigrid
// cycle the first one is the full residual of the solve's first test
bool red_residual_rotated(const mhs_ctx* c, const Hierarchy& H) {
    return red_residual_cycle(c, H) && red_residual_fmg(c, H) && !(c->opts.flags & MHS_FLAG_NO_FMG);
}

static void vcycle_rotated(mhs_ctx* c, Hierarchy& H) {
    const LevelOps<double> o(c, H, 0);
    const double sweep_bytes = o.N * (2 * o.s + o.fs);
    coarse_correction<double>(c, H, 0, o, false, red_residual_rotated(c, H));
    smooth_n<double>(c, H, 0, o.f, c->opts.nu2, o.fine, sweep_bytes, o.N * o.upd_flops);
    smooth_n<double>(c, H, 0, o.f, c->opts.nu1, o.fine, sweep_bytes, o.N * o.upd_flops);
}

// Levels whose red-black sweeps run out of place (u and its twin t taking
// turns as input and output): FP32 3D levels of at least fused_min interior
// nodes, FP64 3D levels with MHS_FLAG_FUSED_SWEEP64; not with z-line smoothing.
template <typename T>
static bool fused_level(const mhs_ctx* c, const Hierarchy& H, int l) {
    if (H.dim != 3 || use_zline(c)) return false;
    if (!arrays<T>(const_cast<Hierarchy&>(H), l).t) return false;
    return sizeof(T) == 8 ? (c->opts.flags & MHS_FLAG_FUSED_SWEEP64) != 0
                          : H.g[l].interior() >= size_t(c->opts.fused_min);
}

// An out-of-place sweep writes interior nodes only and reads t as the old
// iterate on every second sweep, so t's boundary faces must hold u's.  t is
// also scratch of the separable solver (a coarse-grid solve, or the inner
// solve of MHS_FLAG_SEPARABLE) and may hold anything there after a solve with
// other options: every solve, and every smoothing hook, copies the faces of
// u into t on the levels it sweeps out of place first.
template <typename T>
static void sync_twin_faces(mhs_ctx* c, Hierarchy& H, int l) {
    if (!fused_level<T>(c, H, l)) return;
    LevelArrays<T>& A = arrays<T>(H, l);
    launch_copy_faces<T>(H.g[l], A.u, A.t, c->stream);
}

template <typename T>
void smooth_hook(mhs_ctx* c, Hierarchy& H, int l) {
    sync_twin_faces<T>(c, H, l);
    smooth_n<T>(c, H, l, arrays<T>(H, l).f, 1, false, 0.0, 0.0);
}
template void smooth_hook<double>(mhs_ctx*, Hierarchy&, int);
template void smooth_hook<float>(mhs_ctx*, Hierarchy&, int);

// Full multigrid for the correction equation A e = r0 of level 0 (standard
// FMG with one V-cycle per level): r0 is restricted down the hierarchy
// (full weighting, coarse iterates zeroed), the coarsest part is solved by
// one V-cycle from the sub-cycle cut-off (or the coarsest level), and on the
// way up each level starts from the interpolated coarser solution and runs
// one V-cycle.  Level 0 adds the interpolated correction to its iterate
// (FP64: P itself with f; mixed: the FP32 correction e, zeroed beforehand)
// and runs its V-cycle on its own right-hand side.
template <typename T>
void fmg(mhs_ctx* c, Hierarchy& H, const T* r0) {
    const int L = H.nlev();
    if (L < 2) {
        vcycle<T>(c, H, 0);
        return;
    }
    cudaStream_t st = c->stream;
    launch_restrict<T>(H.g[0], H.g[1], H.dim, r0, arrays<T>(H, 1).f, arrays<T>(H, 1).u, st);
    int top = std::min(std::max(cut_of<T>(H), 1), L - 1);
    if (exact_of<T>(H) >= 1) top = std::min(top, exact_of<T>(H));
    for (int l = 1; l < top; ++l)
        launch_restrict<T>(H.g[l], H.g[l + 1], H.dim, arrays<T>(H, l).f, arrays<T>(H, l + 1).f,
                           arrays<T>(H, l + 1).u, st);
    vcycle<T>(c, H, top);
    for (int l = top - 1; l >= 0; --l) {
        launch_prolong<T>(H.g[l + 1], H.g[l], H.dim, arrays<T>(H, l + 1).u, arrays<T>(H, l).u, st);
        vcycle<T>(c, H, l);
    }
}

template void vcycle<double>(mhs_ctx*, Hierarchy&, int);
template void vcycle<float>(mhs_ctx*, Hierarchy&, int);

double read_norm2(mhs_ctx* c, int slot) {
    MHS_CUDA(cudaMemcpyAsync(c->ns.host + slot, c->ns.result + slot, sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
    MHS_CUDA(cudaStreamSynchronize(c->stream));
    return c->ns.host[slot];
}

// ------------------------- solve sequences ---------------------------------
//
// One solve = lower-boundary prologue, while(cond) {lower-boundary cycle},
// interior prologue, while(cond) {interior cycle}.  The convergence test is
// check_kernel on the device; in graph mode it drives the conditional while
// nodes, in eager mode the host reads the control block after each check.

struct Enq {
    mhs_ctx* c;
    int mode;
    bool graph;
    cudaGraphConditionalHandle hnd = 0;
};

// Precision of the lower-boundary solve: that of the solve, except that
// MHS_FLAG_LOWER_FP64 turns a mixed-mode lower-boundary solve into FP64
// cycles (its double-float iterate bounds the residual near 5e-12 on 257^2
// nodes and 2e-11 on 513^2); the interior solve keeps the mode it was given.
static int lower_mode(const mhs_ctx* c, int mode) {
    return (mode == MHS_MIXED && (c->opts.flags & MHS_FLAG_LOWER_FP64)) ? int(MHS_FP64) : mode;
}

// residual of the current iterate (FP64, or FP64 rounded into the FP32
// right-hand side in mixed mode) with norm partials; returns their count
static int residual_partials(mhs_ctx* c, Hierarchy& H, int mode, bool red = false) {
    const Geom& g = H.g[0];
    LevelArrays<double>& A = H.d[0];
    const double N = double(g.interior());
    const bool fz = H.dim == 3 && c->f_zero_finest;   // f = 0: not read
    // bytes: u read, r written, f read unless zero; flops: the residual (10 in 3D
    // without f, 11 with f, 8 in 2D) and the square-accumulate of the norm (2)
    const double fb = fz ? 0.0 : 8.0;
    const double fl = (H.dim == 3 ? (fz ? 10.0 : 11.0) : 8.0) + 2.0;
    if (mode == MHS_MIXED) {
        // double-float residual of P = hi + lo, rounded into the FP32 right-hand side
        TimedScope t(c->timer, MHS_KT_RESID_MIXED, N * (8.0 + (fz ? 0.0 : 8.0) + 4.0), N * 70.0, c->stream,
                     H.dim == 3);
        return launch_df_residual(g, H.dim, H.df.coef, H.df.hi, H.df.lo, fz ? nullptr : H.df.fh,
                                  fz ? nullptr : H.df.fl, H.s[0].f, c->ns.partial, c->ns.max_blocks, c->stream);
    }
    TimedScope t(c->timer, MHS_KT_RESID64, N * (16.0 + fb), N * fl * (red ? 0.5 : 1.0), c->stream, H.dim == 3);
    return launch_residual<double>(g, H.dim, A.coef, A.u, fz ? nullptr : A.f, A.r, c->ns.partial, c->ns.max_blocks,
                                   c->stream, red);
}

static void cycle_body(const Enq& e, Hierarchy& H, SolveCtl* ctl) {
    mhs_ctx* c = e.c;
    const Geom& g = H.g[0];
    if (e.mode == MHS_MIXED) {
        MHS_CUDA(cudaMemsetAsync(H.s[0].u, 0, g.n * sizeof(float), c->stream));
        if (c->opts.flags & MHS_FLAG_SEPARABLE) {
            const double N = double(g.interior());
            TimedScope t(c->timer, MHS_KT_SEPARABLE, N * 4.0 * 2.0, 0.0, c->stream, H.dim == 3);
            sep_solve(c, H);
        } else {
            for (int q = 0; q < c->opts.inner_cycles; ++q) vcycle<float>(c, H, 0);
        }
        TimedScope t(c->timer, MHS_KT_CORRECT, double(g.interior()) * 20.0, double(g.interior()) * 8.0, c->stream,
                     H.dim == 3);
        launch_df_correct(g, H.dim, H.s[0].u, H.df.hi, H.df.lo, c->stream);
    } else if ((c->opts.flags & MHS_FLAG_SEPARABLE) && sep_fp64_available(c)) {
        // direct solve of the correction from the residual of the latest check
        const double N = double(g.interior());
        TimedScope t(c->timer, MHS_KT_SEPARABLE, N * 8.0 * 3.0, 0.0, c->stream, H.dim == 3);
        sep_correct64(c, H);
    } else if (rotated_cycles(c, H)) {
        vcycle_rotated(c, H);
    } else {
        vcycle<double>(c, H, 0);
    }
    const int nb = residual_partials(c, H, e.mode, e.mode == MHS_FP64 && red_residual_cycle(c, H));
    launch_check(c->ns.partial, nb, ctl, 0, e.hnd, e.graph ? 1 : 0, c->stream);
}

// First cycle of a solve by full multigrid (skipped with MHS_FLAG_NO_FMG):
// FP64 mode corrects P from its residual in A.r, mixed mode builds the FP32
// correction from the double-float residual in S.f.  It runs right after the
// first convergence test; when that test already passed, the kernels still
// run (a zero or tiny correction) but no cycle is counted.
static void fmg_cycle(const Enq& e, Hierarchy& H, SolveCtl* ctl) {
    mhs_ctx* c = e.c;
    if (c->opts.flags & MHS_FLAG_NO_FMG) return;
    if ((c->opts.flags & MHS_FLAG_SEPARABLE) && (e.mode == MHS_MIXED || sep_fp64_available(c)))
        return;   // the first separable step already solves the correction equation
    const Geom& g = H.g[0];
    if (e.mode == MHS_MIXED) {
        MHS_CUDA(cudaMemsetAsync(H.s[0].u, 0, g.n * sizeof(float), c->stream));
        fmg<float>(c, H, H.s[0].f);
        TimedScope t(c->timer, MHS_KT_CORRECT, double(g.interior()) * 20.0, double(g.interior()) * 8.0, c->stream,
                     H.dim == 3);
        launch_df_correct(g, H.dim, H.s[0].u, H.df.hi, H.df.lo, c->stream);
    } else {
        fmg<double>(c, H, H.d[0].r);
    }
    const int nb = residual_partials(c, H, e.mode, e.mode == MHS_FP64 && red_residual_fmg(c, H));
    launch_check(c->ns.partial, nb, ctl, 2, e.hnd, e.graph ? 1 : 0, c->stream);
}

static void prologue_2d(const Enq& e) {
    mhs_ctx* c = e.c;
    Hierarchy& H = c->h2;
    const Geom& g = H.g[0];
    {
        TimedScope t(c->timer, MHS_KT_OTHER, 0.0, 0.0, c->stream);
        MHS_CUDA(cudaMemsetAsync(H.d[0].u, 0, g.n * sizeof(double), c->stream));
        launch_lower_rhs(g, c->bz, H.d[0].f, c->stream);
        if (e.mode == MHS_MIXED) {
            MHS_CUDA(cudaMemsetAsync(H.df.hi, 0, g.n * sizeof(float), c->stream));
            MHS_CUDA(cudaMemsetAsync(H.df.lo, 0, g.n * sizeof(float), c->stream));
            launch_df_split(g, 2, H.d[0].f, H.df.fh, H.df.fl, c->stream);
        }
        // with u = 0 the residual is the right-hand side: its norm is ||b||
        const int nb = residual_partials(c, H, e.mode);
        launch_bnorm(c->ns.partial, nb, c->ctl + 0, c->stream);
        launch_check(c->ns.partial, nb, c->ctl + 0, 1, e.hnd, e.graph ? 1 : 0, c->stream);
    }
    // the first cycle's kernels are timed under their own kinds
    fmg_cycle(e, H, c->ctl + 0);
}

static void prologue_3d(const Enq& e) {
    mhs_ctx* c = e.c;
    Hierarchy& H = c->h3;
    const Geom& g = H.g[0];
    {
        TimedScope t(c->timer, MHS_KT_OTHER, 0.0, 0.0, c->stream);
        // P = 0 everywhere (Sect. 2.2, step 1), unless a warm start keeps the resident iterate
        const bool warm = c->opts.flags & MHS_FLAG_WARM;
        if (!warm) MHS_CUDA(cudaMemsetAsync(H.d[0].u, 0, g.n * sizeof(double), c->stream));
        launch_copy_plane(c->h2.g[0], c->h2.d[0].u, g, H.d[0].u, c->stream);
        // the twin of u used by out-of-place sweeps carries the same Dirichlet data
        launch_copy_plane(c->h2.g[0], c->h2.d[0].u, g, H.d[0].t, c->stream);
        if (e.mode == MHS_MIXED) {
            if (warm) {
                launch_df_split(g, 3, H.d[0].u, H.df.hi, H.df.lo, c->stream);
            } else {
                MHS_CUDA(cudaMemsetAsync(H.df.hi, 0, g.n * sizeof(float), c->stream));
                MHS_CUDA(cudaMemsetAsync(H.df.lo, 0, g.n * sizeof(float), c->stream));
            }
            // the Dirichlet plane in double-float form: the lower-boundary iterate itself, or the
            // split of its FP64 solution when that problem ran in FP64 cycles
            if (lower_mode(c, e.mode) != e.mode)
                launch_df_split(c->h2.g[0], 2, c->h2.d[0].u, c->h2.df.hi, c->h2.df.lo, c->stream);
            launch_df_copy_plane(c->h2.g[0], c->h2.df.hi, c->h2.df.lo, g, H.df.hi, H.df.lo, c->stream);
            if (!c->f_zero_finest) launch_df_split(g, 3, H.d[0].f, H.df.fh, H.df.fl, c->stream);
        }
        // twins of the levels swept out of place: u's boundary faces (level 0: the Dirichlet data)
        for (int l = 0; l < H.nlev(); ++l) {
            if (e.mode == MHS_MIXED) sync_twin_faces<float>(c, H, l);
            else sync_twin_faces<double>(c, H, l);
        }
        const int nl = launch_lift_norm(g, H.d[0].coef, H.d[0].u, c->ns.partial, c->stream);
        launch_bnorm(c->ns.partial, nl, c->ctl + 1, c->stream);
        const int nb = residual_partials(c, H, e.mode);
        launch_check(c->ns.partial, nb, c->ctl + 1, 1, e.hnd, e.graph ? 1 : 0, c->stream);
    }
    fmg_cycle(e, H, c->ctl + 1);
}

// Mixed mode keeps the finest iterate as a double-float pair; after the
// cycles it becomes the FP64 solution P that the rest of the library reads.
static void epilogue(const Enq& e, Hierarchy& H) {
    if (e.mode != MHS_MIXED) return;
    TimedScope t(e.c->timer, MHS_KT_OTHER, 0.0, 0.0, e.c->stream);
    launch_df_to_double(H.g[0], H.df.hi, H.df.lo, H.d[0].u, e.c->stream);
}

// Append a while node to the graph being captured on c->stream whose body
// is captured from fn on the second capture stream.
template <typename F>
static void add_while(mhs_ctx* c, cudaGraphConditionalHandle hnd, F&& fn) {
    cudaStreamCaptureStatus status;
    cudaGraph_t graph;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    MHS_CUDA(cudaStreamGetCaptureInfo(c->stream, &status, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MHS_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    MHS_CUDA(cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t outer = c->stream;
    c->stream = c->cap_stream2;
    MHS_CUDA(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    fn();
    cudaGraph_t captured;
    MHS_CUDA(cudaStreamEndCapture(c->stream, &captured));
    c->stream = outer;
}

// The options a captured solve is built from (sweeps, cut-offs, coarse solve,
// thresholds, graph-relevant flags) and the derived choices (smoother, zero
// finest right-hand side).  The tolerance and the cycle limit live in device
// memory, not in the graph.
static GraphKey graph_key(mhs_ctx* c) {
    const int flags = c->opts.flags & ~(MHS_FLAG_NO_GRAPH | MHS_FLAG_ZLINE | MHS_FLAG_POINT | MHS_FLAG_BZ_MIMETIC);
    return GraphKey{{c->opts.nu1, c->opts.nu2, c->opts.inner_cycles, flags, c->opts.cut64, c->opts.cut32,
                     c->opts.fused_min, c->opts.sep_coarse, c->f_zero_finest ? 1 : 0, use_zline(c) ? 1 : 0,
                     c->opts.tile, c->opts.tma_rows}};
}

constexpr size_t GRAPH_CACHE = 8;   // captured solves kept per precision mode

static void build_graph(mhs_ctx* c, int mode) {
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaGraph_t graph = nullptr;
    try {
        MHS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaStreamCaptureStatus status;
        cudaGraph_t g;
        MHS_CUDA(cudaStreamGetCaptureInfo(c->stream, &status, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h2, h3;
        MHS_CUDA(cudaGraphConditionalHandleCreate(&h2, g, 0, cudaGraphCondAssignDefault));
        MHS_CUDA(cudaGraphConditionalHandleCreate(&h3, g, 0, cudaGraphCondAssignDefault));
        Enq e2{c, lower_mode(c, mode), true, h2}, e3{c, mode, true, h3};
        // kernel counts per section (prologues once, bodies once per cycle), so that
        // launch accounting can add what a graph launch actually ran
        const long long l0 = launches();
        prologue_2d(e2);
        const long long l1 = launches();
        add_while(c, h2, [&] { cycle_body(e2, c->h2, c->ctl + 0); });
        const long long l2 = launches();
        epilogue(e2, c->h2);
        prologue_3d(e3);
        const long long l3 = launches();
        add_while(c, h3, [&] { cycle_body(e3, c->h3, c->ctl + 1); });
        const long long l4 = launches();
        epilogue(e3, c->h3);
        const long long l5 = launches();
        count_launches(-(l5 - l0));   // capture records kernels without running them
        CachedGraph e;
        e.count[0] = (l1 - l0) + (l3 - l2) + (l5 - l4);   // run once per solve
        e.count[1] = l2 - l1;                             // per lower-boundary cycle
        e.count[2] = 0;
        e.count[3] = l4 - l3;                             // per interior cycle
        MHS_CUDA(cudaStreamEndCapture(c->stream, &graph));
        MHS_CUDA(cudaGraphInstantiate(&e.exec, graph, 0));
        cudaGraphDestroy(graph);
        graph = nullptr;
        e.key = graph_key(c);
        std::vector<CachedGraph>& v = c->graphs[mode];
        if (v.size() >= GRAPH_CACHE) {   // evict the least recently used
            size_t lru = 0;
            for (size_t q = 1; q < v.size(); ++q)
                if (v[q].used < v[lru].used) lru = q;
            cudaGraphExecDestroy(v[lru].exec);
            v.erase(v.begin() + lru);
        }
        v.push_back(e);
    } catch (...) {
        cudaGraph_t junk;
        if (cudaStreamEndCapture(c->stream, &junk) == cudaSuccess && junk) cudaGraphDestroy(junk);
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        c->stream = user;
        throw;
    }
    c->stream = user;
}

// the cached graph of the current options, captured on first use
static CachedGraph& current_graph(mhs_ctx* c, int mode) {
    const GraphKey k = graph_key(c);
    for (CachedGraph& e : c->graphs[mode])
        if (e.key == k) return e;
    build_graph(c, mode);   // capture records work only; nothing runs until the launch
    return c->graphs[mode].back();
}

static bool read_cont(mhs_ctx* c, int which) {
    MHS_CUDA(cudaMemcpyAsync(c->ctl_host + which, c->ctl + which, sizeof(SolveCtl), cudaMemcpyDeviceToHost, c->stream));
    MHS_CUDA(cudaStreamSynchronize(c->stream));
    return c->ctl_host[which].cont != 0;
}

// Enqueue a solve on c->stream.  In graph mode nothing waits on the host;
// in eager mode (kernel timing enabled) the host drives the cycles.
void solve_begin(mhs_ctx* c, double tol, int mode) {
    cudaStream_t st = c->stream;
    if (c->opts.flags & MHS_FLAG_SEPARABLE) {   // allocations: not inside a graph capture
        sep_prepare(c, mode);
        if (lower_mode(c, mode) != mode && sep_fp64_available(c)) sep_tables<double>(c, c->h2, 0);
    }
    for (int q = 0; q < 2; ++q) {
        c->ctl_host[q] = SolveCtl{};
        c->ctl_host[q].tol = tol;
        c->ctl_host[q].max_cycles = c->opts.max_cycles;
    }
    MHS_CUDA(cudaMemcpyAsync(c->ctl, c->ctl_host, 2 * sizeof(SolveCtl), cudaMemcpyHostToDevice, st));
    MHS_CUDA(cudaMemsetAsync(c->flag + 1, 0, sizeof(int), st));   // bounded-wait expiry flag of the kernels
    MHS_CUDA(cudaEventRecord(c->ev0, st));
    c->pending_graph = c->use_graphs && !c->timer.enabled && !(c->opts.flags & MHS_FLAG_NO_GRAPH);
    if (c->pending_graph) {
        CachedGraph& e = current_graph(c, mode);
        e.used = ++c->graph_clock;
        for (int q = 0; q < 4; ++q) c->launched_count[q] = e.count[q];
        MHS_CUDA(cudaGraphLaunch(e.exec, st));
    } else {
        Enq e{c, mode, false, 0}, e2{c, lower_mode(c, mode), false, 0};
        prologue_2d(e2);
        while (read_cont(c, 0)) cycle_body(e2, c->h2, c->ctl + 0);
        epilogue(e2, c->h2);
        prologue_3d(e);
        while (read_cont(c, 1)) cycle_body(e, c->h3, c->ctl + 1);
        epilogue(e, c->h3);
    }
    MHS_CUDA(cudaEventRecord(c->ev1, st));
    MHS_CUDA(cudaMemcpyAsync(c->ctl_host, c->ctl, 2 * sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
    MHS_CUDA(cudaMemcpyAsync(c->flag_host + 1, c->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
}

// Wait for the solve enqueued by solve_begin and report it.
mhs_status solve_end(mhs_ctx* c, double tol, int mode, mhs_solve_info* info) {
    MHS_CUDA(cudaEventSynchronize(c->ev1));
    MHS_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0;
    MHS_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    const SolveCtl& a = c->ctl_host[0];
    const SolveCtl& b = c->ctl_host[1];
    if (c->pending_graph) {
        const long long* n = c->launched_count;
        count_launches(n[0] + a.bodies * n[1] + n[2] + b.bodies * n[3]);
    }
    if (info) {
        info->cycles_2d = a.cycles;
        info->cycles_3d = b.cycles;
        info->rel_res_2d = a.rel;
        info->rel_res_3d = b.rel;
        info->conv_factor = (b.cycles > 0 && b.rel0 > 0 && b.rel > 0) ? std::pow(b.rel / b.rel0, 1.0 / b.cycles) : 0.0;
        info->ms = ms;
        info->outer_iters_2d = lower_mode(c, mode) == MHS_MIXED ? a.cycles : 0;
        info->outer_iters_3d = mode == MHS_MIXED ? b.cycles : 0;
    }
    c->have_solution = true;
    if (c->flag_host[1]) throw Error(MHS_ERR_TIMEOUT, "a kernel's bounded wait for its TMA loads expired");
    if (a.status != MHS_OK || b.status != MHS_OK) throw Error(MHS_ERR_NONFINITE, "non-finite residual norm");
    const bool ok2 = a.bnorm == 0.0 || a.rel < tol;
    const bool ok3 = b.bnorm == 0.0 || b.rel < tol;
    if (!ok2 || !ok3) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "no convergence to %g in %d cycles (2D rel %.3e, 3D rel %.3e)", tol,
                      c->opts.max_cycles, a.rel, b.rel);
        throw Error(MHS_ERR_NO_CONVERGENCE, buf);
    }
    return MHS_OK;
}

mhs_status solve(mhs_ctx* c, double tol, int mode, mhs_solve_info* info) {
    solve_begin(c, tol, mode);
    return solve_end(c, tol, mode, info);
}

// Batched solve: every handle's solve runs on its own internal stream so that
// instances of different sizes overlap on the GPU; each instance runs exactly
// the kernels of its solo solve, so results do not depend on the batch.
mhs_status batch_solve(mhs_ctx** hs, int n, double tol, int mode, mhs_solve_info* infos, mhs_status* statuses) {
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = hs[q];
        if (!c->bstream) MHS_CUDA(cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
        // order the batch stream after any work already queued on the handle's stream
        MHS_CUDA(cudaEventRecord(c->ev0, c->stream));
        MHS_CUDA(cudaStreamWaitEvent(c->bstream, c->ev0, 0));
    }
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = hs[q];
        cudaStream_t user = c->stream;
        c->stream = c->bstream;
        try {
            solve_begin(c, tol, mode);
        } catch (...) {
            c->stream = user;
            throw;
        }
        c->stream = user;
    }
    mhs_status worst = MHS_OK;
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = hs[q];
        cudaStream_t user = c->stream;
        c->stream = c->bstream;
        mhs_status s = MHS_OK;
        try {
            s = solve_end(c, tol, mode, infos ? infos + q : nullptr);
        } catch (const Error& e) {
            s = e.status;
            if (s == MHS_ERR_CUDA) {
                c->stream = user;
                throw;
            }
        }
        c->stream = user;
        if (statuses) statuses[q] = s;
        if (s != MHS_OK && worst == MHS_OK) worst = s;
    }
    return worst;
}

void ensure_field_buffers(mhs_ctx* c) {
    if (c->fld[0]) return;
    for (int q = 0; q < 5; ++q) c->fld[q] = static_cast<double*>(dev_alloc(c, c->h3.g[0].n * sizeof(double)));
}

void ensure_post_buffers(mhs_ctx* c) {
    if (c->post[0]) return;
    for (int q = 0; q < 5; ++q) c->post[q] = static_cast<double*>(dev_alloc(c, c->h3.g[0].n * sizeof(double)));
}

void ensure_staging(mhs_ctx* c) {
    if (c->staging) return;
    MHS_CUDA(cudaMalloc(&c->staging, c->h3.g[0].n * sizeof(double)));
    c->dev_bytes += round_up(c->h3.g[0].n * sizeof(double), 256);
}

// Device bytes of a handle for an nx*ny*nz grid, from the same level
// geometry as build_hierarchy: per level of the interior and lower-boundary
// hierarchies u, f, r, t in FP64 and FP32 and the plane coefficients; the
// double-float state of each finest level; the norm scratch; the five field
// buffers; and separable-solver tables (mode pivots in both precisions) for
// every coarse level, an upper bound of what any coarse-grid choice builds.
size_t handle_bytes_estimate(int nx, int ny, int nz, double Lx, double Ly, double Lz) {
    const size_t q = 256;
    size_t b = 0;
    for (int dim : {3, 2}) {
        int x = nx, y = ny, z = dim == 3 ? nz : 1;
        for (int l = 0;; ++l) {
            const Geom g = make_geom(x, y, z, Lx, Ly, Lz);
            b += 4 * round_up(g.n * sizeof(double), q) + 4 * round_up(g.n * sizeof(float), q);
            b += round_up(g.nz * sizeof(PlaneCoef<double>), q) + round_up(g.nz * sizeof(PlaneCoef<float>), q);
            if (l == 0) {
                b += 4 * round_up(g.n * sizeof(float), q) + round_up(g.nz * sizeof(PlaneCoefDF), q);
                if (dim == 2) b += round_up(g.n * sizeof(double), q);   // B_z
            } else {
                if (dim == 3) b += 2 * round_up(g.interior() * (sizeof(double) + sizeof(float)), q);
                // mode eigenvalues and twiddles, or sine matrices of short rows, in both precisions
                b += 4 * round_up(size_t(x + y) * 2 * sizeof(double), q);
                if (x <= 66 && y <= 66) b += 2 * round_up(size_t(x * x + y * y) * sizeof(double), q);
            }
            const bool can = coarsenable(x) && coarsenable(y) && (dim == 2 || coarsenable(z));
            if (!can || l + 1 == MAX_SUB_LEVELS) break;
            x = (x - 1) / 2 + 1;
            y = (y - 1) / 2 + 1;
            if (dim == 3) z = (z - 1) / 2 + 1;
        }
    }
    const Geom g0 = make_geom(nx, ny, nz, Lx, Ly, Lz);
    b += 5 * round_up(g0.n * sizeof(double), q);                 // B_x, B_y, B_z, p, rho
    b += 65536 * sizeof(double) + 4096 + 8 * size_t(nz) * sizeof(double);   // norm scratch, flags, profiles
    return b;
}

// Bytes a resident handle holds now, plus the field buffers its first field
// recovery allocates.
size_t handle_bytes_held(const mhs_ctx* c) {
    size_t b = c->dev_bytes;
    if (!c->fld[0]) b += 5 * round_up(c->h3.g[0].n * sizeof(double), 256);
    return b;
}

}  // namespace mhs

namespace mhs {

int KernelTimer::begin(int k, double b, double f, cudaStream_t st, bool finest) {
    if (!enabled) return -1;
    if (2 * (used + 1) > pool.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            MHS_CUDA(cudaEventCreate(&e));
            pool.push_back(e);
        }
    }
    const int rec = int(used++);
    if (kind.size() < used) {
        kind.resize(used);
        fine.resize(used);
        bytes.resize(used);
        flops.resize(used);
    }
    kind[rec] = k;
    fine[rec] = finest ? 1 : 0;
    bytes[rec] = b;
    flops[rec] = f;
    MHS_CUDA(cudaEventRecord(pool[2 * rec], st));
    return rec;
}

void KernelTimer::end(int rec, cudaStream_t st) {
    if (rec < 0) return;
    cudaEventRecord(pool[2 * rec + 1], st);
}

void KernelTimer::collect() {
    for (size_t r = 0; r < used; ++r) {
        MHS_CUDA(cudaEventSynchronize(pool[2 * r + 1]));
        float m = 0;
        MHS_CUDA(cudaEventElapsedTime(&m, pool[2 * r], pool[2 * r + 1]));
        ms[kind[r]] += m;
        count[kind[r]] += 1;
        alg_bytes[kind[r]] += bytes[r];
        alg_flops[kind[r]] += flops[r];
        if (fine[r]) {
            ms0[kind[r]] += m;
            count0[kind[r]] += 1;
            alg_bytes0[kind[r]] += bytes[r];
            alg_flops0[kind[r]] += flops[r];
        }
    }
    used = 0;
}

void KernelTimer::reset() {
    collect();
    for (int k = 0; k < MHS_KT_COUNT; ++k) {
        ms[k] = alg_bytes[k] = alg_flops[k] = 0, count[k] = 0;
        ms0[k] = alg_bytes0[k] = alg_flops0[k] = 0, count0[k] = 0;
    }
}

void KernelTimer::destroy() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    used = 0;
}

}  // namespace mhs
