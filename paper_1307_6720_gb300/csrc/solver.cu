// Host-side multigrid driver: hierarchy construction, V-cycles, the FP64
// and the FP32-in-FP64 (defect correction) solves of Sect. 2.2 steps 2-3, and
// field recovery (steps 4-5).  Every arithmetic step runs in the kernels of
// kernels_mg.cu / kernels_fields.cu; this file only sequences launches.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

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
    MHS_CUDA(cudaMemsetAsync(p, 0, bytes ? bytes : 16, c->stream));
    return p;
}

static void build_hierarchy(mhs_ctx* c, Hierarchy& H, int dim) {
    H.dim = dim;
    int nx = c->nx, ny = c->ny, nz = dim == 3 ? c->nz : 1;
    for (;;) {
        H.g.push_back(make_geom(nx, ny, nz, c->Lx, c->Ly, c->Lz));
        const bool can = coarsenable(nx) && coarsenable(ny) && (dim == 2 || coarsenable(nz));
        if (!can || H.g.size() == 24) break;
        nx = (nx - 1) / 2 + 1;
        ny = (ny - 1) / 2 + 1;
        if (dim == 3) nz = (nz - 1) / 2 + 1;
    }
    const Geom& gc = H.g.back();
    if (2 * gc.n * sizeof(double) > 200 * 1024)
        throw Error(MHS_ERR_INVALID_ARG,
                    "coarsest multigrid level too large (" + std::to_string(gc.nx) + "x" + std::to_string(gc.ny) +
                        "x" + std::to_string(gc.nz) + "); use node counts of the form 2^k m + 1 with small m");
    for (const Geom& g : H.g) {
        LevelArrays<double> d;
        LevelArrays<float> s;
        d.u = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.f = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.r = static_cast<double*>(dev_alloc(c, g.n * sizeof(double)));
        d.coef = static_cast<PlaneCoef<double>*>(dev_alloc(c, g.nz * sizeof(PlaneCoef<double>)));
        s.u = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.f = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.r = static_cast<float*>(dev_alloc(c, g.n * sizeof(float)));
        s.coef = static_cast<PlaneCoef<float>*>(dev_alloc(c, g.nz * sizeof(PlaneCoef<float>)));
        H.d.push_back(d);
        H.s.push_back(s);
    }
}

void compute_coefficients(mhs_ctx* c) {
    for (Hierarchy* H : {&c->h3, &c->h2}) {
        for (int l = 0; l < H->nlev(); ++l) {
            launch_coef<double>(H->g[l], H->dim, c->alpha, c->xi, H->d[l].coef, c->stream);
            launch_coef<float>(H->g[l], H->dim, c->alpha, c->xi, H->s[l].coef, c->stream);
        }
    }
    launch_profiles(c->h3.g[0], c->xi, c->atm, c->prof, c->stream);
}

void create(mhs_ctx* c) {
    MHS_CUDA(cudaEventCreate(&c->ev0));
    MHS_CUDA(cudaEventCreate(&c->ev1));
    build_hierarchy(c, c->h3, 3);
    build_hierarchy(c, c->h2, 2);
    c->ns.max_blocks = 65536;
    c->ns.partial = static_cast<double*>(dev_alloc(c, c->ns.max_blocks * sizeof(double)));
    c->ns.result = static_cast<double*>(dev_alloc(c, 16 * sizeof(double)));
    MHS_CUDA(cudaMallocHost(&c->ns.host, 16 * sizeof(double)));
    c->flag = static_cast<int*>(dev_alloc(c, 16 * sizeof(int)));
    MHS_CUDA(cudaMallocHost(&c->flag_host, 16 * sizeof(int)));
    c->bz = static_cast<double*>(dev_alloc(c, c->h2.g[0].n * sizeof(double)));
    c->prof = static_cast<double*>(dev_alloc(c, 4 * size_t(c->nz) * sizeof(double)));
    compute_coefficients(c);
    MHS_CUDA(cudaStreamSynchronize(c->stream));
}

void destroy(mhs_ctx* c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void* p : c->allocations) cudaFree(p);
    c->allocations.clear();
    if (c->ns.host) cudaFreeHost(c->ns.host);
    if (c->flag_host) cudaFreeHost(c->flag_host);
    if (c->staging) cudaFree(c->staging);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
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
void vcycle(mhs_ctx* c, Hierarchy& H, int l) {
    cudaStream_t st = c->stream;
    LevelArrays<T>& A = arrays<T>(H, l);
    const Geom& g = H.g[l];
    const bool dbl = sizeof(T) == 8;
    const double s = sizeof(T), N = double(g.interior());
    // f vanishes on the finest FP64 interior level (the Dirichlet data sits in u)
    const double fs = (dbl && l == 0 && H.dim == 3 && c->f_zero_finest) ? 0.0 : s;
    const double upd_flops = H.dim == 3 ? 10.0 : 7.0;
    if (l == H.nlev() - 1) {
        TimedScope t(c->timer, dbl ? MHS_KT_COARSE64 : MHS_KT_COARSE32, 2.0 * g.n * s, 0.0, st);
        launch_coarse<T>(g, H.dim, A.coef, A.u, A.f, st);
        return;
    }
    for (int q = 0; q < c->opts.nu1; ++q) {
        TimedScope t(c->timer, dbl ? MHS_KT_SMOOTH64 : MHS_KT_SMOOTH32, N * (2 * s + fs), N * upd_flops, st);
        launch_smooth<T>(g, H.dim, A.coef, A.u, A.f, st);
    }
    {
        TimedScope t(c->timer, dbl ? MHS_KT_RESID64 : MHS_KT_RESID32, N * (2 * s + fs), N * (upd_flops + 1), st);
        launch_residual<T>(g, H.dim, A.coef, A.u, A.f, A.r, &c->ns, NORM_SCRATCH_SLOT, st);
    }
    LevelArrays<T>& C = arrays<T>(H, l + 1);
    const double Nc = double(H.g[l + 1].interior());
    {
        TimedScope t(c->timer, dbl ? MHS_KT_RESTRICT64 : MHS_KT_RESTRICT32, (N + Nc) * s,
                     Nc * (H.dim == 3 ? 54.0 : 18.0), st);
        launch_restrict<T>(g, H.g[l + 1], H.dim, A.r, C.f, st);
        MHS_CUDA(cudaMemsetAsync(C.u, 0, H.g[l + 1].n * sizeof(T), st));
    }
    vcycle<T>(c, H, l + 1);
    {
        TimedScope t(c->timer, dbl ? MHS_KT_PROLONG64 : MHS_KT_PROLONG32, (2 * N + Nc) * s, 4.0 * N, st);
        launch_prolong<T>(H.g[l + 1], g, H.dim, C.u, A.u, st);
    }
    for (int q = 0; q < c->opts.nu2; ++q) {
        TimedScope t(c->timer, dbl ? MHS_KT_SMOOTH64 : MHS_KT_SMOOTH32, N * (2 * s + fs), N * upd_flops, st);
        launch_smooth<T>(g, H.dim, A.coef, A.u, A.f, st);
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

// Solve A u = f on level 0 of H (u's boundary entries carry the Dirichlet
// data) to ||f - A u|| < tol * bnorm.  Returns cycles (or outer steps).
static int mg_solve(mhs_ctx* c, Hierarchy& H, int mode, double tol, double bnorm, double* rel_out,
                    double* conv_out) {
    cudaStream_t st = c->stream;
    const Geom& g = H.g[0];
    LevelArrays<double>& A = H.d[0];
    LevelArrays<float>& S = H.s[0];
    const double N = double(g.interior());
    const double fb = (H.dim == 3 && c->f_zero_finest) ? 0.0 : 8.0;
    const double fl = H.dim == 3 ? 11.0 : 8.0;
    auto residual_norm = [&]() {
        if (mode == MHS_MIXED) {
            TimedScope t(c->timer, MHS_KT_RESID_MIXED, N * (8.0 + fb + 4.0), N * fl, st);
            launch_residual_to_f32(g, H.dim, A.coef, A.u, A.f, S.f, &c->ns, NORM_RES_SLOT, st);
        } else {
            TimedScope t(c->timer, MHS_KT_RESID64, N * (16.0 + fb), N * fl, st);
            launch_residual<double>(g, H.dim, A.coef, A.u, A.f, A.r, &c->ns, NORM_RES_SLOT, st);
        }
        return std::sqrt(read_norm2(c, NORM_RES_SLOT));
    };
    double rn = residual_norm();
    if (!std::isfinite(rn)) throw Error(MHS_ERR_NONFINITE, "non-finite residual norm");
    double rel = bnorm > 0 ? rn / bnorm : 0.0;
    const double rel0 = rel;
    int cyc = 0;
    while (bnorm > 0 && rel >= tol && cyc < c->opts.max_cycles) {
        if (mode == MHS_MIXED) {
            MHS_CUDA(cudaMemsetAsync(S.u, 0, g.n * sizeof(float), st));
            for (int q = 0; q < c->opts.inner_cycles; ++q) vcycle<float>(c, H, 0);
            TimedScope t(c->timer, MHS_KT_CORRECT, N * 20.0, N, st);
            launch_add_correction(g, H.dim, S.u, A.u, st);
        } else {
            vcycle<double>(c, H, 0);
        }
        ++cyc;
        rn = residual_norm();
        if (!std::isfinite(rn)) throw Error(MHS_ERR_NONFINITE, "non-finite residual norm");
        rel = rn / bnorm;
    }
    if (rel_out) *rel_out = rel;
    if (conv_out) *conv_out = (cyc > 0 && rel0 > 0 && rel > 0) ? std::pow(rel / rel0, 1.0 / cyc) : 0.0;
    return (bnorm > 0 && rel >= tol) ? -cyc - 1 : cyc;
}

mhs_status solve(mhs_ctx* c, double tol, int mode, mhs_solve_info* info) {
    cudaStream_t st = c->stream;
    MHS_CUDA(cudaEventRecord(c->ev0, st));
    // step 2: lower boundary, eq. (lower_bound), from P = 0 (step 1)
    Hierarchy& H2 = c->h2;
    const Geom& g2 = H2.g[0];
    MHS_CUDA(cudaMemsetAsync(H2.d[0].u, 0, g2.n * sizeof(double), st));
    launch_lower_rhs(g2, c->bz, H2.d[0].f, st);
    // ||b|| of the 2D problem: residual of u = 0 is f
    launch_residual<double>(g2, 2, H2.d[0].coef, H2.d[0].u, H2.d[0].f, H2.d[0].r, &c->ns, NORM_B_SLOT, st);
    const double b2 = std::sqrt(read_norm2(c, NORM_B_SLOT));
    double rel2 = 0, rel3 = 0, conv = 0;
    int c2 = mg_solve(c, H2, mode, tol, b2, &rel2, nullptr);
    // step 3: interior, eq. (scalar_pot), with the plane k = 0 from step 2
    Hierarchy& H3 = c->h3;
    const Geom& g3 = H3.g[0];
    if (!(c->opts.flags & MHS_FLAG_WARM) || !c->have_solution)
        MHS_CUDA(cudaMemsetAsync(H3.d[0].u, 0, g3.n * sizeof(double), st));
    launch_copy_plane(g2, H2.d[0].u, g3, H3.d[0].u, st);
    launch_lift_norm(g3, H3.d[0].coef, H3.d[0].u, &c->ns, NORM_B_SLOT, st);
    const double b3 = std::sqrt(read_norm2(c, NORM_B_SLOT));
    int c3 = mg_solve(c, H3, mode, tol, b3, &rel3, &conv);
    MHS_CUDA(cudaEventRecord(c->ev1, st));
    MHS_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0;
    MHS_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    const bool ok = c2 >= 0 && c3 >= 0;
    if (c2 < 0) c2 = -c2 - 1;
    if (c3 < 0) c3 = -c3 - 1;
    if (info) {
        info->cycles_2d = c2;
        info->cycles_3d = c3;
        info->rel_res_2d = rel2;
        info->rel_res_3d = rel3;
        info->conv_factor = conv;
        info->ms = ms;
    }
    c->have_solution = true;
    if (!ok) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "no convergence to %g in %d cycles (2D rel %.3e, 3D rel %.3e)", tol,
                      c->opts.max_cycles, rel2, rel3);
        throw Error(MHS_ERR_NO_CONVERGENCE, buf);
    }
    return MHS_OK;
}

void ensure_field_buffers(mhs_ctx* c) {
    if (c->fld[0]) return;
    for (int q = 0; q < 5; ++q) c->fld[q] = static_cast<double*>(dev_alloc(c, c->h3.g[0].n * sizeof(double)));
}

void ensure_staging(mhs_ctx* c) {
    if (c->staging) return;
    MHS_CUDA(cudaMalloc(&c->staging, c->h3.g[0].n * sizeof(double)));
}

}  // namespace mhs

namespace mhs {

int KernelTimer::begin(int k, double b, double f, cudaStream_t st) {
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
        bytes.resize(used);
        flops.resize(used);
    }
    kind[rec] = k;
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
    }
    used = 0;
}

void KernelTimer::reset() {
    collect();
    for (int k = 0; k < MHS_KT_COUNT; ++k) ms[k] = alg_bytes[k] = alg_flops[k] = 0, count[k] = 0;
}

void KernelTimer::destroy() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    used = 0;
}

}  // namespace mhs
