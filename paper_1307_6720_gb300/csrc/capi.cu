// C ABI of libmhs (include/mhs.h): argument checks, status codes, copies
// between caller buffers (dense, host or device) and the pitched device
// hierarchy.  No C++ exception crosses this layer.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "group.h"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {
double fma_rate(int precision, cudaStream_t st);
mhs_status interior_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                                     const mhs_xi_params* xi, const double* P, double* out, cudaStream_t st);
}

namespace {

thread_local std::string g_last_error;

mhs_status fail(mhs_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

template <typename F>
mhs_status guarded(F&& f) {
    try {
        return f();
    } catch (const mhs::Error& e) {
        return fail(e.status, e.what());
    } catch (const std::bad_alloc&) {
        return fail(MHS_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(MHS_ERR_CUDA, e.what());
    } catch (...) {
        return fail(MHS_ERR_CUDA, "unknown internal error");
    }
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mhs_atmos_params default_atmos() { return mhs_atmos_params{1.0, 0.5, 150.0, 5.0, 10.0}; }

mhs_solver_opts default_opts() { return mhs_solver_opts{2, 2, 100, 1, 0, 1200, 4000, 12000000, 300000, 1, 8}; }

void fill_opts(mhs_solver_opts* o, const mhs_solver_opts* in) {
    *o = default_opts();
    if (!in) return;
    if (in->nu1 > 0) o->nu1 = in->nu1;
    if (in->nu2 > 0) o->nu2 = in->nu2;
    if (in->max_cycles > 0) o->max_cycles = in->max_cycles;
    if (in->inner_cycles > 0) o->inner_cycles = in->inner_cycles;
    if (in->cut64 > 0) o->cut64 = in->cut64;
    if (in->cut32 > 0) o->cut32 = in->cut32;
    if (in->fused_min > 0) o->fused_min = in->fused_min;
    if (in->sep_coarse != 0) o->sep_coarse = in->sep_coarse < 0 ? -1 : in->sep_coarse;
    if (in->tile > 0) o->tile = in->tile;
    if (in->tma_rows > 0) o->tma_rows = in->tma_rows;
    o->flags = in->flags;
}

// Argument checks shared by mhs_create and mhs_set_params.
mhs_status check_physics(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                         const mhs_xi_params& xi, const mhs_atmos_params& atm) {
    if (!std::isfinite(alpha)) return fail(MHS_ERR_INVALID_ARG, "alpha must be finite");
    if (xi.kind < MHS_XI_NONE || xi.kind > MHS_XI_EXP_SIN) return fail(MHS_ERR_INVALID_ARG, "unknown xi kind");
    if (!std::isfinite(xi.a) || !std::isfinite(xi.kappa) || !std::isfinite(xi.b) || !std::isfinite(xi.omega))
        return fail(MHS_ERR_INVALID_ARG, "xi parameters must be finite");
    if (!(atm.g > 0) || !(atm.mu0 > 0) || !(atm.T_cor > 0) || atm.T_cor == 1.0 || !(atm.z2 > atm.z1))
        return fail(MHS_ERR_INVALID_ARG, "atmosphere parameters: need g > 0, mu0 > 0, T_cor > 0 and != 1, z2 > z1");
    // eq. (scalar_pot) is elliptic for xi < 1 (Sect. 2.1): check every interior plane
    const double hz = Lz / (nz - 1);
    double min_om = 1.0;
    for (int k = 1; k < nz - 1; ++k) {
        const double om = 1.0 - mhs::xi_host(xi, k * hz);
        if (!(om > 0.0)) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "xi(z) = %.6g >= 1 at z = %.6g: eq. (scalar_pot) is not elliptic",
                          1.0 - om, k * hz);
            return fail(MHS_ERR_NOT_ELLIPTIC, buf);
        }
        if (om < min_om) min_om = om;
    }
    // -A must stay positive definite on every multigrid level: a sufficient
    // condition is alpha^2 below min(1 - xi) * lambda_xy + lambda_z, the
    // smallest eigenvalues of the discrete -(d_xx + d_yy) and -d_zz on the
    // coarsest level (three nodes per axis gives 2/h^2 per axis).
    auto lam = [](int n, double L) {
        const double h = L / (n - 1);
        const double s = std::sin(M_PI / (2.0 * (n - 1)));
        return 4.0 / (h * h) * s * s;
    };
    int cx = nx, cy = ny, cz = nz;
    auto can = [](int n) { return n >= 5 && (n - 1) % 2 == 0; };
    while (can(cx) && can(cy) && can(cz)) {
        cx = (cx - 1) / 2 + 1;
        cy = (cy - 1) / 2 + 1;
        cz = (cz - 1) / 2 + 1;
    }
    const double bound = min_om * (lam(cx, Lx) + lam(cy, Ly)) + lam(cz, Lz);
    if (!(alpha * alpha < bound)) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "alpha^2 = %.6g is not below the definiteness bound %.6g of the coarsest multigrid level",
                      alpha * alpha, bound);
        return fail(MHS_ERR_NOT_ELLIPTIC, buf);
    }
    return MHS_OK;
}

// dense [rows][nx] doubles <-> pitched device array (cudaMemcpyDefault: host or device)
void to_pitched(const mhs::Geom& g, double* dst, const double* src, size_t rows, cudaStream_t st) {
    MHS_CUDA(cudaMemcpy2DAsync(dst, g.px * sizeof(double), src, g.nx * sizeof(double), g.nx * sizeof(double), rows,
                               cudaMemcpyDefault, st));
}
void from_pitched(const mhs::Geom& g, double* dst, const double* src, size_t rows, cudaStream_t st) {
    MHS_CUDA(cudaMemcpy2DAsync(dst, g.nx * sizeof(double), src, g.px * sizeof(double), g.nx * sizeof(double), rows,
                               cudaMemcpyDefault, st));
}
// the same for a result array of the handle, by the packing kernel: into
// device memory directly (a 2D copy of the short pitched rows measured three
// times the time of a plain copy of the array), into host memory through the
// staging buffer, so the transfer is one contiguous copy instead of one short
// row per DMA step
void copy_out(mhs_handle h, const mhs::Geom& g, double* dst, const double* src, size_t rows) {
    if (is_device_ptr(dst)) {
        mhs::launch_pack(src, dst, g.nx, g.px, rows, h->stream);
        return;
    }
    mhs::ensure_staging(h);
    mhs::launch_pack(src, h->staging, g.nx, g.px, rows, h->stream);
    MHS_CUDA(cudaMemcpyAsync(dst, h->staging, size_t(g.nx) * rows * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
}
}  // namespace

extern "C" {

const char* mhs_version(void) { return "mhs-gb300 0.1"; }

long long mhs_kernel_launches(void) { return mhs::launches(); }

mhs_status mhs_probe_fma_rate(int precision, void* stream, double* flops_per_s) {
    if (!flops_per_s || (precision != MHS_FP64 && precision != MHS_MIXED))
        return fail(MHS_ERR_INVALID_ARG, "precision must be MHS_FP64 or MHS_MIXED (FP32) and the result non-NULL");
    return guarded([&] {
        *flops_per_s = mhs::fma_rate(precision, static_cast<cudaStream_t>(stream));
        return MHS_OK;
    });
}

const char* mhs_last_error(void) { return g_last_error.c_str(); }

const char* mhs_status_string(mhs_status s) {
    switch (s) {
    case MHS_OK: return "MHS_OK";
    case MHS_ERR_INVALID_ARG: return "MHS_ERR_INVALID_ARG";
    case MHS_ERR_NOT_ELLIPTIC: return "MHS_ERR_NOT_ELLIPTIC";
    case MHS_ERR_OUT_OF_MEMORY: return "MHS_ERR_OUT_OF_MEMORY";
    case MHS_ERR_CUDA: return "MHS_ERR_CUDA";
    case MHS_ERR_NO_CONVERGENCE: return "MHS_ERR_NO_CONVERGENCE";
    case MHS_ERR_NONFINITE: return "MHS_ERR_NONFINITE";
    case MHS_ERR_BAD_STATE: return "MHS_ERR_BAD_STATE";
    case MHS_ERR_TIMEOUT: return "MHS_ERR_TIMEOUT";
    case MHS_ERR_REJECTED: return "MHS_ERR_REJECTED";
    }
    return "MHS_ERR_UNKNOWN";
}

mhs_status mhs_create(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                      const mhs_xi_params* xi, const mhs_atmos_params* atm, mhs_handle* out) {
    if (!out) return fail(MHS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    for (int n : {nx, ny, nz})
        if (n < 5 || n % 2 == 0 || n > 16385)
            return fail(MHS_ERR_INVALID_ARG, "node counts must be odd and in [5, 16385], got " + std::to_string(n));
    if (nx > 4097 || ny > 4097) return fail(MHS_ERR_INVALID_ARG, "nx and ny must not exceed 4097");
    if (!(Lx > 0) || !(Ly > 0) || !(Lz > 0) || !std::isfinite(Lx) || !std::isfinite(Ly) || !std::isfinite(Lz))
        return fail(MHS_ERR_INVALID_ARG, "domain lengths must be finite and > 0");
    const mhs_xi_params x = xi ? *xi : mhs_xi_params{MHS_XI_NONE, 0, 0, 0, 0};
    const mhs_atmos_params a = atm ? *atm : default_atmos();
    const mhs_status s = check_physics(nx, ny, nz, Lx, Ly, Lz, alpha, x, a);
    if (s != MHS_OK) return s;
    mhs_ctx* c = new (std::nothrow) mhs_ctx();
    if (!c) return fail(MHS_ERR_OUT_OF_MEMORY, "host allocation failed");
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->Lx = Lx; c->Ly = Ly; c->Lz = Lz;
    c->alpha = alpha;
    c->xi = x;
    c->atm = a;
    c->opts = default_opts();
    const mhs_status r = guarded([&] {
        mhs::create(c);
        return MHS_OK;
    });
    if (r != MHS_OK) {
        mhs::destroy(c);
        delete c;
        return r;
    }
    *out = c;
    return MHS_OK;
}

void mhs_destroy(mhs_handle h) {
    if (!h) return;
    mhs::destroy(h);
    delete h;
}

mhs_status mhs_set_stream(mhs_handle h, void* stream) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    h->stream = static_cast<cudaStream_t>(stream);
    return MHS_OK;
}

mhs_status mhs_set_options(mhs_handle h, const mhs_solver_opts* opts) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (opts && (opts->nu1 < 0 || opts->nu2 < 0 || opts->max_cycles < 0 || opts->inner_cycles < 0 ||
                 opts->nu1 > 16 || opts->nu2 > 16 || opts->inner_cycles > 16 ||
                 (opts->tma_rows != 0 && opts->tma_rows != 8 && opts->tma_rows != 16)))
        return fail(MHS_ERR_INVALID_ARG, "options out of range");
    fill_opts(&h->opts, opts);
    return guarded([&] {
        mhs::choose_cuts(h);   // captured solves are cached per option set
        return MHS_OK;
    });
}

mhs_status mhs_set_params(mhs_handle h, double alpha, const mhs_xi_params* xi, const mhs_atmos_params* atm) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    const mhs_xi_params x = xi ? *xi : mhs_xi_params{MHS_XI_NONE, 0, 0, 0, 0};
    const mhs_atmos_params a = atm ? *atm : default_atmos();
    const mhs_status s = check_physics(h->nx, h->ny, h->nz, h->Lx, h->Ly, h->Lz, alpha, x, a);
    if (s != MHS_OK) return s;
    return guarded([&] {
        h->alpha = alpha;
        h->xi = x;
        h->atm = a;
        mhs::compute_coefficients(h);
        h->have_solution = false;
        return MHS_OK;
    });
}

mhs_status mhs_set_lower_bz(mhs_handle h, const double* bz) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!bz) return fail(MHS_ERR_INVALID_ARG, "bz is NULL");
    return guarded([&] {
        const mhs::Geom& g = h->h2.g[0];
        to_pitched(g, h->bz, bz, g.ny, h->stream);
        MHS_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
        mhs::launch_count_nonfinite(g, h->bz, h->flag, h->stream);
        MHS_CUDA(cudaMemcpyAsync(h->flag_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        MHS_CUDA(cudaStreamSynchronize(h->stream));
        if (h->flag_host[0]) {
            h->have_bz = false;
            return fail(MHS_ERR_NONFINITE, "B_z holds a non-finite value at an interior node");
        }
        h->have_bz = true;
        h->have_solution = false;
        return MHS_OK;
    });
}

mhs_status mhs_solve(mhs_handle h, double tol, int mode, mhs_solve_info* info) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!(tol > 0.0 && tol < 1.0)) return fail(MHS_ERR_INVALID_ARG, "tol must be in (0, 1)");
    if (mode != MHS_FP64 && mode != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision mode");
    if (!h->have_bz) return fail(MHS_ERR_BAD_STATE, "mhs_set_lower_bz must come before mhs_solve");
    return guarded([&] { return mhs::solve(h, tol, mode, info); });
}

mhs_status mhs_batch_solve(mhs_handle* hs, int n, double tol, int mode, mhs_solve_info* infos,
                           mhs_status* statuses) {
    if (!hs || n < 0) return fail(MHS_ERR_INVALID_ARG, "bad handle array");
    if (!(tol > 0.0 && tol < 1.0)) return fail(MHS_ERR_INVALID_ARG, "tol must be in (0, 1)");
    if (mode != MHS_FP64 && mode != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision mode");
    for (int q = 0; q < n; ++q) {
        if (!hs[q]) return fail(MHS_ERR_INVALID_ARG, "NULL handle in batch");
        if (!hs[q]->have_bz) return fail(MHS_ERR_BAD_STATE, "every handle needs mhs_set_lower_bz before a batch");
        for (int r = 0; r < q; ++r)
            if (hs[r] == hs[q]) return fail(MHS_ERR_INVALID_ARG, "a handle appears twice in the batch");
    }
    return guarded([&] { return mhs::batch_solve(hs, n, tol, mode, infos, statuses); });
}

mhs_status mhs_group_create(mhs_handle* hs, int n, int mode, size_t part_bytes, int nstreams, mhs_group_t* out) {
    if (!out) return fail(MHS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!hs || n < 1) return fail(MHS_ERR_INVALID_ARG, "group: need at least one handle");
    if (nstreams < 0 || nstreams > 64) return fail(MHS_ERR_INVALID_ARG, "group: nstreams must be in [0, 64]");
    if (mode != MHS_FP64 && mode != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision mode");
    for (int q = 0; q < n; ++q) {
        if (!hs[q]) return fail(MHS_ERR_INVALID_ARG, "NULL handle in group");
        for (int r = 0; r < q; ++r)
            if (hs[r] == hs[q]) return fail(MHS_ERR_INVALID_ARG, "a handle appears twice in the group");
    }
    return guarded([&] {
        *out = mhs::group_create(hs, n, mode, part_bytes, nstreams);
        return MHS_OK;
    });
}

mhs_status mhs_group_solve(mhs_group_t g, double tol, mhs_solve_info* infos, mhs_status* statuses) {
    if (!g) return fail(MHS_ERR_INVALID_ARG, "group is NULL");
    if (!(tol > 0.0 && tol < 1.0)) return fail(MHS_ERR_INVALID_ARG, "tol must be in (0, 1)");
    for (const mhs::GPart* p : g->parts)
        for (const mhs_ctx* c : p->hs)
            if (!c->have_bz) return fail(MHS_ERR_BAD_STATE, "every group member needs mhs_set_lower_bz before a solve");
    return guarded([&] {
        const mhs_status s = mhs::group_solve(g, tol, infos, statuses);
        if (s != MHS_OK) return fail(s, s == MHS_ERR_NO_CONVERGENCE ? "an instance did not converge"
                                                                    : "an instance has a non-finite residual");
        return MHS_OK;
    });
}

void mhs_group_destroy(mhs_group_t g) { mhs::group_destroy(g); }

mhs_status mhs_group_set_eager(mhs_group_t g, int eager) {
    if (!g) return fail(MHS_ERR_INVALID_ARG, "group is NULL");
    mhs::group_set_eager(g, eager != 0);
    return MHS_OK;
}

mhs_status mhs_autotune(mhs_handle h, double tol, int mode, int repeats, mhs_tune_result* out) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!(tol > 0.0 && tol < 1.0)) return fail(MHS_ERR_INVALID_ARG, "tol must be in (0, 1)");
    if (mode != MHS_FP64 && mode != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision mode");
    if (repeats < 1 || repeats > 20) return fail(MHS_ERR_INVALID_ARG, "repeats must be in [1, 20]");
    if (!h->have_bz) return fail(MHS_ERR_BAD_STATE, "mhs_set_lower_bz must come before mhs_autotune");
    return guarded([&] {
        mhs::autotune(h, tol, mode, repeats, out);
        return MHS_OK;
    });
}

mhs_status mhs_tune_lookup(mhs_handle h, int mode, mhs_solver_opts* opts, int* found) {
    if (!h || !opts || !found) return fail(MHS_ERR_INVALID_ARG, "NULL argument");
    if (mode != MHS_FP64 && mode != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision mode");
    *found = mhs::tune_lookup(h, mode, opts) ? 1 : 0;
    return MHS_OK;
}

void mhs_tune_clear(void) { mhs::tune_clear(); }

mhs_status mhs_get_phi(mhs_handle h, double* phi) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!phi) return fail(MHS_ERR_INVALID_ARG, "phi is NULL");
    if (!h->have_solution) return fail(MHS_ERR_BAD_STATE, "no solution yet (call mhs_solve)");
    return guarded([&] {
        const mhs::Geom& g = h->h3.g[0];
        copy_out(h, g, phi, h->h3.d[0].u, size_t(g.ny) * g.nz);
        if (!is_device_ptr(phi)) MHS_CUDA(cudaStreamSynchronize(h->stream));
        return MHS_OK;
    });
}

mhs_status mhs_fields(mhs_handle h, double* Bx, double* By, double* Bz, double* p, double* rho) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!h->have_solution) return fail(MHS_ERR_BAD_STATE, "no solution yet (call mhs_solve)");
    return guarded([&] {
        mhs::ensure_field_buffers(h);
        const mhs::Geom& g = h->h3.g[0];
        {
            const double nodes = double(g.nx) * g.ny * g.nz;
            mhs::TimedScope t(h->timer, MHS_KT_FIELDS, 48.0 * nodes, 60.0 * nodes, h->stream);
            mhs::launch_fields(g, h->alpha, h->atm, h->prof, h->h3.d[0].u, h->fld[0], h->fld[1], h->fld[2],
                               h->fld[3], h->fld[4], (h->opts.flags & MHS_FLAG_BZ_MIMETIC) ? 1 : 0, h->stream);
        }
        double* outs[5] = {Bx, By, Bz, p, rho};
        bool host = false;
        for (int q = 0; q < 5; ++q) {
            if (!outs[q]) continue;
            copy_out(h, g, outs[q], h->fld[q], size_t(g.ny) * g.nz);
            host = host || !is_device_ptr(outs[q]);
        }
        if (host) MHS_CUDA(cudaStreamSynchronize(h->stream));
        return MHS_OK;
    });
}

// B of the latest solve into h->fld (the field recovery of mhs_fields)
static void compute_fields(mhs_handle h) {
    mhs::ensure_field_buffers(h);
    const mhs::Geom& g = h->h3.g[0];
    const double nodes = double(g.nx) * g.ny * g.nz;
    mhs::TimedScope t(h->timer, MHS_KT_FIELDS, 48.0 * nodes, 60.0 * nodes, h->stream);
    mhs::launch_fields(g, h->alpha, h->atm, h->prof, h->h3.d[0].u, h->fld[0], h->fld[1], h->fld[2], h->fld[3],
                       h->fld[4], (h->opts.flags & MHS_FLAG_BZ_MIMETIC) ? 1 : 0, h->stream);
}

mhs_status mhs_current(mhs_handle h, double* jx, double* jy, double* jz, double* jmag, double* bmag) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!h->have_solution) return fail(MHS_ERR_BAD_STATE, "no solution yet (call mhs_solve)");
    return guarded([&] {
        compute_fields(h);
        mhs::ensure_post_buffers(h);
        const mhs::Geom& g = h->h3.g[0];
        mhs::launch_current(g, h->atm.mu0, h->fld[0], h->fld[1], h->fld[2], h->post[0], h->post[1], h->post[2],
                            h->post[3], h->post[4], h->stream);
        double* outs[5] = {jx, jy, jz, jmag, bmag};
        bool host = false;
        for (int q = 0; q < 5; ++q) {
            if (!outs[q]) continue;
            copy_out(h, g, outs[q], h->post[q], size_t(g.ny) * g.nz);
            host = host || !is_device_ptr(outs[q]);
        }
        if (host) MHS_CUDA(cudaStreamSynchronize(h->stream));
        return MHS_OK;
    });
}

// Field lines on B arrays with strides (px, plane); seeds, points and lengths
// may be host or device memory (host ones are staged through the device).
static void trace_any(int nx, int ny, int nz, double Lx, double Ly, double Lz, size_t px, size_t plane,
                      const double* Bx, const double* By, const double* Bz, const double* seeds, int n, double ds,
                      int max_steps, int direction, double* points, int* lengths, cudaStream_t st) {
    const size_t seed_bytes = size_t(n) * 3 * sizeof(double);
    const size_t pts_bytes = size_t(n) * size_t(max_steps + 1) * 3 * sizeof(double);
    const size_t len_bytes = size_t(n) * sizeof(int);
    const bool ds_dev = is_device_ptr(seeds), dp_dev = is_device_ptr(points), dl_dev = is_device_ptr(lengths);
    double* d_seeds = const_cast<double*>(seeds);
    double* d_pts = points;
    int* d_len = lengths;
    if (!ds_dev) MHS_CUDA(cudaMalloc(&d_seeds, seed_bytes));
    if (!dp_dev) MHS_CUDA(cudaMalloc(&d_pts, pts_bytes));
    if (!dl_dev) MHS_CUDA(cudaMalloc(&d_len, len_bytes));
    try {
        if (!ds_dev) MHS_CUDA(cudaMemcpyAsync(d_seeds, seeds, seed_bytes, cudaMemcpyHostToDevice, st));
        mhs::launch_trace(nx, ny, nz, Lx, Ly, Lz, px, plane, Bx, By, Bz, d_seeds, n, ds, max_steps,
                          direction > 0 ? 1.0 : -1.0, d_pts, d_len, st);
        if (!dp_dev) MHS_CUDA(cudaMemcpyAsync(points, d_pts, pts_bytes, cudaMemcpyDeviceToHost, st));
        if (!dl_dev) MHS_CUDA(cudaMemcpyAsync(lengths, d_len, len_bytes, cudaMemcpyDeviceToHost, st));
        if (!ds_dev || !dp_dev || !dl_dev) MHS_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamSynchronize(st);
        if (!ds_dev) cudaFree(d_seeds);
        if (!dp_dev) cudaFree(d_pts);
        if (!dl_dev) cudaFree(d_len);
        throw;
    }
    if (!ds_dev) cudaFree(d_seeds);
    if (!dp_dev) cudaFree(d_pts);
    if (!dl_dev) cudaFree(d_len);
}

static mhs_status check_trace_args(const double* seeds, int n, double ds, int max_steps, int direction,
                                   const double* points, const int* lengths) {
    if (n < 0 || max_steps < 0 || !(ds > 0.0) || !std::isfinite(ds) || (direction != 1 && direction != -1))
        return fail(MHS_ERR_INVALID_ARG, "trace: need n >= 0, max_steps >= 0, ds > 0, direction +1 or -1");
    if (n > 0 && (!seeds || !points || !lengths)) return fail(MHS_ERR_INVALID_ARG, "trace: NULL buffer");
    if (double(n) * double(max_steps + 1) * 24.0 > 64e9)
        return fail(MHS_ERR_INVALID_ARG, "trace: output larger than 64 GB");
    return MHS_OK;
}

mhs_status mhs_trace(mhs_handle h, const double* seeds, int n, double ds, int max_steps, int direction,
                     double* points, int* lengths) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    if (!h->have_solution) return fail(MHS_ERR_BAD_STATE, "no solution yet (call mhs_solve)");
    const mhs_status s = check_trace_args(seeds, n, ds, max_steps, direction, points, lengths);
    if (s != MHS_OK) return s;
    return guarded([&] {
        compute_fields(h);
        const mhs::Geom& g = h->h3.g[0];
        trace_any(g.nx, g.ny, g.nz, h->Lx, h->Ly, h->Lz, size_t(g.px), g.plane, h->fld[0], h->fld[1], h->fld[2],
                  seeds, n, ds, max_steps, direction, points, lengths, h->stream);
        return MHS_OK;
    });
}

mhs_status mhs_trace_field(int nx, int ny, int nz, double Lx, double Ly, double Lz, const double* Bx,
                           const double* By, const double* Bz, const double* seeds, int n, double ds, int max_steps,
                           int direction, double* points, int* lengths, void* stream) {
    if (nx < 2 || ny < 2 || nz < 2 || !(Lx > 0) || !(Ly > 0) || !(Lz > 0))
        return fail(MHS_ERR_INVALID_ARG, "trace: need at least 2 nodes and a positive length per axis");
    if (!Bx || !By || !Bz || !is_device_ptr(Bx) || !is_device_ptr(By) || !is_device_ptr(Bz))
        return fail(MHS_ERR_INVALID_ARG, "trace: Bx, By, Bz must be device arrays");
    const mhs_status s = check_trace_args(seeds, n, ds, max_steps, direction, points, lengths);
    if (s != MHS_OK) return s;
    return guarded([&] {
        trace_any(nx, ny, nz, Lx, Ly, Lz, size_t(nx), size_t(nx) * ny, Bx, By, Bz, seeds, n, ds, max_steps,
                  direction, points, lengths, static_cast<cudaStream_t>(stream));
        return MHS_OK;
    });
}

mhs_status mhs_num_levels(mhs_handle h, int dim, int* nlevels) {
    if (!h || !nlevels || (dim != 2 && dim != 3)) return fail(MHS_ERR_INVALID_ARG, "bad argument");
    *nlevels = (dim == 3 ? h->h3 : h->h2).nlev();
    return MHS_OK;
}

mhs_status mhs_level_shape(mhs_handle h, int dim, int level, int* nx, int* ny, int* nz) {
    if (!h || (dim != 2 && dim != 3)) return fail(MHS_ERR_INVALID_ARG, "bad argument");
    const mhs::Hierarchy& H = dim == 3 ? h->h3 : h->h2;
    if (level < 0 || level >= H.nlev()) return fail(MHS_ERR_INVALID_ARG, "level out of range");
    if (nx) *nx = H.g[level].nx;
    if (ny) *ny = H.g[level].ny;
    if (nz) *nz = H.g[level].nz;
    return MHS_OK;
}

static mhs_status level_check(mhs_handle h, int dim, int level, int field, int prec) {
    if (!h || (dim != 2 && dim != 3)) return fail(MHS_ERR_INVALID_ARG, "bad handle or dim");
    const mhs::Hierarchy& H = dim == 3 ? h->h3 : h->h2;
    if (level < 0 || level >= H.nlev()) return fail(MHS_ERR_INVALID_ARG, "level out of range");
    if (field < MHS_FIELD_U || field > MHS_FIELD_R) return fail(MHS_ERR_INVALID_ARG, "unknown field");
    if (prec != MHS_FP64 && prec != MHS_MIXED) return fail(MHS_ERR_INVALID_ARG, "unknown precision");
    return MHS_OK;
}

mhs_status mhs_level_write(mhs_handle h, int dim, int level, int field, int prec, const double* src) {
    mhs_status s = level_check(h, dim, level, field, prec);
    if (s != MHS_OK) return s;
    if (!src) return fail(MHS_ERR_INVALID_ARG, "src is NULL");
    return guarded([&] {
        mhs::Hierarchy& H = dim == 3 ? h->h3 : h->h2;
        const mhs::Geom& g = H.g[level];
        const size_t rows = size_t(g.ny) * g.nz;
        if (dim == 3 && level == 0 && field == MHS_FIELD_F) h->f_zero_finest = false;
        if (prec == MHS_FP64) {
            double* d = field == MHS_FIELD_U ? H.d[level].u : field == MHS_FIELD_F ? H.d[level].f : H.d[level].r;
            to_pitched(g, d, src, rows, h->stream);
            if (field == MHS_FIELD_U)   // the sweep twin carries the same (Dirichlet) boundary values
                MHS_CUDA(cudaMemcpyAsync(H.d[level].t, d, g.n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        } else {
            float* d = field == MHS_FIELD_U ? H.s[level].u : field == MHS_FIELD_F ? H.s[level].f : H.s[level].r;
            mhs::ensure_staging(h);
            MHS_CUDA(cudaMemsetAsync(h->staging, 0, g.n * sizeof(double), h->stream));
            to_pitched(g, h->staging, src, rows, h->stream);
            mhs::launch_d2f(h->staging, d, g.n, h->stream);
            if (field == MHS_FIELD_U)
                MHS_CUDA(cudaMemcpyAsync(H.s[level].t, d, g.n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
        }
        MHS_CUDA(cudaStreamSynchronize(h->stream));
        return MHS_OK;
    });
}

mhs_status mhs_level_read(mhs_handle h, int dim, int level, int field, int prec, double* dst) {
    mhs_status s = level_check(h, dim, level, field, prec);
    if (s != MHS_OK) return s;
    if (!dst) return fail(MHS_ERR_INVALID_ARG, "dst is NULL");
    return guarded([&] {
        mhs::Hierarchy& H = dim == 3 ? h->h3 : h->h2;
        const mhs::Geom& g = H.g[level];
        const size_t rows = size_t(g.ny) * g.nz;
        if (prec == MHS_FP64) {
            const double* d = field == MHS_FIELD_U ? H.d[level].u : field == MHS_FIELD_F ? H.d[level].f : H.d[level].r;
            from_pitched(g, dst, d, rows, h->stream);
        } else {
            const float* d = field == MHS_FIELD_U ? H.s[level].u : field == MHS_FIELD_F ? H.s[level].f : H.s[level].r;
            mhs::ensure_staging(h);
            mhs::launch_f2d(d, h->staging, g.n, h->stream);
            from_pitched(g, dst, h->staging, rows, h->stream);
        }
        MHS_CUDA(cudaStreamSynchronize(h->stream));
        return MHS_OK;
    });
}

mhs_status mhs_level_op(mhs_handle h, int dim, int level, int op, int prec) {
    mhs_status s = level_check(h, dim, level, MHS_FIELD_U, prec);
    if (s != MHS_OK) return s;
    mhs::Hierarchy& H = dim == 3 ? h->h3 : h->h2;
    if ((op == MHS_OP_RESTRICT || op == MHS_OP_PROLONG || op == MHS_OP_RESID_RESTRICT || op == MHS_OP_RESTRICT_RED) &&
        level >= H.nlev() - 1)
        return fail(MHS_ERR_INVALID_ARG, "no coarser level");
    if (op < MHS_OP_SMOOTH || op > MHS_OP_RESTRICT_RED) return fail(MHS_ERR_INVALID_ARG, "unknown op");
    if (op == MHS_OP_EXACT && !mhs::sep_level_ok(H.g[level]))
        return fail(MHS_ERR_INVALID_ARG, "exact solve needs nx - 1 and ny - 1 powers of two, or nx, ny <= 66");
    return guarded([&] {
        const mhs::Geom& g = H.g[level];
        cudaStream_t st = h->stream;
        auto run = [&](auto& A, auto& C, auto tag) {
            using T = decltype(tag);
            switch (op) {
            case MHS_OP_SMOOTH: mhs::smooth_hook<T>(h, H, level); break;
            case MHS_OP_RESIDUAL:
                mhs::launch_residual<T>(g, dim, A.coef, A.u, A.f, A.r, nullptr, 0, st);
                break;
            case MHS_OP_RESTRICT: mhs::launch_restrict<T>(g, H.g[level + 1], dim, A.r, C.f, (T*)nullptr, st); break;
            case MHS_OP_RESTRICT_RED:
                mhs::launch_restrict<T>(g, H.g[level + 1], dim, A.r, C.f, (T*)nullptr, st, true);
                break;
            case MHS_OP_PROLONG: mhs::launch_prolong<T>(H.g[level + 1], g, dim, C.u, A.u, st); break;
            case MHS_OP_COARSE:
                if (2 * g.n * sizeof(T) > 200 * 1024) throw mhs::Error(MHS_ERR_INVALID_ARG, "level too large for the one-CTA solve");
                MHS_CUDA(cudaMemsetAsync(A.u, 0, g.n * sizeof(T), st));
                mhs::launch_coarse<T>(g, dim, A.coef, A.u, A.f, st);
                break;
            case MHS_OP_VCYCLE: mhs::vcycle<T>(h, H, level); break;
            case MHS_OP_EXACT:
                mhs::sep_tables<T>(h, H, level);
                mhs::sep_exact<T>(h, H, level);
                break;
            case MHS_OP_RESID_RESTRICT:
                mhs::launch_resid_restrict<T>(g, H.g[level + 1], dim, A.coef, A.u, A.f, C.f, C.u, st);
                break;
            }
        };
        const int lc = level + 1 < H.nlev() ? level + 1 : level;
        if (prec == MHS_FP64) run(H.d[level], H.d[lc], double(0));
        else run(H.s[level], H.s[lc], float(0));
        MHS_CUDA(cudaStreamSynchronize(st));
        return MHS_OK;
    });
}

mhs_status mhs_set_kernel_timing(mhs_handle h, int enable) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    return guarded([&] {
        h->timer.collect();
        h->timer.enabled = enable != 0;
        return MHS_OK;
    });
}

mhs_status mhs_kernel_timing(mhs_handle h, int kind, double* total_ms, long long* launches, double* alg_bytes,
                             double* alg_flops) {
    if (!h || kind < 0 || kind >= MHS_KT_COUNT) return fail(MHS_ERR_INVALID_ARG, "bad handle or kind");
    return guarded([&] {
        h->timer.collect();
        if (total_ms) *total_ms = h->timer.ms[kind];
        if (launches) *launches = h->timer.count[kind];
        if (alg_bytes) *alg_bytes = h->timer.alg_bytes[kind];
        if (alg_flops) *alg_flops = h->timer.alg_flops[kind];
        return MHS_OK;
    });
}

mhs_status mhs_kernel_timing_finest(mhs_handle h, int kind, double* total_ms, long long* launches, double* alg_bytes,
                                    double* alg_flops) {
    if (!h || kind < 0 || kind >= MHS_KT_COUNT) return fail(MHS_ERR_INVALID_ARG, "bad handle or kind");
    return guarded([&] {
        h->timer.collect();
        if (total_ms) *total_ms = h->timer.ms0[kind];
        if (launches) *launches = h->timer.count0[kind];
        if (alg_bytes) *alg_bytes = h->timer.alg_bytes0[kind];
        if (alg_flops) *alg_flops = h->timer.alg_flops0[kind];
        return MHS_OK;
    });
}

mhs_status mhs_kernel_timing_reset(mhs_handle h) {
    if (!h) return fail(MHS_ERR_INVALID_ARG, "handle is NULL");
    return guarded([&] {
        h->timer.reset();
        return MHS_OK;
    });
}

const char* mhs_kernel_kind_name(int kind) {
    static const char* names[MHS_KT_COUNT] = {"smooth64", "smooth32", "residual64", "residual32", "restrict64",
                                              "restrict32", "prolong64", "prolong32", "coarse64", "coarse32",
                                              "residual_mixed", "correct", "fields", "other",
                                              "separable"};
    return (kind >= 0 && kind < MHS_KT_COUNT) ? names[kind] : "unknown";
}

mhs_status mhs_interior_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                                         const mhs_xi_params* xi, const double* P, double* out, void* stream) {
    return guarded([&] {
        return mhs::interior_residual_noalloc(nx, ny, nz, Lx, Ly, Lz, alpha, xi, P, out,
                                              static_cast<cudaStream_t>(stream));
    });
}

}  // extern "C"
