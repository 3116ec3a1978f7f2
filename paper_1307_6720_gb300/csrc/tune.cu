// Autotuner: picks a handle's solver options by timing whole solves.
//
// The cost of an option set is the device time of a complete solve of the
// handle's own problem (resident B_z, its grid, alpha and xi) to the caller's
// tolerance through the captured-graph path, so that a cheaper smoother
// that needs more cycles, or a cut-off that moves work into the one-CTA
// sub-cycle, is judged by what it costs end to end.  The search is
// coordinate descent from the handle's current options over
//   - the smoother: red-black point Gauss-Seidel or zebra z-line (MHS_FLAG_POINT,
//     MHS_FLAG_ZLINE),
//   - the sweep counts (nu1, nu2),
//   - the sub-cycle cut-off (cut64 in FP64 mode, cut32 in mixed mode), one
//     candidate per level that the sub-cycle could start from,
//   - the fused TMA sweep threshold on FP32 levels (mixed mode, point smoother)
//     and the height of its tiles (tma_rows),
//   - the full-multigrid first cycle (MHS_FLAG_NO_FMG),
//   - the thread-block shape of the red-black point passes (tile),
// at most two rounds, a change kept only when it saves at least 3 %.  The
// winner is stored in a process-wide table keyed by the problem class
// (grid, mode, anisotropy class), so that other handles of the class, such
// as the instances of a batch or the hierarchies of a server, take it
// without tuning.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mg_bodies.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

struct TuneKey {
    int nx, ny, nz, mode, aniso;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nz, mode, aniso) < std::tie(o.nx, o.ny, o.nz, o.mode, o.aniso);
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, mhs_solver_opts> g_tune_table;

TuneKey key_of(const mhs_ctx* c, int mode) { return TuneKey{c->nx, c->ny, c->nz, mode, aniso_class(c)}; }

bool same_opts(const mhs_solver_opts& a, const mhs_solver_opts& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

void apply_opts(mhs_ctx* c, const mhs_solver_opts& o) {
    c->opts = o;
    choose_cuts(c);
}

// fastest of `repeats` timed solves after one untimed solve (graph capture);
// +inf when a solve of the candidate does not reach the tolerance (no
// convergence within max_cycles, or a non-finite residual): the candidate
// loses, the search goes on.  Other errors propagate.
double time_opts(mhs_ctx* c, const mhs_solver_opts& o, double tol, int mode, int repeats) {
    apply_opts(c, o);
    mhs_solve_info info{};
    try {
        solve(c, tol, mode, &info);
        double best = INFINITY;
        for (int r = 0; r < repeats; ++r) {
            solve(c, tol, mode, &info);
            best = std::min(best, info.ms);
        }
        return best;
    } catch (const Error& e) {
        if (e.status == MHS_ERR_NO_CONVERGENCE || e.status == MHS_ERR_NONFINITE) return INFINITY;
        throw;
    }
}

int clamp_int(size_t v) { return v > size_t(INT_MAX) ? INT_MAX : int(v); }

}  // namespace

int aniso_class(const mhs_ctx* c) {
    const double hx = c->Lx / (c->nx - 1), hy = c->Ly / (c->ny - 1), hz = c->Lz / (c->nz - 1);
    const double hmax = std::max(hx, hy);
    double rho = 1.0;
    for (int k = 1; k < c->nz - 1; ++k) {
        const double om = 1.0 - xi_host(c->xi, k * hz);
        if (om > 0.0) rho = std::max(rho, hmax * hmax / (om * hz * hz));
    }
    return std::max(0, int(std::floor(std::log2(rho))));
}

void autotune(mhs_ctx* c, double tol, int mode, int repeats, mhs_tune_result* out) {
    const mhs_solver_opts start = c->opts;
    int ncand = 0;
    mhs_solver_opts best = start;
    double best_ms = time_opts(c, start, tol, mode, repeats);
    ++ncand;
    const double start_ms = best_ms;
    auto consider = [&](const mhs_solver_opts& o) {
        if (same_opts(o, best)) return;
        const double t = time_opts(c, o, tol, mode, repeats);
        ++ncand;
        if (t < 0.97 * best_ms) {
            best = o;
            best_ms = t;
        }
    };
    // sub-cycle cut-off candidates: the interior node count of every level
    // below the finest (the sub-cycle starts at the first level at or under
    // the cut-off that fits shared memory) and 1 (the coarsest level only)
    std::vector<int> cuts{1};
    for (int l = 1; l < c->h3.nlev(); ++l) cuts.push_back(clamp_int(c->h3.g[l].interior()));
    // coarse-grid solve by the separable solver on any level that allows it, or nowhere
    std::vector<int> exacts{-1};
    for (int l = 1; l < c->h3.nlev(); ++l)
        if (sep_level_ok(c->h3.g[l])) exacts.push_back(clamp_int(c->h3.g[l].interior()));
    const int pairs[][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 3}};
    for (int round = 0; round < 2; ++round) {
        const mhs_solver_opts before = best;
        for (int sm : {MHS_FLAG_POINT, MHS_FLAG_ZLINE}) {
            mhs_solver_opts o = best;
            o.flags = (o.flags & ~(MHS_FLAG_POINT | MHS_FLAG_ZLINE)) | sm;
            consider(o);
        }
        for (const auto& p : pairs) {
            mhs_solver_opts o = best;
            o.nu1 = p[0];
            o.nu2 = p[1];
            consider(o);
        }
        for (int ex : exacts) {
            mhs_solver_opts o = best;
            o.sep_coarse = ex;
            consider(o);
        }
        for (int cut : cuts) {
            mhs_solver_opts o = best;
            (mode == MHS_FP64 ? o.cut64 : o.cut32) = cut;
            consider(o);
        }
        const bool line = (best.flags & MHS_FLAG_ZLINE) || (!(best.flags & MHS_FLAG_POINT) && c->aniso >= 5);
        if (mode == MHS_MIXED && !line && c->h3.nlev() > 1) {
            // fused sweep on the finest FP32 level, on the two finest, or nowhere
            for (int fm : {clamp_int(c->h3.g[0].interior()), clamp_int(c->h3.g[1].interior()), INT_MAX}) {
                mhs_solver_opts o = best;
                o.fused_min = fm;
                consider(o);
            }
            if (best.fused_min != INT_MAX)
                for (int rows : {8, 16}) {   // tile height of the fused sweep
                    mhs_solver_opts o = best;
                    o.tma_rows = rows;
                    consider(o);
                }
        }
        {
            mhs_solver_opts o = best;
            o.flags ^= MHS_FLAG_NO_FMG;
            consider(o);
        }
        if (!line) {   // thread-block shape of the point passes
            for (int t = 1; t <= N_TILES; ++t) {
                mhs_solver_opts o = best;
                o.tile = t;
                consider(o);
            }
        }
        if (same_opts(before, best)) break;
    }
    apply_opts(c, best);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_table[key_of(c, mode)] = best;
    }
    if (out) {
        out->opts = best;
        out->ms = best_ms;
        out->ms_start = start_ms;
        out->candidates = ncand;
        out->aniso_class = aniso_class(c);
    }
}

bool tune_lookup(const mhs_ctx* c, int mode, mhs_solver_opts* o) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_table.find(key_of(c, mode));
    if (it == g_tune_table.end()) return false;
    *o = it->second;
    return true;
}

void tune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_table.clear();
}

}  // namespace mhs
