// Grouped solves: many independent instances (uneven grids, own parameters
// and options) solved together, one kernel launch per multigrid operation
// and level for all of them, the whole solve captured in one CUDA graph with
// device-side convergence control (a while node per problem that runs while
// any instance still iterates; converged instances drop out of every launch).
//
// The sequence per instance is exactly that of its solo solve (solver.cu):
// lower-boundary prologue, full-multigrid first cycle, V-cycles until the
// relative residual is below the tolerance, then the same for the interior
// problem; every operation runs the solo kernels' bodies with the solo block
// decomposition, so each instance's result is bitwise the same as solving
// it alone.  What changes is the launch structure: a V-cycle of the whole
// group costs about (11 per global level + 1) launches instead of that
// number for every instance.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "df_bodies.cuh"
#include "group.h"
#include "line_body.cuh"
#include "mg_bodies.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

void* galloc(GPart* G, size_t bytes) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error(MHS_ERR_OUT_OF_MEMORY, "group: cudaMalloc failed");
    }
    G->allocs.push_back(p);
    return p;
}

GTable upload(GPart* G, std::vector<GItem>& v) {
    GTable t;
    long long off = 0;
    for (GItem& it : v) {
        it.first = int(off);
        off += (long long)it.gx * it.gy * it.gz;
    }
    if (off > 0x7fffffffLL) throw Error(MHS_ERR_INVALID_ARG, "group: a grouped launch needs more than 2^31 blocks");
    t.n = int(v.size());
    t.blocks = int(off);
    if (t.n) {
        t.items = static_cast<GItem*>(galloc(G, v.size() * sizeof(GItem)));
        MHS_CUDA(cudaMemcpy(t.items, v.data(), v.size() * sizeof(GItem), cudaMemcpyHostToDevice));
    }
    return t;
}

GItem item(int q, dim3 grid, const Geom& g, SolveCtl* ctl) {
    GItem it;
    std::memset(&it, 0, sizeof it);
    it.q = q;
    it.gx = int(grid.x);
    it.gy = int(grid.y);
    it.gz = int(grid.z);
    it.g = g;
    it.ctl = ctl;
    return it;
}

template <typename T>
LevelArrays<T>& arr(Hierarchy& H, int l);
template <>
LevelArrays<double>& arr<double>(Hierarchy& H, int l) { return H.d[l]; }
template <>
LevelArrays<float>& arr<float>(Hierarchy& H, int l) { return H.s[l]; }

int top_level(int L, int cut) { return std::min(std::max(cut, 1), L - 1); }

// level whose system the instance's cycles solve exactly (as in the solo
// V-cycle), or -1
template <typename T>
int exact_level(const Hierarchy& H) { return sizeof(T) == 8 ? H.exact64 : H.exact32; }

template <typename T>
std::vector<GSepTable<T>>& exact_tables(GDim& D);
template <>
std::vector<GSepTable<float>>& exact_tables<float>(GDim& D) { return D.exact32; }
template <>
std::vector<GSepTable<double>>& exact_tables<double>(GDim& D) { return D.exact64; }

// stage tables of the exact coarse-grid solves: items of stage s and kind k
// share a launch; block shapes of the plain mode solves follow the launch's
// thread count
template <typename T>
void upload_exact(GPart* G, GDim& D, std::vector<std::vector<GSepItem<T>>>& by_stage) {
    std::vector<GSepTable<T>>& out = exact_tables<T>(D);
    out.clear();
    for (auto& items : by_stage) {
        for (int kind = SEP_DST; kind <= SEP_DIVIDE; ++kind) {
            std::vector<GSepItem<T>> v;
            for (const GSepItem<T>& it : items)
                if (it.st.kind == kind) v.push_back(it);
            if (v.empty()) continue;
            GSepTable<T> t;
            t.kind = kind;
            for (const GSepItem<T>& it : v) {
                t.threads = std::max(t.threads, it.st.threads);
                t.smem = std::max(t.smem, it.st.smem);
            }
            long long off = 0;
            for (GSepItem<T>& it : v) {
                if (kind == SEP_THOMAS || kind == SEP_DIVIDE)
                    it.st.grid.x = unsigned((it.st.mode.nfast + t.threads - 1) / t.threads);
                it.gx = int(it.st.grid.x);
                it.gy = int(it.st.grid.y);
                it.gz = int(it.st.grid.z);
                it.first = int(off);
                off += (long long)it.gx * it.gy * it.gz;
            }
            if (off > 0x7fffffffLL) throw Error(MHS_ERR_INVALID_ARG, "group: a grouped launch needs more than 2^31 blocks");
            t.n = int(v.size());
            t.blocks = int(off);
            t.items = static_cast<GSepItem<T>*>(galloc(G, v.size() * sizeof(GSepItem<T>)));
            MHS_CUDA(cudaMemcpy(t.items, v.data(), v.size() * sizeof(GSepItem<T>), cudaMemcpyHostToDevice));
            out.push_back(t);
        }
    }
}

// Operations whose result does not depend on the block decomposition (every
// node written by one thread from values the launch does not write: colour
// passes, residuals without norms, transfers, elementwise updates) run in
// grouped launches with fewer, fatter blocks: the planes of an item are
// spread over at most 8 blocks along z, so a launch over hundreds of
// instances does not pay the per-block item lookup hundreds of thousands of
// times, and parts launched on concurrent streams share the GPU (sizing the
// cap to fill the GPU from each part alone was measured slower: 1,818 against
// 2,610 solves/s on a 256-instance mix).  Norm partials keep the solo
// decomposition (it fixes the summation order).
constexpr int kZCap = 8;
dim3 fat(dim3 grid) {
    grid.z = std::min<unsigned>(grid.z, kZCap);
    return grid;
}

// Build the tables of one problem for cycles in precision T.
template <typename T>
void build_dim(GPart* G, GDim& D, int dim) {
    const int n = int(G->hs.size());
    const bool dbl = sizeof(T) == 8, mixed = G->mode == MHS_MIXED;
    const int d3 = dim == 3;
    D.dim = dim;
    D.L = 0;
    for (mhs_ctx* c : G->hs) D.L = std::max(D.L, (dim == 3 ? c->h3 : c->h2).nlev());
    const int L = D.L;
    std::vector<std::vector<GItem>> pre_pt(L), post_pt(L), pre_ln(L), post_ln(L), res(L), restr(L), resr(L), prol(L),
        fmg_restr(L), fmg_prol(L);
    std::vector<GItem> sub, sub8, subz, subz8, zero_u, lower_rhs, zero_hi, zero_lo, split, copy_u, copy_t, df_copy, lift, bnorm, check1,
        res_norm0, res_norm, check, fmg_res_norm, fmg_check, zero_e, correct, fmg_zero_e, fmg_correct, to_double;
    std::vector<SubParams<T>> params;
    std::vector<std::vector<GSepItem<T>>> exact_items;   // per stage of the separable solves
    D.max_nu1 = D.max_nu2 = 0;
    D.max_top = -1;
    D.sub_smem = 0;
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = G->hs[q];
        Hierarchy& H = dim == 3 ? c->h3 : c->h2;
        SolveCtl* ctl = c->ctl + (dim == 3 ? 1 : 0);
        const int Lq = H.nlev();
        const int cut = dbl ? H.cut64 : H.cut32;
        const int ex = exact_level<T>(H);
        const int stop = ex >= 0 ? ex : cut;   // first level not cycled by per-level launches
        const bool fmg = !(c->opts.flags & MHS_FLAG_NO_FMG);
        const int top = fmg ? (ex >= 1 ? std::min(top_level(Lq, cut), ex) : top_level(Lq, cut)) : -1;
        const bool line = dim == 3 && use_zline(c);
        const int nu1 = c->opts.nu1, nu2 = c->opts.nu2;
        D.max_nu1 = std::max(D.max_nu1, nu1);
        D.max_nu2 = std::max(D.max_nu2, nu2);
        D.max_top = std::max(D.max_top, top);
        const bool fz = dbl && dim == 3 && c->f_zero_finest;   // f = 0 on the finest FP64 interior level
        // ---- V-cycle levels above the sub-cycle or the exact coarse-grid solve ----
        for (int l = 0; l < stop; ++l) {
            LevelArrays<T>& A = arr<T>(H, l);
            LevelArrays<T>& C = arr<T>(H, l + 1);
            const Geom& g = H.g[l];
            const Geom& gc = H.g[l + 1];
            T* f = (fz && l == 0) ? nullptr : A.f;
            GItem s = item(q, line ? (sizeof(T) == 4 ? zline_part_grid(g) : zline_grid(g)) : fat(smooth_grid_t<T>(g, d3)),
                           g, ctl);
            s.coef = A.coef;
            s.p[0] = A.u;
            s.p[1] = f;
            s.p[2] = A.r;
            s.ia[1] = top;
            s.ia[0] = nu1;
            (line ? pre_ln : pre_pt)[l].push_back(s);
            s.ia[0] = nu2;
            (line ? post_ln : post_pt)[l].push_back(s);
            if (dbl) {
                const bool red_l = red_residual_level(c, H);   // red nodes only, as the solo V-cycle
                GItem r = item(q, fat(red_l ? residual_red_grid(g, d3, false, 0) : residual_grid_plain_t<T>(g, d3)),
                               g, ctl);
                r.coef = A.coef;
                r.p[0] = A.u;
                r.p[1] = f;
                r.p[2] = A.r;
                r.ia[1] = top;
                r.ia[2] = red_l ? 1 : 0;
                res[l].push_back(r);
                GItem rs = item(q, fat(restrict_grid(gc, d3)), g, ctl);
                rs.g2 = gc;
                rs.p[0] = A.r;
                rs.p[1] = C.f;
                rs.p[2] = C.u;
                rs.ia[1] = top;
                rs.ia[2] = red_l ? 1 : 0;                                      // after this level's residual
                rs.ia[3] = (l == 0 && red_residual_rotated(c, H)) ? 1 : 0;    // in a rotated cycle
                restr[l].push_back(rs);
            } else {   // FP32 levels: the solo V-cycle's fused residual and restriction
                GItem r = item(q, fat(resid_restrict_grid(gc, d3)), g, ctl);
                r.g2 = gc;
                r.coef = A.coef;
                r.p[0] = A.u;
                r.p[1] = f;
                r.p[2] = C.f;
                r.p[3] = C.u;
                r.ia[1] = top;
                resr[l].push_back(r);
            }
            GItem pr = item(q, fat(prolong_grid(gc, d3)), gc, ctl);
            pr.g2 = g;
            pr.p[0] = C.u;
            pr.p[1] = A.u;
            pr.ia[1] = top;
            prol[l].push_back(pr);
        }
        // ---- full multigrid transfers ----
        for (int l = 0; l < top; ++l) {
            LevelArrays<T>& A = arr<T>(H, l);
            LevelArrays<T>& C = arr<T>(H, l + 1);
            const Geom& g = H.g[l];
            const Geom& gc = H.g[l + 1];
            GItem rs = item(q, fat(restrict_grid(gc, d3)), g, ctl);
            rs.g2 = gc;
            // the residual of the first test: FP64 mode in A.r of level 0, mixed mode the
            // double-float residual rounded into S.f of level 0
            rs.p[0] = l == 0 ? static_cast<void*>(mixed ? static_cast<void*>(H.s[0].f) : static_cast<void*>(H.d[0].r))
                             : static_cast<void*>(A.f);
            rs.p[1] = C.f;
            rs.p[2] = C.u;
            rs.ia[1] = top;
            fmg_restr[l].push_back(rs);
            GItem pr = item(q, fat(prolong_grid(gc, d3)), gc, ctl);
            pr.g2 = g;
            pr.p[0] = C.u;
            pr.p[1] = A.u;
            pr.ia[1] = top;
            fmg_prol[l].push_back(pr);
        }
        // ---- exact coarse-grid solve: the solo solve's stages ----
        if (ex >= 0) {
            std::vector<SepStage<T>> stages;
            sep_exact_plan<T>(c, H, ex, stages);
            if (exact_items.size() < stages.size()) exact_items.resize(stages.size());
            for (size_t k = 0; k < stages.size(); ++k) {
                GSepItem<T> it;
                std::memset(&it, 0, sizeof it);
                it.ctl = ctl;
                it.top = top;
                it.st = stages[k];
                exact_items[k].push_back(it);
            }
        }
        // ---- sub-cycle parameters for every start level from the cut-off down ----
        GItem sb = item(q, dim3(1, 1, 1), H.g[std::min(cut, Lq - 1)], ctl);
        sb.ia[1] = top;
        sb.ia[2] = int(params.size());
        sb.ia[3] = cut;
        const int rows = subcycle_rows(H.g[std::min(cut, Lq - 1)].interior());
        for (int s0 = cut; s0 < Lq; ++s0) {
            SubParams<T> p{};
            p.nlev = Lq - s0;
            p.dim = dim;
            p.nu1 = nu1;
            p.nu2 = nu2;
            p.line = line ? 1 : 0;
            p.rows = rows;
            size_t off = 0, ncoef = 0;
            for (int m = 0; m < p.nlev; ++m) {
                const Geom& gm = H.g[s0 + m];
                p.L[m].g = gm;
                p.L[m].coef = arr<T>(H, s0 + m).coef;
                p.L[m].off_u = int(off);
                off += round_up(gm.n, 4);
                p.L[m].off_f = int(off);
                off += round_up(gm.n, 4);
                ncoef += size_t(gm.nz);
            }
            p.u_g = arr<T>(H, s0).u;
            p.f_g = arr<T>(H, s0).f;
            p.smem_bytes = round_up(ncoef * sizeof(PlaneCoef<T>), 16) + off * sizeof(T);
            if (p.smem_bytes > subcycle_smem_limit())
                throw Error(MHS_ERR_INVALID_ARG, "group: a sub-cycle does not fit shared memory");
            D.sub_smem = std::max(D.sub_smem, p.smem_bytes);
            params.push_back(p);
        }
        if (ex < 0) {
            if (cut == 0) (rows == 8 ? subz8 : subz).push_back(sb);
            else (rows == 8 ? sub8 : sub).push_back(sb);
        }
        // ---- prologue, cycle end, epilogue ----
        const Geom& g0 = H.g[0];
        auto words = [](size_t elems, size_t bytes) { return int(elems * bytes / 4); };
        auto zero_item = [&](void* ptr, size_t elems, size_t bytes) {
            const int w = words(elems, bytes);
            GItem z = item(q, dim3(std::max(1, std::min(64, (w + 4095) / 4096)), 1, 1), g0, ctl);
            z.p[0] = ptr;
            z.ia[0] = w;
            return z;
        };
        // residual with norm partials of the first test, at the end of a cycle and after the
        // full-multigrid cycle (FP64: the last two on red nodes only where the solo solve does so)
        GItem rn;
        int nb;
        GItem rn_cyc, rn_fmg;
        int nb_cyc = 0, nb_fmg = 0;
        if (mixed) {
            const dim3 grid = df_residual_grid(g0, d3, c->ns.max_blocks);
            rn = item(q, grid, g0, ctl);
            const bool fz3 = dim == 3 && c->f_zero_finest;
            rn.coef = H.df.coef;
            rn.p[0] = H.df.hi;
            rn.p[1] = H.df.lo;
            rn.p[2] = fz3 ? nullptr : H.df.fh;
            rn.p[3] = fz3 ? nullptr : H.df.fl;
            rn.p[4] = H.s[0].f;
            rn.p[5] = c->ns.partial;
            nb = int(grid.x * grid.y * grid.z);
            rn_cyc = rn_fmg = rn;
            nb_cyc = nb_fmg = nb;
        } else {
            auto rn64 = [&](bool red, int& count) {
                const dim3 grid = red ? residual_red_grid(g0, d3, true, c->ns.max_blocks)
                                      : residual_grid(g0, d3, true, c->ns.max_blocks);
                GItem it = item(q, grid, g0, ctl);
                it.coef = H.d[0].coef;
                it.p[0] = H.d[0].u;
                it.p[1] = H.d[0].f;
                it.p[2] = H.d[0].r;
                it.p[3] = c->ns.partial;
                it.ia[2] = red ? 1 : 0;
                count = int(grid.x * grid.y * grid.z);
                return it;
            };
            rn = rn64(false, nb);
            rn_cyc = rn64(red_residual_cycle(c, H), nb_cyc);
            rn_fmg = rn64(red_residual_fmg(c, H), nb_fmg);
        }
        res_norm0.push_back(rn);
        res_norm.push_back(rn_cyc);
        GItem ck = item(q, dim3(1, 1, 1), g0, ctl);
        ck.p[0] = c->ns.partial;
        ck.ia[0] = nb;
        check1.push_back(ck);
        GItem ck_cyc = ck, ck_fmg = ck;
        ck_cyc.ia[0] = nb_cyc;
        ck_fmg.ia[0] = nb_fmg;
        check.push_back(ck_cyc);
        if (fmg) {
            fmg_res_norm.push_back(rn_fmg);
            fmg_check.push_back(ck_fmg);
        }
        if (dim == 2) {
            zero_u.push_back(zero_item(H.d[0].u, g0.n, sizeof(double)));
            GItem lr = item(q, mg_grid(g0, 0, g0.nx - 2, 0), g0, ctl);
            lr.p[0] = c->bz;
            lr.p[1] = H.d[0].f;
            lower_rhs.push_back(lr);
            if (mixed) {
                GItem sp = item(q, df_grid(g0, 0, 0), g0, ctl);
                sp.p[0] = H.d[0].f;
                sp.p[1] = H.df.fh;
                sp.p[2] = H.df.fl;
                split.push_back(sp);
            }
            GItem bn = ck;   // ||b|| from the residual of P = 0
            bnorm.push_back(bn);
        } else {
            Hierarchy& H2 = c->h2;
            const Geom& g2 = H2.g[0];
            zero_u.push_back(zero_item(H.d[0].u, g0.n, sizeof(double)));
            GItem cu = item(q, plane_grid(g2), g2, ctl);
            cu.g2 = g0;
            cu.p[0] = H2.d[0].u;
            cu.p[1] = H.d[0].u;
            copy_u.push_back(cu);
            cu.p[1] = H.d[0].t;
            copy_t.push_back(cu);
            if (mixed) {
                GItem dc = item(q, df_plane_grid(g2), g2, ctl);
                dc.g2 = g0;
                dc.p[0] = H2.df.hi;
                dc.p[1] = H2.df.lo;
                dc.p[2] = H.df.hi;
                dc.p[3] = H.df.lo;
                df_copy.push_back(dc);
                if (!c->f_zero_finest) {
                    GItem sp = item(q, fat(df_grid(g0, 1, 0)), g0, ctl);
                    sp.p[0] = H.d[0].f;
                    sp.p[1] = H.df.fh;
                    sp.p[2] = H.df.fl;
                    split.push_back(sp);
                }
            }
            const dim3 lg = lift_grid(g0);
            GItem lf = item(q, lg, g0, ctl);
            lf.coef = H.d[0].coef;
            lf.p[0] = H.d[0].u;
            lf.p[1] = c->ns.partial;
            lift.push_back(lf);
            GItem bn = ck;
            bn.ia[0] = int(lg.x * lg.y * lg.z);
            bnorm.push_back(bn);
        }
        if (mixed) {
            zero_hi.push_back(zero_item(H.df.hi, g0.n, sizeof(float)));
            zero_lo.push_back(zero_item(H.df.lo, g0.n, sizeof(float)));
            GItem ze = zero_item(H.s[0].u, g0.n, sizeof(float));
            zero_e.push_back(ze);
            GItem cr = item(q, fat(df_grid(g0, d3, 0)), g0, ctl);
            cr.p[0] = H.s[0].u;
            cr.p[1] = H.df.hi;
            cr.p[2] = H.df.lo;
            correct.push_back(cr);
            if (fmg) {
                fmg_zero_e.push_back(ze);
                fmg_correct.push_back(cr);
            }
            GItem td = item(q, dim3(std::max<size_t>(1, std::min<size_t>(64, (g0.n + 16 * DF_TO_DOUBLE_THREADS - 1) /
                                                                                 (16 * DF_TO_DOUBLE_THREADS))),
                                    1, 1),
                            g0, ctl);
            td.p[0] = H.df.hi;
            td.p[1] = H.df.lo;
            td.p[2] = H.d[0].u;
            to_double.push_back(td);
        }
    }
    auto up = [&](std::vector<std::vector<GItem>>& src, std::vector<GTable>& dst) {
        dst.resize(src.size());
        for (size_t l = 0; l < src.size(); ++l) dst[l] = upload(G, src[l]);
    };
    up(pre_pt, D.pre_pt);
    up(post_pt, D.post_pt);
    up(pre_ln, D.pre_ln);
    up(post_ln, D.post_ln);
    // launch shape of the partitioned FP32 z-line passes: the most segments and
    // the largest shared-memory need among the items of a launch
    for (auto* pr : {&pre_ln, &post_ln}) {
        std::vector<GTable>& dst = pr == &pre_ln ? D.pre_ln : D.post_ln;
        for (size_t l = 0; l < pr->size(); ++l)
            for (const GItem& it : (*pr)[l]) {
                const int n = it.g.nz - 2, S = zpart_segments(n);
                dst[l].ty = std::max(dst[l].ty, S);
                dst[l].smem = std::max(dst[l].smem, unsigned(zpart_smem(n, S)));
            }
    }
    up(res, D.res);
    up(restr, D.restr);
    up(resr, D.resr);
    up(prol, D.prol);
    up(fmg_restr, D.fmg_restr);
    up(fmg_prol, D.fmg_prol);
    D.sub = upload(G, sub);
    D.sub8 = upload(G, sub8);
    D.subz = upload(G, subz);
    D.subz8 = upload(G, subz8);
    upload_exact<T>(G, D, exact_items);
    D.params = galloc(G, params.size() * sizeof(SubParams<T>));
    MHS_CUDA(cudaMemcpy(D.params, params.data(), params.size() * sizeof(SubParams<T>), cudaMemcpyHostToDevice));
    D.zero_u = upload(G, zero_u);
    D.lower_rhs = upload(G, lower_rhs);
    D.zero_hi = upload(G, zero_hi);
    D.zero_lo = upload(G, zero_lo);
    D.split = upload(G, split);
    D.copy_u = upload(G, copy_u);
    D.copy_t = upload(G, copy_t);
    D.df_copy = upload(G, df_copy);
    D.lift = upload(G, lift);
    D.bnorm = upload(G, bnorm);
    D.check1 = upload(G, check1);
    D.res_norm0 = upload(G, res_norm0);
    D.res_norm = upload(G, res_norm);
    D.check = upload(G, check);
    D.fmg_res_norm = upload(G, fmg_res_norm);
    D.fmg_check = upload(G, fmg_check);
    D.zero_e = upload(G, zero_e);
    D.correct = upload(G, correct);
    D.fmg_zero_e = upload(G, fmg_zero_e);
    D.fmg_correct = upload(G, fmg_correct);
    D.to_double = upload(G, to_double);
}

}  // namespace

}  // namespace mhs

namespace mhs {

namespace {

// One V-cycle from level s for every instance: levels s .. of each instance
// above its sub-cycle cut-off, then its sub-cycle from max(s, cut-off).
// fmg_step >= 0 restricts the launch to instances whose full-multigrid top
// level is at least fmg_step (the up-sweep of the first cycle).
template <typename T>
void gsmooth(GPart* G, GDim& D, std::vector<GTable>& pt, std::vector<GTable>& ln, int l, int nsweep, int fmg_step,
             int gate) {
    const int d3 = D.dim == 3;
    for (int w = 0; w < nsweep; ++w) {
        for (int colour = 0; colour < 2; ++colour) glaunch_colour<T>(pt[l], d3, colour, w, fmg_step, gate, G->stream);
        for (int colour = 0; colour < 2; ++colour) glaunch_zline<T>(ln[l], colour, w, fmg_step, gate, G->stream);
    }
}

// levels s.. of the instances above their cut-off, their sub-cycles or exact
// solves, and back up to level s (with_z: also the instances whose sub-cycle
// starts at level 0)
template <typename T>
void gvcycle_from(GPart* G, GDim& D, int s, int fmg_step, int gate, bool with_z) {
    cudaStream_t st = G->stream;
    const int d3 = D.dim == 3;
    for (int l = s; l < D.L - 1; ++l) {
        gsmooth<T>(G, D, D.pre_pt, D.pre_ln, l, D.max_nu1, fmg_step, gate);
        glaunch_residual<T>(D.res[l], d3, fmg_step, gate, st);
        glaunch_restrict<T>(D.restr[l], d3, fmg_step, gate, st);
        glaunch_resid_restrict<T>(D.resr[l], d3, fmg_step, gate, st);
    }
    const SubParams<T>* params = static_cast<const SubParams<T>*>(D.params);
    glaunch_subcycle<T>(D.sub, params, d3, s, fmg_step, gate, D.sub_smem, 32, st);
    glaunch_subcycle<T>(D.sub8, params, d3, s, fmg_step, gate, D.sub_smem, 8, st);
    if (with_z) {
        glaunch_subcycle<T>(D.subz, params, d3, s, fmg_step, gate, D.sub_smem, 32, st);
        glaunch_subcycle<T>(D.subz8, params, d3, s, fmg_step, gate, D.sub_smem, 8, st);
    }
    for (const GSepTable<T>& t : exact_tables<T>(D)) glaunch_sep<T>(t, fmg_step, gate, st);
    for (int l = D.L - 2; l >= s; --l) {
        glaunch_prolong<T>(D.prol[l], d3, fmg_step, gate, st);
        gsmooth<T>(G, D, D.post_pt, D.post_ln, l, D.max_nu2, fmg_step, gate);
    }
}

template <typename T>
void gvcycle(GPart* G, GDim& D, int s, int fmg_step, int gate) {
    gvcycle_from<T>(G, D, s, fmg_step, gate, true);
}

// FP64 cycles with the convergence test after the pre-smoothing (as the solo
// solve): instances above their cut-off at level 0 take the coarse-grid
// correction of the latest residual, post- and then pre-smoothing; instances
// whose sub-cycle starts at level 0 take a whole sub-cycle
void gvcycle_rotated(GPart* G, GDim& D, int gate) {
    cudaStream_t st = G->stream;
    const int d3 = D.dim == 3;
    glaunch_restrict<double>(D.restr[0], d3, -1, gate, st, 1);
    gvcycle_from<double>(G, D, 1, -1, gate, false);
    const SubParams<double>* params = static_cast<const SubParams<double>*>(D.params);
    glaunch_subcycle<double>(D.subz, params, d3, 0, -1, gate, D.sub_smem, 32, st);
    glaunch_subcycle<double>(D.subz8, params, d3, 0, -1, gate, D.sub_smem, 8, st);
    glaunch_prolong<double>(D.prol[0], d3, -1, gate, st);
    gsmooth<double>(G, D, D.post_pt, D.post_ln, 0, D.max_nu2, -1, gate);
    gsmooth<double>(G, D, D.pre_pt, D.pre_ln, 0, D.max_nu1, -1, gate);
}

// first cycle by full multigrid on the correction equation (instances
// without MHS_FLAG_NO_FMG): restrict the first residual to each instance's
// top level, then up level by level: prolongate and run a V-cycle
template <typename T>
void gfmg(GPart* G, GDim& D) {
    cudaStream_t st = G->stream;
    const int d3 = D.dim == 3;
    const bool mixed = G->mode == MHS_MIXED;
    if (D.max_top < 0) return;
    if (mixed) glaunch_zero(D.fmg_zero_e, G_ALL, st);
    for (int l = 0; l < D.L - 1; ++l) glaunch_restrict<T>(D.fmg_restr[l], d3, -1, G_ALL, st);
    for (int s = D.max_top; s >= 0; --s) {
        if (s < D.L - 1) glaunch_prolong<T>(D.fmg_prol[s], d3, -1, G_ALL, st);
        gvcycle<T>(G, D, s, s, G_ALL);
    }
    if (mixed) glaunch_df_correct(D.fmg_correct, d3, G_ALL, st);
    if (mixed) glaunch_df_residual(D.fmg_res_norm, d3, G_ALL, st);
    else glaunch_residual_norm<double>(D.fmg_res_norm, d3, G_ALL, st);
    glaunch_check(D.fmg_check, 2, G_ALL, st);
}

template <typename T>
void gprologue(GPart* G, GDim& D) {
    cudaStream_t st = G->stream;
    const int d3 = D.dim == 3;
    const bool mixed = G->mode == MHS_MIXED;
    glaunch_zero(D.zero_u, G_ALL, st);
    if (!d3) {
        glaunch_lower_rhs(D.lower_rhs, st);
        if (mixed) {
            glaunch_zero(D.zero_hi, G_ALL, st);
            glaunch_zero(D.zero_lo, G_ALL, st);
            glaunch_df_split(D.split, 0, st);
        }
        if (mixed) glaunch_df_residual(D.res_norm0, 0, G_ALL, st);
        else glaunch_residual_norm<double>(D.res_norm0, 0, G_ALL, st);
        glaunch_bnorm(D.bnorm, st);
    } else {
        glaunch_copy_plane(D.copy_u, st);
        glaunch_copy_plane(D.copy_t, st);
        if (mixed) {
            glaunch_zero(D.zero_hi, G_ALL, st);
            glaunch_zero(D.zero_lo, G_ALL, st);
            glaunch_df_copy_plane(D.df_copy, st);
            glaunch_df_split(D.split, 1, st);
        }
        glaunch_lift_norm(D.lift, st);
        glaunch_bnorm(D.bnorm, st);
        if (mixed) glaunch_df_residual(D.res_norm0, 1, G_ALL, st);
        else glaunch_residual_norm<double>(D.res_norm0, 1, G_ALL, st);
    }
    glaunch_check(D.check1, 1, G_ALL, st);
    gfmg<T>(G, D);
}

template <typename T>
void gcycle(GPart* G, GDim& D, SolveCtl* const* ctls, cudaGraphConditionalHandle h, bool graph = true) {
    cudaStream_t st = G->stream;
    const int d3 = D.dim == 3;
    const bool mixed = G->mode == MHS_MIXED;
    if (mixed) glaunch_zero(D.zero_e, G_ACTIVE, st);
    if (mixed || D.L < 2) gvcycle<T>(G, D, 0, -1, G_ACTIVE);
    else gvcycle_rotated(G, D, G_ACTIVE);
    if (mixed) {
        glaunch_df_correct(D.correct, d3, G_ACTIVE, st);
        glaunch_df_residual(D.res_norm, d3, G_ACTIVE, st);
    } else {
        glaunch_residual_norm<double>(D.res_norm, d3, G_ACTIVE, st);
    }
    glaunch_check(D.check, 0, G_ACTIVE, st);
    if (graph) glaunch_any(ctls, int(G->hs.size()), h, 1, nullptr, st);
}

// append a while node (condition handle h) to the graph captured on
// G->stream, its body captured from fn on the second capture stream
template <typename F>
void gadd_while(GPart* G, cudaGraphConditionalHandle h, F&& fn) {
    cudaStreamCaptureStatus status;
    cudaGraph_t graph;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    MHS_CUDA(cudaStreamGetCaptureInfo(G->stream, &status, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MHS_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    MHS_CUDA(cudaStreamUpdateCaptureDependencies(G->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t outer = G->stream;
    G->stream = G->cap2;
    MHS_CUDA(cudaStreamBeginCaptureToGraph(G->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    fn();
    cudaGraph_t captured;
    MHS_CUDA(cudaStreamEndCapture(G->stream, &captured));
    G->stream = outer;
}

template <typename T>
void gbuild_graph(GPart* G) {
    const int n = int(G->hs.size());
    cudaStream_t user = G->stream;
    G->stream = G->cap;
    cudaGraph_t graph = nullptr;
    try {
        MHS_CUDA(cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeThreadLocal));
        cudaStreamCaptureStatus status;
        cudaGraph_t g;
        MHS_CUDA(cudaStreamGetCaptureInfo(G->stream, &status, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h2, h3;
        MHS_CUDA(cudaGraphConditionalHandleCreate(&h2, g, 0, cudaGraphCondAssignDefault));
        MHS_CUDA(cudaGraphConditionalHandleCreate(&h3, g, 0, cudaGraphCondAssignDefault));
        const long long l0 = launches();
        gprologue<T>(G, G->d2);
        glaunch_any(G->ctls, n, h2, 1, nullptr, G->stream);
        const long long l1 = launches();
        gadd_while(G, h2, [&] { gcycle<T>(G, G->d2, G->ctls, h2); });
        const long long l2 = launches();
        if (G->mode == MHS_MIXED) glaunch_df_to_double(G->d2.to_double, G->stream);
        gprologue<T>(G, G->d3);
        glaunch_any(G->ctls + n, n, h3, 1, nullptr, G->stream);
        const long long l3 = launches();
        gadd_while(G, h3, [&] { gcycle<T>(G, G->d3, G->ctls + n, h3); });
        const long long l4 = launches();
        if (G->mode == MHS_MIXED) glaunch_df_to_double(G->d3.to_double, G->stream);
        glaunch_gather_ctl(G->ctls, 2 * n, G->gathered, G->stream);
        const long long l5 = launches();
        MHS_CUDA(cudaStreamEndCapture(G->stream, &graph));
        MHS_CUDA(cudaGraphInstantiate(&G->exec, graph, 0));
        cudaGraphDestroy(graph);
        // capture records launches without running them: take them back and
        // keep the counts per section, added per executed cycle after a solve
        G->n_fixed = (l1 - l0) + (l3 - l2) + (l5 - l4);
        G->n_cycle2 = l2 - l1;
        G->n_cycle3 = l4 - l3;
        count_launches(-(l5 - l0));
    } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(G->stream, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        (void)cudaGetLastError();
        G->stream = user;
        throw;
    }
    G->stream = user;
}

}  // namespace

GPart* part_create(mhs_ctx** hs, int n, int mode) {
    auto G = std::make_unique<GPart>();
    G->mode = mode;
    G->hs.assign(hs, hs + n);
    for (mhs_ctx* c : G->hs) {
        if (c->opts.flags & MHS_FLAG_WARM) throw Error(MHS_ERR_INVALID_ARG, "group: warm starts are not supported");
        if (c->opts.inner_cycles != 1) throw Error(MHS_ERR_INVALID_ARG, "group: inner_cycles must be 1");
        if (c->opts.flags & MHS_FLAG_SEPARABLE)
            throw Error(MHS_ERR_INVALID_ARG, "group: the separable inner solver is not available in groups");
        if (mode == MHS_MIXED && (c->opts.flags & MHS_FLAG_LOWER_FP64))
            throw Error(MHS_ERR_INVALID_ARG, "group: MHS_FLAG_LOWER_FP64 is not available in groups");
    }
    if (n == 1) {   // its own launch stream, as the instance of a batched solve has
        G->solo = true;
        MHS_CUDA(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
        return G.release();
    }
    gsubcycle_prepare();
    MHS_CUDA(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
    MHS_CUDA(cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking));
    MHS_CUDA(cudaStreamCreateWithFlags(&G->cap2, cudaStreamNonBlocking));
    MHS_CUDA(cudaEventCreate(&G->ev0));
    MHS_CUDA(cudaEventCreate(&G->ev1));
    std::vector<SolveCtl*> ctls(2 * size_t(n));
    for (int q = 0; q < n; ++q) {
        ctls[q] = G->hs[q]->ctl + 0;
        ctls[n + q] = G->hs[q]->ctl + 1;
    }
    G->ctls = static_cast<SolveCtl**>(galloc(G.get(), ctls.size() * sizeof(SolveCtl*)));
    MHS_CUDA(cudaMemcpy(G->ctls, ctls.data(), ctls.size() * sizeof(SolveCtl*), cudaMemcpyHostToDevice));
    G->gathered = static_cast<SolveCtl*>(galloc(G.get(), 2 * size_t(n) * sizeof(SolveCtl)));
    MHS_CUDA(cudaMallocHost(&G->gathered_host, 2 * size_t(n) * sizeof(SolveCtl)));
    G->any_dev = static_cast<int*>(galloc(G.get(), sizeof(int)));
    MHS_CUDA(cudaMallocHost(&G->any_host, sizeof(int)));
    if (mode == MHS_MIXED) {
        build_dim<float>(G.get(), G->d2, 2);
        build_dim<float>(G.get(), G->d3, 3);
        gbuild_graph<float>(G.get());
    } else {
        build_dim<double>(G.get(), G->d2, 2);
        build_dim<double>(G.get(), G->d3, 3);
        gbuild_graph<double>(G.get());
    }
    return G.release();
}

void part_destroy(GPart* G) {
    if (!G) return;
    if (G->stream) cudaStreamSynchronize(G->stream);
    if (G->exec) cudaGraphExecDestroy(G->exec);
    for (void* p : G->allocs) cudaFree(p);
    if (G->gathered_host) cudaFreeHost(G->gathered_host);
    if (G->any_host) cudaFreeHost(G->any_host);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    if (G->stream) cudaStreamDestroy(G->stream);
    if (G->cap) cudaStreamDestroy(G->cap);
    if (G->cap2) cudaStreamDestroy(G->cap2);
    delete G;
}

// Host-driven form of the graph's sequence (the same launches; the loops
// read the OR of the continuation flags back after each cycle), for
// profilers that cannot see kernels inside conditional graph nodes.
template <typename T>
void geager(GPart* G) {
    const int n = int(G->hs.size());
    auto any = [&](SolveCtl* const* ctls) {
        glaunch_any(ctls, n, 0, 0, G->any_dev, G->stream);
        MHS_CUDA(cudaMemcpyAsync(G->any_host, G->any_dev, sizeof(int), cudaMemcpyDeviceToHost, G->stream));
        MHS_CUDA(cudaStreamSynchronize(G->stream));
        return *G->any_host != 0;
    };
    gprologue<T>(G, G->d2);
    while (any(G->ctls)) gcycle<T>(G, G->d2, G->ctls, 0, false);
    if (G->mode == MHS_MIXED) glaunch_df_to_double(G->d2.to_double, G->stream);
    gprologue<T>(G, G->d3);
    while (any(G->ctls + n)) gcycle<T>(G, G->d3, G->ctls + n, 0, false);
    if (G->mode == MHS_MIXED) glaunch_df_to_double(G->d3.to_double, G->stream);
    glaunch_gather_ctl(G->ctls, 2 * n, G->gathered, G->stream);
}

// Enqueue one grouped solve on the group's stream: control blocks
// initialised on the host and copied in, the graph (or the eager sequence)
// launched, the control blocks gathered back into pinned memory.
void part_launch(GPart* G, double tol, cudaStream_t st) {
    const int n = int(G->hs.size());
    G->tol = tol;
    if (G->solo) {
        mhs_ctx* c = G->hs[0];
        const cudaStream_t user = c->stream;
        const bool graphs = c->use_graphs;
        c->stream = st;
        c->use_graphs = !G->eager;
        try {
            solve_begin(c, tol, G->mode);
        } catch (...) {
            c->stream = user;
            c->use_graphs = graphs;
            throw;
        }
        c->stream = user;
        c->use_graphs = graphs;
        G->launch_stream = st;
        return;
    }
    const cudaStream_t own = G->stream;
    G->stream = st;
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = G->hs[q];
        for (int k = 0; k < 2; ++k) {
            c->ctl_host[k] = SolveCtl{};
            c->ctl_host[k].tol = tol;
            c->ctl_host[k].max_cycles = c->opts.max_cycles;
        }
        MHS_CUDA(cudaMemcpyAsync(c->ctl, c->ctl_host, 2 * sizeof(SolveCtl), cudaMemcpyHostToDevice, G->stream));
    }
    MHS_CUDA(cudaEventRecord(G->ev0, G->stream));
    try {
        if (G->eager) {
            if (G->mode == MHS_MIXED) geager<float>(G);
            else geager<double>(G);
        } else {
            MHS_CUDA(cudaGraphLaunch(G->exec, G->stream));
        }
    } catch (...) {
        G->stream = own;
        throw;
    }
    MHS_CUDA(cudaEventRecord(G->ev1, G->stream));
    MHS_CUDA(cudaMemcpyAsync(G->gathered_host, G->gathered, 2 * size_t(n) * sizeof(SolveCtl), cudaMemcpyDeviceToHost,
                             G->stream));
    G->launch_stream = st;
    G->stream = own;
}

// Wait for the solve enqueued by part_launch and report it.  Returns the
// first failing instance's status (per-instance statuses in `statuses`).
mhs_status part_wait(GPart* G, mhs_solve_info* infos, mhs_status* statuses, double* ms_out) {
    const int n = int(G->hs.size());
    const double tol = G->tol;
    if (G->solo) {
        mhs_ctx* c = G->hs[0];
        const cudaStream_t user = c->stream;
        c->stream = G->launch_stream;
        mhs_solve_info info{};
        mhs_status s = MHS_OK;
        try {
            s = solve_end(c, tol, G->mode, &info);
        } catch (const Error& e) {
            s = e.status;
            if (s == MHS_ERR_CUDA) {
                c->stream = user;
                throw;
            }
        }
        c->stream = user;
        if (infos) infos[0] = info;
        if (statuses) statuses[0] = s;
        if (ms_out) *ms_out = info.ms;
        return s;
    }
    MHS_CUDA(cudaEventSynchronize(G->ev1));
    MHS_CUDA(cudaStreamSynchronize(G->launch_stream));
    float ms = 0.f;
    MHS_CUDA(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
    if (ms_out) *ms_out = ms;
    int max2 = 0, max3 = 0;
    mhs_status worst = MHS_OK;
    for (int q = 0; q < n; ++q) {
        mhs_ctx* c = G->hs[q];
        const SolveCtl& a = G->gathered_host[q];
        const SolveCtl& b = G->gathered_host[n + q];
        c->ctl_host[0] = a;
        c->ctl_host[1] = b;
        max2 = std::max(max2, a.bodies);   // while iterations: the most bodies any instance ran
        max3 = std::max(max3, b.bodies);
        mhs_status s = MHS_OK;
        if (a.status != MHS_OK || b.status != MHS_OK) s = MHS_ERR_NONFINITE;
        else if (!(a.bnorm == 0.0 || a.rel < tol) || !(b.bnorm == 0.0 || b.rel < tol)) s = MHS_ERR_NO_CONVERGENCE;
        if (infos) {
            mhs_solve_info& i = infos[q];
            i.cycles_2d = a.cycles;
            i.cycles_3d = b.cycles;
            i.rel_res_2d = a.rel;
            i.rel_res_3d = b.rel;
            i.conv_factor = (b.cycles > 0 && b.rel0 > 0 && b.rel > 0) ? std::pow(b.rel / b.rel0, 1.0 / b.cycles) : 0.0;
            i.ms = ms;
            i.outer_iters_2d = G->mode == MHS_MIXED ? a.cycles : 0;
            i.outer_iters_3d = G->mode == MHS_MIXED ? b.cycles : 0;
        }
        if (statuses) statuses[q] = s;
        if (s != MHS_OK && worst == MHS_OK) worst = s;
        c->have_solution = true;
    }
    // graph: the prologues and epilogues once, each while body once per cycle of the slowest instance
    if (!G->eager) count_launches(G->n_fixed + (long long)max2 * G->n_cycle2 + (long long)max3 * G->n_cycle3);
    return worst;
}

// Device bytes one multigrid cycle of a handle's interior problem touches:
// the arrays of every level in the precision of the cycles, plus the
// double-float state of the finest level in mixed mode.
size_t cycle_bytes(const mhs_ctx* c, int mode) {
    size_t b = 0;
    const Hierarchy& H = c->h3;
    const size_t s = mode == MHS_MIXED ? sizeof(float) : sizeof(double);
    for (int l = 0; l < H.nlev(); ++l) b += 3 * H.g[l].n * s;
    if (mode == MHS_MIXED) b += 2 * H.g[0].n * sizeof(float);
    return b;
}

// ---- groups: parts of L2-sized working sets on a few launch streams ----

mhs_group* group_create(mhs_ctx** hs, int n, int mode, size_t part_bytes, int nstreams) {
    if (part_bytes == 0) {
        int dev = 0, l2 = 0;
        MHS_CUDA(cudaGetDevice(&dev));
        MHS_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        part_bytes = size_t(l2) / 2;
    }
    if (nstreams <= 0) nstreams = 16;
    auto G = std::make_unique<mhs_group>();
    G->n = n;
    // instances by decreasing cycle working set (stable), then greedy: a part
    // takes instances until the next would push its working set over
    // part_bytes.  Similar sizes share a part, so a part's lock-step cycles
    // do not make small instances wait on large ones, large instances get
    // parts of their own that run concurrently, and small ones pack into
    // few launches.
    std::vector<size_t> bytes(n);
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) {
        bytes[q] = cycle_bytes(hs[q], mode);
        order[q] = q;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes[a] > bytes[b]; });
    // An instance whose working set exceeds a sixteenth of part_bytes takes a part of its own (it runs
    // its own solve): grouping pays where launch latency dominates, and a larger instance's own graph
    // (TMA-staged sweeps, vector passes, cluster transforms) on its own stream beats lock-step grouped
    // launches (measured on the 256-instance mix: grouping its 65^3 instances cost 7 %).
    std::vector<int> cur;
    size_t acc = 0;
    for (int q : order) {
        const size_t b = bytes[q];
        if (b > part_bytes / 16) {
            G->members.push_back({q});
            continue;
        }
        if (!cur.empty() && acc + b > part_bytes) {
            G->members.push_back(cur);
            cur.clear();
            acc = 0;
        }
        cur.push_back(q);
        acc += b;
    }
    if (!cur.empty()) G->members.push_back(cur);
    try {
        for (const auto& m : G->members) {
            std::vector<mhs_ctx*> part;
            for (int q : m) part.push_back(hs[q]);
            G->parts.push_back(part_create(part.data(), int(part.size()), mode));
        }
        const int k = std::min<int>(nstreams, int(G->parts.size()));
        for (int s = 0; s < k; ++s) {
            cudaStream_t st;
            MHS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            G->streams.push_back(st);
        }
    } catch (...) {
        group_destroy(G.release());
        throw;
    }
    return G.release();
}

void group_destroy(mhs_group* G) {
    if (!G) return;
    for (GPart* p : G->parts) part_destroy(p);
    for (cudaStream_t s : G->streams) cudaStreamDestroy(s);
    delete G;
}

void group_set_eager(mhs_group* G, bool eager) {
    G->eager = eager;
    for (GPart* p : G->parts) p->eager = eager;
}

mhs_status group_solve(mhs_group* G, double tol, mhs_solve_info* infos, mhs_status* statuses) {
    const size_t P = G->parts.size();
    // the single-instance parts first, each on its own stream, in the caller's instance order (sizes as
    // they come, rather than the size order of the packing, spread the load over the device's hardware
    // queues); then the grouped parts, round-robin on the launch streams: their lock-step cycles of
    // small instances fill the device while the large instances drain (on the 256-instance mix this
    // order measured 3,142-3,151 solves/s against 3,105 with the grouped parts launched first)
    size_t k = 0;
    std::vector<size_t> solo;
    for (size_t p = 0; p < P; ++p)
        if (G->parts[p]->solo) solo.push_back(p);
    std::sort(solo.begin(), solo.end(), [&](size_t a, size_t b) { return G->members[a][0] < G->members[b][0]; });
    for (size_t p : solo) part_launch(G->parts[p], tol, G->parts[p]->stream);
    for (size_t p = 0; p < P; ++p)
        if (!G->parts[p]->solo) part_launch(G->parts[p], tol, G->streams[k++ % G->streams.size()]);
    mhs_status worst = MHS_OK;
    std::vector<mhs_solve_info> pi;
    std::vector<mhs_status> ps;
    double ms_max = 0.0;
    for (size_t p = 0; p < P; ++p) {
        const auto& m = G->members[p];
        pi.assign(m.size(), mhs_solve_info{});
        ps.assign(m.size(), MHS_OK);
        double ms = 0.0;
        const mhs_status s = part_wait(G->parts[p], pi.data(), ps.data(), &ms);
        ms_max = std::max(ms_max, ms);
        if (s != MHS_OK && worst == MHS_OK) worst = s;
        for (size_t i = 0; i < m.size(); ++i) {
            if (infos) infos[m[i]] = pi[i];
            if (statuses) statuses[m[i]] = ps[i];
        }
    }
    (void)ms_max;
    return worst;
}

}  // namespace mhs
