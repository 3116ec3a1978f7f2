// Device-side convergence control and the one-CTA multigrid sub-cycle, as
// bodies shared by the solver's own kernels (kernels_ctl.cu) and the
// grouped launches over many instances (kernels_group.cu).
//
// check_body finishes a residual norm in a fixed summation order, forms the
// relative residual ||b - A u|| / ||b|| (the stopping test of a multigrid
// solve) and counts cycles.
//
// subcycle_body runs a complete V(nu1,nu2)-cycle over the coarse levels of
// a hierarchy (from a cut-off level down to the coarsest) inside one CTA,
// with every level held in shared memory: red-black Gauss-Seidel (or zebra
// z-line) sweeps, residual and full-weighting restriction fused into one
// pass, (bi/tri)linear prolongation, and relaxation to convergence on the
// coarsest level.  Coarse levels are too small to occupy the GPU, so one
// launch replaces the dozens of latency-bound launches they would take.
#pragma once

#include <cmath>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

// ||b|| of a solve from its norm partials; resets the control block
__device__ __forceinline__ void bnorm_body(const double* __restrict__ partial, int n, SolveCtl* ctl) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        ctl->bnorm = sqrt(s);
        ctl->cycles = 0;
        ctl->status = MHS_OK;
        ctl->cont = 0;
        ctl->bodies = 0;
    }
}

// Convergence test after a cycle: finishes the residual norm in a fixed
// order, updates the control block and returns (in thread 0) whether
// another cycle is needed.  first = 1: the initial test; first = 2: after
// the full-multigrid cycle of the prologue, which counts as a cycle only if
// the initial test asked for one; first = 0: after a cycle.
__device__ __forceinline__ int check_body(const double* __restrict__ partial, int n, SolveCtl* ctl, int first) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    s = block_sum(s);
    int cont = 0;
    if (threadIdx.x == 0) {
        const double rn = sqrt(s);
        const double b = ctl->bnorm;
        const double rel = b > 0.0 ? rn / b : 0.0;
        if (first == 0 || (first == 2 && ctl->cont)) ctl->cycles += 1;
        if (first == 0) ctl->bodies += 1;
        ctl->rel = rel;
        if (first == 1) ctl->rel0 = rel;
        cont = (b > 0.0 && rel >= ctl->tol && ctl->cycles < ctl->max_cycles) ? 1 : 0;
        if (!isfinite(rn)) {
            ctl->status = MHS_ERR_NONFINITE;
            cont = 0;
        }
        ctl->cont = cont;
    }
    return cont;
}

// ---------------------------------------------------------------------------
// one-CTA sub-cycle
// ---------------------------------------------------------------------------
//
// Threads are arranged as SX x rows (x fastest; rows = blockDim.y, 8 or 32).  Every phase walks the rows
// (j, k) of a level with threadIdx.y and the x positions with threadIdx.x,
// so index decoding costs one division per row, and reads only shared
// memory: the levels' arrays, geometry and per-plane coefficients are
// staged there at the start.

constexpr int SX = 32, SY = 32;

struct SubGeom {
    int nx, ny, nz, px;
    int plane;          // px * ny
    int n;              // allocated elements of the level
    int off_u, off_f;   // offsets in the array area of shared memory (elements)
    int off_c;          // offset of the level's coefficients in the coefficient area
    int nxi, nyi, hx;   // interior counts along x and y, nodes of one colour per row (ceil(nxi/2))
    float inv_nxi, inv_nyi, inv_hx;
};

// floor(q / d) for 0 <= q < 2^18 and 1 <= d <= 2^10 from a float reciprocal:
// (q + 1/2) / d lies at least 1/(2d) from an integer, far more than the
// rounding error of the product.
__device__ __forceinline__ int fdiv(int q, float inv_d) { return int((float(q) + 0.5f) * inv_d); }

template <typename T, bool D3>
struct SubSmem {
    T* a;                       // arrays
    const PlaneCoef<T>* c;      // coefficients of all levels
    const SubGeom* g;
};

template <typename T, bool D3>
__device__ __forceinline__ T sub_off(const SubGeom& g, const PlaneCoef<T>& c, const T* u, int o) {
    T off = c.cx * (u[o + 1] + u[o - 1]) + c.cy * (u[o + g.px] + u[o - g.px]);
    if (D3) off += c.cz * (u[o + g.plane] + u[o - g.plane]);
    return off;
}

// one red-black sweep (colour 0 = (i+j+k) even first)
template <typename T, bool D3>
__device__ void sub_smooth(const SubSmem<T, D3>& S, int l) {
    const SubGeom g = S.g[l];
    T* u = S.a + g.off_u;
    const T* f = S.a + g.off_f;
    const PlaneCoef<T>* cf = S.c + g.off_c;
    const int nw = g.hx * g.nyi * (D3 ? g.nz - 2 : 1);
    const int tid = threadIdx.x + SX * threadIdx.y;
    for (int colour = 0; colour < 2; ++colour) {
        for (int q = tid; q < nw; q += SX * blockDim.y) {
            const int row = fdiv(q, g.inv_hx);
            const int t = q - row * g.hx;
            const int kk = D3 ? fdiv(row, g.inv_nyi) : 0;
            const int j = 1 + row - kk * g.nyi;
            const int k = D3 ? 1 + kk : 0;
            const int i = 1 + (((1 + j + k) & 1) != colour) + 2 * t;
            if (i > g.nx - 2) continue;
            const PlaneCoef<T> c = cf[k];
            const int o = i + g.px * (j + g.ny * k);
            u[o] = (f[o] - sub_off<T, D3>(g, c, u, o)) * c.inv_d;
        }
        __syncthreads();
    }
}

// one zebra z-line sweep (columns with i + j even first): each thread solves
// the tridiagonal system of one column exactly (elimination factors lm, lsup
// of the level's coefficient records), the eliminated right-hand side held
// in the column's own entries of u until the back substitution
template <typename T>
__device__ void sub_zline(const SubSmem<T, true>& S, int l) {
    const SubGeom g = S.g[l];
    T* u = S.a + g.off_u;
    const T* f = S.a + g.off_f;
    const PlaneCoef<T>* cf = S.c + g.off_c;
    const int ncol = g.hx * g.nyi, nzi = g.nz - 2;
    const int tid = threadIdx.x + SX * threadIdx.y;
    for (int colour = 0; colour < 2; ++colour) {
        for (int q = tid; q < ncol; q += SX * blockDim.y) {
            const int jj = fdiv(q, g.inv_hx);
            const int t = q - jj * g.hx;
            const int j = 1 + jj;
            const int i = 1 + (((1 + j) & 1) != colour) + 2 * t;
            if (i > g.nx - 2) continue;
            int o = i + g.px * (j + g.ny);
            T dprev = T(0);
            for (int k = 1; k <= nzi; ++k, o += g.plane) {
                const PlaneCoef<T> c = cf[k];
                T v = f[o] - c.cx * (u[o + 1] + u[o - 1]) - c.cy * (u[o + g.px] + u[o - g.px]);
                if (k == 1) v -= c.cz * u[o - g.plane];
                if (k == nzi) v -= c.cz * u[o + g.plane];
                dprev = (v - c.cz * dprev) * c.lm;
                u[o] = dprev;
            }
            o -= g.plane;   // plane nzi: u = w there
            T unext = u[o];
            for (int k = nzi - 1; k >= 1; --k) {
                o -= g.plane;
                unext = u[o] - cf[k].lsup * unext;
                u[o] = unext;
            }
        }
        __syncthreads();
    }
}

template <typename T, bool D3>
__device__ __forceinline__ void sub_relax(const SubSmem<T, D3>& S, int l, int line) {
    if constexpr (D3) {
        if (line) {
            sub_zline<T>(S, l);
            return;
        }
    }
    sub_smooth<T, D3>(S, l);
}

// f[l+1] = full weighting of (f - A u) on level l; u[l+1] = 0 at interior nodes
template <typename T, bool D3>
__device__ void sub_restrict_residual(const SubSmem<T, D3>& S, int l) {
    const SubGeom gf = S.g[l], gc = S.g[l + 1];
    const T* u = S.a + gf.off_u;
    const T* f = S.a + gf.off_f;
    T* fc = S.a + gc.off_f;
    T* uc = S.a + gc.off_u;
    const PlaneCoef<T>* cf = S.c + gf.off_c;
    const int nw = gc.nxi * gc.nyi * (D3 ? gc.nz - 2 : 1);
    for (int q = threadIdx.x + SX * threadIdx.y; q < nw; q += SX * blockDim.y) {
        const int row = fdiv(q, gc.inv_nxi);
        const int I = 1 + q - row * gc.nxi;
        const int KK = D3 ? fdiv(row, gc.inv_nyi) : 0;
        const int J = 1 + row - KK * gc.nyi;
        const int K = D3 ? 1 + KK : 0;
        {
            T acc = T(0);
            for (int c3 = (D3 ? -1 : 0); c3 <= (D3 ? 1 : 0); ++c3) {
                const int k = D3 ? 2 * K + c3 : 0;
                const PlaneCoef<T> c = cf[k];
                T sb = T(0);
                for (int b = -1; b <= 1; ++b) {
                    const int o = 2 * I + gf.px * (2 * J + b + gf.ny * k);
                    const T r0 = f[o - 1] - sub_off<T, D3>(gf, c, u, o - 1) - c.d * u[o - 1];
                    const T r1 = f[o] - sub_off<T, D3>(gf, c, u, o) - c.d * u[o];
                    const T r2 = f[o + 1] - sub_off<T, D3>(gf, c, u, o + 1) - c.d * u[o + 1];
                    const T sa = T(0.25) * (r0 + r2) + T(0.5) * r1;
                    sb += (b == 0 ? T(0.5) : T(0.25)) * sa;
                }
                acc += (D3 ? (c3 == 0 ? T(0.5) : T(0.25)) : T(1)) * sb;
            }
            const int oc = I + gc.px * (J + gc.ny * K);
            fc[oc] = acc;
            uc[oc] = T(0);
        }
    }
    __syncthreads();
}

// u[l] += I u[l+1] at interior nodes
template <typename T, bool D3>
__device__ void sub_prolong(const SubSmem<T, D3>& S, int l) {
    const SubGeom gf = S.g[l], gc = S.g[l + 1];
    T* uf = S.a + gf.off_u;
    const T* uc = S.a + gc.off_u;
    const int nw = gf.nxi * gf.nyi * (D3 ? gf.nz - 2 : 1);
    for (int q = threadIdx.x + SX * threadIdx.y; q < nw; q += SX * blockDim.y) {
        const int row = fdiv(q, gf.inv_nxi);
        const int i = 1 + q - row * gf.nxi;
        const int kk = D3 ? fdiv(row, gf.inv_nyi) : 0;
        const int j = 1 + row - kk * gf.nyi;
        const int k = D3 ? 1 + kk : 0;
        const int J0 = j >> 1, J1 = (j + 1) >> 1, K0 = k >> 1, K1 = (k + 1) >> 1;
        {
            const int I0 = i >> 1, I1 = (i + 1) >> 1;
            auto pl = [&](int K) {
                const int b = gc.ny * K;
                return T(0.25) * ((uc[I0 + gc.px * (J0 + b)] + uc[I1 + gc.px * (J0 + b)]) +
                                  (uc[I0 + gc.px * (J1 + b)] + uc[I1 + gc.px * (J1 + b)]));
            };
            const T v = D3 ? T(0.5) * (pl(K0) + pl(K1)) : pl(0);
            uf[i + gf.px * (j + gf.ny * k)] += v;
        }
    }
    __syncthreads();
}

// sum of squares of (f - A u) (res = true) or of f over the interior of level l
template <typename T, bool D3>
__device__ double sub_norm2(const SubSmem<T, D3>& S, int l, bool res) {
    const SubGeom g = S.g[l];
    const T* u = S.a + g.off_u;
    const T* f = S.a + g.off_f;
    const PlaneCoef<T>* cf = S.c + g.off_c;
    const int nw = g.nxi * g.nyi * (D3 ? g.nz - 2 : 1);
    double a = 0.0;
    for (int q = threadIdx.x + SX * threadIdx.y; q < nw; q += SX * blockDim.y) {
        const int row = fdiv(q, g.inv_nxi);
        const int i = 1 + q - row * g.nxi;
        const int kk = D3 ? fdiv(row, g.inv_nyi) : 0;
        const int j = 1 + row - kk * g.nyi;
        const int k = D3 ? 1 + kk : 0;
        const PlaneCoef<T> c = cf[k];
        {
            const int o = i + g.px * (j + g.ny * k);
            const double v = res ? double(f[o] - sub_off<T, D3>(g, c, u, o) - c.d * u[o]) : double(f[o]);
            a += v * v;
        }
    }
    return block_sum(a);
}

// coarsest level: one exact update when it has a single unknown, else sweep
// until ||f - A u|| <= tol ||f|| (checked every 4 sweeps, at most 2000)
template <typename T, bool D3>
__device__ void sub_coarsest(const SubSmem<T, D3>& S, int l, int line) {
    const SubGeom g = S.g[l];
    const int nint = (g.nx - 2) * (g.ny - 2) * (D3 ? g.nz - 2 : 1);
    if (nint == 1) {
        sub_relax<T, D3>(S, l, line);
        return;
    }
    const double tol = sizeof(T) == 8 ? 1e-10 : 1e-5;
    __shared__ double s_fn;
    __shared__ int s_done;
    const double fn = sub_norm2<T, D3>(S, l, false);
    const int tid = threadIdx.x + SX * threadIdx.y;
    if (tid == 0) {
        s_fn = fn;
        s_done = fn == 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 2000 && !s_done; ++sweep) {
        sub_relax<T, D3>(S, l, line);
        if ((sweep & 3) == 3) {
            const double rr = sub_norm2<T, D3>(S, l, true);
            if (tid == 0) s_done = rr <= tol * tol * s_fn;
            __syncthreads();
        }
    }
}

template <typename T, bool D3>
__device__ __forceinline__ void subcycle_body(const SubParams<T>& p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SubGeom sg[MAX_SUB_LEVELS];
    const int tid = threadIdx.x + SX * threadIdx.y, nt = SX * blockDim.y;
    // layout: [coefficients of all levels][level arrays]
    PlaneCoef<T>* sc = reinterpret_cast<PlaneCoef<T>*>(smem_raw);
    int ncoef = 0;
    for (int l = 0; l < p.nlev; ++l) ncoef += p.L[l].g.nz;
    T* sa = reinterpret_cast<T*>(smem_raw + round_up(size_t(ncoef) * sizeof(PlaneCoef<T>), 16));
    if (tid < p.nlev) {
        const Geom& g = p.L[tid].g;
        int oc = 0;
        for (int m = 0; m < tid; ++m) oc += p.L[m].g.nz;
        const int nxi = g.nx - 2, nyi = g.ny - 2, hx = (nxi + 1) / 2;
        sg[tid] = SubGeom{g.nx, g.ny, g.nz, g.px, int(g.plane), int(g.n), p.L[tid].off_u, p.L[tid].off_f, oc,
                          nxi, nyi, hx, 1.0f / float(nxi), 1.0f / float(nyi), 1.0f / float(hx)};
    }
    for (int l = 0, oc = 0; l < p.nlev; oc += p.L[l].g.nz, ++l)
        for (int k = tid; k < p.L[l].g.nz; k += nt) sc[oc + k] = p.L[l].coef[k];
    {
        const Geom& g0 = p.L[0].g;
        T* u0 = sa + p.L[0].off_u;
        T* f0 = sa + p.L[0].off_f;
        for (size_t o = tid; o < g0.n; o += nt) {
            u0[o] = p.u_g[o];
            f0[o] = p.f_g[o];
        }
        for (int l = 1; l < p.nlev; ++l) {
            T* ul = sa + p.L[l].off_u;
            T* fl = sa + p.L[l].off_f;
            for (size_t o = tid; o < p.L[l].g.n; o += nt) {
                ul[o] = T(0);
                fl[o] = T(0);
            }
        }
    }
    __syncthreads();
    const SubSmem<T, D3> S{sa, sc, sg};
    for (int l = 0; l < p.nlev - 1; ++l) {
        for (int q = 0; q < p.nu1; ++q) sub_relax<T, D3>(S, l, p.line);
        sub_restrict_residual<T, D3>(S, l);
    }
    sub_coarsest<T, D3>(S, p.nlev - 1, p.line);
    for (int l = p.nlev - 2; l >= 0; --l) {
        sub_prolong<T, D3>(S, l);
        for (int q = 0; q < p.nu2; ++q) sub_relax<T, D3>(S, l, p.line);
    }
    const SubGeom g0 = sg[0];
    const T* u0 = sa + g0.off_u;
    const int nw = g0.nxi * g0.nyi * (D3 ? g0.nz - 2 : 1);
    for (int q = tid; q < nw; q += nt) {
        const int row = fdiv(q, g0.inv_nxi);
        const int i = 1 + q - row * g0.nxi;
        const int kk = D3 ? fdiv(row, g0.inv_nyi) : 0;
        const int j = 1 + row - kk * g0.nyi;
        const int k = D3 ? 1 + kk : 0;
        const int o = i + g0.px * (j + g0.ny * k);
        p.u_g[o] = u0[o];
    }
}


}  // namespace mhs
