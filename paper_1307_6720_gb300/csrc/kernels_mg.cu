// Multigrid building blocks for the lower-boundary problem (eq. lower_bound,
// 5-point stencil) and the interior problem (eq. scalar_pot, 7-point stencil
// with per-plane coefficients), in FP64 and FP32.
//
// The paper parallelises every multigrid stage with one thread per node
// (Sect. 4: relaxation, residual, restriction and prolongation).  These are
// the plain per-node kernels of that design, adapted to red-black
// Gauss-Seidel; the fused sweeps live in kernels_sweep.cu and kernels_tma.cu,
// the z-line smoother in kernels_line.cu.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "device_util.cuh"
#include "line_body.cuh"
#include "mg_bodies.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

constexpr int BX = MG_BX, BY = MG_BY;

// -------------------------------------------------------------------------
// a1: per-plane coefficients and height profiles (Sect. 2.1, eq. scalar_pot;
// Sect. 3 background atmosphere and the xi families of Sect. 3.2).
// -------------------------------------------------------------------------

__device__ double xi_of(const mhs_xi_params& x, double z) {
    switch (x.kind) {
    case MHS_XI_EXP: return x.a * exp(-x.kappa * z);
    case MHS_XI_EXP_SIN: return (x.a + x.b * sin(x.omega * z)) * exp(-x.kappa * z);
    default: return 0.0;
    }
}

__device__ double dxi_of(const mhs_xi_params& x, double z) {
    switch (x.kind) {
    case MHS_XI_EXP: return -x.kappa * x.a * exp(-x.kappa * z);
    case MHS_XI_EXP_SIN:
        return (x.b * x.omega * cos(x.omega * z) - x.kappa * (x.a + x.b * sin(x.omega * z))) * exp(-x.kappa * z);
    default: return 0.0;
    }
}

__device__ void plane_coef(const Geom& g, int dim, double alpha, const mhs_xi_params& xi, int k, double& cx,
                           double& cy, double& cz, double& d) {
    if (dim == 3) {
        const double om = 1.0 - xi_of(xi, k * g.hz);
        cx = om / (g.hx * g.hx);
        cy = om / (g.hy * g.hy);
        cz = 1.0 / (g.hz * g.hz);
        d = -2.0 * (cx + cy + cz) + alpha * alpha;
    } else {
        cx = 1.0 / (g.hx * g.hx);
        cy = 1.0 / (g.hy * g.hy);
        cz = 0.0;
        d = -2.0 * (cx + cy);
    }
}

template <typename T>
__global__ void coef_kernel(Geom g, int dim, double alpha, mhs_xi_params xi, PlaneCoef<T>* coef) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nz) return;
    double cx, cy, cz, d;
    plane_coef(g, dim, alpha, xi, k, cx, cy, cz, d);
    coef[k] = PlaneCoef<T>{T(cx),     T(cy),     T(cz),     T(d), T(1.0 / d), T(cx / d),
                           T(cy / d), T(cz / d), T(0),      T(0), T(alpha * alpha - 2.0 * cz)};
}

// Elimination factors of the z-line smoother's column systems: the plane
// coefficients in FP64 by all threads of the block (into shared memory),
// then the pivot recursion over the interior planes by one thread; rounded
// to T at the end.  Levels have at most 1026 planes.  Also the factors of the
// partitioned column solve (line_body.cuh): one thread per segment forms the
// segment's pivots and its responses g = T_p^-1 e_first, h = T_p^-1 e_last to
// unit interface values, then one thread the interface system's factors.
template <typename T>
__global__ void line_coef_kernel(Geom g, double alpha, mhs_xi_params xi, PlaneCoef<T>* coef) {
    __shared__ double sd[1026], sg[1026], sh[1026];
    __shared__ double scz;
    for (int k = threadIdx.x; k < g.nz && k < 1026; k += blockDim.x) {
        double cx, cy, cz, d;
        plane_coef(g, 3, alpha, xi, k, cx, cy, cz, d);
        sd[k] = d;
        if (k == 0) scz = cz;
    }
    __syncthreads();
    const double cz = scz;
    const int n = min(g.nz - 2, 1024);
    const int S = zpart_segments(n), m = zpart_len(n, S);
    if (threadIdx.x == 0) {
        double sup = 0.0;
        for (int k = 1; k <= n; ++k) {
            const double lm = 1.0 / (sd[k] - (k > 1 ? cz * sup : 0.0));
            sup = cz * lm;
            coef[k].lm = T(lm);
            coef[k].lsup = T(sup);
        }
    }
    const int p = int(threadIdx.x) - 32;   // warp 1: one thread per segment
    if (p >= 0 && p < S) {
        const int a = 1 + p * (m + 1), e = min(a + m - 1, n);
        double lm[ZP_MMAX], sup[ZP_MMAX], wg[ZP_MMAX];
        for (int k = a; k <= e; ++k) {
            const int q = k - a;
            lm[q] = 1.0 / (sd[k] - (q > 0 ? cz * sup[q - 1] : 0.0));
            sup[q] = cz * lm[q];
            wg[q] = (q > 0 ? -cz * wg[q - 1] : 1.0) * lm[q];   // forward elimination of e_first
        }
        double gk = 0.0, hk = 0.0;
        for (int k = e; k >= a; --k) {
            const int q = k - a;
            gk = k == e ? wg[q] : wg[q] - sup[q] * gk;
            hk = k == e ? lm[q] : -sup[q] * hk;   // e_last: forward values vanish above the last row
            sg[k] = gk;
            sh[k] = hk;
            coef[k].zlm = T(lm[q]);
            coef[k].zsup = T(sup[q]);
            coef[k].zg = T(gk);
            coef[k].zh = T(hk);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && S > 1) {
        const double cz2 = cz * cz;
        double rsup = 0.0;
        for (int q = 1; q < S; ++q) {
            const int c = q * (m + 1);   // interface plane: last of segment q-1 below, first of segment q above
            const double L = q >= 2 ? -cz2 * sg[c - 1] : 0.0;
            const double D = sd[c] - cz2 * (sh[c - 1] + sg[c + 1]);
            const double U = q <= S - 2 ? -cz2 * sh[c + 1] : 0.0;
            const double rlm = 1.0 / (D - L * rsup);
            rsup = U * rlm;
            coef[c].zlm = T(rlm);
            coef[c].zsup = T(rsup);
            coef[c].zg = T(L);
            coef[c].zh = T(0);
        }
    }
}

// Background atmosphere: T_b piecewise (1, T_cor^((z-z1)/(z2-z1)), T_cor);
// p_b from dp_b/dz = -g p_b/T_b integrated in closed form per piece
// (1/T_b is constant or exponential in z); rho_b = p_b / T_b.
__device__ void background(const mhs_atmos_params& a, double z, double* pb, double* rhob) {
    const double d = a.z2 - a.z1, lnT = log(a.T_cor);
    double p, T;
    if (z <= a.z1) {
        p = exp(-a.g * z);
        T = 1.0;
    } else if (z <= a.z2) {
        const double s = (z - a.z1) / d;
        p = exp(-a.g * a.z1) * exp(-a.g * d * (1.0 - pow(a.T_cor, -s)) / lnT);
        T = pow(a.T_cor, s);
    } else {
        const double p2 = exp(-a.g * a.z1) * exp(-a.g * d * (1.0 - 1.0 / a.T_cor) / lnT);
        p = p2 * exp(-a.g * (z - a.z2) / a.T_cor);
        T = a.T_cor;
    }
    *pb = p;
    *rhob = p / T;
}

// per plane: xi, xi', p_b, rho_b and the folded field-recovery constants
// xi/(2 mu0) (eq. pressure), xi'/(2 mu0 g) and xi/(mu0 g) (eq. density)
__global__ void profile_kernel(Geom g, mhs_xi_params xi, mhs_atmos_params atm, double* prof) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nz) return;
    const double z = k * g.hz;
    double pb, rb;
    background(atm, z, &pb, &rb);
    const double x = xi_of(xi, z), dx = dxi_of(xi, z);
    prof[8 * k + 0] = x;
    prof[8 * k + 1] = dx;
    prof[8 * k + 2] = pb;
    prof[8 * k + 3] = rb;
    prof[8 * k + 4] = x / (2.0 * atm.mu0);
    prof[8 * k + 5] = dx / (2.0 * atm.mu0 * atm.g);
    prof[8 * k + 6] = x / (atm.mu0 * atm.g);
    prof[8 * k + 7] = 0.0;
}

template <typename T>
__global__ void fill_kernel(T* a, size_t n, T v) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) a[i] = v;
}

template <typename T, bool D3>
__global__ void colour_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef, T* __restrict__ u,
                              const T* __restrict__ f, int colour) {
    colour_body<T, D3>(g, coef, u, f, colour, blockIdx, gridDim);
}

__global__ void colour_v4_kernel(Geom g, const PlaneCoef<float>* __restrict__ coef, float* __restrict__ u,
                                 const float* __restrict__ f, int colour) {
    colour_body_v4(g, coef, u, f, colour, blockIdx, gridDim);
}

__global__ void residual_v4_kernel(Geom g, const PlaneCoef<float>* __restrict__ coef, const float* __restrict__ u,
                                   const float* __restrict__ f, float* __restrict__ r) {
    residual_body_v4(g, coef, u, f, r, blockIdx, gridDim);
}

template <typename T, bool D3, bool NORM>
__global__ void residual_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef, const T* __restrict__ u,
                                const T* __restrict__ f, T* __restrict__ r, double* __restrict__ partial) {
    residual_body<T, D3, NORM>(g, coef, u, f, r, partial, blockIdx, gridDim);
}

template <typename T, bool D3, bool NORM>
__global__ void residual_red_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef, const T* __restrict__ u,
                                    const T* __restrict__ f, T* __restrict__ r, double* __restrict__ partial) {
    residual_red_body<T, D3, NORM>(g, coef, u, f, r, partial, blockIdx, gridDim);
}

template <typename T, bool D3>
__global__ void __launch_bounds__(RR_THREADS) resid_restrict_kernel(Geom gf, Geom gc, const PlaneCoef<T>* __restrict__ coef,
                                                                   const T* __restrict__ u, const T* __restrict__ f,
                                                                   T* __restrict__ fc, T* __restrict__ uc) {
    resid_restrict_body<T, D3>(gf, gc, coef, u, f, fc, uc, blockIdx, gridDim);
}

__global__ void norm_finish_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    // one block, fixed summation order: thread t sums t, t+blockDim, ...; then a fixed tree
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

template <typename T, bool D3>
__global__ void restrict_kernel(Geom gf, Geom gc, const T* __restrict__ rf, T* __restrict__ fc, T* __restrict__ uc,
                                int red) {
    restrict_body<T, D3>(gf, gc, rf, fc, uc, blockIdx, gridDim, red != 0);
}

template <typename T, bool D3>
__global__ void prolong_kernel(Geom gc, Geom gf, const T* __restrict__ uc, T* __restrict__ uf) {
    prolong_body<T, D3>(gc, gf, uc, uf, blockIdx, gridDim);
}

// Coarsest level: one CTA sweeps red-black Gauss-Seidel in shared memory
// until ||f - A u|| <= tol_rel ||f|| (checked every 4 sweeps) or max_sweeps.
template <typename T, bool D3>
__global__ void coarse_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef, T* __restrict__ u_g,
                              const T* __restrict__ f_g, double tol_rel, int max_sweeps) {
    extern __shared__ unsigned char smem_raw[];
    T* u = reinterpret_cast<T*>(smem_raw);
    T* f = u + g.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (size_t o = tid; o < g.n; o += nt) {
        u[o] = u_g[o];
        f[o] = f_g[o];
    }
    __syncthreads();
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = D3 ? g.nz - 2 : 1;
    const int nint = nxi * nyi * nzi;
    auto node = [&](int q, int& i, int& j, int& k) {
        i = 1 + q % nxi;
        j = 1 + (q / nxi) % nyi;
        k = D3 ? 1 + q / (nxi * nyi) : 0;
    };
    auto au_off = [&](int i, int j, int k, const PlaneCoef<T>& c, size_t o) {
        T off = c.cx * (u[o + 1] + u[o - 1]) + c.cy * (u[o + g.px] + u[o - g.px]);
        if (D3) off += c.cz * (u[o + g.plane] + u[o - g.plane]);
        return off;
    };
    double fn = 0.0;
    for (int q = tid; q < nint; q += nt) {
        int i, j, k;
        node(q, i, j, k);
        const double v = f[at(g, i, j, k)];
        fn += v * v;
    }
    fn = block_sum(fn);
    __shared__ double s_fn;
    __shared__ int s_done;
    if (tid == 0) {
        s_fn = fn;
        s_done = (fn == 0.0);
    }
    __syncthreads();
    if (s_done) {
        for (size_t o = tid; o < g.n; o += nt) u_g[o] = T(0);
        return;
    }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int colour = 0; colour < 2; ++colour) {
            for (int q = tid; q < nint; q += nt) {
                int i, j, k;
                node(q, i, j, k);
                if (((i + j + k) & 1) != colour) continue;
                const PlaneCoef<T> c = coef[k];
                const size_t o = at(g, i, j, k);
                u[o] = (f[o] - au_off(i, j, k, c, o)) * c.inv_d;
            }
            __syncthreads();
        }
        if ((sweep & 3) == 3) {
            double rr = 0.0;
            for (int q = tid; q < nint; q += nt) {
                int i, j, k;
                node(q, i, j, k);
                const PlaneCoef<T> c = coef[k];
                const size_t o = at(g, i, j, k);
                const double rv = double(f[o] - au_off(i, j, k, c, o) - c.d * u[o]);
                rr += rv * rv;
            }
            rr = block_sum(rr);
            if (tid == 0) s_done = (rr <= tol_rel * tol_rel * s_fn);
            __syncthreads();
            if (s_done) break;
        }
    }
    for (size_t o = tid; o < g.n; o += nt) u_g[o] = u[o];
}

__global__ void lower_rhs_kernel(Geom g, const double* __restrict__ bz, double* __restrict__ f) {
    lower_rhs_body(g, bz, f, blockIdx);
}

template <typename T>
__global__ void zero_interior_kernel(Geom g, int d3, T* __restrict__ u) {
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    for (int k = d3 ? 1 + blockIdx.z : 0; k <= (d3 ? g.nz - 2 : 0); k += gridDim.z) u[at(g, i, j, k)] = T(0);
}

__global__ void copy_plane_kernel(Geom g2, const double* __restrict__ src, Geom g3, double* __restrict__ dst) {
    copy_plane_body(g2, src, g3, dst, blockIdx);
}

// dst = src on the six boundary faces of a 3D level (face nodes enumerated:
// the planes k = 0 and nz - 1, then the rows j = 0 and ny - 1 of the other
// planes, then the columns i = 0 and nx - 1 of the remaining rows)
template <typename T>
__global__ void copy_faces_kernel(Geom g, const T* __restrict__ src, T* __restrict__ dst) {
    const long long nxy = (long long)g.nx * g.ny, nxz = (long long)g.nx * (g.nz - 2),
                    nyz = (long long)(g.ny - 2) * (g.nz - 2);
    const long long total = 2 * (nxy + nxz + nyz);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (e < 2 * nxy) {
            const long long q = e % nxy;
            k = e < nxy ? 0 : g.nz - 1;
            j = int(q / g.nx);
            i = int(q - (long long)j * g.nx);
        } else if (e < 2 * (nxy + nxz)) {
            const long long q = (e - 2 * nxy) % nxz;
            j = e - 2 * nxy < nxz ? 0 : g.ny - 1;
            k = 1 + int(q / g.nx);
            i = int(q - (long long)(k - 1) * g.nx);
        } else {
            const long long r = e - 2 * (nxy + nxz);
            const long long q = r % nyz;
            i = r < nyz ? 0 : g.nx - 1;
            k = 1 + int(q / (g.ny - 2));
            j = 1 + int(q - (long long)(k - 1) * (g.ny - 2));
        }
        const size_t o = at(g, i, j, k);
        dst[o] = src[o];
    }
}

__global__ void nonfinite_kernel(Geom g, const double* __restrict__ bz, int* flag) {
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    if (!isfinite(bz[at(g, i, j, 0)])) atomicExch(flag, 1);
}

__global__ void lift_norm_kernel(Geom g, const PlaneCoef<double>* __restrict__ coef, const double* __restrict__ u,
                                 double* __restrict__ partial) {
    lift_norm_body(g, coef, u, partial, blockIdx, gridDim);
}

dim3 grid_for(const Geom& g, int d3, int xcount, int max_blocks) { return mg_grid(g, d3, xcount, max_blocks); }


}  // namespace

// ------------------------------- launchers -------------------------------

template <typename T>
void launch_coef(const Geom& g, int dim, double alpha, const mhs_xi_params& xi, PlaneCoef<T>* coef,
                 cudaStream_t st) {
    coef_kernel<T><<<(g.nz + 127) / 128, 128, 0, st>>>(g, dim, alpha, xi, coef);
    count_launches(1);
    if (dim == 3 && g.nz > 2) {
        line_coef_kernel<T><<<1, 256, 0, st>>>(g, alpha, xi, coef);
        count_launches(1);
    }
    MHS_CUDA(cudaGetLastError());
}

void launch_profiles(const Geom& g, const mhs_xi_params& xi, const mhs_atmos_params& atm, double* prof,
                     cudaStream_t st) {
    profile_kernel<<<(g.nz + 127) / 128, 128, 0, st>>>(g, xi, atm, prof);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_fill(T* a, size_t n, T v, cudaStream_t st) {
    if (n == 0) return;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    fill_kernel<T><<<unsigned(blocks), 256, 0, st>>>(a, n, v);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_smooth(const Geom& g, int dim, const PlaneCoef<T>* coef, T* u, const T* f, cudaStream_t st, int tile) {
    const int d3 = dim == 3;
    const dim3 blk = tile_block(tile);
    if constexpr (sizeof(T) == 4) {
        if (d3 && use_v4(g)) {
            const dim3 grid = tile_grid(g, 1, (g.nx - 2) / 4 + 1, blk);
            for (int colour = 0; colour < 2; ++colour) {
                colour_v4_kernel<<<grid, blk, 0, st>>>(g, coef, u, f, colour);
                count_launches(1);
            }
            MHS_CUDA(cudaGetLastError());
            return;
        }
    }
    const dim3 grid = tile_grid(g, d3, (g.nx - 2 + 1) / 2, blk);
    for (int colour = 0; colour < 2; ++colour) {
        if (d3) colour_kernel<T, true><<<grid, blk, 0, st>>>(g, coef, u, f, colour);
        else colour_kernel<T, false><<<grid, blk, 0, st>>>(g, coef, u, f, colour);
        count_launches(1);
    }
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
int launch_residual(const Geom& g, int dim, const PlaneCoef<T>* coef, const T* u, const T* f, T* r, double* partial,
                    int max_blocks, cudaStream_t st, bool red) {
    const int d3 = dim == 3;
    if (red) {   // right after a red-black sweep: red nodes computed, black nodes 0
        const dim3 grid = residual_red_grid(g, d3, partial != nullptr, max_blocks);
        if (partial) {
            if (d3) residual_red_kernel<T, true, true><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
            else residual_red_kernel<T, false, true><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
        } else {
            if (d3) residual_red_kernel<T, true, false><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
            else residual_red_kernel<T, false, false><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
        }
        count_launches(1);
        MHS_CUDA(cudaGetLastError());
        return int(grid.x * grid.y * grid.z);
    }
    // with norm partials, few enough blocks (a multiple of the SM count) that
    // the fixed-order finish stays short; every thread then covers several planes
    if constexpr (sizeof(T) == 4) {
        if (d3 && !partial && use_v4(g)) {
            residual_v4_kernel<<<quad_grid(g), dim3(BX, BY), 0, st>>>(g, coef, u, f, r);
            count_launches(1);
            MHS_CUDA(cudaGetLastError());
            return int(quad_grid(g).x * quad_grid(g).y * quad_grid(g).z);
        }
    }
    const dim3 grid = residual_grid(g, d3, partial != nullptr, max_blocks);
    if (partial) {
        if (d3) residual_kernel<T, true, true><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
        else residual_kernel<T, false, true><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
    } else {
        if (d3) residual_kernel<T, true, false><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
        else residual_kernel<T, false, false><<<grid, dim3(BX, BY), 0, st>>>(g, coef, u, f, r, partial);
    }
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    return int(grid.x * grid.y * grid.z);
}

template <typename T>
void launch_resid_restrict(const Geom& gf, const Geom& gc, int dim, const PlaneCoef<T>* coef, const T* u, const T* f,
                           T* fc, T* uc, cudaStream_t st) {
    const int d3 = dim == 3;
    const dim3 grid = resid_restrict_grid(gc, d3);
    if (d3) resid_restrict_kernel<T, true><<<grid, RR_THREADS, 0, st>>>(gf, gc, coef, u, f, fc, uc);
    else resid_restrict_kernel<T, false><<<grid, RR_THREADS, 0, st>>>(gf, gc, coef, u, f, fc, uc);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_norm_finish(const double* partial, int n, double* out, cudaStream_t st) {
    norm_finish_kernel<<<1, 1024, 0, st>>>(partial, n, out);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_restrict(const Geom& gf, const Geom& gc, int dim, const T* rf, T* fc, T* uc_zero, cudaStream_t st,
                     bool red) {
    const int d3 = dim == 3;
    const dim3 grid = restrict_grid(gc, d3);
    if (d3) restrict_kernel<T, true><<<grid, dim3(BX, BY), 0, st>>>(gf, gc, rf, fc, uc_zero, red ? 1 : 0);
    else restrict_kernel<T, false><<<grid, dim3(BX, BY), 0, st>>>(gf, gc, rf, fc, uc_zero, red ? 1 : 0);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_prolong(const Geom& gc, const Geom& gf, int dim, const T* uc, T* uf, cudaStream_t st) {
    const int d3 = dim == 3;
    const dim3 grid = prolong_grid(gc, d3);   // one thread per coarse cell
    if (d3) prolong_kernel<T, true><<<grid, dim3(BX, BY), 0, st>>>(gc, gf, uc, uf);
    else prolong_kernel<T, false><<<grid, dim3(BX, BY), 0, st>>>(gc, gf, uc, uf);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_coarse(const Geom& g, int dim, const PlaneCoef<T>* coef, T* u, const T* f, cudaStream_t st) {
    const size_t smem = 2 * g.n * sizeof(T);
    const double tol = sizeof(T) == 8 ? 1e-13 : 1e-6;
    const int max_sweeps = 4000;
    if (dim == 3) {
        MHS_CUDA(cudaFuncSetAttribute(coarse_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        coarse_kernel<T, true><<<1, 512, smem, st>>>(g, coef, u, f, tol, max_sweeps);
        count_launches(1);
    } else {
        MHS_CUDA(cudaFuncSetAttribute(coarse_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        coarse_kernel<T, false><<<1, 512, smem, st>>>(g, coef, u, f, tol, max_sweeps);
        count_launches(1);
    }
    MHS_CUDA(cudaGetLastError());
}

void launch_lower_rhs(const Geom& g, const double* bz, double* f64, cudaStream_t st) {
    const dim3 grid = grid_for(g, 0, g.nx - 2, 0);
    lower_rhs_kernel<<<grid, dim3(BX, BY), 0, st>>>(g, bz, f64);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_zero_interior(const Geom& g, int dim, T* u, cudaStream_t st) {
    const int d3 = dim == 3;
    const dim3 grid = grid_for(g, d3, g.nx - 2, 0);
    zero_interior_kernel<T><<<grid, dim3(BX, BY), 0, st>>>(g, d3, u);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_copy_plane(const Geom& g2, const double* src2d, const Geom& g3, double* dst3d, cudaStream_t st) {
    const dim3 grid = plane_grid(g2);
    copy_plane_kernel<<<grid, dim3(BX, BY), 0, st>>>(g2, src2d, g3, dst3d);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_copy_faces(const Geom& g, const T* src, T* dst, cudaStream_t st) {
    const long long total = 2 * ((long long)g.nx * g.ny + (long long)g.nx * (g.nz - 2) + (long long)(g.ny - 2) * (g.nz - 2));
    const int blocks = int(std::min<long long>((total + 255) / 256, 152 * 4));
    copy_faces_kernel<T><<<blocks, 256, 0, st>>>(g, src, dst);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_count_nonfinite(const Geom& g, const double* bz, int* flag, cudaStream_t st) {
    const dim3 grid = grid_for(g, 0, g.nx - 2, 0);
    nonfinite_kernel<<<grid, dim3(BX, BY), 0, st>>>(g, bz, flag);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

int launch_lift_norm(const Geom& g3, const PlaneCoef<double>* coef, const double* u, double* partial,
                     cudaStream_t st) {
    const dim3 grid = lift_grid(g3);
    lift_norm_kernel<<<grid, dim3(BX, BY), 0, st>>>(g3, coef, u, partial);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    return int(grid.x * grid.y);
}

#define MHS_INST(T)                                                                                          \
    template void launch_coef<T>(const Geom&, int, double, const mhs_xi_params&, PlaneCoef<T>*, cudaStream_t); \
    template void launch_fill<T>(T*, size_t, T, cudaStream_t);                                                 \
    template void launch_smooth<T>(const Geom&, int, const PlaneCoef<T>*, T*, const T*, cudaStream_t, int);    \
    template int launch_residual<T>(const Geom&, int, const PlaneCoef<T>*, const T*, const T*, T*, double*,    \
                                    int, cudaStream_t, bool);                                                  \
    template void launch_restrict<T>(const Geom&, const Geom&, int, const T*, T*, T*, cudaStream_t, bool);           \
    template void launch_resid_restrict<T>(const Geom&, const Geom&, int, const PlaneCoef<T>*, const T*, const T*, \
                                           T*, T*, cudaStream_t);                                                 \
    template void launch_prolong<T>(const Geom&, const Geom&, int, const T*, T*, cudaStream_t);                \
    template void launch_coarse<T>(const Geom&, int, const PlaneCoef<T>*, T*, const T*, cudaStream_t);         \
    template void launch_zero_interior<T>(const Geom&, int, T*, cudaStream_t);                                \
    template void launch_copy_faces<T>(const Geom&, const T*, T*, cudaStream_t);
MHS_INST(double)
MHS_INST(float)
#undef MHS_INST

}  // namespace mhs

namespace mhs {
namespace {
__global__ void d2f_kernel(const double* __restrict__ s, float* __restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        d[i] = float(s[i]);
}
__global__ void f2d_kernel(const float* __restrict__ s, double* __restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        d[i] = double(s[i]);
}
// rows of nx doubles at pitch px -> dense rows (a row per block-stride step)
__global__ void pack_kernel(const double* __restrict__ s, double* __restrict__ d, int nx, int px, size_t rows) {
    for (size_t r = blockIdx.x; r < rows; r += gridDim.x)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) d[r * nx + i] = s[r * px + i];
}
}  // namespace
void launch_pack(const double* src, double* dst, int nx, int px, size_t rows, cudaStream_t st) {
    if (rows == 0) return;
    const unsigned blocks = unsigned(rows < 152 * 16 ? rows : 152 * 16);
    pack_kernel<<<blocks, 128, 0, st>>>(src, dst, nx, px, rows);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_d2f(const double* src, float* dst, size_t n, cudaStream_t st) {
    d2f_kernel<<<152 * 8, 256, 0, st>>>(src, dst, n);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}
void launch_f2d(const float* src, double* dst, size_t n, cudaStream_t st) {
    f2d_kernel<<<152 * 8, 256, 0, st>>>(src, dst, n);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}
}  // namespace mhs
