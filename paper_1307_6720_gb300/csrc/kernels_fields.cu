// Field recovery (Sect. 2.2, eqs. b_iden, t, pressure, density), FP64.
//
//   B_x = alpha dP/dy + d2P/dxdz,  B_y = -alpha dP/dx + d2P/dydz,
//   B_z = -(d2P/dx2 + d2P/dy2),
//   p   = p_b(z) - xi(z) B_z^2 / (2 mu0),
//   rho = rho_b(z) + [xi'(z) B_z^2/(2 mu0) + xi(z) B.grad(B_z) / mu0] / g.
//
// Derivatives are second-order finite differences: central at inner nodes,
// one-sided three-point (first derivative) and four-point (second
// derivative) stencils on the first and last node of an axis; the mixed
// derivative applies the first-derivative operator along x (or y) to the
// first derivative along z.  B_z takes the compact three-point second
// difference (the operator of eq. lower_bound) or, with bz_mode = 1, the
// first-difference operator applied twice.
#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

struct St {
    int off[4];
    double w[4];
    int n;
};

// first derivative at position t of an axis of n nodes with spacing h
__device__ __forceinline__ St d1(int t, int n, double h) {
    const double a = 1.0 / (2.0 * h);
    if (t == 0) return St{{0, 1, 2, 0}, {-3.0 * a, 4.0 * a, -a, 0.0}, 3};
    if (t == n - 1) return St{{0, -1, -2, 0}, {3.0 * a, -4.0 * a, a, 0.0}, 3};
    return St{{-1, 1, 0, 0}, {-a, a, 0.0, 0.0}, 2};
}

// second derivative (compact)
__device__ __forceinline__ St d2(int t, int n, double h) {
    const double a = 1.0 / (h * h);
    if (t == 0) return St{{0, 1, 2, 3}, {2.0 * a, -5.0 * a, 4.0 * a, -a}, 4};
    if (t == n - 1) return St{{0, -1, -2, -3}, {2.0 * a, -5.0 * a, 4.0 * a, -a}, 4};
    return St{{-1, 0, 1, 0}, {a, -2.0 * a, a, 0.0}, 3};
}

// d/dx_a applied along axis a (0,1,2) of array f at (i,j,k)
__device__ double D1(const Geom& g, const double* f, int i, int j, int k, int a) {
    const int t = a == 0 ? i : a == 1 ? j : k;
    const int n = a == 0 ? g.nx : a == 1 ? g.ny : g.nz;
    const double h = a == 0 ? g.hx : a == 1 ? g.hy : g.hz;
    const ptrdiff_t s = a == 0 ? 1 : a == 1 ? (ptrdiff_t)g.px : (ptrdiff_t)g.plane;
    const St st = d1(t, n, h);
    const size_t o = at(g, i, j, k);
    double v = 0.0;
    for (int q = 0; q < st.n; ++q) v += st.w[q] * f[o + st.off[q] * s];
    return v;
}

__device__ double D2(const Geom& g, const double* f, int i, int j, int k, int a) {
    const int t = a == 0 ? i : j;
    const int n = a == 0 ? g.nx : g.ny;
    const double h = a == 0 ? g.hx : g.hy;
    const ptrdiff_t s = a == 0 ? 1 : (ptrdiff_t)g.px;
    const St st = d2(t, n, h);
    const size_t o = at(g, i, j, k);
    double v = 0.0;
    for (int q = 0; q < st.n; ++q) v += st.w[q] * f[o + st.off[q] * s];
    return v;
}

// mixed derivative: D1 along axis a (x or y) of D1 along z
__device__ double D1z_then(const Geom& g, const double* P, int i, int j, int k, int a) {
    const int t = a == 0 ? i : j;
    const int n = a == 0 ? g.nx : g.ny;
    const double h = a == 0 ? g.hx : g.hy;
    const St st = d1(t, n, h);
    double v = 0.0;
    for (int q = 0; q < st.n; ++q) {
        const int ii = a == 0 ? i + st.off[q] : i;
        const int jj = a == 1 ? j + st.off[q] : j;
        v += st.w[q] * D1(g, P, ii, jj, k, 2);
    }
    return v;
}

// D1 along axis a applied twice (the mimetic B_z option)
__device__ double D1D1(const Geom& g, const double* P, int i, int j, int k, int a) {
    const int t = a == 0 ? i : j;
    const int n = a == 0 ? g.nx : g.ny;
    const double h = a == 0 ? g.hx : g.hy;
    const St st = d1(t, n, h);
    double v = 0.0;
    for (int q = 0; q < st.n; ++q) {
        const int ii = a == 0 ? i + st.off[q] : i;
        const int jj = a == 1 ? j + st.off[q] : j;
        v += st.w[q] * D1(g, P, ii, jj, k, a);
    }
    return v;
}

__global__ void field_b_kernel(Geom g, double alpha, double inv2mu0, const double* __restrict__ prof,
                               const double* __restrict__ P, double* __restrict__ Bx, double* __restrict__ By,
                               double* __restrict__ Bz, double* __restrict__ p, int bz_mode) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const size_t o = at(g, i, j, k);
        const double bx = alpha * D1(g, P, i, j, k, 1) + D1z_then(g, P, i, j, k, 0);
        const double by = -alpha * D1(g, P, i, j, k, 0) + D1z_then(g, P, i, j, k, 1);
        const double bz = bz_mode == 1 ? -(D1D1(g, P, i, j, k, 0) + D1D1(g, P, i, j, k, 1))
                                       : -(D2(g, P, i, j, k, 0) + D2(g, P, i, j, k, 1));
        Bx[o] = bx;
        By[o] = by;
        Bz[o] = bz;
        p[o] = prof[4 * k + 2] - prof[4 * k + 0] * bz * bz * inv2mu0;
    }
}

__global__ void field_rho_kernel(Geom g, double inv2mu0, double invmu0, double invg, const double* __restrict__ prof,
                                 const double* __restrict__ Bx, const double* __restrict__ By,
                                 const double* __restrict__ Bz, double* __restrict__ rho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const size_t o = at(g, i, j, k);
        const double bz = Bz[o];
        const double bgb = Bx[o] * D1(g, Bz, i, j, k, 0) + By[o] * D1(g, Bz, i, j, k, 1) + bz * D1(g, Bz, i, j, k, 2);
        const double xi = prof[4 * k + 0], dxi = prof[4 * k + 1], rb = prof[4 * k + 3];
        rho[o] = rb + (dxi * bz * bz * inv2mu0 + xi * bgb * invmu0) * invg;
    }
}

}  // namespace

void launch_fields(const Geom& g, double alpha, const mhs_atmos_params& atm, const double* prof, const double* P,
                   double* Bx, double* By, double* Bz, double* p, double* rho, int bz_mode, cudaStream_t st) {
    const dim3 blk(32, 8);
    int gz = g.nz;
    if (gz > 65535) gz = 65535;
    const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, gz);
    const double inv2mu0 = 1.0 / (2.0 * atm.mu0);
    field_b_kernel<<<grid, blk, 0, st>>>(g, alpha, inv2mu0, prof, P, Bx, By, Bz, p, bz_mode);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    field_rho_kernel<<<grid, blk, 0, st>>>(g, inv2mu0, 1.0 / atm.mu0, 1.0 / atm.g, prof, Bx, By, Bz, rho);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
