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

// Per-plane constants: prof[8k + ...] = xi, xi', p_b, rho_b, xi/(2 mu0),
// xi'/(2 mu0 g), xi/(mu0 g).
// Generic (face) path for node (i,j,k): any position, one-sided stencils where needed.
__device__ void field_b_node(const Geom& g, double alpha, const double* __restrict__ prof, const double* __restrict__ P,
                             double* __restrict__ Bx, double* __restrict__ By, double* __restrict__ Bz,
                             double* __restrict__ p, int bz_mode, int i, int j, int k) {
    const size_t o = at(g, i, j, k);
    const double bx = alpha * D1(g, P, i, j, k, 1) + D1z_then(g, P, i, j, k, 0);
    const double by = -alpha * D1(g, P, i, j, k, 0) + D1z_then(g, P, i, j, k, 1);
    const double bz = bz_mode == 1 ? -(D1D1(g, P, i, j, k, 0) + D1D1(g, P, i, j, k, 1))
                                   : -(D2(g, P, i, j, k, 0) + D2(g, P, i, j, k, 1));
    Bx[o] = bx;
    By[o] = by;
    Bz[o] = bz;
    p[o] = fma(-prof[8 * k + 4], bz * bz, prof[8 * k + 2]);
}

__device__ void field_rho_node(const Geom& g, const double* __restrict__ prof, const double* __restrict__ Bx,
                               const double* __restrict__ By, const double* __restrict__ Bz, double* __restrict__ rho,
                               int i, int j, int k) {
    const size_t o = at(g, i, j, k);
    const double bz = Bz[o];
    const double bgb = fma(Bx[o], D1(g, Bz, i, j, k, 0), fma(By[o], D1(g, Bz, i, j, k, 1), bz * D1(g, Bz, i, j, k, 2)));
    rho[o] = fma(prof[8 * k + 5], bz * bz, fma(prof[8 * k + 6], bgb, prof[8 * k + 3]));
}

// Boundary nodes (the six faces), enumerated as a flat list so that every
// warp runs the generic path together: planes k = 0 and nz-1, then rows
// j = 0 and ny-1 of the inner planes, then columns i = 0 and nx-1 of the
// remaining nodes.
__device__ bool face_node(const Geom& g, long long q, int& i, int& j, int& k) {
    const long long pl = (long long)g.nx * g.ny;
    if (q < 2 * pl) {
        k = q < pl ? 0 : g.nz - 1;
        const long long r = q % pl;
        i = int(r % g.nx);
        j = int(r / g.nx);
        return true;
    }
    q -= 2 * pl;
    const long long rows = (long long)(g.nz - 2) * 2 * g.nx;
    if (q < rows) {
        k = 1 + int(q / (2 * g.nx));
        const int r = int(q % (2 * g.nx));
        j = r < g.nx ? 0 : g.ny - 1;
        i = r % g.nx;
        return true;
    }
    q -= rows;
    const long long cols = (long long)(g.nz - 2) * (g.ny - 2) * 2;
    if (q < cols) {
        k = 1 + int(q / (2 * (g.ny - 2)));
        const int r = int(q % (2 * (g.ny - 2)));
        j = 1 + r / 2;
        i = (r & 1) ? g.nx - 1 : 0;
        return true;
    }
    return false;
}

__global__ void field_b_face_kernel(Geom g, double alpha, const double* __restrict__ prof, const double* __restrict__ P,
                                    double* __restrict__ Bx, double* __restrict__ By, double* __restrict__ Bz,
                                    double* __restrict__ p, int bz_mode) {
    int i, j, k;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; face_node(g, q, i, j, k);
         q += (long long)gridDim.x * blockDim.x)
        field_b_node(g, alpha, prof, P, Bx, By, Bz, p, bz_mode, i, j, k);
}

__global__ void field_rho_face_kernel(Geom g, const double* __restrict__ prof, const double* __restrict__ Bx,
                                      const double* __restrict__ By, const double* __restrict__ Bz,
                                      double* __restrict__ rho) {
    int i, j, k;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; face_node(g, q, i, j, k);
         q += (long long)gridDim.x * blockDim.x)
        field_rho_node(g, prof, Bx, By, Bz, rho, i, j, k);
}

// Inner nodes (1 <= i, j, k <= n-2): fixed central stencils.  The
// difference weights come precomputed from the host (FieldWeights).
struct FieldWeights {
    double ax, ay;     // alpha/(2 hy), alpha/(2 hx): alpha dP/dy and alpha dP/dx
    double mxz, myz;   // 1/(4 hx hz), 1/(4 hy hz): mixed derivatives
    double cx, cy;     // 1/hx^2, 1/hy^2: compact second differences
    double dx, dy, dz; // 1/(2 h): central first differences of B_z
};

__global__ void field_b_kernel(Geom g, FieldWeights w, double alpha, const double* __restrict__ prof,
                               const double* __restrict__ P, double* __restrict__ Bx, double* __restrict__ By,
                               double* __restrict__ Bz, double* __restrict__ p, int bz_mode) {
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const ptrdiff_t sx = 1, sy = g.px, sz = (ptrdiff_t)g.plane;
    const double ax = w.ax, ay = w.ay, mxz = w.mxz, myz = w.myz, cx = w.cx, cy = w.cy;
    for (int k = 1 + blockIdx.z; k <= g.nz - 2; k += gridDim.z) {
        const size_t o = at(g, i, j, k);
        double bx, by, bz;
        if (bz_mode == 0) {
            const double* q = P + o;
            const double pxz = ((q[sx + sz] - q[sx - sz]) - (q[-sx + sz] - q[-sx - sz])) * mxz;
            const double pyz = ((q[sy + sz] - q[sy - sz]) - (q[-sy + sz] - q[-sy - sz])) * myz;
            bx = fma(ax, q[sy] - q[-sy], pxz);
            by = fma(-ay, q[sx] - q[-sx], pyz);
            const double c = q[0];
            bz = -fma(cx, fma(-2.0, c, q[sx] + q[-sx]), cy * fma(-2.0, c, q[sy] + q[-sy]));
        } else {
            field_b_node(g, alpha, prof, P, Bx, By, Bz, p, bz_mode, i, j, k);
            continue;
        }
        Bx[o] = bx;
        By[o] = by;
        Bz[o] = bz;
        p[o] = fma(-prof[8 * k + 4], bz * bz, prof[8 * k + 2]);
    }
}

__global__ void field_rho_kernel(Geom g, FieldWeights w, const double* __restrict__ prof, const double* __restrict__ Bx,
                                 const double* __restrict__ By, const double* __restrict__ Bz,
                                 double* __restrict__ rho) {
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const double dx = w.dx, dy = w.dy, dz = w.dz;
    for (int k = 1 + blockIdx.z; k <= g.nz - 2; k += gridDim.z) {
        const size_t o = at(g, i, j, k);
        const double bz = Bz[o];
        const double* q = Bz + o;
        const double gx = (q[1] - q[-1]) * dx;
        const double gy = (q[g.px] - q[-(ptrdiff_t)g.px]) * dy;
        const double gz = (q[g.plane] - q[-(ptrdiff_t)g.plane]) * dz;
        const double bgb = fma(Bx[o], gx, fma(By[o], gy, bz * gz));
        rho[o] = fma(prof[8 * k + 5], bz * bz, fma(prof[8 * k + 6], bgb, prof[8 * k + 3]));
    }
}

}  // namespace

void launch_fields(const Geom& g, double alpha, const mhs_atmos_params& atm, const double* prof, const double* P,
                   double* Bx, double* By, double* Bz, double* p, double* rho, int bz_mode, cudaStream_t st) {
    const dim3 blk(32, 8);
    // a few planes per thread so that per-thread set-up is amortised
    int gz = (g.nz - 2 + 3) / 4;
    if (gz > 65535) gz = 65535;
    FieldWeights w;
    w.ax = alpha / (2.0 * g.hy);
    w.ay = alpha / (2.0 * g.hx);
    w.mxz = 1.0 / (4.0 * g.hx * g.hz);
    w.myz = 1.0 / (4.0 * g.hy * g.hz);
    w.cx = 1.0 / (g.hx * g.hx);
    w.cy = 1.0 / (g.hy * g.hy);
    w.dx = 1.0 / (2.0 * g.hx);
    w.dy = 1.0 / (2.0 * g.hy);
    w.dz = 1.0 / (2.0 * g.hz);
    const dim3 grid((g.nx - 2 + 31) / 32, (g.ny - 2 + 7) / 8, gz);
    const long long faces = 2LL * g.nx * g.ny + 2LL * (g.nz - 2) * g.nx + 2LL * (g.nz - 2) * (g.ny - 2);
    const int fblocks = int((faces + 255) / 256 < 152 * 16 ? (faces + 255) / 256 : 152 * 16);
    (void)atm;
    field_b_kernel<<<grid, blk, 0, st>>>(g, w, alpha, prof, P, Bx, By, Bz, p, bz_mode);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    field_b_face_kernel<<<fblocks, 256, 0, st>>>(g, alpha, prof, P, Bx, By, Bz, p, bz_mode);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    field_rho_kernel<<<grid, blk, 0, st>>>(g, w, prof, Bx, By, Bz, rho);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    field_rho_face_kernel<<<fblocks, 256, 0, st>>>(g, prof, Bx, By, Bz, rho);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
