// Post-processing of an equilibrium: the quantities the paper's figures show
// (Sect. 3): current density j = curl B / mu0 with its magnitude, |B|, and
// magnetic field lines.
//
// current_kernel: one thread per node, the difference operators of the
// field recovery (central inside, second-order one-sided at the first and
// last node of an axis), FP64.
//
// trace_kernel: one thread per seed; classical fourth-order Runge-Kutta
// along dr/ds = dir B/|B| with B interpolated trilinearly (x, then y, then
// z) from the nodes of the cell holding the point.  A step is taken only
// when its four stage points and its end point lie in the closed box and
// |B| does not vanish at the stage points; otherwise the line ends.  All
// arithmetic uses explicitly rounded FP64 operations (no fused
// multiply-add), in a fixed order, so that a line depends only on B and the
// seed, not on how the compiler schedules the arithmetic.
#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int BX = 32, BY = 8;

// d/dx_a at node t of n along one axis, element stride s
__device__ __forceinline__ double dif1(const double* __restrict__ f, size_t c, size_t s, int t, int n, double inv2h) {
    if (t == 0) return (-3.0 * f[c] + 4.0 * f[c + s] - f[c + 2 * s]) * inv2h;
    if (t == n - 1) return (3.0 * f[c] - 4.0 * f[c - s] + f[c - 2 * s]) * inv2h;
    return (f[c + s] - f[c - s]) * inv2h;
}

__global__ void current_kernel(Geom g, double inv_mu0, const double* __restrict__ Bx, const double* __restrict__ By,
                               const double* __restrict__ Bz, double* __restrict__ jx, double* __restrict__ jy,
                               double* __restrict__ jz, double* __restrict__ jmag, double* __restrict__ bmag) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double ix = 0.5 / g.hx, iy = 0.5 / g.hy, iz = 0.5 / g.hz;
    const size_t sy = g.px, sz = g.plane;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const size_t c = at(g, i, j, k);
        const double cx = (dif1(Bz, c, sy, j, g.ny, iy) - dif1(By, c, sz, k, g.nz, iz)) * inv_mu0;
        const double cy = (dif1(Bx, c, sz, k, g.nz, iz) - dif1(Bz, c, 1, i, g.nx, ix)) * inv_mu0;
        const double cz = (dif1(By, c, 1, i, g.nx, ix) - dif1(Bx, c, sy, j, g.ny, iy)) * inv_mu0;
        if (jx) jx[c] = cx;
        if (jy) jy[c] = cy;
        if (jz) jz[c] = cz;
        if (jmag) jmag[c] = sqrt(cx * cx + cy * cy + cz * cz);
        if (bmag) bmag[c] = sqrt(Bx[c] * Bx[c] + By[c] * By[c] + Bz[c] * Bz[c]);
    }
}

struct TraceGeom {
    int n[3];
    double L[3];
    size_t px, plane;   // element strides of the B arrays along y and z
};

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }

// dir * B/|B| at r; false outside the closed box or where |B| = 0
__device__ bool trace_dir(const TraceGeom& G, const double* __restrict__ Bx, const double* __restrict__ By,
                          const double* __restrict__ Bz, double dir, const double r[3], double v[3]) {
    int c[3];
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(r[a] >= 0.0 && r[a] <= G.L[a])) return false;
        const double h = __ddiv_rn(G.L[a], double(G.n[a] - 1));
        const double s = __ddiv_rn(r[a], h);
        int i = int(floor(s));
        if (i > G.n[a] - 2) i = G.n[a] - 2;
        if (i < 0) i = 0;
        c[a] = i;
        f[a] = sub(s, double(i));
    }
    const double* B[3] = {Bx, By, Bz};
    double b[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double* F = B[q];
        double e[2][2];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const size_t o = size_t(c[0]) + G.px * size_t(c[1] + dy) + G.plane * size_t(c[2] + dz);
                e[dz][dy] = add(mul(F[o], sub(1.0, f[0])), mul(F[o + 1], f[0]));
            }
        const double e0 = add(mul(e[0][0], sub(1.0, f[1])), mul(e[0][1], f[1]));
        const double e1 = add(mul(e[1][0], sub(1.0, f[1])), mul(e[1][1], f[1]));
        b[q] = add(mul(e0, sub(1.0, f[2])), mul(e1, f[2]));
    }
    const double m = __dsqrt_rn(add(add(mul(b[0], b[0]), mul(b[1], b[1])), mul(b[2], b[2])));
    if (!(m > 0.0)) return false;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = __ddiv_rn(mul(dir, b[q]), m);
    return true;
}

__global__ void trace_kernel(TraceGeom G, const double* __restrict__ Bx, const double* __restrict__ By,
                             const double* __restrict__ Bz, const double* __restrict__ seeds, int n, double ds,
                             int max_steps, double dir, double* __restrict__ points, int* __restrict__ lengths) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double r[3] = {seeds[3 * size_t(q)], seeds[3 * size_t(q) + 1], seeds[3 * size_t(q) + 2]};
    double* out = points + size_t(q) * size_t(max_steps + 1) * 3;
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) inside = inside && r[a] >= 0.0 && r[a] <= G.L[a];
    if (!inside) {
        lengths[q] = 0;
        return;
    }
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
    int len = 1;
    const double hs = mul(0.5, ds), s6 = __ddiv_rn(ds, 6.0);
    for (int step = 0; step < max_steps; ++step) {
        double k1[3], k2[3], k3[3], k4[3], t[3], e[3];
        if (!trace_dir(G, Bx, By, Bz, dir, r, k1)) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = add(r[a], mul(hs, k1[a]));
        if (!trace_dir(G, Bx, By, Bz, dir, t, k2)) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = add(r[a], mul(hs, k2[a]));
        if (!trace_dir(G, Bx, By, Bz, dir, t, k3)) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = add(r[a], mul(ds, k3[a]));
        if (!trace_dir(G, Bx, By, Bz, dir, t, k4)) break;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            e[a] = add(r[a], mul(s6, add(add(add(k1[a], mul(2.0, k2[a])), mul(2.0, k3[a])), k4[a])));
            ok = ok && e[a] >= 0.0 && e[a] <= G.L[a];
        }
        if (!ok) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[a] = e[a];
            out[3 * size_t(len) + a] = e[a];
        }
        ++len;
    }
    lengths[q] = len;
}

}  // namespace

void launch_current(const Geom& g, double mu0, const double* Bx, const double* By, const double* Bz, double* jx,
                    double* jy, double* jz, double* jmag, double* bmag, cudaStream_t st) {
    int gz = g.nz;
    const int tiles = ((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY);
    if (gz * tiles > 152 * 16) gz = std::max(1, 152 * 16 / tiles);
    const dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, gz);
    current_kernel<<<grid, dim3(BX, BY), 0, st>>>(g, 1.0 / mu0, Bx, By, Bz, jx, jy, jz, jmag, bmag);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_trace(int nx, int ny, int nz, double Lx, double Ly, double Lz, size_t px, size_t plane, const double* Bx,
                  const double* By, const double* Bz, const double* seeds, int n, double ds, int max_steps,
                  double dir, double* points, int* lengths, cudaStream_t st) {
    if (n <= 0) return;
    TraceGeom G{{nx, ny, nz}, {Lx, Ly, Lz}, px, plane};
    trace_kernel<<<(n + 63) / 64, 64, 0, st>>>(G, Bx, By, Bz, seeds, n, ds, max_steps, dir, points, lengths);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
