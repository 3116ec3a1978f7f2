// Per-block body of the zebra z-line Gauss-Seidel pass (kernels_line.cu),
// with an explicit block index for grouped launches (see mg_bodies.cuh).
//
// Zebra z-line Gauss-Seidel: the line-relaxation form of the smoother for
// the interior operator of eq. (scalar_pot) when the vertical coupling is
// strong ([1 - xi(z)] small, or h_z < h_x), where point red-black
// Gauss-Seidel smooths poorly.
//
// The columns (i, j) are coloured by the parity of i + j; a pass solves, for
// every column of one colour, the nz - 2 interior rows of A u = f along the
// column exactly, the neighbouring columns (the other colour) and the
// Dirichlet ends held fixed:
//   cz u[k-1] + d[k] u[k] + cz u[k+1] = f[k] - cx[k] (u_E + u_W) - cy[k] (u_N + u_S).
// Gaussian elimination without pivoting (the Thomas algorithm): -A is
// symmetric positive definite, so no pivot vanishes.  The pivots do not
// depend on the column, so their reciprocals lm and the eliminated
// super-diagonal lsup = cz lm are precomputed once per level (PlaneCoef).
//
// One thread per column.  The forward sweep stores the eliminated right-hand
// side in a scratch array laid out by (column of the colour, plane), so
// that a warp writes and reads it in consecutive words; the back
// substitution overwrites u.  Loads of U planes are issued together so that
// several memory round trips overlap along the sequential recursion; the
// neighbour columns (the other colour) are not written by the pass, so they
// are read through the read-only data path.
#pragma once

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

constexpr int LX = 32, LY = 2, MAXZ = 1026;   // block shape; most planes per level

// coefficients the line solve needs, per plane, staged in shared memory
template <typename T>
struct LineCoef {
    T cx, cy, lm, lsup;
};

// U planes at a time: all loads of a chunk are issued before the recursion
// consumes them, so U memory round trips overlap.  Full chunks run without
// guards; the last, partial chunk one plane at a time.
template <typename T, int U>
__device__ __forceinline__ void zline_body(const Geom& g, const PlaneCoef<T>* __restrict__ coef, T* __restrict__ u,
                                           const T* __restrict__ f, T* __restrict__ w, int colour, int hx, dim3 b) {
    __shared__ LineCoef<T> sc[MAXZ];
    const int nzi = g.nz - 2;
    for (int k = threadIdx.x + LX * threadIdx.y; k <= nzi; k += LX * LY) {
        const PlaneCoef<T> c = coef[k];
        sc[k] = LineCoef<T>{c.cx, c.cy, c.lm, c.lsup};
    }
    const T cz = coef[1].cz;
    __syncthreads();
    const int t = b.x * LX + threadIdx.x;
    const int jj = b.y * LY + threadIdx.y;
    const int nyi = g.ny - 2;
    if (t >= hx || jj >= nyi) return;
    const int j = 1 + jj;
    const int i = 1 + ((1 + j + colour) & 1) + 2 * t;   // (i + j) & 1 == colour
    if (i > g.nx - 2) return;
    const size_t plane = g.plane;
    const size_t wplane = size_t(hx) * nyi;
    const T* __restrict__ uc = u + at(g, i, j, 1);         // this column at plane 1
    const T* __restrict__ fc = f ? f + at(g, i, j, 1) : nullptr;
    T* __restrict__ wc = w + t + size_t(hx) * jj;           // this column's scratch, stride wplane
    const int px = g.px;
    const T u_bot = __ldg(uc - plane);                      // Dirichlet ends of the column
    const T u_top = __ldg(uc + size_t(nzi) * plane);
    auto rhs = [&](int k) {                                 // k = 1 .. nzi
        const T* o = uc + size_t(k - 1) * plane;
        T v = fc ? __ldg(fc + size_t(k - 1) * plane) : T(0);
        const T e = __ldg(o + 1), ww = __ldg(o - 1), n = __ldg(o + px), s = __ldg(o - px);
        v = fma(-sc[k].cx, e + ww, v);
        v = fma(-sc[k].cy, n + s, v);
        if (k == 1) v = fma(-cz, u_bot, v);
        if (k == nzi) v = fma(-cz, u_top, v);
        return v;
    };
    // forward elimination: w_k = (b_k - cz w_{k-1}) lm_k
    T dprev = T(0);
    int k0 = 1;
    for (; k0 + U - 1 <= nzi; k0 += U) {
        T b[U];
#pragma unroll
        for (int q = 0; q < U; ++q) b[q] = rhs(k0 + q);
#pragma unroll
        for (int q = 0; q < U; ++q) {
            dprev = fma(-cz, dprev, b[q]) * sc[k0 + q].lm;
            wc[size_t(k0 + q - 1) * wplane] = dprev;
        }
    }
    for (; k0 <= nzi; ++k0) {
        dprev = fma(-cz, dprev, rhs(k0)) * sc[k0].lm;
        wc[size_t(k0 - 1) * wplane] = dprev;
    }
    // back substitution: u_k = w_k - lsup_k u_{k+1}; u_nzi = w_nzi = dprev
    T* __restrict__ uo = u + at(g, i, j, 1);
    uo[size_t(nzi - 1) * plane] = dprev;
    T unext = dprev;
    int k1 = nzi - 1;
    for (; k1 - U + 1 >= 1; k1 -= U) {
        T d[U];
#pragma unroll
        for (int q = 0; q < U; ++q) d[q] = wc[size_t(k1 - q - 1) * wplane];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            unext = fma(-sc[k1 - q].lsup, unext, d[q]);
            uo[size_t(k1 - q - 1) * plane] = unext;
        }
    }
    for (; k1 >= 1; --k1) {
        unext = fma(-sc[k1].lsup, unext, wc[size_t(k1 - 1) * wplane]);
        uo[size_t(k1 - 1) * plane] = unext;
    }
}

// planes per chunk of loads
template <typename T>
constexpr int ZLINE_U = sizeof(T) == 8 ? 8 : 16;

// columns of one colour per row, and the grid of a pass
__host__ __device__ inline int zline_hx(const Geom& g) { return (g.nx - 2 + 1) / 2; }
inline dim3 zline_grid(const Geom& g) {
    const int hx = zline_hx(g);
    return dim3((hx + LX - 1) / LX, (g.ny - 2 + LY - 1) / LY);
}

}  // namespace mhs
