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

// ---------------------------------------------------------------------------
// Partitioned column solve (FP32 levels).  One thread per column leaves the
// pass latency-bound (one warp per 32 columns walks nz planes twice, and the
// eliminated right-hand side round-trips through memory).  Here a block of
// 32 x S threads owns 32 columns of one colour in one row: the n interior
// planes of a column split into S segments of m planes separated by single
// interface planes c_q = q (m + 1), q = 1 .. S-1.  Warp p solves segment p of
// its 32 columns in shared memory with the local system's own elimination
// factors, taking the interface values as zero: y.  With the responses g, h
// of the segment solution to unit values at its lower and upper interface
// (column-independent, precomputed per level), the column solution is
//   x_k = y_k - cz (g_k x_{c_p} + h_k x_{c_{p+1}})      (k inside segment p),
// and substituting it into the rows of the interface planes gives a
// tridiagonal system in the S - 1 interface values,
//   L_q x_{c_{q-1}} + D_q x_{c_q} + U_q x_{c_{q+1}} = b_{c_q} - cz (y_{q-1,last} + y_{q,first}),
// L_q = -cz^2 g_{q-1,last}, D_q = d_{c_q} - cz^2 (h_{q-1,last} + g_{q,first}),
// U_q = -cz^2 h_{q,first}, whose factors are precomputed too: warp 0 solves it
// per column from the segments' end values in shared memory, then every warp
// forms its segment's x.  The same exact column solve as the Thomas form (the
// matrix is diagonally dominant, so the partitioning is stable), in a
// different rounding order; no scratch array.

constexpr int ZP_MMAX = 32;   // most planes per segment
constexpr int ZB = 8;         // planes whose loads a thread keeps in flight together

// segments of a column of n interior planes: about 24 planes each, at most
// 32, every segment non-empty
__host__ __device__ inline int zpart_segments(int n) {
    int S = 1;
    while (S < 32 && n + 1 > 24 * S) S *= 2;
    while (S > 1 && (S - 1) * ((n + S) / S) > n - 1) S /= 2;
    return S;
}
// planes per segment (the last one may be shorter): ceil((n + 1) / S) - 1
__host__ __device__ inline int zpart_len(int n, int S) { return (n + S) / S - 1; }

// dynamic shared memory of a pass: per-plane factors and (cx, cy), the
// segments' end values and interface right-hand sides, the interface values,
// and the segments' planes (with the interface plane above) of the block's 32
// columns
__host__ __device__ inline size_t zpart_smem(int n, int S) {
    return size_t(n + 2) * (sizeof(float4) + sizeof(float2)) +
           (size_t(4 * S + 1) + size_t(S) * (zpart_len(n, S) + 1)) * 32 * sizeof(float);
}

// columns of one colour per row in blocks of 32, one row of columns per block
inline dim3 zline_part_grid(const Geom& g) { return dim3((zline_hx(g) + 31) / 32, g.ny - 2); }

// One colour pass; the block is 32 x ty threads with ty >= S (warps beyond S
// idle but take part in the barriers).
__device__ __forceinline__ void zline_part_body(const Geom& g, const PlaneCoef<float>* __restrict__ coef,
                                                float* __restrict__ u, const float* __restrict__ f, int colour,
                                                int hx, dim3 b) {
    extern __shared__ __align__(16) unsigned char zline_smem[];
    const int n = g.nz - 2;
    const int S = zpart_segments(n), m = zpart_len(n, S);
    float4* st = reinterpret_cast<float4*>(zline_smem);            // per plane: zlm, zsup, zg, zh
    float2* sxy = reinterpret_cast<float2*>(st + (n + 2));          // per plane: cx, cy
    float* yF = reinterpret_cast<float*>(sxy + (n + 2));            // [segment][lane]: y at its first plane
    float* yL = yF + S * 32;                                        // y at its last plane
    float* bq = yL + S * 32;                                        // right-hand side of the plane above it
    float* xq = bq + S * 32;                                        // [interface q][lane], q = 1 .. S-1
    const int tid = threadIdx.x + 32 * threadIdx.y, nt = 32 * blockDim.y;
    for (int k = 1 + tid; k <= n; k += nt) {
        const PlaneCoef<float> c = coef[k];
        st[k] = make_float4(c.zlm, c.zsup, c.zg, c.zh);
        sxy[k] = make_float2(c.cx, c.cy);
    }
    const float cz = coef[1].cz;
    __syncthreads();

    const int lane = threadIdx.x, p = threadIdx.y;
    const int t = b.x * 32 + lane, j = 1 + int(b.y);
    const int i = 1 + ((1 + j + colour) & 1) + 2 * t;            // (i + j) & 1 == colour
    const bool act = t < hx && i <= g.nx - 2 && p < S;
    const int a = 1 + p * (m + 1);                                  // first plane of the segment
    const int len = act ? min(m, n - a + 1) : 0;
    const bool upper = p < S - 1;                                   // an interface plane above the segment
    const size_t plane = g.plane;
    const ptrdiff_t px = g.px;
    const size_t o0 = act ? at(g, i, j, 0) : 0;
    // right-hand sides f - cx (E + W) - cy (N + S) of the segment's planes and
    // of the interface plane above it, ZB planes' loads in flight together,
    // into shared memory: plane a + q of the lane's column at yp[32 q]
    float* yp = xq + (S + 1) * 32 + p * (m + 1) * 32 + lane;
    const int cnt = len + ((act && upper) ? 1 : 0);
    for (int q0 = 0; q0 < cnt; q0 += ZB) {
        float fe[ZB], ew[ZB], ns[ZB];
#pragma unroll
        for (int q = 0; q < ZB; ++q)
            if (q0 + q < cnt) {
                const size_t o = o0 + size_t(a + q0 + q) * plane;
                fe[q] = f ? __ldg(f + o) : 0.f;
                ew[q] = __ldg(u + o + 1) + __ldg(u + o - 1);
                ns[q] = __ldg(u + o + px) + __ldg(u + o - px);
            }
#pragma unroll
        for (int q = 0; q < ZB; ++q)
            if (q0 + q < cnt) {
                const float2 c = sxy[a + q0 + q];
                yp[(q0 + q) * 32] = fmaf(-c.y, ns[q], fmaf(-c.x, ew[q], fe[q]));
            }
    }
    // the Dirichlet ends of the column, folded into its first and last rows
    if (act && p == 0) yp[0] = fmaf(-cz, __ldg(u + o0), yp[0]);
    if (act && p == S - 1) yp[(len - 1) * 32] = fmaf(-cz, __ldg(u + o0 + size_t(n + 1) * plane), yp[(len - 1) * 32]);
    const float bup = (act && upper) ? yp[len * 32] : 0.f;
    // the segment's own solve with the interface values taken as zero, in place
    float prev = 0.f;
    for (int q = 0; q < len; ++q) {
        prev = fmaf(-cz, prev, yp[q * 32]) * st[a + q].x;
        yp[q * 32] = prev;
    }
    const float ylast = prev;
    float nxt = prev;
    for (int q = len - 2; q >= 0; --q) {
        nxt = fmaf(-st[a + q].y, nxt, yp[q * 32]);
        yp[q * 32] = nxt;
    }
    if (p < S) {
        yF[p * 32 + lane] = len > 0 ? yp[0] : 0.f;
        yL[p * 32 + lane] = ylast;
        bq[p * 32 + lane] = bup;
    }
    __syncthreads();
    // the interface system, one column per lane of warp 0
    if (p == 0 && S > 1) {
        float w = 0.f;
        for (int q = 1; q < S; ++q) {
            const float4 c = st[q * (m + 1)];
            const float r = fmaf(-cz, yL[(q - 1) * 32 + lane] + yF[q * 32 + lane], bq[(q - 1) * 32 + lane]);
            w = fmaf(-c.z, w, r) * c.x;
            xq[q * 32 + lane] = w;
        }
        float x = 0.f;
        for (int q = S - 1; q >= 1; --q) {
            x = q == S - 1 ? xq[q * 32 + lane] : fmaf(-st[q * (m + 1)].y, x, xq[q * 32 + lane]);
            xq[q * 32 + lane] = x;
        }
    }
    __syncthreads();
    if (!act) return;
    const float xl = p > 0 ? xq[p * 32 + lane] : 0.f;
    const float xr = upper ? xq[(p + 1) * 32 + lane] : 0.f;
    for (int q = 0; q < len; ++q) {
        const float4 c = st[a + q];
        u[o0 + size_t(a + q) * plane] = fmaf(-cz, fmaf(c.z, xl, c.w * xr), yp[q * 32]);
    }
    if (upper) u[o0 + size_t(a + len) * plane] = xr;
}


}  // namespace mhs
