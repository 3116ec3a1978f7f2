// Per-block bodies of the multigrid building blocks (kernels_mg.cu) for the
// lower-boundary problem (eq. lower_bound, 5-point stencil) and the interior
// problem (eq. scalar_pot, 7-point stencil with per-plane coefficients).
//
// Each body takes the block's index b and the grid's dimensions gd
// explicitly, so that the same code runs as a kernel of its own
// (b = blockIdx, gd = gridDim) and inside a grouped launch that covers many
// instances, where every instance keeps its own block decomposition: a
// grouped solve is then bitwise identical to solving each instance alone.
// Blocks are BX x BY threads.
#pragma once

#include <algorithm>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

constexpr int MG_BX = 32, MG_BY = 8;

// Red-black Gauss-Seidel colour pass (in place): colour c updates the
// interior nodes with (i + j + k) % 2 == c by solving their own row of
// A u = f for u_ijk with the current neighbour values; thread t of row
// (j, k) takes i = i0 + 2t.  f == nullptr means f = 0.
template <typename T, bool D3>
__device__ __forceinline__ void colour_body(const Geom& g, const PlaneCoef<T>* __restrict__ coef,
                                            T* __restrict__ u, const T* __restrict__ f, int colour, dim3 b,
                                            dim3 gd) {
    const int t = b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (j > g.ny - 2) return;
    for (int k = D3 ? 1 + b.z : 0; k <= (D3 ? g.nz - 2 : 0); k += gd.z) {
        const int i = 1 + (((1 + j + k) & 1) != colour) + 2 * t;
        if (i > g.nx - 2) continue;
        const PlaneCoef<T> c = coef[k];
        const size_t o = at(g, i, j, k);
        // u = f/d - ax (E + W) - ay (N + S) - az (U + D)
        T v = f ? f[o] * c.inv_d : T(0);
        if (D3) v = fma(-c.az, u[o + g.plane] + u[o - g.plane], v);
        v = fma(-c.ay, u[o + g.px] + u[o - g.px], v);
        u[o] = fma(-c.ax, u[o + 1] + u[o - 1], v);
    }
}

// r = f - A u at interior nodes; with NORM also this block's sum of r^2 (in
// double), stored at partial[b.x + gd.x (b.y + gd.y b.z)] and finished in a
// fixed order by the norm / check kernels.  Every thread of the block must
// call it.
template <typename T, bool D3, bool NORM>
__device__ __forceinline__ void residual_body(const Geom& g, const PlaneCoef<T>* __restrict__ coef,
                                              const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ r,
                                              double* __restrict__ partial, dim3 b, dim3 gd) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (i <= g.nx - 2 && j <= g.ny - 2) {
        for (int k = D3 ? 1 + b.z : 0; k <= (D3 ? g.nz - 2 : 0); k += gd.z) {
            const PlaneCoef<T> c = coef[k];
            const size_t o = at(g, i, j, k);
            // r = f - cz (U + D) - cy (N + S) - cx (E + W) - d u: one FMA per
            // term, f (or 0) as the first addend
            T v = f ? f[o] : T(0);
            if (D3) v = fma(-c.cz, u[o + g.plane] + u[o - g.plane], v);
            v = fma(-c.cy, u[o + g.px] + u[o - g.px], v);
            v = fma(-c.cx, u[o + 1] + u[o - 1], v);
            const T rv = fma(-c.d, u[o], v);
            r[o] = rv;
            if (NORM) acc += double(rv) * double(rv);
        }
    }
    if (!NORM) return;
    const double s = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[b.x + gd.x * (b.y + gd.y * b.z)] = s;
}

// The residual right after a red-black sweep: the black nodes, updated last,
// satisfy their own rows of A u = f given the final red values, so their
// residual is zero to rounding and is stored as 0; the red nodes' residual is
// computed as in residual_body (same operations).  Thread t of row (j, k)
// takes the pair of nodes 1 + 2t and 2 + 2t, one red and one black (the
// colour pass's mapping), so the FP64 work is that of half the nodes.  NORM:
// the block's sum of r^2 over its red nodes, at the same partial index as
// residual_body.  Every thread of the block must call it.
template <typename T, bool D3, bool NORM>
__device__ __forceinline__ void residual_red_body(const Geom& g, const PlaneCoef<T>* __restrict__ coef,
                                                  const T* __restrict__ u, const T* __restrict__ f,
                                                  T* __restrict__ r, double* __restrict__ partial, dim3 b, dim3 gd) {
    const int t = b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (j <= g.ny - 2 && 1 + 2 * t <= g.nx - 2) {
        for (int k = D3 ? 1 + b.z : 0; k <= (D3 ? g.nz - 2 : 0); k += gd.z) {
            const int red = ((1 + j + k) & 1);   // the red node of the pair is 1 + red + 2t
            const int ir = 1 + red + 2 * t, ib = 2 - red + 2 * t;
            if (ib <= g.nx - 2) r[at(g, ib, j, k)] = T(0);
            if (ir > g.nx - 2) continue;
            const PlaneCoef<T> c = coef[k];
            const size_t o = at(g, ir, j, k);
            T v = f ? f[o] : T(0);
            if (D3) v = fma(-c.cz, u[o + g.plane] + u[o - g.plane], v);
            v = fma(-c.cy, u[o + g.px] + u[o - g.px], v);
            v = fma(-c.cx, u[o + 1] + u[o - 1], v);
            const T rv = fma(-c.d, u[o], v);
            r[o] = rv;
            if (NORM) acc += double(rv) * double(rv);
        }
    }
    if (!NORM) return;
    const double s = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[b.x + gd.x * (b.y + gd.y * b.z)] = s;
}

// FP32 3D forms of the colour pass and the residual that give each thread
// the four consecutive nodes i0 .. i0+3 (i0 = 4t) of a row: the centre row,
// the four neighbour rows and f are read as 16-byte vectors (rows start on
// 16-byte boundaries), the two outer neighbours as scalars, and the result
// is stored as one vector.  Per node the arithmetic is that of the scalar
// bodies above.  For odd nx only (the padded row, px >= nx + 1, then holds
// every vector a thread touches), and for levels of at least 4M interior
// nodes: there the passes are DRAM-bound and the quads raise the rate from
// 58 % (colour pass) and 45 % (residual) to about 70 % of the measured copy
// bandwidth, while on smaller, cache-resident levels the scalar forms'
// twice as many threads hide latency better.
__host__ __device__ inline bool use_v4(const Geom& g) {
    return (g.nx & 1) != 0 && double(g.nx - 2) * double(g.ny - 2) * double(g.nz - 2) >= 4.0e6;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float lane(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// colour pass: the quad's two nodes of the colour are updated; the other two
// (neighbours of this colour, unchanged by the pass) are stored back as read
__device__ __forceinline__ void colour_body_v4(const Geom& g, const PlaneCoef<float>* __restrict__ coef,
                                               float* __restrict__ u, const float* __restrict__ f, int colour,
                                               dim3 b, dim3 gd) {
    const int i0 = 4 * int(b.x * blockDim.x + threadIdx.x);
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (j > g.ny - 2 || i0 > g.nx - 2) return;
    for (int k = 1 + b.z; k <= g.nz - 2; k += gd.z) {
        const PlaneCoef<float> c = coef[k];
        const size_t o = at(g, i0, j, k);
        const float4 cc = ld4(u + o);
        const float4 nn = ld4(u + o + g.px), ss = ld4(u + o - g.px);
        const float4 uu = ld4(u + o + g.plane), dd = ld4(u + o - g.plane);
        const float4 ff = f ? ld4(f + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float west = i0 > 0 ? u[o - 1] : 0.f, east = u[o + 4];
        float res[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q;
            if (i < 1 || i > g.nx - 2 || ((i + j + k) & 1) != colour) continue;
            const float e = q < 3 ? lane(cc, q + 1) : east;
            const float w = q > 0 ? lane(cc, q - 1) : west;
            float v = f ? lane(ff, q) * c.inv_d : 0.f;
            v = fmaf(-c.az, lane(uu, q) + lane(dd, q), v);
            v = fmaf(-c.ay, lane(nn, q) + lane(ss, q), v);
            res[q] = fmaf(-c.ax, e + w, v);
        }
        *reinterpret_cast<float4*>(u + o) = make_float4(res[0], res[1], res[2], res[3]);
    }
}

// r = f - A u on the quad (0 at the quad's boundary and padding positions)
__device__ __forceinline__ void residual_body_v4(const Geom& g, const PlaneCoef<float>* __restrict__ coef,
                                                 const float* __restrict__ u, const float* __restrict__ f,
                                                 float* __restrict__ r, dim3 b, dim3 gd) {
    const int i0 = 4 * int(b.x * blockDim.x + threadIdx.x);
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (j > g.ny - 2 || i0 > g.nx - 2) return;
    for (int k = 1 + b.z; k <= g.nz - 2; k += gd.z) {
        const PlaneCoef<float> c = coef[k];
        const size_t o = at(g, i0, j, k);
        const float4 cc = ld4(u + o);
        const float4 nn = ld4(u + o + g.px), ss = ld4(u + o - g.px);
        const float4 uu = ld4(u + o + g.plane), dd = ld4(u + o - g.plane);
        const float4 ff = f ? ld4(f + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float west = i0 > 0 ? u[o - 1] : 0.f, east = u[o + 4];
        float res[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q;
            res[q] = 0.f;
            if (i < 1 || i > g.nx - 2) continue;
            const float e = q < 3 ? lane(cc, q + 1) : east;
            const float w = q > 0 ? lane(cc, q - 1) : west;
            float v = f ? lane(ff, q) : 0.f;
            v = fmaf(-c.cz, lane(uu, q) + lane(dd, q), v);
            v = fmaf(-c.cy, lane(nn, q) + lane(ss, q), v);
            v = fmaf(-c.cx, e + w, v);
            res[q] = fmaf(-c.d, lane(cc, q), v);
        }
        *reinterpret_cast<float4*>(r + o) = make_float4(res[0], res[1], res[2], res[3]);
    }
}

// Full weighting: tensor product of (1/4, 1/2, 1/4) around the fine node
// (2I, 2J, 2K) coincident with coarse interior node (I, J, K), formed as the
// tensor product of (1, 2, 1) sums (two operations per triple: a + c, then
// an FMA with 2b) scaled once by 1/64 (2D: 1/16); the power-of-two weights
// make this the same weighted sum up to the order of the additions.  With
// uc != nullptr the coarse iterate is zeroed at the same nodes (the initial
// guess of the coarse-grid correction).
//
// red: rf is a residual taken right after a red-black sweep, zero (stored as
// +0) at the black nodes, those with i + j + k odd.  The fine node under a
// coarse one is red, so of its 27 neighbours only the centre and the 12 edge
// neighbours (two offsets non-zero) can be non-zero, and each (1, 2, 1) triple
// has either zero ends (fma(2, b, +0) = 2b) or a zero middle
// (fma(2, +0, a + c) = a + c): the same sums are formed from the 13 red
// values with 18 instead of 27 FP64 operations, equal to the full form's
// (up to the sign of a zero result).
template <typename T, bool D3>
__device__ __forceinline__ void restrict_body(const Geom& gf, const Geom& gc, const T* __restrict__ rf,
                                              T* __restrict__ fc, T* __restrict__ uc, dim3 b, dim3 gd,
                                              bool red = false) {
    const int I = 1 + b.x * blockDim.x + threadIdx.x;
    const int J = 1 + b.y * blockDim.y + threadIdx.y;
    if (I > gc.nx - 2 || J > gc.ny - 2) return;
    const ptrdiff_t sy = (ptrdiff_t)gf.px, sz = (ptrdiff_t)gf.plane;
    for (int K = D3 ? 1 + b.z : 0; K <= (D3 ? gc.nz - 2 : 0); K += gd.z) {
        const size_t o = at(gf, 2 * I, 2 * J, D3 ? 2 * K : 0);
        T acc;
        if (red) {
            const T* q = rf + o;
            // a plane whose centre node is red: centre row 2b, the two off rows a + c
            auto plane_r = [&](const T* c) { return fma(T(2), fma(T(2), c[0], T(0)), (c[-sy - 1] + c[-sy + 1]) + (c[sy - 1] + c[sy + 1])); };
            if (D3) {
                // a plane whose centre node is black: centre row a + c, the two off rows 2b
                auto plane_b = [&](const T* c) { return fma(T(2), c[-1] + c[1], fma(T(2), c[-sy], T(0)) + fma(T(2), c[sy], T(0))); };
                acc = fma(T(2), plane_r(q), plane_b(q - sz) + plane_b(q + sz)) * T(1.0 / 64.0);
            } else {
                acc = plane_r(q) * T(1.0 / 16.0);
            }
        } else {
            auto row = [&](size_t ob) { return fma(T(2), rf[ob], rf[ob - 1] + rf[ob + 1]); };
            auto plane = [&](size_t oc) { return fma(T(2), row(oc), row(oc - gf.px) + row(oc + gf.px)); };
            if (D3) {
                const T lo = plane(o - gf.plane), mid = plane(o), hi = plane(o + gf.plane);
                acc = fma(T(2), mid, lo + hi) * T(1.0 / 64.0);
            } else {
                acc = plane(o) * T(1.0 / 16.0);
            }
        }
        fc[at(gc, I, J, K)] = acc;
        if (uc) uc[at(gc, I, J, K)] = T(0);
    }
}

// u_f += I u_c at fine interior nodes: along each axis an even fine index
// takes coarse node i/2, an odd one the mean of (i-1)/2 and (i+1)/2.  One
// thread per coarse cell (I..I+1, J..J+1, K..K+1) produces its 8 (2D: 4)
// fine nodes (2I+a, 2J+b, 2K+c), a, b, c in {0, 1}, sharing the partial sums
// of the corner values; an even fine index is interior only when its coarse
// index is >= 1.
template <typename T, bool D3>
__device__ __forceinline__ void prolong_body(const Geom& gc, const Geom& gf, const T* __restrict__ uc,
                                             T* __restrict__ uf, dim3 b, dim3 gd) {
    const int I = b.x * blockDim.x + threadIdx.x;
    const int J = b.y * blockDim.y + threadIdx.y;
    if (I > gc.nx - 2 || J > gc.ny - 2) return;
    const ptrdiff_t cx = 1, cy = gc.px, cz = (ptrdiff_t)gc.plane;
    const ptrdiff_t fx = 1, fy = gf.px, fz = (ptrdiff_t)gf.plane;
    const bool ex = I >= 1, ey = J >= 1;
    for (int K = D3 ? b.z : 0; K <= (D3 ? gc.nz - 2 : 0); K += gd.z) {
        const T* c = uc + at(gc, I, J, K);
        T* f = uf + at(gf, 2 * I, 2 * J, D3 ? 2 * K : 0);
        const T c000 = c[0], c100 = c[cx], c010 = c[cy], c110 = c[cx + cy];
        const T e100 = c000 + c100, e010 = c000 + c010, e110 = e100 + (c010 + c110);
        const bool ez = !D3 || K >= 1;
        if (ex && ey && ez) f[0] += c000;
        if (ey && ez) f[fx] = fma(T(0.5), e100, f[fx]);
        if (ex && ez) f[fy] = fma(T(0.5), e010, f[fy]);
        if (ez) f[fx + fy] = fma(T(0.25), e110, f[fx + fy]);
        if (D3) {
            const T c001 = c[cz], c101 = c[cx + cz], c011 = c[cy + cz], c111 = c[cx + cy + cz];
            const T s01 = c001 + c101, s02 = c001 + c011;
            if (ex && ey) f[fz] = fma(T(0.5), c000 + c001, f[fz]);
            if (ey) f[fx + fz] = fma(T(0.25), e100 + s01, f[fx + fz]);
            if (ex) f[fy + fz] = fma(T(0.25), e010 + s02, f[fy + fz]);
            f[fx + fy + fz] = fma(T(0.125), e110 + (s01 + (c011 + c111)), f[fx + fy + fz]);
        }
    }
}

// Residual and full-weighting restriction in one pass (Sect. 4: the
// residual of the smoothed iterate, restricted to the coarse right-hand
// side), without storing the residual: a block owns a tile of RX x RR_Y
// coarse nodes and a chunk of coarse planes, and marches up the fine planes
// of the chunk's support.  The tile's fine window is the fine nodes 2I - 1 ..
// 2I + 1, 2J - 1 .. 2J + 1 of its coarse nodes (2 RX + 1 by 2 RR_Y + 1).  On
// each fine plane the residual r = f - A u of the window is formed by quads
// of four consecutive x nodes (x from 2 RX bx, a multiple of four, so FP32
// quads are 16-byte vectors of u, of its four neighbour rows and of f, the
// outer x neighbours scalars; stencil reuse across quads, rows and planes
// comes from L1) into shared memory; then the x row sums at the coarse x
// positions, the y sums at the coarse nodes, and three consecutive fine
// planes give f_c.  Per node these are the operations of residual_body and
// of restrict_body, in their order, so the result equals the two separate
// launches bit for bit.  Fine planes shared by two chunks and fine columns
// and rows shared by two tiles are computed by both.  uc != nullptr: the
// coarse iterate is zeroed at the same nodes.  RX = 32 coarse nodes along x
// (threads 32 x 8, one per coarse node in the last step).  The V-cycles run
// it on FP32 levels, which are bound by memory traffic; on FP64 levels the
// FP64 pipe is the bound and the pass saves no FP64 operation.  Blocks of
// RR_THREADS threads; every thread must call it.
constexpr int RR_X = 32, RR_Y = 8, RR_THREADS = 256;

template <typename T, bool D3>
__device__ __forceinline__ void resid_restrict_body(const Geom& gf, const Geom& gc, const PlaneCoef<T>* __restrict__ coef,
                                                    const T* __restrict__ u, const T* __restrict__ f,
                                                    T* __restrict__ fc, T* __restrict__ uc, dim3 b, dim3 gd) {
    constexpr int WX = 2 * RR_X + 1, WY = 2 * RR_Y + 1;   // residual window
    constexpr int NQ = (WX + 1 + 3) / 4;                   // quads per window row (from one node left of it)
    constexpr int RP = NQ * 4 + 1;                         // row pitch of r (odd)
    __shared__ T rw[WY][RP];                               // rw[y][x]: r at (x0 + x, fy0 + y)
    __shared__ T rs[WY][RR_X];                             // row sums at the coarse x positions
    const int tid = threadIdx.x;
    const int tx = tid % RR_X, ty = tid / RR_X;
    const int Ib = 1 + int(b.x) * RR_X, Jb = 1 + int(b.y) * RR_Y;
    const int fy0 = 2 * Jb - 1;                            // first window row
    const int x0 = 2 * Ib - 2;                             // first quad column: one node left of the window
    const int I = Ib + tx, J = Jb + ty;
    const bool node = I <= gc.nx - 2 && J <= gc.ny - 2;
    // residual of the quad (x0 + 4 q .. + 3, fy0 + y) of fine plane kf into rw (0 off the interior)
    auto resid_quad = [&](int q, int y, int kf, const PlaneCoef<T>& c) {
        const int i0 = x0 + 4 * q, j = fy0 + y;
        T res[4] = {T(0), T(0), T(0), T(0)};
        if (j <= gf.ny - 2 && i0 <= gf.nx - 2) {
            const size_t o = at(gf, i0, j, kf);
            T cc[4], nn[4], ss[4], uu[4], dd[4], ff[4];
            if constexpr (sizeof(T) == 4) {
                // the quad lies inside the padded row (px a multiple of four, i0 < nx)
                auto ld4 = [](const T* ptr, T* out) {
                    const float4 v = *reinterpret_cast<const float4*>(ptr);
                    out[0] = v.x, out[1] = v.y, out[2] = v.z, out[3] = v.w;
                };
                ld4(u + o, cc);
                ld4(u + o + gf.px, nn);
                ld4(u + o - gf.px, ss);
                if (D3) {
                    ld4(u + o + gf.plane, uu);
                    ld4(u + o - gf.plane, dd);
                }
                if (f) ld4(f + o, ff);
            } else {
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    cc[l] = u[o + l];
                    nn[l] = u[o + l + gf.px];
                    ss[l] = u[o + l - gf.px];
                    if (D3) {
                        uu[l] = u[o + l + gf.plane];
                        dd[l] = u[o + l - gf.plane];
                    }
                    if (f) ff[l] = f[o + l];
                }
            }
            const T west = i0 > 0 ? u[o - 1] : T(0);
            const T east = i0 + 3 <= gf.nx - 2 ? u[o + 4] : T(0);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int i = i0 + l;
                if (i < 1 || i > gf.nx - 2) continue;
                const T e = l < 3 ? cc[l + 1] : east;
                const T w = l > 0 ? cc[l - 1] : west;
                T v = f ? ff[l] : T(0);
                if (D3) v = fma(-c.cz, uu[l] + dd[l], v);
                v = fma(-c.cy, nn[l] + ss[l], v);
                v = fma(-c.cx, e + w, v);
                res[l] = fma(-c.d, cc[l], v);
            }
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) rw[y][4 * q + l] = res[l];
    };
    auto resid_plane = [&](int kf) {
        const PlaneCoef<T> c = coef[kf];
        for (int e = tid; e < WY * NQ; e += RR_THREADS) {
            const int y = e / NQ, q = e - y * NQ;
            resid_quad(q, y, kf, c);
        }
    };
    // full-weighting y-x sum of the window at this thread's coarse node (window node x at rw
    // column x + 1)
    auto plane_sum = [&]() {
        __syncthreads();
        for (int y = ty; y < WY; y += RR_THREADS / RR_X) {
            const int w = 2 * tx + 2;
            rs[y][tx] = fma(T(2), rw[y][w], rw[y][w - 1] + rw[y][w + 1]);
        }
        __syncthreads();
        const int w = 2 * ty + 1;
        return node ? fma(T(2), rs[w][tx], rs[w - 1][tx] + rs[w + 1][tx]) : T(0);
    };
    if (D3) {
        const int nkc = gc.nz - 2;
        const int per = (nkc + int(gd.z) - 1) / int(gd.z);
        const int K0 = 1 + int(b.z) * per, K1 = min(nkc, K0 + per - 1);
        if (K0 <= K1) {
            resid_plane(2 * K0 - 1);
            T lo = plane_sum();
            for (int K = K0; K <= K1; ++K) {
                // plane_sum's barriers order these writes of rw after every read of the previous plane
                resid_plane(2 * K);
                const T mid = plane_sum();
                resid_plane(2 * K + 1);
                const T hi = plane_sum();
                if (node) {
                    fc[at(gc, I, J, K)] = fma(T(2), mid, lo + hi) * T(1.0 / 64.0);
                    if (uc) uc[at(gc, I, J, K)] = T(0);
                }
                lo = hi;
            }
        }
    } else {
        resid_plane(0);
        const T sum = plane_sum();
        if (node) {
            fc[at(gc, I, J, 0)] = sum * T(1.0 / 16.0);
            if (uc) uc[at(gc, I, J, 0)] = T(0);
        }
    }
}

// grid of resid_restrict_body: coarse tiles in x and y, chunks of `per`
// coarse planes along z, per chosen so that the grid is about eight blocks per
// SM while a chunk spans at least four coarse planes where the level has them
// (every chunk recomputes one fine plane of its neighbour)
inline dim3 resid_restrict_grid(const Geom& gc, int d3) {
    const int gx = (gc.nx - 2 + RR_X - 1) / RR_X, gy = (gc.ny - 2 + RR_Y - 1) / RR_Y;
    if (!d3) return dim3(gx, gy, 1);
    const int nkc = gc.nz - 2;
    int per = std::max(1, (nkc * gx * gy + 152 * 8 - 1) / (152 * 8));
    per = std::max(per, std::min(4, nkc));
    return dim3(gx, gy, (nkc + per - 1) / per);
}

// f = -B_z on the interior of the lower-boundary plane (eq. lower_bound)
__device__ __forceinline__ void lower_rhs_body(const Geom& g, const double* __restrict__ bz, double* __restrict__ f,
                                               dim3 b) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const size_t o = at(g, i, j, 0);
    f[o] = -bz[o];
}

// the lower-boundary solution as the z = 0 plane of a 3D array
__device__ __forceinline__ void copy_plane_body(const Geom& g2, const double* __restrict__ src, const Geom& g3,
                                                double* __restrict__ dst, dim3 b) {
    const int i = b.x * blockDim.x + threadIdx.x;
    const int j = b.y * blockDim.y + threadIdx.y;
    if (i >= g2.nx || j >= g2.ny) return;
    dst[at(g3, i, j, 0)] = src[at(g2, i, j, 0)];
}

// ||b||^2 partials of the lifted interior right-hand side: the Dirichlet data
// on k = 0 enters row (i, j, 1) as cz * P(i, j, 0).  Every thread calls it.
__device__ __forceinline__ void lift_norm_body(const Geom& g, const PlaneCoef<double>* __restrict__ coef,
                                               const double* __restrict__ u, double* __restrict__ partial, dim3 b,
                                               dim3 gd) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (i <= g.nx - 2 && j <= g.ny - 2) {
        const double v = coef[1].cz * u[at(g, i, j, 0)];
        acc = v * v;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[b.x + gd.x * b.y] = s;
}

// grid of the per-node kernels: xcount threads along x, one row of blocks per
// BY rows, planes spread over gridDim.z (capped by max_blocks when > 0)
inline dim3 mg_grid(const Geom& g, int d3, int xcount, int max_blocks) {
    const int gx = (xcount + MG_BX - 1) / MG_BX;
    const int gy = (g.ny - 2 + MG_BY - 1) / MG_BY;
    int gz = 1;
    if (d3) {
        gz = g.nz - 2;
        const int cap = max_blocks > 0 ? max_blocks / (gx * gy) : 65535;
        if (gz > cap) gz = cap > 0 ? cap : 1;
        if (gz > 65535) gz = 65535;
    }
    return dim3(gx, gy, gz);
}

// thread-block shapes of the red-black colour passes (option `tile`, 1-based)
constexpr int N_TILES = 5;
inline dim3 tile_block(int tile) {
    switch (tile) {
    case 2: return dim3(64, 4);
    case 3: return dim3(16, 16);
    case 4: return dim3(32, 16);
    case 5: return dim3(128, 2);
    default: return dim3(MG_BX, MG_BY);
    }
}
// grid of a colour pass with block shape blk (xcount threads along x)
inline dim3 tile_grid(const Geom& g, int d3, int xcount, dim3 blk) {
    const int gx = (xcount + int(blk.x) - 1) / int(blk.x);
    const int gy = (g.ny - 2 + int(blk.y) - 1) / int(blk.y);
    int gz = d3 ? g.nz - 2 : 1;
    if (gz > 65535) gz = 65535;
    return dim3(gx, gy, gz);
}

// the grids the solver launches each operation with (quad forms for FP32 3D
// levels with odd nx: one thread per 4 consecutive x positions from 0)
inline dim3 smooth_grid(const Geom& g, int d3) { return mg_grid(g, d3, (g.nx - 2 + 1) / 2, 0); }
inline dim3 quad_grid(const Geom& g) { return mg_grid(g, 1, (g.nx - 2) / 4 + 1, 0); }
template <typename T>
inline dim3 smooth_grid_t(const Geom& g, int d3) {
    return (sizeof(T) == 4 && d3 && use_v4(g)) ? quad_grid(g) : smooth_grid(g, d3);
}
template <typename T>
inline dim3 residual_grid_plain_t(const Geom& g, int d3) {
    return (sizeof(T) == 4 && d3 && use_v4(g)) ? quad_grid(g) : mg_grid(g, d3, g.nx - 2, 0);
}
// with norm partials, a few blocks per SM (each then covers several planes):
// one block per (tile, plane) was slower, every block paying a block-wide
// reduction for 256 nodes; the fixed-order finish stays short too
inline dim3 residual_grid(const Geom& g, int d3, bool norm, int max_blocks) {
    return mg_grid(g, d3, g.nx - 2, norm ? (max_blocks < 152 * 8 ? max_blocks : 152 * 8) : 0);
}
// the same for residual_red_body: one thread per pair of x positions
inline dim3 residual_red_grid(const Geom& g, int d3, bool norm, int max_blocks) {
    return mg_grid(g, d3, (g.nx - 2 + 1) / 2, norm ? (max_blocks < 152 * 8 ? max_blocks : 152 * 8) : 0);
}
inline dim3 restrict_grid(const Geom& gc, int d3) { return mg_grid(gc, d3, gc.nx - 2, 0); }
inline dim3 prolong_grid(const Geom& gc, int d3) {
    Geom cells = gc;   // one thread per coarse cell: nc - 1 cells per axis
    cells.ny = gc.ny + 1;
    cells.nz = gc.nz + 1;
    return mg_grid(cells, d3, gc.nx - 1, 0);
}
inline dim3 plane_grid(const Geom& g2) { return dim3((g2.nx + MG_BX - 1) / MG_BX, (g2.ny + MG_BY - 1) / MG_BY); }
inline dim3 lift_grid(const Geom& g3) {
    return dim3((g3.nx - 2 + MG_BX - 1) / MG_BX, (g3.ny - 2 + MG_BY - 1) / MG_BY);
}

}  // namespace mhs
