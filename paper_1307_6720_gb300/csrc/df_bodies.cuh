// Per-block bodies of the double-float kernels of mixed-precision defect
// correction (kernels_df.cu), with explicit block index b and grid
// dimensions gd, so that grouped launches over many instances run the same
// code with each instance's own block decomposition (see mg_bodies.cuh).
//
// The iterate of the finest level is carried as an unevaluated sum of two
// FP32 words, P = hi + lo (|lo| <= ulp(hi)/2, about 48 significant bits), and
// the outer residual r = f - A P is evaluated with error-free
// transformations instead of FP64 instructions:
//   - TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   - Fast2Sum (Dekker 1971): the same when |a| >= |b|;
//   - TwoProd with a fused multiply-add: p + e = a * b exactly.
// Intrinsics with explicit rounding (__fadd_rn, ...) keep the compiler from
// contracting or reassociating the transformations.
#pragma once

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

constexpr int DF_BX = 32, DF_BY = 8;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// r = f - A (hi + lo) at one interior node from its stencil values:
// centre C, x neighbours E W, y neighbours N S, z neighbours U D of the high
// and the low words.
template <bool D3>
__device__ __forceinline__ float df_stencil(const PlaneCoefDF& c, float hE, float hW, float hN, float hS, float hU,
                                           float hD, float hC, float lE, float lW, float lN, float lS, float lU,
                                           float lD, float lC, float fh, float fl) {
    // neighbour pair sums of the high words, exactly as (sum, error)
    float s1, e1, s2, e2, s3 = 0.f, e3 = 0.f;
    two_sum(hE, hW, s1, e1);
    two_sum(hN, hS, s2, e2);
    if (D3) two_sum(hU, hD, s3, e3);
    const float ch = hC;
    // leading products, exactly as (product, error)
    float px, qx, py, qy, pz = 0.f, qz = 0.f, pd, qd;
    two_prod(c.cxh, s1, px, qx);
    two_prod(c.cyh, s2, py, qy);
    if (D3) two_prod(c.czh, s3, pz, qz);
    two_prod(c.dh, ch, pd, qd);
    // second-order terms (each ~2^-24 of its leading product): plain FP32
    float t = qx + qy + qd;
    t = __fmaf_rn(c.cxh, e1, t);
    t = __fmaf_rn(c.cxl, s1, t);
    t = __fmaf_rn(c.cyh, e2, t);
    t = __fmaf_rn(c.cyl, s2, t);
    t = __fmaf_rn(c.dl, ch, t);
    if (D3) {
        t += qz;
        t = __fmaf_rn(c.czh, e3, t);
        t = __fmaf_rn(c.czl, s3, t);
    }
    // A applied to the low words (about 2^-24 of the total): plain FP32
    float al = c.cxh * (lE + lW) + c.cyh * (lN + lS) + c.dh * lC;
    if (D3) al += c.czh * (lU + lD);
    t += al;
    // exact sum of the leading products, which cancel down to the residual
    float s, e, err;
    two_sum(px, py, s, err);
    if (D3) {
        two_sum(s, pz, s, e);
        err += e;
    }
    two_sum(s, pd, s, e);
    err += e;
    // r = (fh - s) + (fl - err - t)
    float a, b;
    two_sum(fh, -s, a, b);
    return a + (b + (fl - (err + t)));
}

// outer residual rounded to FP32 (r32) with this block's sum of r^2 in
// partial[b.x + gd.x (b.y + gd.y b.z)]; every thread of the block calls it.
// 3D: block b.z takes a contiguous chunk of planes and each thread marches up
// its column, the column's own and vertical-neighbour words kept in
// registers (10 loads per node instead of 14).
template <bool D3>
__device__ __forceinline__ void df_residual_body(const Geom& g, const PlaneCoefDF* __restrict__ cdf,
                                                 const float* __restrict__ hi, const float* __restrict__ lo,
                                                 const float* __restrict__ fh, const float* __restrict__ fl,
                                                 float* __restrict__ r32, double* __restrict__ partial, dim3 b,
                                                 dim3 gd) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    float acc = 0.f;
    if (i <= g.nx - 2 && j <= g.ny - 2) {
        const ptrdiff_t sy = g.px, sz = (ptrdiff_t)g.plane;
        if (D3) {
            const int nzi = g.nz - 2, chunk = (nzi + int(gd.z) - 1) / int(gd.z);
            const int k0 = 1 + int(b.z) * chunk, k1 = min(g.nz - 2, k0 + chunk - 1);
            if (k0 <= k1) {
                // one plane ahead: the next plane's loads are issued before the
                // current plane's double-float arithmetic, so their latency overlaps it
                size_t o = at(g, i, j, k0);
                float hD = hi[o - sz], hC = hi[o], lD = lo[o - sz], lC = lo[o];
                float hE = hi[o + 1], hW = hi[o - 1], hN = hi[o + sy], hS = hi[o - sy], hU = hi[o + sz];
                float lE = lo[o + 1], lW = lo[o - 1], lN = lo[o + sy], lS = lo[o - sy], lU = lo[o + sz];
                float fa = fh ? fh[o] : 0.f, fb = fl ? fl[o] : 0.f;
                for (int k = k0; k <= k1; ++k, o += sz) {
                    float nhE = 0.f, nhW = 0.f, nhN = 0.f, nhS = 0.f, nhU = 0.f;
                    float nlE = 0.f, nlW = 0.f, nlN = 0.f, nlS = 0.f, nlU = 0.f, nfa = 0.f, nfb = 0.f;
                    if (k < k1) {
                        const size_t p = o + sz;
                        nhE = hi[p + 1], nhW = hi[p - 1], nhN = hi[p + sy], nhS = hi[p - sy], nhU = hi[p + sz];
                        nlE = lo[p + 1], nlW = lo[p - 1], nlN = lo[p + sy], nlS = lo[p - sy], nlU = lo[p + sz];
                        nfa = fh ? fh[p] : 0.f;
                        nfb = fl ? fl[p] : 0.f;
                    }
                    const float r = df_stencil<true>(cdf[k], hE, hW, hN, hS, hU, hD, hC, lE, lW, lN, lS, lU, lD, lC,
                                                     fa, fb);
                    r32[o] = r;
                    acc = __fmaf_rn(r, r, acc);
                    hD = hC;
                    hC = hU;
                    lD = lC;
                    lC = lU;
                    hE = nhE, hW = nhW, hN = nhN, hS = nhS, hU = nhU;
                    lE = nlE, lW = nlW, lN = nlN, lS = nlS, lU = nlU;
                    fa = nfa, fb = nfb;
                }
            }
        } else {
            const size_t o = at(g, i, j, 0);
            const float r = df_stencil<false>(cdf[0], hi[o + 1], hi[o - 1], hi[o + sy], hi[o - sy], 0.f, 0.f, hi[o],
                                              lo[o + 1], lo[o - 1], lo[o + sy], lo[o - sy], 0.f, 0.f, lo[o],
                                              fh ? fh[o] : 0.f, fl ? fl[o] : 0.f);
            r32[o] = r;
            acc = __fmaf_rn(r, r, acc);
        }
    }
    const double s = block_sum(double(acc));
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[b.x + gd.x * (b.y + gd.y * b.z)] = s;
}

// (hi, lo) += e: TwoSum of the high word and e, the low word folded into the
// error, then renormalised with Fast2Sum.
__device__ __forceinline__ void df_correct_body(const Geom& g, int d3, const float* __restrict__ e,
                                                float* __restrict__ hi, float* __restrict__ lo, dim3 b, dim3 gd) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    for (int k = d3 ? 1 + b.z : 0; k <= (d3 ? g.nz - 2 : 0); k += gd.z) {
        const size_t o = at(g, i, j, k);
        float s, t;
        two_sum(hi[o], e[o], s, t);
        t = __fadd_rn(t, lo[o]);
        float h, l;
        fast_two_sum(s, t, h, l);
        hi[o] = h;
        lo[o] = l;
    }
}

// split a double into hi = fl32(x), lo = fl32(x - hi) at interior nodes (zero when f is absent)
__device__ __forceinline__ void df_split_body(const Geom& g, int d3, const double* __restrict__ f,
                                              float* __restrict__ hi, float* __restrict__ lo, dim3 b, dim3 gd) {
    const int i = 1 + b.x * blockDim.x + threadIdx.x;
    const int j = 1 + b.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    for (int k = d3 ? 1 + b.z : 0; k <= (d3 ? g.nz - 2 : 0); k += gd.z) {
        const size_t o = at(g, i, j, k);
        const double x = f ? f[o] : 0.0;
        const float h = float(x);
        hi[o] = h;
        lo[o] = float(x - double(h));
    }
}

// P = hi + lo over the whole array (grid-stride over gd.x blocks)
__device__ __forceinline__ void df_to_double_body(size_t n, const float* __restrict__ hi,
                                                  const float* __restrict__ lo, double* __restrict__ P, dim3 b,
                                                  dim3 gd) {
    for (size_t o = b.x * size_t(blockDim.x) + threadIdx.x; o < n; o += size_t(gd.x) * blockDim.x)
        P[o] = double(hi[o]) + double(lo[o]);
}

__device__ __forceinline__ void df_copy_plane_body(const Geom& g2, const float* __restrict__ hi2,
                                                   const float* __restrict__ lo2, const Geom& g3,
                                                   float* __restrict__ hi3, float* __restrict__ lo3, dim3 b) {
    const int i = b.x * blockDim.x + threadIdx.x;
    const int j = b.y * blockDim.y + threadIdx.y;
    if (i >= g2.nx || j >= g2.ny) return;
    hi3[at(g3, i, j, 0)] = hi2[at(g2, i, j, 0)];
    lo3[at(g3, i, j, 0)] = lo2[at(g2, i, j, 0)];
}

inline dim3 df_grid(const Geom& g, int d3, int max_blocks) {
    const int gx = (g.nx - 2 + DF_BX - 1) / DF_BX;
    const int gy = (g.ny - 2 + DF_BY - 1) / DF_BY;
    int gz = d3 ? g.nz - 2 : 1;
    if (d3 && max_blocks > 0) {
        const int cap = max_blocks / (gx * gy);
        gz = gz > cap ? (cap > 0 ? cap : 1) : gz;
    }
    if (gz > 65535) gz = 65535;
    return dim3(gx, gy, gz);
}
// norm partials: a few blocks per SM, each covering several planes (see residual_grid)
inline dim3 df_residual_grid(const Geom& g, int d3, int max_blocks) {
    return df_grid(g, d3, max_blocks < 152 * 8 ? max_blocks : 152 * 8);
}
inline dim3 df_plane_grid(const Geom& g2) { return dim3((g2.nx + DF_BX - 1) / DF_BX, (g2.ny + DF_BY - 1) / DF_BY); }
constexpr int DF_TO_DOUBLE_BLOCKS = 152 * 8, DF_TO_DOUBLE_THREADS = 256;

}  // namespace mhs
