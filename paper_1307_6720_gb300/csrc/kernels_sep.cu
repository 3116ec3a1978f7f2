// Exact separable solver of the discrete problems: the inner solver of the
// mixed-precision defect correction, the FP64 direct correction, and the
// coarse-grid solve of the V-cycles.
//
// xi depends on z only (Sect. 2.1, eq. scalar_pot) and the side faces are
// Dirichlet (Sect. 2.2), so the discrete sine vectors
//   s_m(i) = sin(pi m i / (nx - 1)),  m = 1 .. nx-2
// diagonalise the horizontal second differences: on plane k the operator
// cx_k (E + W - 2) + cy_k (N + S - 2) becomes cx_k mu_x(m) + cy_k mu_y(n)
// with mu(m) = -4 sin^2(pi m / (2 (n - 1))).  A = f on one level then splits
// into one tridiagonal system along z per mode (m, n):
//   cz (e[k-1] + e[k+1]) + D_k e[k] = rhat[k],
//   D_k = (alpha^2 - 2 cz) + cx_k mu_x(m) + cy_k mu_y(n),
// and the lower-boundary problem (eq. lower_bound) into a division per mode.
// Every multigrid level is a rediscretisation with the same structure, so
// the same solver applies on any level.  The sine transforms are fast
// transforms (kernels_dst.cu) when nx - 1 and ny - 1 are powers of two, else
// dense products with the (symmetric) sine matrices done as batched GEMMs over
// the planes; the inverse is the same transform scaled by
// (2/(nx-1)) (2/(ny-1)).  In FP32 the solve is accurate to about 1e-6
// relative, which the double-float outer loop of mixed mode then corrects.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "dst_body.cuh"
#include "group.h"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

// C_b = scale A_b B_b (+ C_b): 64 x 64 output tile per block of 256 threads,
// 4 x 4 outputs per thread (rows ty + 16 r, columns tx + 16 c), K staged
// through shared memory 16 at a time; block (bx, by, bz) = (column tile, row
// tile, batch).
constexpr int TM = 64, TN = 64, TK = 16;

template <typename T>
__device__ __forceinline__ void gemm_body(const GemmArgs<T>& g, int bx, int by, int bz) {
    __shared__ T As[TK][TM + 4];
    __shared__ T Bs[TK][TN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = by * TM, col0 = bx * TN;
    const long long b = bz;
    const T* A = g.A + b * g.sA;
    const T* B = g.B + b * g.sB;
    T* C = g.C + b * g.sC;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += TK) {
        // A tile: 64 rows x 16 k (k fastest in global memory)
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int r = e / TK, kk = e % TK;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < g.M && gk < g.K) ? A[gr * g.lda + gk] : T(0);
        }
        // B tile: 16 k x 64 columns (columns fastest)
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            const int kk = e / TN, c = e % TN;
            const int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < g.K && gc < g.N) ? B[gk * g.ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gr = row0 + ty + 16 * r;
        if (gr >= g.M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gc = col0 + tx + 16 * c;
            if (gc < g.N) {
                const T v = g.scale * acc[r][c];
                C[gr * g.ldc + gc] = g.accumulate ? C[gr * g.ldc + gc] + v : v;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs<T> g) {
    gemm_body(g, int(blockIdx.x), int(blockIdx.y), int(blockIdx.z));
}

// Elimination factors of the mode systems of one 3D level, one thread per
// mode (fast index m, slow index n; the layout of the transformed data),
// formed in FP64 from the FP64 plane coefficients and rounded to T:
//   D_k = base_k + c_k^fast mu_fast(m) + c_k^slow mu_slow(n),
//   pivot_1 = D_1, pivot_k = D_k - cz sup_{k-1}, inv_k = 1 / pivot_k,
//   sup_k = cz inv_k,
// with mu(m) = -4 sin^2(pi (m + 1) / (2 (n_nodes - 1))).  ytrans: the fast
// index is the y mode (fast transforms), else the x mode (dense transforms).
template <typename T>
__global__ void sep_pivot_kernel(int nfast, int nslow, int nzi, int nodes_fast, int nodes_slow,
                                 const PlaneCoef<double>* __restrict__ coef, int ytrans, T* __restrict__ inv,
                                 T* __restrict__ sup) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m >= nfast) return;
    const double sf = sinpi(double(m + 1) / (2.0 * (nodes_fast - 1)));
    const double ss = sinpi(double(n + 1) / (2.0 * (nodes_slow - 1)));
    const double af = -4.0 * sf * sf, as = -4.0 * ss * ss;
    const double cz = coef[1].cz;
    const size_t stride = size_t(nfast) * nslow, o = size_t(n) * nfast + m;
    double prev = 0.0;
    for (int k = 0; k < nzi; ++k) {
        const PlaneCoef<double> c = coef[k + 1];
        const double d = ytrans ? c.base + c.cy * af + c.cx * as : c.base + c.cx * af + c.cy * as;
        const double iv = 1.0 / (k ? d - cz * prev : d);
        prev = cz * iv;
        inv[k * stride + o] = T(iv);
        sup[k * stride + o] = T(prev);
    }
}

// One thread per mode (m fast, n slow) of the transformed data t[k][n][m]
// (k = 0 .. nzi-1 standing for planes 1 .. nzi): the mode's tridiagonal
// system along k solved with its precomputed elimination factors,
//   forward  e_k <- (t_k - cz e_{k-1}) inv_k,
//   backward e_k <- e_k - sup_k e_{k+1},
// t overwritten by the solution.  U planes of right-hand sides (and, going
// back, of eliminated values) are loaded before the recursion consumes them,
// so U memory round trips overlap (the factor tables through the read-only
// path); the recursion is an FMA and a multiply per plane.
template <typename T>
__device__ __forceinline__ void thomas_body(const ModeArgs<T>& a, int bx, int by) {
    constexpr int U = 16;
    const int m = bx * blockDim.x + threadIdx.x;
    const int n = by;
    if (m >= a.nfast) return;
    const int nzi = a.nzi;
    const size_t stride = size_t(a.nfast) * a.nslow, o = size_t(n) * a.nfast + m;
    T* tc = a.t + o;
    const T* ic = a.inv + o;
    const T* sc = a.sup + o;
    const T cz = a.coef[1].cz;
    T dp = T(0);
    for (int k0 = 0; k0 < nzi; k0 += U) {
        T rhs[U], iv[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 + q < nzi) {
                rhs[q] = tc[(k0 + q) * stride];
                iv[q] = __ldg(ic + (k0 + q) * stride);
            }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = k0 + q;
            if (k < nzi) {
                dp = (k ? fma(-cz, dp, rhs[q]) : rhs[q]) * iv[q];
                tc[k * stride] = dp;
            }
        }
    }
    T x = dp;
    for (int k0 = nzi - 2; k0 >= 0; k0 -= U) {
        T dd[U], cc[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 - q >= 0) {
                dd[q] = tc[(k0 - q) * stride];
                cc[q] = __ldg(sc + (k0 - q) * stride);
            }
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 - q >= 0) {
                x = fma(-cc[q], x, dd[q]);
                tc[(k0 - q) * stride] = x;
            }
    }
}

template <typename T>
__global__ void sep_thomas_kernel(ModeArgs<T> a) {
    thomas_body(a, int(blockIdx.x), int(blockIdx.y));
}

// The same mode systems with more parallelism, for levels whose planes fit
// shared memory: a block takes 32 consecutive fast modes of one slow index,
// stages their right-hand sides and factors for every plane through shared
// memory (coalesced rows; the tile is padded to 33 columns), and a warp solves
// one mode at a time with its lanes over the planes.  Each recurrence of the
// elimination is affine in its carried value,
//   forward  e_k = a_k e_{k-1} + b_k,  a_k = -cz inv_k (a_0 = 0), b_k = t_k inv_k,
//   backward e_k = alpha_k e_{k+1} + e_k,  alpha_k = -sup_k (0 on the top plane),
// so every lane composes the maps of its run of consecutive planes, a warp
// scan of the composed maps (shuffles) gives each lane the value entering its
// run, and the lane then repeats the sequential steps of its run from it.
template <typename T>
__device__ __forceinline__ void scan_body(const ModeArgs<T>& ma, int bx, int by) {
    extern __shared__ __align__(16) unsigned char scan_smem[];
    const int nfast = ma.nfast, nslow = ma.nslow, nzi = ma.nzi;
    const T* __restrict__ inv = ma.inv;
    const T* __restrict__ sup = ma.sup;
    T* __restrict__ t = ma.t;
    constexpr int W = 33;
    T* st = reinterpret_cast<T*>(scan_smem);   // [nzi][W]: right-hand sides, then solution
    T* si = st + size_t(nzi) * W;              // inverse pivots
    T* ss = si + size_t(nzi) * W;              // eliminated super-diagonals
    const int m0 = bx * 32, n = by;
    const int nc = min(32, nfast - m0);
    const size_t stride = size_t(nfast) * nslow, base = size_t(n) * nfast + m0;
    const T cz = ma.coef[1].cz;
    // rows in batches of R per thread, every load of a batch issued before its
    // values are stored (one memory round trip per batch instead of per row)
    constexpr int R = 8;
    const int c_ld = threadIdx.x & 31, r_ld = threadIdx.x >> 5, rstep = blockDim.x >> 5;
    for (int k0 = r_ld; k0 < nzi; k0 += R * rstep) {
        T vt[R], vi[R], vs[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k = k0 + q * rstep;
            if (k < nzi && c_ld < nc) {
                const size_t gi = k * stride + base + c_ld;
                vt[q] = t[gi];
                vi[q] = __ldg(inv + gi);
                vs[q] = __ldg(sup + gi);
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k = k0 + q * rstep;
            if (k < nzi && c_ld < nc) {
                st[k * W + c_ld] = vt[q];
                si[k * W + c_ld] = vi[q];
                ss[k * W + c_ld] = vs[q];
            }
        }
    }
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int run = (nzi + 31) / 32;
    const int k0 = min(nzi, lane * run), k1 = min(nzi, k0 + run);
    for (int c = warp; c < nc; c += nw) {
        // forward: compose this lane's maps, scan, then the sequential steps
        T A = T(1), B = T(0);
        for (int k = k0; k < k1; ++k) {
            const T iv = si[k * W + c];
            const T a = k ? -cz * iv : T(0);
            B = fma(a, B, st[k * W + c] * iv);
            A = a * A;
        }
        for (int off = 1; off < 32; off <<= 1) {
            const T Ap = __shfl_up_sync(full, A, off), Bp = __shfl_up_sync(full, B, off);
            if (lane >= off) {
                B = fma(A, Bp, B);
                A = A * Ap;
            }
        }
        T d = __shfl_up_sync(full, B, 1);
        if (lane == 0) d = T(0);
        for (int k = k0; k < k1; ++k) {
            const T iv = si[k * W + c];
            d = (k ? fma(-cz, d, st[k * W + c]) : st[k * W + c]) * iv;
            st[k * W + c] = d;
        }
        __syncwarp();
        // backward: the same from the top plane down
        A = T(1);
        B = T(0);
        for (int k = k1 - 1; k >= k0; --k) {
            const T al = k == nzi - 1 ? T(0) : -ss[k * W + c];
            B = fma(al, B, st[k * W + c]);
            A = al * A;
        }
        for (int off = 1; off < 32; off <<= 1) {
            const T An = __shfl_down_sync(full, A, off), Bn = __shfl_down_sync(full, B, off);
            if (lane + off < 32) {
                B = fma(A, Bn, B);
                A = A * An;
            }
        }
        T x = __shfl_down_sync(full, B, 1);
        if (lane == 31) x = T(0);
        for (int k = k1 - 1; k >= k0; --k) {
            x = k == nzi - 1 ? st[k * W + c] : fma(-ss[k * W + c], x, st[k * W + c]);
            st[k * W + c] = x;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nzi * 32; e += blockDim.x) {
        const int k = e >> 5, c = e & 31;
        if (c < nc) t[k * stride + base + c] = st[k * W + c];
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) sep_scan_kernel(ModeArgs<T> a) {
    scan_body(a, int(blockIdx.x), int(blockIdx.y));
}

constexpr size_t SCAN_SMEM_MAX = 200 * 1024;
template <typename T>
size_t scan_smem_bytes(int nzi) { return size_t(3) * size_t(nzi) * 33 * sizeof(T); }

// lower-boundary plane: that = rhat / (cf mu_fast(m) + cs mu_slow(n))
template <typename T>
__device__ __forceinline__ void divide_body(const ModeArgs<T>& a, int bx, int by) {
    const int m = bx * blockDim.x + threadIdx.x;
    const int n = by;
    if (m >= a.nfast) return;
    T& t = a.t[size_t(n) * a.nfast + m];
    t = mode_divide(t, a.cf, a.mufast[m], a.cs, a.muslow[n]);
}

template <typename T>
__global__ void sep_divide_kernel(ModeArgs<T> a) {
    divide_body(a, int(blockIdx.x), int(blockIdx.y));
}

// one stage of every item's separable solve (grouped launches)
template <typename T, int KIND>
__global__ void __launch_bounds__(1024) g_sep_kernel(const GSepItem<T>* items, int n, int fmg_step, int gate) {
    int lb;
    const GSepItem<T>* it = glocate(items, n, gate, fmg_step, lb);
    if (!it) return;
    const int bx = lb % it->gx, by = (lb / it->gx) % it->gy, bz = lb / (it->gx * it->gy);
    if constexpr (KIND == SEP_GEMM) gemm_body(it->st.gemm, bx, by, bz);
    else if constexpr (KIND == SEP_SCAN) scan_body(it->st.mode, bx, by);
    else if constexpr (KIND == SEP_THOMAS) thomas_body(it->st.mode, bx, by);
    else divide_body(it->st.mode, bx, by);
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

// the mode-solve stage on transformed data t (fast index nfast): tridiagonal
// systems along z with the level's elimination factors (3D; a warp scan per
// mode on FP32 levels whose planes fit shared memory, the plain recurrence
// otherwise) or a division per mode (2D)
template <typename T>
SepStage<T> mode_stage(const Geom& g, int dim, const PlaneCoef<T>* coef, const SepTables& tab, int nfast, int nslow,
                       const T* mufast, const T* muslow, bool ytrans, T* t) {
    SepStage<T> s;
    ModeArgs<T>& m = s.mode;
    m.nfast = nfast;
    m.nslow = nslow;
    m.nzi = dim == 3 ? g.nz - 2 : 1;
    m.coef = coef;
    m.t = t;
    if (dim == 3) {
        m.inv = static_cast<const T*>(tab.inv);
        m.sup = static_cast<const T*>(tab.sup);
        // the scan costs about four times the arithmetic of the plain
        // recurrence: FP32 levels only (in FP64 the plain recurrence is faster)
        if (sizeof(T) == 4 && scan_smem_bytes<T>(m.nzi) <= SCAN_SMEM_MAX) {
            s.kind = SEP_SCAN;
            s.threads = 32 * std::min(32, nfast);   // a warp per mode of the block's 32
            s.grid = dim3((nfast + 31) / 32, nslow);
            s.smem = scan_smem_bytes<T>(m.nzi);
            return s;
        }
        s.kind = SEP_THOMAS;
    } else {
        s.kind = SEP_DIVIDE;
        m.mufast = mufast;
        m.muslow = muslow;
        m.cf = T(1.0 / (ytrans ? g.hy * g.hy : g.hx * g.hx));
        m.cs = T(1.0 / (ytrans ? g.hx * g.hx : g.hy * g.hy));
    }
    s.threads = nfast <= 64 ? 64 : 128;
    s.grid = dim3((nfast + s.threads - 1) / s.threads, nslow);
    return s;
}

template <typename T>
SepStage<T> gemm_stage(const GemmArgs<T>& g, int batch) {
    SepStage<T> s;
    s.kind = SEP_GEMM;
    s.gemm = g;
    s.threads = 256;
    s.grid = dim3((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, batch);
    return s;
}

// The stages of A e = f on one level, e = out (stored, or added with
// accumulate), f and out pitched level arrays (interior read / written), t1
// and t2 dense scratch of the interior size (t2 may be the array of f).
// Fast transforms: x lines of f -> t1[k][m][j] (transposed), y lines ->
// t2[k][m][n], mode solves, inverse y -> t1[k][j][m] (transposed), inverse
// x -> out, scaled.
// Dense transforms: t1[k][j][m] = sum_i f[k][j][i] Sx[m][i], t2[k][n][m] =
// sum_j Sy[n][j] t1[k][j][m], mode solves, and back the same way.
template <typename T>
void plan_level(const Geom& g, int dim, const PlaneCoef<T>* coef, const SepTables& tab, const T* f, T* t1, T* t2,
                T* out, bool accumulate, std::vector<SepStage<T>>& stages) {
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = dim == 3 ? g.nz - 2 : 1;
    if (nxi < 1 || nyi < 1 || nzi < 1) return;
    const long long pl = (long long)nxi * nyi;
    const long long off = dim == 3 ? (long long)g.plane + g.px + 1 : (long long)g.px + 1;
    const long long sA = dim == 3 ? (long long)g.plane : 0;
    const T* mux = static_cast<const T*>(tab.mux);
    const T* muy = static_cast<const T*>(tab.muy);
    const T scale = T((2.0 / (g.nx - 1)) * (2.0 / (g.ny - 1)));
    if (tab.twx) {
        auto dst = [&](const DstArgs<T>& a) {
            SepStage<T> s;
            s.kind = SEP_DST;
            s.dst = a;
            dst_shape<T>(s.dst, s.grid, s.threads, s.smem);
            stages.push_back(s);
        };
        const int Lx = g.nx - 1, Ly = g.ny - 1;
        DstArgs<T> a{};
        a.L = Lx; a.log2n = ilog2(Lx); a.lines = nyi; a.planes = nzi; a.tw = tab.twx; a.scale = T(1);
        a.in = f + off; a.in_plane = sA; a.in_line = g.px;
        a.out = t1; a.out_plane = pl; a.out_line = 1; a.out_elem = nyi;
        dst(a);
        DstArgs<T> b{};
        b.L = Ly; b.log2n = ilog2(Ly); b.lines = nxi; b.planes = nzi; b.tw = tab.twy; b.scale = T(1);
        b.in = t1; b.in_plane = pl; b.in_line = nyi;
        b.out = t2; b.out_plane = pl; b.out_line = nyi; b.out_elem = 1;
        dst(b);
        stages.push_back(mode_stage<T>(g, dim, coef, tab, nyi, nxi, muy, mux, true, t2));
        b.in = t2; b.out = t1; b.out_line = 1; b.out_elem = nxi;
        dst(b);
        a.in = t1; a.in_plane = pl; a.in_line = nxi;
        a.out = out + off; a.out_plane = sA; a.out_line = g.px; a.out_elem = 1;
        a.scale = scale;
        a.accumulate = accumulate ? 1 : 0;
        dst(a);
        return;
    }
    const T* Sx = static_cast<const T*>(tab.sx);
    const T* Sy = static_cast<const T*>(tab.sy);
    stages.push_back(gemm_stage<T>(GemmArgs<T>{nyi, nxi, nxi, f + off, g.px, sA, Sx, nxi, 0, t1, nxi, pl, T(1), 0}, nzi));
    stages.push_back(gemm_stage<T>(GemmArgs<T>{nyi, nxi, nyi, Sy, nyi, 0, t1, nxi, pl, t2, nxi, pl, T(1), 0}, nzi));
    stages.push_back(mode_stage<T>(g, dim, coef, tab, nxi, nyi, mux, muy, false, t2));
    stages.push_back(gemm_stage<T>(GemmArgs<T>{nyi, nxi, nyi, Sy, nyi, 0, t2, nxi, pl, t1, nxi, pl, T(1), 0}, nzi));
    stages.push_back(gemm_stage<T>(
        GemmArgs<T>{nyi, nxi, nxi, t1, nxi, pl, Sx, nxi, 0, out + off, g.px, sA, scale, accumulate ? 1 : 0}, nzi));
}

template <typename T>
void launch_stage(const SepStage<T>& s, cudaStream_t st) {
    switch (s.kind) {
    case SEP_DST: launch_dst_stage<T>(s, st); return;
    case SEP_GEMM: gemm_kernel<T><<<s.grid, s.threads, 0, st>>>(s.gemm); break;
    case SEP_SCAN: {
        static bool configured = false;   // per template instance
        if (!configured) {
            MHS_CUDA(cudaFuncSetAttribute(sep_scan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(SCAN_SMEM_MAX)));
            configured = true;
        }
        sep_scan_kernel<T><<<s.grid, s.threads, s.smem, st>>>(s.mode);
        break;
    }
    case SEP_THOMAS: sep_thomas_kernel<T><<<s.grid, s.threads, 0, st>>>(s.mode); break;
    default: sep_divide_kernel<T><<<s.grid, s.threads, 0, st>>>(s.mode); break;
    }
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace

template <typename T>
void launch_sep_stage(const SepStage<T>& s, cudaStream_t st) {
    launch_stage<T>(s, st);
}
template void launch_sep_stage<double>(const SepStage<double>&, cudaStream_t);
template void launch_sep_stage<float>(const SepStage<float>&, cudaStream_t);

namespace {

template <typename T>
void level_solve(mhs_ctx* c, const Geom& g, int dim, const PlaneCoef<T>* coef, const SepTables& tab, const T* f,
                 T* t1, T* t2, T* out, bool accumulate) {
    std::vector<SepStage<T>> stages;
    plan_level<T>(g, dim, coef, tab, f, t1, t2, out, accumulate, stages);
    for (const SepStage<T>& s : stages) launch_stage<T>(s, c->stream);
}

template <typename T>
LevelArrays<T>& arrays_of(Hierarchy& H, int l);
template <>
LevelArrays<double>& arrays_of<double>(Hierarchy& H, int l) { return H.d[l]; }
template <>
LevelArrays<float>& arrays_of<float>(Hierarchy& H, int l) { return H.s[l]; }
template <typename T>
std::vector<SepTables>& tables_of(Hierarchy& H) { return sizeof(T) == 8 ? H.sep64 : H.sep32; }

// elimination factors of level l's mode systems from the current coefficients
template <typename T>
void compute_pivots(mhs_ctx* c, Hierarchy& H, int l, SepTables& t) {
    const Geom& g = H.g[l];
    if (H.dim != 3 || !t.inv) return;
    const bool ytrans = t.twx != nullptr;
    const int nxi = g.nx - 2, nyi = g.ny - 2;
    const int nfast = ytrans ? nyi : nxi, nslow = ytrans ? nxi : nyi;
    const int threads = nfast <= 64 ? 64 : 128;
    sep_pivot_kernel<T><<<dim3((nfast + threads - 1) / threads, nslow), threads, 0, c->stream>>>(
        nfast, nslow, g.nz - 2, ytrans ? g.ny : g.nx, ytrans ? g.nx : g.ny, H.d[l].coef, ytrans ? 1 : 0,
        static_cast<T*>(t.inv), static_cast<T*>(t.sup));
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
const SepTables& tables(Hierarchy& H, int l) {
    std::vector<SepTables>& v = tables_of<T>(H);
    if (size_t(l) >= v.size() || !v[l].ready) throw Error(MHS_ERR_BAD_STATE, "separable solver tables not built");
    return v[l];
}

}  // namespace

bool sep_level_ok(const Geom& g) {
    return (pow2(g.nx - 1) && pow2(g.ny - 1)) || (g.nx <= 66 && g.ny <= 66);
}

// Mode eigenvalues, and twiddles or sine matrices, of level l in T, built once
// (FP64 on the host, rounded to T).  Any level: the dense transforms serve
// whatever the node counts (the mixed-mode finest-level solve of long
// non-power-of-two rows among them); the callers that must stay cheap check
// sep_level_ok first.
template <typename T>
void sep_tables(mhs_ctx* c, Hierarchy& H, int l) {
    std::vector<SepTables>& v = tables_of<T>(H);
    if (v.size() < size_t(H.nlev())) v.resize(H.nlev());
    SepTables& t = v[l];
    if (t.ready) return;
    const Geom& g = H.g[l];
    auto upload = [&](const std::vector<T>& h) {
        void* p = nullptr;
        MHS_CUDA(cudaMalloc(&p, std::max<size_t>(h.size(), 1) * sizeof(T)));
        c->allocations.push_back(p);
        c->dev_bytes += round_up(std::max<size_t>(h.size(), 1) * sizeof(T), 256);
        MHS_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        return p;
    };
    auto mu = [](int n) {
        std::vector<T> m(n - 2);
        for (int q = 1; q <= n - 2; ++q) {
            const double s = std::sin(M_PI * q / (2.0 * (n - 1)));
            m[q - 1] = T(-4.0 * s * s);
        }
        return m;
    };
    auto sine = [](int n) {   // S[m-1][i-1] = sin(pi m i / (n - 1))
        const int ni = n - 2;
        std::vector<T> s(size_t(ni) * ni);
        for (int m = 1; m <= ni; ++m)
            for (int i = 1; i <= ni; ++i) {
                // reduce m i modulo 2 (n - 1) before the sine for an accurate argument
                const long long p = (long long)m * i % (2LL * (n - 1));
                s[size_t(m - 1) * ni + (i - 1)] = T(std::sin(M_PI * double(p) / double(n - 1)));
            }
        return s;
    };
    t.mux = upload(mu(g.nx));
    t.muy = upload(mu(g.ny));
    if (pow2(g.nx - 1) && pow2(g.ny - 1)) {
        size_t tb = 0;
        t.twx = make_twiddles<T>(g.nx - 1, &tb);
        c->allocations.push_back(t.twx);
        c->dev_bytes += round_up(tb, 256);
        t.twy = make_twiddles<T>(g.ny - 1, &tb);
        c->allocations.push_back(t.twy);
        c->dev_bytes += round_up(tb, 256);
    } else {
        t.sx = upload(sine(g.nx));
        t.sy = upload(sine(g.ny));
    }
    if (H.dim == 3 && g.nz > 2) {
        const size_t n = size_t(g.nx - 2) * size_t(g.ny - 2) * size_t(g.nz - 2);
        for (void** p : {&t.inv, &t.sup}) {
            MHS_CUDA(cudaMalloc(p, n * sizeof(T)));
            c->allocations.push_back(*p);
            c->dev_bytes += round_up(n * sizeof(T), 256);
        }
        compute_pivots<T>(c, H, l, t);
    }
    t.ready = true;
}

void sep_refresh(mhs_ctx* c, Hierarchy& H) {
    for (size_t l = 0; l < H.sep64.size(); ++l)
        if (H.sep64[l].ready) compute_pivots<double>(c, H, int(l), H.sep64[l]);
    for (size_t l = 0; l < H.sep32.size(); ++l)
        if (H.sep32[l].ready) compute_pivots<float>(c, H, int(l), H.sep32[l]);
}

template <typename T>
void sep_exact(mhs_ctx* c, Hierarchy& H, int l) {
    LevelArrays<T>& A = arrays_of<T>(H, l);
    const Geom& g = H.g[l];
    const SepTables& tab = tables<T>(H, l);
    if (!(c->opts.flags & MHS_FLAG_STAGED_TRANSFORMS) && tab.twx) {
        // per-plane transforms in thread-block clusters (same results as the staged passes)
        const SepStage<T> ms = mode_stage<T>(g, H.dim, A.coef, tab, g.ny - 2, g.nx - 2, static_cast<const T*>(tab.muy),
                                             static_cast<const T*>(tab.mux), true, A.t);
        if (plane_level_solve<T>(g, H.dim, tab, A.f, A.t, A.u, false, &ms, c->stream)) return;
    }
    level_solve<T>(c, g, H.dim, A.coef, tab, A.f, A.r, A.t, A.u, false);
}

template <typename T>
void sep_exact_plan(mhs_ctx* c, Hierarchy& H, int l, std::vector<SepStage<T>>& stages) {
    (void)c;
    LevelArrays<T>& A = arrays_of<T>(H, l);
    plan_level<T>(H.g[l], H.dim, A.coef, tables<T>(H, l), A.f, A.r, A.t, A.u, false, stages);
}

template <typename T>
void glaunch_sep(const GSepTable<T>& t, int fmg_step, int gate, cudaStream_t st) {
    if (t.n == 0) return;
    switch (t.kind) {
    case SEP_DST: glaunch_dst<T>(t, fmg_step, gate, st); return;
    case SEP_GEMM: g_sep_kernel<T, SEP_GEMM><<<t.blocks, t.threads, 0, st>>>(t.items, t.n, fmg_step, gate); break;
    case SEP_SCAN: {
        static bool configured = false;
        if (!configured) {
            MHS_CUDA(cudaFuncSetAttribute(g_sep_kernel<T, SEP_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(SCAN_SMEM_MAX)));
            configured = true;
        }
        g_sep_kernel<T, SEP_SCAN><<<t.blocks, t.threads, t.smem, st>>>(t.items, t.n, fmg_step, gate);
        break;
    }
    case SEP_THOMAS: g_sep_kernel<T, SEP_THOMAS><<<t.blocks, t.threads, 0, st>>>(t.items, t.n, fmg_step, gate); break;
    default: g_sep_kernel<T, SEP_DIVIDE><<<t.blocks, t.threads, 0, st>>>(t.items, t.n, fmg_step, gate); break;
    }
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void sep_prepare(mhs_ctx* c, int mode) {
    for (Hierarchy* H : {&c->h3, &c->h2}) {
        if (mode == MHS_MIXED) sep_tables<float>(c, *H, 0);
        else if (sep_fp64_available(c)) sep_tables<double>(c, *H, 0);
    }
}

// e = A^{-1} f on the finest FP32 level of H (interior; e's boundary is left
// as it is); the level's r and t arrays are scratch.
void sep_solve(mhs_ctx* c, Hierarchy& H) { sep_exact<float>(c, H, 0); }

bool sep_fp64_available(const mhs_ctx* c) { return sep_level_ok(c->h3.g[0]); }

// FP64 mode: P += A^{-1} r on the finest level of H, r the residual of the
// latest check (in A.r, consumed), the level's twin t as scratch.
void sep_correct64(mhs_ctx* c, Hierarchy& H) {
    LevelArrays<double>& A = H.d[0];
    level_solve<double>(c, H.g[0], H.dim, A.coef, tables<double>(H, 0), A.r, A.t, A.r, A.u, true);
}

template void sep_tables<double>(mhs_ctx*, Hierarchy&, int);
template void sep_tables<float>(mhs_ctx*, Hierarchy&, int);
template void sep_exact<double>(mhs_ctx*, Hierarchy&, int);
template void sep_exact<float>(mhs_ctx*, Hierarchy&, int);
template void sep_exact_plan<double>(mhs_ctx*, Hierarchy&, int, std::vector<SepStage<double>>&);
template void sep_exact_plan<float>(mhs_ctx*, Hierarchy&, int, std::vector<SepStage<float>>&);
template void glaunch_sep<double>(const GSepTable<double>&, int, int, cudaStream_t);
template void glaunch_sep<float>(const GSepTable<float>&, int, int, cudaStream_t);

}  // namespace mhs
