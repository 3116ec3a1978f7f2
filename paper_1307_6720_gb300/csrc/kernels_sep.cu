// Exact separable solver of the discrete problems (an alternative inner
// solver for the mixed-precision defect correction).
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
// The sine transforms are fast transforms (kernels_dst.cu) when nx - 1 and
// ny - 1 are powers of two, else dense products with the (symmetric) sine
// matrices done as batched FP32 GEMMs over the planes; the inverse is the
// same transform scaled by (2/(nx-1)) (2/(ny-1)).  In FP32 the solve is accurate to
// about 1e-6 relative, which the double-float outer loop of mixed mode then
// corrects: each outer step cuts the error by about that factor.
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

// C_b = scale * A_b * B_b for b < batch, row-major with leading dimensions
// and batch strides (0: shared by the batch).  64 x 64 output tile per block
// of 256 threads, 4 x 4 outputs per thread (rows ty + 16 r, columns tx + 16 c),
// K staged through shared memory 16 at a time.
struct GemmArgs {
    int M, N, K;
    const float* A;
    long long lda, sA;
    const float* B;
    long long ldb, sB;
    float* C;
    long long ldc, sC;
    float scale;
};

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) sgemm_kernel(GemmArgs g) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const long long b = blockIdx.z;
    const float* A = g.A + b * g.sA;
    const float* B = g.B + b * g.sB;
    float* C = g.C + b * g.sC;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += TK) {
        // A tile: 64 rows x 16 k (k fastest in global memory), 4 elements per thread
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int r = e / TK, kk = e % TK;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < g.M && gk < g.K) ? A[gr * g.lda + gk] : 0.f;
        }
        // B tile: 16 k x 64 columns (columns fastest)
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            const int kk = e / TN, c = e % TN;
            const int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < g.K && gc < g.N) ? B[gk * g.ldb + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bb[c], acc[r][c]);
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
            if (gc < g.N) C[gr * g.ldc + gc] = g.scale * acc[r][c];
        }
    }
}

void sgemm(const GemmArgs& g, int batch, cudaStream_t st) {
    const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, batch);
    sgemm_kernel<<<grid, 256, 0, st>>>(g);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

// One thread per mode (n, m) of the transformed data t[k][n][m] (k = 0 ..
// nzi-1 standing for planes 1 .. nzi): Thomas elimination along k with the
// mode's diagonal, the eliminated super-diagonal kept in w; t is overwritten
// by the solution.
// (ytrans: the fast index is the y mode, the layout [k][m][n] of the FFT path)
template <typename T>
__global__ void sep_thomas_kernel(int nxi, int nyi, int nzi, const PlaneCoef<T>* __restrict__ coef,
                                  const T* __restrict__ mux, const T* __restrict__ muy, T base, T cz,
                                  T* __restrict__ t, T* __restrict__ w, int ytrans) {
    // U planes of right-hand sides (and, going back, of eliminated values)
    // are loaded before the recursion consumes them, so U memory round trips
    // overlap; the recursion itself is a chain of a few FMAs per plane
    constexpr int U = 8;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m >= nxi) return;
    const size_t stride = size_t(nxi) * nyi;
    T* tc = t + size_t(n) * nxi + m;
    T* wc = w + size_t(n) * nxi + m;
    const T ax = mux[m], ay = muy[n];
    T cp = T(0), dp = T(0);
    for (int k0 = 0; k0 < nzi; k0 += U) {
        T rhs[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 + q < nzi) rhs[q] = tc[(k0 + q) * stride];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = k0 + q;
            if (k < nzi) {
                const PlaneCoef<T> c = coef[k + 1];
                const T d = ytrans ? base + c.cy * ax + c.cx * ay : base + c.cx * ax + c.cy * ay;
                const T piv = k ? fma(-cz, cp, d) : d;
                const T inv = T(1) / piv;
                dp = (k ? fma(-cz, dp, rhs[q]) : rhs[q]) * inv;
                cp = cz * inv;
                tc[k * stride] = dp;
                wc[k * stride] = cp;
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
                cc[q] = wc[(k0 - q) * stride];
            }
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 - q >= 0) {
                x = fma(-cc[q], x, dd[q]);
                tc[(k0 - q) * stride] = x;
            }
    }
}

// lower-boundary plane: that = rhat / (cx mu_x(m) + cy mu_y(n))
template <typename T>
__global__ void sep_divide_kernel(int nxi, int nyi, T cx, T cy, const T* __restrict__ mux, const T* __restrict__ muy,
                                  T* __restrict__ t) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m >= nxi) return;
    t[size_t(n) * nxi + m] /= cx * mux[m] + cy * muy[n];
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

// A e = f on one level through fast sine transforms (nx - 1, ny - 1 powers
// of two): x lines of f -> t1[k][m][j] (transposed), y lines -> t2[k][m][n],
// mode solves (t1 as scratch), inverse y -> t1[k][j][m] (transposed), inverse
// x -> out, scaled, stored or added (accumulate).  f and out are pitched level
// arrays (interior read / written); t2 may be the array of f.
template <typename T>
void sep_fft(mhs_ctx* c, const Geom& g, int dim, const PlaneCoef<T>* coef, const T* f, T* t1, T* t2, T* out,
             bool accumulate, const void* twx, const void* twy, const T* mux, const T* muy) {
    cudaStream_t st = c->stream;
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = dim == 3 ? g.nz - 2 : 1;
    const long long pl = (long long)nxi * nyi;
    const long long off = dim == 3 ? (long long)g.plane + g.px + 1 : (long long)g.px + 1;
    const long long sA = dim == 3 ? (long long)g.plane : 0;
    const int Lx = g.nx - 1, Ly = g.ny - 1;
    DstArgs<T> a;
    a.L = Lx; a.log2n = ilog2(2 * Lx); a.lines = nyi; a.planes = nzi; a.tw = twx;
    a.in = f + off; a.in_plane = sA; a.in_line = g.px;
    a.out = t1; a.out_plane = pl; a.out_line = 1; a.out_elem = nyi;
    launch_dst<T>(a, st);
    DstArgs<T> b;
    b.L = Ly; b.log2n = ilog2(2 * Ly); b.lines = nxi; b.planes = nzi; b.tw = twy;
    b.in = t1; b.in_plane = pl; b.in_line = nyi;
    b.out = t2; b.out_plane = pl; b.out_line = nyi; b.out_elem = 1;
    launch_dst<T>(b, st);
    if (dim == 3) {
        // diagonal base alpha^2 - 2 cz in FP64, so that it does not cancel against cx, cy
        const double czd = 1.0 / (g.hz * g.hz);
        sep_thomas_kernel<T><<<dim3((nyi + 127) / 128, nxi), 128, 0, st>>>(
            nyi, nxi, nzi, coef, muy, mux, T(c->alpha * c->alpha - 2.0 * czd), T(czd), t2, t1, 1);
    } else {
        sep_divide_kernel<T><<<dim3((nyi + 127) / 128, nxi), 128, 0, st>>>(
            nyi, nxi, T(1.0 / (g.hy * g.hy)), T(1.0 / (g.hx * g.hx)), muy, mux, t2);
    }
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    b.in = t2; b.out = t1; b.out_line = 1; b.out_elem = nxi;
    launch_dst<T>(b, st);
    a.in = t1; a.in_plane = pl; a.in_line = nxi;
    a.out = out + off; a.out_plane = sA; a.out_line = g.px; a.out_elem = 1;
    a.scale = T((2.0 / (g.nx - 1)) * (2.0 / (g.ny - 1)));
    a.accumulate = accumulate ? 1 : 0;
    launch_dst<T>(a, st);
}

}  // namespace

// Sine matrices and mode eigenvalues of a grid (FP32, device), built once.
void sep_prepare(mhs_ctx* c) {
    if (c->sep.sx) return;
    auto alloc = [&](size_t n) {
        float* p = nullptr;
        MHS_CUDA(cudaMalloc(&p, n * sizeof(float)));
        c->allocations.push_back(p);
        return p;
    };
    auto sine = [](int n) {   // S[m-1][i-1] = sin(pi m i / (n - 1)), FP64 then rounded
        const int ni = n - 2;
        std::vector<float> s(size_t(ni) * ni);
        for (int m = 1; m <= ni; ++m)
            for (int i = 1; i <= ni; ++i) {
                // reduce m i modulo 2 (n - 1) before the sine for an accurate argument
                const long long p = (long long)m * i % (2LL * (n - 1));
                s[size_t(m - 1) * ni + (i - 1)] = float(std::sin(M_PI * double(p) / double(n - 1)));
            }
        return s;
    };
    auto mu = [](int n) {
        std::vector<float> v(n - 2);
        for (int m = 1; m <= n - 2; ++m) {
            const double s = std::sin(M_PI * m / (2.0 * (n - 1)));
            v[m - 1] = float(-4.0 * s * s);
        }
        return v;
    };
    const std::vector<float> sx = sine(c->nx), sy = sine(c->ny), mx = mu(c->nx), my = mu(c->ny);
    c->sep.sx = alloc(sx.size());
    c->sep.sy = alloc(sy.size());
    c->sep.mux = alloc(mx.size());
    c->sep.muy = alloc(my.size());
    MHS_CUDA(cudaMemcpy(c->sep.sx, sx.data(), sx.size() * sizeof(float), cudaMemcpyHostToDevice));
    MHS_CUDA(cudaMemcpy(c->sep.sy, sy.data(), sy.size() * sizeof(float), cudaMemcpyHostToDevice));
    MHS_CUDA(cudaMemcpy(c->sep.mux, mx.data(), mx.size() * sizeof(float), cudaMemcpyHostToDevice));
    MHS_CUDA(cudaMemcpy(c->sep.muy, my.data(), my.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (pow2(c->nx - 1) && pow2(c->ny - 1)) {
        c->sep.twx = make_twiddles<float>(c->nx - 1);
        c->allocations.push_back(c->sep.twx);
        c->sep.twy = make_twiddles<float>(c->ny - 1);
        c->allocations.push_back(c->sep.twy);
    }
}

// e = A^{-1} f on the finest FP32 level of H (interior; e's boundary is left
// as it is), through the sine transforms; the level's r and t arrays are
// scratch.
void sep_solve(mhs_ctx* c, Hierarchy& H) {
    const Geom& g = H.g[0];
    LevelArrays<float>& A = H.s[0];
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = H.dim == 3 ? g.nz - 2 : 1;
    if (nxi < 1 || nyi < 1 || nzi < 1) return;
    cudaStream_t st = c->stream;
    const long long pl = (long long)nxi * nyi;     // one transformed plane
    float* t1 = A.r;
    float* t2 = A.t;
    const long long off = H.dim == 3 ? (long long)g.plane + g.px + 1 : (long long)g.px + 1;
    const long long sA = H.dim == 3 ? (long long)g.plane : 0;
    const float scale = float((2.0 / (g.nx - 1)) * (2.0 / (g.ny - 1)));
    if (c->sep.twx) {
        sep_fft<float>(c, g, H.dim, A.coef, A.f, t1, t2, A.u, false, c->sep.twx, c->sep.twy, c->sep.mux, c->sep.muy);
        return;
    }
    // along x: t1[k][j][m] = sum_i f[k][j][i] Sx[m][i]
    sgemm(GemmArgs{nyi, nxi, nxi, A.f + off, g.px, sA, c->sep.sx, nxi, 0, t1, nxi, pl, 1.f}, nzi, st);
    // along y: t2[k][n][m] = sum_j Sy[n][j] t1[k][j][m]
    sgemm(GemmArgs{nyi, nxi, nyi, c->sep.sy, nyi, 0, t1, nxi, pl, t2, nxi, pl, 1.f}, nzi, st);
    if (H.dim == 3) {
        // mode systems along z; base = alpha^2 - 2 cz from the FP64 coefficients
        const double hz = g.hz, czd = 1.0 / (hz * hz);
        const float base = float(c->alpha * c->alpha - 2.0 * czd);
        sep_thomas_kernel<float><<<dim3((nxi + 127) / 128, nyi), 128, 0, st>>>(nxi, nyi, nzi, A.coef, c->sep.mux,
                                                                        c->sep.muy, base, float(czd), t2, t1, 0);
    } else {
        const float cx = float(1.0 / (g.hx * g.hx)), cy = float(1.0 / (g.hy * g.hy));
        sep_divide_kernel<float><<<dim3((nxi + 127) / 128, nyi), 128, 0, st>>>(nxi, nyi, cx, cy, c->sep.mux, c->sep.muy, t2);
    }
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    // inverse along y: t1[k][j][m] = sum_n Sy[j][n] t2[k][n][m]
    sgemm(GemmArgs{nyi, nxi, nyi, c->sep.sy, nyi, 0, t2, nxi, pl, t1, nxi, pl, 1.f}, nzi, st);
    // inverse along x with the normalisation: e[k][j][i] = s sum_m t1[k][j][m] Sx[m][i]
    sgemm(GemmArgs{nyi, nxi, nxi, t1, nxi, pl, c->sep.sx, nxi, 0, A.u + off, g.px, sA, scale}, nzi, st);
}

bool sep_fp64_available(const mhs_ctx* c) { return pow2(c->nx - 1) && pow2(c->ny - 1); }

// FP64 mode: mode eigenvalues and twiddles in FP64 (fast transforms only)
void sep_prepare64(mhs_ctx* c) {
    if (c->sep.mux64 || !sep_fp64_available(c)) return;
    auto mu = [](int n) {
        std::vector<double> v(n - 2);
        for (int m = 1; m <= n - 2; ++m) {
            const double s = std::sin(M_PI * m / (2.0 * (n - 1)));
            v[m - 1] = -4.0 * s * s;
        }
        return v;
    };
    for (int axis = 0; axis < 2; ++axis) {
        const std::vector<double> v = mu(axis == 0 ? c->nx : c->ny);
        double* p = nullptr;
        MHS_CUDA(cudaMalloc(&p, v.size() * sizeof(double)));
        c->allocations.push_back(p);
        MHS_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        (axis == 0 ? c->sep.mux64 : c->sep.muy64) = p;
    }
    c->sep.twx64 = make_twiddles<double>(c->nx - 1);
    c->allocations.push_back(c->sep.twx64);
    c->sep.twy64 = make_twiddles<double>(c->ny - 1);
    c->allocations.push_back(c->sep.twy64);
}

// FP64 mode: P += A^{-1} r on the finest level of H, r the residual of the
// latest check (in A.r, consumed), the level's twin t as scratch
void sep_correct64(mhs_ctx* c, Hierarchy& H) {
    LevelArrays<double>& A = H.d[0];
    sep_fft<double>(c, H.g[0], H.dim, A.coef, A.r, A.t, A.r, A.u, true, c->sep.twx64, c->sep.twy64, c->sep.mux64,
                    c->sep.muy64);
}

}  // namespace mhs
