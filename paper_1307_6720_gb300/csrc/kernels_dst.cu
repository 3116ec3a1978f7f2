// Fast discrete sine transforms (DST-I) for the separable solver.
//
// For a line x_1 .. x_{N-1} (N = L a power of two) the transform is
//   X_m = sum_i x_i sin(pi m i / N),  m = 1 .. N-1;
// the inverse is the same transform scaled by 2/N.  With s_i = x_i + x_{N-i},
// d_i = x_i - x_{N-i} (x_0 = x_N = 0) form the real sequence
//   y_0 = 0,  y_i = sin(pi i / N) s_i + d_i / 2,  i = 1 .. N-1,
// and its DFT Y_k = R_k + i I_k (length N).  Because s is even and d odd
// about N/2, and sin(pi i / N) cos(2 pi i k / N) = (sin(pi i (2k+1)/N) -
// sin(pi i (2k-1)/N)) / 2, the real and imaginary parts give
//   X_{2k} = -I_k,   X_{2k+1} - X_{2k-1} = R_k  (X_{-1} = -X_1),
// so the even outputs come directly and the odd ones as the prefix sums
// X_{2k+1} = R_0/2 + R_1 + ... + R_k.  Two real lines a and b share one
// complex FFT of length N as z = y_a + i y_b; with Z its transform,
// Y_a,k = (Z_k + conj Z_{N-k}) / 2 and Y_b,k = (Z_k - conj Z_{N-k}) / (2i).
// This is half the FFT length of transforming the odd extensions (length
// 2N) directly, which FP64 transforms use (the FP64 pipe is their bound).
// FP32 transforms keep the odd extensions: y_0 = 0, y_i = x_i, y_N = 0,
// y_{2N-i} = -x_i transforms to -2i X_m, so with two lines in one complex FFT
// of length 2N, X_a = -Im(Z_m)/2 and X_b = Re(Z_m)/2; the prefix sums of the
// half-length form lose about a factor of three in accuracy, which in FP32
// slows the mixed-precision outer loop, while these short FP32 transforms are
// bound by latency, not arithmetic.
//
// One block handles P pairs of lines in shared memory: the pairs' z are
// stored in bit-reversed order, then the log2 N radix-2 decimation-in-time
// stages (Cooley and Tukey) run three at a time in registers (radix-8
// passes), with twiddles e^{-2 pi i q / (2N)} from a table staged in shared
// memory (the FFT of length N uses its even entries).  A warp per line then
// forms R and I from Z_k and Z_{N-k} and the prefix sums by a warp scan
// (each lane a run of consecutive k), into a staging area from which the
// block writes the lines (element m of line l at out + l * out_line + m) or
// the transposed lines (at out + m * out_elem + l), consecutive threads on
// consecutive addresses.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "group.h"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
    using type = float2;
};
template <>
struct Cplx<double> {
    using type = double2;
};

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// shared-memory position of point i of a pair: one padding element per 8
// points, which spreads the first passes' strided accesses over the banks
__device__ __forceinline__ int phys(int i) { return i + (i >> 3); }

template <typename C>
__device__ __forceinline__ void bfly(C& a, C& b, const C w) {
    const C t = C{b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x};
    b = C{a.x - t.x, a.y - t.y};
    a = C{a.x + t.x, a.y + t.y};
}

// Q consecutive radix-2 decimation-in-time stages (half-sizes h = 2^s ..
// 2^(s+Q-1)) in registers: each unit holds the 2^Q points base + j h that
// those stages combine; sub-stage t pairs j with j + 2^t under the twiddle
// e^{-2 pi i rr / (2H)}, H = h 2^t, rr = r + (j mod 2^t) h, taken from the
// table e^{-2 pi i q / (2L)} at q = rr L / H.
template <int Q, typename C>
__device__ __forceinline__ void fft_pass(C* z, const C* tw, int P, int PS, int bits, int L, int s) {
    constexpr int R = 1 << Q;
    const int h = 1 << s, ub = bits - Q;
    const int units = P << ub;
    for (int e = threadIdx.x; e < units; e += blockDim.x) {
        const int pair = e >> ub, u = e & ((1 << ub) - 1);
        const int r = u & (h - 1);
        const int base = ((u >> s) << (Q + s)) + r;
        C* zp = z + pair * PS;
        C v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = zp[phys(base + j * h)];
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            const int d = 1 << t;
            const int tstride = L >> (s + t);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (j & d) continue;
                const int rr = r + (j & (d - 1)) * h;
                bfly(v[j], v[j + d], tw[rr * tstride]);
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) zp[phys(base + j * h)] = v[j];
    }
}

// The first three stages (half-sizes 1, 2, 4) as one radix-8 pass whose
// twiddles are the eighth roots of unity e^{-i pi q / 4}: multiplications by
// 1 and -i become additions and swaps, those by (+-1 - i)/sqrt(2) two
// additions and two multiplications.
template <typename C>
__device__ __forceinline__ void fft_first(C* z, int P, int PS, int bits) {
    using T = decltype(C{}.x);
    const T c = T(0.70710678118654752440);
    const int ub = bits - 3;
    const int units = P << ub;
    for (int e = threadIdx.x; e < units; e += blockDim.x) {
        const int pair = e >> ub, u = e & ((1 << ub) - 1);
        const int base = u << 3;
        C* zp = z + pair * PS;
        C v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = zp[phys(base + j)];
        auto add = [](C& a, C& b, const C t) {   // a, b <- a + t, a - t
            b = C{a.x - t.x, a.y - t.y};
            a = C{a.x + t.x, a.y + t.y};
        };
        // half-size 1: twiddle 1
#pragma unroll
        for (int j = 0; j < 8; j += 2) add(v[j], v[j + 1], v[j + 1]);
        // half-size 2: twiddles 1, -i
        add(v[0], v[2], v[2]);
        add(v[4], v[6], v[6]);
        add(v[1], v[3], C{v[3].y, -v[3].x});
        add(v[5], v[7], C{v[7].y, -v[7].x});
        // half-size 4: twiddles 1, (1 - i)/sqrt2, -i, (-1 - i)/sqrt2
        add(v[0], v[4], v[4]);
        add(v[1], v[5], C{(v[5].x + v[5].y) * c, (v[5].y - v[5].x) * c});
        add(v[2], v[6], C{v[6].y, -v[6].x});
        add(v[3], v[7], C{(v[7].y - v[7].x) * c, -(v[7].x + v[7].y) * c});
#pragma unroll
        for (int j = 0; j < 8; ++j) zp[phys(base + j)] = v[j];
    }
}

// complex elements between the pairs of a block: the padded F points of the
// FFT, made odd so that consecutive pairs start on different banks
__host__ __device__ inline int pair_stride(int F) {
    const int padded = (F - 1) + ((F - 1) >> 3) + 1;
    return padded | 1;
}

// block (bx, by) = (line block, plane) of the transform a; every thread of
// the block calls it
template <typename T>
__device__ __forceinline__ void dst_body(const DstArgs<T>& a, int bx, int by) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char dst_smem[];
    constexpr bool HALF = sizeof(T) == 8;              // half-length form (FP64) or odd extensions (FP32)
    const int N = a.L, H = N / 2;
    const int F = HALF ? N : 2 * N, bits = HALF ? a.log2n : a.log2n + 1;   // FFT length, log2
    const int PS = pair_stride(F);
    const int P = a.pairs;
    C* z = reinterpret_cast<C*>(dst_smem);            // P pairs, PS points apart
    C* tw = z + P * PS;                                // twiddle table, L entries
    T* ob = reinterpret_cast<T*>(tw + a.L);            // results: 2P lines of N - 1
    const int plane = by;
    const int line0 = bx * 2 * P;                     // first line of the block in its plane
    const int nl = min(2 * P, a.lines - line0);       // lines of the block
    const T* in = a.in + plane * a.in_plane + (long long)line0 * a.in_line;
    const C* twg = static_cast<const C*>(a.tw);
    for (int e = threadIdx.x; e < a.L; e += blockDim.x) tw[e] = twg[e];
    // y_0 = 0 (and, odd extensions, y_N = 0 at bit-reversed position 1) of
    // every pair; a pair with one line has a zero imaginary part
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        z[p * PS + phys(0)] = C{T(0), T(0)};
        if (!HALF) z[p * PS + phys(1)] = C{T(0), T(0)};
    }
    if (nl & 1)
        for (int e = threadIdx.x; e < F; e += blockDim.x) reinterpret_cast<T*>(&z[(nl >> 1) * PS + phys(e)])[1] = T(0);
    __syncthreads();
    // y_i and y_{N-i} from x_i and x_{N-i} (i = 1 .. N/2) into bit-reversed
    // positions; element e of the block's nl * N/2 is (line e / (N/2), i);
    // U pairs of loads per thread are in flight before their values are used
    if (HALF) {
        constexpr int U = 4;
        const int total = nl * H;
        for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
            T xi[U], xr[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / H, i = e - l * H + 1;
                    const T* src = in + (long long)l * a.in_line;
                    xi[q] = src[i - 1];
                    xr[q] = src[N - i - 1];
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / H, i = e - l * H + 1;
                    const T sm = xi[q] + xr[q], df = xi[q] - xr[q];
                    const T t = -tw[i].y * sm;   // sin(pi i / N) s_i
                    C* zp = z + (l >> 1) * PS;
                    reinterpret_cast<T*>(&zp[phys(bitrev(i, bits))])[l & 1] = fma(T(0.5), df, t);
                    reinterpret_cast<T*>(&zp[phys(bitrev(N - i, bits))])[l & 1] = fma(T(-0.5), df, t);
                }
            }
        }
    } else {
        // odd extensions: x_i at i and -x_i at 2N - i (element e = l (N-1) + i - 1)
        constexpr int U = 8;
        const int M = N - 1, total = nl * M;
        for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
            T v[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / M, i = e - l * M;
                    v[q] = in[(long long)l * a.in_line + i];
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / M, i = e - l * M + 1;
                    C* zp = z + (l >> 1) * PS;
                    reinterpret_cast<T*>(&zp[phys(bitrev(i, bits))])[l & 1] = v[q];
                    reinterpret_cast<T*>(&zp[phys(bitrev(F - i, bits))])[l & 1] = -v[q];
                }
            }
        }
    }
    __syncthreads();
    // FFT of length N: radix-8 passes (the first with constant twiddles), the
    // remaining one or two stages last
    int s = 0;
    if (bits >= 3) {
        fft_first(z, P, PS, bits);
        __syncthreads();
        s = 3;
    }
    for (; s + 3 <= bits; s += 3) {
        fft_pass<3>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    }
    if (bits - s == 2) {
        fft_pass<2>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    } else if (bits - s == 1) {
        fft_pass<1>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    }
    // a warp per line: R_k, I_k from Z_k and Z_{N-k}; X_{2k} = -I_k and the
    // prefix sums X_{2k+1} = R_0/2 + R_1 + .. + R_k (lane runs of `per` k's,
    // then a warp scan of the run totals)
    if (HALF) {
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        const int per = (H + 31) / 32, j0 = lane * per;
        for (int l = warp; l < nl; l += nwarps) {
            const C* zp = z + (l >> 1) * PS;
            const int comp = l & 1;
            T* o = ob + l * N;
            auto rk = [&](int j, T& R, T& I) {
                const C zk = zp[phys(j)], zr = zp[phys((N - j) & (N - 1))];
                R = T(0.5) * (comp ? zk.y + zr.y : zk.x + zr.x);
                I = T(0.5) * (comp ? zr.x - zk.x : zk.y - zr.y);
                if (j == 0) R *= T(0.5);
            };
            T run = T(0);
            for (int q = 0; q < per; ++q) {
                const int j = j0 + q;
                if (j < H) {
                    T R, I;
                    rk(j, R, I);
                    run += R;
                }
            }
            T incl = run;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const T v = __shfl_up_sync(full, incl, off);
                if (lane >= off) incl += v;
            }
            T acc = incl - run;
            for (int q = 0; q < per; ++q) {
                const int j = j0 + q;
                if (j < H) {
                    T R, I;
                    rk(j, R, I);
                    acc += R;
                    o[2 * j] = acc;              // X_{2j+1}
                    if (j >= 1) o[2 * j - 1] = -I;   // X_{2j}
                }
            }
        }
    } else {
        // odd extensions: X_a = -Im(Z_m)/2, X_b = Re(Z_m)/2
        const int M = N - 1, total = nl * M;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int l = e / M, m = e - l * M + 1;
            const C zm = z[(l >> 1) * PS + phys(m)];
            ob[l * N + m - 1] = (l & 1) ? T(0.5) * zm.x : T(-0.5) * zm.y;
        }
    }
    __syncthreads();
    // the block's nl * (N - 1) results, scaled, flattened so that consecutive
    // threads write consecutive addresses: line layout (m fastest) or
    // transposed (line fastest)
    const int M = N - 1;
    T* out = a.out + plane * a.out_plane;
    const int total = nl * M;
    const bool lines_out = a.out_elem == 1;
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
        T v[U], old[U];
        long long at[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < total) {
                int l, m;
                if (lines_out) {
                    l = e / M;
                    m = e - l * M;
                } else {
                    m = e / nl;
                    l = e - m * nl;
                }
                v[q] = a.scale * ob[l * N + m];
                at[q] = lines_out ? (long long)(line0 + l) * a.out_line + m : (long long)m * a.out_elem + line0 + l;
                if (a.accumulate) old[q] = out[at[q]];
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < total) out[at[q]] = a.accumulate ? old[q] + v[q] : v[q];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) dst_kernel(DstArgs<T> a) {
    dst_body(a, int(blockIdx.x), int(blockIdx.y));
}

// one stage of every item's separable solve (grouped launch)
template <typename T>
__global__ void __launch_bounds__(256) g_dst_kernel(const GSepItem<T>* items, int n, int fmg_step, int gate) {
    int lb;
    const GSepItem<T>* it = glocate(items, n, gate, fmg_step, lb);
    if (!it) return;
    dst_body(it->st.dst, lb % it->gx, lb / it->gx);
}

}  // namespace

// shared memory of a block: P pairs of FFT points (N in FP64, 2N in FP32)
// with one padding element per 8, the twiddle table of L entries, and the
// results of 2P lines
template <typename T>
int fft_length(int L) { return sizeof(T) == 8 ? L : 2 * L; }

template <typename T>
size_t dst_smem_bytes(int L, int P) {
    return (size_t(P) * size_t(pair_stride(fft_length<T>(L))) + size_t(L)) * 2 * sizeof(T) +
           size_t(2 * P) * size_t(L) * sizeof(T);
}

template <typename T>
int dst_pairs(int L) {
    // up to 16 pairs per block within 48 KB of shared memory (several blocks per
    // SM), but at least 4 pairs (up to 96 KB) where that budget would leave
    // fewer, and fewer pairs only for lines that need it
    int p = 16;
    while (p > 4 && dst_smem_bytes<T>(L, p) > 48 * 1024) p >>= 1;
    while (p > 1 && dst_smem_bytes<T>(L, p) > 96 * 1024) p >>= 1;
    return p;
}

// opt-in shared memory per block of the GPU (227 KB); one pair of the
// longest lines (L = 4096, FP64) takes 205 KB
constexpr size_t DST_SMEM_MAX = 227 * 1024;

template <typename T>
void dst_shape(DstArgs<T>& a, dim3& grid, int& threads, size_t& smem) {
    a.pairs = dst_pairs<T>(a.L);
    // small transforms (coarse levels): fewer pairs per block, so that the
    // blocks cover every SM about twice
    auto blocks = [&](int p) { return size_t((a.lines + 2 * p - 1) / (2 * p)) * size_t(a.planes); };
    while (a.pairs > 2 && blocks(a.pairs) < 2 * 152) a.pairs >>= 1;
    // one thread per radix-8 unit of the block's pairs, 64 .. 256
    const int units = a.pairs * std::max(1, fft_length<T>(a.L) / 8);
    threads = std::min(256, std::max(64, (units + 31) / 32 * 32));
    smem = dst_smem_bytes<T>(a.L, a.pairs);
    if (smem > DST_SMEM_MAX) throw Error(MHS_ERR_INVALID_ARG, "sine transform lines too long for shared memory");
    grid = dim3((a.lines + 2 * a.pairs - 1) / (2 * a.pairs), a.planes);
}

template <typename T>
void launch_dst_stage(const SepStage<T>& s, cudaStream_t st) {
    static bool configured = false;   // per template instance
    if (!configured) {
        MHS_CUDA(cudaFuncSetAttribute(dst_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(DST_SMEM_MAX)));
        configured = true;
    }
    dst_kernel<T><<<s.grid, s.threads, s.smem, st>>>(s.dst);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template <typename T>
void glaunch_dst(const GSepTable<T>& t, int fmg_step, int gate, cudaStream_t st) {
    if (t.n == 0) return;
    static bool configured = false;
    if (!configured) {
        MHS_CUDA(
            cudaFuncSetAttribute(g_dst_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(DST_SMEM_MAX)));
        configured = true;
    }
    g_dst_kernel<T><<<t.blocks, t.threads, t.smem, st>>>(t.items, t.n, fmg_step, gate);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

// twiddles e^{-2 pi i q / (2L)}, q < L, computed in FP64
template <typename T>
void* make_twiddles(int L) {
    using C = typename Cplx<T>::type;
    std::vector<C> tw(L);
    for (int q = 0; q < L; ++q) {
        const double ang = -M_PI * double(q) / double(L);
        tw[q] = C{T(std::cos(ang)), T(std::sin(ang))};
    }
    void* p = nullptr;
    MHS_CUDA(cudaMalloc(&p, tw.size() * sizeof(C)));
    MHS_CUDA(cudaMemcpy(p, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice));
    return p;
}

template void dst_shape<float>(DstArgs<float>&, dim3&, int&, size_t&);
template void dst_shape<double>(DstArgs<double>&, dim3&, int&, size_t&);
template void launch_dst_stage<float>(const SepStage<float>&, cudaStream_t);
template void launch_dst_stage<double>(const SepStage<double>&, cudaStream_t);
template void glaunch_dst<float>(const GSepTable<float>&, int, int, cudaStream_t);
template void glaunch_dst<double>(const GSepTable<double>&, int, int, cudaStream_t);
template void* make_twiddles<float>(int);
template void* make_twiddles<double>(int);

}  // namespace mhs
