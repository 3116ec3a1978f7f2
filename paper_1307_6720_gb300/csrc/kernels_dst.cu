// Fast discrete sine transforms (DST-I) for the separable solver.
//
// For a line x_1 .. x_N (N = L - 1, L a power of two) the transform
//   X_m = sum_i x_i sin(pi m i / L),  m = 1 .. N,
// follows from a complex FFT of length 2L of the odd extension
//   y_0 = 0, y_i = x_i, y_L = 0, y_{2L-i} = -x_i:
// its transform is -2i X_m.  Two real lines a and b go through one complex
// FFT as y_a + i y_b; since each odd extension transforms to a purely
// imaginary sequence, the result Z gives X_a = -Im(Z)/2 and X_b = Re(Z)/2.
// The inverse of the DST-I is the same transform scaled by 2/L.
//
// One block handles P pairs of lines in shared memory: the extended pairs
// are stored in bit-reversed order, then the log2(2L) radix-2
// decimation-in-time stages (Cooley and Tukey) run three at a time in
// registers (radix-8 passes), with twiddles e^{-2 pi i q / (2L)} from a table
// staged in shared memory.  Lines are read contiguously; results are written either as lines
// (element m of line l at out + l * out_line + m) or transposed (at
// out + m * out_elem + l), in both cases with consecutive threads on
// consecutive addresses.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
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
// LAST: these are the final stages; the last one only needs its lower
// outputs (positions below L hold the modes the transform returns), so the
// upper half is neither formed nor stored.
template <int Q, bool LAST, typename C>
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
                if (LAST && t == Q - 1) {
                    const C w = tw[rr * tstride];
                    const C b = v[j + d];
                    v[j] = C{v[j].x + (b.x * w.x - b.y * w.y), v[j].y + (b.x * w.y + b.y * w.x)};
                } else {
                    bfly(v[j], v[j + d], tw[rr * tstride]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < (LAST ? R / 2 : R); ++j) zp[phys(base + j * h)] = v[j];
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

// complex elements between the pairs of a block: the padded 2L points, made
// odd so that consecutive pairs start on different banks (the output gather
// reads one element of every pair in a warp)
__host__ __device__ inline int pair_stride(int L) {
    const int padded = (2 * L - 1) + ((2 * L - 1) >> 3) + 1;
    return padded | 1;
}

template <typename T>
__global__ void __launch_bounds__(256) dst_kernel(DstArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char dst_smem[];
    const int L2 = 2 * a.L, N = a.L - 1, bits = a.log2n;
    const int PS = pair_stride(a.L);
    const int P = a.pairs;
    C* z = reinterpret_cast<C*>(dst_smem);            // P pairs, PS points apart
    C* tw = z + P * PS;                                // twiddle table, L entries
    const int plane = blockIdx.y;
    const int line0 = blockIdx.x * 2 * P;             // first line of the block in its plane
    const int nl = min(2 * P, a.lines - line0);       // lines of the block
    const T* in = a.in + plane * a.in_plane + (long long)line0 * a.in_line;
    const C* twg = static_cast<const C*>(a.tw);
    for (int e = threadIdx.x; e < a.L; e += blockDim.x) tw[e] = twg[e];
    // positions 0 and L (bit-reversed: 0 and 1) of every pair are zero; a pair
    // with one line has a zero imaginary part everywhere
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        z[p * PS + phys(0)] = C{T(0), T(0)};
        z[p * PS + phys(1)] = C{T(0), T(0)};
    }
    if (nl & 1)
        for (int e = threadIdx.x; e < L2; e += blockDim.x) reinterpret_cast<T*>(&z[(nl >> 1) * PS + phys(e)])[1] = T(0);
    __syncthreads();
    // scatter the odd extensions into bit-reversed positions: element e of the
    // block's nl * N inputs is x_i of line l (e = l N + i - 1), consecutive
    // threads on consecutive inputs; U loads per thread are in flight before
    // their values are placed
    {
        constexpr int U = 8;
        const int total = nl * N;
        for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
            T v[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / N, i = e - l * N;
                    v[q] = in[(long long)l * a.in_line + i];
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / N, i = e - l * N + 1;
                    C* zp = z + (l >> 1) * PS;
                    reinterpret_cast<T*>(&zp[phys(bitrev(i, bits))])[l & 1] = v[q];
                    reinterpret_cast<T*>(&zp[phys(bitrev(L2 - i, bits))])[l & 1] = -v[q];
                }
            }
        }
    }
    __syncthreads();
    // radix-8 passes (three stages each; the first with constant twiddles), the
    // remaining one or two stages last
    int s = 0;
    if (bits >= 3) {
        fft_first(z, P, PS, bits);
        __syncthreads();
        s = 3;
    }
    for (; s + 3 <= bits; s += 3) {
        if (s + 3 == bits) fft_pass<3, true>(z, tw, P, PS, bits, a.L, s);
        else fft_pass<3, false>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    }
    if (bits - s == 2) {
        fft_pass<2, true>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    } else if (bits - s == 1) {
        fft_pass<1, true>(z, tw, P, PS, bits, a.L, s);
        __syncthreads();
    }
    // X_a = -Im(Z)/2, X_b = Re(Z)/2, m = 1 .. N, scaled; the block's nl * N
    // outputs flattened so that consecutive threads write consecutive
    // addresses: line layout (m fastest) or transposed (line fastest)
    const T hs = T(0.5) * a.scale;
    T* out = a.out + plane * a.out_plane;
    const int total = nl * N;
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
                    l = e / N;
                    m = e - l * N + 1;
                } else {
                    m = e / nl + 1;
                    l = e - (m - 1) * nl;
                }
                const C zm = z[(l >> 1) * PS + phys(m)];
                v[q] = (l & 1) ? hs * zm.x : -hs * zm.y;
                at[q] = lines_out ? (long long)(line0 + l) * a.out_line + (m - 1)
                                  : (long long)(m - 1) * a.out_elem + line0 + l;
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

}  // namespace

// shared memory of a block: P pairs of 2L points with one padding element per
// 8, and the twiddle table of L entries
template <typename T>
size_t dst_smem_bytes(int L, int P) {
    return (size_t(P) * size_t(pair_stride(L)) + size_t(L)) * 2 * sizeof(T);
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
// longest lines (L = 4096, FP64) takes 213 KB
constexpr size_t DST_SMEM_MAX = 227 * 1024;

template <typename T>
void launch_dst(DstArgs<T> a, cudaStream_t st) {
    a.pairs = dst_pairs<T>(a.L);
    // small transforms (coarse levels): fewer pairs per block, so that the
    // blocks cover every SM about twice
    auto blocks = [&](int p) { return size_t((a.lines + 2 * p - 1) / (2 * p)) * size_t(a.planes); };
    while (a.pairs > 2 && blocks(a.pairs) < 2 * 152) a.pairs >>= 1;
    // one thread per radix-8 unit of the block's pairs, 64 .. 256
    const int units = a.pairs * std::max(1, (2 * a.L) / 8);
    const int threads = std::min(256, std::max(64, (units + 31) / 32 * 32));
    const size_t smem = dst_smem_bytes<T>(a.L, a.pairs);
    if (smem > DST_SMEM_MAX) throw Error(MHS_ERR_INVALID_ARG, "sine transform lines too long for shared memory");
    static bool configured = false;   // per template instance
    if (!configured) {
        MHS_CUDA(cudaFuncSetAttribute(dst_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(DST_SMEM_MAX)));
        configured = true;
    }
    const dim3 grid((a.lines + 2 * a.pairs - 1) / (2 * a.pairs), a.planes);
    dst_kernel<T><<<grid, threads, smem, st>>>(a);
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

template void launch_dst<float>(DstArgs<float>, cudaStream_t);
template void launch_dst<double>(DstArgs<double>, cudaStream_t);
template void* make_twiddles<float>(int);
template void* make_twiddles<double>(int);

}  // namespace mhs
