// Building blocks of the fast discrete sine transforms (DST-I) of lines held
// in shared memory, shared by the one-pass-per-launch transforms of
// kernels_dst.cu and the plane kernels of kernels_sepplane.cu.  Whatever
// kernel runs them, a line pair's transform performs the same operations in
// the same order (the pairing of lines (2q, 2q + 1), the FFT units, the
// prefix sums), so the two kernel families give bitwise equal results.
//
// The transform (see kernels_dst.cu for the derivation): for a line x_1 ..
// x_{N-1} (N = L a power of two), X_m = sum_i x_i sin(pi m i / N).  FP64
// lines use the half-length form (two real lines share one complex FFT of
// length N, the odd outputs come from prefix sums), FP32 lines the odd
// extensions (one complex FFT of length 2N per pair).
#pragma once

#include "mhs_internal.h"

namespace mhs {

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

// products and sums rounded separately (no contraction into a fused
// multiply-add), where an expression could otherwise compile differently in
// different kernels
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// shared-memory position of point i of a pair: one padding element per 8
// points, which spreads the first passes' strided accesses over the banks
__device__ __forceinline__ int phys(int i) { return i + (i >> 3); }

// complex elements between the pairs of a block: the padded F points of the
// FFT, made odd so that consecutive pairs start on different banks
__host__ __device__ inline int pair_stride(int F) {
    const int padded = (F - 1) + ((F - 1) >> 3) + 1;
    return padded | 1;
}

// FFT length of a line pair: N (FP64 half-length form) or 2N (FP32 odd extensions)
template <typename T>
__host__ __device__ inline int fft_length(int L) { return sizeof(T) == 8 ? L : 2 * L; }

// radix-2 butterfly a, b <- a + w b, a - w b; the complex product with one
// explicit fused multiply-add per component, so that its rounding is fixed
template <typename C>
__device__ __forceinline__ void bfly(C& a, C& b, const C w) {
    const C t = C{fma(b.x, w.x, -mul_rn(b.y, w.y)), fma(b.x, w.y, mul_rn(b.y, w.x))};
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

// Butterfly of the first three stages (half-sizes 1, 2, 4), whose twiddles
// are eighth roots of unity e^{-i pi q / 4}: multiplications by 1 and -i
// become additions and swaps, those by (+-1 - i)/sqrt(2) two additions and
// two rounded multiplications.  a, b <- a + t, a - t with t = b e^{-i pi q / 4}.
template <typename C>
__device__ __forceinline__ void first_bfly(C& a, C& b, int q) {
    using T = decltype(C{}.x);
    const T c = T(0.70710678118654752440);
    C t;
    if (q == 0) t = b;
    else if (q == 1) t = C{mul_rn(b.x + b.y, c), mul_rn(b.y - b.x, c)};
    else if (q == 2) t = C{b.y, -b.x};
    else t = C{mul_rn(b.y - b.x, c), -mul_rn(b.x + b.y, c)};
    b = C{a.x - t.x, a.y - t.y};
    a = C{a.x + t.x, a.y + t.y};
}

// The first three stages as one radix-8 pass in registers.
template <typename C>
__device__ __forceinline__ void fft_first(C* z, int P, int PS, int bits) {
    const int ub = bits - 3;
    const int units = P << ub;
    for (int e = threadIdx.x; e < units; e += blockDim.x) {
        const int pair = e >> ub, u = e & ((1 << ub) - 1);
        const int base = u << 3;
        C* zp = z + pair * PS;
        C v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = zp[phys(base + j)];
        // half-size 1: twiddle 1
#pragma unroll
        for (int j = 0; j < 8; j += 2) first_bfly(v[j], v[j + 1], 0);
        // half-size 2: twiddles 1, -i
        first_bfly(v[0], v[2], 0);
        first_bfly(v[4], v[6], 0);
        first_bfly(v[1], v[3], 2);
        first_bfly(v[5], v[7], 2);
        // half-size 4: twiddles 1, (1 - i)/sqrt2, -i, (-1 - i)/sqrt2
#pragma unroll
        for (int j = 0; j < 4; ++j) first_bfly(v[j], v[j + 4], j);
#pragma unroll
        for (int j = 0; j < 8; ++j) zp[phys(base + j)] = v[j];
    }
}

// One radix-2 stage (half-size H = 2^s) of every pair, one butterfly per
// unit: the operations of the radix-8 passes, butterfly for butterfly
// (first_bfly below half-size 8, bfly with the table twiddle from there on),
// spread over more threads, for blocks with few pairs.
template <typename C>
__device__ __forceinline__ void fft_stage(C* z, const C* tw, int P, int PS, int bits, int L, int s) {
    const int H = 1 << s, hb = bits - 1;
    const int units = P << hb;
    for (int e = threadIdx.x; e < units; e += blockDim.x) {
        const int pair = e >> hb, b = e & ((1 << hb) - 1);
        const int r = b & (H - 1);
        const int i0 = ((b >> s) << (s + 1)) + r;
        C* zp = z + pair * PS;
        C va = zp[phys(i0)], vb = zp[phys(i0 + H)];
        if (s < 3) first_bfly(va, vb, r << (2 - s));
        else bfly(va, vb, tw[r * (L >> s)]);
        zp[phys(i0)] = va;
        zp[phys(i0 + H)] = vb;
    }
}

// The fixed points of every pair (y_0, and y_N for the odd extensions) and,
// for an odd line count nl, the imaginary part of the lone last line, set to
// zero.  The caller synchronises before the loads.
template <typename T>
__device__ __forceinline__ void dst_zero(typename Cplx<T>::type* z, int P, int PS, int N, int nl) {
    using C = typename Cplx<T>::type;
    constexpr bool HALF = sizeof(T) == 8;
    const int F = fft_length<T>(N);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        z[p * PS + phys(0)] = C{T(0), T(0)};
        if (!HALF) z[p * PS + phys(1)] = C{T(0), T(0)};
    }
    if (nl & 1)
        for (int e = threadIdx.x; e < F; e += blockDim.x) reinterpret_cast<T*>(&z[(nl >> 1) * PS + phys(e)])[1] = T(0);
}

// The FFT input of nl lines from ld(l, i) = x_{i+1} of line l (i = 0 .. N-2),
// at bit-reversed positions: FP64 y_i and y_{N-i} from x_i and x_{N-i}
// (i = 1 .. N/2), FP32 the odd extensions.  U loads per thread are in flight
// before their values are used.  tw: the twiddle table (FP64 pre-processing
// uses sin(pi i / N) = -Im tw[i]).  The caller synchronises afterwards.
template <typename T, typename Ld>
__device__ __forceinline__ void dst_load(typename Cplx<T>::type* z, int PS, int nl, int N, int bits,
                                         const typename Cplx<T>::type* tw, Ld ld) {
    using C = typename Cplx<T>::type;
    if constexpr (sizeof(T) == 8) {
        constexpr int U = 4;
        const int H = N / 2, total = nl * H;
        for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
            T xi[U], xr[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / H, i = e - l * H + 1;
                    xi[q] = ld(l, i - 1);
                    xr[q] = ld(l, N - i - 1);
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
        const int F = 2 * N, M = N - 1, total = nl * M;
        for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
            T v[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < total) {
                    const int l = e / M, i = e - l * M;
                    v[q] = ld(l, i);
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
}

// The FFT of every pair of the block: radix-8 passes (the first with
// constant twiddles), the remaining one or two stages last.  Synchronises
// after every pass.  An FP64 block with fewer radix-8 units than four
// warps' lanes (few pairs) runs the same butterflies stage by stage instead:
// the FP64 pipe charges each warp instruction whatever its active lanes, so a
// lone warp's radix-8 units cost their full length in issue time, while one
// butterfly per thread per stage spreads them over several warps.  Both
// schedules give the same words.  Not inlined: a kernel that transforms along
// x and y, forward and back, runs one copy of this code (fetched once into
// the instruction cache) instead of four, and every kernel family runs the
// same compiled operations.
template <typename T>
__device__ __noinline__ void dst_fft(typename Cplx<T>::type* z, const typename Cplx<T>::type* tw, int P, int PS,
                                        int bits, int L) {
    if (sizeof(T) == 8 && bits >= 3 && (P << (bits - 3)) < 128) {
        for (int s = 0; s < bits; ++s) {
            fft_stage(z, tw, P, PS, bits, L, s);
            __syncthreads();
        }
        return;
    }
    int s = 0;
    if (bits >= 3) {
        fft_first(z, P, PS, bits);
        __syncthreads();
        s = 3;
    }
    for (; s + 3 <= bits; s += 3) {
        fft_pass<3>(z, tw, P, PS, bits, L, s);
        __syncthreads();
    }
    if (bits - s == 2) {
        fft_pass<2>(z, tw, P, PS, bits, L, s);
        __syncthreads();
    } else if (bits - s == 1) {
        fft_pass<1>(z, tw, P, PS, bits, L, s);
        __syncthreads();
    }
}

// The transforms X_1 .. X_{N-1} of the nl lines into ob (element m - 1 of
// line l at ob[l N + m - 1]).  FP64: lanes form R_k, I_k from Z_k and
// Z_{N-k}, X_{2k} = -I_k and the prefix sums X_{2k+1} = R_0/2 + R_1 + .. + R_k
// (lane runs of `per` consecutive k's, at least 4 on lines of 8 points or
// more, then a scan of the run totals over the line's lanes); FP32:
// X_a = -Im(Z_m)/2, X_b = Re(Z_m)/2.  The caller synchronises afterwards.
template <typename T>
__device__ __noinline__ void dst_post(const typename Cplx<T>::type* z, int PS, int nl, int N, T* ob) {
    using C = typename Cplx<T>::type;
    if constexpr (sizeof(T) == 8) {
        const int H = N / 2;
        const unsigned full = 0xffffffffu;
        // lpl lanes per line, each over a run of at least 4 consecutive k's
        // (up to 32 lanes): the scan's FP64 steps, each a full warp
        // instruction, are shared by the run; a warp takes 32 / lpl lines at once
        int lpl = 32;
        while (lpl > 1 && 4 * lpl > H) lpl >>= 1;
        const int per = (H + lpl - 1) / lpl;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        const int lpw = 32 / lpl, sub = lane / lpl, sl = lane - sub * lpl;
        const int j0 = sl * per;
        for (int l0 = warp * lpw; l0 < nl; l0 += nwarps * lpw) {   // warp-uniform: every lane takes part in the scan
            const int l = l0 + sub;
            const bool has = l < nl;
            const C* zp = z + (has ? (l >> 1) * PS : 0);
            const int comp = l & 1;
            T* o = ob + (has ? l * N : 0);
            auto rk = [&](int j, T& R, T& I) {
                const C zk = zp[phys(j)], zr = zp[phys((N - j) & (N - 1))];
                R = T(0.5) * (comp ? zk.y + zr.y : zk.x + zr.x);
                I = T(0.5) * (comp ? zr.x - zk.x : zk.y - zr.y);
                if (j == 0) R *= T(0.5);
            };
            // R and I of a lane's first KEEP k's stay in registers between the two loops;
            // longer runs (N > 256) recompute the rest
            constexpr int KEEP = 4;
            T Rk[KEEP], Ik[KEEP];
            T run = T(0);
#pragma unroll
            for (int q = 0; q < KEEP; ++q) {
                const int j = j0 + q;
                if (has && q < per && j < H) {
                    rk(j, Rk[q], Ik[q]);
                    run = add_rn(run, Rk[q]);
                }
            }
            for (int q = KEEP; q < per; ++q) {
                const int j = j0 + q;
                if (has && j < H) {
                    T R, I;
                    rk(j, R, I);
                    run = add_rn(run, R);
                }
            }
            T incl = run;
            for (int off = 1; off < lpl; off <<= 1) {
                const T v = __shfl_up_sync(full, incl, off, lpl);
                if (sl >= off) incl += v;
            }
            if (!has) continue;
            T acc = incl - run;
#pragma unroll
            for (int q = 0; q < KEEP; ++q) {
                const int j = j0 + q;
                if (q < per && j < H) {
                    acc = add_rn(acc, Rk[q]);
                    o[2 * j] = acc;                       // X_{2j+1}
                    if (j >= 1) o[2 * j - 1] = -Ik[q];    // X_{2j}
                }
            }
            for (int q = KEEP; q < per; ++q) {
                const int j = j0 + q;
                if (j < H) {
                    T R, I;
                    rk(j, R, I);
                    acc = add_rn(acc, R);
                    o[2 * j] = acc;
                    if (j >= 1) o[2 * j - 1] = -I;
                }
            }
        }
    } else {
        const int M = N - 1, total = nl * M;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int l = e / M, m = e - l * M + 1;
            const C zm = z[(l >> 1) * PS + phys(m)];
            ob[l * N + m - 1] = (l & 1) ? T(0.5) * zm.x : T(-0.5) * zm.y;
        }
    }
}

// stored result of a transform: scale * X (+ the old value with accumulate),
// each operation rounded on its own
template <typename T>
__device__ __forceinline__ T dst_result(T scale, T x, bool accumulate, T old) {
    const T v = mul_rn(scale, x);
    return accumulate ? add_rn(old, v) : v;
}

// the lower-boundary mode division t / (cf mu_fast + cs mu_slow)
template <typename T>
__device__ __forceinline__ T mode_divide(T t, T cf, T mufast, T cs, T muslow) {
    return t / fma(cf, mufast, mul_rn(cs, muslow));
}

}  // namespace mhs
