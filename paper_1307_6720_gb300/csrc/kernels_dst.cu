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
#include "dst_body.cuh"
#include "group.h"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

// block (bx, by) = (line block, plane) of the transform a; every thread of
// the block calls it
template <typename T>
__device__ __forceinline__ void dst_body(const DstArgs<T>& a, int bx, int by) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char dst_smem[];
    const int N = a.L;
    const int bits = sizeof(T) == 8 ? a.log2n : a.log2n + 1;   // log2 of the FFT length
    const int PS = pair_stride(fft_length<T>(N));
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
    dst_zero<T>(z, P, PS, N, nl);
    __syncthreads();
    const long long il = a.in_line;
    dst_load<T>(z, PS, nl, N, bits, tw, [&](int l, int i) { return in[(long long)l * il + i]; });
    __syncthreads();
    dst_fft<T>(z, tw, P, PS, bits, a.L);
    dst_post<T>(z, PS, nl, N, ob);
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
                v[q] = ob[l * N + m];
                at[q] = lines_out ? (long long)(line0 + l) * a.out_line + m : (long long)m * a.out_elem + line0 + l;
                old[q] = a.accumulate ? out[at[q]] : T(0);
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < total) out[at[q]] = dst_result(a.scale, v[q], a.accumulate != 0, old[q]);
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
void* make_twiddles(int L, size_t* bytes) {
    using C = typename Cplx<T>::type;
    std::vector<C> tw(L);
    for (int q = 0; q < L; ++q) {
        const double ang = -M_PI * double(q) / double(L);
        tw[q] = C{T(std::cos(ang)), T(std::sin(ang))};
    }
    void* p = nullptr;
    MHS_CUDA(cudaMalloc(&p, tw.size() * sizeof(C)));
    MHS_CUDA(cudaMemcpy(p, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice));
    if (bytes) *bytes = tw.size() * sizeof(C);
    return p;
}

template void dst_shape<float>(DstArgs<float>&, dim3&, int&, size_t&);
template void dst_shape<double>(DstArgs<double>&, dim3&, int&, size_t&);
template void launch_dst_stage<float>(const SepStage<float>&, cudaStream_t);
template void launch_dst_stage<double>(const SepStage<double>&, cudaStream_t);
template void glaunch_dst<float>(const GSepTable<float>&, int, int, cudaStream_t);
template void glaunch_dst<double>(const GSepTable<double>&, int, int, cudaStream_t);
template void* make_twiddles<float>(int, size_t*);
template void* make_twiddles<double>(int, size_t*);

}  // namespace mhs
