// Fused red-black Gauss-Seidel sweep (both colours in one pass), out of place.
//
// A CTA owns a TX x TY tile of interior (x, y) positions and marches up a
// chunk of z-planes.  Per plane k it keeps in shared memory:
//   - the old iterate of planes k, k+1, k+2 on the tile with a 2-node halo,
//   - the new red values of planes k-1, k, k+1 on the tile with a 1-node halo,
//   - f of planes k and k+1 on the tile with a 1-node halo;
// it computes the red update of plane k+1 (halo included, from old values
// only), then the black update of plane k from the new red values, and writes
// plane k of the output.  The result equals the in-place sweep (all red nodes,
// then all black nodes) because red updates read only old black values and
// black updates read only new red values.  Reading from one buffer and
// writing another lets neighbouring tiles overlap in their halos without any
// race, and each sweep reads u and f once and writes u once (one launch),
// where the two colour passes read u twice and write it twice.
#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int OX = TX + 4, OY = TY + 4;   // old planes: 2-node halo
constexpr int RX = TX + 2, RY = TY + 2;   // new red values and f: 1-node halo

template <typename T>
struct SweepSmem {
    T old[3][OY][OX];
    T red[3][RY][RX];
    T f[2][RY][RX];
};

template <typename T>
__global__ void __launch_bounds__(TX* TY) rb_sweep_kernel(Geom g, const PlaneCoef<T>* __restrict__ coef,
                                                          const T* __restrict__ uin, const T* __restrict__ f,
                                                          T* __restrict__ uout, int kchunk) {
    __shared__ SweepSmem<T> s;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int x0 = 1 + blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;   // first interior node of the tile
    const int k0 = 1 + blockIdx.z * kchunk;
    if (k0 > g.nz - 2) return;
    const int k1 = min(k0 + kchunk, g.nz - 1);   // planes k0 .. k1-1

    auto load_old = [&](int kk) {
        T(*dst)[OX] = s.old[kk % 3];
        for (int q = tid; q < OX * OY; q += TX * TY) {
            const int xx = q % OX, yy = q / OX;
            const int gx = x0 - 2 + xx, gy = y0 - 2 + yy;
            T v = T(0);
            if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) v = uin[at(g, gx, gy, kk)];
            dst[yy][xx] = v;
        }
    };
    auto load_f = [&](int kk) {
        T(*dst)[RX] = s.f[kk & 1];
        for (int q = tid; q < RX * RY; q += TX * TY) {
            const int xx = q % RX, yy = q / RX;
            const int gx = x0 - 1 + xx, gy = y0 - 1 + yy;
            T v = T(0);
            if (f && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) v = f[at(g, gx, gy, kk)];
            dst[yy][xx] = v;
        }
    };
    // new red values of plane kk on the tile and its 1-node halo; black and
    // boundary positions keep their old (respectively Dirichlet) values
    auto red = [&](int kk) {
        T(*dst)[RX] = s.red[kk % 3];
        const T(*o0)[OX] = s.old[kk % 3];
        const bool inner_plane = kk >= 1 && kk <= g.nz - 2;
        PlaneCoef<T> c{};
        if (inner_plane) c = coef[kk];
        for (int q = tid; q < RX * RY; q += TX * TY) {
            const int xx = q % RX, yy = q / RX;
            const int gx = x0 - 1 + xx, gy = y0 - 1 + yy;
            const int ox = xx + 1, oy = yy + 1;   // same node in the old-plane arrays
            T v = o0[oy][ox];
            if (inner_plane && gx >= 1 && gx <= g.nx - 2 && gy >= 1 && gy <= g.ny - 2 && ((gx + gy + kk) & 1) == 0) {
                const T(*om)[OX] = s.old[(kk + 2) % 3];   // plane kk-1
                const T(*op)[OX] = s.old[(kk + 1) % 3];   // plane kk+1
                T w = s.f[kk & 1][yy][xx] * c.inv_d;
                w = fma(-c.az, om[oy][ox] + op[oy][ox], w);
                w = fma(-c.ay, o0[oy + 1][ox] + o0[oy - 1][ox], w);
                v = fma(-c.ax, o0[oy][ox + 1] + o0[oy][ox - 1], w);
            }
            dst[yy][xx] = v;
        }
    };
    // black update of plane k on the tile, written with the new red values
    auto black_store = [&](int k) {
        const PlaneCoef<T> c = coef[k];
        const T(*r0)[RX] = s.red[k % 3];
        const T(*rm)[RX] = s.red[(k + 2) % 3];   // plane k-1
        const T(*rp)[RX] = s.red[(k + 1) % 3];   // plane k+1
        const int xx = threadIdx.x, yy = threadIdx.y;
        const int gx = x0 + xx, gy = y0 + yy;
        if (gx > g.nx - 2 || gy > g.ny - 2) return;
        const int rx = xx + 1, ry = yy + 1;
        T v = r0[ry][rx];
        if ((gx + gy + k) & 1) {
            T w = s.f[k & 1][ry][rx] * c.inv_d;
            w = fma(-c.az, rm[ry][rx] + rp[ry][rx], w);
            w = fma(-c.ay, r0[ry + 1][rx] + r0[ry - 1][rx], w);
            v = fma(-c.ax, r0[ry][rx + 1] + r0[ry][rx - 1], w);
        }
        uout[at(g, gx, gy, k)] = v;
    };

    // warm-up: new red values of planes k0-1 and k0
    if (k0 - 2 >= 0) load_old(k0 - 2);
    load_old(k0 - 1);
    load_old(k0);
    if (k0 - 1 >= 1) load_f(k0 - 1);
    __syncthreads();
    red(k0 - 1);
    __syncthreads();
    load_old(k0 + 1);
    load_f(k0);
    __syncthreads();
    red(k0);
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        if (k + 2 <= g.nz - 1) load_old(k + 2);
        if (k + 1 <= g.nz - 2) load_f(k + 1);
        __syncthreads();
        red(k + 1);
        __syncthreads();
        black_store(k);
        __syncthreads();
    }
}

}  // namespace

template <typename T>
void launch_sweep(const Geom& g, const PlaneCoef<T>* coef, const T* uin, const T* f, T* uout, cudaStream_t st) {
    const int gx = (g.nx - 2 + TX - 1) / TX, gy = (g.ny - 2 + TY - 1) / TY;
    const int nzi = g.nz - 2;
    // about four CTAs per SM; chunks of at least 4 planes amortise the warm-up
    int chunks = (4 * 152 + gx * gy - 1) / (gx * gy);
    if (chunks > nzi / 4) chunks = nzi / 4;
    if (chunks < 1) chunks = 1;
    const int kchunk = (nzi + chunks - 1) / chunks;
    const dim3 grid(gx, gy, (nzi + kchunk - 1) / kchunk);
    rb_sweep_kernel<T><<<grid, dim3(TX, TY), 0, st>>>(g, coef, uin, f, uout, kchunk);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template void launch_sweep<float>(const Geom&, const PlaneCoef<float>*, const float*, const float*, float*,
                                  cudaStream_t);
template void launch_sweep<double>(const Geom&, const PlaneCoef<double>*, const double*, const double*, double*,
                                   cudaStream_t);

}  // namespace mhs
