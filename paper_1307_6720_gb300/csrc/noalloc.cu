// Allocation-free variant of the interior residual-norm kernel.
//
// mhs_interior_residual_noalloc() evaluates ||b - A P||_2 and ||b||_2 of the
// interior problem for a potential P supplied by the caller, without any
// device allocation: its scratch (per-block partial sums and the per-plane
// coefficient table) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library keeps until the process exits.
// b is the right-hand side after lifting every Dirichlet face of P (the
// values on the six faces enter the rows of their interior neighbours); the
// interior source is zero, as in the paper's problem (Sect. 2.2).
//
// Host code may not use the array's name as a device address (it is a host
// stand-in), so the address is looked up once per device with
// cudaGetSymbolAddress and cached.  That look-up happens inside the first
// call on each device.  A cudaDeviceReset destroys the context the address
// belongs to; the cached address is then stale.
//
// All calls share the one array and it keeps the last call's contents:
// every slot a call reads is written earlier by that same call (partials by
// every block, coefficients by every plane), so no clearing is needed, but
// two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int NA_BLOCKS = 1024;     // residual blocks (fixed grid)
constexpr int NA_MAX_NZ = 4097;     // largest nz accepted
constexpr size_t NA_DOUBLES = 2 * size_t(NA_BLOCKS) + 5 * size_t(NA_MAX_NZ);   // about 176 KB

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

std::mutex g_mu;
double* g_addr[256] = {};   // device address of g_noalloc_scratch per device ordinal

__device__ double xi_na(const mhs_xi_params& x, double z) {
    switch (x.kind) {
    case MHS_XI_EXP: return x.a * exp(-x.kappa * z);
    case MHS_XI_EXP_SIN: return (x.a + x.b * sin(x.omega * z)) * exp(-x.kappa * z);
    default: return 0.0;
    }
}

// coefficient table: [cx, cy, cz, d, unused] per plane, the same formulas as the solver's
__global__ void na_coef_kernel(int nz, double hx, double hy, double hz, double alpha, mhs_xi_params xi,
                               double* tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    const double om = 1.0 - xi_na(xi, k * hz);
    const double cx = om / (hx * hx), cy = om / (hy * hy), cz = 1.0 / (hz * hz);
    tab[5 * k + 0] = cx;
    tab[5 * k + 1] = cy;
    tab[5 * k + 2] = cz;
    tab[5 * k + 3] = -2.0 * (cx + cy + cz) + alpha * alpha;
    tab[5 * k + 4] = 0.0;
}

// r = 0 - A P on interior nodes of a dense [nz][ny][nx] array (every face of
// P is Dirichlet data); the lifted right-hand side b of a node is minus the
// coefficient-weighted sum of its neighbours that lie on a face
__global__ void na_residual_kernel(int nx, int ny, int nz, const double* __restrict__ P,
                                   const double* __restrict__ tab, double* __restrict__ part_r,
                                   double* __restrict__ part_b) {
    const size_t nxi = nx - 2, nyi = ny - 2, nzi = nz - 2;
    const size_t total = nxi * nyi * nzi;
    const size_t plane = size_t(nx) * ny;
    double ar = 0.0, ab = 0.0;
    for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < total; q += size_t(gridDim.x) * blockDim.x) {
        const int i = 1 + int(q % nxi);
        const int j = 1 + int((q / nxi) % nyi);
        const int k = 1 + int(q / (nxi * nyi));
        const size_t o = size_t(i) + size_t(nx) * (size_t(j) + size_t(ny) * size_t(k));
        const double cx = tab[5 * k], cy = tab[5 * k + 1], cz = tab[5 * k + 2], d = tab[5 * k + 3];
        double au = cx * (P[o + 1] + P[o - 1]) + cy * (P[o + nx] + P[o - nx]) + d * P[o];
        au += cz * (P[o + plane] + P[o - plane]);
        const double rv = 0.0 - au;
        ar += rv * rv;
        double lift = 0.0;
        if (i == 1) lift += cx * P[o - 1];
        if (i == nx - 2) lift += cx * P[o + 1];
        if (j == 1) lift += cy * P[o - nx];
        if (j == ny - 2) lift += cy * P[o + nx];
        if (k == 1) lift += cz * P[o - plane];
        if (k == nz - 2) lift += cz * P[o + plane];
        ab += lift * lift;
    }
    const double sr = block_sum(ar);
    const double sb = block_sum(ab);
    if (threadIdx.x == 0) {
        part_r[blockIdx.x] = sr;
        part_b[blockIdx.x] = sb;
    }
}

__global__ void na_finish_kernel(const double* __restrict__ part_r, const double* __restrict__ part_b, int n,
                                 double* out) {
    double sr = 0.0, sb = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        sr += part_r[b];
        sb += part_b[b];
    }
    sr = block_sum(sr);
    sb = block_sum(sb);
    if (threadIdx.x == 0) {
        const double rn = sqrt(sr), bn = sqrt(sb);
        out[0] = rn;
        out[1] = bn;
        out[2] = bn > 0.0 ? rn / bn : 0.0;
    }
}

bool is_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Device address of the scratch array on the current device (looked up once per device).
static double* noalloc_scratch() {
    int dev = 0;
    MHS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) throw Error(MHS_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            throw Error(MHS_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                          cudaGetErrorString(e));
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    return g_addr[dev];
}

mhs_status interior_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                                     const mhs_xi_params* xi, const double* P, double* out, cudaStream_t st) {
    if (nx < 3 || ny < 3 || nz < 3) throw Error(MHS_ERR_INVALID_ARG, "node counts must be >= 3");
    if (nz > NA_MAX_NZ)
        throw Error(MHS_ERR_INVALID_ARG, "nz = " + std::to_string(nz) + " exceeds the allocation-free limit of " +
                                             std::to_string(NA_MAX_NZ) + " planes");
    if (!(Lx > 0) || !(Ly > 0) || !(Lz > 0) || !std::isfinite(Lx) || !std::isfinite(Ly) || !std::isfinite(Lz))
        throw Error(MHS_ERR_INVALID_ARG, "domain lengths must be finite and > 0");
    if (!std::isfinite(alpha)) throw Error(MHS_ERR_INVALID_ARG, "alpha must be finite");
    if (xi) {
        if (xi->kind < MHS_XI_NONE || xi->kind > MHS_XI_EXP_SIN) throw Error(MHS_ERR_INVALID_ARG, "unknown xi kind");
        if (!std::isfinite(xi->a) || !std::isfinite(xi->kappa) || !std::isfinite(xi->b) || !std::isfinite(xi->omega))
            throw Error(MHS_ERR_INVALID_ARG, "xi parameters must be finite");
    }
    if (!P || !out || !is_device(P) || !is_device(out))
        throw Error(MHS_ERR_INVALID_ARG, "P and out must be device pointers");
    const mhs_xi_params x = xi ? *xi : mhs_xi_params{MHS_XI_NONE, 0, 0, 0, 0};
    double* base = noalloc_scratch();
    double* part_r = base;
    double* part_b = base + NA_BLOCKS;
    double* tab = base + 2 * NA_BLOCKS;
    na_coef_kernel<<<(nz + 127) / 128, 128, 0, st>>>(nz, Lx / (nx - 1), Ly / (ny - 1), Lz / (nz - 1), alpha, x, tab);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    na_residual_kernel<<<NA_BLOCKS, 256, 0, st>>>(nx, ny, nz, P, tab, part_r, part_b);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    na_finish_kernel<<<1, 1024, 0, st>>>(part_r, part_b, NA_BLOCKS, out);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
    return MHS_OK;
}

}  // namespace mhs
