// Device-side convergence control and the one-CTA multigrid sub-cycle.
//
// check_kernel finishes a residual norm in a fixed summation order, forms
// the relative residual ||b - A u|| / ||b|| (the stopping test of a
// multigrid solve), counts cycles and, inside a CUDA graph, sets the
// condition of the enclosing while node.
//
// subcycle_kernel runs a complete V(nu1,nu2)-cycle over the coarse levels
// of a hierarchy (from a cut-off level down to the coarsest) inside one
// CTA, with every level held in shared memory: red-black Gauss-Seidel
// sweeps, residual and full-weighting restriction fused into one pass,
// (bi/tri)linear prolongation, and Gauss-Seidel to convergence on the
// coarsest level.  Coarse levels are too small to occupy the GPU, so one
// launch replaces the dozens of latency-bound launches they would take.
#include <cmath>

#include "device_util.cuh"
#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

__global__ void bnorm_kernel(const double* __restrict__ partial, int n, SolveCtl* ctl) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        ctl->bnorm = sqrt(s);
        ctl->cycles = 0;
        ctl->status = MHS_OK;
        ctl->cont = 0;
    }
}

__global__ void check_kernel(const double* __restrict__ partial, int n, SolveCtl* ctl, int first,
                             cudaGraphConditionalHandle handle, int use_handle) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        const double rn = sqrt(s);
        const double b = ctl->bnorm;
        const double rel = b > 0.0 ? rn / b : 0.0;
        if (!first) ctl->cycles += 1;
        ctl->rel = rel;
        if (first) ctl->rel0 = rel;
        int cont = (b > 0.0 && rel >= ctl->tol && ctl->cycles < ctl->max_cycles) ? 1 : 0;
        if (!isfinite(rn)) {
            ctl->status = MHS_ERR_NONFINITE;
            cont = 0;
        }
        ctl->cont = cont;
        if (use_handle) cudaGraphSetConditional(handle, cont);
    }
}

// ---------------------------------------------------------------------------
// one-CTA sub-cycle
// ---------------------------------------------------------------------------

template <typename T, bool D3>
struct SubCtx {
    T* base;
    const SubParams<T>* p;
    __device__ T* u(int l) const { return base + p->L[l].off_u; }
    __device__ T* f(int l) const { return base + p->L[l].off_f; }
};

template <typename T, bool D3>
__device__ __forceinline__ T apply_off(const Geom& g, const PlaneCoef<T>& c, const T* u, size_t o) {
    T off = c.cx * (u[o + 1] + u[o - 1]) + c.cy * (u[o + g.px] + u[o - g.px]);
    if (D3) off += c.cz * (u[o + g.plane] + u[o - g.plane]);
    return off;
}

// one red-black sweep on level l (colour 0 = (i+j+k) even first)
template <typename T, bool D3>
__device__ void sub_smooth(const SubCtx<T, D3>& s, int l) {
    const Geom& g = s.p->L[l].g;
    const PlaneCoef<T>* coef = s.p->L[l].coef;
    T* u = s.u(l);
    const T* f = s.f(l);
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = D3 ? g.nz - 2 : 1;
    const int hx = (nxi + 1) / 2;
    const int nq = hx * nyi * nzi;
    for (int colour = 0; colour < 2; ++colour) {
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int t = q % hx;
            const int row = q / hx;
            const int j = 1 + row % nyi;
            const int k = D3 ? 1 + row / nyi : 0;
            const int i = 1 + (((1 + j + k) & 1) != colour) + 2 * t;
            if (i > g.nx - 2) continue;
            const PlaneCoef<T> c = coef[k];
            const size_t o = at(g, i, j, k);
            u[o] = (f[o] - apply_off<T, D3>(g, c, u, o)) * c.inv_d;
        }
        __syncthreads();
    }
}

// f[l+1] = full weighting of (f - A u) on level l; u[l+1] = 0 at interior nodes
template <typename T, bool D3>
__device__ void sub_restrict_residual(const SubCtx<T, D3>& s, int l) {
    const Geom& gf = s.p->L[l].g;
    const Geom& gc = s.p->L[l + 1].g;
    const PlaneCoef<T>* coef = s.p->L[l].coef;
    const T* u = s.u(l);
    const T* f = s.f(l);
    T* fc = s.f(l + 1);
    T* uc = s.u(l + 1);
    const int nxi = gc.nx - 2, nyi = gc.ny - 2, nzi = D3 ? gc.nz - 2 : 1;
    const int nq = nxi * nyi * nzi;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int I = 1 + q % nxi;
        const int J = 1 + (q / nxi) % nyi;
        const int K = D3 ? 1 + q / (nxi * nyi) : 0;
        T acc = T(0);
        for (int c3 = (D3 ? -1 : 0); c3 <= (D3 ? 1 : 0); ++c3) {
            const int k = D3 ? 2 * K + c3 : 0;
            const PlaneCoef<T> c = coef[k];
            const T wc = D3 ? (c3 == 0 ? T(0.5) : T(0.25)) : T(1);
            T sb = T(0);
            for (int b = -1; b <= 1; ++b) {
                const T wb = b == 0 ? T(0.5) : T(0.25);
                T sa = T(0);
                for (int a = -1; a <= 1; ++a) {
                    const T wa = a == 0 ? T(0.5) : T(0.25);
                    const size_t o = at(gf, 2 * I + a, 2 * J + b, k);
                    const T r = f[o] - apply_off<T, D3>(gf, c, u, o) - c.d * u[o];
                    sa += wa * r;
                }
                sb += wb * sa;
            }
            acc += wc * sb;
        }
        const size_t oc = at(gc, I, J, K);
        fc[oc] = acc;
        uc[oc] = T(0);
    }
    __syncthreads();
}

// u[l] += I u[l+1] at interior nodes
template <typename T, bool D3>
__device__ void sub_prolong(const SubCtx<T, D3>& s, int l) {
    const Geom& gf = s.p->L[l].g;
    const Geom& gc = s.p->L[l + 1].g;
    T* uf = s.u(l);
    const T* uc = s.u(l + 1);
    const int nxi = gf.nx - 2, nyi = gf.ny - 2, nzi = D3 ? gf.nz - 2 : 1;
    const int nq = nxi * nyi * nzi;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int i = 1 + q % nxi;
        const int j = 1 + (q / nxi) % nyi;
        const int k = D3 ? 1 + q / (nxi * nyi) : 0;
        const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
        auto plane = [&](int K) {
            return T(0.25) * ((uc[at(gc, I0, J0, K)] + uc[at(gc, I1, J0, K)]) +
                              (uc[at(gc, I0, J1, K)] + uc[at(gc, I1, J1, K)]));
        };
        const T v = D3 ? T(0.5) * (plane(k >> 1) + plane((k + 1) >> 1)) : plane(0);
        uf[at(gf, i, j, k)] += v;
    }
    __syncthreads();
}

// coarsest level: sweep until ||f - A u|| <= tol ||f|| (checked every 4 sweeps)
template <typename T, bool D3>
__device__ void sub_coarsest(const SubCtx<T, D3>& s, int l) {
    const Geom& g = s.p->L[l].g;
    const PlaneCoef<T>* coef = s.p->L[l].coef;
    const T* u = s.u(l);
    const T* f = s.f(l);
    const int nxi = g.nx - 2, nyi = g.ny - 2, nzi = D3 ? g.nz - 2 : 1;
    const int nq = nxi * nyi * nzi;
    const double tol = sizeof(T) == 8 ? 1e-10 : 1e-5;
    __shared__ double s_fn;
    __shared__ int s_done;
    auto rnorm2 = [&](bool res) {
        double a = 0.0;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int i = 1 + q % nxi, j = 1 + (q / nxi) % nyi, k = D3 ? 1 + q / (nxi * nyi) : 0;
            const size_t o = at(g, i, j, k);
            double v = double(f[o]);
            if (res) {
                const PlaneCoef<T> c = coef[k];
                v = double(f[o] - apply_off<T, D3>(g, c, u, o) - c.d * u[o]);
            }
            a += v * v;
        }
        return block_sum(a);
    };
    const double fn = rnorm2(false);
    if (threadIdx.x == 0) {
        s_fn = fn;
        s_done = fn == 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 2000 && !s_done; ++sweep) {
        sub_smooth<T, D3>(s, l);
        if ((sweep & 3) == 3) {
            const double rr = rnorm2(true);
            if (threadIdx.x == 0) s_done = rr <= tol * tol * s_fn;
            __syncthreads();
        }
    }
}

template <typename T, bool D3>
__global__ void __launch_bounds__(512) subcycle_kernel(const SubParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SubCtx<T, D3> s{reinterpret_cast<T*>(smem_raw), &p};
    const int nt = blockDim.x;
    {
        const Geom& g0 = p.L[0].g;
        T* u0 = s.u(0);
        T* f0 = s.f(0);
        for (size_t o = threadIdx.x; o < g0.n; o += nt) {
            u0[o] = p.u_g[o];
            f0[o] = p.f_g[o];
        }
        for (int l = 1; l < p.nlev; ++l) {
            T* ul = s.u(l);
            T* fl = s.f(l);
            for (size_t o = threadIdx.x; o < p.L[l].g.n; o += nt) {
                ul[o] = T(0);
                fl[o] = T(0);
            }
        }
    }
    __syncthreads();
    for (int l = 0; l < p.nlev - 1; ++l) {
        for (int q = 0; q < p.nu1; ++q) sub_smooth<T, D3>(s, l);
        sub_restrict_residual<T, D3>(s, l);
    }
    sub_coarsest<T, D3>(s, p.nlev - 1);
    for (int l = p.nlev - 2; l >= 0; --l) {
        sub_prolong<T, D3>(s, l);
        for (int q = 0; q < p.nu2; ++q) sub_smooth<T, D3>(s, l);
    }
    const Geom& g0 = p.L[0].g;
    const T* u0 = s.u(0);
    const int nxi = g0.nx - 2, nyi = g0.ny - 2, nzi = D3 ? g0.nz - 2 : 1;
    for (int q = threadIdx.x; q < nxi * nyi * nzi; q += nt) {
        const int i = 1 + q % nxi, j = 1 + (q / nxi) % nyi, k = D3 ? 1 + q / (nxi * nyi) : 0;
        const size_t o = at(g0, i, j, k);
        p.u_g[o] = u0[o];
    }
}

}  // namespace

void launch_bnorm(const double* partial, int n, SolveCtl* ctl, cudaStream_t st) {
    bnorm_kernel<<<1, 1024, 0, st>>>(partial, n, ctl);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

void launch_check(const double* partial, int n, SolveCtl* ctl, int first, cudaGraphConditionalHandle handle,
                  int use_handle, cudaStream_t st) {
    check_kernel<<<1, 1024, 0, st>>>(partial, n, ctl, first, handle, use_handle);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

size_t subcycle_smem_limit() { return 220 * 1024; }

void subcycle_prepare() {
    const int lim = int(subcycle_smem_limit());
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    MHS_CUDA(cudaFuncSetAttribute(subcycle_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
}

template <typename T>
void launch_subcycle(const SubParams<T>& p, cudaStream_t st) {
    if (p.dim == 3) subcycle_kernel<T, true><<<1, 512, p.smem_bytes, st>>>(p);
    else subcycle_kernel<T, false><<<1, 512, p.smem_bytes, st>>>(p);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

template void launch_subcycle<double>(const SubParams<double>&, cudaStream_t);
template void launch_subcycle<float>(const SubParams<float>&, cudaStream_t);

}  // namespace mhs
