// Fused red-black sweep for FP32 levels with TMA plane staging.
//
// Same sweep as kernels_sweep.cu (out of place, both colours, z-marching
// over a chunk of planes per CTA), but the planes of the old iterate and of f
// arrive by TMA: one thread issues cp.async.bulk.tensor loads of a
// (TX+8) x (TY+4) box per plane three z-steps ahead, into a four-slot
// shared-memory ring, and each stage completes on an mbarrier (transaction
// bytes).  The loads of later planes are therefore in flight while the
// current plane is computed, which hides L2/HBM latency.
//
// TMA rules honoured: the box's innermost start coordinate is a multiple of 4
// floats (16 bytes; the box starts 4 nodes left of the tile's halo-2 origin
// and is 40 floats wide); loads may start at negative coordinates (zero
// fill); every shared-memory destination is 128-byte aligned.  Every mbarrier
// wait has an iteration limit: on expiry the CTA records an error flag,
// waits (again bounded) for its own copies in flight, and exits.
#include <cuda.h>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int BW = TX + 8, BH = TY + 4;   // TMA box: 40 x 12 floats (row of 160 bytes)
constexpr int RX = TX + 2, RY = TY + 2;   // new red values: 1-node halo
constexpr unsigned BOX_BYTES = BW * BH * 4;
constexpr int WAIT_LIMIT = 1 << 22;

struct __align__(128) TmaSmem {
    float old[4][BH][BW];   // 1920 bytes per slot (a multiple of 128)
    float f[4][BH][BW];
    float red[3][RY][RX];
    unsigned long long bar[4];
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for a phase of an mbarrier
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    for (int it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_plane(void* dst, const CUtensorMap* map, int x, int y, int z,
                                               unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_addr(bar))
        : "memory");
}

__global__ void __launch_bounds__(TX* TY)
    rb_sweep_tma_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_f, Geom g,
                        const PlaneCoef<float>* __restrict__ coef, float* __restrict__ uout, int kchunk,
                        int* __restrict__ err) {
    __shared__ TmaSmem s;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int x0 = 1 + blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * kchunk;
    if (k0 > g.nz - 2) return;
    const int k1 = min(k0 + kchunk, g.nz - 1);
    const int bx = x0 - 5, by = y0 - 2;   // box origin: bx = 32 * blockIdx.x - 4, a multiple of 4

    if (tid == 0) {
        for (int q = 0; q < 4; ++q) mbar_init(&s.bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // stage t: old planes and f planes to load (t = 0 is the warm-up stage)
    auto issue = [&](int t) {
        if (tid != 0) return;
        int po[3], npo = 0, pf = -1;
        if (t == 0) {
            if (k0 - 2 >= 0) po[npo++] = k0 - 2;
            po[npo++] = k0 - 1;
            po[npo++] = k0;
            if (k0 - 1 >= 1) pf = k0 - 1;
        } else {
            if (k0 + t <= g.nz - 1) po[npo++] = k0 + t;
            if (k0 + t - 1 <= g.nz - 2) pf = k0 + t - 1;
        }
        unsigned long long* b = &s.bar[t & 3];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(b, BOX_BYTES * unsigned(npo + (pf >= 0 ? 1 : 0)));
        for (int q = 0; q < npo; ++q) tma_load_plane(&s.old[po[q] & 3][0][0], &tm_in, bx, by, po[q], b);
        if (pf >= 0) tma_load_plane(&s.f[pf & 3][0][0], &tm_f, bx, by, pf, b);
    };
    int issued = 0;   // stages issued so far
    auto drain_and_fail = [&](int waited) {
        // record the failure, then wait (bounded) for every stage still in flight
        if (tid == 0) {
            atomicExch(err, 1);
            for (int t = waited; t < issued; ++t) (void)mbar_wait(&s.bar[t & 3], (t >> 2) & 1);
        }
    };
    auto wait_stage = [&](int t) -> bool {
        const bool ok = mbar_wait(&s.bar[t & 3], (t >> 2) & 1);
        if (__syncthreads_or(!ok)) {
            drain_and_fail(t);
            return false;
        }
        return true;
    };

    auto red = [&](int kk) {
        float(*dst)[RX] = s.red[kk % 3];
        const float(*o0)[BW] = s.old[kk & 3];
        const bool inner_plane = kk >= 1 && kk <= g.nz - 2;
        PlaneCoef<float> c{};
        if (inner_plane) c = coef[kk];
        for (int q = tid; q < RX * RY; q += TX * TY) {
            const int hx = q % RX, hy = q / RX;
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
            const int ox = hx + 4, oy = hy + 1;
            float v = o0[oy][ox];
            if (inner_plane && gx >= 1 && gx <= g.nx - 2 && gy >= 1 && gy <= g.ny - 2 && ((gx + gy + kk) & 1) == 0) {
                const float(*om)[BW] = s.old[(kk + 3) & 3];   // plane kk-1
                const float(*op)[BW] = s.old[(kk + 1) & 3];   // plane kk+1
                float w = s.f[kk & 3][oy][ox] * c.inv_d;
                w = fmaf(-c.az, om[oy][ox] + op[oy][ox], w);
                w = fmaf(-c.ay, o0[oy + 1][ox] + o0[oy - 1][ox], w);
                v = fmaf(-c.ax, o0[oy][ox + 1] + o0[oy][ox - 1], w);
            }
            dst[hy][hx] = v;
        }
    };
    auto black_store = [&](int k) {
        const PlaneCoef<float> c = coef[k];
        const float(*r0)[RX] = s.red[k % 3];
        const float(*rm)[RX] = s.red[(k + 2) % 3];
        const float(*rp)[RX] = s.red[(k + 1) % 3];
        const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
        if (gx > g.nx - 2 || gy > g.ny - 2) return;
        const int rx = threadIdx.x + 1, ry = threadIdx.y + 1;
        float v = r0[ry][rx];
        if ((gx + gy + k) & 1) {
            float w = s.f[k & 3][ry + 1][rx + 4] * c.inv_d;
            w = fmaf(-c.az, rm[ry][rx] + rp[ry][rx], w);
            w = fmaf(-c.ay, r0[ry + 1][rx] + r0[ry - 1][rx], w);
            v = fmaf(-c.ax, r0[ry][rx + 1] + r0[ry][rx - 1], w);
        }
        uout[at(g, gx, gy, k)] = v;
    };

    issue(0);
    issue(1);
    issued = 2;
    if (!wait_stage(0)) return;
    red(k0 - 1);
    __syncthreads();
    issue(2);
    issued = 3;
    if (!wait_stage(1)) return;
    red(k0);
    __syncthreads();
    for (int k = k0, j = 0; k < k1; ++k, ++j) {
        issue(j + 3);
        issued = j + 4;
        if (!wait_stage(j + 2)) return;
        red(k + 1);
        __syncthreads();
        black_store(k);
        __syncthreads();
    }
    // the stage issued during the last step is still in flight: complete it
    for (int t = (k1 - k0) + 2; t < issued; ++t)
        if (!wait_stage(t)) return;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        MHS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw Error(MHS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

// 3D tensor map over a pitched FP32 level array (x fastest) with a
// (TX+8) x (TY+4) x 1 box: one plane of a tile with its halo.
void make_plane_map(CUtensorMap* map, const Geom& g, const float* base) {
    const cuuint64_t dims[3] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz)};
    const cuuint64_t strides[2] = {cuuint64_t(g.px) * 4, cuuint64_t(g.plane) * 4};   // multiples of 16 bytes
    const cuuint32_t box[3] = {cuuint32_t(BW), cuuint32_t(BH), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(MHS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
}

void launch_sweep_tma(const Geom& g, const CUtensorMap& tm_in, const CUtensorMap& tm_f,
                      const PlaneCoef<float>* coef, float* uout, int* err, cudaStream_t st) {
    const int gx = (g.nx - 2 + TX - 1) / TX, gy = (g.ny - 2 + TY - 1) / TY;
    const int nzi = g.nz - 2;
    // about six CTAs per SM; chunks of at least 6 planes amortise the warm-up
    int chunks = (6 * 152 + gx * gy - 1) / (gx * gy);
    if (chunks > nzi / 6) chunks = nzi / 6;
    if (chunks < 1) chunks = 1;
    const int kchunk = (nzi + chunks - 1) / chunks;
    const dim3 grid(gx, gy, (nzi + kchunk - 1) / kchunk);
    rb_sweep_tma_kernel<<<grid, dim3(TX, TY), 0, st>>>(tm_in, tm_f, g, coef, uout, kchunk, err);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
