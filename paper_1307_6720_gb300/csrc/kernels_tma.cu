// Fused red-black sweep for FP32 levels with TMA plane staging.
//
// Same sweep as kernels_sweep.cu (out of place, both colours, z-marching
// over a chunk of planes per CTA), but the planes of the old iterate and of f
// arrive by TMA: one thread issues cp.async.bulk.tensor loads of a 72 x 12
// box per plane three z-steps ahead, into a four-slot shared-memory ring, and
// each stage completes on an mbarrier (transaction bytes).  The loads of later
// planes are therefore in flight while the current plane is computed, which
// hides L2/HBM latency.
//
// A CTA of 32 x 8 threads owns a 64 x 8 tile; every thread takes an x-pair
// of nodes, of which exactly one is red and one black, so all lanes do the
// same work: per z-step it forms the red value of plane k+1 (tile plus a
// 1-node halo: 33 pairs x 10 rows over the 256 threads), then the black value
// of plane k and writes both nodes of its pair.
//
// TMA rules honoured: the box's innermost start coordinate is a multiple of 4
// floats (16 bytes: the box starts at x = 64 bx - 4, 5 nodes left of the
// tile) and 72 floats wide; loads may start at negative coordinates (zero
// fill); every shared-memory destination is 128-byte aligned.  Every mbarrier
// wait has an iteration limit: on expiry the CTA records an error flag,
// waits (again bounded) for its own copies in flight, and exits.
#include <cuda.h>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int TX = 64, TY = 8;            // tile of outputs; threads 32 x 8, an x-pair each
constexpr int BW = 72, BH = 12;           // TMA box (floats): x from 64 bx - 4, y from y0 - 2
constexpr int RX = TX + 2, RY = TY + 2;   // red values: tile + 1-node halo
constexpr int RPAIRS = RX / 2;            // x-pairs per red row = red values per row (stored densely)
constexpr unsigned BOX_BYTES = BW * BH * 4;
constexpr int WAIT_LIMIT = 1 << 22;

struct __align__(128) TmaSmem {
    float old[4][BH][BW];   // 3456 bytes per slot (27 x 128)
    float f[4][BH][BW];
    float red[3][RY][RPAIRS];   // row hy: the red value of pair j at [hy][j]
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

__global__ void __launch_bounds__(256)
    rb_sweep_tma_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_f, Geom g,
                        const PlaneCoef<float>* __restrict__ coef, float* __restrict__ uout, int kchunk,
                        int* __restrict__ err) {
    __shared__ TmaSmem s;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int x0 = 1 + blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * kchunk;
    if (k0 > g.nz - 2) return;
    const int k1 = min(k0 + kchunk, g.nz - 1);
    const int bx = x0 - 5, by = y0 - 2;   // box origin: bx = 64 * blockIdx.x - 4, a multiple of 4
    // shared-memory box coordinates of node (x, y): (x - bx, y - by)

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

    // red values of plane kk on the tile and its halo: pair e = (row hy, pair j)
    // holds nodes x0 - 1 + 2j and x0 + 2j of row y0 - 1 + hy, the red one at
    // offset (x0 - 1 + y + kk) & 1 in the pair; stored densely at [hy][j]
    PlaneCoef<float> c_red{};   // coefficients of the latest red plane (the next black plane's)
    auto red = [&](int kk) {
        float(*dst)[RPAIRS] = s.red[kk % 3];
        const float(*o0)[BW] = s.old[kk & 3];
        const float(*om)[BW] = s.old[(kk + 3) & 3];   // plane kk-1
        const float(*op)[BW] = s.old[(kk + 1) & 3];   // plane kk+1
        const float(*fk)[BW] = s.f[kk & 3];
        const bool inner_plane = kk >= 1 && kk <= g.nz - 2;
        PlaneCoef<float> c{};
        if (inner_plane) c = coef[kk];
        c_red = c;
        for (int e = tid; e < RPAIRS * RY; e += 256) {
            const int hy = e / RPAIRS, j = e - hy * RPAIRS;
            const int gy = y0 - 1 + hy;
            const int gx = x0 - 1 + 2 * j + ((x0 - 1 + gy + kk) & 1);
            const int ox = gx - bx, oy = gy - by;
            float v = o0[oy][ox];
            if (inner_plane && gx >= 1 && gx <= g.nx - 2 && gy >= 1 && gy <= g.ny - 2) {
                float w = fk[oy][ox] * c.inv_d;
                w = fmaf(-c.az, om[oy][ox] + op[oy][ox], w);
                w = fmaf(-c.ay, o0[oy + 1][ox] + o0[oy - 1][ox], w);
                v = fmaf(-c.ax, o0[oy][ox + 1] + o0[oy][ox - 1], w);
            }
            dst[hy][j] = v;
        }
    };
    // plane k of the tile: the thread's pair (x0 + 2 tx, x0 + 2 tx + 1) in row
    // y0 + ty: the black node updated from the red values of planes k-1, k,
    // k+1, the red node copied from its red entry.  With p the red offset of
    // the row, the black node is at offset p, its west and east red neighbours
    // are entries tx and tx + 1 of the row, the red node of the pair entry
    // tx + 1 - p, and the red values above, below and in planes k -+ 1 (rows of
    // the other parity) entry tx + p.
    auto black_store = [&](int k, const PlaneCoef<float>& c) {
        const int gy = y0 + threadIdx.y;
        if (gy > g.ny - 2) return;
        const int xa = x0 + 2 * threadIdx.x;
        if (xa > g.nx - 2) return;
        const int p = (x0 - 1 + gy + k) & 1;
        const int gb = xa + p, gr = xa + 1 - p;
        const int tx = threadIdx.x, ry = threadIdx.y + 1;
        const float(*r0)[RPAIRS] = s.red[k % 3];
        const float(*rm)[RPAIRS] = s.red[(k + 2) % 3];
        const float(*rp)[RPAIRS] = s.red[(k + 1) % 3];
        const int jv = tx + p;
        float w = s.f[k & 3][gy - by][gb - bx] * c.inv_d;
        w = fmaf(-c.az, rm[ry][jv] + rp[ry][jv], w);
        w = fmaf(-c.ay, r0[ry + 1][jv] + r0[ry - 1][jv], w);
        const float vb = fmaf(-c.ax, r0[ry][tx + 1] + r0[ry][tx], w);
        const float vr = r0[ry][tx + 1 - p];
        float* row = uout + at(g, 0, gy, k);
        if (gb <= g.nx - 2) row[gb] = vb;
        if (gr <= g.nx - 2) row[gr] = vr;
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
        const PlaneCoef<float> ck = c_red;   // plane k's coefficients, loaded by red(k)
        issue(j + 3);
        issued = j + 4;
        if (!wait_stage(j + 2)) return;
        red(k + 1);
        __syncthreads();
        black_store(k, ck);
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
// 72 x 12 x 1 box: one plane of a 64 x 8 tile with its halo.
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
    rb_sweep_tma_kernel<<<grid, dim3(32, TY), 0, st>>>(tm_in, tm_f, g, coef, uout, kchunk, err);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace mhs
