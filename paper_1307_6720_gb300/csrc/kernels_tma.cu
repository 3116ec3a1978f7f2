// Fused red-black sweep for FP32 levels with TMA plane staging.
//
// Same sweep as kernels_sweep.cu (out of place, both colours, z-marching
// over a chunk of planes per CTA), but the planes of the old iterate and of f
// arrive by TMA: one thread issues cp.async.bulk.tensor loads of a
// 72 x (TY + 4) box per plane, one z-step ahead of the plane consumed next,
// into four-slot shared-memory rings, and each stage completes on an mbarrier
// (transaction bytes).  The loads of later planes are therefore in flight
// while the current plane is computed, which hides L2/HBM latency.
//
// A CTA of 32 x TY threads (TY = 8 or 16) owns a 64 x TY tile; every thread
// takes an x-pair of nodes, of which exactly one is red and one black, so all
// lanes do the same work: per z-step it forms red values of plane k+1 (tile
// plus a 1-node halo: 33 pairs x (TY + 2) rows over the threads), then the
// black value of plane k, and writes both nodes of its pair.  The per-thread
// index work (offsets, parities, interior masks) is formed once before the
// z-march; only thread 0 polls the mbarrier, and a block barrier passes the
// completed stage on.
//
// TMA rules honoured: the box's innermost start coordinate is a multiple of 4
// floats (16 bytes: the box starts at x = 64 bx - 4, 5 nodes left of the
// tile) and 72 floats wide; loads may start at negative coordinates (zero
// fill); every shared-memory destination is 128-byte aligned.  Every mbarrier
// wait has an iteration limit: on expiry the CTA records an error flag,
// waits (again bounded) for its own copies in flight, and exits.
#include <cuda.h>

#include <algorithm>

#include "device_util.cuh"
#include "mhs_internal.h"

namespace mhs {

namespace {

// A CTA owns a TX x TY tile of outputs: 32 x TY threads, an x-pair each.
// The TMA box of one plane is BW x (TY + 4) floats: x from 64 bx - 4 (five
// nodes left of the tile, a multiple of 4 floats), y from two rows above it.
// Planes of the old iterate and of f stream through rings of NS slots; the
// loads run NS - 3 z-steps ahead of the one consumed next.
constexpr int TX = 64;
constexpr int BW = 72;
constexpr int RP = TX / 2 + 1;   // red values per row of the tile plus halo: pairs of nodes x0 - 1 + 2j, x0 + 2j
constexpr int WAIT_LIMIT = 1 << 22;

template <int TY, int NS>
struct TmaShape {
    static constexpr int BH = TY + 4;                  // box rows
    static constexpr int RY = TY + 2;                  // red rows: tile + 1-row halo
    static constexpr int NT = 32 * TY;                 // threads
    static constexpr int NRED = RY * RP;               // red values per plane
    static constexpr int NI = (NRED + NT - 1) / NT;    // red values per thread (at most)
    static constexpr int SLOT = BH * BW;               // floats per staged plane (a multiple of 32: 128-byte slots)
    static constexpr int AHEAD = NS - 3;               // stages in flight beyond the next one
    static constexpr unsigned BOX_BYTES = SLOT * 4;
    // dynamic shared memory: NS old-iterate slots, NS f slots, 3 red planes, NS mbarriers
    static constexpr size_t RED_OFF = size_t(2 * NS) * SLOT * 4;
    static constexpr size_t BAR_OFF = (RED_OFF + size_t(3) * NRED * 4 + 15) / 16 * 16;
    static constexpr size_t BYTES = BAR_OFF + NS * 8 + 128;   // + 128: alignment of the base
    static_assert(SLOT % 32 == 0, "TMA slots must stay 128-byte aligned");
    static_assert(NI <= 2, "at most two red values per thread");
    static_assert(NS >= 4, "the ring holds planes k-1, k, k+1 and at least one in flight");
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

// Everything a thread needs per plane that does not depend on the plane is
// formed once before the z-march: the shared-memory offsets of its red items
// and of its pair, the parity of its rows, which of its nodes are interior,
// and the global address of its pair.  Per plane only the red offset of the
// row (parity of x0 - 1 + y + k) changes.  The arithmetic of every update is
// the plain fused sweep's, in the same order, so both give identical words.
template <int TY, int NS>
__global__ void __launch_bounds__(32 * TY, TY == 16 ? 3 : 6)
    rb_sweep_tma_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_f, Geom g,
                        const PlaneCoef<float>* __restrict__ coef, float* __restrict__ uout, int kchunk,
                        int* __restrict__ err) {
    using S = TmaShape<TY, NS>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float* s_old = reinterpret_cast<float*>(base);
    float* s_f = s_old + NS * S::SLOT;
    float* s_red = reinterpret_cast<float*>(base + S::RED_OFF);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + S::BAR_OFF);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + 32 * ty;
    const int x0 = 1 + blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * kchunk;
    if (k0 > g.nz - 2) return;
    const int k1 = min(k0 + kchunk, g.nz - 1);
    const int bx = x0 - 5, by = y0 - 2;   // box origin: bx = 64 * blockIdx.x - 4, a multiple of 4
    // shared-memory box coordinates of node (x, y): (x - bx, y - by)

    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // red items e = tid + NT i: row hy = e / RP, pair j = e % RP, nodes
    // x0 - 1 + 2j and x0 + 2j of row gy = y0 - 1 + hy; the red one sits at
    // offset (x0 - 1 + gy + kk) & 1 of the pair.  mask bit b: the node at
    // offset b is interior (updated), else the red value is the old one.
    int r_off[S::NI], r_q[S::NI], r_mask[S::NI];
#pragma unroll
    for (int i = 0; i < S::NI; ++i) {
        const int e = tid + S::NT * i;
        const int hy = e / RP, j = e - (e / RP) * RP;
        const int gy = y0 - 1 + hy, xb = x0 - 1 + 2 * j;
        r_off[i] = (hy + 1) * BW + (xb - bx);
        r_q[i] = (xb + gy) & 1;
        const bool yin = gy >= 1 && gy <= g.ny - 2;
        r_mask[i] = (e < S::NRED && yin) ? ((xb >= 1 && xb <= g.nx - 2 ? 1 : 0) | (xb + 1 >= 1 && xb + 1 <= g.nx - 2 ? 2 : 0)) : 0;
    }
    // the thread's pair: nodes xa, xa + 1 of row gy; the black node sits at
    // offset p = (x0 - 1 + gy + k) & 1, the red one at 1 - p
    const int gy = y0 + ty, xa = x0 + 2 * tx;
    const bool active = gy <= g.ny - 2 && xa <= g.nx - 2;
    const bool hi_in = xa + 1 <= g.nx - 2;
    const int b_q = (x0 - 1 + gy) & 1;
    const int b_f = (gy - by) * BW + (xa - bx);   // f of node xa in a slot
    const int b_r = (ty + 1) * RP + tx;           // red entry of pair tx (nodes xa - 1, xa) in the red plane
    float* out = uout + (active ? at(g, xa, gy, k0) : 0);

    // stage 0 loads old planes k0-2 (if any), k0-1, k0 and f plane k0-1 (if
    // interior); stage t >= 1 old plane k0+t (if any) and f plane k0+t-1 (if
    // interior).  Plane q sits in slot q % NS of its ring, stage t completes
    // on mbarrier t % NS.  Stages 0 .. last are needed.
    const int last = (k1 - k0) + 1;
    auto issue = [&](int t) {
        if (tid != 0 || t > last) return;
        int olo, ohi, pf;
        if (t == 0) {
            olo = max(k0 - 2, 0);
            ohi = k0;
            pf = k0 - 1 >= 1 ? k0 - 1 : -1;
        } else {
            olo = k0 + t;
            ohi = min(k0 + t, g.nz - 1);
            pf = k0 + t - 1 <= g.nz - 2 ? k0 + t - 1 : -1;
        }
        const int nload = max(ohi - olo + 1, 0) + (pf >= 0 ? 1 : 0);
        unsigned long long* b = &bar[t % NS];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(b, S::BOX_BYTES * unsigned(nload));
        for (int q = olo; q <= ohi; ++q) tma_load_plane(s_old + (q % NS) * S::SLOT, &tm_in, bx, by, q, b);
        if (pf >= 0) tma_load_plane(s_f + (pf % NS) * S::SLOT, &tm_f, bx, by, pf, b);
    };
    int issued = 0;   // stages issued so far (0 .. issued - 1)
    auto issue_upto = [&](int t) {   // issue every stage up to t
        for (; issued <= min(t, last); ++issued) issue(issued);
    };
    // thread 0 alone waits on the stage's mbarrier; the block barrier that
    // follows hands the completed loads (and a failure) to every thread
    auto wait_stage = [&](int t) -> bool {
        bool ok = true;
        if (tid == 0) ok = mbar_wait(&bar[t % NS], (t / NS) & 1);
        if (__syncthreads_or(!ok)) {
            // record the failure, then wait (bounded) for every stage still in flight
            if (tid == 0) {
                atomicExch(err, 1);
                for (int u = t; u < issued; ++u) (void)mbar_wait(&bar[u % NS], (u / NS) & 1);
            }
            return false;
        }
        return true;
    };

    PlaneCoef<float> c_red{};   // coefficients of the latest red plane (the next black plane's)
    // red values of plane kk (in slot sk of the rings) on the tile and its
    // halo, stored densely at [hy][j]
    auto red = [&](int kk, int sk, float* dst) {
        const float* o0 = s_old + sk * S::SLOT;
        const float* om = s_old + (sk == 0 ? NS - 1 : sk - 1) * S::SLOT;   // plane kk-1
        const float* op = s_old + (sk == NS - 1 ? 0 : sk + 1) * S::SLOT;   // plane kk+1
        const float* fk = s_f + sk * S::SLOT;
        const bool inner_plane = kk >= 1 && kk <= g.nz - 2;
        PlaneCoef<float> c{};
        if (inner_plane) c = coef[kk];
        c_red = c;
        const int kp = kk & 1;
#pragma unroll
        for (int i = 0; i < S::NI; ++i) {
            const int e = tid + S::NT * i;
            if (S::NI * S::NT > S::NRED && e >= S::NRED) break;
            const int par = r_q[i] ^ kp;
            const int a = r_off[i] + par;
            float v = o0[a];
            if (inner_plane && ((r_mask[i] >> par) & 1)) {
                float w = fk[a] * c.inv_d;
                w = fmaf(-c.az, om[a] + op[a], w);
                w = fmaf(-c.ay, o0[a + BW] + o0[a - BW], w);
                v = fmaf(-c.ax, o0[a + 1] + o0[a - 1], w);
            }
            dst[e] = v;
        }
    };
    // plane k (f in slot sk) of the tile: the black node of the thread's pair
    // from the red values of planes k-1, k, k+1, the red node copied from its
    // red entry.  With p the red offset of the row, the west and east red
    // neighbours of the black node are entries tx and tx + 1 of the row, the
    // red node of the pair entry tx + 1 - p, and the red values above, below
    // and in planes k -+ 1 (rows of the other parity) entry tx + p.
    auto black_store = [&](int k, int sk, const PlaneCoef<float>& c, const float* r0, const float* rm,
                           const float* rp) {
        if (!active) return;
        const int p = b_q ^ (k & 1);
        const int jv = b_r + p;
        float w = s_f[sk * S::SLOT + b_f + p] * c.inv_d;
        w = fmaf(-c.az, rm[jv] + rp[jv], w);
        w = fmaf(-c.ay, r0[jv + RP] + r0[jv - RP], w);
        const float re = r0[b_r + 1], rw = r0[b_r];   // east and west red neighbours
        const float vb = fmaf(-c.ax, re + rw, w);
        const float vr = p ? rw : re;                 // the pair's red node
        out[0] = p ? vr : vb;
        if (hi_in) out[1] = p ? vb : vr;
        out += g.plane;
    };

    // red planes rotate through three buffers
    float* rb0 = s_red;                 // plane k - 1
    float* rb1 = s_red + S::NRED;       // plane k
    float* rb2 = s_red + 2 * S::NRED;   // plane k + 1
    int sk = (k0 - 1) % NS;             // ring slot of plane k0 - 1

    issue_upto(S::AHEAD);   // stage AHEAD + 1 would refill the slot of plane k0 - 2, still needed
    if (!wait_stage(0)) return;
    red(k0 - 1, sk, rb0);
    __syncthreads();
    sk = sk == NS - 1 ? 0 : sk + 1;
    issue_upto(S::AHEAD + 1);
    if (!wait_stage(1)) return;
    red(k0, sk, rb1);
    __syncthreads();   // red(k0) read plane k0 - 1's slot, which the next stage refills
    for (int k = k0, j = 0; k < k1; ++k, ++j) {
        const PlaneCoef<float> ck = c_red;   // plane k's coefficients, loaded by red(k)
        const int sn = sk == NS - 1 ? 0 : sk + 1;   // slot of plane k + 1
        // stage j + AHEAD + 2 refills the slots of old plane k - 1 and f plane k - 2
        issue_upto(j + S::AHEAD + 2);
        // the wait's block barrier also orders black_store(k - 1) before
        // red(k + 1) overwrites the buffer of plane k - 2
        if (!wait_stage(j + 2)) return;
        red(k + 1, sn, rb2);
        __syncthreads();
        black_store(k, sk, ck, rb1, rb0, rb2);
        float* t = rb0;
        rb0 = rb1;
        rb1 = rb2;
        rb2 = t;
        sk = sn;
    }
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
// 72 x (rows + 4) x 1 box: one plane of a 64 x rows tile with its halo.
void make_plane_map(CUtensorMap* map, const Geom& g, const float* base, int rows) {
    const cuuint64_t dims[3] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz)};
    const cuuint64_t strides[2] = {cuuint64_t(g.px) * 4, cuuint64_t(g.plane) * 4};   // multiples of 16 bytes
    const cuuint32_t box[3] = {cuuint32_t(BW), cuuint32_t(rows + 4), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(MHS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
}

namespace {

template <int TY, int NS>
void launch_tma(const Geom& g, const CUtensorMap& tm_in, const CUtensorMap& tm_f, const PlaneCoef<float>* coef,
                float* uout, int* err, cudaStream_t st) {
    using S = TmaShape<TY, NS>;
    static bool attr = false;
    if (!attr) {
        MHS_CUDA(cudaFuncSetAttribute(rb_sweep_tma_kernel<TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(S::BYTES)));
        attr = true;
    }
    int per_sm = 0;
    MHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rb_sweep_tma_kernel<TY, NS>, 32 * TY, S::BYTES));
    const int gx = (g.nx - 2 + TX - 1) / TX, gy = (g.ny - 2 + TY - 1) / TY;
    const int nzi = g.nz - 2;
    // at most one wave of resident CTAs (a second, partial wave would run
    // alone); chunks of at least 6 planes amortise the warm-up
    const int want = 152 * std::max(per_sm, 1);
    int chunks = want / (gx * gy);
    if (chunks > nzi / 6) chunks = nzi / 6;
    if (chunks < 1) chunks = 1;
    const int kchunk = (nzi + chunks - 1) / chunks;
    const dim3 grid(gx, gy, (nzi + kchunk - 1) / kchunk);
    rb_sweep_tma_kernel<TY, NS><<<grid, dim3(32, TY), S::BYTES, st>>>(tm_in, tm_f, g, coef, uout, kchunk, err);
    count_launches(1);
    MHS_CUDA(cudaGetLastError());
}

}  // namespace

void launch_sweep_tma(const Geom& g, int rows, const CUtensorMap& tm_in, const CUtensorMap& tm_f,
                      const PlaneCoef<float>* coef, float* uout, int* err, cudaStream_t st) {
    // four-slot rings: deeper rings (6 or 8 slots, more loads in flight) cost
    // resident CTAs and measured slower on 129^3 to 513^3 grids
    if (rows == 16)
        launch_tma<16, 4>(g, tm_in, tm_f, coef, uout, err, st);
    else if (rows == 8)
        launch_tma<8, 4>(g, tm_in, tm_f, coef, uout, err, st);
    else
        throw Error(MHS_ERR_INVALID_ARG, "TMA sweep tiles are 8 or 16 rows high");
}

}  // namespace mhs
