// gemm_tc.cu -- the surrogate's bf16 GEMM on the fifth-generation tensor
// cores (surrogate.h: sur_gemm_bf16 with both operands K-major, and
// sur_gemm_bf16_batched).
//
// Output tiles of 128 x 128, f32 accumulators in tensor memory, operands
// staged by TMA (cp.async.bulk.tensor) into rings of mbarrier stages, MMAs by
// tcgen05.mma (kind::f16, M = 128, N = 128, K = 16 per instruction, bf16
// operands read from shared memory through matrix descriptors), stages freed
// by tcgen05.commit; the accumulator read back with tcgen05.ld (32 lanes x 32
// columns per warp) and stored through a 32 x 33 transpose tile in shared
// memory, so that each row is written by 32 lanes together, with the fused
// epilogue (row scale, accumulate, bias, ReLU, f32 store and bf16 copy).
// Two kernels:
//   k_gemm_tcp (128-byte swizzled 64-element K slices, the default):
//     persistent, two CTAs per SM, warp-specialised -- one thread loads, one
//     issues MMAs into two accumulators in turn, four warps run the epilogue
//     of the previous tile meanwhile (below);
//   k_gemm_tc<0> (unswizzled core-matrix slices, 8 x 16 bytes from a 3-D
//     tensor map over (8 elements, rows, K / 8)): one CTA per tile, thread 0
//     loads and issues, the four warps run the epilogue at the end.
// Out-of-range rows and K columns read as zeros (TMA bounds), so any M, N, K
// work; the row strides must be multiples of 8 elements (16 bytes).
// Every mbarrier wait is bounded; on expiry the CTA records a failure
// (sur_gemm_tc_failed), stops, lets its MMAs and loads in flight complete and
// frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "../../include/fdtd.h"
#include "../../include/surrogate.h"
#include "tma_pipe.cuh"

namespace fdtd {
namespace gtc {
namespace {

using namespace tma;

constexpr int BM = 128, BN = 128, NT = 128;
constexpr uint32_t TMEM_COLS = BN;   // f32 accumulator: one column per N

template <int SW> struct Cfg;
template <> struct Cfg<1> {
    static constexpr int BK = 64;
};
template <> struct Cfg<0> {
    static constexpr int BK = 32, NS = 4;
};
template <int SW> __host__ __device__ constexpr int a_bytes() { return BM * Cfg<SW>::BK * 2; }
template <int SW> __host__ __device__ constexpr int stage_bytes() { return (BM + BN) * Cfg<SW>::BK * 2; }
// shared memory of a CTA with ns stages (fewer stages than Cfg::NS when K
// has fewer slices, so that more CTAs share an SM; two at least, which hold
// the epilogue's four 32 x 33 transpose tiles)
template <int SW> __host__ __device__ constexpr int smem_bytes(int ns) { return 1024 + ns * stage_bytes<SW>() + 256; }
static_assert(2 * stage_bytes<0>() >= 4 * 32 * 33 * 4 && 2 * stage_bytes<1>() >= 4 * 32 * 33 * 4,
              "transpose tiles fit in two stages");

// instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units, 14 bits each), the fixed 0b001 at bit 46, swizzle
// mode at bit 61 (0 none, 2 128-byte)
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)swz << 61);
}

__device__ __forceinline__ void tma_load2(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load3b(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// the mbarrier arrives once every tcgen05 operation this thread issued has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive f32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ int g_fail;   // a bounded wait gave up in some CTA

// Epilogue and batch: Y[b] = alpha diag(row_scale) A[b] B[b]^T (+ Y if
// accumulate, + bias, ReLU if relu), Y[b] at Y + b sy; Yb a bf16 copy
struct Epi {
    float *Y;
    long long sy;
    unsigned short *Yb;
    const float *bias, *row_scale;
    float alpha;
    int ldy, relu, accumulate;
    int a3, b3;   // A, B tensor maps carry a batch dimension (else shared by the batch)
    int ystore;   // the persistent kernel stores Y by TMA (no accumulate, no bf16 copy)
};

template <int SW>
__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ma,
                                                   const __grid_constant__ CUtensorMap mb, const Epi E, int M, int N,
                                                   int K, int NS) {
    typedef Cfg<SW> C;
    constexpr int BK = C::BK, KSTEPS = BK / 16;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned stages (the 128-byte swizzle repeats every 8 rows of 128 bytes)
    const uint32_t base = sa(smem_raw);
    unsigned char *sm = smem_raw + ((1024u - (base & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + NS * stage_bytes<SW>());
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;
    uint32_t *tholder = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int s_ok;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, bz = blockIdx.z;
    const int nk = (K + BK - 1) / BK;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tholder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tholder;

    if (tid == 0) {
        auto issue = [&](int c, int s) {
            unsigned char *a = sm + s * stage_bytes<SW>();
            unsigned char *b = a + a_bytes<SW>();
            mbar_expect_tx(&full[s], (uint32_t)stage_bytes<SW>());
            if (SW) {
                if (E.a3) tma_load3b(a, &ma, &full[s], c * BK, m0, bz);
                else tma_load2(a, &ma, &full[s], c * BK, m0);
                if (E.b3) tma_load3b(b, &mb, &full[s], c * BK, n0, bz);
                else tma_load2(b, &mb, &full[s], c * BK, n0);
            } else {
                tma_load3b(a, &ma, &full[s], 0, m0, c * (BK / 8));
                tma_load3b(b, &mb, &full[s], 0, n0, c * (BK / 8));
            }
        };
        bool ok = true;
        int issued = 0;   // slices whose loads were issued
        for (int c = 0; c < NS && c < nk; ++c) issue(c, c), ++issued;
        int c = 0;
        for (; c < nk; ++c) {
            const int s = c % NS;
            if (!mbar_wait(&full[s], (uint32_t)(c / NS) & 1u)) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t a0 = sa(sm + s * stage_bytes<SW>()), b0 = a0 + a_bytes<SW>();
#pragma unroll
            for (int k = 0; k < KSTEPS; ++k) {
                uint64_t da, db;
                if (SW) {
                    da = mdesc(a0 + 32u * k, 16u, 1024u, 2u);
                    db = mdesc(b0 + 32u * k, 16u, 1024u, 2u);
                } else {
                    da = mdesc(a0 + 2u * k * (BM * 16u), BM * 16u, 128u, 0u);
                    db = mdesc(b0 + 2u * k * (BN * 16u), BN * 16u, 128u, 0u);
                }
                mma_f16(tmem, da, db, IDESC, (c | k) != 0);
            }
            mma_commit(&empty[s]);
            // refill the stage of the previous slice, whose MMAs have had a slice's time to finish
            if (c >= 1 && c - 1 + NS < nk) {
                const int sp = (c - 1) % NS;
                if (!mbar_wait(&empty[sp], (uint32_t)((c - 1) / NS) & 1u)) {
                    ok = false;
                    break;
                }
                issue(c - 1 + NS, sp);
                ++issued;
            }
        }
        mma_commit(done);   // completes once every MMA issued above has
        if (!ok) {
            atomicOr(&g_fail, 1);
            s_ok = 0;
            // let the loads in flight land before the CTA ends
            for (int r = c + 1; r < issued; ++r) mbar_wait(&full[r % NS], (uint32_t)(r / NS) & 1u);
        }
    }
    const bool dok = mbar_wait(done, 0);
    fence_after();
    __syncthreads();
    if (dok && s_ok) {
        // each warp moves its 32 rows through a 32 x 32 transpose tile in the
        // (now idle) stage memory, so that a row is stored by 32 lanes at once
        float *tile = reinterpret_cast<float *>(sm) + warp * (32 * 33);
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cc = 0; cc < BN; cc += 32) {
            uint32_t r[32];
            tmem_ld32(trow + (uint32_t)cc, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const int n = n0 + cc + lane;
            const float bn = (E.bias && n < N) ? E.bias[n] : 0.f;
            float *Yz = E.Y + (long long)bz * E.sy;
            unsigned short *Ybz = E.Yb ? E.Yb + (long long)bz * E.sy : nullptr;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int row = m0 + warp * 32 + rr;
                if (row < M && n < N) {
                    const long long o = (long long)row * E.ldy + n;
                    float v = tile[rr * 33 + lane];
                    if (E.row_scale) v *= E.alpha * E.row_scale[row];
                    else if (E.alpha != 1.f) v *= E.alpha;
                    if (E.accumulate) v += Yz[o];
                    v += bn;
                    if (E.relu) v = fmaxf(v, 0.f);
                    Yz[o] = v;
                    if (Ybz) Ybz[o] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
                }
            }
            __syncwarp();
        }
    } else if (!dok && tid == 0) {
        atomicOr(&g_fail, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---- the persistent form (128-byte swizzled slices) ----
//
// One CTA per half SM walks the output tiles t = blockIdx.x, + gridDim.x, ...
// (n fastest, then m, then the batch) with its warps in three roles:
//   warp 4 (one thread): TMA producer of the K slices, a ring of stages;
//   warp 5 (one thread): MMA issuer, into one of two 128-column accumulators
//     in tensor memory (tile parity), committing each stage back to the
//     producer and each finished accumulator to the epilogue;
//   warps 0-3: epilogue of the previous tile (tensor-memory lanes 32w ..
//     32w+31) through a 32 x 33 transpose tile each, then they hand the
//     accumulator back to the MMA issuer.
// So one tile's loads and MMAs run under the previous tile's epilogue.
constexpr int PNT = 192;
constexpr int PNS = 2;                    // stages of 64-element slices (two CTAs per SM)
constexpr uint32_t PTMEM_COLS = 2 * BN;   // two accumulators
constexpr int PTILE_FLOATS = 4 * 2 * 32 * 32;   // per epilogue warp: two 32 x 32 f32 staging tiles
static_assert(PTILE_FLOATS >= 4 * 32 * 33, "the transpose tiles fit too");
__host__ __device__ constexpr int psmem_bytes() { return 1024 + PNS * stage_bytes<1>() + PTILE_FLOATS * 4 + 256; }

__device__ __forceinline__ void tma_store3(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(sa(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__global__ void __launch_bounds__(PNT, 1) k_gemm_tcp(const __grid_constant__ CUtensorMap ma,
                                                     const __grid_constant__ CUtensorMap mb,
                                                     const __grid_constant__ CUtensorMap my, const Epi E, int M,
                                                     int N, int K, int total_tiles) {
    constexpr int BK = Cfg<1>::BK, KSTEPS = BK / 16;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = sa(smem_raw);
    unsigned char *sm = smem_raw + ((1024u - (base & 1023u)) & 1023u);
    float *tiles = reinterpret_cast<float *>(sm + PNS * stage_bytes<1>());
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + PTILE_FLOATS);
    uint64_t *empty = full + PNS;
    uint64_t *acc_full = empty + PNS;     // [2]
    uint64_t *acc_empty = acc_full + 2;   // [2]
    uint64_t *drain = acc_empty + 2;
    uint32_t *tholder = reinterpret_cast<uint32_t *>(drain + 1);
    __shared__ int s_fail, s_issued, s_consumed;
    volatile int *fail = &s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tn = (N + BN - 1) / BN, tpb = tn * ((M + BM - 1) / BM);
    const int nk = (K + BK - 1) / BK;

    if (tid == 0) {
        for (int s = 0; s < PNS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);   // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = s_consumed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tholder)),
                     "r"(PTMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tholder;

    if (warp == 4) {
        if (lane == 0) {   // producer
            int it = 0;
            for (int t = blockIdx.x; t < total_tiles && !*fail; t += gridDim.x) {
                const int b = t / tpb, r = t % tpb, m0 = (r / tn) * BM, n0 = (r % tn) * BN;
                for (int c = 0; c < nk; ++c, ++it) {
                    const int s = it % PNS, u = it / PNS;
                    if (u >= 1 && !mbar_wait(&empty[s], (uint32_t)(u - 1) & 1u)) {
                        *fail = 1;
                        break;
                    }
                    unsigned char *a = sm + s * stage_bytes<1>();
                    mbar_expect_tx(&full[s], (uint32_t)stage_bytes<1>());
                    if (E.a3) tma_load3b(a, &ma, &full[s], c * BK, m0, b);
                    else tma_load2(a, &ma, &full[s], c * BK, m0);
                    if (E.b3) tma_load3b(a + a_bytes<1>(), &mb, &full[s], c * BK, n0, b);
                    else tma_load2(a + a_bytes<1>(), &mb, &full[s], c * BK, n0);
                }
            }
            s_issued = it;
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            int it = 0, lt = 0;
            for (int t = blockIdx.x; t < total_tiles && !*fail; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (lt >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((lt >> 1) - 1) & 1u)) {
                    *fail = 1;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int c = 0; c < nk; ++c, ++it) {
                    const int s = it % PNS;
                    if (!mbar_wait(&full[s], (uint32_t)(it / PNS) & 1u)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t a0 = sa(sm + s * stage_bytes<1>()), b0 = a0 + a_bytes<1>();
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k)
                        mma_f16(d, mdesc(a0 + 32u * k, 16u, 1024u, 2u), mdesc(b0 + 32u * k, 16u, 1024u, 2u), IDESC,
                                (c | k) != 0);
                    mma_commit(&empty[s]);
                }
                mma_commit(&acc_full[buf]);
                if (!ok) {
                    *fail = 1;
                    break;
                }
            }
            s_consumed = it;
            // completes once every MMA issued here has
            mma_commit(drain);
        }
    } else {   // epilogue warps 0-3
        float *tile = tiles + warp * (32 * 33);
        float *stage_y = tiles + warp * (2 * 32 * 32);   // two 4 KB staging tiles, 1024-byte aligned
        int lt = 0, ny = 0;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            const bool ok = mbar_wait(&acc_full[buf], (uint32_t)(lt >> 1) & 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *fail = 1;
                break;
            }
            if (*fail) break;
            fence_after();
            const int b = t / tpb, r = t % tpb, m0 = (r / tn) * BM, n0 = (r % tn) * BN;
            const uint32_t trow = tmem + (uint32_t)(buf * BN) + ((uint32_t)(warp * 32) << 16);
            if (E.ystore) {
                // row m0 + 32 w + lane in registers; scaled, biased, ReLU'd there,
                // written to a 128-byte-swizzled staging tile and stored by TMA
                const int row = m0 + warp * 32 + lane;
                const float rs = E.row_scale ? (row < M ? E.alpha * E.row_scale[row] : 0.f) : E.alpha;
#pragma unroll 1
                for (int cc = 0; cc < BN; cc += 32, ++ny) {
                    uint32_t rr32[32];
                    tmem_ld32(trow + (uint32_t)cc, rr32);
                    float *st = stage_y + (ny & 1) * (32 * 32);
                    // the staging tile written two chunks ago has been read by its store
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 v;
                        float *pv = reinterpret_cast<float *>(&v);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int n = n0 + cc + 4 * q + e;
                            float x = __uint_as_float(rr32[4 * q + e]) * rs;
                            if (E.bias) x += n < N ? E.bias[n] : 0.f;
                            if (E.relu) x = fmaxf(x, 0.f);
                            pv[e] = x;
                        }
                        sts4(st + lane * 32 + ((q ^ (lane & 7)) * 4), v);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        if (m0 + warp * 32 < M && n0 + cc < N) tma_store3(&my, st, n0 + cc, m0 + warp * 32, b);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
            } else {
                float *Yz = E.Y + (long long)b * E.sy;
                unsigned short *Ybz = E.Yb ? E.Yb + (long long)b * E.sy : nullptr;
#pragma unroll 1
                for (int cc = 0; cc < BN; cc += 32) {
                    uint32_t rr32[32];
                    tmem_ld32(trow + (uint32_t)cc, rr32);
#pragma unroll
                    for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(rr32[j]);
                    __syncwarp();
                    const int n = n0 + cc + lane;
                    const float bn = (E.bias && n < N) ? E.bias[n] : 0.f;
#pragma unroll 4
                    for (int rr = 0; rr < 32; ++rr) {
                        const int row = m0 + warp * 32 + rr;
                        if (row < M && n < N) {
                            const long long o = (long long)row * E.ldy + n;
                            float v = tile[rr * 33 + lane];
                            if (E.row_scale) v *= E.alpha * E.row_scale[row];
                            else if (E.alpha != 1.f) v *= E.alpha;
                            if (E.accumulate) v += Yz[o];
                            v += bn;
                            if (E.relu) v = fmaxf(v, 0.f);
                            Yz[o] = v;
                            if (Ybz) Ybz[o] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
                        }
                    }
                    __syncwarp();
                }
            }
            // the accumulator is read: hand it back to the MMA issuer
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        // the output stores complete before the CTA ends
        if (E.ystore && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    __syncthreads();
    if (warp == 5 && lane == 0) {
        // every MMA this CTA issued has completed before its tensor memory is
        // freed; after a failure, the loads still in flight land first
        if (!mbar_wait(drain, 0)) *fail = 1;
        for (int u = s_consumed; u < s_issued; ++u) mbar_wait(&full[u % PNS], (uint32_t)(u / PNS) & 1u);
    }
    __syncthreads();
    if (tid == 0 && *fail) atomicOr(&g_fail, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PTMEM_COLS) : "memory");
    }
}

// batch > 1 with stride > 0 (elements): a third dimension over the batch
bool encode_kmajor(EncodeTiled enc, CUtensorMap *m, const void *p, int rows, int K, int ld, int box_rows, int sw,
                   int batch = 1, long long stride = 0) {
    if (sw) {
        const int nd = batch > 1 && stride > 0 ? 3 : 2;
        cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
        cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)stride * 2};
        cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
        cuuint32_t es[3] = {1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, nd, const_cast<void *>(p), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    // (8 elements, rows, K / 8): core matrices of 8 rows x 16 bytes
    cuuint64_t dims[3] = {8, (cuuint64_t)rows, (cuuint64_t)(K / 8)};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, 16};
    cuuint32_t box[3] = {8, (cuuint32_t)box_rows, (cuuint32_t)(Cfg<0>::BK / 8)};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_path = 0;                 // sur_gemm_set_path
long long g_launches = 0;       // launches of k_gemm_tc

}  // namespace

int tc_path() { return g_path; }

// Whether (and how) the tcgen05 kernel runs this product: 1 (128-byte
// swizzle), 0 (core matrices), -1 (it cannot: sur_gemm_bf16 runs mma.sync).
int tc_layout(const void *A, int lda, int a_kmajor, const void *B, int ldb, int b_kmajor, int K) {
    if (g_path == 1) return -1;
    const bool kmajor = a_kmajor && b_kmajor && lda % 8 == 0 && ldb % 8 == 0 &&
                        (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    if (!kmajor) return -1;
    if (g_path == 3) return K % 8 == 0 ? 0 : -1;
    return 1;
}

namespace {
// launch of k_gemm_tc over batch products (layout 1 only when batch > 1)
int launch_tc(int layout, const void *A, int lda, long long sa, const void *B, int ldb, long long sb, int batch,
              Epi E, int M, int N, int K, cudaStream_t s) {
    static bool attr_set[2] = {false, false};
    EncodeTiled enc = encoder();
    if (!enc) return FDTD_ERR_CUDA;
    CUtensorMap ma, mb, my;
    E.a3 = batch > 1 && sa > 0;
    E.b3 = batch > 1 && sb > 0;
    // Y by TMA (persistent kernel): no accumulate, no bf16 copy, 16-byte rows and batch stride
    E.ystore = layout == 1 && !E.accumulate && !E.Yb && E.ldy % 4 == 0 && E.sy % 4 == 0 &&
               (reinterpret_cast<uintptr_t>(E.Y) & 15) == 0;
    if (E.ystore) {
        cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)batch};
        cuuint64_t strides[2] = {(cuuint64_t)E.ldy * 4, (cuuint64_t)(batch > 1 ? E.sy : (long long)M * E.ldy) * 4};
        cuuint32_t box[3] = {32, 32, 1};
        cuuint32_t es[3] = {1, 1, 1};
        E.ystore = enc(&my, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, E.Y, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (!E.ystore) std::memset(&my, 0, sizeof(my));   // unused
    if (!encode_kmajor(enc, &ma, A, M, K, lda, BM, layout, batch, sa) ||
        !encode_kmajor(enc, &mb, B, N, K, ldb, BN, layout, batch, sb))
        return FDTD_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (layout == 1) {
        // persistent: two CTAs per SM over all output tiles of the batch
        static int sms = 0;
        if (sms == 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                sms = 0;
            if (sms <= 0) {
                cudaGetLastError();
                return FDTD_ERR_CUDA;
            }
        }
        const long long tiles = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * batch;
        if (tiles > (1LL << 31) - 1) return FDTD_ERR_ARG;
        const int grid = (int)std::min<long long>(tiles, 2LL * sms);
        if (!attr_set[1])
            e = cudaFuncSetAttribute(k_gemm_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem_bytes());
        attr_set[1] = e == cudaSuccess;
        if (e == cudaSuccess) k_gemm_tcp<<<grid, PNT, psmem_bytes(), s>>>(ma, mb, my, E, M, N, K, (int)tiles);
    } else {
        const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
        const int nk = (K + Cfg<0>::BK - 1) / Cfg<0>::BK, ns = nk < 2 ? 2 : nk < Cfg<0>::NS ? nk : Cfg<0>::NS;
        if (!attr_set[0])
            e = cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<0>(Cfg<0>::NS));
        attr_set[0] = e == cudaSuccess;
        if (e == cudaSuccess) k_gemm_tc<0><<<grid, NT, smem_bytes<0>(ns), s>>>(ma, mb, E, M, N, K, ns);
    }
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return FDTD_ERR_CUDA;
    ++g_launches;
    return FDTD_OK;
}
}  // namespace

int gemm_tc(int layout, const void *A, int lda, const void *B, int ldb, float *Y, int ldy, void *Yb, int M, int N,
            int K, const float *bias, int relu, int accumulate, cudaStream_t s) {
    Epi E;
    E.Y = Y;
    E.sy = 0;
    E.Yb = static_cast<unsigned short *>(Yb);
    E.bias = bias;
    E.row_scale = nullptr;
    E.alpha = 1.f;
    E.ldy = ldy;
    E.relu = relu;
    E.accumulate = accumulate;
    return launch_tc(layout, A, lda, 0, B, ldb, 0, 1, E, M, N, K, s);
}

}  // namespace gtc
}  // namespace fdtd

extern "C" {

int sur_gemm_set_path(int path) {
    if (path < 0 || path > 3) return FDTD_ERR_ARG;
    fdtd::gtc::g_path = path;
    return FDTD_OK;
}

long long sur_gemm_tc_launches(void) { return fdtd::gtc::g_launches; }

int sur_gemm_bf16_batched(const void *A, int lda, long long sa, const void *B, int ldb, long long sb, float *Y, int ldy,
                          long long sy, int M, int N, int K, int batch, const float *row_scale, float alpha,
                          void *stream) {
    using namespace fdtd::gtc;
    if (!A || !B || !Y || M < 1 || N < 1 || K < 1 || batch < 1 || batch > 65535 || lda < K || ldb < K || ldy < N ||
        sa < 0 || sb < 0 || lda % 8 || ldb % 8 || sa % 8 || sb % 8 ||
        (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) ||
        (batch > 1 && sy < (long long)M * ldy) || g_path == 1 || g_path == 3)
        return FDTD_ERR_ARG;
    Epi E;
    E.Y = Y;
    E.sy = sy;
    E.Yb = nullptr;
    E.bias = nullptr;
    E.row_scale = row_scale;
    E.alpha = alpha;
    E.ldy = ldy;
    E.relu = 0;
    E.accumulate = 0;
    return launch_tc(1, A, lda, sa, B, ldb, sb, batch, E, M, N, K, static_cast<cudaStream_t>(stream));
}

int sur_gemm_tc_failed(void) {
    int f = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&f, fdtd::gtc::g_fail, sizeof(int)) != cudaSuccess ||
        cudaMemcpyToSymbol(fdtd::gtc::g_fail, &zero, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    return f;
}

}  // extern "C"
