// kernels_vtile.cu -- one-pass leapfrog step over the CPML-free interior box:
// TMA-staged planes, four columns per lane.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B): a step reads E^n and H^{n-1/2}
// once and writes H^{n+1/2} and E^{n+1} once, 24 B + 24 B per cell.
//
// A block owns a tile of 128 columns [i0, i0+128) (i0 a multiple of 128) by
// BY rows and marches up a chunk of z planes.  For every plane p of the input
// set, one thread issues six TMA loads (cp.async.bulk.tensor.3d), one box per
// component of 136 columns x (BY+2) rows starting at (i0-4, jb-1): the tile
// plus a one-cell halo on every side, the x origin on a 16-byte boundary.
// Planes stream into a ring of NS stages tracked by mbarriers, several planes
// ahead of the compute.
//
// Warps 0..BY-1 each own one row of the tile; lane L holds the four columns
// i0+4L .. i0+4L+3 as float4.  Per plane k:
//   H phase: H^{n+1/2}(k) of the own cells from the stages of planes k and k+1
//     (y neighbour j+1 and x neighbour i+1 are vector reads of the stage);
//     warp BY computes the halo H the E update needs: row jb-1 (Hx, Hz) and
//     column i0-1 (Hy, Hz).  All of it goes to a shared H plane; own H is
//     stored to global memory.
//   barrier
//   E phase: E^{n+1}(k) from the H plane (neighbours j-1 and i-1) and the
//     own H^{n+1/2}(k-1) Hx, Hy kept in registers; stored.
//   barrier; the stage of plane k is refilled with plane k+NS.
// A chunk that starts above the box's first plane first runs the H phase of
// plane k0-1 without stores.  Every mbarrier wait is bounded; on expiry the
// block records the failure in a device flag and stops.
#include <cuda.h>
#include <cuda_runtime.h>

#include <new>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

#ifndef VT_BY
#define VT_BY 8
#endif
#ifndef VT_NS
#define VT_NS 4
#endif
constexpr int BY = VT_BY;              // rows per tile (one warp each)
constexpr int NS = VT_NS;              // pipeline stages
constexpr int NW = BY + 1;             // warps: BY row warps + one halo warp
constexpr int NT = 32 * NW;
constexpr int TXC = 128;               // tile columns
constexpr int BXC = TXC + 8;           // box columns: i0-4 .. i0+131
constexpr int BYR = BY + 2;            // box rows: jb-1 .. jb+BY
constexpr int BOX = BXC * BYR;         // floats per component box
constexpr int BOXP = (BOX + 31) / 32 * 32;  // box stride (128-byte aligned)
constexpr int STAGE = 6 * BOXP;        // floats per stage
constexpr unsigned STAGE_BYTES = 6u * BOX * 4u;
constexpr int HR = BY + 1;             // H plane rows: jb-1 .. jb+BY-1
constexpr int HPL = HR * BXC;          // floats per H-plane component
constexpr size_t BAR_BYTES = 128;
constexpr size_t SMEM_BYTES = BAR_BYTES + (size_t)NS * STAGE * 4 + 3 * (size_t)HPL * 4;
static_assert((BXC * 4) % 16 == 0, "box rows must be a multiple of 16 bytes");
static_assert(NS * 8 <= (int)BAR_BYTES, "barrier area");

struct Maps {
    CUtensorMap m[2][6];  // [set][component]
};

struct Args {
    Grid g;
    float *oex, *oey, *oez, *ohx, *ohy, *ohz;   // output set
    int ilo, ihi, jlo, jhi, klo, khi;           // interior box (ilo, ihi+1 multiples of 4)
    int tx0, tiles_x, tiles_y, chunk;
    int cur;
    Source src;
    SourceStep ss;
    float kE, kH;
    int *flags;
};

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: gives up after about two seconds of clock cycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (4LL << 30)) return false;
    return true;
}
__device__ __forceinline__ void tma_load(float *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// box offset of (box column bc, box row br) for component c
__device__ __forceinline__ int bo(int c, int br, int bc) { return c * BOXP + br * BXC + bc; }

__device__ __forceinline__ void issue_plane(const CUtensorMap *mp, float *stage, uint64_t *bar, int i0, int jb, int z) {
    mbar_expect_tx(bar, STAGE_BYTES);
    for (int c = 0; c < 6; ++c) tma_load(stage + c * BOXP, &mp[c], bar, i0 - 4, jb - 1, z);
}

__global__ void __launch_bounds__(NT, 1) k_vtile(const Args A, const __grid_constant__ Maps maps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *stages = reinterpret_cast<float *>(smem_raw + BAR_BYTES);
    float *HS = stages + NS * STAGE;   // [3][HR][BXC]: Hx, Hy, Hz of plane k, column index col - i0 + 4

    const Grid &g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tx = (int)blockIdx.x % A.tiles_x, ty = (int)blockIdx.x / A.tiles_x;
    const int i0 = (A.tx0 + tx) * TXC;
    const int jb = A.jlo + ty * BY;
    const int k0 = A.klo + (int)blockIdx.y * A.chunk;
    const int k1 = min(A.khi + 1, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    const int nplanes = k1 - kstart + 1;   // input planes kstart .. k1
    const CUtensorMap *mp = maps.m[A.cur];

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int r = 0; r < NS && r < nplanes; ++r) issue_plane(mp, stages + r * STAGE, &bar[r], i0, jb, kstart + r);

    // row warps: row j, columns c0..c0+3 (box column bc0 = 4 + 4 lane)
    const bool roww = w < BY;
    const int j = jb + w;
    const int c0 = i0 + 4 * lane;
    const int bc0 = 4 + 4 * lane;
    const int br = w + 1;                 // box row of j
    const bool storable = roww && j <= A.jhi && c0 >= A.ilo && c0 + 3 <= A.ihi;
    const unsigned goff = (unsigned)c0 + (unsigned)j * (unsigned)g.pitch;
    const bool src_blk = A.src.active && i0 <= A.src.ic + A.src.L && i0 + TXC - 1 >= A.src.ic - A.src.L &&
                         jb <= A.src.jc + A.src.L && jb + BY - 1 >= A.src.jc - A.src.L;
    float4 hxp = make_float4(0.f, 0.f, 0.f, 0.f), hyp = hxp;   // own H^{n+1/2}(k-1) Hx, Hy
    const float kH = A.kH, kE = A.kE;

    for (int rel = 0; kstart + rel < k1; ++rel) {
        const int k = kstart + rel;
        bool ok = true;
        if (rel == 0) ok = mbar_wait(&bar[0], 0);
        ok = ok && mbar_wait(&bar[(rel + 1) % NS], ((rel + 1) / NS) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(A.flags, 1);
                for (int r = rel; r < nplanes && r < rel + NS; ++r) mbar_wait(&bar[r % NS], (r / NS) & 1);
            }
            __syncthreads();
            return;
        }
        const float *s0 = stages + (rel % NS) * STAGE;        // plane k
        const float *s1 = stages + ((rel + 1) % NS) * STAGE;  // plane k+1
        const bool own = k >= k0;
        const unsigned goffk = goff + (unsigned)k * (unsigned)g.plane;

        float4 ex0, ey0, ez0, hxn, hyn, hzn;
        if (roww) {
            // ---- H phase, own cells ----
            ex0 = lds4(s0 + bo(0, br, bc0));
            ey0 = lds4(s0 + bo(1, br, bc0));
            ez0 = lds4(s0 + bo(2, br, bc0));
            const float4 hx = lds4(s0 + bo(3, br, bc0));
            const float4 hy = lds4(s0 + bo(4, br, bc0));
            const float4 hz = lds4(s0 + bo(5, br, bc0));
            const float4 exU = lds4(s0 + bo(0, br + 1, bc0));      // row j+1
            const float4 ezU = lds4(s0 + bo(2, br + 1, bc0));
            const float4 eyR = lds4(s0 + bo(1, br, bc0 + 4));      // columns +4: .x is i+1 of .w
            const float4 ezR = lds4(s0 + bo(2, br, bc0 + 4));
            const float4 ex1 = lds4(s1 + bo(0, br, bc0));
            const float4 ey1 = lds4(s1 + bo(1, br, bc0));
            hxn.x = hx.x - kH * ((ezU.x - ez0.x) - (ey1.x - ey0.x));
            hxn.y = hx.y - kH * ((ezU.y - ez0.y) - (ey1.y - ey0.y));
            hxn.z = hx.z - kH * ((ezU.z - ez0.z) - (ey1.z - ey0.z));
            hxn.w = hx.w - kH * ((ezU.w - ez0.w) - (ey1.w - ey0.w));
            hyn.x = hy.x - kH * ((ex1.x - ex0.x) - (ez0.y - ez0.x));
            hyn.y = hy.y - kH * ((ex1.y - ex0.y) - (ez0.z - ez0.y));
            hyn.z = hy.z - kH * ((ex1.z - ex0.z) - (ez0.w - ez0.z));
            hyn.w = hy.w - kH * ((ex1.w - ex0.w) - (ezR.x - ez0.w));
            hzn.x = hz.x - kH * ((ey0.y - ey0.x) - (exU.x - ex0.x));
            hzn.y = hz.y - kH * ((ey0.z - ey0.y) - (exU.y - ex0.y));
            hzn.z = hz.z - kH * ((ey0.w - ey0.z) - (exU.z - ex0.z));
            hzn.w = hz.w - kH * ((eyR.x - ey0.w) - (exU.w - ex0.w));
            if (own) {
                sts4(HS + 0 * HPL + br * BXC + bc0, hxn);
                sts4(HS + 1 * HPL + br * BXC + bc0, hyn);
                sts4(HS + 2 * HPL + br * BXC + bc0, hzn);
                if (storable) {
                    // components on the grid's low faces are not updated
                    float4 sx = hxn, sy = hyn, sz = hzn;
                    if (c0 == 0) sx.x = 0.f;
                    if (j == 0) sy = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k == 0) sz = make_float4(0.f, 0.f, 0.f, 0.f);
                    *reinterpret_cast<float4 *>(A.ohx + goffk) = sx;
                    *reinterpret_cast<float4 *>(A.ohy + goffk) = sy;
                    *reinterpret_cast<float4 *>(A.ohz + goffk) = sz;
                }
            }
        } else if (own) {
            // ---- halo warp: H at row jb-1 (Hx, Hz), columns i0-4 .. i0+127 ----
            for (int q = lane; q < TXC / 4 + 1; q += 32) {
                const int bc = 4 * q;   // box columns bc .. bc+3
                const float4 ex = lds4(s0 + bo(0, 0, bc)), ey = lds4(s0 + bo(1, 0, bc)), ez = lds4(s0 + bo(2, 0, bc));
                const float4 hx = lds4(s0 + bo(3, 0, bc)), hz = lds4(s0 + bo(5, 0, bc));
                const float4 exU = lds4(s0 + bo(0, 1, bc)), ezU = lds4(s0 + bo(2, 1, bc));
                const float4 ey1 = lds4(s1 + bo(1, 0, bc));
                const float eyRx = s0[bo(1, 0, bc + 4)];
                float4 ox, oz;
                ox.x = hx.x - kH * ((ezU.x - ez.x) - (ey1.x - ey.x));
                ox.y = hx.y - kH * ((ezU.y - ez.y) - (ey1.y - ey.y));
                ox.z = hx.z - kH * ((ezU.z - ez.z) - (ey1.z - ey.z));
                ox.w = hx.w - kH * ((ezU.w - ez.w) - (ey1.w - ey.w));
                oz.x = hz.x - kH * ((ey.y - ey.x) - (exU.x - ex.x));
                oz.y = hz.y - kH * ((ey.z - ey.y) - (exU.y - ex.y));
                oz.z = hz.z - kH * ((ey.w - ey.z) - (exU.z - ex.z));
                oz.w = hz.w - kH * ((eyRx - ey.w) - (exU.w - ex.w));
                sts4(HS + 0 * HPL + 0 * BXC + bc, ox);
                sts4(HS + 2 * HPL + 0 * BXC + bc, oz);
            }
            // column i0-1 (box column 3), rows jb .. jb+BY-1 (Hy, Hz)
            if (lane < BY) {
                const int b = lane + 1;
                const float ey = s0[bo(1, b, 3)], eyR = s0[bo(1, b, 4)];
                const float ex = s0[bo(0, b, 3)], exU = s0[bo(0, b + 1, 3)], ex1 = s1[bo(0, b, 3)];
                const float ez = s0[bo(2, b, 3)], ezR = s0[bo(2, b, 4)];
                const float hy = s0[bo(4, b, 3)], hz = s0[bo(5, b, 3)];
                HS[1 * HPL + b * BXC + 3] = hy - kH * ((ex1 - ex) - (ezR - ez));
                HS[2 * HPL + b * BXC + 3] = hz - kH * ((eyR - ey) - (exU - ex));
            }
        }
        __syncthreads();

        // ---- E phase ----
        if (roww && own) {
            const float4 hzD = lds4(HS + 2 * HPL + (br - 1) * BXC + bc0);   // row j-1
            const float4 hxD = lds4(HS + 0 * HPL + (br - 1) * BXC + bc0);
            const float hzL = HS[2 * HPL + br * BXC + bc0 - 1];             // column i-1 of .x
            const float hyL = HS[1 * HPL + br * BXC + bc0 - 1];
            float4 nex, ney, nez;
            nex.x = ex0.x + kE * ((hzn.x - hzD.x) - (hyn.x - hyp.x));
            nex.y = ex0.y + kE * ((hzn.y - hzD.y) - (hyn.y - hyp.y));
            nex.z = ex0.z + kE * ((hzn.z - hzD.z) - (hyn.z - hyp.z));
            nex.w = ex0.w + kE * ((hzn.w - hzD.w) - (hyn.w - hyp.w));
            ney.x = ey0.x + kE * ((hxn.x - hxp.x) - (hzn.x - hzL));
            ney.y = ey0.y + kE * ((hxn.y - hxp.y) - (hzn.y - hzn.x));
            ney.z = ey0.z + kE * ((hxn.z - hxp.z) - (hzn.z - hzn.y));
            ney.w = ey0.w + kE * ((hxn.w - hxp.w) - (hzn.w - hzn.z));
            nez.x = ez0.x + kE * ((hyn.x - hyL) - (hxn.x - hxD.x));
            nez.y = ez0.y + kE * ((hyn.y - hyn.x) - (hxn.y - hxD.y));
            nez.z = ez0.z + kE * ((hyn.z - hyn.y) - (hxn.z - hxD.z));
            nez.w = ez0.w + kE * ((hyn.w - hyn.z) - (hxn.w - hxD.w));
            if (storable) {
                if (src_blk) {
                    nez.x += source_at(A.src, A.ss, c0, j, k);
                    nez.y += source_at(A.src, A.ss, c0 + 1, j, k);
                    nez.z += source_at(A.src, A.ss, c0 + 2, j, k);
                    nez.w += source_at(A.src, A.ss, c0 + 3, j, k);
                }
                if (j == 0 || k == 0) nex = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k == 0) ney = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c0 == 0) { ney.x = 0.f; nez.x = 0.f; }
                if (j == 0) nez = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(A.oex + goffk) = nex;
                *reinterpret_cast<float4 *>(A.oey + goffk) = ney;
                *reinterpret_cast<float4 *>(A.oez + goffk) = nez;
            }
        }
        if (roww) { hxp = hxn; hyp = hyn; }
        __syncthreads();  // stage of plane k and the H plane are free
        if (tid == 0 && rel + NS < nplanes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_plane(mp, stages + ((rel + NS) % NS) * STAGE, &bar[(rel + NS) % NS], i0, jb, kstart + rel + NS);
        }
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct HostState {
    Maps maps;
    Args proto;
    int blocks_x, chunks;
};

}  // namespace

const char *vtile_name() { return "fused-vtile-128x" "8"; }

int vtile_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    if ((unsigned long long)g.comp >= (1ull << 32) || g.pitch % 4 != 0) return FDTD_ERR_ARG;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    EncodeTiled encode = reinterpret_cast<EncodeTiled>(fn);
    HostState *st = new (std::nothrow) HostState();
    if (!st) return FDTD_ERR_OOM;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx + 1, (cuuint64_t)g.ny + 1, (cuuint64_t)g.nz + 1};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    cuuint32_t box[3] = {BXC, BYR, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 6; ++c)
            if (encode(&st->maps.m[s][c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->fields[s] + (size_t)c * g.comp, dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
                delete st;
                return FDTD_ERR_CUDA;
            }
    if (cudaFuncSetAttribute(k_vtile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FDTD_ERR_CUDA;
    }
    int lo[3], hi[3];
    interior_box(h, lo, hi);
    Args &a = st->proto;
    a.ilo = lo[0]; a.ihi = hi[0]; a.jlo = lo[1]; a.jhi = hi[1]; a.klo = lo[2]; a.khi = hi[2];
    if (a.ihi < a.ilo || a.jhi < a.jlo || a.khi < a.klo) { delete st; return FDTD_ERR_ARG; }
    a.tx0 = a.ilo / TXC;
    a.tiles_x = a.ihi / TXC - a.tx0 + 1;
    a.tiles_y = (a.jhi - a.jlo + BY) / BY;
    const int ez = a.khi - a.klo + 1;
    const int sms = h->num_sms > 0 ? h->num_sms : 1;
    const long long want = 8LL * sms;
    long long chunks = (want + (long long)a.tiles_x * a.tiles_y - 1) / ((long long)a.tiles_x * a.tiles_y);
    if (chunks > ez / 16) chunks = ez / 16;
    if (chunks < 1) chunks = 1;
    a.chunk = (int)((ez + chunks - 1) / chunks);
    st->chunks = (ez + a.chunk - 1) / a.chunk;
    st->blocks_x = a.tiles_x * a.tiles_y;
    h->vtile = st;
    return FDTD_OK;
}

void vtile_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->vtile);
    h->vtile = nullptr;
}

long long vtile_cells(const fdtd_ctx *h) {
    const Args &a = static_cast<const HostState *>(h->vtile)->proto;
    return (long long)(a.ihi - a.ilo + 1) * (a.jhi - a.jlo + 1) * (a.khi - a.klo + 1);
}

void launch_vtile(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->vtile);
    const Grid &g = h->g;
    Args a = st->proto;
    a.g = g;
    float *out = h->fields[h->cur ^ 1];
    const size_t c = (size_t)g.comp;
    a.oex = out; a.oey = out + c; a.oez = out + 2 * c; a.ohx = out + 3 * c; a.ohy = out + 4 * c; a.ohz = out + 5 * c;
    a.cur = h->cur;
    a.src = h->src;
    a.ss = source_window(h->src, h->steps);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.flags = h->d_flags;
    dim3 grid(st->blocks_x, st->chunks);
    k_vtile<<<grid, NT, SMEM_BYTES, s>>>(a, st->maps);
}

}  // namespace fdtd
