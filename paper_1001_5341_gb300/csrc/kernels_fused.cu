// kernels_fused.cu -- one-pass leapfrog step: H^{n+1/2} and E^{n+1} in a single
// sweep over z (Yee scheme, Sec. III.A; source of Sec. III.B).
//
// Each CTA owns a TX x TY column of cells and marches up a chunk of z planes.
// For every plane k it
//   A. computes H^{n+1/2}(k) on its cells plus a one-cell halo at i0-1 / j0-1
//      (recomputed from E^n and H^{n-1/2}, never stored), keeping the plane in
//      shared memory and storing its own cells to the output set;
//   B. computes E^{n+1}(k) on its cells from H^{n+1/2}(k) (shared memory) and
//      H^{n+1/2}(k-1) (registers: each thread keeps its own cells' Hx, Hy from
//      the previous plane), adds the shower's current and stores.
// So every field value is read once and written once per step: 24 B read and
// 24 B written per cell, against 72 B for an H sweep followed by an E sweep.
//
// Planes of the input set (E^n and H^{n-1/2}, six components, each a box of
// (TX+8) x (TY+2) floats from x = i0-4, y = j0-1, the x origin kept on a
// 16-byte boundary) are brought into a ring of NS shared-memory stages by TMA
// (cp.async.bulk.tensor.3d) and tracked with one mbarrier per stage; plane
// k+1 and the planes after it stream in while plane k is computed.  Out-of-grid
// parts of a box read as zero.  A chunk that starts at k0 > 0 first recomputes
// H^{n+1/2}(k0-1) for its own cells (no stores).  Every wait on an mbarrier is
// bounded; on expiry the CTA records the failure in a device flag and stops.
#include <cuda.h>
#include <cuda_runtime.h>

#include <new>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

constexpr int TX = 64;              // cells per tile in x
constexpr int TY = 8;               // cells per tile in y
constexpr int NT = 256;             // threads per CTA
constexpr int NS = 4;               // pipeline stages (planes in shared memory)
constexpr int RY = TY / (NT / TX);  // cells per thread (stacked in y)
constexpr int BX = TX + 8;          // box width: x from i0-4 to i0+TX+3
constexpr int BY = TY + 2;          // box height: y from j0-1 to j0+TY
constexpr int BOX = BX * BY;        // floats per component plane
constexpr int BOXP = (BOX + 31) / 32 * 32;  // box stride: every box starts on 128 bytes
constexpr int STAGE = 6 * BOXP;     // floats per stage (Ex Ey Ez Hx Hy Hz)
constexpr int HP = TX + 1;          // row pitch of the H^{n+1/2} plane (halo column first)
constexpr int HSZ = HP * (TY + 1);  // floats per component of that plane
constexpr unsigned STAGE_BYTES = 6u * BOX * 4u;  // bytes the TMA writes per stage
constexpr size_t BAR_BYTES = 128;   // mbarriers first, stages from offset 128
constexpr size_t SMEM_BYTES = BAR_BYTES + (size_t)NS * STAGE * 4 + 3 * (size_t)HSZ * 4;
static_assert(NS * 8 <= BAR_BYTES, "barrier area");
static_assert(NT % TX == 0 && TY % (NT / TX) == 0, "thread layout");
static_assert((BX * 4) % 16 == 0, "TMA box row must be a multiple of 16 bytes");
static_assert(TY <= NT - 2 * TX, "halo column threads");

struct Maps {
    CUtensorMap m[2][6];  // [set][component]
};

struct Args {
    Grid g;
    float *eout;          // Ex of the output set (Ey, Ez follow at +comp)
    float *hout;          // Hx of the output set
    Cpml pml;
    Source src;
    float kE, kH;
    long long n;          // step index (source position)
    int cur;              // input set
    int tiles_x;
    int chunk;            // planes per CTA
    int *flags;
};

struct HostState {
    Maps maps;
    int tiles_x, tiles_y, chunks, chunk;
};

// ---- PTX wrappers (TMA, mbarrier) ---------------------------------------------

__device__ __forceinline__ uint32_t sa(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes)
                 : "memory");
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

// Bounded wait: gives up after about two seconds of clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (4LL << 30)) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_box(float *dst, const CUtensorMap *map, uint64_t *bar,
                                             int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

// ---- stencil pieces on the shared-memory planes --------------------------------

// index of cell (ii, jj) (relative to i0, j0) in a stage box
__device__ __forceinline__ int bx(int ii, int jj) { return (jj + 1) * BX + (ii + 4); }
// index of cell (ii, jj) in the H^{n+1/2} plane (ii, jj >= -1)
__device__ __forceinline__ int hx(int ii, int jj) { return (jj + 1) * HP + (ii + 1); }

// psi of the H update: read step n-1/2, optionally write step n+1/2
__device__ __forceinline__ void psi_h(const float *pin, float *pout, long long q, const float *a,
                                      const float *b, int pos, float &d, bool write) {
    float p = b[pos] * pin[q] + a[pos] * d;
    if (write) pout[q] = p;
    d = d + p;
}
__device__ __forceinline__ void psi_e(float *pe, long long q, const float *a, const float *b,
                                      int pos, float &d) {
    float p = b[pos] * pe[q] + a[pos] * d;
    pe[q] = p;
    d = d + p;
}

// H^{n+1/2} components at cell (i, j, k) = (i0+ii, j0+jj, k); sa_/sb_: stage of planes k, k+1
__device__ __forceinline__ float calc_hx(const Args &A, const float *s0, const float *s1, int ii,
                                         int jj, int i, int j, int k, bool w) {
    float dy = s0[2 * BOXP + bx(ii, jj + 1)] - s0[2 * BOXP + bx(ii, jj)];
    float dz = s1[1 * BOXP + bx(ii, jj)] - s0[1 * BOXP + bx(ii, jj)];
    const Cpml &p = A.pml;
    if (p.P > 0) {
        int ly = slab_cell(j, A.g.ny, p.P), lz = slab_cell(k, A.g.nz, p.P);
        if (ly >= 0) psi_h(p.hin[1][0], p.hout[1][0], psi_y(A.g, p.W, i, ly, k), p.aH[1], p.bH[1], j, dy, w);
        if (lz >= 0) psi_h(p.hin[2][0], p.hout[2][0], psi_z(A.g, p.W, i, j, lz), p.aH[2], p.bH[2], k, dz, w);
    }
    return s0[3 * BOXP + bx(ii, jj)] - A.kH * (dy - dz);
}

__device__ __forceinline__ float calc_hy(const Args &A, const float *s0, const float *s1, int ii,
                                         int jj, int i, int j, int k, bool w) {
    float dz = s1[0 * BOXP + bx(ii, jj)] - s0[0 * BOXP + bx(ii, jj)];
    float dx = s0[2 * BOXP + bx(ii + 1, jj)] - s0[2 * BOXP + bx(ii, jj)];
    const Cpml &p = A.pml;
    if (p.P > 0) {
        int lz = slab_cell(k, A.g.nz, p.P), lx = psi_x_pos(i, A.g.nx, p.P);
        if (lz >= 0) psi_h(p.hin[2][1], p.hout[2][1], psi_z(A.g, p.W, i, j, lz), p.aH[2], p.bH[2], k, dz, w);
        if (lx >= 0) psi_h(p.hin[0][0], p.hout[0][0], psi_x(A.g, p.P, lx, j, k), p.aH[0], p.bH[0], i, dx, w);
    }
    return s0[4 * BOXP + bx(ii, jj)] - A.kH * (dz - dx);
}

__device__ __forceinline__ float calc_hz(const Args &A, const float *s0, int ii, int jj, int i,
                                         int j, int k, bool w) {
    float dx = s0[1 * BOXP + bx(ii + 1, jj)] - s0[1 * BOXP + bx(ii, jj)];
    float dy = s0[0 * BOXP + bx(ii, jj + 1)] - s0[0 * BOXP + bx(ii, jj)];
    const Cpml &p = A.pml;
    if (p.P > 0) {
        int lx = psi_x_pos(i, A.g.nx, p.P), ly = slab_cell(j, A.g.ny, p.P);
        if (lx >= 0) psi_h(p.hin[0][1], p.hout[0][1], psi_x(A.g, p.P, lx, j, k), p.aH[0], p.bH[0], i, dx, w);
        if (ly >= 0) psi_h(p.hin[1][1], p.hout[1][1], psi_y(A.g, p.W, i, ly, k), p.aH[1], p.bH[1], j, dy, w);
    }
    return s0[5 * BOXP + bx(ii, jj)] - A.kH * (dx - dy);
}

__global__ void __launch_bounds__(NT, 2) k_fused(const Args A, const __grid_constant__ Maps maps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *stages = reinterpret_cast<float *>(smem_raw + BAR_BYTES);
    float *Hs = stages + NS * STAGE;  // [3][TY+1][TX+1]: Hx, Hy, Hz of plane k

    const Grid &g = A.g;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int i0 = (tile % A.tiles_x) * TX;
    const int j0 = (tile / A.tiles_x) * TY;
    const int k0 = blockIdx.y * A.chunk;
    if (k0 >= g.nz) return;
    const int k1 = min(g.nz, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    const int nplanes = k1 - kstart + 1;  // planes kstart..k1 of the input set
    const CUtensorMap *mp = maps.m[A.cur];

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int r = 0; r < NS && r < nplanes; ++r) {
            float *dst = stages + r * STAGE;
            mbar_expect_tx(&bar[r], STAGE_BYTES);
            for (int c = 0; c < 6; ++c) tma_load_box(dst + c * BOXP, &mp[c], &bar[r], i0 - 4, j0 - 1, kstart + r);
        }
    }

    const int tx = tid % TX;
    const int ty = tid / TX;
    const int i = i0 + tx;
    float hxp[RY], hyp[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) { hxp[r] = 0.0f; hyp[r] = 0.0f; }

    for (int rel = 0; rel + kstart < k1; ++rel) {
        const int k = kstart + rel;
        bool ok = true;
        if (rel == 0) ok = mbar_wait(&bar[0], 0);
        ok = ok && mbar_wait(&bar[(rel + 1) % NS], ((rel + 1) / NS) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.flags, 1);
            // let the copies already issued land before the CTA's memory is released
            if (tid == 0)
                for (int r = rel; r < nplanes && r < rel + NS; ++r) mbar_wait(&bar[r % NS], (r / NS) & 1);
            __syncthreads();
            return;
        }
        const float *s0 = stages + (rel % NS) * STAGE;
        const float *s1 = stages + ((rel + 1) % NS) * STAGE;
        const bool own = k >= k0;  // false: recompute H(k0-1) only

        // ---- A: H^{n+1/2}(k) ----
        float hxv[RY], hyv[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int jj = ty + r * (NT / TX);
            const int j = j0 + jj;
            float vx = 0.0f, vy = 0.0f, vz = 0.0f;
            if (i < g.nx && j < g.ny) {
                if (i >= 1) vx = calc_hx(A, s0, s1, tx, jj, i, j, k, own);
                if (j >= 1) vy = calc_hy(A, s0, s1, tx, jj, i, j, k, own);
                if (own && k >= 1) vz = calc_hz(A, s0, tx, jj, i, j, k, true);
                if (own) {
                    const long long c = gidx(g, i, j, k);
                    if (i >= 1) A.hout[c] = vx;
                    if (j >= 1) A.hout[g.comp + c] = vy;
                    if (k >= 1) A.hout[2 * g.comp + c] = vz;
                }
            }
            hxv[r] = vx;
            hyv[r] = vy;
            if (own) {
                Hs[0 * HSZ + hx(tx, jj)] = vx;
                Hs[1 * HSZ + hx(tx, jj)] = vy;
                Hs[2 * HSZ + hx(tx, jj)] = vz;
            }
        }
        if (own) {
            // halo row j0-1 (Hx, Hz) and halo column i0-1 (Hy, Hz), not stored
            if (ty == 0 && j0 >= 1) {
                const int j = j0 - 1;
                float vx = 0.0f, vz = 0.0f;
                if (i < g.nx) {
                    if (i >= 1) vx = calc_hx(A, s0, s1, tx, -1, i, j, k, false);
                    if (k >= 1) vz = calc_hz(A, s0, tx, -1, i, j, k, false);
                }
                Hs[0 * HSZ + hx(tx, -1)] = vx;
                Hs[2 * HSZ + hx(tx, -1)] = vz;
            }
            const int hc = tid - 2 * TX;
            if (hc >= 0 && hc < TY && i0 >= 1) {
                const int j = j0 + hc, ih = i0 - 1;
                float vy = 0.0f, vz = 0.0f;
                if (j < g.ny) {
                    if (j >= 1) vy = calc_hy(A, s0, s1, -1, hc, ih, j, k, false);
                    if (k >= 1) vz = calc_hz(A, s0, -1, hc, ih, j, k, false);
                }
                Hs[1 * HSZ + hx(-1, hc)] = vy;
                Hs[2 * HSZ + hx(-1, hc)] = vz;
            }
        }
        __syncthreads();

        // ---- B: E^{n+1}(k) ----
        if (own) {
            const Cpml &p = A.pml;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int jj = ty + r * (NT / TX);
                const int j = j0 + jj;
                if (i < g.nx && j < g.ny) {
                    const long long c = gidx(g, i, j, k);
                    const int lx = psi_x_pos(i, g.nx, p.P), ly = slab_cell(j, g.ny, p.P),
                              lz = slab_cell(k, g.nz, p.P);
                    if (j >= 1 && k >= 1) {  // Ex
                        float dy = Hs[2 * HSZ + hx(tx, jj)] - Hs[2 * HSZ + hx(tx, jj - 1)];
                        float dz = hyv[r] - hyp[r];
                        if (ly >= 0) psi_e(p.e[1][0], psi_y(g, p.W, i, ly, k), p.aE[1], p.bE[1], j, dy);
                        if (lz >= 0) psi_e(p.e[2][0], psi_z(g, p.W, i, j, lz), p.aE[2], p.bE[2], k, dz);
                        A.eout[c] = s0[0 * BOXP + bx(tx, jj)] + A.kE * (dy - dz);
                    }
                    if (i >= 1 && k >= 1) {  // Ey
                        float dz = hxv[r] - hxp[r];
                        float dx = Hs[2 * HSZ + hx(tx, jj)] - Hs[2 * HSZ + hx(tx - 1, jj)];
                        if (lz >= 0) psi_e(p.e[2][1], psi_z(g, p.W, i, j, lz), p.aE[2], p.bE[2], k, dz);
                        if (lx >= 0) psi_e(p.e[0][0], psi_x(g, p.P, lx, j, k), p.aE[0], p.bE[0], i, dx);
                        A.eout[g.comp + c] = s0[1 * BOXP + bx(tx, jj)] + A.kE * (dz - dx);
                    }
                    if (i >= 1 && j >= 1) {  // Ez
                        float dx = Hs[1 * HSZ + hx(tx, jj)] - Hs[1 * HSZ + hx(tx - 1, jj)];
                        float dy = Hs[0 * HSZ + hx(tx, jj)] - Hs[0 * HSZ + hx(tx, jj - 1)];
                        if (lx >= 0) psi_e(p.e[0][1], psi_x(g, p.P, lx, j, k), p.aE[0], p.bE[0], i, dx);
                        if (ly >= 0) psi_e(p.e[1][1], psi_y(g, p.W, i, ly, k), p.aE[1], p.bE[1], j, dy);
                        float e = s0[2 * BOXP + bx(tx, jj)] + A.kE * (dx - dy);
                        if (A.src.active) e += source_term(A.src, i, j, k, A.n);
                        A.eout[2 * g.comp + c] = e;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) { hxp[r] = hxv[r]; hyp[r] = hyv[r]; }
        __syncthreads();  // plane rel fully consumed; H plane free for reuse
        if (tid == 0 && rel + NS < nplanes) {
            const int r = rel + NS;
            float *dst = stages + (r % NS) * STAGE;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[r % NS], STAGE_BYTES);
            for (int c = 0; c < 6; ++c) tma_load_box(dst + c * BOXP, &mp[c], &bar[r % NS], i0 - 4, j0 - 1, kstart + r);
        }
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

const char *fused_name() { return "fused-tma-64x8"; }

int fused_prepare(fdtd_ctx *h) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->dev);
    if (major < 10) return FDTD_ERR_CUDA;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    EncodeTiled encode = reinterpret_cast<EncodeTiled>(fn);
    HostState *st = new (std::nothrow) HostState();
    if (!st) return FDTD_ERR_OOM;
    const Grid &g = h->g;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx + 1, (cuuint64_t)g.ny + 1, (cuuint64_t)g.nz + 1};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    cuuint32_t box[3] = {BX, BY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 6; ++c) {
            CUresult r = encode(&st->maps.m[s][c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                h->fields[s] + (size_t)c * g.comp, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                delete st;
                return FDTD_ERR_CUDA;
            }
        }
    if (cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) !=
        cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FDTD_ERR_CUDA;
    }
    st->tiles_x = (g.nx + TX - 1) / TX;
    st->tiles_y = (g.ny + TY - 1) / TY;
    // split z so that there are at least ~16 CTAs per SM in flight over the step
    const int tiles = st->tiles_x * st->tiles_y;
    int want = 16 * h->num_sms;
    int chunks = (want + tiles - 1) / tiles;
    int max_chunks = g.nz / 16 > 0 ? g.nz / 16 : 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    st->chunk = (g.nz + chunks - 1) / chunks;
    st->chunks = (g.nz + st->chunk - 1) / st->chunk;
    h->fused = st;
    return FDTD_OK;
}

void fused_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->fused);
    h->fused = nullptr;
}

void launch_fused(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->fused);
    const Grid &g = h->g;
    Args a;
    a.g = g;
    a.eout = h->fields[h->cur ^ 1];
    a.hout = h->fields[h->cur ^ 1] + 3 * g.comp;
    a.pml = cpml_view(h);
    a.src = h->src;
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.n = h->steps;
    a.cur = h->cur;
    a.tiles_x = st->tiles_x;
    a.chunk = st->chunk;
    a.flags = h->d_flags;
    dim3 grid(st->tiles_x * st->tiles_y, st->chunks);
    k_fused<<<grid, NT, SMEM_BYTES, s>>>(a, st->maps);
}

}  // namespace fdtd
