// vtile_tile.cuh -- the block body of the one-pass leapfrog step: TMA-staged
// planes, four columns per lane, CPML folded in.  kernels_vtile.cu launches one
// block per (tile, z chunk) of a grid; batch.cu runs the same body over the
// tiles of many grids in one persistent kernel.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B; the paper names no absorbing
// boundary, so the CPML is this library's choice, Roden-Gedney): a step reads
// E^n and H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once, 24 B + 24 B
// per cell, plus the CPML memory of the cells in the layers (16 B read and
// 16 B written per cell and layer axis).
//
// A block owns a tile of 128 columns [i0, i0+128) (i0 a multiple of 128) by
// BY rows and marches up a chunk of z planes.  For every plane of the input
// set, one thread issues the TMA loads (cp.async.bulk.tensor.3d) of one
// pipeline stage: one box per field component holding the tile and the halo
// that component is read at (the x origin on a 16-byte boundary; outside the
// node grid a box reads zeros) -- Ex: columns i0-4..i0+127, rows jb-1..jb+BY;
// Ey: i0-4..i0+131, jb-1..jb+BY-1; Ez: i0-4..i0+131, jb-1..jb+BY; Hx:
// i0..i0+127, jb-1..jb+BY-1; Hy: i0-4..i0+127, jb..jb+BY-1; Hz: i0-4..i0+127,
// jb-1..jb+BY-1 -- and, where the block touches a CPML layer, boxes of the
// four psi arrays of that axis (below).  Stages form a ring tracked by mbarriers; a block
// without CPML work holds up to NSMAX planes in flight, a block with it as
// many as its larger stages leave room for (at least two).
//
// Warps 0..BY-1 each own one row of the tile; lane L holds the four columns
// i0+4L .. i0+4L+3 as float4.  Per plane k:
//   H phase: H^{n+1/2}(k) of the own cells from the stages of planes k and k+1
//     (y neighbour j+1 and x neighbour i+1 are vector reads of the stage);
//     warp BY computes the halo H the E update needs: row jb-1 (Hx, Hz) and
//     column i0-1 (Hy, Hz).  Hx, Hz of the rows a warp below needs and the
//     halo go to a shared H plane (two of them, used by alternate planes);
//     own H is stored to global memory.
//   E phase: E^{n+1}(k) from the H plane (neighbour j-1), the lane to the
//     left (neighbour i-1, a warp shuffle) and the own H^{n+1/2}(k-1) Hx, Hy
//     kept in registers; stored.
// Each thread waits on the mbarrier of the stages it reads itself.  Between
// the phases the body has two forms (tile_block's NB):
//   without block barriers (k_vtile): a row warp's E phase waits only for
//     the H row below and the halo warp's row and column, each signalled on
//     an mbarrier of its writer, and a tenth warp refills a stage once every
//     warp that reads it has signalled it empty (tile_block states the
//     order of waits that keeps every parity wait within one phase);
//   with block barriers (the batch kernel): one block barrier between the
//     phases, after which no thread reads the stage of plane k and thread 0
//     refills it with plane k+ns; blocks with CPML boxes read E psi from the
//     stage in the E phase and refill it after a second barrier.
// A chunk that starts above plane 0 first runs the H phase of plane k0-1
// without stores.  Every mbarrier wait is bounded; on expiry the block records
// the failure in a device flag and stops.
//
// CPML.  psi boxes of a stage (rows jb-1 .. jb+BY-1, so that the halo H has
// its terms too):
//   x: the half of the x rows (low layer or high layer, psi_x_pos) that the
//      tile or its halo column meets;
//   y: 132 columns from i0-4, BY+1 slab rows from l0, when a row of the tile
//      (or the halo row) lies in a y layer; the slab rows of BY+1 consecutive
//      grid rows are consecutive in the slab index, so one box holds them;
//   z: 132 columns x BY+1 rows at slab plane lz, when plane k lies in a z layer.
// A warp is one row, so "row j lies in a y layer" is uniform over the warp;
// "plane k lies in a z layer" is uniform over the block.  In a tile that meets
// an x layer every lane runs the x recursion on its float4: the coefficients
// are zero outside the layer, where it leaves the derivative unchanged, and
// only the lanes with layer columns store psi.  The z chunks are split at the
// z layers, so only the short layer chunks carry z boxes (a middle chunk whose
// warm-up plane lies in a layer reads that plane's H psi directly).  The halo H that a
// block recomputes uses its neighbours' H psi at n-1/2 (read only); the E psi
// are updated in place and the H psi written to the n+1/2 copy by the owner.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "fdtd_internal.h"
#include "source_term.cuh"
#include "tma_pipe.cuh"

namespace fdtd {
namespace vt {

using namespace tma;

#ifndef VT_BY
#define VT_BY 8
#endif
#ifndef VT_NSMAX
#define VT_NSMAX 8
#endif
#ifndef VT_L2PROMO
#define VT_L2PROMO 2   // L2 promotion of the TMA loads: 0 none, 1 64 B, 2 128 B, 3 256 B
#endif
constexpr int BY = VT_BY;              // rows per tile (one warp each)
constexpr int NSMAX = VT_NSMAX;        // most pipeline stages
constexpr int NW = BY + 1;             // warps: BY row warps + one halo warp
constexpr int NT = 32 * NW;
constexpr int TXC = 128;               // tile columns
// field boxes, component c (Ex Ey Ez Hx Hy Hz): columns from i0-4+fb_cb(c),
// rows from jb-1+fb_rb(c), fb_w(c) x fb_r(c) (box column bc = column - i0 + 4,
// box row br = row - jb + 1 in the accessors)
__host__ __device__ constexpr int fb_cb(int c) { return c == 3 ? 4 : 0; }
__host__ __device__ constexpr int fb_rb(int c) { return c == 4 ? 1 : 0; }
__host__ __device__ constexpr int fb_w(int c) { return c == 1 || c == 2 ? TXC + 8 : c == 3 ? TXC : TXC + 4; }
__host__ __device__ constexpr int fb_r(int c) { return c == 0 || c == 2 ? BY + 2 : c == 4 ? BY : BY + 1; }
__host__ __device__ constexpr int fb_size(int c) { return (fb_w(c) * fb_r(c) + 31) / 32 * 32; }
__host__ __device__ constexpr int fb_off(int c) {
    return (c > 0 ? fb_size(0) : 0) + (c > 1 ? fb_size(1) : 0) + (c > 2 ? fb_size(2) : 0) +
           (c > 3 ? fb_size(3) : 0) + (c > 4 ? fb_size(4) : 0);
}
constexpr int FIELDS = fb_off(5) + fb_size(5);   // floats of the field boxes of a stage
constexpr unsigned FIELD_BYTES = 4u * (fb_w(0) * fb_r(0) + fb_w(1) * fb_r(1) + fb_w(2) * fb_r(2) +
                                       fb_w(3) * fb_r(3) + fb_w(4) * fb_r(4) + fb_w(5) * fb_r(5));
constexpr int PW = TXC + 4;            // y/z psi box columns: i0-4 .. i0+127
constexpr int PR = BY + 1;             // psi box rows: jb-1 .. jb+BY-1
constexpr int PBOX = PW * PR;
constexpr int PBOXP = (PBOX + 31) / 32 * 32;
constexpr int HR = BY + 1;             // rows jb-1 .. jb+BY-1 (coefficient table)
// shared H plane (one of two): Hx and Hz of rows jb-1 .. jb+BY-2 (the rows
// below each row warp), columns i0 .. i0+127; Hz and Hy of column i0-1, rows
// jb .. jb+BY-1
constexpr int HS_X = 0, HS_Z = BY * TXC, HS_ZC = 2 * BY * TXC, HS_YC = HS_ZC + BY;
constexpr int HSB = (HS_YC + BY + 31) / 32 * 32;
constexpr int BAR_BYTES = 384;
// CPML coefficient table: aH, bH, aE, bE of the tile's columns i0-4 .. i0+127
// (CXN each; column c at c - i0 + 4, 16-byte aligned per lane), of its rows
// jb-1 .. jb+BY-1 (HR each), of the chunk's planes kstart .. k1-1 (zc each)
constexpr int CXN = PW;
constexpr int CY = 4 * CXN;
constexpr int CZ = CY + 4 * HR;
static_assert((PW * 4) % 16 == 0 && (fb_w(0) * 4) % 16 == 0 && (fb_w(1) * 4) % 16 == 0 &&
                  (fb_w(3) * 4) % 16 == 0 && (fb_cb(3) * 4) % 16 == 0,
              "box rows and origins must be multiples of 16 bytes");
// mbarriers of a block (the ring's full barriers first, which is all the
// block-barrier form uses): the stage ring (full: the stage's copies landed;
// empty: every warp that reads it is done), and for the form without block
// barriers the shared H plane (hrow: a row warp's H row is written; halo: the
// halo warp's row and column, by plane parity; edone, eall: a row warp's /
// every row warp's E phase is done, eall by plane parity)
struct Bars {
    uint64_t full[NSMAX], empty[NSMAX];
    uint64_t hrow[BY - 1], halo[2], edone[BY], eall[2];
};
static_assert(sizeof(Bars) <= BAR_BYTES, "barrier area");
static_assert(BY <= 32, "one halo lane per row");

// shared memory: barriers, H plane, coefficient table, then the stage ring
__host__ __device__ constexpr int head_floats(int zc) { return (2 * HSB + CZ + 4 * zc + 31) / 32 * 32; }

struct Maps {
    CUtensorMap f[2][6];    // fields [set][component]
    CUtensorMap x[4][2];    // psi x: xHy, xHz (H, [field set]) then xEy, xEz (E, [E psi set])
    CUtensorMap y[4][2];    // psi y: yHx, yHz, yEx, yEz
    CUtensorMap z[4][2];    // psi z: zHx, zHy, zEx, zEy
};

struct Args {
    Grid g;
    float *oex, *oey, *oez, *ohx, *ohy, *ohz;   // output set
    Cpml pml;
    int tiles_x, tiles_y;
    int za, zb, cm, m;                          // z chunks: m of cm planes over [za, zb), then [0, za), [zb, nz)
    int zc;                                     // planes of the coefficient table (longest chunk + 1)
    int ring;                                   // floats available to the stage ring
    int xlo4, xhb, xbw;                         // x psi: high half start, first column of the high
                                                // half, box width
    int cur, ecur;                              // field set read; E psi set (updated in place)
    Source src;
    SourceStep ss;
    float kE, kH;
    int *flags;
};

// stage offset of component c at box row br (row jb-1+br), box column bc
// (column i0-4+bc)
template <int C>
__device__ __forceinline__ int bo(int br, int bc) {
    constexpr int off = fb_off(C) - fb_rb(C) * fb_w(C) - fb_cb(C), w = fb_w(C);
    return off + br * w + bc;
}

// Block geometry and stage layout, fixed for the whole march.
struct Blk {
    int i0, jb, k0, k1, kstart, nplanes;
    bool src_blk;
    bool hx, hy, hz;     // the stages carry x / y / z psi boxes
    int l0;              // first y slab row of the y box
    int xo, yo, zo;      // psi region offsets inside a stage
    int stage, ns;       // floats per stage, stages in the ring
    int xlo, xhi;        // x box index of the low / high half, or -1
    int nxb, xb;         // x boxes per array, floats per x box (128-byte aligned)
};

__device__ __forceinline__ void issue_plane(const Args &A, const Maps &M, const Blk &B, float *st, uint64_t *bar,
                                            int r) {
    const int z = B.kstart + r;
    const int set = A.cur;
    const int lz = (B.hz && z < B.k1) ? slab_cell(z, A.g.nz, A.pml.P) : -1;
    unsigned bytes = FIELD_BYTES;
    if (B.hx) bytes += 4u * (unsigned)B.nxb * (unsigned)A.xbw * PR * 4u;
    if (B.hy) bytes += 4u * PBOX * 4u;
    if (lz >= 0) bytes += 4u * PBOX * 4u;
    mbar_expect_tx(bar, bytes);
#pragma unroll
    for (int c = 0; c < 6; ++c)
        tma_load(st + fb_off(c), &M.f[set][c], bar, B.i0 - 4 + fb_cb(c), B.jb - 1 + fb_rb(c), z);
    if (B.hx)
        for (int a = 0; a < 4; ++a) {
            float *d = st + B.xo + a * B.nxb * B.xb;
            if (B.xlo >= 0) tma_load(d + B.xlo * B.xb, &M.x[a][a < 2 ? set : A.ecur], bar, 0, B.jb - 1, z);
            if (B.xhi >= 0) tma_load(d + B.xhi * B.xb, &M.x[a][a < 2 ? set : A.ecur], bar, A.xlo4, B.jb - 1, z);
        }
    if (B.hy)
        for (int a = 0; a < 4; ++a) tma_load(st + B.yo + a * PBOXP, &M.y[a][a < 2 ? set : A.ecur], bar, B.i0 - 4, B.l0, z);
    if (lz >= 0)
        for (int a = 0; a < 4; ++a) tma_load(st + B.zo + a * PBOXP, &M.z[a][a < 2 ? set : A.ecur], bar, B.i0 - 4, B.jb - 1, lz);
}

// Per-lane geometry, fixed for the whole march.
struct Lane {
    int lane, w, c0, nval;
    bool roww, colin;
    int j;          // row of the lane's cells (row warps) or jb-1 (halo warp)
    bool rowin;     // 0 <= j < ny
    int ly;         // y slab index of row j, or -1 (also -1 off the grid)
    bool xl;        // some column lies in an x layer (and the row on the grid)
    int xpos;       // x psi position of column c0 (xl lanes)
    int xs;         // offset of the lane's x psi in a stage's x region (row jb-1 based)
    // halo column i0-1 (halo warp, lanes < BY): row jc
    int jc, lyc;
    int xsc;        // offset of column i0-1's x psi (row 0 based), or -1
    bool cin;
};

// One plane: H phase, barrier, E phase, barrier, refill.  Returns false when
// a wait expired (the block then stops).
// Ring position of plane rel: its stage s0, the stage s1 of plane rel+1 and
// the phase parity of that stage's barrier
struct RingPos {
    int s0, s1;
    uint32_t ph1;
};

// One plane: H phase, barrier, E phase, barrier, refill.  HX: the block
// meets an x layer; HYZ: it meets a y layer or a z layer (or its warm-up plane
// lies in one).  A block runs the instance of its case, so the plain update of
// the CPML-free interior carries no layer code at all.  Returns false when a
// wait expired (the block then stops).
// ---- the form without block barriers (k_vtile): warp-level waits and signals ----
constexpr unsigned FULLM = 0xffffffffu;
// a warp's signal: its lanes' shared stores before one arrival
__device__ __forceinline__ void wsignal(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}
// a bounded wait, taken by the whole warp; false when it expired for any lane
__device__ __forceinline__ bool wwait(uint64_t *bar, uint32_t parity) {
    return !__any_sync(FULLM, !mbar_wait(bar, parity));
}
// a warp's wait expired: record it and stop (the warps that wait for this
// one give up in turn; the refill warp lets the copies in flight land)
__device__ __forceinline__ bool wfail(const Args &A) {
    if ((threadIdx.x & 31) == 0) atomicOr(A.flags, 1);
    return false;
}

template <bool HX, bool HYZ, bool NB>
__device__ __forceinline__ bool plane(const Args &A, const Maps &M, const Lane &L, const Blk &B, uint64_t *bar,
                                      float *ring, float *HS, const float *CT, int rel, RingPos &rp,
                                      float4 &hxp, float4 &hyp) {
    const Grid &g = A.g;
    const Cpml &pm = A.pml;
    const int tid = threadIdx.x;
    const int k = B.kstart + rel;
    const bool own = k >= B.k0;
    const int s0i = rp.s0, s1i = rp.s1;

    // psi in the stage: the E phase reads the stage too
    constexpr bool STAGE_IN_E = HX || HYZ;
    bool ok = true;
    if (rel == 0) ok = mbar_wait(&bar[0], 0);
    ok = ok && mbar_wait(&bar[s1i], rp.ph1);
    Bars *vb = reinterpret_cast<Bars *>(bar);
    if (NB) {
        if (__any_sync(FULLM, !ok)) return wfail(A);
        // the halo warp rewrites this parity's halo row and column once every
        // row warp is done with them (its E phase two planes back)
        if (!L.roww && rel >= 2 && !wwait(&vb->eall[rel & 1], ((rel >> 1) - 1) & 1)) return wfail(A);
    }
    float *H = HS + (rel & 1) * HSB;          // this plane's shared H plane
    const float *s0 = ring + s0i * B.stage;   // plane k
    const float *s1 = ring + s1i * B.stage;   // plane k+1
    const int lzk = slab_cell(k, g.nz, pm.P);
    const int lz = B.hz ? lzk : -1;   // z layer plane with z boxes in the stage
    const float kH = A.kH, kE = A.kE;
    const int bc0 = 4 + 4 * L.lane;
    const unsigned goffk = (unsigned)L.c0 + (unsigned)L.j * (unsigned)g.pitch + (unsigned)k * (unsigned)g.plane;
    const bool storable = L.roww && L.rowin && L.colin;
    const bool zl = HYZ && lz >= 0 && L.rowin && L.colin;
    // psi of this lane's cells in the stage of plane k
    const float *PX = s0 + B.xo + L.xs + (L.j - B.jb + 1) * A.xbw;
    const int XA = B.nxb * B.xb;   // floats per x psi array in a stage
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float *PY = s0 + B.yo + (L.ly - B.l0) * PW + bc0;
    const float *PZ = s0 + B.zo + (L.j - B.jb + 1) * PW + bc0;

    float4 ex0, ey0, ez0, hxn, hyn, hzn;
    if (L.roww) {
        const int br = L.w + 1;  // box row of j
        ex0 = lds4(s0 + bo<0>(br, bc0));
        ey0 = lds4(s0 + bo<1>(br, bc0));
        ez0 = lds4(s0 + bo<2>(br, bc0));
        const float4 hx = lds4(s0 + bo<3>(br, bc0));
        const float4 hy = lds4(s0 + bo<4>(br, bc0));
        const float4 hz = lds4(s0 + bo<5>(br, bc0));
        const float4 exU = lds4(s0 + bo<0>(br + 1, bc0));  // row j+1
        const float4 ezU = lds4(s0 + bo<2>(br + 1, bc0));
        const float eyR = s0[bo<1>(br, bc0 + 4)];         // column c0+4
        const float ezR = s0[bo<2>(br, bc0 + 4)];
        const float4 ex1 = lds4(s1 + bo<0>(br, bc0));
        const float4 ey1 = lds4(s1 + bo<1>(br, bc0));
        float4 dyEz = ezU - ez0, dzEy = ey1 - ey0;                                    // Hx
        float4 dzEx = ex1 - ex0, dxEz = make_float4(ez0.y, ez0.z, ez0.w, ezR) - ez0;  // Hy
        float4 dxEy = make_float4(ey0.y, ey0.z, ey0.w, eyR) - ey0, dyEx = exU - ex0;  // Hz
        float4 qy0, qy1, qz0, qz1, qx0, qx1;
        if (HYZ && L.ly >= 0) {
            const float a = CT[CY + br], b = CT[CY + HR + br];
            qy0 = lds4(PY);
            qy1 = lds4(PY + PBOXP);
            dyEz = cpml4(qy0, a, b, dyEz);
            dyEx = cpml4(qy1, a, b, dyEx);
        }
        if (zl) {
            const float a = CT[CZ + rel], b = CT[CZ + A.zc + rel];
            qz0 = lds4(PZ);
            qz1 = lds4(PZ + PBOXP);
            dzEy = cpml4(qz0, a, b, dzEy);
            dzEx = cpml4(qz1, a, b, dzEx);
        } else if (HYZ && !own && lzk >= 0 && L.rowin && L.colin) {
            // warm-up plane in a z layer, the stage has no z boxes
            const unsigned o = (unsigned)psi_z(g, pm.W, L.c0, L.j, lzk);
            const float a = CT[CZ + rel], b = CT[CZ + A.zc + rel];
            qz0 = *reinterpret_cast<const float4 *>(pm.hin[2][0] + o);
            qz1 = *reinterpret_cast<const float4 *>(pm.hin[2][1] + o);
            dzEy = cpml4(qz0, a, b, dzEy);
            dzEx = cpml4(qz1, a, b, dzEx);
        }
        if (HX) {
            const float4 a = lds4(CT + bc0), b = lds4(CT + CXN + bc0);
            qx0 = L.xl ? lds4(PX) : z4;
            qx1 = L.xl ? lds4(PX + XA) : z4;
            dxEz = cpmlv(qx0, a, b, dxEz);
            dxEy = cpmlv(qx1, a, b, dxEy);
        }
        hxn = axpy(hx, -kH, dyEz - dzEy);
        hyn = axpy(hy, -kH, dzEx - dxEz);
        hzn = axpy(hz, -kH, dxEy - dyEx);
        if (own) {
            if (L.w < BY - 1) {   // the warp above reads this row
                sts4(H + HS_X + br * TXC + 4 * L.lane, hxn);
                sts4(H + HS_Z + br * TXC + 4 * L.lane, hzn);
            }
            if (storable) {
                const bool f0 = L.c0 == 0, j0 = L.j == 0, k0 = k == 0;
                st4n(A.ohx + goffk, mask(hxn, false, f0), L.nval);
                st4n(A.ohy + goffk, mask(hyn, j0, false), L.nval);
                st4n(A.ohz + goffk, mask(hzn, k0, false), L.nval);
                if (HYZ && L.ly >= 0) {
                    const unsigned o = (unsigned)psi_y(g, pm.W, L.c0, L.ly, k);
                    st4n(pm.hout[1][0] + o, mask(qy0, false, f0), L.nval);
                    st4n(pm.hout[1][1] + o, mask(qy1, k0, false), L.nval);
                }
                if (zl) {
                    const unsigned o = (unsigned)psi_z(g, pm.W, L.c0, L.j, lz);
                    st4n(pm.hout[2][0] + o, mask(qz0, false, f0), L.nval);
                    st4n(pm.hout[2][1] + o, mask(qz1, j0, false), L.nval);
                }
                if (L.xl) {
                    const unsigned o = (unsigned)psi_x(g, pm.P, L.xpos, L.j, k);
                    st4n(pm.hout[0][0] + o, mask(qx0, j0, false), L.nval);
                    st4n(pm.hout[0][1] + o, mask(qx1, k0, false), L.nval);
                }
            }
        }
    } else if (own) {
        // halo warp: H at row jb-1 (Hx, Hz) over the tile's columns
        {
            const float4 ex = lds4(s0 + bo<0>(0, bc0)), ey = lds4(s0 + bo<1>(0, bc0)), ez = lds4(s0 + bo<2>(0, bc0));
            const float4 hx = lds4(s0 + bo<3>(0, bc0)), hz = lds4(s0 + bo<5>(0, bc0));
            const float4 exU = lds4(s0 + bo<0>(1, bc0)), ezU = lds4(s0 + bo<2>(1, bc0));
            const float4 ey1 = lds4(s1 + bo<1>(0, bc0));
            const float eyR = s0[bo<1>(0, bc0 + 4)];
            float4 dyEz = ezU - ez, dzEy = ey1 - ey;
            float4 dxEy = make_float4(ey.y, ey.z, ey.w, eyR) - ey, dyEx = exU - ex;
            if (HYZ && L.ly >= 0) {
                const float a = CT[CY], b = CT[CY + HR];
                float4 q0 = lds4(PY), q1 = lds4(PY + PBOXP);
                dyEz = cpml4(q0, a, b, dyEz);
                dyEx = cpml4(q1, a, b, dyEx);
            }
            if (zl) {
                float4 q0 = lds4(PZ);
                dzEy = cpml4(q0, CT[CZ + rel], CT[CZ + A.zc + rel], dzEy);
            }
            if (HX) {
                float4 q1 = L.xl ? lds4(PX + XA) : z4;
                dxEy = cpmlv(q1, lds4(CT + bc0), lds4(CT + CXN + bc0), dxEy);
            }
            sts4(H + HS_X + 4 * L.lane, axpy(hx, -kH, dyEz - dzEy));
            sts4(H + HS_Z + 4 * L.lane, axpy(hz, -kH, dxEy - dyEx));
        }
        // column i0-1 (box column 3), rows jb .. jb+BY-1 (Hy, Hz)
        if (L.lane < BY) {
            const int b = L.lane + 1;
            const float ey = s0[bo<1>(b, 3)], eyR = s0[bo<1>(b, 4)];
            const float ex = s0[bo<0>(b, 3)], exU = s0[bo<0>(b + 1, 3)], ex1 = s1[bo<0>(b, 3)];
            const float ez = s0[bo<2>(b, 3)], ezR = s0[bo<2>(b, 4)];
            const float hy = s0[bo<4>(b, 3)], hz = s0[bo<5>(b, 3)];
            float dzEx = ex1 - ex, dxEz = ezR - ez, dxEy = eyR - ey, dyEx = exU - ex;
            if (L.cin) {
                if (HYZ && lz >= 0) {
                    float q = s0[B.zo + PBOXP + b * PW + 3];
                    dzEx = cpml1(q, CT[CZ + rel], CT[CZ + A.zc + rel], dzEx);
                }
                if (HX && L.xsc >= 0) {
                    const float *px = s0 + B.xo + L.xsc + b * A.xbw;
                    float q0 = px[0], q1 = px[XA];
                    dxEz = cpml1(q0, CT[3], CT[CXN + 3], dxEz);
                    dxEy = cpml1(q1, CT[3], CT[CXN + 3], dxEy);
                }
                if (HYZ && L.lyc >= 0) {
                    float q = s0[B.yo + PBOXP + (L.lyc - B.l0) * PW + 3];
                    dyEx = cpml1(q, CT[CY + b], CT[CY + HR + b], dyEx);
                }
            }
            H[HS_YC + b - 1] = hy - kH * (dzEx - dxEz);
            H[HS_ZC + b - 1] = hz - kH * (dxEy - dyEx);
        }
    }
    if (NB) {
        if (L.roww) {
            // before its H row is signalled, a row warp waits until the warp
            // above is done with its E phase of the last plane: the warp above
            // then cannot finish this plane's E before this warp's later waits,
            // so no barrier runs two phases ahead of a wait, and its next
            // rewrite of this parity's row comes after that E phase read it
            if (L.w < BY - 1) {
                if (rel >= 1 && !wwait(&vb->edone[L.w + 1], (rel - 1) & 1)) return wfail(A);
                wsignal(&vb->hrow[L.w]);
            }
            if (!STAGE_IN_E) wsignal(&vb->empty[s0i]);
        } else {
            wsignal(&vb->halo[rel & 1]);
            wsignal(&vb->empty[s0i]);   // the halo warp reads the stage in the H phase only
        }
    } else if (__syncthreads_or(!ok)) {
        // a wait expired: record it, let the copies in flight land, stop
        if (tid == 0) {
            atomicOr(A.flags, 1);
            // a copy that still has not landed after these waits may write the
            // block's shared memory after it ends: flag bit 8 (the handle's
            // status is sticky, it is not stepped again)
            for (int r = rel; r < B.nplanes && r < rel + B.ns; ++r) {
                bool landed = false;
                for (int t = 0; t < 4 && !landed; ++t) landed = mbar_wait(&bar[r % B.ns], (r / B.ns) & 1);
                if (!landed) atomicOr(A.flags, 8);
            }
        }
        __syncthreads();
        return false;
    }
    // the block barrier above orders every thread's reads of the stage
    // before the refill (the release/acquire a consumer barrier would give)
    if (!NB && !STAGE_IN_E && tid == 0 && rel + B.ns < B.nplanes)
        issue_plane(A, M, B, ring + s0i * B.stage, &bar[s0i], rel + B.ns);

    // ---- E phase ----
    // the H row below (the warp below's, or the halo warp's for row 0) and
    // the halo column
    if (NB && L.roww) {
        if (L.w >= 1 && !wwait(&vb->hrow[L.w - 1], rel & 1)) return wfail(A);
        if (!wwait(&vb->halo[rel & 1], (rel >> 1) & 1)) return wfail(A);
    }
    if (L.roww && own) {
        const int br = L.w + 1;
        const float4 hzD = lds4(H + HS_Z + L.w * TXC + 4 * L.lane);   // row j-1
        const float4 hxD = lds4(H + HS_X + L.w * TXC + 4 * L.lane);
        float hzL = __shfl_up_sync(0xffffffffu, hzn.w, 1);           // column c0-1
        float hyL = __shfl_up_sync(0xffffffffu, hyn.w, 1);
        if (L.lane == 0) {
            hzL = H[HS_ZC + L.w];
            hyL = H[HS_YC + L.w];
        }
        float4 dyHz = hzn - hzD, dzHy = hyn - hyp;                                       // Ex
        float4 dzHx = hxn - hxp, dxHz = hzn - make_float4(hzL, hzn.x, hzn.y, hzn.z);     // Ey
        float4 dxHy = hyn - make_float4(hyL, hyn.x, hyn.y, hyn.z), dyHx = hxn - hxD;     // Ez
        float4 qy0, qy1, qz0, qz1, qx0, qx1;
        if (HYZ && L.ly >= 0) {
            const float a = CT[CY + 2 * HR + br], b = CT[CY + 3 * HR + br];
            qy0 = lds4(PY + 2 * PBOXP);
            qy1 = lds4(PY + 3 * PBOXP);
            dyHz = cpml4(qy0, a, b, dyHz);
            dyHx = cpml4(qy1, a, b, dyHx);
        }
        if (zl) {
            const float a = CT[CZ + 2 * A.zc + rel], b = CT[CZ + 3 * A.zc + rel];
            qz0 = lds4(PZ + 2 * PBOXP);
            qz1 = lds4(PZ + 3 * PBOXP);
            dzHy = cpml4(qz0, a, b, dzHy);
            dzHx = cpml4(qz1, a, b, dzHx);
        }
        if (HX) {
            const float4 a = lds4(CT + 2 * CXN + bc0), b = lds4(CT + 3 * CXN + bc0);
            qx0 = L.xl ? lds4(PX + 2 * XA) : z4;
            qx1 = L.xl ? lds4(PX + 3 * XA) : z4;
            dxHz = cpmlv(qx0, a, b, dxHz);
            dxHy = cpmlv(qx1, a, b, dxHy);
        }
        float4 nex = axpy(ex0, kE, dyHz - dzHy);
        float4 ney = axpy(ey0, kE, dzHx - dxHz);
        float4 nez = axpy(ez0, kE, dxHy - dyHx);
        if (storable) {
            if (B.src_blk) {
                nez.x += source_at(A.src, A.ss, L.c0, L.j, k);
                nez.y += source_at(A.src, A.ss, L.c0 + 1, L.j, k);
                nez.z += source_at(A.src, A.ss, L.c0 + 2, L.j, k);
                nez.w += source_at(A.src, A.ss, L.c0 + 3, L.j, k);
            }
            const bool f0 = L.c0 == 0, j0 = L.j == 0, k0 = k == 0;
            st4n(A.oex + goffk, mask(nex, j0 || k0, false), L.nval);
            st4n(A.oey + goffk, mask(ney, k0, f0), L.nval);
            st4n(A.oez + goffk, mask(nez, j0, f0), L.nval);
            if (HYZ && L.ly >= 0) {
                const unsigned o = (unsigned)psi_y(g, pm.W, L.c0, L.ly, k);
                st4n(pm.e[1][0] + o, mask(qy0, j0 || k0, false), L.nval);
                st4n(pm.e[1][1] + o, mask(qy1, j0, f0), L.nval);
            }
            if (zl) {
                const unsigned o = (unsigned)psi_z(g, pm.W, L.c0, L.j, lz);
                st4n(pm.e[2][0] + o, mask(qz0, j0 || k0, false), L.nval);
                st4n(pm.e[2][1] + o, mask(qz1, k0, f0), L.nval);
            }
            if (L.xl) {
                const unsigned o = (unsigned)psi_x(g, pm.P, L.xpos, L.j, k);
                st4n(pm.e[0][0] + o, mask(qx0, k0, f0), L.nval);
                st4n(pm.e[0][1] + o, mask(qx1, j0, f0), L.nval);
            }
        }
    }
    if (L.roww) { hxp = hxn; hyp = hyn; }
    if (NB) {
        if (L.roww) {
            if (STAGE_IN_E) wsignal(&vb->empty[s0i]);
            wsignal(&vb->edone[L.w]);
            wsignal(&vb->eall[rel & 1]);
        }
    } else if (STAGE_IN_E) {
        __syncthreads();  // the E psi of plane k are read: its stage is free
        if (tid == 0 && rel + B.ns < B.nplanes) issue_plane(A, M, B, ring + s0i * B.stage, &bar[s0i], rel + B.ns);
    }
    rp.s0 = s1i;
    rp.s1 = s1i + 1;
    if (rp.s1 == B.ns) {
        rp.s1 = 0;
        rp.ph1 ^= 1u;
    }
    return true;
}

template <bool HX, bool HYZ, bool NB>
__device__ __forceinline__ void march(const Args &A, const Maps &M, const Lane &L, const Blk &B, uint64_t *bar,
                                      float *ring, float *HS, const float *CT) {
    float4 hxp = make_float4(0.f, 0.f, 0.f, 0.f), hyp = hxp;   // own H^{n+1/2}(k-1) Hx, Hy
    RingPos rp{0, 1, 0u};   // two stages at least
    int rel = 0;
    // a warm-up plane in a z layer (stages without z boxes) needs the layer
    // code once
    if (!HYZ && B.kstart < B.k0 && slab_cell(B.kstart, A.g.nz, A.pml.P) >= 0) {
        if (!plane<HX, true, NB>(A, M, L, B, bar, ring, HS, CT, rel, rp, hxp, hyp)) return;
        ++rel;
    }
    for (; B.kstart + rel < B.k1; ++rel)
        if (!plane<HX, HYZ, NB>(A, M, L, B, bar, ring, HS, CT, rel, rp, hxp, hyp)) return;
}

// The refill warp of the form without block barriers (one thread): planes
// 0 .. ns-1 into the empty ring, then plane r into stage r % ns once every
// warp that reads the stage is done with plane r - ns.
__device__ __forceinline__ void refill(const Args &A, const Maps &M, const Blk &B, Bars *vb, float *ring) {
    for (int r = 0; r < B.ns && r < B.nplanes; ++r) issue_plane(A, M, B, ring + r * B.stage, &vb->full[r], r);
    for (int r = B.ns; r < B.nplanes; ++r) {
        const int s = r % B.ns;
        if (!mbar_wait(&vb->empty[s], ((r - B.ns) / B.ns) & 1)) {
            // a warp stopped: let the copies in flight (planes r-ns .. r-1)
            // land before the block ends; one that does not land within these
            // waits may land after it: flag bit 8 (the handle's status is sticky)
            atomicOr(A.flags, 1);
            for (int t = r - B.ns; t < r; ++t) {
                bool landed = false;
                for (int n = 0; n < 4 && !landed; ++n) landed = mbar_wait(&vb->full[t % B.ns], (t / B.ns) & 1);
                if (!landed) atomicOr(A.flags, 8);
            }
            return;
        }
        issue_plane(A, M, B, ring + s * B.stage, &vb->full[s], r);
    }
}

// One block's tile: tile column and row `tile` (row-major over tiles_x), z
// chunk `chunk`, in the shared memory at smem_raw (barriers, H planes,
// coefficient table, then A.ring floats of stage ring).  The block may have
// run another tile before (the persistent batch kernel): every thread's
// earlier shared-memory accesses are ordered before the new TMA writes, and
// the barriers of the ring are initialised afresh (the caller invalidates
// them after each tile, see end_tile).
// LAYERS false: a grid without CPML layers (only the plain instance is
// compiled in, which keeps the register count of a caller that reads A from
// memory within a block of NW warps).
// NB true: the form without block barriers in the march, for a block of NW
// warps plus a refill warp (NT + 32 threads): each row warp waits only for
// the H rows it reads (the warp below's, the halo warp's) and signals its
// own; the halo warp waits until every row warp is done with its row and
// column of two planes back; the refill warp reloads a stage once every warp
// that reads it has signalled it empty.  The waits are parity waits and the
// order of waits and signals keeps every barrier within one phase of its
// waiters (checked on a CPU model of the warps, tests/test_tb2_sync_cpu.py).
// NB false: two block barriers per plane at most; the block's thread 0
// refills (the batch kernel, blocks of NT threads).
template <bool LAYERS = true, bool NB = false>
__device__ __forceinline__ int tile_block(const Args &A, const Maps &M, int tile, int chunk,
                                          unsigned char *smem_raw) {
    constexpr int NTB = NB ? NT + 32 : NT;   // threads of the block
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *HS = reinterpret_cast<float *>(smem_raw + BAR_BYTES);  // two shared H planes
    float *CT = HS + 2 * HSB;                                     // CPML coefficient table
    float *ring = HS + head_floats(A.zc);                         // stage ring

    const Grid &g = A.g;
    const Cpml &pm = A.pml;
    const int P = pm.P;
    const int tid = threadIdx.x;
    Blk B;
    const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
    B.i0 = tx * TXC;
    B.jb = ty * BY;
    {
        // chunk-major launch order: the m middle chunks first, so the tiles
        // of a chunk start together; the short layer chunks last, where they
        // fill the SMs of the final wave
        const int c = chunk;
        if (c < A.m) {
            B.k0 = A.za + c * A.cm;
            B.k1 = min(A.zb, B.k0 + A.cm);
        } else if (c == A.m && A.za > 0) {
            B.k0 = 0;
            B.k1 = A.za;
        } else {
            B.k0 = A.zb;
            B.k1 = g.nz;
        }
    }
    B.kstart = B.k0 > 0 ? B.k0 - 1 : 0;
    B.nplanes = B.k1 - B.kstart + 1;   // input planes kstart .. k1
    B.src_blk = A.src.active && B.i0 <= A.src.ic + A.src.L && B.i0 + TXC - 1 >= A.src.ic - A.src.L &&
                B.jb <= A.src.jc + A.src.L && B.jb + BY - 1 >= A.src.jc - A.src.L;
    // which psi boxes the stages carry
    B.hx = B.hy = B.hz = false;
    B.l0 = 0;
    B.xlo = B.xhi = -1;
    B.nxb = 0;
    B.xb = (A.xbw * PR + 31) / 32 * 32;
    if (P > 0) {
        const int ilo = max(B.i0 - 1, 0), ihi = min(B.i0 + TXC - 1, g.nx - 1);
        if (ilo <= P) B.xlo = B.nxb++;
        if (ihi >= g.nx - P) B.xhi = B.nxb++;
        B.hx = B.nxb > 0;
        int lmin = 1 << 30;
        for (int j = max(B.jb - 1, 0); j < min(B.jb + BY, g.ny); ++j) {
            const int l = slab_cell(j, g.ny, P);
            if (l >= 0 && l < lmin) lmin = l;
        }
        B.hy = lmin < (1 << 30);
        B.l0 = B.hy ? lmin : 0;
        B.hz = B.k0 < A.za || B.k0 >= A.zb;   // a layer chunk
    }
    B.xo = FIELDS;
    B.yo = B.xo + 4 * B.nxb * B.xb;
    B.zo = B.yo + (B.hy ? 4 * PBOXP : 0);
    B.stage = B.zo + (B.hz ? 4 * PBOXP : 0);
    B.ns = min(NSMAX, A.ring / B.stage);

    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    Bars *vb = reinterpret_cast<Bars *>(smem_raw);
    if (tid == 0) {
        for (int s = 0; s < B.ns; ++s) mbar_init(&bar[s], 1);
        if (NB) {
            for (int s = 0; s < B.ns; ++s) mbar_init(&vb->empty[s], NW);
            for (int w = 0; w < BY - 1; ++w) mbar_init(&vb->hrow[w], 1);
            for (int w = 0; w < BY; ++w) mbar_init(&vb->edone[w], 1);
            for (int b = 0; b < 2; ++b) {
                mbar_init(&vb->halo[b], 1);
                mbar_init(&vb->eall[b], BY);
            }
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (P > 0) {
        for (int t = tid; t < CXN; t += NTB) {
            const int i = B.i0 - 4 + t;
            const bool in = i >= 0 && i < g.nx;
            CT[t] = in ? pm.aH[0][i] : 0.f;
            CT[CXN + t] = in ? pm.bH[0][i] : 0.f;
            CT[2 * CXN + t] = in ? pm.aE[0][i] : 0.f;
            CT[3 * CXN + t] = in ? pm.bE[0][i] : 0.f;
        }
        for (int t = tid; t < HR; t += NTB) {
            const int j = B.jb - 1 + t;
            const bool in = j >= 0 && j < g.ny;
            CT[CY + t] = in ? pm.aH[1][j] : 0.f;
            CT[CY + HR + t] = in ? pm.bH[1][j] : 0.f;
            CT[CY + 2 * HR + t] = in ? pm.aE[1][j] : 0.f;
            CT[CY + 3 * HR + t] = in ? pm.bE[1][j] : 0.f;
        }
        for (int t = tid; t < A.zc; t += NTB) {
            const int k = B.kstart + t;
            const bool in = k < B.k1;
            CT[CZ + t] = in ? pm.aH[2][k] : 0.f;
            CT[CZ + A.zc + t] = in ? pm.bH[2][k] : 0.f;
            CT[CZ + 2 * A.zc + t] = in ? pm.aE[2][k] : 0.f;
            CT[CZ + 3 * A.zc + t] = in ? pm.bE[2][k] : 0.f;
        }
    }
    __syncthreads();
    if (NB) {
        if (tid >= NT) {   // the refill warp
            if (tid == NT) refill(A, M, B, vb, ring);
            return B.ns;
        }
    } else if (tid == 0) {
        for (int r = 0; r < B.ns && r < B.nplanes; ++r) issue_plane(A, M, B, ring + r * B.stage, &bar[r], r);
    }

    Lane L;
    L.lane = tid & 31;
    L.w = tid >> 5;
    L.roww = L.w < BY;
    L.c0 = B.i0 + 4 * L.lane;
    L.colin = L.c0 < g.nx;
    L.nval = L.colin ? min(4, g.nx - L.c0) : 0;
    L.j = L.roww ? B.jb + L.w : B.jb - 1;
    L.rowin = L.j >= 0 && L.j < g.ny;
    L.ly = (L.rowin && L.colin) ? slab_cell(L.j, g.ny, P) : -1;
    L.xl = false;
    L.xpos = L.xs = 0;
    if (B.hx && L.rowin && L.colin) {
        if (L.c0 <= P) {
            L.xl = true;
            L.xpos = L.c0;
            L.xs = B.xlo * B.xb + L.c0;
        } else if (L.c0 + 3 >= g.nx - P) {
            L.xl = true;
            L.xpos = A.xlo4 + L.c0 - A.xhb;
            L.xs = B.xhi * B.xb + (L.c0 - A.xhb);
        }
    }
    L.jc = B.jb + L.lane;
    L.cin = !L.roww && L.lane < BY && L.jc < g.ny && B.i0 >= 1;
    L.lyc = L.cin ? slab_cell(L.jc, g.ny, P) : -1;
    L.xsc = -1;
    if (L.cin && B.hx) {
        const int ic = B.i0 - 1;
        if (ic <= P) L.xsc = B.xlo * B.xb + ic;
        else if (ic >= g.nx - P) L.xsc = B.xhi * B.xb + (ic - A.xhb);
    }

    if (!LAYERS) {
        march<false, false, NB>(A, M, L, B, bar, ring, HS, CT);
    } else if (B.hy || B.hz) {
        if (B.hx) march<true, true, NB>(A, M, L, B, bar, ring, HS, CT);
        else march<false, true, NB>(A, M, L, B, bar, ring, HS, CT);
    } else {
        if (B.hx) march<true, false, NB>(A, M, L, B, bar, ring, HS, CT);
        else march<false, false, NB>(A, M, L, B, bar, ring, HS, CT);
    }
    return B.ns;
}

// After a tile (all threads, every wait of its march done): invalidate the
// ring's barriers so that the next tile can initialise them again.
__device__ __forceinline__ void end_tile(unsigned char *smem_raw, int ns) {
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < ns; ++s) mbar_inval(reinterpret_cast<uint64_t *>(smem_raw) + s);
    __syncthreads();
}

// ---- host ----

// Host state of a handle's tile path: its tensor maps, tiles and z chunks.
// z chunks of a grid: the layers [0, za) and [zb, nz) as chunks of their own
// (none on a grid without CPML), the planes between in m chunks of cm; zc the
// planes of the coefficient table (longest chunk + 1), ring the floats left
// for the stage ring
struct Chunks {
    int za, zb, cm, m, zc, chunks, ring;
};

// Chunks for about m middle chunks, more where the coefficient table of a
// long chunk leaves the ring (of `floats` shared floats after the barriers)
// too small for two of the largest stages.  False when one-plane chunks
// still leave too little.
inline bool z_chunks(int nz, int P, int xbw, long long m, long long floats, Chunks &c) {
    c.za = P > 0 ? P + 1 : 0;
    c.zb = P > 0 ? nz - P : nz;
    const int mid = c.zb - c.za;
    if (mid < 1) return false;
    const long long xb = (xbw * PR + 31) / 32 * 32;
    const long long big = FIELDS + 8 * xb + 8LL * PBOXP;   // largest stage: two x boxes, y and z
    if (m < 1) m = 1;
    long long ring = 0;
    for (;;) {
        c.cm = (int)((mid + m - 1) / m);
        c.zc = (c.cm > c.za ? c.cm : c.za) + 1;
        ring = floats - head_floats(c.zc);
        if (ring >= 2 * big || c.cm <= 1) break;
        ++m;
    }
    c.m = (mid + c.cm - 1) / c.cm;
    c.chunks = (c.za > 0 ? 1 : 0) + c.m + (c.zb < nz ? 1 : 0);
    c.ring = (int)ring;
    return ring >= 2 * big;
}

struct HostState {
    Maps maps;
    int tiles_x, tiles_y;
    Chunks z;
    int xlo4, xhb, xbw;
    size_t smem;
};

}  // namespace vt
}  // namespace fdtd
