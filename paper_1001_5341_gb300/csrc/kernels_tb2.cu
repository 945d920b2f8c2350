// kernels_tb2.cu -- two leapfrog steps per pass over the whole grid
// (temporal blocking of the Yee scheme, Sec. III.A; shower current of
// Sec. III.B; the CPML, this library's choice of absorbing boundary, and the
// detectors included).
//
// One launch takes E^n, H^{n-1/2} (set cur) to E^{n+2}, H^{n+3/2} (set cur^1):
// the fields are read once and written once for two steps, 24 B + 24 B per
// cell, so 24 B per cell-update instead of 48 B.
//
// Tiles.  A block owns 120 columns [i0, i0+120) (i0 = 120 tx) by TY = 8 rows
// [j0, j0+8) and marches up a chunk of z planes [k0, k1).  It computes the
// first step (level 1: H^{n+1/2}, E^{n+1}) on a larger region and the second
// (level 2: H^{n+3/2}, E^{n+2}) on its own cells:
//   lanes: lane L holds the four columns i0-4+4L .. i0-4+4L+3 as float4, so
//     the block computes columns [i0-4, i0+124); the values of a level stay
//     correct where their stencil stays inside that range, which leaves two
//     correct columns left and three right of the owned ones after level 2
//     (x neighbours by warp shuffle);
//   warps: warp w (0..10) is row j0-2+w; level-1 H on rows j0-2 .. j0+8,
//     level-1 E on j0-1 .. j0+8, level-2 H on j0-1 .. j0+7, level-2 E on the
//     owned rows (y neighbours through shared exchange rows).
// Every value of the halo is computed from the same inputs with the same
// arithmetic as by the tile that owns it, so it is that tile's value; values
// of nodes outside the grid, and the components a cell owns on the grid's low
// faces, are zero, as the one-step paths leave them.
//
// z march.  Iteration p (from k0-2 to k1) waits for input plane p+1 (TMA ring
// of stages, one mbarrier each, bounded waits), then:
//   A  level-1 H at plane p (planes p, p+1 of the stage);
//   -- barrier --
//   B  level-1 E at plane p (level-1 H of plane p-1 kept in registers);
//   C  level-2 H at plane q = p-1 (level-1 E of plane p-1 kept in registers,
//      and of plane p from B);
//   -- barrier --
//   D  level-2 E at plane q (level-2 H of plane q-1 kept in registers);
//      stores of the owned H and E of plane q.
// Exchange rows: A writes Hx, Hz of its row for B (row below); D writes the
// level-1 Ex, Ez of plane p for the next iteration's C (row above); C writes
// level-2 Hx, Hz for D (row below).
//
// CPML.  The first step of a halo cell needs the CPML memory of that cell, so
// the stages carry psi boxes (x, y, z) where the tile meets a layer.  The
// level-1 memory stays in registers for level 2; level 2 writes the H psi to
// the other H set (as the one-step path does) and the E psi to the other E
// set (the one-step paths update E psi in place, which a neighbour's halo
// would read after it changed).  z chunks are split so that only the chunks
// of the two layers carry z boxes.
//
// Detectors.  The level-1 E of the six cells of a detector's readout (Ex at
// i-1, i; Ey at j-1, j; Ez at k-1, k) go to a small buffer from the tile that
// owns them (records sorted by plane per block); the readout of step n+1 reads
// them, that of step n+2 reads the fields.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fdtd_internal.h"
#include "source_term.cuh"
#include "tma_pipe.cuh"

namespace fdtd {
namespace {

using namespace tma;

constexpr int TY = 8;                 // owned rows
constexpr int NWR = TY + 3;           // warps: rows j0-2 .. j0+TY
constexpr int NT = 32 * NWR;
constexpr int TXC = 128;              // computed columns i0-4 .. i0+123
constexpr int TXO = 120;              // owned columns (lanes 1 .. 30)
constexpr int BR = TY + 4;            // box rows j0-2 .. j0+TY+1
constexpr int BOX = TXC * BR;         // floats of a field or y/z psi box
constexpr int FIELDS = 6 * BOX;
constexpr unsigned FIELD_BYTES = 4u * FIELDS;
constexpr int XROW = 2 * TXC;         // exchange floats per warp row (two components)
constexpr int XBUF = NWR * XROW;      // one exchange buffer
constexpr int NSMAX = 8;
constexpr int BAR_BYTES = 128;
// CPML coefficient table (floats): aH, bH, aE, bE of the columns i0-4 ..
// i0+123, of the rows j0-2 .. j0+TY+1, of the planes kstart .. kstart+zt-1
constexpr int CX = 0;
constexpr int CY = 4 * TXC;
constexpr int CZ = CY + 4 * BR;
static_assert(NSMAX * 8 <= BAR_BYTES, "barrier area");
static_assert(TXO % 4 == 0 && TXC == TXO + 8, "owned columns: lanes 1 .. 30");

// shared memory: barriers, three exchange buffers, coefficient table, ring
__host__ __device__ constexpr int head_floats(int zt) { return (3 * XBUF + CZ + 4 * zt + 31) / 32 * 32; }

struct Maps {
    CUtensorMap f[2][6];    // fields [set][component]
    CUtensorMap x[4][2];    // psi x: xHy, xHz [field set], xEy, xEz [E psi set]
    CUtensorMap y[4][2];    // psi y: yHx, yHz, yEx, yEz
    CUtensorMap z[4][2];    // psi z: zHx, zHy, zEx, zEy
};

struct Args {
    Grid g;
    float *out[6];          // output field set
    Cpml pm;                // psi read (hin: H set cur, e: E set ecur) and coefficients
    float *eout[3][2];      // E psi written (set ecur^1); H psi: pm.hout
    int tiles_x, tiles_y;
    int za, zb, cm, m;      // z chunks: m of cm planes over [za, zb), then [0, za), [zb, nz)
    int zt;                 // planes of the z coefficient table
    int ring;               // floats of the stage ring
    int xlo4, xhb, xbw;     // x psi: high half start, first column of the high half, box width
    int cur, ecur;
    Source src;
    SourceStep ss1, ss2;    // current of steps n and n+1
    float kE, kH;
    int *flags;
    const int4 *prec;       // detector records {k, j, i, slot * 4 + component}
    const int *pidx;        // records of block b: [pidx[b], pidx[b+1])
    float *pbuf;            // level-1 values of the records
};

struct Blk {
    int i0, j0, k0, k1, kstart, nplanes;
    bool src_blk, hx, hy, hz;
    int l0;                 // first y slab row of the y box
    int xo, yo, zo, stage, ns;
    int xlo, xhi, nxb, xb;
    int pbeg, pend;
};

__device__ __forceinline__ void issue_plane(const Args &A, const Maps &M, const Blk &B, float *st, uint64_t *bar,
                                            int r) {
    const int p = B.kstart + r;
    const int lz = (B.hz && p >= 0 && p < A.g.nz) ? slab_cell(p, A.g.nz, A.pm.P) : -1;
    unsigned bytes = FIELD_BYTES;
    if (B.hx) bytes += 16u * (unsigned)(B.nxb * A.xbw * BR);
    if (B.hy) bytes += 16u * BOX;
    if (lz >= 0) bytes += 16u * BOX;
    mbar_expect_tx(bar, bytes);
#pragma unroll
    for (int c = 0; c < 6; ++c) tma_load(st + c * BOX, &M.f[A.cur][c], bar, B.i0 - 4, B.j0 - 2, p);
    if (B.hx)
        for (int a = 0; a < 4; ++a) {
            float *d = st + B.xo + a * B.nxb * B.xb;
            const CUtensorMap *mp = &M.x[a][a < 2 ? A.cur : A.ecur];
            if (B.xlo >= 0) tma_load(d + B.xlo * B.xb, mp, bar, 0, B.j0 - 2, p);
            if (B.xhi >= 0) tma_load(d + B.xhi * B.xb, mp, bar, A.xlo4, B.j0 - 2, p);
        }
    if (B.hy)
        for (int a = 0; a < 4; ++a) tma_load(st + B.yo + a * BOX, &M.y[a][a < 2 ? A.cur : A.ecur], bar, B.i0 - 4, B.l0, p);
    if (lz >= 0)
        for (int a = 0; a < 4; ++a) tma_load(st + B.zo + a * BOX, &M.z[a][a < 2 ? A.cur : A.ecur], bar, B.i0 - 4, B.j0 - 2, lz);
}

struct Lane {
    int lane, w, c0, j;
    bool rowin;
    bool own;          // stores level-2 values: owned lane and row, on the grid
    int nval;          // columns of the lane on the grid
    uint4 mcol;        // all bits of an element whose column lies in [0, nx)
    uint4 mcol0;       // the same without column 0
    int ly;            // y slab row of j, or -1
    bool xl;           // the lane's columns lie in an x half (row on the grid)
    int xs, xpos;      // x psi: offset in a stage's x array (box row 0), position of column c0
};

// Per-plane element masks of the six components: the state a cell keeps
// (all bits) or a zero that the one-step paths leave there (no bits): nodes
// outside the grid, and the components a cell owns on the grid's low faces.
struct Masks {
    uint4 hx, hy, hz, ex, ey, ez;
};
__device__ __forceinline__ Masks masks(const Lane &L, int k, int nz) {
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const bool in = L.rowin && k >= 0 && k < nz, fj = L.j != 0, fk = k != 0;
    Masks m;
    m.hx = in ? L.mcol0 : z;
    m.hy = in && fj ? L.mcol : z;
    m.hz = in && fk ? L.mcol : z;
    m.ex = in && fj && fk ? L.mcol : z;
    m.ey = in && fk ? L.mcol0 : z;
    m.ez = in && fj ? L.mcol0 : z;
    return m;
}
// v with the elements outside the mask set to +0 (bitwise, so a non-finite
// value outside the state never leaks in)
template <bool MASK>
__device__ __forceinline__ float4 keep(float4 v, uint4 b) {
    if (!MASK) return v;
    return make_float4(__uint_as_float(__float_as_uint(v.x) & b.x), __uint_as_float(__float_as_uint(v.y) & b.y),
                       __uint_as_float(__float_as_uint(v.z) & b.z), __uint_as_float(__float_as_uint(v.w) & b.w));
}
// the vector one column to the right (x+1) / left (x-1), edge element given
__device__ __forceinline__ float4 right(float4 v, float r) { return make_float4(v.y, v.z, v.w, r); }
__device__ __forceinline__ float4 left(float4 v, float l) { return make_float4(l, v.x, v.y, v.z); }
__device__ __forceinline__ float elem(float4 v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

constexpr unsigned FULL = 0xffffffffu;

// Register state carried from one iteration to the next.
struct State {
    float4 ex1p, ey1p, ez1p;   // level-1 E at plane p-1
    float4 hx1p, hy1p, hz1p;   // level-1 H at plane p-1
    float4 hx2p, hy2p;         // level-2 H at plane p-2
    // level-1 CPML memory at plane p-1 (H terms 0, 1; E terms 0, 1 per axis)
    float4 yH0, yH1, yE0, yE1, zH0, zH1, zE0, zE1, xH0, xH1, xE0, xE1;
};

struct RingPos {
    int s0, s1;
    uint32_t ph1;
};

template <bool HX, bool HY, bool HZ, bool MASK>
__device__ __forceinline__ bool plane(const Args &A, const Maps &M, const Lane &L, const Blk &B, uint64_t *bar,
                                      float *ring, float *X, const float *CT, int rel, RingPos &rp, State &S,
                                      int &pc) {
    const Grid &g = A.g;
    const Cpml &pm = A.pm;
    const int tid = threadIdx.x, w = L.w;
    const int p = B.kstart + rel, q = p - 1;
    const float kH = A.kH, kE = A.kE;
    constexpr bool STAGE_IN_B = HX || HY || HZ;   // B reads E psi from the stage
    bool ok = true;
    if (rel == 0) ok = mbar_wait(&bar[0], 0);
    ok = ok && mbar_wait(&bar[rp.s1], rp.ph1);
    const float *s0 = ring + rp.s0 * B.stage;   // plane p
    const float *s1 = ring + rp.s1 * B.stage;   // plane p+1
    float *XA = X, *XB = X + XBUF, *XC = X + 2 * XBUF;
    const int bc0 = 4 * L.lane;
    const int lzp = (HZ && p >= 0 && p < g.nz) ? slab_cell(p, g.nz, pm.P) : -1;
    const int lzq = (HZ && q >= 0 && q < g.nz) ? slab_cell(q, g.nz, pm.P) : -1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool yl = HY && L.ly >= 0;
    const float *PY = s0 + B.yo + (L.ly - B.l0) * TXC + bc0;
    const float *PZ = s0 + B.zo + w * TXC + bc0;
    const float *PX = s0 + B.xo + L.xs + w * A.xbw;
    const int XA4 = B.nxb * B.xb;   // floats per x psi array in a stage
    Masks mp, mq;
    if (MASK) mp = masks(L, p, g.nz);

    // ---- A: level-1 H at plane p (rows j0-2 .. j0+TY) ----
    const float4 ex0 = lds4(s0 + 0 * BOX + w * TXC + bc0);
    const float4 ey0 = lds4(s0 + 1 * BOX + w * TXC + bc0);
    const float4 ez0 = lds4(s0 + 2 * BOX + w * TXC + bc0);
    float4 hx1, hy1, hz1;
    float4 yH0 = z4, yH1 = z4, zH0 = z4, zH1 = z4, xH0 = z4, xH1 = z4;
    {
        const float4 hx = lds4(s0 + 3 * BOX + w * TXC + bc0);
        const float4 hy = lds4(s0 + 4 * BOX + w * TXC + bc0);
        const float4 hz = lds4(s0 + 5 * BOX + w * TXC + bc0);
        const float4 exU = lds4(s0 + 0 * BOX + (w + 1) * TXC + bc0);   // row j+1
        const float4 ezU = lds4(s0 + 2 * BOX + (w + 1) * TXC + bc0);
        const float4 exN = lds4(s1 + 0 * BOX + w * TXC + bc0);         // plane p+1
        const float4 eyN = lds4(s1 + 1 * BOX + w * TXC + bc0);
        const float eyR = __shfl_down_sync(FULL, ey0.x, 1);             // column +4 (lane 31: unused)
        const float ezR = __shfl_down_sync(FULL, ez0.x, 1);
        float4 dyEz = ezU - ez0, dzEy = eyN - ey0;                      // Hx
        float4 dzEx = exN - ex0, dxEz = right(ez0, ezR) - ez0;          // Hy
        float4 dxEy = right(ey0, eyR) - ey0, dyEx = exU - ex0;          // Hz
        if (yl) {
            const float a = CT[CY + w], b = CT[CY + BR + w];
            yH0 = lds4(PY);
            yH1 = lds4(PY + BOX);
            dyEz = cpml4(yH0, a, b, dyEz);
            dyEx = cpml4(yH1, a, b, dyEx);
        }
        if (HZ && lzp >= 0) {
            const float a = CT[CZ + rel], b = CT[CZ + A.zt + rel];
            zH0 = lds4(PZ);
            zH1 = lds4(PZ + BOX);
            dzEy = cpml4(zH0, a, b, dzEy);
            dzEx = cpml4(zH1, a, b, dzEx);
        }
        if (HX) {
            const float4 a = lds4(CT + CX + bc0), b = lds4(CT + CX + TXC + bc0);
            xH0 = L.xl ? lds4(PX) : z4;
            xH1 = L.xl ? lds4(PX + XA4) : z4;
            dxEz = cpmlv(xH0, a, b, dxEz);
            dxEy = cpmlv(xH1, a, b, dxEy);
        }
        hx1 = keep<MASK>(axpy(hx, -kH, dyEz - dzEy), mp.hx);
        hy1 = keep<MASK>(axpy(hy, -kH, dzEx - dxEz), mp.hy);
        hz1 = keep<MASK>(axpy(hz, -kH, dxEy - dyEx), mp.hz);
        yH0 = keep<MASK>(yH0, mp.hx); yH1 = keep<MASK>(yH1, mp.hz);
        zH0 = keep<MASK>(zH0, mp.hx); zH1 = keep<MASK>(zH1, mp.hy);
        xH0 = keep<MASK>(xH0, mp.hy); xH1 = keep<MASK>(xH1, mp.hz);
        sts4(XA + w * XROW + bc0, hx1);
        sts4(XA + w * XROW + TXC + bc0, hz1);
    }
    if (__syncthreads_or(!ok)) {
        // a wait expired: record it, let the copies in flight land, stop
        if (tid == 0) {
            atomicOr(A.flags, 1);
            for (int r = rel; r < B.nplanes && r < rel + B.ns; ++r)
                if (!mbar_wait(&bar[r % B.ns], (r / B.ns) & 1)) atomicOr(A.flags, 8);
        }
        __syncthreads();
        return false;
    }
    // the barrier orders every thread's reads of stage p before its refill
    if (!STAGE_IN_B && tid == 0 && rel + B.ns < B.nplanes)
        issue_plane(A, M, B, ring + rp.s0 * B.stage, &bar[rp.s0], rel + B.ns);

    // ---- B: level-1 E at plane p (rows j0-1 .. j0+TY) ----
    float4 ex1 = z4, ey1 = z4, ez1 = z4;
    float4 yE0 = z4, yE1 = z4, zE0 = z4, zE1 = z4, xE0 = z4, xE1 = z4;
    if (w >= 1) {
        const float4 hzD = lds4(XA + (w - 1) * XROW + TXC + bc0);   // row j-1
        const float4 hxD = lds4(XA + (w - 1) * XROW + bc0);
        const float hzL = __shfl_up_sync(FULL, hz1.w, 1);           // column -1 (lane 0: unused)
        const float hyL = __shfl_up_sync(FULL, hy1.w, 1);
        float4 dyHz = hz1 - hzD, dzHy = hy1 - S.hy1p;                  // Ex
        float4 dzHx = hx1 - S.hx1p, dxHz = hz1 - left(hz1, hzL);       // Ey
        float4 dxHy = hy1 - left(hy1, hyL), dyHx = hx1 - hxD;          // Ez
        if (yl) {
            const float a = CT[CY + 2 * BR + w], b = CT[CY + 3 * BR + w];
            yE0 = lds4(PY + 2 * BOX);
            yE1 = lds4(PY + 3 * BOX);
            dyHz = cpml4(yE0, a, b, dyHz);
            dyHx = cpml4(yE1, a, b, dyHx);
        }
        if (HZ && lzp >= 0) {
            const float a = CT[CZ + 2 * A.zt + rel], b = CT[CZ + 3 * A.zt + rel];
            zE0 = lds4(PZ + 2 * BOX);
            zE1 = lds4(PZ + 3 * BOX);
            dzHy = cpml4(zE0, a, b, dzHy);
            dzHx = cpml4(zE1, a, b, dzHx);
        }
        if (HX) {
            const float4 a = lds4(CT + CX + 2 * TXC + bc0), b = lds4(CT + CX + 3 * TXC + bc0);
            xE0 = L.xl ? lds4(PX + 2 * XA4) : z4;
            xE1 = L.xl ? lds4(PX + 3 * XA4) : z4;
            dxHz = cpmlv(xE0, a, b, dxHz);
            dxHy = cpmlv(xE1, a, b, dxHy);
        }
        ex1 = axpy(ex0, kE, dyHz - dzHy);
        ey1 = axpy(ey0, kE, dzHx - dxHz);
        ez1 = axpy(ez0, kE, dxHy - dyHx);
        if (B.src_blk) {
            ez1.x += source_at(A.src, A.ss1, L.c0, L.j, p);
            ez1.y += source_at(A.src, A.ss1, L.c0 + 1, L.j, p);
            ez1.z += source_at(A.src, A.ss1, L.c0 + 2, L.j, p);
            ez1.w += source_at(A.src, A.ss1, L.c0 + 3, L.j, p);
        }
        ex1 = keep<MASK>(ex1, mp.ex);
        ey1 = keep<MASK>(ey1, mp.ey);
        ez1 = keep<MASK>(ez1, mp.ez);
        yE0 = keep<MASK>(yE0, mp.ex); yE1 = keep<MASK>(yE1, mp.ez);
        zE0 = keep<MASK>(zE0, mp.ex); zE1 = keep<MASK>(zE1, mp.ey);
        xE0 = keep<MASK>(xE0, mp.ey); xE1 = keep<MASK>(xE1, mp.ez);
    }
    // detector records of plane p (block-uniform walk of the block's list)
    while (pc < B.pend) {
        const int4 r = A.prec[pc];
        if (r.x != p) break;
        if (w >= 1 && r.y == L.j && r.z >= L.c0 && r.z < L.c0 + 4) {
            const int c = r.w & 3;
            A.pbuf[r.w >> 2] = elem(c == 0 ? ex1 : c == 1 ? ey1 : ez1, r.z - L.c0);
        }
        ++pc;
    }

    // ---- C: level-2 H at plane q = p-1 (rows j0-1 .. j0+TY-1) ----
    float4 hx2 = z4, hy2 = z4, hz2 = z4;
    if (MASK) mq = masks(L, q, g.nz);
    if (p >= B.k0 && w >= 1 && w <= TY + 1) {
        const float4 exU = lds4(XB + (w + 1) * XROW + bc0);         // level-1 E of plane q, row j+1
        const float4 ezU = lds4(XB + (w + 1) * XROW + TXC + bc0);
        const float eyR = __shfl_down_sync(FULL, S.ey1p.x, 1);
        const float ezR = __shfl_down_sync(FULL, S.ez1p.x, 1);
        float4 dyEz = ezU - S.ez1p, dzEy = ey1 - S.ey1p;
        float4 dzEx = ex1 - S.ex1p, dxEz = right(S.ez1p, ezR) - S.ez1p;
        float4 dxEy = right(S.ey1p, eyR) - S.ey1p, dyEx = exU - S.ex1p;
        if (yl) {
            const float a = CT[CY + w], b = CT[CY + BR + w];
            dyEz = cpml4(S.yH0, a, b, dyEz);
            dyEx = cpml4(S.yH1, a, b, dyEx);
        }
        if (HZ && lzq >= 0) {
            const float a = CT[CZ + rel - 1], b = CT[CZ + A.zt + rel - 1];
            dzEy = cpml4(S.zH0, a, b, dzEy);
            dzEx = cpml4(S.zH1, a, b, dzEx);
        }
        if (HX) {
            const float4 a = lds4(CT + CX + bc0), b = lds4(CT + CX + TXC + bc0);
            dxEz = cpmlv(S.xH0, a, b, dxEz);
            dxEy = cpmlv(S.xH1, a, b, dxEy);
        }
        hx2 = keep<MASK>(axpy(S.hx1p, -kH, dyEz - dzEy), mq.hx);
        hy2 = keep<MASK>(axpy(S.hy1p, -kH, dzEx - dxEz), mq.hy);
        hz2 = keep<MASK>(axpy(S.hz1p, -kH, dxEy - dyEx), mq.hz);
        sts4(XC + w * XROW + bc0, hx2);
        sts4(XC + w * XROW + TXC + bc0, hz2);
        if (L.own && q >= B.k0 && q < B.k1) {
            const unsigned o = (unsigned)L.c0 + (unsigned)L.j * (unsigned)g.pitch + (unsigned)q * (unsigned)g.plane;
            st4n(A.out[3] + o, hx2, L.nval);
            st4n(A.out[4] + o, hy2, L.nval);
            st4n(A.out[5] + o, hz2, L.nval);
            if (yl) {
                const unsigned oy = (unsigned)psi_y(g, pm.W, L.c0, L.ly, q);
                st4n(pm.hout[1][0] + oy, keep<MASK>(S.yH0, mq.hx), L.nval);
                st4n(pm.hout[1][1] + oy, keep<MASK>(S.yH1, mq.hz), L.nval);
            }
            if (HZ && lzq >= 0) {
                const unsigned oz = (unsigned)psi_z(g, pm.W, L.c0, L.j, lzq);
                st4n(pm.hout[2][0] + oz, keep<MASK>(S.zH0, mq.hx), L.nval);
                st4n(pm.hout[2][1] + oz, keep<MASK>(S.zH1, mq.hy), L.nval);
            }
            if (HX && L.xl) {
                const unsigned ox = (unsigned)psi_x(g, pm.P, L.xpos, L.j, q);
                st4n(pm.hout[0][0] + ox, keep<MASK>(S.xH0, mq.hy), L.nval);
                st4n(pm.hout[0][1] + ox, keep<MASK>(S.xH1, mq.hz), L.nval);
            }
        }
    }
    __syncthreads();
    if (STAGE_IN_B && tid == 0 && rel + B.ns < B.nplanes)
        issue_plane(A, M, B, ring + rp.s0 * B.stage, &bar[rp.s0], rel + B.ns);

    // ---- D: level-1 E rows for the next C; level-2 E at plane q (owned rows) ----
    if (w >= 1) {
        sts4(XB + w * XROW + bc0, ex1);
        sts4(XB + w * XROW + TXC + bc0, ez1);
    }
    if (p >= B.k0 + 1 && w >= 2 && w <= TY + 1) {
        const float4 hzD = lds4(XC + (w - 1) * XROW + TXC + bc0);
        const float4 hxD = lds4(XC + (w - 1) * XROW + bc0);
        const float hzL = __shfl_up_sync(FULL, hz2.w, 1);
        const float hyL = __shfl_up_sync(FULL, hy2.w, 1);
        float4 dyHz = hz2 - hzD, dzHy = hy2 - S.hy2p;
        float4 dzHx = hx2 - S.hx2p, dxHz = hz2 - left(hz2, hzL);
        float4 dxHy = hy2 - left(hy2, hyL), dyHx = hx2 - hxD;
        if (yl) {
            const float a = CT[CY + 2 * BR + w], b = CT[CY + 3 * BR + w];
            dyHz = cpml4(S.yE0, a, b, dyHz);
            dyHx = cpml4(S.yE1, a, b, dyHx);
        }
        if (HZ && lzq >= 0) {
            const float a = CT[CZ + 2 * A.zt + rel - 1], b = CT[CZ + 3 * A.zt + rel - 1];
            dzHy = cpml4(S.zE0, a, b, dzHy);
            dzHx = cpml4(S.zE1, a, b, dzHx);
        }
        if (HX) {
            const float4 a = lds4(CT + CX + 2 * TXC + bc0), b = lds4(CT + CX + 3 * TXC + bc0);
            dxHz = cpmlv(S.xE0, a, b, dxHz);
            dxHy = cpmlv(S.xE1, a, b, dxHy);
        }
        float4 ex2 = axpy(S.ex1p, kE, dyHz - dzHy);
        float4 ey2 = axpy(S.ey1p, kE, dzHx - dxHz);
        float4 ez2 = axpy(S.ez1p, kE, dxHy - dyHx);
        if (L.own && q < B.k1) {
            if (B.src_blk) {
                ez2.x += source_at(A.src, A.ss2, L.c0, L.j, q);
                ez2.y += source_at(A.src, A.ss2, L.c0 + 1, L.j, q);
                ez2.z += source_at(A.src, A.ss2, L.c0 + 2, L.j, q);
                ez2.w += source_at(A.src, A.ss2, L.c0 + 3, L.j, q);
            }
            const unsigned o = (unsigned)L.c0 + (unsigned)L.j * (unsigned)g.pitch + (unsigned)q * (unsigned)g.plane;
            st4n(A.out[0] + o, keep<MASK>(ex2, mq.ex), L.nval);
            st4n(A.out[1] + o, keep<MASK>(ey2, mq.ey), L.nval);
            st4n(A.out[2] + o, keep<MASK>(ez2, mq.ez), L.nval);
            if (yl) {
                const unsigned oy = (unsigned)psi_y(g, pm.W, L.c0, L.ly, q);
                st4n(A.eout[1][0] + oy, keep<MASK>(S.yE0, mq.ex), L.nval);
                st4n(A.eout[1][1] + oy, keep<MASK>(S.yE1, mq.ez), L.nval);
            }
            if (HZ && lzq >= 0) {
                const unsigned oz = (unsigned)psi_z(g, pm.W, L.c0, L.j, lzq);
                st4n(A.eout[2][0] + oz, keep<MASK>(S.zE0, mq.ex), L.nval);
                st4n(A.eout[2][1] + oz, keep<MASK>(S.zE1, mq.ey), L.nval);
            }
            if (HX && L.xl) {
                const unsigned ox = (unsigned)psi_x(g, pm.P, L.xpos, L.j, q);
                st4n(A.eout[0][0] + ox, keep<MASK>(S.xE0, mq.ey), L.nval);
                st4n(A.eout[0][1] + ox, keep<MASK>(S.xE1, mq.ez), L.nval);
            }
        }
    }
    // carry to the next plane
    S.ex1p = ex1; S.ey1p = ey1; S.ez1p = ez1;
    S.hx1p = hx1; S.hy1p = hy1; S.hz1p = hz1;
    S.hx2p = hx2; S.hy2p = hy2;
    S.yH0 = yH0; S.yH1 = yH1; S.yE0 = yE0; S.yE1 = yE1;
    S.zH0 = zH0; S.zH1 = zH1; S.zE0 = zE0; S.zE1 = zE1;
    S.xH0 = xH0; S.xH1 = xH1; S.xE0 = xE0; S.xE1 = xE1;
    rp.s0 = rp.s1;
    rp.s1 = rp.s1 + 1;
    if (rp.s1 == B.ns) {
        rp.s1 = 0;
        rp.ph1 ^= 1u;
    }
    return true;
}

template <bool HX, bool HY, bool HZ, bool MASK>
__device__ __forceinline__ void march(const Args &A, const Maps &M, const Lane &L, const Blk &B, uint64_t *bar,
                                      float *ring, float *X, const float *CT) {
    State S;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    S.ex1p = S.ey1p = S.ez1p = S.hx1p = S.hy1p = S.hz1p = S.hx2p = S.hy2p = z4;
    S.yH0 = S.yH1 = S.yE0 = S.yE1 = S.zH0 = S.zH1 = S.zE0 = S.zE1 = S.xH0 = S.xH1 = S.xE0 = S.xE1 = z4;
    RingPos rp{0, 1, 0u};   // two stages at least
    int pc = B.pbeg;
    for (int rel = 0; rel + 1 < B.nplanes; ++rel)
        if (!plane<HX, HY, HZ, MASK>(A, M, L, B, bar, ring, X, CT, rel, rp, S, pc)) return;
}

// the instance of a block's case: which psi boxes it carries, whether it
// meets a face of the grid
template <bool HX, bool HY, bool HZ>
__device__ __forceinline__ void march_edge(bool edge, const Args &A, const Maps &M, const Lane &L, const Blk &B,
                                           uint64_t *bar, float *ring, float *X, const float *CT) {
    if (edge) march<HX, HY, HZ, true>(A, M, L, B, bar, ring, X, CT);
    else march<HX, HY, HZ, false>(A, M, L, B, bar, ring, X, CT);
}
template <bool HX, bool HY>
__device__ __forceinline__ void march_z(bool hz, bool edge, const Args &A, const Maps &M, const Lane &L,
                                        const Blk &B, uint64_t *bar, float *ring, float *X, const float *CT) {
    if (hz) march_edge<HX, HY, true>(edge, A, M, L, B, bar, ring, X, CT);
    else march_edge<HX, HY, false>(edge, A, M, L, B, bar, ring, X, CT);
}

__global__ void __launch_bounds__(NT, 1) k_tb2(const Args A, const __grid_constant__ Maps M) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *X = reinterpret_cast<float *>(smem_raw + BAR_BYTES);   // exchange rows
    float *CT = X + 3 * XBUF;                                      // CPML coefficients
    float *ring = X + head_floats(A.zt);                           // stage ring

    const Grid &g = A.g;
    const Cpml &pm = A.pm;
    const int P = pm.P;
    const int tid = threadIdx.x;
    Blk B;
    const int tile = (int)blockIdx.x;
    const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
    B.i0 = tx * TXO;
    B.j0 = ty * TY;
    {
        // chunk-major launch order: the middle chunks first, the two layer
        // chunks last
        const int c = (int)blockIdx.y;
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
        B.hz = P > 0 && c >= A.m;
        const int b = c * A.tiles_x * A.tiles_y + tile;
        B.pbeg = A.pidx ? A.pidx[b] : 0;
        B.pend = A.pidx ? A.pidx[b + 1] : 0;
    }
    B.kstart = B.k0 - 2;
    B.nplanes = B.k1 - B.k0 + 4;   // input planes k0-2 .. k1+1
    B.src_blk = A.src.active && B.i0 - 4 <= A.src.ic + A.src.L && B.i0 + TXC - 5 >= A.src.ic - A.src.L &&
                B.j0 - 2 <= A.src.jc + A.src.L && B.j0 + TY + 1 >= A.src.jc - A.src.L;
    B.hx = B.hy = false;
    B.l0 = 0;
    B.xlo = B.xhi = -1;
    B.nxb = 0;
    B.xb = (A.xbw * BR + 31) / 32 * 32;
    if (P > 0) {
        const int ilo = max(B.i0 - 4, 0), ihi = min(B.i0 + TXC - 5, g.nx - 1);
        if (ilo <= P) B.xlo = B.nxb++;
        if (ihi >= g.nx - P) B.xhi = B.nxb++;
        B.hx = B.nxb > 0;
        int lmin = 1 << 30;
        for (int j = max(B.j0 - 2, 0); j < min(B.j0 + TY + 2, g.ny); ++j) {
            const int l = slab_cell(j, g.ny, P);
            if (l >= 0 && l < lmin) lmin = l;
        }
        B.hy = lmin < (1 << 30);
        B.l0 = B.hy ? lmin : 0;
    }
    B.xo = FIELDS;
    B.yo = B.xo + 4 * B.nxb * B.xb;
    B.zo = B.yo + (B.hy ? 4 * BOX : 0);
    B.stage = B.zo + (B.hz ? 4 * BOX : 0);
    B.ns = min(NSMAX, A.ring / B.stage);

    if (tid == 0) {
        for (int s = 0; s < B.ns; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (P > 0) {
        for (int t = tid; t < TXC; t += NT) {
            const int i = B.i0 - 4 + t;
            const bool in = i >= 0 && i < g.nx;
            CT[CX + t] = in ? pm.aH[0][i] : 0.f;
            CT[CX + TXC + t] = in ? pm.bH[0][i] : 0.f;
            CT[CX + 2 * TXC + t] = in ? pm.aE[0][i] : 0.f;
            CT[CX + 3 * TXC + t] = in ? pm.bE[0][i] : 0.f;
        }
        for (int t = tid; t < BR; t += NT) {
            const int j = B.j0 - 2 + t;
            const bool in = j >= 0 && j < g.ny;
            CT[CY + t] = in ? pm.aH[1][j] : 0.f;
            CT[CY + BR + t] = in ? pm.bH[1][j] : 0.f;
            CT[CY + 2 * BR + t] = in ? pm.aE[1][j] : 0.f;
            CT[CY + 3 * BR + t] = in ? pm.bE[1][j] : 0.f;
        }
        if (B.hz)
            for (int t = tid; t < A.zt; t += NT) {
                const int k = B.kstart + t;
                const bool in = k >= 0 && k < g.nz;
                CT[CZ + t] = in ? pm.aH[2][k] : 0.f;
                CT[CZ + A.zt + t] = in ? pm.bH[2][k] : 0.f;
                CT[CZ + 2 * A.zt + t] = in ? pm.aE[2][k] : 0.f;
                CT[CZ + 3 * A.zt + t] = in ? pm.bE[2][k] : 0.f;
            }
    }
    __syncthreads();
    if (tid == 0)
        for (int r = 0; r < B.ns && r < B.nplanes; ++r) issue_plane(A, M, B, ring + r * B.stage, &bar[r], r);

    Lane L;
    L.lane = tid & 31;
    L.w = tid >> 5;
    L.c0 = B.i0 - 4 + 4 * L.lane;
    L.j = B.j0 - 2 + L.w;
    L.rowin = L.j >= 0 && L.j < g.ny;
    {
        unsigned m[4];
        for (int e = 0; e < 4; ++e) m[e] = (L.c0 + e >= 0 && L.c0 + e < g.nx) ? 0xffffffffu : 0u;
        L.mcol = make_uint4(m[0], m[1], m[2], m[3]);
        L.mcol0 = make_uint4(L.c0 == 0 ? 0u : m[0], m[1], m[2], m[3]);
    }
    L.nval = L.c0 >= 0 && L.c0 < g.nx ? min(4, g.nx - L.c0) : 0;
    L.own = L.lane >= 1 && L.lane <= 30 && L.w >= 2 && L.w <= TY + 1 && L.rowin && L.nval > 0;
    L.ly = (P > 0 && L.rowin) ? slab_cell(L.j, g.ny, P) : -1;
    L.xl = false;
    L.xs = L.xpos = 0;
    if (B.hx && L.rowin && L.nval > 0) {
        if (B.xlo >= 0 && L.c0 < A.xlo4) {
            L.xl = true;
            L.xpos = L.c0;
            L.xs = B.xlo * B.xb + L.c0;
        } else if (B.xhi >= 0 && L.c0 >= A.xhb) {
            L.xl = true;
            L.xpos = A.xlo4 + L.c0 - A.xhb;
            L.xs = B.xhi * B.xb + (L.c0 - A.xhb);
        }
    }

    // blocks whose computed region stays clear of the faces need no masks
    const bool edge = B.i0 - 4 < 1 || B.i0 + TXC - 5 > g.nx - 1 || B.j0 - 2 < 1 || B.j0 + TY > g.ny - 1 ||
                      B.k0 - 2 < 1 || B.k1 > g.nz - 1;
    if (B.hx) {
        if (B.hy) march_z<true, true>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
        else march_z<true, false>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
    } else {
        if (B.hy) march_z<false, true>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
        else march_z<false, false>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
    }
}

constexpr CUtensorMapL2promotion kPromotion = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;

struct HostState {
    Maps maps;
    int tiles_x, tiles_y, za, zb, cm, m, zt, chunks, ring;
    int xlo4, xhb, xbw;
    size_t smem;
    // detector records, rebuilt when the handle's detectors change
    int probe_ver;
    std::vector<int4> h_rec;
    std::vector<int> h_idx;
    int4 *d_rec;
    int *d_idx;
    float *d_pbuf;
};

// chunk of plane k (the kernel's chunk decoding, inverted)
int chunk_of(const HostState *st, int k) {
    if (k < st->za) return st->m;
    if (k >= st->zb) return st->m + (st->za > 0 ? 1 : 0);
    return (k - st->za) / st->cm;
}

int build_records(fdtd_ctx *h, HostState *st) {
    cudaFree(st->d_rec);
    cudaFree(st->d_idx);
    cudaFree(st->d_pbuf);
    st->d_rec = nullptr;
    st->d_idx = nullptr;
    st->d_pbuf = nullptr;
    st->probe_ver = h->probe_ver;
    if (h->np == 0) return FDTD_OK;
    const int tiles = st->tiles_x * st->tiles_y;
    const int blocks = tiles * st->chunks;
    // the six cells of each detector's readout: Ex at i-1, i; Ey at j-1, j; Ez at k-1, k
    struct Rec { int b; int4 r; };
    std::vector<Rec> recs;
    recs.reserve(6 * (size_t)h->np);
    for (int t = 0; t < h->np; ++t) {
        const int i = h->h_ijk[3 * t], j = h->h_ijk[3 * t + 1], k = h->h_ijk[3 * t + 2];
        const int cell[6][4] = {{i - 1, j, k, 0}, {i, j, k, 0}, {i, j - 1, k, 1},
                                {i, j, k, 1},     {i, j, k - 1, 2}, {i, j, k, 2}};
        for (int s = 0; s < 6; ++s) {
            const int ci = cell[s][0], cj = cell[s][1], ck = cell[s][2];
            const int b = chunk_of(st, ck) * tiles + (cj / TY) * st->tiles_x + ci / TXO;
            recs.push_back({b, make_int4(ck, cj, ci, (6 * t + s) * 4 + cell[s][3])});
        }
    }
    std::stable_sort(recs.begin(), recs.end(),
                     [](const Rec &a, const Rec &b) { return a.b < b.b || (a.b == b.b && a.r.x < b.r.x); });
    st->h_rec.resize(recs.size());
    st->h_idx.assign(blocks + 1, 0);
    for (size_t n = 0; n < recs.size(); ++n) {
        st->h_rec[n] = recs[n].r;
        st->h_idx[recs[n].b + 1]++;
    }
    for (int b = 0; b < blocks; ++b) st->h_idx[b + 1] += st->h_idx[b];
    if (cudaMalloc(&st->d_rec, sizeof(int4) * recs.size()) != cudaSuccess ||
        cudaMalloc(&st->d_idx, sizeof(int) * (blocks + 1)) != cudaSuccess ||
        cudaMalloc(&st->d_pbuf, sizeof(float) * 6 * (size_t)h->np) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    if (cudaMemcpy(st->d_rec, st->h_rec.data(), sizeof(int4) * recs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(st->d_idx, st->h_idx.data(), sizeof(int) * (blocks + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    return FDTD_OK;
}

}  // namespace

const char *tb2_name() { return "tblock2-120x8"; }

int tb2_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    const int P = h->P;
    if (h->boundary == FDTD_MUR1) return FDTD_ERR_ARG;   // the Mur faces need E^{n+1} between the steps
    if ((unsigned long long)g.comp >= (1ull << 32) || g.pitch % 4 != 0) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    const int xlo4 = P > 0 ? psi_x_lo4(P) : 0, xhb = P > 0 ? psi_x_hb(g.nx, P) : 0;
    const int WX = P > 0 ? psi_x_row(g.nx, P) : 0;
    const int xbw = P > 0 ? (xlo4 > WX - xlo4 ? xlo4 : WX - xlo4) : 4;
    if (P > 0 && (g.nx < 2 * P + 8 || xbw > 256 || !h->epsi2)) return FDTD_ERR_ARG;
    EncodeTiled encode = encoder();
    if (!encode) return FDTD_ERR_CUDA;
    HostState *st = new (std::nothrow) HostState();
    if (!st) return FDTD_ERR_OOM;
    st->xlo4 = xlo4;
    st->xhb = xhb;
    st->xbw = xbw;
    bool ok = true;
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 6; ++c)
            ok = ok && encode3(encode, &st->maps.f[s][c], h->fields[s] + (size_t)c * g.comp, g.nx + 1, g.ny + 1,
                               g.nz + 1, g.pitch, g.plane, TXC, BR, kPromotion);
    if (P > 0) {
        // H psi sets follow the field set; E psi sets are psi_block's first
        // third and epsi2
        const size_t set = 2 * (h->psi_axis[0] + h->psi_axis[1] + h->psi_axis[2]);
        const int W = 2 * P + 1;
        for (int s = 0; s < 2; ++s) {
            size_t off = 0;
            for (int axis = 0; axis < 3; ++axis)
                for (int t = 0; t < 2; ++t) {
                    const float *hp = h->psi_block + set * (1 + s) + off;
                    const float *ep = (s == 0 ? h->psi_block : h->epsi2) + off;
                    off += h->psi_axis[axis];
                    for (int half = 0; half < 2; ++half) {
                        const float *base = half == 0 ? hp : ep;
                        const int a = 2 * half + t;
                        CUtensorMap *m = axis == 0 ? &st->maps.x[a][s] : axis == 1 ? &st->maps.y[a][s] : &st->maps.z[a][s];
                        if (axis == 0)
                            ok = ok && encode3(encode, m, base, WX, g.ny, g.nz, WX, (cuuint64_t)g.ny * WX, xbw, BR, kPromotion);
                        else if (axis == 1)
                            ok = ok && encode3(encode, m, base, g.nx, W, g.nz, g.pitch, (cuuint64_t)W * g.pitch, TXC, BR, kPromotion);
                        else
                            ok = ok && encode3(encode, m, base, g.nx, g.ny, W, g.pitch, (cuuint64_t)g.ny * g.pitch, TXC, BR, kPromotion);
                    }
                }
        }
    }
    if (!ok) {
        delete st;
        return FDTD_ERR_CUDA;
    }
    st->tiles_x = (g.nx + TXO - 1) / TXO;
    st->tiles_y = (g.ny + TY - 1) / TY;
    // z chunks: the planes of a middle chunk (k0-2 .. k1+1) stay clear of the
    // z layers, so only the two layer chunks [0, za), [zb, nz) carry z boxes;
    // a grid too short for a middle part is one layer chunk
    if (P > 0) {
        st->za = P + 3;
        st->zb = g.nz - P - 2;
        if (st->zb - st->za < 8) st->za = st->zb = g.nz;
    } else {
        st->za = 0;
        st->zb = g.nz;
    }
    const int mid = st->zb - st->za;
    const long long sms = h->num_sms > 0 ? h->num_sms : 1;
    const long long tiles = (long long)st->tiles_x * st->tiles_y;
    long long m = 0, best = -1;
    if (mid > 0)
        for (long long mm = 1; mm <= (mid / 16 > 1 ? mid / 16 : 1); ++mm) {
            const long long cm = (mid + mm - 1) / mm;
            const long long cost = (tiles * mm + sms - 1) / sms * (cm + 7);
            if (best < 0 || cost < best) { best = cost; m = mm; }
        }
    st->cm = m > 0 ? (int)((mid + m - 1) / m) : 1;
    st->m = m > 0 ? (mid + st->cm - 1) / st->cm : 0;
    st->chunks = st->m + (st->za > 0 ? 1 : 0) + (st->zb < g.nz ? 1 : 0);
    const int layer = std::max(st->za, g.nz - st->zb);
    st->zt = P > 0 ? layer + 4 : 1;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const long long xb = (xbw * BR + 31) / 32 * 32;
    const long long big = FIELDS + 8 * xb + 8LL * BOX;   // largest stage: two x halves, y and z
    const long long ring = (long long)max_smem / 4 - BAR_BYTES / 4 - head_floats(st->zt);
    st->ring = (int)ring;
    st->smem = BAR_BYTES + 4 * (size_t)(head_floats(st->zt) + st->ring);
    if (ring < 2 * big ||
        cudaFuncSetAttribute(k_tb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem) != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FDTD_ERR_CUDA;
    }
    st->probe_ver = -1;
    h->tb2 = st;
    return FDTD_OK;
}

void tb2_release(fdtd_ctx *h) {
    HostState *st = static_cast<HostState *>(h->tb2);
    if (st) {
        cudaFree(st->d_rec);
        cudaFree(st->d_idx);
        cudaFree(st->d_pbuf);
    }
    delete st;
    h->tb2 = nullptr;
}

void launch_tb2(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->tb2);
    if (st->probe_ver != h->probe_ver) {
        const int rc = build_records(h, st);
        if (rc != FDTD_OK && h->status == FDTD_OK) h->status = rc;
    }
    const Grid &g = h->g;
    Args a;
    a.g = g;
    float *out = h->fields[h->cur ^ 1];
    for (int c = 0; c < 6; ++c) a.out[c] = out + (size_t)c * g.comp;
    a.pm = cpml_view(h);
    h->ecur ^= 1;   // the E psi set this pass writes
    const Cpml other = cpml_view(h);
    h->ecur ^= 1;
    for (int ax = 0; ax < 3; ++ax)
        for (int t = 0; t < 2; ++t) a.eout[ax][t] = other.e[ax][t];
    a.tiles_x = st->tiles_x;
    a.tiles_y = st->tiles_y;
    a.za = st->za;
    a.zb = st->zb;
    a.cm = st->cm;
    a.m = st->m;
    a.zt = st->zt;
    a.ring = st->ring;
    a.xlo4 = st->xlo4;
    a.xhb = st->xhb;
    a.xbw = st->xbw;
    a.cur = h->cur;
    a.ecur = h->ecur;
    a.src = h->src;
    a.ss1 = source_window(h->src, h->steps);
    a.ss2 = source_window(h->src, h->steps + 1);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.flags = h->d_flags;
    a.prec = st->d_rec;
    a.pidx = st->d_idx;
    a.pbuf = st->d_pbuf;
    dim3 grid(st->tiles_x * st->tiles_y, st->chunks);
    k_tb2<<<grid, NT, st->smem, s>>>(a, st->maps);
}

float *tb2_probe_values(fdtd_ctx *h) {
    HostState *st = static_cast<HostState *>(h->tb2);
    return st ? st->d_pbuf : nullptr;
}

}  // namespace fdtd
