// kernels_strip.cu -- one-pass leapfrog step as a register-strip z-march.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B), so a step reads E^n and
// H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once: 24 B read and 24 B
// written per cell, plus the CPML memory of the cells in the layers.
//
// The grid is covered by up to seven boxes of cells, all updated by one
// launch: the interior box [P+1, N-P-1]^3 (x range shrunk to whole groups of
// four columns), where no CPML term exists, and up to six shell boxes (two z
// slabs over the whole x-y plane, two y slabs over the interior z range, two x
// slabs over the interior y and z ranges).  Every box
// reads only the input set and writes only its own cells of the output set, so
// the boxes are independent.  Interior blocks run the plain update with a
// register double buffer; shell blocks run the update with the CPML memory
// loads issued together with the field loads of the same plane.
//
// Work decomposition inside a box.  A warp owns 30 consecutive x columns and
// a strip of TY rows in y, and marches up a chunk of z planes.  Lane L sits on
// column i = ilo + 30 t - 1 + L: lanes 1..30 own their column, lane 0 carries
// the column to the left (its H is needed by lane 1's E update) and lane 31 the
// column to the right (its E is needed by lane 30's H update).  Per plane k a
// lane
//   - loads E^n(k) Ez, E^n(k+1) Ex/Ey and H^{n-1/2}(k) for rows j0-1 .. j0+TY
//     of its column (E^n(k) Ex/Ey carried from plane k-1);
//   - computes H^{n+1/2}(k) on rows j0-1 .. j0+TY-1; the x neighbour i+1 comes
//     from lane L+1 by a warp shuffle, the y neighbour from the next register;
//   - computes E^{n+1}(k) on its own rows; the x neighbour i-1 of H comes from
//     lane L-1 by a shuffle, the z neighbour k-1 of Hx, Hy from registers kept
//     from the previous plane;
//   - stores its own H and E.
// Row j0-1 and lanes 0/31 are recomputed halo and never stored; the halo of a
// box never needs CPML memory it does not own (the interior box's halo cells
// at P lie outside the layers).  There is no shared memory and no block-level
// barrier: warps are independent.  A chunk that starts above its box's first
// plane first recomputes H^{n+1/2}(k0-1) of its own rows (no stores).
#include <cuda_runtime.h>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

#ifndef STRIP_TY
#define STRIP_TY 8
#endif
#ifndef STRIP_TY_PML
#define STRIP_TY_PML 2
#endif
#ifndef STRIP_MINB
#define STRIP_MINB 1
#endif
#ifndef STRIP_WARPS
#define STRIP_WARPS 8
#endif
constexpr int TYI = STRIP_TY;       // rows per lane, interior box
constexpr int TYP = STRIP_TY_PML;   // rows per lane, CPML shell boxes
constexpr int OWN = 30;             // owned columns per warp
constexpr int WARPS = STRIP_WARPS;  // warps per block, stacked in y
constexpr int NT = 32 * WARPS;
constexpr int MAXBOX = 7;

struct Box {
    int lo[3], hi[3];   // cells, inclusive
    int pml;            // 1: the box lies in the CPML shell
    int tx, ty;         // tiles (blocks) in x and y
    int chunk;          // planes per block
    int first;          // first block index of the box
};

struct Args {
    Grid g;
    const float *ex, *ey, *ez, *hx, *hy, *hz;   // input set
    float *oex, *oey, *oez, *ohx, *ohy, *ohz;   // output set
    Cpml pml;
    Source src;
    SourceStep ss;      // this step's window of planes that may carry current
    float kE, kH;
    int nbox;
    Box box[MAXBOX];
};

template <int TY>
struct Plane {
    float ez0[TY + 2];  // Ez^n(k), rows j0-1 .. j0+TY
    float ex1[TY + 2];  // Ex^n(k+1)
    float ey1[TY + 1];  // Ey^n(k+1), rows j0-1 .. j0+TY-1
    float hx[TY + 1];   // Hx^{n-1/2}(k), becomes H^{n+1/2}(k)
    float hz[TY + 1];   // Hz
    float hy[TY];       // Hy, own rows
};

// CPML memory of one plane for the lane's column: H terms on rows j0-1 ..
// j0+TY-1 (index a), E terms on the own rows (index r).
template <int TY>
struct PlanePsi {
    float xHy[TY], xHz[TY + 1], yHx[TY + 1], yHz[TY + 1], zHx[TY + 1], zHy[TY];
    float xEy[TY], xEz[TY], yEx[TY], yEz[TY], zEx[TY], zEy[TY];
};

struct Col {
    int i;            // lane's column
    int j0;           // first own row
    bool colok;       // column lies on the node grid (loads)
    bool owns;        // lane owns its column in this box
    unsigned cofs;    // offset of (i, j0) inside one component plane
    int jhi;          // last row of the box
};

__device__ __forceinline__ float ld(const float *p, unsigned off, bool ok) {
    return ok ? __ldg(p + off) : 0.0f;
}

template <int TY>
__device__ __forceinline__ void load_plane(const Args &A, Plane<TY> &p, int k, const Col &c) {
    const Grid &g = A.g;
    const unsigned base = c.cofs + (unsigned)k * (unsigned)g.plane;
    const unsigned up = (unsigned)g.plane;
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) {
        const int j = c.j0 + a - 1;
        const bool ok = c.colok && j >= 0 && j <= g.ny;
        const unsigned o = base + (unsigned)(a - 1) * (unsigned)g.pitch;
        p.ez0[a] = ld(A.ez, o, ok);
        p.ex1[a] = ld(A.ex, o + up, ok);
        if (a < TY + 1) {
            p.ey1[a] = ld(A.ey, o + up, ok);
            p.hx[a] = ld(A.hx, o, ok);
            p.hz[a] = ld(A.hz, o, ok);
        }
        if (a >= 1 && a < TY + 1) p.hy[a - 1] = ld(A.hy, o, ok);
    }
}

// CPML memory of plane k (read step: H terms from the n-1/2 copy, E terms in
// place); zero where the cell is not in the matching layer.
template <int TY>
__device__ __forceinline__ void load_psi(const Args &A, PlanePsi<TY> &q, int k, const Col &c) {
    const Grid &g = A.g;
    const Cpml &p = A.pml;
    const bool xin = c.colok && c.i < g.nx;
    const int lx = xin ? psi_x_pos(c.i, g.nx, p.P) : -1;
    const int lz = slab_cell(k, g.nz, p.P);
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const int j = c.j0 + a - 1;
        const bool in = xin && j >= 0 && j < g.ny;
        const int ly = in ? slab_cell(j, g.ny, p.P) : -1;
        const bool bx = in && lx >= 0, bz = in && lz >= 0;
        const unsigned ix = bx ? (unsigned)psi_x(g, p.P, lx, j, k) : 0u;
        const unsigned iy = ly >= 0 ? (unsigned)psi_y(g, p.W, c.i, ly, k) : 0u;
        const unsigned iz = bz ? (unsigned)psi_z(g, p.W, c.i, j, lz) : 0u;
        q.xHz[a] = bx ? p.hin[0][1][ix] : 0.f;
        q.yHx[a] = ly >= 0 ? p.hin[1][0][iy] : 0.f;
        q.yHz[a] = ly >= 0 ? p.hin[1][1][iy] : 0.f;
        q.zHx[a] = bz ? p.hin[2][0][iz] : 0.f;
        if (a >= 1) {
            const int r = a - 1;
            q.xHy[r] = bx ? p.hin[0][0][ix] : 0.f;
            q.zHy[r] = bz ? p.hin[2][1][iz] : 0.f;
            q.xEy[r] = bx ? p.e[0][0][ix] : 0.f;
            q.xEz[r] = bx ? p.e[0][1][ix] : 0.f;
            q.yEx[r] = ly >= 0 ? p.e[1][0][iy] : 0.f;
            q.yEz[r] = ly >= 0 ? p.e[1][1][iy] : 0.f;
            q.zEx[r] = bz ? p.e[2][0][iz] : 0.f;
            q.zEy[r] = bz ? p.e[2][1][iz] : 0.f;
        }
    }
}

// psi^{new} = b psi + a d; returns d + psi^{new}
__device__ __forceinline__ float cpml(float &psi, float a, float b, float d) {
    psi = b * psi + a * d;
    return d + psi;
}

template <int TY, bool PML>
__device__ __forceinline__ void compute_plane(const Args &A, Plane<TY> &p, PlanePsi<TY> &q, int k,
                                              bool own, const Col &c, bool src_here,
                                              float (&ex0)[TY + 2], float (&ey0)[TY + 1],
                                              float (&hxp)[TY], float (&hyp)[TY]) {
    const Grid &g = A.g;
    const Cpml &pm = A.pml;
    const int i = c.i;
    const float kH = A.kH;
    int lx = -1, lz = -1;
    if (PML) {
        lx = (c.colok && i < g.nx) ? psi_x_pos(i, g.nx, pm.P) : -1;
        lz = slab_cell(k, g.nz, pm.P);
    }
    // ---- H^{n+1/2}(k) on rows j0-1 .. j0+TY-1 ----
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const int j = c.j0 + a - 1;
        const float ezR = __shfl_down_sync(0xffffffffu, p.ez0[a], 1);
        const float eyR = __shfl_down_sync(0xffffffffu, ey0[a], 1);
        float dyx = p.ez0[a + 1] - p.ez0[a];   // Hx: dEz/dy
        float dzx = p.ey1[a] - ey0[a];         //     dEy/dz
        float dxz = eyR - ey0[a];              // Hz: dEy/dx
        float dyz = ex0[a + 1] - ex0[a];       //     dEx/dy
        if (PML) {
            const bool in = c.colok && i < g.nx && j >= 0 && j < g.ny;
            const int ly = in ? slab_cell(j, g.ny, pm.P) : -1;
            if (ly >= 0) {
                const float aa = pm.aH[1][j], bb = pm.bH[1][j];
                dyx = cpml(q.yHx[a], aa, bb, dyx);
                dyz = cpml(q.yHz[a], aa, bb, dyz);
            }
            if (in && lz >= 0) dzx = cpml(q.zHx[a], pm.aH[2][k], pm.bH[2][k], dzx);
            if (in && lx >= 0) dxz = cpml(q.xHz[a], pm.aH[0][i], pm.bH[0][i], dxz);
        }
        p.hx[a] = p.hx[a] - kH * (dyx - dzx);
        p.hz[a] = p.hz[a] - kH * (dxz - dyz);
        if (a >= 1) {
            const int r = a - 1;
            float dzy = p.ex1[a] - ex0[a];     // Hy: dEx/dz
            float dxy = ezR - p.ez0[a];        //     dEz/dx
            if (PML) {
                const bool in = c.colok && i < g.nx && j >= 0 && j < g.ny;
                if (in && lz >= 0) dzy = cpml(q.zHy[r], pm.aH[2][k], pm.bH[2][k], dzy);
                if (in && lx >= 0) dxy = cpml(q.xHy[r], pm.aH[0][i], pm.bH[0][i], dxy);
            }
            p.hy[r] = p.hy[r] - kH * (dzy - dxy);
        }
    }

    if (own) {
        const unsigned base = c.cofs + (unsigned)k * (unsigned)g.plane;
        const float kE = A.kE;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = c.j0 + r;
            const int a = r + 1;
            const float hzL = __shfl_up_sync(0xffffffffu, p.hz[a], 1);
            const float hyL = __shfl_up_sync(0xffffffffu, p.hy[r], 1);
            if (c.owns && j <= c.jhi) {
                const unsigned o = base + (unsigned)r * (unsigned)g.pitch;
                float dyEx = p.hz[a] - p.hz[a - 1];
                float dzEx = p.hy[r] - hyp[r];
                float dzEy = p.hx[a] - hxp[r];
                float dxEy = p.hz[a] - hzL;
                float dxEz = p.hy[r] - hyL;
                float dyEz = p.hx[a] - p.hx[a - 1];
                if (PML) {
                    const int ly = slab_cell(j, g.ny, pm.P);
                    if (ly >= 0) {
                        const float aa = pm.aE[1][j], bb = pm.bE[1][j];
                        dyEx = cpml(q.yEx[r], aa, bb, dyEx);
                        dyEz = cpml(q.yEz[r], aa, bb, dyEz);
                        const unsigned iy = (unsigned)psi_y(g, pm.W, i, ly, k);
                        if (j >= 1 && k >= 1) pm.e[1][0][iy] = q.yEx[r];
                        if (i >= 1 && j >= 1) pm.e[1][1][iy] = q.yEz[r];
                        if (i >= 1) pm.hout[1][0][iy] = q.yHx[a];
                        if (k >= 1) pm.hout[1][1][iy] = q.yHz[a];
                    }
                    if (lz >= 0) {
                        const float aa = pm.aE[2][k], bb = pm.bE[2][k];
                        dzEx = cpml(q.zEx[r], aa, bb, dzEx);
                        dzEy = cpml(q.zEy[r], aa, bb, dzEy);
                        const unsigned iz = (unsigned)psi_z(g, pm.W, i, j, lz);
                        if (j >= 1 && k >= 1) pm.e[2][0][iz] = q.zEx[r];
                        if (i >= 1 && k >= 1) pm.e[2][1][iz] = q.zEy[r];
                        if (i >= 1) pm.hout[2][0][iz] = q.zHx[a];
                        if (j >= 1) pm.hout[2][1][iz] = q.zHy[r];
                    }
                    if (lx >= 0) {
                        const float aa = pm.aE[0][i], bb = pm.bE[0][i];
                        dxEy = cpml(q.xEy[r], aa, bb, dxEy);
                        dxEz = cpml(q.xEz[r], aa, bb, dxEz);
                        const unsigned ix = (unsigned)psi_x(g, pm.P, lx, j, k);
                        if (i >= 1 && k >= 1) pm.e[0][0][ix] = q.xEy[r];
                        if (i >= 1 && j >= 1) pm.e[0][1][ix] = q.xEz[r];
                        if (j >= 1) pm.hout[0][0][ix] = q.xHy[r];
                        if (k >= 1) pm.hout[0][1][ix] = q.xHz[a];
                    }
                }
                float src = 0.0f;
                if (src_here) src = source_at(A.src, A.ss, i, j, k);
                // components a cell owns on the grid's low faces are not updated
                if (i >= 1) A.ohx[o] = p.hx[a];
                if (j >= 1) A.ohy[o] = p.hy[r];
                if (k >= 1) A.ohz[o] = p.hz[a];
                if (j >= 1 && k >= 1) A.oex[o] = ex0[a] + kE * (dyEx - dzEx);
                if (i >= 1 && k >= 1) A.oey[o] = ey0[a] + kE * (dzEy - dxEy);
                if (i >= 1 && j >= 1) A.oez[o] = p.ez0[a] + kE * (dxEz - dyEz) + src;
            }
        }
    }
    // carry to the next plane
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        hxp[r] = p.hx[r + 1];
        hyp[r] = p.hy[r];
    }
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) ex0[a] = p.ex1[a];
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) ey0[a] = p.ey1[a];
}

template <int TY, bool PML>
__device__ __forceinline__ void march(const Args &A, const Box &B, int tile, int lane, int warp) {
    const Grid &g = A.g;
    Col c;
    const int bxi = tile % B.tx, byi = (tile / B.tx) % B.ty, ch = tile / (B.tx * B.ty);
    c.i = B.lo[0] + bxi * OWN - 1 + lane;
    c.j0 = B.lo[1] + (byi * WARPS + warp) * TY;
    if (c.j0 > B.hi[1]) return;  // the whole warp is outside the box
    const int k0 = B.lo[2] + ch * B.chunk;
    if (k0 > B.hi[2]) return;
    const int k1 = min(B.hi[2] + 1, k0 + B.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    c.colok = c.i >= 0 && c.i <= g.nx;
    c.owns = lane >= 1 && lane <= OWN && c.i <= B.hi[0];
    c.jhi = B.hi[1];
    // (the unsigned wrap-around at row j0-1 = -1 is never dereferenced: the
    // load predicate tests j >= 0)
    c.cofs = c.colok ? (unsigned)c.i + (unsigned)c.j0 * (unsigned)g.pitch : 0u;
    const int xlo = B.lo[0] + bxi * OWN;
    const bool src_xy = A.src.active && xlo <= A.src.ic + A.src.L && xlo + OWN - 1 >= A.src.ic - A.src.L &&
                        c.j0 <= A.src.jc + A.src.L && c.j0 + TY - 1 >= A.src.jc - A.src.L;

    float ex0[TY + 2], ey0[TY + 1], hxp[TY], hyp[TY];
    {
        const unsigned o0 = c.cofs + (unsigned)kstart * (unsigned)g.plane;
#pragma unroll
        for (int a = 0; a < TY + 2; ++a) {
            const int j = c.j0 + a - 1;
            const bool ok = c.colok && j >= 0 && j <= g.ny;
            ex0[a] = ld(A.ex, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
            if (a < TY + 1) ey0[a] = ld(A.ey, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) { hxp[r] = 0.0f; hyp[r] = 0.0f; }
    }
    if (PML) {
        // one buffer: the CPML memory loads go out with the field loads of the
        // same plane, so they add no round trip of their own
        Plane<TY> p;
        PlanePsi<TY> q;
        for (int k = kstart; k < k1; ++k) {
            load_plane(A, p, k, c);
            load_psi(A, q, k, c);
            compute_plane<TY, true>(A, p, q, k, k >= k0, c, src_xy && k >= A.ss.klo && k <= A.ss.khi,
                                    ex0, ey0, hxp, hyp);
        }
    } else {
        // two buffers: while plane k is computed from one, the loads of plane
        // k+1 are in flight into the other
        Plane<TY> pa, pb;
        PlanePsi<TY> q;  // unused on this path
        load_plane(A, pa, kstart, c);
        int k = kstart;
        while (k < k1) {
            if (k + 1 < k1) load_plane(A, pb, k + 1, c);
            compute_plane<TY, false>(A, pa, q, k, k >= k0, c, src_xy && k >= A.ss.klo && k <= A.ss.khi,
                                     ex0, ey0, hxp, hyp);
            ++k;
            if (k >= k1) break;
            if (k + 1 < k1) load_plane(A, pa, k + 1, c);
            compute_plane<TY, false>(A, pb, q, k, k >= k0, c, src_xy && k >= A.ss.klo && k <= A.ss.khi,
                                     ex0, ey0, hxp, hyp);
            ++k;
        }
    }
}

__global__ void __launch_bounds__(NT, STRIP_MINB) k_strip(const Args A) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int blk = (int)blockIdx.x;
    int b = 0;
    while (b + 1 < A.nbox && blk >= A.box[b + 1].first) ++b;
    const Box &B = A.box[b];
    const int tile = blk - B.first;
    if (B.pml)
        march<TYP, true>(A, B, tile, lane, warp);
    else
        march<TYI, false>(A, B, tile, lane, warp);
}

struct HostState {
    int nbox;
    Box box[MAXBOX];
    int blocks;
    long long interior_cells;
};

}  // namespace

const char *strip_name() { return "fused-strip-30"; }

int strip_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    // 32-bit offsets inside one component array and one psi array
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    HostState *st = new HostState();
    int blo[3], bhi[3];
    interior_box(h, blo, bhi);
    const int ilo = blo[0], ihi = bhi[0], lo = blo[1], jhi = bhi[1], khi = bhi[2];
    st->nbox = 0;
    const int sms = h->num_sms > 0 ? h->num_sms : 1;
    int first = 0;
    auto add = [&](int i0, int i1, int j0, int j1, int k0, int k1, int pml) {
        if (i1 < i0 || j1 < j0 || k1 < k0) return;
        Box &B = st->box[st->nbox++];
        B.lo[0] = i0; B.hi[0] = i1; B.lo[1] = j0; B.hi[1] = j1; B.lo[2] = k0; B.hi[2] = k1;
        B.pml = pml;
        const int ty = pml ? TYP : TYI;
        B.tx = (i1 - i0 + 1 + OWN - 1) / OWN;
        B.ty = (j1 - j0 + 1 + WARPS * ty - 1) / (WARPS * ty);
        const int ez = k1 - k0 + 1;
        // the interior box: about eight waves of blocks, chunks of >= 16 planes;
        // the thin shell boxes: one chunk per 32 planes
        long long chunks;
        if (!pml) {
            const long long want = 8LL * STRIP_MINB * sms;
            chunks = (want + (long long)B.tx * B.ty - 1) / ((long long)B.tx * B.ty);
            if (chunks > ez / 16) chunks = ez / 16;
        } else {
            chunks = (ez + 31) / 32;
        }
        if (chunks < 1) chunks = 1;
        B.chunk = (int)((ez + chunks - 1) / chunks);
        chunks = (ez + B.chunk - 1) / B.chunk;
        B.first = first;
        first += B.tx * B.ty * (int)chunks;
    };
    add(ilo, ihi, lo, jhi, lo, khi, 0);
    st->interior_cells = (long long)(ihi - ilo + 1) * (jhi - lo + 1) * (khi - lo + 1);
    // the shell: empty boxes are skipped (no CPML: at most the x+ columns
    // beyond the last whole group of four)
    add(0, g.nx - 1, 0, g.ny - 1, 0, lo - 1, 1);           // z- slab
    add(0, g.nx - 1, 0, g.ny - 1, khi + 1, g.nz - 1, 1);   // z+ slab
    add(0, g.nx - 1, 0, lo - 1, lo, khi, 1);               // y- slab
    add(0, g.nx - 1, jhi + 1, g.ny - 1, lo, khi, 1);       // y+ slab
    add(0, ilo - 1, lo, jhi, lo, khi, 1);                  // x- slab
    add(ihi + 1, g.nx - 1, lo, jhi, lo, khi, 1);           // x+ slab
    st->blocks = first;
    h->strip = st;
    return FDTD_OK;
}

void strip_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->strip);
    h->strip = nullptr;
}

void launch_strip(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->strip);
    const Grid &g = h->g;
    Args a;
    a.g = g;
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    const size_t c = (size_t)g.comp;
    a.ex = in; a.ey = in + c; a.ez = in + 2 * c; a.hx = in + 3 * c; a.hy = in + 4 * c; a.hz = in + 5 * c;
    a.oex = out; a.oey = out + c; a.oez = out + 2 * c; a.ohx = out + 3 * c; a.ohy = out + 4 * c; a.ohz = out + 5 * c;
    a.pml = cpml_view(h);
    a.src = h->src;
    a.ss = source_window(h->src, h->steps);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.nbox = st->nbox;
    for (int b = 0; b < st->nbox; ++b) a.box[b] = st->box[b];
    if (st->blocks > 0) k_strip<<<st->blocks, NT, 0, s>>>(a);
}

}  // namespace fdtd
