// kernels_tile.cu -- one-pass leapfrog step over the CPML-free interior box as
// a z-march of aligned 32-column tiles.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B), so a step reads E^n and
// H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once: 24 B read and 24 B
// written per cell.
//
// A block owns the 32 columns [i0, i0+32) (i0 a multiple of 32, so every
// warp-wide load and store is one aligned 128-byte line) and BY = WY*TY rows,
// and marches up a chunk of z planes.  Warp w holds rows j0 + w*TY .. +TY-1,
// one column per lane, in registers.  Per plane k:
//   1. each lane loads its own cells: E^n(k) Ez, E^n(k+1) Ex/Ey, H^{n-1/2}(k)
//      (E^n(k) Ex/Ey carried from the previous plane), one plane ahead in a
//      second register buffer;
//   2. each warp puts its lowest row of Ez^n(k), Ex^n(k) into shared memory for
//      the warp below; barrier;
//   3. H^{n+1/2}(k) of the own cells: x neighbour i+1 by warp shuffle (lane 31
//      loads column i0+32), y neighbour j+1 from the next register or the warp
//      above (the top warp loads row j0+BY);
//   4. each warp puts its highest row of Hx, Hz into shared memory for the
//      warp above; barrier;
//   5. E^{n+1}(k): x neighbour i-1 of H by shuffle (lane 0 recomputes H at
//      column i0-1 from E^n and H^{n-1/2} there), y neighbour j-1 from the
//      previous register or the warp below (the bottom warp recomputes row
//      j0-1), z neighbour k-1 of Hx, Hy from registers of the previous plane;
//      store H and E of the own cells.
// Cells of the tile outside the box are computed as halo and not stored.  The
// box's halo (cells at P) lies outside the CPML layers, so no CPML memory is
// needed.  A chunk that starts above the box's first plane first recomputes
// H^{n+1/2}(k0-1) of its cells (no stores).
#include <cuda_runtime.h>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

#ifndef TILE_TY
#define TILE_TY 4
#endif
#ifndef TILE_WY
#define TILE_WY 8
#endif
#ifndef TILE_MINB
#define TILE_MINB 1
#endif
constexpr int TY = TILE_TY;   // rows per warp
constexpr int WY = TILE_WY;   // warps per block, stacked in y
constexpr int BY = WY * TY;   // rows per block
constexpr int NT = 32 * WY;

struct Args {
    Grid g;
    const float *ex, *ey, *ez, *hx, *hy, *hz;   // input set
    float *oex, *oey, *oez, *ohx, *ohy, *ohz;   // output set
    int ilo, ihi, jlo, jhi, klo, khi;           // interior box (cells, inclusive)
    int bx0;                                    // first 32-column tile index
    int tiles_x, tiles_y, chunk;
    Source src;
    SourceStep ss;
    float kE, kH;
};

// One plane's loads of a lane's own cells (rows r = 0..TY-1).
struct Own {
    float ez0[TY], ex1[TY], ey1[TY], hx[TY], hy[TY], hz[TY];
};

__device__ __forceinline__ float ld(const float *p, unsigned off, bool ok) {
    return ok ? __ldg(p + off) : 0.0f;
}

struct Ctx {
    int i, j0;          // lane column, warp's first row
    int w, lane;
    unsigned cofs;      // offset of (i, j0) in a component plane
    bool colok;         // column on the node grid
    bool owns;          // column inside the box
    bool rowok[TY];     // own rows on the node grid
    bool left;          // lane 0 must recompute H at column i0-1
    bool right;         // lane 31 must load E at column i0+32
};

__device__ __forceinline__ void load_own(const Args &A, const Ctx &c, Own &o, int k) {
    const Grid &g = A.g;
    const unsigned base = c.cofs + (unsigned)k * (unsigned)g.plane;
    const unsigned up = (unsigned)g.plane;
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        const bool ok = c.colok && c.rowok[r];
        const unsigned q = base + (unsigned)r * (unsigned)g.pitch;
        o.ez0[r] = ld(A.ez, q, ok);
        o.ex1[r] = ld(A.ex, q + up, ok);
        o.ey1[r] = ld(A.ey, q + up, ok);
        o.hx[r] = ld(A.hx, q, ok);
        o.hy[r] = ld(A.hy, q, ok);
        o.hz[r] = ld(A.hz, q, ok);
    }
}

// Carried from plane to plane.
struct Carry {
    float ex0[TY], ey0[TY];   // E^n(k) Ex, Ey of the own cells
    float hxp[TY], hyp[TY];   // H^{n+1/2}(k-1) Hx, Hy of the own cells
    float exT0;               // top warp: Ex^n(k) at the row above the block
    float exB0, eyB0;         // bottom warp: Ex^n(k), Ey^n(k) at the row below
    float exL0[TY + 1];       // lane 0: Ex^n(k) at column i0-1, rows j0..j0+TY
};

struct Blk {
    int i0, jb;
    bool top, bot, jt_ok, jbm_ok, src_blk;
};

__device__ __forceinline__ void step_plane(const Args &A, const Ctx &c, const Blk &b, int k, bool own,
                                           const Own &o, Carry &s, float (*sEz)[32], float (*sEx)[32],
                                           float (*sHx)[32], float (*sHz)[32]) {
    const Grid &g = A.g;
    const unsigned pitch = (unsigned)g.pitch, planeo = (unsigned)g.plane;
    const unsigned base = c.cofs + (unsigned)k * planeo;

    // halo loads of this plane (single lanes / single warps; mostly L2 hits)
    float ezT = 0.f, exT1 = 0.f;                                   // top warp, row above
    float ezB = 0.f, exB1 = 0.f, eyB1 = 0.f, hxB = 0.f, hzB = 0.f;  // bottom warp, row below
    if (b.top && b.jt_ok && c.colok) {
        const unsigned q = base + (unsigned)TY * pitch;
        ezT = __ldg(A.ez + q);
        exT1 = __ldg(A.ex + q + planeo);
    }
    if (b.bot && b.jbm_ok && c.colok) {
        const unsigned q = base - pitch;
        ezB = __ldg(A.ez + q);
        exB1 = __ldg(A.ex + q + planeo);
        eyB1 = __ldg(A.ey + q + planeo);
        hxB = __ldg(A.hx + q);
        hzB = __ldg(A.hz + q);
    }
    float ezR[TY], eyR[TY], eyRB = 0.f;   // lane 31: E at column i0+32
    {
        const bool ok = c.lane == 31 && c.right;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const bool okr = ok && c.rowok[r];
            ezR[r] = ld(A.ez, base + 1u + (unsigned)r * pitch, okr);
            eyR[r] = ld(A.ey, base + 1u + (unsigned)r * pitch, okr);
        }
        if (b.bot && b.jbm_ok) eyRB = ld(A.ey, base + 1u - pitch, ok);
    }
    float eyL[TY], ezL[TY], hzL0[TY], hyL0[TY], exL1[TY + 1];  // lane 0: column i0-1
    {
        const bool ok = c.lane == 0 && c.left;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const bool okr = ok && c.rowok[r];
            const unsigned q = base - 1u + (unsigned)r * pitch;
            eyL[r] = ld(A.ey, q, okr);
            ezL[r] = ld(A.ez, q, okr);
            hzL0[r] = ld(A.hz, q, okr);
            hyL0[r] = ld(A.hy, q, okr);
        }
#pragma unroll
        for (int r = 0; r <= TY; ++r)
            exL1[r] = ld(A.ex, base - 1u + planeo + (unsigned)r * pitch, ok && c.j0 + r <= g.ny);
    }

    // lowest E row for the warp below
    sEz[c.w][c.lane] = o.ez0[0];
    sEx[c.w][c.lane] = s.ex0[0];
    __syncthreads();

    // H^{n+1/2}(k) of own rows
    const float kH = A.kH;
    float hxn[TY], hyn[TY], hzn[TY];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        const float ezUp = r + 1 < TY ? o.ez0[r + 1] : (b.top ? ezT : sEz[min(c.w + 1, WY - 1)][c.lane]);
        const float exUp = r + 1 < TY ? s.ex0[r + 1] : (b.top ? s.exT0 : sEx[min(c.w + 1, WY - 1)][c.lane]);
        float ezRt = __shfl_down_sync(0xffffffffu, o.ez0[r], 1);
        float eyRt = __shfl_down_sync(0xffffffffu, s.ey0[r], 1);
        if (c.lane == 31) { ezRt = ezR[r]; eyRt = eyR[r]; }
        hxn[r] = o.hx[r] - kH * ((ezUp - o.ez0[r]) - (o.ey1[r] - s.ey0[r]));
        hyn[r] = o.hy[r] - kH * ((o.ex1[r] - s.ex0[r]) - (ezRt - o.ez0[r]));
        hzn[r] = o.hz[r] - kH * ((eyRt - s.ey0[r]) - (exUp - s.ex0[r]));
    }
    // bottom warp: H at the row below the block (Hx, Hz)
    float hxB1 = 0.f, hzB1 = 0.f;
    {
        float eyRb = __shfl_down_sync(0xffffffffu, s.eyB0, 1);
        if (c.lane == 31) eyRb = eyRB;
        if (b.bot) {
            hxB1 = hxB - kH * ((o.ez0[0] - ezB) - (eyB1 - s.eyB0));
            hzB1 = hzB - kH * ((eyRb - s.eyB0) - (s.ex0[0] - s.exB0));
        }
    }
    // lane 0: H at column i0-1 (Hz, Hy), own rows
    float hzLn[TY], hyLn[TY];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        hzLn[r] = hzL0[r] - kH * ((s.ey0[r] - eyL[r]) - (s.exL0[r + 1] - s.exL0[r]));
        hyLn[r] = hyL0[r] - kH * ((exL1[r] - s.exL0[r]) - (o.ez0[r] - ezL[r]));
    }

    // highest H row for the warp above
    sHx[c.w][c.lane] = hxn[TY - 1];
    sHz[c.w][c.lane] = hzn[TY - 1];
    __syncthreads();

    // E^{n+1}(k) of own rows, stores
    if (own) {
        const float kE = A.kE;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = c.j0 + r;
            const float hxDn = r > 0 ? hxn[r - 1] : (b.bot ? hxB1 : sHx[max(c.w - 1, 0)][c.lane]);
            const float hzDn = r > 0 ? hzn[r - 1] : (b.bot ? hzB1 : sHz[max(c.w - 1, 0)][c.lane]);
            float hzLt = __shfl_up_sync(0xffffffffu, hzn[r], 1);
            float hyLt = __shfl_up_sync(0xffffffffu, hyn[r], 1);
            if (c.lane == 0) { hzLt = hzLn[r]; hyLt = hyLn[r]; }
            if (c.owns && j <= A.jhi) {
                const unsigned q = base + (unsigned)r * pitch;
                float src = 0.f;
                if (b.src_blk) src = source_at(A.src, A.ss, c.i, j, k);
                if (c.i >= 1) A.ohx[q] = hxn[r];
                if (j >= 1) A.ohy[q] = hyn[r];
                if (k >= 1) A.ohz[q] = hzn[r];
                if (j >= 1 && k >= 1) A.oex[q] = s.ex0[r] + kE * ((hzn[r] - hzDn) - (hyn[r] - s.hyp[r]));
                if (c.i >= 1 && k >= 1) A.oey[q] = s.ey0[r] + kE * ((hxn[r] - s.hxp[r]) - (hzn[r] - hzLt));
                if (c.i >= 1 && j >= 1)
                    A.oez[q] = o.ez0[r] + kE * ((hyn[r] - hyLt) - (hxn[r] - hxDn)) + src;
            }
        }
    }
    // carry to plane k+1
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        s.hxp[r] = hxn[r];
        s.hyp[r] = hyn[r];
        s.ex0[r] = o.ex1[r];
        s.ey0[r] = o.ey1[r];
    }
    s.exT0 = exT1;
    s.exB0 = exB1;
    s.eyB0 = eyB1;
#pragma unroll
    for (int r = 0; r <= TY; ++r) s.exL0[r] = exL1[r];
}

__global__ void __launch_bounds__(NT, TILE_MINB) k_tile(const Args A) {
    __shared__ float sEz[WY][32], sEx[WY][32];   // lowest row of each warp, E^n(k)
    __shared__ float sHx[WY][32], sHz[WY][32];   // highest row of each warp, H^{n+1/2}(k)
    const Grid &g = A.g;
    Ctx c;
    Blk b;
    c.lane = threadIdx.x & 31;
    c.w = threadIdx.x >> 5;
    const int tx = (int)blockIdx.x % A.tiles_x, ty = (int)blockIdx.x / A.tiles_x;
    b.i0 = (A.bx0 + tx) * 32;
    b.jb = A.jlo + ty * BY;
    c.i = b.i0 + c.lane;
    c.j0 = b.jb + c.w * TY;
    const int k0 = A.klo + (int)blockIdx.y * A.chunk;
    const int k1 = min(A.khi + 1, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    c.colok = c.i <= g.nx;
    c.owns = c.i >= A.ilo && c.i <= A.ihi;
#pragma unroll
    for (int r = 0; r < TY; ++r) c.rowok[r] = c.j0 + r <= g.ny;
    c.left = b.i0 >= 1 && b.i0 > A.ilo;        // lane 0's E needs H at i0-1
    c.right = b.i0 + 32 <= g.nx;               // lane 31's H needs E at i0+32
    c.cofs = c.colok ? (unsigned)c.i + (unsigned)c.j0 * (unsigned)g.pitch : 0u;
    b.top = c.w == WY - 1;
    b.bot = c.w == 0;
    b.jt_ok = b.jb + BY <= g.ny;
    b.jbm_ok = b.jb >= 1;
    b.src_blk = A.src.active && b.i0 <= A.src.ic + A.src.L && b.i0 + 31 >= A.src.ic - A.src.L &&
                b.jb <= A.src.jc + A.src.L && b.jb + BY - 1 >= A.src.jc - A.src.L;

    Carry s;
    {
        const unsigned pitch = (unsigned)g.pitch;
        const unsigned o0 = c.cofs + (unsigned)kstart * (unsigned)g.plane;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const bool ok = c.colok && c.rowok[r];
            s.ex0[r] = ld(A.ex, o0 + (unsigned)r * pitch, ok);
            s.ey0[r] = ld(A.ey, o0 + (unsigned)r * pitch, ok);
            s.hxp[r] = 0.f;
            s.hyp[r] = 0.f;
        }
        s.exT0 = (b.top && b.jt_ok && c.colok) ? __ldg(A.ex + o0 + (unsigned)TY * pitch) : 0.f;
        s.exB0 = (b.bot && b.jbm_ok && c.colok) ? __ldg(A.ex + o0 - pitch) : 0.f;
        s.eyB0 = (b.bot && b.jbm_ok && c.colok) ? __ldg(A.ey + o0 - pitch) : 0.f;
#pragma unroll
        for (int r = 0; r <= TY; ++r)
            s.exL0[r] = ld(A.ex, o0 - 1u + (unsigned)r * pitch, c.lane == 0 && c.left && c.j0 + r <= g.ny);
    }
    // two register buffers: while plane k is computed from one, the loads of
    // plane k+1 are in flight into the other
    Own pa, pb;
    load_own(A, c, pa, kstart);
    int k = kstart;
    while (k < k1) {
        if (k + 1 < k1) load_own(A, c, pb, k + 1);
        step_plane(A, c, b, k, k >= k0, pa, s, sEz, sEx, sHx, sHz);
        ++k;
        if (k >= k1) break;
        if (k + 1 < k1) load_own(A, c, pa, k + 1);
        step_plane(A, c, b, k, k >= k0, pb, s, sEz, sEx, sHx, sHz);
        ++k;
    }
}

struct HostState {
    Args proto;
    int blocks_x, chunks;
};

}  // namespace

const char *tile_name() { return "fused-tile-32"; }

int tile_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
    HostState *st = new HostState();
    Args &a = st->proto;
    const int P = h->P;
    const int lo = P > 0 ? P + 1 : 0;
    a.ilo = lo; a.ihi = g.nx - 1 - P;
    a.jlo = lo; a.jhi = g.ny - 1 - P;
    a.klo = lo; a.khi = g.nz - 1 - P;
    a.bx0 = a.ilo / 32;
    a.tiles_x = a.ihi / 32 - a.bx0 + 1;
    a.tiles_y = (a.jhi - a.jlo + BY) / BY;
    const int ez = a.khi - a.klo + 1;
    const int sms = h->num_sms > 0 ? h->num_sms : 1;
    const long long want = 8LL * TILE_MINB * sms;
    long long chunks = (want + (long long)a.tiles_x * a.tiles_y - 1) / ((long long)a.tiles_x * a.tiles_y);
    if (chunks > ez / 16) chunks = ez / 16;
    if (chunks < 1) chunks = 1;
    a.chunk = (int)((ez + chunks - 1) / chunks);
    st->chunks = (ez + a.chunk - 1) / a.chunk;
    st->blocks_x = a.tiles_x * a.tiles_y;
    h->tile = st;
    return FDTD_OK;
}

void tile_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->tile);
    h->tile = nullptr;
}

long long tile_cells(const fdtd_ctx *h) {
    const Args &a = static_cast<const HostState *>(h->tile)->proto;
    return (long long)(a.ihi - a.ilo + 1) * (a.jhi - a.jlo + 1) * (a.khi - a.klo + 1);
}

void launch_tile(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->tile);
    const Grid &g = h->g;
    Args a = st->proto;
    a.g = g;
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    const size_t c = (size_t)g.comp;
    a.ex = in; a.ey = in + c; a.ez = in + 2 * c; a.hx = in + 3 * c; a.hy = in + 4 * c; a.hz = in + 5 * c;
    a.oex = out; a.oey = out + c; a.oez = out + 2 * c; a.ohx = out + 3 * c; a.ohy = out + 4 * c; a.ohz = out + 5 * c;
    a.src = h->src;
    a.ss = source_window(h->src, h->steps);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    dim3 grid(st->blocks_x, st->chunks);
    k_tile<<<grid, NT, 0, s>>>(a);
}

}  // namespace fdtd
