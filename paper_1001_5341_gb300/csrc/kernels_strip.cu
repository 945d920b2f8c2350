// kernels_strip.cu -- one-pass leapfrog step over the interior box as a
// register-strip z-march.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B), so a step reads E^n and
// H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once: 24 B read and 24 B
// written per cell.
//
// The kernel covers the interior box of cells [P+1, N-P-1] on each axis (the
// whole grid without a CPML).  No CPML memory is touched there: the E-type
// positions of the box lie outside the layers, and so do the H-type positions
// P+1/2 .. N-P-3/2 and the halo H at cell P that the box's first cells need.
// The shell of cells around the box is updated afterwards by kernels_basic.cu.
//
// Work decomposition.  A warp owns 30 consecutive x columns and a strip of TY
// rows in y, and marches up a chunk of z planes.  Lane L sits on column
// i = ilo + 30 t - 1 + L: lanes 1..30 own their column, lane 0 carries the
// column to the left (its H is needed by lane 1's E update) and lane 31 the
// column to the right (its E is needed by lane 30's H update).  Per plane k a
// lane
//   - has in registers E^n(k) Ez, E^n(k+1) Ex/Ey and H^{n-1/2}(k) for rows
//     j0-1 .. j0+TY of its column (E^n(k) Ex/Ey carried from plane k-1), and
//     issues the loads of plane k+1 into a second register buffer before it
//     computes, so every warp keeps a plane of loads in flight;
//   - computes H^{n+1/2}(k) on rows j0-1 .. j0+TY-1; the x neighbour i+1 comes
//     from lane L+1 by a warp shuffle, the y neighbour from the next register;
//   - computes E^{n+1}(k) on its own rows; the x neighbour i-1 of H comes from
//     lane L-1 by a shuffle, the z neighbour k-1 of Hx, Hy from registers kept
//     from the previous plane;
//   - stores its own H and E.
// Row j0-1 and lanes 0/31 are recomputed halo and never stored.  There is no
// shared memory and no block-level barrier: warps are independent.  A chunk
// that starts above the box's first plane first recomputes H^{n+1/2}(k0-1) of
// its own rows (no stores).
#include <cuda_runtime.h>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

#ifndef STRIP_TY
#define STRIP_TY 4
#endif
#ifndef STRIP_MINB
#define STRIP_MINB 2
#endif
#ifndef STRIP_WARPS
#define STRIP_WARPS 8
#endif
constexpr int TY = STRIP_TY;        // rows per lane
constexpr int OWN = 30;             // owned columns per warp
constexpr int WARPS = STRIP_WARPS;  // warps per block, stacked in y
constexpr int NT = 32 * WARPS;

struct Args {
    Grid g;
    const float *ex, *ey, *ez, *hx, *hy, *hz;   // input set
    float *oex, *oey, *oez, *ohx, *ohy, *ohz;   // output set
    int ilo, ihi, jlo, jhi, klo, khi;           // interior box (cells, inclusive)
    Source src;
    SourceStep ss;      // this step's window of planes that may carry current
    float kE, kH;
    int chunk;          // planes per block
};

// One plane's loads: rows r = -1..TY of the lane's column at index a = r + 1.
struct Plane {
    float ez0[TY + 2];  // Ez^n(k)
    float ex1[TY + 2];  // Ex^n(k+1)
    float ey1[TY + 1];  // Ey^n(k+1)
    float hx[TY + 1];   // Hx^{n-1/2}(k), becomes H^{n+1/2}(k)
    float hz[TY + 1];   // Hz
    float hy[TY];       // Hy (own rows only)
};

__device__ __forceinline__ float ld(const float *p, unsigned off, bool ok) {
    return ok ? __ldg(p + off) : 0.0f;
}

// Loads of plane k (E^n(k) Ez, E^n(k+1) Ex/Ey, H^{n-1/2}(k)) for the lane's
// column; a row is loaded if it lies on the node grid.
__device__ __forceinline__ void load_plane(const Args &A, Plane &p, int k, unsigned cofs,
                                           bool colok, int j0) {
    const Grid &g = A.g;
    const unsigned base = cofs + (unsigned)k * (unsigned)g.plane;
    const unsigned up = (unsigned)g.plane;
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) {
        const int j = j0 + a - 1;
        const bool ok = colok && j >= 0 && j <= g.ny;
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

__device__ __forceinline__ void compute_plane(const Args &A, Plane &p, int k, bool own, int i,
                                              int j0, bool lane_owns, unsigned cofs, bool src_here,
                                              float (&ex0)[TY + 2], float (&ey0)[TY + 1],
                                              float (&hxp)[TY], float (&hyp)[TY]) {
    const Grid &g = A.g;
    const float kH = A.kH;
    // ---- H^{n+1/2}(k) on rows j0-1 .. j0+TY-1 ----
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const float ezR = __shfl_down_sync(0xffffffffu, p.ez0[a], 1);
        const float eyR = __shfl_down_sync(0xffffffffu, ey0[a], 1);
        p.hx[a] = p.hx[a] - kH * ((p.ez0[a + 1] - p.ez0[a]) - (p.ey1[a] - ey0[a]));
        p.hz[a] = p.hz[a] - kH * ((eyR - ey0[a]) - (ex0[a + 1] - ex0[a]));
        if (a >= 1) p.hy[a - 1] = p.hy[a - 1] - kH * ((p.ex1[a] - ex0[a]) - (ezR - p.ez0[a]));
    }

    if (own) {
        const unsigned base = cofs + (unsigned)k * (unsigned)g.plane;
        const float kE = A.kE;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = j0 + r;
            const int a = r + 1;
            const float hzL = __shfl_up_sync(0xffffffffu, p.hz[a], 1);
            const float hyL = __shfl_up_sync(0xffffffffu, p.hy[r], 1);
            if (lane_owns && j <= A.jhi) {
                const unsigned o = base + (unsigned)r * (unsigned)g.pitch;
                float src = 0.0f;
                if (src_here) src = source_at(A.src, A.ss, i, j, k);
                // components a cell owns on the grid's low faces are not updated
                if (i >= 1) A.ohx[o] = p.hx[a];
                if (j >= 1) A.ohy[o] = p.hy[r];
                if (k >= 1) A.ohz[o] = p.hz[a];
                if (j >= 1 && k >= 1)
                    A.oex[o] = ex0[a] + kE * ((p.hz[a] - p.hz[a - 1]) - (p.hy[r] - hyp[r]));
                if (i >= 1 && k >= 1)
                    A.oey[o] = ey0[a] + kE * ((p.hx[a] - hxp[r]) - (p.hz[a] - hzL));
                if (i >= 1 && j >= 1)
                    A.oez[o] = p.ez0[a] + kE * ((p.hy[r] - hyL) - (p.hx[a] - p.hx[a - 1])) + src;
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

__global__ void __launch_bounds__(NT, STRIP_MINB) k_strip(const Args A) {
    const Grid &g = A.g;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int i = A.ilo + (int)blockIdx.x * OWN - 1 + lane;
    const int j0 = A.jlo + ((int)blockIdx.y * WARPS + warp) * TY;
    if (j0 > A.jhi) return;  // the whole warp is outside the box
    const int k0 = A.klo + (int)blockIdx.z * A.chunk;
    if (k0 > A.khi) return;
    const int k1 = min(A.khi + 1, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    const bool colok = i >= 0 && i <= g.nx;
    const bool lane_owns = lane >= 1 && lane <= OWN && i <= A.ihi;
    // offset of (i, j0) inside one component plane; row j0 + r is cofs + r * pitch
    // (the unsigned wrap-around at r = -1, j0 = 0 is never dereferenced: the load
    // predicate tests j >= 0)
    const unsigned cofs = colok ? (unsigned)i + (unsigned)j0 * (unsigned)g.pitch : 0u;
    // warp-uniform: does the strip meet the current's footprint?
    const int xlo = A.ilo + (int)blockIdx.x * OWN;
    const bool src_xy = A.src.active && xlo <= A.src.ic + A.src.L && xlo + OWN - 1 >= A.src.ic - A.src.L &&
                        j0 <= A.src.jc + A.src.L && j0 + TY - 1 >= A.src.jc - A.src.L;

    float ex0[TY + 2], ey0[TY + 1], hxp[TY], hyp[TY];
    {
        const unsigned o0 = cofs + (unsigned)kstart * (unsigned)g.plane;
#pragma unroll
        for (int a = 0; a < TY + 2; ++a) {
            const int j = j0 + a - 1;
            const bool ok = colok && j >= 0 && j <= g.ny;
            ex0[a] = ld(A.ex, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
            if (a < TY + 1) ey0[a] = ld(A.ey, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) { hxp[r] = 0.0f; hyp[r] = 0.0f; }
    }
    // two register buffers: while plane k is computed from one, the loads of
    // plane k+1 are in flight into the other
    Plane pa, pb;
    load_plane(A, pa, kstart, cofs, colok, j0);
    int k = kstart;
    while (k < k1) {
        if (k + 1 < k1) load_plane(A, pb, k + 1, cofs, colok, j0);
        compute_plane(A, pa, k, k >= k0, i, j0, lane_owns, cofs,
                      src_xy && k >= A.ss.klo && k <= A.ss.khi, ex0, ey0, hxp, hyp);
        ++k;
        if (k >= k1) break;
        if (k + 1 < k1) load_plane(A, pa, k + 1, cofs, colok, j0);
        compute_plane(A, pb, k, k >= k0, i, j0, lane_owns, cofs,
                      src_xy && k >= A.ss.klo && k <= A.ss.khi, ex0, ey0, hxp, hyp);
        ++k;
    }
}

struct HostState {
    int ilo, ihi, jlo, jhi, klo, khi;
    int bx, by, chunks, chunk;
    Shell shell;
};

}  // namespace

const char *strip_name() { return "fused-strip-30x4"; }

int strip_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    // 32-bit offsets inside one component array
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
    HostState *st = new HostState();
    const int P = h->P;
    const int lo = P > 0 ? P + 1 : 0;
    st->ilo = lo; st->ihi = g.nx - 1 - (P > 0 ? P : 0);
    st->jlo = lo; st->jhi = g.ny - 1 - (P > 0 ? P : 0);
    st->klo = lo; st->khi = g.nz - 1 - (P > 0 ? P : 0);
    const int ex = st->ihi - st->ilo + 1, ey = st->jhi - st->jlo + 1, ez = st->khi - st->klo + 1;
    st->bx = (ex + OWN - 1) / OWN;
    st->by = (ey + WARPS * TY - 1) / (WARPS * TY);
    int sms = h->num_sms > 0 ? h->num_sms : 1;
    // about eight waves of resident blocks, chunks of >= 16 planes
    const long long want = 8LL * STRIP_MINB * sms;
    long long chunks = (want + (long long)st->bx * st->by - 1) / ((long long)st->bx * st->by);
    if (chunks > ez / 16) chunks = ez / 16;
    if (chunks < 1) chunks = 1;
    st->chunk = (int)((ez + chunks - 1) / chunks);
    st->chunks = (ez + st->chunk - 1) / st->chunk;
    // the shell: z slabs, y slabs of the remaining planes, x slabs of the rest
    Shell &sh = st->shell;
    sh.n = 0;
    auto add = [&](int i0, int i1, int j0, int j1, int k0, int k1) {
        if (i1 < i0 || j1 < j0 || k1 < k0) return;
        sh.lo[sh.n][0] = i0; sh.hi[sh.n][0] = i1;
        sh.lo[sh.n][1] = j0; sh.hi[sh.n][1] = j1;
        sh.lo[sh.n][2] = k0; sh.hi[sh.n][2] = k1;
        sh.n++;
    };
    if (P > 0) {
        add(0, g.nx - 1, 0, g.ny - 1, 0, st->klo - 1);
        add(0, g.nx - 1, 0, g.ny - 1, st->khi + 1, g.nz - 1);
        add(0, g.nx - 1, 0, st->jlo - 1, st->klo, st->khi);
        add(0, g.nx - 1, st->jhi + 1, g.ny - 1, st->klo, st->khi);
        add(0, st->ilo - 1, st->jlo, st->jhi, st->klo, st->khi);
        add(st->ihi + 1, g.nx - 1, st->jlo, st->jhi, st->klo, st->khi);
    }
    sh.start[0] = 0;
    for (int b = 0; b < sh.n; ++b)
        sh.start[b + 1] = sh.start[b] + (long long)(sh.hi[b][0] - sh.lo[b][0] + 1) *
                                            (sh.hi[b][1] - sh.lo[b][1] + 1) * (sh.hi[b][2] - sh.lo[b][2] + 1);
    h->strip = st;
    return FDTD_OK;
}

void strip_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->strip);
    h->strip = nullptr;
}

long long strip_interior_cells(const fdtd_ctx *h) {
    const HostState *st = static_cast<const HostState *>(h->strip);
    return (long long)(st->ihi - st->ilo + 1) * (st->jhi - st->jlo + 1) * (st->khi - st->klo + 1);
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
    a.ilo = st->ilo; a.ihi = st->ihi; a.jlo = st->jlo; a.jhi = st->jhi; a.klo = st->klo; a.khi = st->khi;
    a.src = h->src;
    a.ss = source_window(h->src, h->steps);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.chunk = st->chunk;
    dim3 grid(st->bx, st->by, st->chunks);
    k_strip<<<grid, NT, 0, s>>>(a);
}

int launch_strip_shell(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->strip);
    int n = 0;
    launch_shell(h, st->shell, s, &n);
    return n;
}

}  // namespace fdtd
