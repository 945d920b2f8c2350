// kernels_strip.cu -- one-pass leapfrog step as a register-strip z-march.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B), so a step reads E^n and
// H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once: 24 B read and 24 B
// written per cell (plus CPML memory in the slabs).
//
// Work decomposition.  A warp owns 30 consecutive x columns and a strip of TY
// rows in y, and marches up a chunk of z planes.  Lane L sits on column
// i = 30 t - 1 + L: lanes 1..30 own their column, lane 0 carries the column to
// the left (its H is needed by lane 1's E update) and lane 31 the column to
// the right (its E is needed by lane 30's H update).  Per plane k a lane
//   - has in registers E^n(k) Ez, E^n(k+1) Ex/Ey and H^{n-1/2}(k) for rows
//     j0-1 .. j0+TY of its column (E^n(k) Ex/Ey carried from plane k-1), and
//     issues the loads of plane k+1 into a second register buffer before it
//     computes, so every warp always has a plane of loads in flight;
//   - computes H^{n+1/2}(k) on rows j0-1 .. j0+TY-1; the x neighbour i+1 comes
//     from lane L+1 by a warp shuffle, the y neighbour from the next register;
//   - computes E^{n+1}(k) on its own rows; the x neighbour i-1 of H comes from
//     lane L-1 by a shuffle, the z neighbour k-1 of Hx, Hy from registers kept
//     from the previous plane;
//   - stores its own H and E.
// Row j0-1 and lanes 0/31 are recomputed halo and never stored.  There is no
// shared memory and no block-level barrier: warps are independent.
//
// The CPML terms and the shower current are only evaluated in a warp-uniform
// slow path taken by warps whose strip meets a PML slab or the current's
// footprint in this plane.  A chunk that starts at k0 > 0 first recomputes
// H^{n+1/2}(k0-1) of its own rows (no stores).
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
    Cpml pml;
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

// Loads of plane k (E^n(k) Ez, E^n(k+1) Ex/Ey, H^{n-1/2}(k)); rowok[a] says row
// j0 - 1 + a exists, colok the lane's column.
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

// psi^{new} = b psi + a d; the derivative gains psi^{new}.  H terms read the
// step n-1/2 copy and write the n+1/2 copy only for the cell's owner.
__device__ __forceinline__ float psih(const float *pin, float *pout, unsigned q, float a, float b,
                                      float d, bool write) {
    float p = b * pin[q] + a * d;
    if (write) pout[q] = p;
    return d + p;
}
__device__ __forceinline__ float psie(float *pe, unsigned q, float a, float b, float d) {
    float p = b * pe[q] + a * d;
    pe[q] = p;
    return d + p;
}

template <bool SLOW>
__device__ __forceinline__ void compute_plane(const Args &A, Plane &p, int k, bool own, int i,
                                              int j0, bool colok, bool lane_owns, unsigned cofs,
                                              float (&ex0)[TY + 2], float (&ey0)[TY + 1],
                                              float (&hxp)[TY], float (&hyp)[TY]) {
    const Grid &g = A.g;
    const Cpml &pm = A.pml;
    // ---- H^{n+1/2}(k) on rows j0-1 .. j0+TY-1 ----
    const float kH = A.kH;
    int lx = -1, lz = -1;
    if (SLOW) {
        lx = (colok && i < g.nx) ? slab_cell(i, g.nx, pm.P) : -1;
        lz = slab_cell(k, g.nz, pm.P);
    }
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const int j = j0 + a - 1;
        const float ezR = __shfl_down_sync(0xffffffffu, p.ez0[a], 1);
        const float eyR = __shfl_down_sync(0xffffffffu, ey0[a], 1);
        float dyx = p.ez0[a + 1] - p.ez0[a];   // Hx: dEz/dy
        float dzx = p.ey1[a] - ey0[a];         //     dEy/dz
        float dxz = eyR - ey0[a];              // Hz: dEy/dx
        float dyz = ex0[a + 1] - ex0[a];       //     dEx/dy
        float dzy = 0.0f, dxy = 0.0f;          // Hy (own rows only)
        if (a >= 1) {
            dzy = p.ex1[a] - ex0[a];
            dxy = ezR - p.ez0[a];
        }
        if (SLOW) {
            const bool in = colok && i < g.nx && j >= 0 && j < g.ny;
            const bool w = in && own && a >= 1 && lane_owns;
            const bool wx = w && i >= 1, wy = w && j >= 1, wz = w && k >= 1;
            const int ly = in ? slab_cell(j, g.ny, pm.P) : -1;
            if (ly >= 0) {
                const unsigned q = (unsigned)psi_y(g, pm.W, i, ly, k);
                const float aa = pm.aH[1][j], bb = pm.bH[1][j];
                dyx = psih(pm.hin[1][0], pm.hout[1][0], q, aa, bb, dyx, wx);
                dyz = psih(pm.hin[1][1], pm.hout[1][1], q, aa, bb, dyz, wz);
            }
            if (lz >= 0 && in) {
                const unsigned q = (unsigned)psi_z(g, pm.W, i, j, lz);
                const float aa = pm.aH[2][k], bb = pm.bH[2][k];
                dzx = psih(pm.hin[2][0], pm.hout[2][0], q, aa, bb, dzx, wx);
                if (a >= 1) dzy = psih(pm.hin[2][1], pm.hout[2][1], q, aa, bb, dzy, wy);
            }
            if (lx >= 0 && in) {
                const unsigned q = (unsigned)psi_x(g, pm.W, lx, j, k);
                const float aa = pm.aH[0][i], bb = pm.bH[0][i];
                if (a >= 1) dxy = psih(pm.hin[0][0], pm.hout[0][0], q, aa, bb, dxy, wy);
                dxz = psih(pm.hin[0][1], pm.hout[0][1], q, aa, bb, dxz, wz);
            }
        }
        p.hx[a] = p.hx[a] - kH * (dyx - dzx);
        p.hz[a] = p.hz[a] - kH * (dxz - dyz);
        if (a >= 1) p.hy[a - 1] = p.hy[a - 1] - kH * (dzy - dxy);
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
            float dyEx = p.hz[a] - p.hz[a - 1];
            float dzEx = p.hy[r] - hyp[r];
            float dzEy = p.hx[a] - hxp[r];
            float dxEy = p.hz[a] - hzL;
            float dxEz = p.hy[r] - hyL;
            float dyEz = p.hx[a] - p.hx[a - 1];
            const bool store = lane_owns && j < g.ny;
            float src = 0.0f;
            if (SLOW && store) {
                const int ly = slab_cell(j, g.ny, pm.P);
                if (ly >= 0) {
                    const unsigned q = (unsigned)psi_y(g, pm.W, i, ly, k);
                    const float aa = pm.aE[1][j], bb = pm.bE[1][j];
                    if (j >= 1 && k >= 1) dyEx = psie(pm.e[1][0], q, aa, bb, dyEx);
                    if (i >= 1 && j >= 1) dyEz = psie(pm.e[1][1], q, aa, bb, dyEz);
                }
                if (lz >= 0) {
                    const unsigned q = (unsigned)psi_z(g, pm.W, i, j, lz);
                    const float aa = pm.aE[2][k], bb = pm.bE[2][k];
                    if (j >= 1 && k >= 1) dzEx = psie(pm.e[2][0], q, aa, bb, dzEx);
                    if (i >= 1 && k >= 1) dzEy = psie(pm.e[2][1], q, aa, bb, dzEy);
                }
                if (lx >= 0) {
                    const unsigned q = (unsigned)psi_x(g, pm.W, lx, j, k);
                    const float aa = pm.aE[0][i], bb = pm.bE[0][i];
                    if (i >= 1 && k >= 1) dxEy = psie(pm.e[0][0], q, aa, bb, dxEy);
                    if (i >= 1 && j >= 1) dxEz = psie(pm.e[0][1], q, aa, bb, dxEz);
                }
                src = source_at(A.src, A.ss, i, j, k);
            }
            if (store) {
                const unsigned o = base + (unsigned)r * (unsigned)g.pitch;
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

__device__ __forceinline__ void do_plane(const Args &A, Plane &p, int k, bool own, int i, int j0,
                                         bool colok, bool lane_owns, unsigned cofs, bool xy_slow,
                                         bool src_xy, float (&ex0)[TY + 2], float (&ey0)[TY + 1],
                                         float (&hxp)[TY], float (&hyp)[TY]) {
    const int P = A.pml.P;
    const bool slow = xy_slow || (P > 0 && (k <= P || k >= A.g.nz - P)) ||
                      (src_xy && k >= A.ss.klo && k <= A.ss.khi);
    if (slow)
        compute_plane<true>(A, p, k, own, i, j0, colok, lane_owns, cofs, ex0, ey0, hxp, hyp);
    else
        compute_plane<false>(A, p, k, own, i, j0, colok, lane_owns, cofs, ex0, ey0, hxp, hyp);
}

__global__ void __launch_bounds__(NT, STRIP_MINB) k_strip(const Args A) {
    const Grid &g = A.g;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int i = (int)blockIdx.x * OWN - 1 + lane;
    const int j0 = ((int)blockIdx.y * WARPS + warp) * TY;
    if (j0 >= g.ny) return;  // the whole warp is above the grid
    const int k0 = (int)blockIdx.z * A.chunk;
    if (k0 >= g.nz) return;
    const int k1 = min(g.nz, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    const bool colok = i >= 0 && i <= g.nx;
    const bool lane_owns = lane >= 1 && lane <= OWN && i < g.nx;
    // offset of (i, j0) inside one component plane; row j0 + r is cofs + r * pitch
    // (the unsigned wrap-around at r = -1, j0 = 0 is never dereferenced: the load
    // predicate tests j >= 0)
    const unsigned cofs = colok ? (unsigned)i + (unsigned)j0 * (unsigned)g.pitch : 0u;

    // warp-uniform: does the strip meet an x/y PML slab or the current's footprint?
    const int P = A.pml.P;
    const int ilo = (int)blockIdx.x * OWN - 1, ihi = ilo + 31;
    const bool xy_slow = P > 0 && (ilo <= P || ihi >= g.nx - P || j0 - 1 <= P || j0 + TY - 1 >= g.ny - P);
    const bool src_xy = A.src.active && ilo <= A.src.ic + A.src.L && ihi >= A.src.ic - A.src.L &&
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
        do_plane(A, pa, k, k >= k0, i, j0, colok, lane_owns, cofs, xy_slow, src_xy, ex0, ey0, hxp, hyp);
        ++k;
        if (k >= k1) break;
        if (k + 1 < k1) load_plane(A, pa, k + 1, cofs, colok, j0);
        do_plane(A, pb, k, k >= k0, i, j0, colok, lane_owns, cofs, xy_slow, src_xy, ex0, ey0, hxp, hyp);
        ++k;
    }
}

struct HostState {
    int bx, by, chunks, chunk;
};

}  // namespace

const char *strip_name() { return "fused-strip-30x4"; }

int strip_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    // 32-bit offsets inside one component array and inside one psi array
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    HostState *st = new HostState();
    st->bx = (g.nx + OWN - 1) / OWN;
    st->by = (g.ny + WARPS * TY - 1) / (WARPS * TY);
    int sms = h->num_sms > 0 ? h->num_sms : 1;
    // about eight waves of two resident blocks per SM, chunks of >= 16 planes
    const long long want = 16LL * sms;
    long long chunks = (want + (long long)st->bx * st->by - 1) / ((long long)st->bx * st->by);
    if (chunks > g.nz / 16) chunks = g.nz / 16;
    if (chunks < 1) chunks = 1;
    st->chunk = (int)((g.nz + chunks - 1) / chunks);
    st->chunks = (g.nz + st->chunk - 1) / st->chunk;
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
    a.chunk = st->chunk;
    dim3 grid(st->bx, st->by, st->chunks);
    k_strip<<<grid, NT, 0, s>>>(a);
}

}  // namespace fdtd
