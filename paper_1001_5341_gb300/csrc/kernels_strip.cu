// kernels_strip.cu -- one-pass leapfrog step as a vectorised register-strip
// z-march.
//
// H^{n+1/2} and E^{n+1} of a plane are computed together (Yee scheme,
// Sec. III.A; shower current of Sec. III.B), so a step reads E^n and
// H^{n-1/2} once and writes H^{n+1/2} and E^{n+1} once: 24 B read and 24 B
// written per cell (plus CPML memory in the slabs).
//
// Work decomposition.  A lane holds four consecutive x columns (one 16-byte
// vector per row and component); a warp spans 128 columns starting at
// x0 = 120 t - 4, and lanes 1..30 own their 120 columns while lane 0 (the four
// columns to the left) and lane 31 (the four to the right) are halo.  Each
// warp takes a strip of TY rows in y and marches up a chunk of z planes.  Per
// plane k a lane
//   - loads E^n(k) Ez, E^n(k+1) Ex/Ey and H^{n-1/2}(k) for rows j0-1 .. j0+TY
//     (E^n(k) Ex/Ey are carried from the previous plane), 16 B per load;
//   - computes H^{n+1/2}(k) on rows j0-1 .. j0+TY-1; the x neighbour of its
//     last column is the next lane's first (warp shuffle), y neighbours are
//     the next row's registers;
//   - computes E^{n+1}(k) on its own rows; the x neighbour of its first column
//     is the previous lane's last (shuffle), the z neighbours k-1 of Hx, Hy are
//     kept in registers from the previous plane;
//   - stores its own H and E as 16-byte vectors.  Entries the step does not
//     update (faces, edges, the grid's padding) are written as zero: the
//     boundary kernel that runs after overwrites the Mur faces, and PEC faces
//     stay zero.
// Row j0-1 and lanes 0/31 are recomputed halo and never stored.  There is no
// shared memory and no block-level barrier: warps are independent.
//
// The CPML terms and the shower current are evaluated only in a warp-uniform
// slow path taken by warps whose strip meets a PML slab or the current's
// footprint in this plane.  A chunk that starts at k0 > 0 first recomputes
// H^{n+1/2}(k0-1) of its own rows (no stores).
#include <cuda_runtime.h>

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {
namespace {

#ifndef STRIP_TY
#define STRIP_TY 2
#endif
#ifndef STRIP_WARPS
#define STRIP_WARPS 4
#endif
#ifndef STRIP_MINB
#define STRIP_MINB 3
#endif
constexpr int TY = STRIP_TY;        // rows per lane
constexpr int OWN = 120;            // owned columns per warp (lanes 1..30)
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

__device__ __forceinline__ float4 ld4(const float *p, unsigned off, bool ok) {
    if (!ok) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4 *>(p + off));
}

__device__ __forceinline__ float &el(float4 &v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ float elc(const float4 &v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
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

struct Lane {
    int c0;          // first of the lane's four columns
    unsigned cofs;   // offset of (c0, j0) inside a component plane
    bool colok;      // the lane's vector lies inside the padded row
    bool owner;      // lanes 1..30
    int j0;
};

template <bool SLOW>
__device__ __forceinline__ void plane_step(const Args &A, const Lane &L, int k, bool own,
                                           float4 (&ex0)[TY + 2], float4 (&ey0)[TY + 1],
                                           float4 (&hxp)[TY], float4 (&hyp)[TY]) {
    const Grid &g = A.g;
    const unsigned pitch = (unsigned)g.pitch;
    const unsigned base = L.cofs + (unsigned)k * (unsigned)g.plane;
    const unsigned up = (unsigned)g.plane;
    // rows r = -1..TY at index a = r + 1
    float4 ez0[TY + 2], ex1[TY + 2], ey1[TY + 1], hx[TY + 1], hz[TY + 1], hy[TY];
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) {
        const int j = L.j0 + a - 1;
        const bool ok = L.colok && j >= 0 && j <= g.ny;
        const unsigned o = base + (unsigned)(a - 1) * pitch;
        ez0[a] = ld4(A.ez, o, ok);
        ex1[a] = ld4(A.ex, o + up, ok);
        if (a < TY + 1) {
            ey1[a] = ld4(A.ey, o + up, ok);
            hx[a] = ld4(A.hx, o, ok);
            hz[a] = ld4(A.hz, o, ok);
        }
        if (a >= 1 && a < TY + 1) hy[a - 1] = ld4(A.hy, o, ok);
    }

    const Cpml &pm = A.pml;
    const float kH = A.kH, kE = A.kE;
    const int lz = SLOW ? slab_cell(k, g.nz, pm.P) : -1;

    // ---- H^{n+1/2}(k) on rows j0-1 .. j0+TY-1 ----
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const int j = L.j0 + a - 1;
        // the column right of the lane's last one: the next lane's first
        const float ezR = __shfl_down_sync(0xffffffffu, ez0[a].x, 1);
        const float eyR = __shfl_down_sync(0xffffffffu, ey0[a].x, 1);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = L.c0 + e;
            const float ezr = e < 3 ? elc(ez0[a], e + 1) : ezR;
            const float eyr = e < 3 ? elc(ey0[a], e + 1) : eyR;
            float dyx = elc(ez0[a + 1], e) - elc(ez0[a], e);   // Hx: dEz/dy
            float dzx = elc(ey1[a], e) - elc(ey0[a], e);       //     dEy/dz
            float dxz = eyr - elc(ey0[a], e);                  // Hz: dEy/dx
            float dyz = elc(ex0[a + 1], e) - elc(ex0[a], e);   //     dEx/dy
            float dzy = 0.f, dxy = 0.f;                        // Hy (own rows)
            if (a >= 1) {
                dzy = elc(ex1[a], e) - elc(ex0[a], e);
                dxy = ezr - elc(ez0[a], e);
            }
            if (SLOW) {
                const bool in = L.colok && i >= 0 && i < g.nx && j >= 0 && j < g.ny;
                const bool w = in && own && a >= 1 && L.owner;
                const bool wx = w && i >= 1, wy = w && j >= 1, wz = w && k >= 1;
                const int lx = in ? slab_cell(i, g.nx, pm.P) : -1;
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
                if (lx >= 0) {
                    const unsigned q = (unsigned)psi_x(g, pm.W, lx, j, k);
                    const float aa = pm.aH[0][i], bb = pm.bH[0][i];
                    if (a >= 1) dxy = psih(pm.hin[0][0], pm.hout[0][0], q, aa, bb, dxy, wy);
                    dxz = psih(pm.hin[0][1], pm.hout[0][1], q, aa, bb, dxz, wz);
                }
            }
            el(hx[a], e) = elc(hx[a], e) - kH * (dyx - dzx);
            el(hz[a], e) = elc(hz[a], e) - kH * (dxz - dyz);
            if (a >= 1) el(hy[a - 1], e) = elc(hy[a - 1], e) - kH * (dzy - dxy);
        }
    }

    if (own) {
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = L.j0 + r;
            const int a = r + 1;
            // the column left of the lane's first one: the previous lane's last
            const float hzL = __shfl_up_sync(0xffffffffu, hz[a].w, 1);
            const float hyL = __shfl_up_sync(0xffffffffu, hy[r].w, 1);
            float4 nex, ney, nez, ohx = hx[a], ohy = hy[r], ohz = hz[a];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = L.c0 + e;
                const float hzl = e > 0 ? elc(hz[a], e - 1) : hzL;
                const float hyl = e > 0 ? elc(hy[r], e - 1) : hyL;
                float dyEx = elc(hz[a], e) - elc(hz[a - 1], e);
                float dzEx = elc(hy[r], e) - elc(hyp[r], e);
                float dzEy = elc(hx[a], e) - elc(hxp[r], e);
                float dxEy = elc(hz[a], e) - hzl;
                float dxEz = elc(hy[r], e) - hyl;
                float dyEz = elc(hx[a], e) - elc(hx[a - 1], e);
                float src = 0.f;
                const bool inx = i >= 1 && i < g.nx;   // Ey, Ez, Hx live here
                if (SLOW && L.owner && i >= 0 && i < g.nx && j < g.ny) {
                    const int lx = slab_cell(i, g.nx, pm.P), ly = slab_cell(j, g.ny, pm.P);
                    if (ly >= 0) {
                        const unsigned q = (unsigned)psi_y(g, pm.W, i, ly, k);
                        const float aa = pm.aE[1][j], bb = pm.bE[1][j];
                        if (j >= 1 && k >= 1) dyEx = psie(pm.e[1][0], q, aa, bb, dyEx);
                        if (inx && j >= 1) dyEz = psie(pm.e[1][1], q, aa, bb, dyEz);
                    }
                    if (lz >= 0) {
                        const unsigned q = (unsigned)psi_z(g, pm.W, i, j, lz);
                        const float aa = pm.aE[2][k], bb = pm.bE[2][k];
                        if (j >= 1 && k >= 1) dzEx = psie(pm.e[2][0], q, aa, bb, dzEx);
                        if (inx && k >= 1) dzEy = psie(pm.e[2][1], q, aa, bb, dzEy);
                    }
                    if (lx >= 0) {
                        const unsigned q = (unsigned)psi_x(g, pm.W, lx, j, k);
                        const float aa = pm.aE[0][i], bb = pm.bE[0][i];
                        if (inx && k >= 1) dxEy = psie(pm.e[0][0], q, aa, bb, dxEy);
                        if (inx && j >= 1) dxEz = psie(pm.e[0][1], q, aa, bb, dxEz);
                    }
                    if (inx && j >= 1) src = source_at(A.src, A.ss, i, j, k);
                }
                // entries the step does not update are written as zero
                const bool ix = i >= 0 && i < g.nx;
                el(nex, e) = (ix && j >= 1 && k >= 1) ? elc(ex0[a], e) + kE * (dyEx - dzEx) : 0.f;
                el(ney, e) = (inx && k >= 1) ? elc(ey0[a], e) + kE * (dzEy - dxEy) : 0.f;
                el(nez, e) = (inx && j >= 1) ? elc(ez0[a], e) + kE * (dxEz - dyEz) + src : 0.f;
                if (!inx) el(ohx, e) = 0.f;
                if (!(ix && j >= 1)) el(ohy, e) = 0.f;
                if (!(ix && k >= 1)) el(ohz, e) = 0.f;
            }
            if (L.owner && L.colok && j < g.ny) {
                const unsigned o = base + (unsigned)r * pitch;
                *reinterpret_cast<float4 *>(A.ohx + o) = ohx;
                *reinterpret_cast<float4 *>(A.ohy + o) = ohy;
                *reinterpret_cast<float4 *>(A.ohz + o) = ohz;
                *reinterpret_cast<float4 *>(A.oex + o) = nex;
                *reinterpret_cast<float4 *>(A.oey + o) = ney;
                *reinterpret_cast<float4 *>(A.oez + o) = nez;
            }
        }
    }
    // carry to the next plane
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        hxp[r] = hx[r + 1];
        hyp[r] = hy[r];
    }
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) ex0[a] = ex1[a];
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) ey0[a] = ey1[a];
}

__global__ void __launch_bounds__(NT, STRIP_MINB) k_strip(const Args A) {
    const Grid &g = A.g;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Lane L;
    const int x0 = (int)blockIdx.x * OWN - 4;
    L.c0 = x0 + 4 * lane;
    L.j0 = ((int)blockIdx.y * WARPS + warp) * TY;
    if (L.j0 >= g.ny) return;  // the whole warp is above the grid
    const int k0 = (int)blockIdx.z * A.chunk;
    if (k0 >= g.nz) return;
    const int k1 = min(g.nz, k0 + A.chunk);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    // a vector is loaded/stored only if it lies inside the padded row; pitch is
    // a multiple of 32 and c0 of 4, so it lies wholly inside or wholly outside
    L.colok = L.c0 >= 0 && L.c0 < g.pitch;
    L.owner = lane >= 1 && lane <= 30 && L.c0 < g.nx;
    // offset of (c0, j0) inside a component plane; row j0 + r is cofs + r*pitch
    // (the unsigned wrap-around at r = -1, j0 = 0 is never dereferenced)
    L.cofs = L.colok ? (unsigned)L.c0 + (unsigned)L.j0 * (unsigned)g.pitch : 0u;

    // warp-uniform: does the strip meet an x/y PML slab or the current's footprint?
    const int P = A.pml.P;
    const int ilo = x0, ihi = x0 + 127;
    const bool xy_slow = P > 0 && (ilo <= P || ihi >= g.nx - P || L.j0 - 1 <= P || L.j0 + TY - 1 >= g.ny - P);
    const bool src_xy = A.src.active && ilo <= A.src.ic + A.src.L && ihi >= A.src.ic - A.src.L &&
                        L.j0 <= A.src.jc + A.src.L && L.j0 + TY - 1 >= A.src.jc - A.src.L;

    float4 ex0[TY + 2], ey0[TY + 1], hxp[TY], hyp[TY];
    {
        const unsigned o0 = L.cofs + (unsigned)kstart * (unsigned)g.plane;
#pragma unroll
        for (int a = 0; a < TY + 2; ++a) {
            const int j = L.j0 + a - 1;
            const bool ok = L.colok && j >= 0 && j <= g.ny;
            ex0[a] = ld4(A.ex, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
            if (a < TY + 1) ey0[a] = ld4(A.ey, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            hxp[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            hyp[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int k = kstart; k < k1; ++k) {
        const bool own = k >= k0;
        const bool slow = xy_slow || (P > 0 && (k <= P || k >= g.nz - P)) ||
                          (src_xy && k >= A.ss.klo && k <= A.ss.khi);
        if (slow)
            plane_step<true>(A, L, k, own, ex0, ey0, hxp, hyp);
        else
            plane_step<false>(A, L, k, own, ex0, ey0, hxp, hyp);
    }
}

struct HostState {
    int bx, by, chunks, chunk;
};

}  // namespace

const char *strip_name() { return "fused-strip-v4x120"; }

int strip_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    // 32-bit offsets inside one component array and inside one psi array
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    if (g.pitch % 4 != 0) return FDTD_ERR_ARG;
    HostState *st = new HostState();
    st->bx = (g.nx + OWN - 1) / OWN;
    st->by = (g.ny + WARPS * TY - 1) / (WARPS * TY);
    int sms = h->num_sms > 0 ? h->num_sms : 1;
    // about eight waves of resident blocks, chunks of >= 16 planes
    const long long want = 8LL * STRIP_MINB * sms;
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
