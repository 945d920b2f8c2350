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
//   - loads E^n(k) Ez, E^n(k+1) Ex/Ey and H^{n-1/2}(k) for rows j0-1 .. j0+TY
//     of its column (E^n(k) Ex/Ey are carried from the previous plane);
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

constexpr int TY = 8;        // rows per lane
constexpr int OWN = 30;      // owned columns per warp
constexpr int WARPS = 8;     // warps per block, stacked in y
constexpr int NT = 32 * WARPS;

struct Args {
    Grid g;
    const float *ein;   // Ex of the input set (Ey, Ez, Hx, Hy, Hz follow at +comp)
    float *eout;        // Ex of the output set
    Cpml pml;
    Source src;
    SourceStep ss;      // this step's charge position and window
    float kE, kH;
    int chunk;          // planes per block
};

__device__ __forceinline__ float ld(const float *p, unsigned off, bool ok) {
    return ok ? __ldg(p + off) : 0.0f;
}

// psi^{new} = b psi + a d (H terms: read step n-1/2, write n+1/2 if owned)
__device__ __forceinline__ float psih(const float *pin, float *pout, long long q, float a, float b,
                                      float d, bool write) {
    float p = b * pin[q] + a * d;
    if (write) pout[q] = p;
    return d + p;
}
__device__ __forceinline__ float psie(float *pe, long long q, float a, float b, float d) {
    float p = b * pe[q] + a * d;
    pe[q] = p;
    return d + p;
}

template <bool SLOW>
__device__ __forceinline__ void plane(const Args &A, int k, bool own, int lane, int i, int j0,
                                      bool colok, bool lane_owns, unsigned cofs, float (&ex0)[TY + 2],
                                      float (&ey0)[TY + 1], float (&hxp)[TY], float (&hyp)[TY]) {
    const Grid &g = A.g;
    const size_t comp = (size_t)g.comp;  // component stride (pointer arithmetic in 64 bits)
    const unsigned plane_off = (unsigned)k * (unsigned)g.plane;  // offsets inside one component
    const unsigned pitch = (unsigned)g.pitch;
    const float *Exi = A.ein, *Eyi = Exi + comp, *Ezi = Eyi + comp;
    const float *Hxi = Ezi + comp, *Hyi = Hxi + comp, *Hzi = Hyi + comp;
    // rows r = -1..TY map to array index a = r + 1; row j = j0 + r
    float ez0[TY + 2], ex1[TY + 2], ey1[TY + 1], hx[TY + 1], hy[TY], hz[TY + 1];
#pragma unroll
    for (int a = 0; a < TY + 2; ++a) {
        const int j = j0 + a - 1;
        const bool ok = colok && j >= 0 && j <= g.ny;
        const unsigned o = cofs + plane_off + (unsigned)(a - 1) * pitch;
        ez0[a] = ld(Ezi, o, ok);
        ex1[a] = ld(Exi, o + (unsigned)g.plane, ok);
        if (a < TY + 1) {
            ey1[a] = ld(Eyi, o + (unsigned)g.plane, ok);
            hx[a] = ld(Hxi, o, ok);
            hz[a] = ld(Hzi, o, ok);
        }
        if (a >= 1 && a < TY + 1) hy[a - 1] = ld(Hyi, o, ok);
    }

    // ---- H^{n+1/2}(k) on rows j0-1 .. j0+TY-1 ----
    const float kH = A.kH;
#pragma unroll
    for (int a = 0; a < TY + 1; ++a) {
        const int j = j0 + a - 1;
        const float ezR = __shfl_down_sync(0xffffffffu, ez0[a], 1);
        const float eyR = __shfl_down_sync(0xffffffffu, ey0[a], 1);
        float dyx = ez0[a + 1] - ez0[a];      // Hx: dEz/dy
        float dzx = ey1[a] - ey0[a];          //     dEy/dz
        float dxz = eyR - ey0[a];             // Hz: dEy/dx
        float dyz = ex0[a + 1] - ex0[a];      //     dEx/dy
        float dzy = 0.0f, dxy = 0.0f;         // Hy (own rows only)
        if (a >= 1) {
            dzy = ex1[a] - ex0[a];
            dxy = ezR - ez0[a];
        }
        if (SLOW) {
            // psi of the H update: read at n-1/2 always, written at n+1/2 only by
            // the owner of the cell and only for components the step updates
            const Cpml &p = A.pml;
            const bool w = own && a >= 1 && lane_owns && j >= 0 && j < g.ny && i < g.nx;
            const bool wx = w && i >= 1, wy = w && j >= 1, wz = w && k >= 1;
            const bool in = colok && i < g.nx && j >= 0 && j < g.ny;
            const int lx = in ? slab_cell(i, g.nx, p.P) : -1;
            const int ly = in ? slab_cell(j, g.ny, p.P) : -1;
            const int lz = in ? slab_cell(k, g.nz, p.P) : -1;
            if (ly >= 0) {
                const long long q = psi_y(g, p.W, i, ly, k);
                const float aa = p.aH[1][j], bb = p.bH[1][j];
                dyx = psih(p.hin[1][0], p.hout[1][0], q, aa, bb, dyx, wx);
                dyz = psih(p.hin[1][1], p.hout[1][1], q, aa, bb, dyz, wz);
            }
            if (lz >= 0) {
                const long long q = psi_z(g, p.W, i, j, lz);
                const float aa = p.aH[2][k], bb = p.bH[2][k];
                dzx = psih(p.hin[2][0], p.hout[2][0], q, aa, bb, dzx, wx);
                if (a >= 1) dzy = psih(p.hin[2][1], p.hout[2][1], q, aa, bb, dzy, wy);
            }
            if (lx >= 0) {
                const long long q = psi_x(g, p.W, lx, j, k);
                const float aa = p.aH[0][i], bb = p.bH[0][i];
                if (a >= 1) dxy = psih(p.hin[0][0], p.hout[0][0], q, aa, bb, dxy, wy);
                dxz = psih(p.hin[0][1], p.hout[0][1], q, aa, bb, dxz, wz);
            }
        }
        hx[a] = hx[a] - kH * (dyx - dzx);
        hz[a] = hz[a] - kH * (dxz - dyz);
        if (a >= 1) hy[a - 1] = hy[a - 1] - kH * (dzy - dxy);
    }

    if (own) {
        // ---- store H^{n+1/2}(k), own rows ----
        float *Hxo = A.eout + 3 * comp, *Hyo = Hxo + comp, *Hzo = Hyo + comp;
        float *Exo = A.eout, *Eyo = Exo + comp, *Ezo = Eyo + comp;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = j0 + r;
            if (lane_owns && j < g.ny) {
                const unsigned o = cofs + plane_off + (unsigned)r * pitch;
                if (i >= 1) Hxo[o] = hx[r + 1];
                if (j >= 1) Hyo[o] = hy[r];
                if (k >= 1) Hzo[o] = hz[r + 1];
            }
        }
        // ---- E^{n+1}(k), own rows ----
        const float kE = A.kE;
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const int j = j0 + r;
            const int a = r + 1;
            const float hzL = __shfl_up_sync(0xffffffffu, hz[a], 1);
            const float hyL = __shfl_up_sync(0xffffffffu, hy[r], 1);
            float dyEx = hz[a] - hz[a - 1];
            float dzEx = hy[r] - hyp[r];
            float dzEy = hx[a] - hxp[r];
            float dxEy = hz[a] - hzL;
            float dxEz = hy[r] - hyL;
            float dyEz = hx[a] - hx[a - 1];
            const bool store = lane_owns && j < g.ny;
            float src = 0.0f;
            if (SLOW && store) {
                const Cpml &p = A.pml;
                const int lx = slab_cell(i, g.nx, p.P), ly = slab_cell(j, g.ny, p.P),
                          lz = slab_cell(k, g.nz, p.P);
                if (ly >= 0) {
                    const long long q = psi_y(g, p.W, i, ly, k);
                    const float aa = p.aE[1][j], bb = p.bE[1][j];
                    if (j >= 1 && k >= 1) dyEx = psie(p.e[1][0], q, aa, bb, dyEx);
                    if (i >= 1 && j >= 1) dyEz = psie(p.e[1][1], q, aa, bb, dyEz);
                }
                if (lz >= 0) {
                    const long long q = psi_z(g, p.W, i, j, lz);
                    const float aa = p.aE[2][k], bb = p.bE[2][k];
                    if (j >= 1 && k >= 1) dzEx = psie(p.e[2][0], q, aa, bb, dzEx);
                    if (i >= 1 && k >= 1) dzEy = psie(p.e[2][1], q, aa, bb, dzEy);
                }
                if (lx >= 0) {
                    const long long q = psi_x(g, p.W, lx, j, k);
                    const float aa = p.aE[0][i], bb = p.bE[0][i];
                    if (i >= 1 && k >= 1) dxEy = psie(p.e[0][0], q, aa, bb, dxEy);
                    if (i >= 1 && j >= 1) dxEz = psie(p.e[0][1], q, aa, bb, dxEz);
                }
                src = source_at(A.src, A.ss, i, j, k);
            }
            if (store) {
                const unsigned o = cofs + plane_off + (unsigned)r * pitch;
                if (j >= 1 && k >= 1) Exo[o] = ex0[a] + kE * (dyEx - dzEx);
                if (i >= 1 && k >= 1) Eyo[o] = ey0[a] + kE * (dzEy - dxEy);
                if (i >= 1 && j >= 1) Ezo[o] = ez0[a] + kE * (dxEz - dyEz) + src;
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

__global__ void __launch_bounds__(NT, 2) k_strip(const Args A) {
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
    // offset of (i, j0) inside a component plane; row j0 + r is cofs + r * pitch
    // (unsigned wrap-around for r = -1 at j0 = 0 is never dereferenced: the load
    // predicate tests j >= 0)
    const unsigned cofs = colok ? (unsigned)i + (unsigned)j0 * (unsigned)g.pitch : 0u;

    // warp-uniform: does the strip meet an x/y PML slab or the current's footprint?
    const int P = A.pml.P;
    const int ilo = (int)blockIdx.x * OWN - 1, ihi = ilo + 31;
    bool xy_pml = P > 0 && (ilo <= P || ihi >= g.nx - P || j0 - 1 <= P || j0 + TY - 1 >= g.ny - P);
    bool src_xy = A.src.active && ilo <= A.src.ic + A.src.L && ihi >= A.src.ic - A.src.L &&
                  j0 <= A.src.jc + A.src.L && j0 + TY - 1 >= A.src.jc - A.src.L;

    float ex0[TY + 2], ey0[TY + 1], hxp[TY], hyp[TY];
    {
        const unsigned o0 = cofs + (unsigned)kstart * (unsigned)g.plane;
#pragma unroll
        for (int a = 0; a < TY + 2; ++a) {
            const int j = j0 + a - 1;
            const bool ok = colok && j >= 0 && j <= g.ny;
            ex0[a] = ld(A.ein, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
            if (a < TY + 1) ey0[a] = ld(A.ein + (size_t)g.comp, o0 + (unsigned)(a - 1) * (unsigned)g.pitch, ok);
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) { hxp[r] = 0.0f; hyp[r] = 0.0f; }
    }
    for (int k = kstart; k < k1; ++k) {
        const bool own = k >= k0;
        const bool slow = xy_pml || (P > 0 && (k <= P || k >= g.nz - P)) ||
                          (src_xy && k >= A.ss.klo && k <= A.ss.khi);
        if (slow)
            plane<true>(A, k, own, lane, i, j0, colok, lane_owns, cofs, ex0, ey0, hxp, hyp);
        else
            plane<false>(A, k, own, lane, i, j0, colok, lane_owns, cofs, ex0, ey0, hxp, hyp);
    }
}

struct HostState {
    int bx, by, chunks, chunk;
};

}  // namespace

const char *strip_name() { return "fused-strip-30x8"; }

int strip_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    // 32-bit offsets inside one component array
    if ((unsigned long long)g.comp >= (1ull << 32)) return FDTD_ERR_ARG;
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
    Args a;
    a.g = h->g;
    a.ein = h->fields[h->cur];
    a.eout = h->fields[h->cur ^ 1];
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
