// cell_update.cuh -- the per-cell field updates of one step (Yee leapfrog,
// Sec. III.A), shared by the unfused sweeps and the batched persistent kernel.
//
// One call updates the up-to-six components owned by one cell (i,j,k),
// 0 <= i < nx etc.:
//   Hx(i,j+1/2,k+1/2) i>=1   Hy(i+1/2,j,k+1/2) j>=1   Hz(i+1/2,j+1/2,k) k>=1
//   Ex(i+1/2,j,k) j,k>=1     Ey(i,j+1/2,k) i,k>=1     Ez(i,j,k+1/2) i,j>=1
// Cells at i = 0 skip the components that lie on the x = 0 face (tangential
// E, boundary owned) and the H normal to it (it drives no updated E); the far
// faces i = nx etc. are never touched.
#pragma once

#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {

// psi^{new} = b psi + a d; the derivative d gains psi^{new}.
__device__ __forceinline__ void cpml_inplace(float *psi, const float *a, const float *b, int pos,
                                             float &d) {
    float p = b[pos] * (*psi) + a[pos] * d;
    *psi = p;
    d = d + p;
}
__device__ __forceinline__ void cpml_pingpong(const float *pin, float *pout, const float *a,
                                              const float *b, int pos, float &d) {
    float p = b[pos] * (*pin) + a[pos] * d;
    *pout = p;
    d = d + p;
}

// H^{n+1/2} of the components owned by cell (i,j,k).
// Ein: Ex (Ey, Ez follow at +comp); Hin, Hout: Hx (Hy, Hz follow at +comp).
__device__ __forceinline__ void cell_h(const Grid &g, const float *__restrict__ Ein,
                                       const float *__restrict__ Hin, float *__restrict__ Hout,
                                       const Cpml &pml, float kH, int i, int j, int k) {
    const float *Ex = Ein, *Ey = Ein + g.comp, *Ez = Ein + 2 * g.comp;
    long long c = gidx(g, i, j, k);
    const int P = pml.P, W = pml.W;
    int lx = psi_x_pos(i, g.nx, P), ly = slab_cell(j, g.ny, P), lz = slab_cell(k, g.nz, P);
    if (i >= 1) {  // Hx
        float dy = Ez[c + g.pitch] - Ez[c];
        float dz = Ey[c + g.plane] - Ey[c];
        if (ly >= 0) { long long q = psi_y(g, W, i, ly, k); cpml_pingpong(pml.hin[1][0] + q, pml.hout[1][0] + q, pml.aH[1], pml.bH[1], j, dy); }
        if (lz >= 0) { long long q = psi_z(g, W, i, j, lz); cpml_pingpong(pml.hin[2][0] + q, pml.hout[2][0] + q, pml.aH[2], pml.bH[2], k, dz); }
        Hout[c] = Hin[c] - kH * (dy - dz);
    }
    if (j >= 1) {  // Hy
        float dz = Ex[c + g.plane] - Ex[c];
        float dx = Ez[c + 1] - Ez[c];
        if (lz >= 0) { long long q = psi_z(g, W, i, j, lz); cpml_pingpong(pml.hin[2][1] + q, pml.hout[2][1] + q, pml.aH[2], pml.bH[2], k, dz); }
        if (lx >= 0) { long long q = psi_x(g, P, lx, j, k); cpml_pingpong(pml.hin[0][0] + q, pml.hout[0][0] + q, pml.aH[0], pml.bH[0], i, dx); }
        Hout[g.comp + c] = Hin[g.comp + c] - kH * (dz - dx);
    }
    if (k >= 1) {  // Hz
        float dx = Ey[c + 1] - Ey[c];
        float dy = Ex[c + g.pitch] - Ex[c];
        if (lx >= 0) { long long q = psi_x(g, P, lx, j, k); cpml_pingpong(pml.hin[0][1] + q, pml.hout[0][1] + q, pml.aH[0], pml.bH[0], i, dx); }
        if (ly >= 0) { long long q = psi_y(g, W, i, ly, k); cpml_pingpong(pml.hin[1][1] + q, pml.hout[1][1] + q, pml.aH[1], pml.bH[1], j, dy); }
        Hout[2 * g.comp + c] = Hin[2 * g.comp + c] - kH * (dx - dy);
    }
}

// E^{n+1} of the components owned by cell (i,j,k).
// Ein, Eout: Ex of sets cur / cur^1; Hnew: Hx of set cur^1.
__device__ __forceinline__ void cell_e(const Grid &g, const float *__restrict__ Ein,
                                       const float *__restrict__ Hnew, float *__restrict__ Eout,
                                       const Cpml &pml, float kE, const Source &src, long long n,
                                       int i, int j, int k) {
    const float *Hx = Hnew, *Hy = Hnew + g.comp, *Hz = Hnew + 2 * g.comp;
    long long c = gidx(g, i, j, k);
    const int P = pml.P, W = pml.W;
    int lx = psi_x_pos(i, g.nx, P), ly = slab_cell(j, g.ny, P), lz = slab_cell(k, g.nz, P);
    if (j >= 1 && k >= 1) {  // Ex
        float dy = Hz[c] - Hz[c - g.pitch];
        float dz = Hy[c] - Hy[c - g.plane];
        if (ly >= 0) cpml_inplace(pml.e[1][0] + psi_y(g, W, i, ly, k), pml.aE[1], pml.bE[1], j, dy);
        if (lz >= 0) cpml_inplace(pml.e[2][0] + psi_z(g, W, i, j, lz), pml.aE[2], pml.bE[2], k, dz);
        Eout[c] = Ein[c] + kE * (dy - dz);
    }
    if (i >= 1 && k >= 1) {  // Ey
        float dz = Hx[c] - Hx[c - g.plane];
        float dx = Hz[c] - Hz[c - 1];
        if (lz >= 0) cpml_inplace(pml.e[2][1] + psi_z(g, W, i, j, lz), pml.aE[2], pml.bE[2], k, dz);
        if (lx >= 0) cpml_inplace(pml.e[0][0] + psi_x(g, P, lx, j, k), pml.aE[0], pml.bE[0], i, dx);
        Eout[g.comp + c] = Ein[g.comp + c] + kE * (dz - dx);
    }
    if (i >= 1 && j >= 1) {  // Ez
        float dx = Hy[c] - Hy[c - 1];
        float dy = Hx[c] - Hx[c - g.pitch];
        if (lx >= 0) cpml_inplace(pml.e[0][1] + psi_x(g, P, lx, j, k), pml.aE[0], pml.bE[0], i, dx);
        if (ly >= 0) cpml_inplace(pml.e[1][1] + psi_y(g, W, i, ly, k), pml.aE[1], pml.bE[1], j, dy);
        float e = Ein[2 * g.comp + c] + kE * (dx - dy);
        if (src.active) e += source_term(src, i, j, k, n);
        Eout[2 * g.comp + c] = e;
    }
}

// First-order Mur on the tangential E of face f (0..5 = x-, x+, y-, y+, z-, z+):
// E0^{n+1} = E1^n + m (E1^{n+1} - E0^n); edge entries are not touched (PEC).
__device__ __forceinline__ void mur_cell(const Grid &g, const float *__restrict__ Eold, float *__restrict__ Enew,
                                         float m, int f, int a, int b) {
    int ax = f >> 1, hi = f & 1;
    if (ax == 0) {  // (a, b) = (j, k)
        int i0 = hi ? g.nx : 0, i1 = hi ? g.nx - 1 : 1;
        if (a <= g.ny && b <= g.nz) {
            const long long o0 = gidx(g, i0, a, b), o1 = gidx(g, i1, a, b);
            if (a <= g.ny - 1 && b >= 1 && b <= g.nz - 1) {
                const float *eo = Eold + g.comp; float *en = Enew + g.comp;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
            if (a >= 1 && a <= g.ny - 1 && b <= g.nz - 1) {
                const float *eo = Eold + 2 * g.comp; float *en = Enew + 2 * g.comp;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
        }
    } else if (ax == 1) {  // (a, b) = (i, k)
        int j0 = hi ? g.ny : 0, j1 = hi ? g.ny - 1 : 1;
        if (a <= g.nx && b <= g.nz) {
            const long long o0 = gidx(g, a, j0, b), o1 = gidx(g, a, j1, b);
            if (a <= g.nx - 1 && b >= 1 && b <= g.nz - 1) {
                const float *eo = Eold; float *en = Enew;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
            if (a >= 1 && a <= g.nx - 1 && b <= g.nz - 1) {
                const float *eo = Eold + 2 * g.comp; float *en = Enew + 2 * g.comp;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
        }
    } else {  // (a, b) = (i, j)
        int k0 = hi ? g.nz : 0, k1 = hi ? g.nz - 1 : 1;
        if (a <= g.nx && b <= g.ny) {
            const long long o0 = gidx(g, a, b, k0), o1 = gidx(g, a, b, k1);
            if (a <= g.nx - 1 && b >= 1 && b <= g.ny - 1) {
                const float *eo = Eold; float *en = Enew;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
            if (a >= 1 && a <= g.nx - 1 && b <= g.ny - 1) {
                const float *eo = Eold + g.comp; float *en = Enew + g.comp;
                en[o0] = eo[o1] + m * (en[o1] - eo[o0]);
            }
        }
    }
}

}  // namespace fdtd
