// adjoint.cu -- transposed steps and the gradient of a detector misfit with
// respect to the shower's charge table (PEC, Mur and CPML grids).
//
// The step of Sec. III.A maps u^n = (E^n, H^{n-1/2}) to u^{n+1} linearly:
//   H' = H - kH C_E E,   E' = E + kE C_H H' + S^n,
// with C_E the forward-difference curl and C_H the backward-difference curl.
// On the Yee grid with PEC walls C_H = C_E^T entry by entry, so the transpose
// of the step, acting on the adjoint state mu = (mu_E, mu_H), is again a
// leapfrog (Mur grids: below):
//   mu_H' = mu_H + kE C_E mu_E,   mu_E' = mu_E - kH C_H mu_H',
// i.e. the forward field update with (kE, kH) replaced by (-kH, -kE), no
// source.  The traces y^{n} = C u^{n} (detector slot n-1) and the source S^n
// (linear in the charge table, Sec. III.B) are linear too, so for a loss L(y)
// with g = dL/dy the adjoint recursion
//   mu^n = M^T mu^{n+1} + C^T g^{n-1},   n = N .. 1   (mu^{N+1} = 0)
// gives dL/dS^{n-1} = mu_E^n, and from the deposit pattern of step n-1 the
// derivative with respect to the interpolated charge qbar^{n-1}, which the
// linear interpolation of the table spreads over two bins.  The recursion
// needs no forward state.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "cell_update.cuh"
#include "fdtd_internal.h"
#include "source_term.cuh"

using namespace fdtd;

namespace {

// C^T g: the transpose of the detector reading of k_probes (two-sample means
// of Ex, Ey, Ez around the node, E_r = X/r Ex + Y/r Ey), added to mu_E.
__global__ void k_adj_probes(Grid g, float *E, Probes p, const float *__restrict__ dl, int slot) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n) return;
    const int i = p.ijk[3 * t], j = p.ijk[3 * t + 1], k = p.ijk[3 * t + 2];
    const long long c = gidx(g, i, j, k);
    const float gz = dl[((long long)t * p.max_steps + slot) * 2];
    const float gr = dl[((long long)t * p.max_steps + slot) * 2 + 1];
    float *Ex = E, *Ey = E + g.comp, *Ez = E + 2 * g.comp;
    const float ax = 0.5f * p.cxy[2 * t] * gr, ay = 0.5f * p.cxy[2 * t + 1] * gr;
    atomicAdd(&Ez[c - g.plane], 0.5f * gz);
    atomicAdd(&Ez[c], 0.5f * gz);
    atomicAdd(&Ex[c - 1], ax);
    atomicAdd(&Ex[c], ax);
    atomicAdd(&Ey[c - g.pitch], ay);
    atomicAdd(&Ey[c], ay);
}

// dL/dqbar of step n: the sum over the footprint edges of mu_Ez times the E
// increment per unit qbar (the deposit pattern of source_term without qbar).
constexpr int ADJ_THREADS = 256;

__global__ void k_adj_source(Grid g, const float *__restrict__ E, Source s, SourceStep w, double *__restrict__ out) {
    const float *Ez = E + 2 * g.comp;
    const int side = 2 * s.L + 1;
    const int planes = w.khi >= w.klo ? w.khi - w.klo + 1 : 0;
    const long long n = w.n;
    const double za = s.z0 + s.v * (double)n * s.dt, zb = s.z0 + s.v * (double)(n + 1) * s.dt;
    const double ua = za / s.dx, ub = zb / s.dx;
    const double ka = floor(ua), kb = floor(ub);
    double acc = 0.0;
    for (int e = threadIdx.x; e < side * side * planes; e += ADJ_THREADS) {
        const int k = w.klo + e / (side * side);
        const int r = e % (side * side);
        const int dj = r / side - s.L, di = r % side - s.L;
        if (k < s.kmin || k > s.kmax) continue;
        const double ca = (double)k < ka ? 0.0 : ((double)k == ka ? 1.0 - (ua - ka) : 1.0);
        const double cb = (double)k < kb ? 0.0 : ((double)k == kb ? 1.0 - (ub - kb) : 1.0);
        const double dC = cb - ca;
        if (dC == 0.0) continue;
        const double pattern = s.w[r] * s.coef * dC;
        acc += pattern * (double)Ez[gidx(g, s.ic + di, s.jc + dj, k)];
    }
    // block reduction: warp shuffles, then one value per warp
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[ADJ_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < ADJ_THREADS / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[n] = v;
    }
}

// dL/dq_b: the per-step derivatives spread over the bins the way qbar of
// each step interpolates the table (one thread per bin, steps in order).
__global__ void k_adj_bins(Source s, const double *__restrict__ gstep, int n_steps, double *__restrict__ grad) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= s.nbins) return;
    double acc = 0.0;
    for (int n = 0; n < n_steps; ++n) {
        const double zm = s.z0 + s.v * ((double)n + 0.5) * s.dt;
        const double u = (zm - s.z0) / s.bin_dz;
        if (!(u >= 0.0) || u > (double)(s.nbins - 1)) continue;
        const int bb = (int)floor(u);
        if (bb >= s.nbins - 1) {
            if (b == s.nbins - 1) acc += gstep[n];
        } else if (b == bb) {
            acc += (1.0 - (u - bb)) * gstep[n];
        } else if (b == bb + 1) {
            acc += (u - bb) * gstep[n];
        }
    }
    grad[b] = acc;
}

// ---- Mur grids --------------------------------------------------------------
// The Mur step is  Etilde = E + kE C_H H' on the interior E cells (the cells
// cell_e updates), then  E'_b = E_1^n + m (Etilde_1 - E_b^n)  on each face cell
// b (tangential E of a face, edges excluded) with inward neighbour 1.  Its
// transpose, from (mu_E', mu_H') in set cur to set cur^1:
//   1. muEt = mu_E' on interior cells plus m mu_E'_b from each face cell b
//      next to them; zero on face cells;
//   2. mu_H = mu_H' + kE C_E muEt                  (cell_h, coefficient -kE);
//   3. mu_E = muEt - kH C_H mu_H on interior cells (cell_e, coefficient -kH);
//   4. face cells: mu_E_b = -kH (C_E^T mu_H)_b - m mu_E'_b, and each inward
//      neighbour gains mu_E'_b.
// (C_E^T mu_H)_b is the backward-difference curl at b with H outside the
// grid taken as zero (H cells the step does not update hold zero).

// whether E component c at node (i,j,k) is updated by cell_e
__device__ __forceinline__ bool e_interior(const Grid &g, int c, int i, int j, int k) {
    const bool xi = i >= 1 && i <= g.nx - 1, yi = j >= 1 && j <= g.ny - 1, zi = k >= 1 && k <= g.nz - 1;
    if (c == 0) return i <= g.nx - 1 && yi && zi;
    if (c == 1) return j <= g.ny - 1 && xi && zi;
    return k <= g.nz - 1 && xi && yi;
}

__global__ void k_adj_mur_gather(Grid g, const float *__restrict__ Ein, float *__restrict__ Et, float m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i > g.nx) return;
    const long long o = gidx(g, i, j, k);
    for (int c = 0; c < 3; ++c) {
        const float *e = Ein + c * g.comp;
        float v = 0.f;
        if (e_interior(g, c, i, j, k)) {
            v = e[o];
            // face neighbours: the component must be tangential to the face
            if (c != 0) {
                if (i == 1) v += m * e[o - 1];
                if (i == g.nx - 1) v += m * e[o + 1];
            }
            if (c != 1) {
                if (j == 1) v += m * e[o - g.pitch];
                if (j == g.ny - 1) v += m * e[o + g.pitch];
            }
            if (c != 2) {
                if (k == 1) v += m * e[o - g.plane];
                if (k == g.nz - 1) v += m * e[o + g.plane];
            }
        }
        Et[c * g.comp + o] = v;
    }
}

__global__ void __launch_bounds__(256) k_adj_h(Grid g, const float *__restrict__ Et, const float *__restrict__ Hin,
                                               float *__restrict__ Hout, Cpml pml, float kH) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    cell_h(g, Et, Hin, Hout, pml, kH, i, j, k);
}

__global__ void __launch_bounds__(256) k_adj_e(Grid g, float *E, const float *__restrict__ H, Cpml pml, float kE,
                                               Source src) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    cell_e(g, E, H, E, pml, kE, src, 0, i, j, k);   // in place: each cell reads and writes only itself
}

__device__ __forceinline__ float hval(const Grid &g, const float *Hc, int i, int j, int k) {
    return (i < 0 || j < 0 || k < 0) ? 0.f : Hc[gidx(g, i, j, k)];
}

// Face f (0..5 = x-, x+, y-, y+, z-, z+), tangential components, (a, b) as mur_cell.
__global__ void k_adj_mur_faces(Grid g, const float *__restrict__ Ein, float *E, const float *__restrict__ H,
                                float kH, float m) {
    const int f = blockIdx.z, ax = f >> 1, hi = f & 1;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
    const float *Hx = H, *Hy = H + g.comp, *Hz = H + 2 * g.comp;
    for (int t = 0; t < 2; ++t) {
        // component c on face f and its index range (as in mur_cell)
        int c, i, j, k, di = 0, dj = 0, dk = 0;
        bool ok;
        if (ax == 0) {
            c = t == 0 ? 1 : 2;
            i = hi ? g.nx : 0; j = a; k = b; di = hi ? -1 : 1;
            ok = c == 1 ? (a <= g.ny - 1 && b >= 1 && b <= g.nz - 1) : (a >= 1 && a <= g.ny - 1 && b <= g.nz - 1);
        } else if (ax == 1) {
            c = t == 0 ? 0 : 2;
            i = a; j = hi ? g.ny : 0; k = b; dj = hi ? -1 : 1;
            ok = c == 0 ? (a <= g.nx - 1 && b >= 1 && b <= g.nz - 1) : (a >= 1 && a <= g.nx - 1 && b <= g.nz - 1);
        } else {
            c = t == 0 ? 0 : 1;
            i = a; j = b; k = hi ? g.nz : 0; dk = hi ? -1 : 1;
            ok = c == 0 ? (a <= g.nx - 1 && b >= 1 && b <= g.ny - 1) : (a >= 1 && a <= g.nx - 1 && b <= g.ny - 1);
        }
        if (!ok) continue;
        float curl;
        if (c == 0)
            curl = (hval(g, Hz, i, j, k) - hval(g, Hz, i, j - 1, k)) - (hval(g, Hy, i, j, k) - hval(g, Hy, i, j, k - 1));
        else if (c == 1)
            curl = (hval(g, Hx, i, j, k) - hval(g, Hx, i, j, k - 1)) - (hval(g, Hz, i, j, k) - hval(g, Hz, i - 1, j, k));
        else
            curl = (hval(g, Hy, i, j, k) - hval(g, Hy, i - 1, j, k)) - (hval(g, Hx, i, j, k) - hval(g, Hx, i, j - 1, k));
        const long long o = gidx(g, i, j, k), o1 = gidx(g, i + di, j + dj, k + dk);
        const float eb = Ein[c * g.comp + o];
        E[c * g.comp + o] = -kH * curl - m * eb;
        atomicAdd(&E[c * g.comp + o1], eb);
    }
}

void adj_field_step_mur(fdtd_ctx *h) {
    const Grid &g = h->g;
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    const float m = (float)h->mur_m;
    Source none{};
    const Cpml pml = cpml_view(h);   // P = 0 on a Mur grid
    k_adj_mur_gather<<<dim3((g.nx + 1 + 127) / 128, g.ny + 1, g.nz + 1), 128, 0, h->stream>>>(g, in, out, m);
    const dim3 blk(32, 8, 1), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    k_adj_h<<<grd, blk, 0, h->stream>>>(g, out, in + 3 * g.comp, out + 3 * g.comp, pml, (float)-h->kE);
    k_adj_e<<<grd, blk, 0, h->stream>>>(g, out, out + 3 * g.comp, pml, (float)-h->kH, none);
    int amax = (g.nx > g.ny ? g.nx : g.ny) + 1;
    int bmax = (g.ny > g.nz ? g.ny : g.nz) + 1;
    if (g.nz + 1 > bmax) bmax = g.nz + 1;
    k_adj_mur_faces<<<dim3((amax + 31) / 32, (bmax + 7) / 8, 6), dim3(32, 8, 1), 0, h->stream>>>(
        g, in, out, out + 3 * g.comp, (float)h->kH, m);
    h->launches += 4;
    h->cur ^= 1;
}

// ---- CPML grids -------------------------------------------------------------
// A term of an update reads a difference d of one component along one axis;
// inside that axis' layer psi' = b psi + a d and the term becomes d + psi'.
// For an E term of sign s: Ec' += kE s (d + psi'); for an H term:
// Hc' -= kH s (d + psi').  With the adjoints mu (output) of the component and
// of psi', the adjoint of d is
//   E term:  G = kE s (1 + a) mu_E' + a mu_psi'
//   H term:  F = -kH s (1 + a) mu_H + a mu_psi'
// and the adjoint of the old psi is b (kE s mu_E' + mu_psi') (E) or
// b (-kH s mu_H + mu_psi') (H).  d is a backward difference of H for an E
// term (d = H(c) - H(c - off)) and a forward difference of E for an H term
// (d = E(c + off) - E(c)); its adjoint G (or F) at cell c is added to the
// component at c (at c + off) and subtracted at c - off (at c).
// Stage 1 (per cell, the three H components): mu_H = mu_H' + the G of every E
// term that reads it, then the adjoint of the H psi into the other psi set.
// Stage 2 (per node, the three E components): mu_E = mu_E' + the F of every H
// term that reads it, then the adjoint of the E psi in place.
struct Term {
    int comp;        // component the term differentiates (0..2 within E or H)
    int axis;        // axis of the difference (0 x, 1 y, 2 z)
    int sign;        // +1 first term of the curl, -1 second
    int psi;         // index t of the psi array of this axis
};
// terms of the E update (cell_e) and of the H update (cell_h), per component
__device__ __constant__ Term kETerms[3][2] = {{{2, 1, +1, 0}, {1, 2, -1, 0}},    // Ex: dy Hz, dz Hy
                                              {{0, 2, +1, 1}, {2, 0, -1, 0}},    // Ey: dz Hx, dx Hz
                                              {{1, 0, +1, 1}, {0, 1, -1, 1}}};   // Ez: dx Hy, dy Hx
__device__ __constant__ Term kHTerms[3][2] = {{{2, 1, +1, 0}, {1, 2, -1, 0}},    // Hx: dy Ez, dz Ey
                                              {{0, 2, +1, 1}, {2, 0, -1, 0}},    // Hy: dz Ex, dx Ez
                                              {{1, 0, +1, 1}, {0, 1, -1, 1}}};   // Hz: dx Ey, dy Ex

// psi offset of cell (i,j,k) in the layer of axis a, or -1 outside it
__device__ __forceinline__ long long psi_at(const Grid &g, const Cpml &pml, int a, int i, int j, int k) {
    if (a == 0) {
        const int l = psi_x_pos(i, g.nx, pml.P);
        return l < 0 ? -1 : psi_x(g, pml.P, l, j, k);
    }
    if (a == 1) {
        const int l = slab_cell(j, g.ny, pml.P);
        return l < 0 ? -1 : psi_y(g, pml.W, i, l, k);
    }
    const int l = slab_cell(k, g.nz, pml.P);
    return l < 0 ? -1 : psi_z(g, pml.W, i, j, l);
}

__device__ __forceinline__ bool e_updated(const Grid &g, int c, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) return false;
    return c == 0 ? (j >= 1 && k >= 1) : c == 1 ? (i >= 1 && k >= 1) : (i >= 1 && j >= 1);
}
__device__ __forceinline__ bool h_updated(const Grid &g, int c, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) return false;
    return c == 0 ? i >= 1 : c == 1 ? j >= 1 : k >= 1;
}

// G of E term (ec, t) at cell (i,j,k): from mu_E' (E set in) and mu_psiE'
__device__ __forceinline__ float g_term(const Grid &g, const Cpml &pml, const float *Ein, float kE, int ec, int t,
                                        int i, int j, int k) {
    if (!e_updated(g, ec, i, j, k)) return 0.f;
    const Term T = kETerms[ec][t];
    const long long o = gidx(g, i, j, k);
    const float mu = Ein[ec * g.comp + o];
    const long long q = psi_at(g, pml, T.axis, i, j, k);
    if (q < 0) return kE * T.sign * mu;
    const int pos = T.axis == 0 ? i : T.axis == 1 ? j : k;
    const float a = pml.aE[T.axis][pos];
    return kE * T.sign * (1.f + a) * mu + a * pml.e[T.axis][T.psi][q];
}

// F of H term (hc, t) at cell (i,j,k): from mu_H (H set out) and mu_psiH' (psi set in)
__device__ __forceinline__ float f_term(const Grid &g, const Cpml &pml, const float *Hout, float kH, int hc, int t,
                                        int i, int j, int k) {
    if (!h_updated(g, hc, i, j, k)) return 0.f;
    const Term T = kHTerms[hc][t];
    const long long o = gidx(g, i, j, k);
    const float mu = Hout[hc * g.comp + o];
    const long long q = psi_at(g, pml, T.axis, i, j, k);
    if (q < 0) return -kH * T.sign * mu;
    const int pos = T.axis == 0 ? i : T.axis == 1 ? j : k;
    const float a = pml.aH[T.axis][pos];
    return -kH * T.sign * (1.f + a) * mu + a * pml.hin[T.axis][T.psi][q];
}

__global__ void __launch_bounds__(256) k_adjc_h(Grid g, Cpml pml, const float *__restrict__ Ein,
                                                const float *__restrict__ Hin, float *__restrict__ Hout, float kE,
                                                float kH) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long o = gidx(g, i, j, k);
    for (int hc = 0; hc < 3; ++hc) {
        if (!h_updated(g, hc, i, j, k)) continue;
        float v = Hin[hc * g.comp + o];
        // E terms that read H_hc: a backward difference at c = h (+G) and at c = h + off (-G)
        for (int ec = 0; ec < 3; ++ec)
            for (int t = 0; t < 2; ++t) {
                const Term T = kETerms[ec][t];
                if (T.comp != hc) continue;
                const int di = T.axis == 0, dj = T.axis == 1, dk = T.axis == 2;
                v += g_term(g, pml, Ein, kE, ec, t, i, j, k) - g_term(g, pml, Ein, kE, ec, t, i + di, j + dj, k + dk);
            }
        Hout[hc * g.comp + o] = v;
        // adjoint of the old H psi: b (-kH s mu_H + mu_psi')
        for (int t = 0; t < 2; ++t) {
            const Term T = kHTerms[hc][t];
            const long long q = psi_at(g, pml, T.axis, i, j, k);
            if (q < 0) continue;
            const int pos = T.axis == 0 ? i : T.axis == 1 ? j : k;
            pml.hout[T.axis][T.psi][q] = pml.bH[T.axis][pos] * (-kH * T.sign * v + pml.hin[T.axis][T.psi][q]);
        }
    }
}

__global__ void __launch_bounds__(256) k_adjc_e(Grid g, Cpml pml, const float *__restrict__ Ein, float *__restrict__ Eout,
                                                const float *__restrict__ Hout, float kE, float kH) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (i > g.nx || j > g.ny) return;
    const long long o = gidx(g, i, j, k);
    for (int ec = 0; ec < 3; ++ec) {
        // state cells: PEC walls keep the tangential E of the faces at zero
        const bool state = ec == 0 ? (i <= g.nx - 1 && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz - 1)
                         : ec == 1 ? (j <= g.ny - 1 && i >= 1 && i <= g.nx - 1 && k >= 1 && k <= g.nz - 1)
                                   : (k <= g.nz - 1 && i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny - 1);
        if (!state) continue;
        float v = Ein[ec * g.comp + o];
        // H terms that read E_ec: a forward difference at c = e - off (+F) and at c = e (-F)
        for (int hc = 0; hc < 3; ++hc)
            for (int t = 0; t < 2; ++t) {
                const Term T = kHTerms[hc][t];
                if (T.comp != ec) continue;
                const int di = T.axis == 0, dj = T.axis == 1, dk = T.axis == 2;
                v += f_term(g, pml, Hout, kH, hc, t, i - di, j - dj, k - dk) - f_term(g, pml, Hout, kH, hc, t, i, j, k);
            }
        Eout[ec * g.comp + o] = v;
        // adjoint of the old E psi, in place: b (kE s mu_E' + mu_psi')
        if (!e_updated(g, ec, i, j, k)) continue;
        const float mu = Ein[ec * g.comp + o];
        for (int t = 0; t < 2; ++t) {
            const Term T = kETerms[ec][t];
            const long long q = psi_at(g, pml, T.axis, i, j, k);
            if (q < 0) continue;
            const int pos = T.axis == 0 ? i : T.axis == 1 ? j : k;
            float &p = pml.e[T.axis][T.psi][q];
            p = pml.bE[T.axis][pos] * (kE * T.sign * mu + p);
        }
    }
}

void adj_field_step_cpml(fdtd_ctx *h) {
    const Grid &g = h->g;
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    const Cpml pml = cpml_view(h);   // H psi: adjoint in from set cur, out to set cur^1
    const dim3 blk(32, 8, 1), gh((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz), ge((g.nx + 32) / 32, (g.ny + 8) / 8, g.nz + 1);
    k_adjc_h<<<gh, blk, 0, h->stream>>>(g, pml, in, in + 3 * g.comp, out + 3 * g.comp, (float)h->kE, (float)h->kH);
    k_adjc_e<<<ge, blk, 0, h->stream>>>(g, pml, in, out, out + 3 * g.comp, (float)h->kE, (float)h->kH);
    h->launches += 2;
    h->cur ^= 1;
}

int note(fdtd_ctx *h, cudaError_t e) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->status == FDTD_OK) h->status = FDTD_ERR_CUDA;
        return FDTD_ERR_CUDA;
    }
    return FDTD_OK;
}

// One transposed step on the current field set (result in the other set).
void adj_field_step(fdtd_ctx *h) {
    if (h->boundary == FDTD_MUR1) {
        adj_field_step_mur(h);
        return;
    }
    if (h->P > 0) {
        adj_field_step_cpml(h);
        return;
    }
    const double kE = h->kE, kH = h->kH;
    const int active = h->src.active;
    h->kE = -kH;
    h->kH = -kE;
    h->src.active = 0;
    switch (h->kernel) {
    case 1: launch_vtile(h, h->stream); h->launches++; break;
    default:
        launch_update_h(h, h->stream);
        launch_update_e(h, h->stream);
        h->launches += 2;
    }
    h->kE = kE;
    h->kH = kH;
    h->src.active = active;
    h->cur ^= 1;
}

bool adjoint_ok(const fdtd_ctx *h) { return h->boundary == FDTD_PEC || h->boundary == FDTD_MUR1 || h->boundary == FDTD_CPML; }

size_t field_bytes(const fdtd_ctx *h) { return 6 * (size_t)h->g.comp * sizeof(float); }

}  // namespace

extern "C" {

int fdtd_adjoint_step(fdtd_t h, int n) {
    if (!h || n < 0) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (!adjoint_ok(h)) return FDTD_ERR_ARG;
    for (int s = 0; s < n; ++s) adj_field_step(h);
    return note(h, cudaGetLastError());
}

int fdtd_adjoint_gradient(fdtd_t h, const float *dl_dtrace, int n_steps, double *grad_q, int on_device) {
    if (!h || !dl_dtrace || !grad_q || n_steps < 1) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (!adjoint_ok(h) || !h->src.active || h->np < 1 || n_steps > h->max_steps) return FDTD_ERR_ARG;
    double *gstep = nullptr, *dgrad = nullptr;
    if (cudaMalloc(&gstep, sizeof(double) * n_steps) != cudaSuccess ||
        (!on_device && cudaMalloc(&dgrad, sizeof(double) * h->src.nbins) != cudaSuccess)) {
        cudaGetLastError();
        if (gstep) cudaFree(gstep);
        return FDTD_ERR_OOM;
    }
    double *out = on_device ? grad_q : dgrad;
    int rc = FDTD_OK;
    for (int s = 0; s < 2 && rc == FDTD_OK; ++s)
        rc = note(h, cudaMemsetAsync(h->fields[s], 0, field_bytes(h), h->stream));
    if (h->psi_block && rc == FDTD_OK)
        rc = note(h, cudaMemsetAsync(h->psi_block, 0, h->psi_floats * sizeof(float), h->stream));
    h->cur = 0;
    h->ecur = 0;
    const Probes p{h->np, h->max_steps, h->d_ijk, h->d_cxy, h->d_trace};
    for (int n = n_steps; n >= 1 && rc == FDTD_OK; --n) {
        if (n < n_steps) adj_field_step(h);   // mu^n = M^T mu^{n+1}
        float *E = h->fields[h->cur];
        k_adj_probes<<<(h->np + 127) / 128, 128, 0, h->stream>>>(h->g, E, p, dl_dtrace, n - 1);
        const SourceStep w = source_window(h->src, n - 1);
        k_adj_source<<<1, ADJ_THREADS, 0, h->stream>>>(h->g, E, h->src, w, gstep);
        h->launches += 2;
        rc = note(h, cudaGetLastError());
    }
    if (rc == FDTD_OK) {
        k_adj_bins<<<(h->src.nbins + 127) / 128, 128, 0, h->stream>>>(h->src, gstep, n_steps, out);
        h->launches++;
        rc = note(h, cudaGetLastError());
    }
    // the adjoint state used the field memory: leave the handle reset
    for (int s = 0; s < 2 && rc == FDTD_OK; ++s)
        rc = note(h, cudaMemsetAsync(h->fields[s], 0, field_bytes(h), h->stream));
    if (h->psi_block && rc == FDTD_OK)
        rc = note(h, cudaMemsetAsync(h->psi_block, 0, h->psi_floats * sizeof(float), h->stream));
    h->cur = 0;
    h->ecur = 0;
    h->steps = 0;
    if (rc == FDTD_OK && !on_device)
        rc = note(h, cudaMemcpyAsync(grad_q, dgrad, sizeof(double) * h->src.nbins, cudaMemcpyDeviceToHost, h->stream));
    if (rc == FDTD_OK) rc = note(h, cudaStreamSynchronize(h->stream));
    cudaFree(gstep);
    if (dgrad) cudaFree(dgrad);
    return rc;
}

}  // extern "C"
