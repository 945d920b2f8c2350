// kernels_basic.cu -- the unfused field update (one H sweep, one E sweep) and
// the small kernels every path shares: Mur faces, detector readout, field
// copies, energy/stability reduction.
//
// The H sweep reads E^n, H^{n-1/2} from set `cur` and writes H^{n+1/2} to set
// `cur^1`; the E sweep reads E^n from `cur` and H^{n+1/2} from `cur^1` and writes
// E^{n+1} to `cur^1` (Yee leapfrog, Sec. III.A; curl differences as in the
// paper's central-difference scheme).  One thread updates the up-to-six
// components owned by one cell (i,j,k), 0 <= i < nx etc.:
//   Hx(i,j+1/2,k+1/2) i>=1   Hy(i+1/2,j,k+1/2) j>=1   Hz(i+1/2,j+1/2,k) k>=1
//   Ex(i+1/2,j,k) j,k>=1     Ey(i,j+1/2,k) i,k>=1     Ez(i,j,k+1/2) i,j>=1
// Cells at i = 0 skip the components that lie on the x = 0 face (tangential
// E, boundary owned) and the H normal to it (it drives no updated E); the
// far faces i = nx etc. are never touched by the sweeps.
#include <cuda_runtime.h>
#include <math.h>

#include "cell_update.cuh"
#include "fdtd_internal.h"
#include "source_term.cuh"

namespace fdtd {

__global__ void __launch_bounds__(256) k_update_h(Grid g, const float *__restrict__ Ein,
                                                  const float *__restrict__ Hin,
                                                  float *__restrict__ Hout, Cpml pml, float kH) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    cell_h(g, Ein, Hin, Hout, pml, kH, i, j, k);
}

__global__ void __launch_bounds__(256) k_update_e(Grid g, const float *__restrict__ Ein,
                                                  const float *__restrict__ Hnew,
                                                  float *__restrict__ Eout, Cpml pml, float kE,
                                                  Source src, long long n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    cell_e(g, Ein, Hnew, Eout, pml, kE, src, n, i, j, k);
}

void launch_update_h(const fdtd_ctx *h, cudaStream_t s) {
    const Grid &g = h->g;
    dim3 blk(32, 8, 1), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    k_update_h<<<grd, blk, 0, s>>>(g, in, in + 3 * g.comp, out + 3 * g.comp, cpml_view(h), (float)h->kH);
}

void launch_update_e(const fdtd_ctx *h, cudaStream_t s) {
    const Grid &g = h->g;
    dim3 blk(32, 8, 1), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    const float *in = h->fields[h->cur];
    float *out = h->fields[h->cur ^ 1];
    k_update_e<<<grd, blk, 0, s>>>(g, in, out + 3 * g.comp, out, cpml_view(h), (float)h->kE, h->src, h->steps);
}

__global__ void k_mur(Grid g, const float *__restrict__ Eold, float *__restrict__ Enew, float m) {
    mur_cell(g, Eold, Enew, m, blockIdx.z, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

void launch_mur(const fdtd_ctx *h, cudaStream_t s) {
    const Grid &g = h->g;
    int amax = (g.nx > g.ny ? g.nx : g.ny) + 1;
    int bmax = (g.ny > g.nz ? g.ny : g.nz) + 1;
    if (g.nz + 1 > bmax) bmax = g.nz + 1;
    dim3 blk(32, 8, 1), grd((amax + 31) / 32, (bmax + 7) / 8, 6);
    k_mur<<<grd, blk, 0, s>>>(g, h->fields[h->cur], h->fields[h->cur ^ 1], (float)h->mur_m);
}

// Readout of detector t into trace slot `slot` from the six E values around
// its node: Ex at i-1, i; Ey at j-1, j; Ez at k-1, k (node averages); E_r
// about the shower axis.
__device__ __forceinline__ void readout(const Probes &p, int t, long long slot, const float *v) {
    float ex = 0.5f * (v[0] + v[1]);
    float ey = 0.5f * (v[2] + v[3]);
    float ez = 0.5f * (v[4] + v[5]);
    float er = p.cxy[2 * t] * ex + p.cxy[2 * t + 1] * ey;
    float *o = p.trace + ((long long)t * p.max_steps + slot) * 2;
    o[0] = ez;
    o[1] = er;
}

__device__ __forceinline__ void readout_fields(const Grid &g, const float *E, const Probes &p, int t,
                                               long long slot) {
    const int i = p.ijk[3 * t], j = p.ijk[3 * t + 1], k = p.ijk[3 * t + 2];
    const long long c = gidx(g, i, j, k);
    const float *Ex = E, *Ey = E + g.comp, *Ez = E + 2 * g.comp;
    const float v[6] = {Ex[c - 1], Ex[c], Ey[c - g.pitch], Ey[c], Ez[c - g.plane], Ez[c]};
    readout(p, t, slot, v);
}

// Detector readout of E^{n+1} (set cur^1) into trace slot n.
__global__ void k_probes(Grid g, const float *__restrict__ E, Probes p, long long slot) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n) return;
    readout_fields(g, E, p, t, slot);
}

// After a two-step pass: slot n from the pass's records of E^{n+1} (six
// values per detector), slot n+1 from E^{n+2} (set cur^1).
__global__ void k_probes2(Grid g, const float *__restrict__ E, Probes p, long long slot,
                          const float *__restrict__ rec) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n) return;
    float v[6];
    for (int s = 0; s < 6; ++s) v[s] = rec[6 * t + s];
    readout(p, t, slot, v);
    readout_fields(g, E, p, t, slot + 1);
}

void launch_probes(const fdtd_ctx *h, cudaStream_t s) {
    Probes p{h->np, h->max_steps, h->d_ijk, h->d_cxy, h->d_trace};
    k_probes<<<(h->np + 127) / 128, 128, 0, s>>>(h->g, h->fields[h->cur ^ 1], p, h->steps);
}

void launch_tb2_probes(fdtd_ctx *h, cudaStream_t s) {
    Probes p{h->np, h->max_steps, h->d_ijk, h->d_cxy, h->d_trace};
    const float *rec = tb2_probe_values(h);
    if (!rec) return;
    k_probes2<<<(h->np + 127) / 128, 128, 0, s>>>(h->g, h->fields[h->cur ^ 1], p, h->steps, rec);
}

// Watchdog of the step path: block (x, y) scans plane k = min(y * stride,
// nz) of the six components in chunks of 4 floats per thread; a non-finite
// value anywhere sets flag bit 2.  An instability, or a non-finite value put
// into any cell, spreads one plane per step (each Yee half step couples
// neighbouring planes only), so it reaches a sampled plane within stride / 2
// steps.
__global__ void __launch_bounds__(256) k_watch(Grid g, const float *__restrict__ f, int stride, int *flags) {
    const int k = min((int)blockIdx.y * stride, g.nz);
    const long long n4 = g.plane / 4;   // plane is a multiple of 32 floats
    bool bad = false;
    for (int c = 0; c < 6; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f + c * g.comp + (long long)k * g.plane);
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n4;
             t += (long long)gridDim.x * blockDim.x) {
            const float4 v = p[t];
            bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, FLAG_UNSTABLE);
}

void launch_watch(const fdtd_ctx *h, cudaStream_t s) {
    const Grid &g = h->g;
    const int planes = (g.nz + WATCH_STRIDE - 1) / WATCH_STRIDE + 1;
    const long long n4 = g.plane / 4;
    const int bx = (int)((n4 + 255) / 256 < 8 ? (n4 + 255) / 256 : 8);
    k_watch<<<dim3(bx, planes), 256, 0, s>>>(g, h->fields[h->cur], WATCH_STRIDE, h->d_flags);
}

// ---- field copies -----------------------------------------------------------

// Whether node-grid entry (i,j,k) of component c is state the update keeps.
__device__ __forceinline__ bool kept(const Grid &g, int c, int i, int j, int k, bool mur) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    switch (c) {
    case 0: {
        if (i > nx - 1) return false;
        bool jin = j >= 1 && j <= ny - 1, kin = k >= 1 && k <= nz - 1;
        return (jin && kin) || (mur && (jin || kin));
    }
    case 1: {
        if (j > ny - 1) return false;
        bool iin = i >= 1 && i <= nx - 1, kin = k >= 1 && k <= nz - 1;
        return (iin && kin) || (mur && (iin || kin));
    }
    case 2: {
        if (k > nz - 1) return false;
        bool iin = i >= 1 && i <= nx - 1, jin = j >= 1 && j <= ny - 1;
        return (iin && jin) || (mur && (iin || jin));
    }
    case 3: return i >= 1 && i <= nx - 1 && j <= ny - 1 && k <= nz - 1;
    case 4: return i <= nx - 1 && j >= 1 && j <= ny - 1 && k <= nz - 1;
    default: return i <= nx - 1 && j <= ny - 1 && k >= 1 && k <= nz - 1;
    }
}

__global__ void k_set_field(Grid g, int c, const float *__restrict__ in, float *__restrict__ f,
                            bool mur) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, k = blockIdx.z;
    if (i > g.nx) return;
    long long s = ((long long)k * (g.ny + 1) + j) * (g.nx + 1) + i;
    f[c * g.comp + gidx(g, i, j, k)] = kept(g, c, i, j, k, mur) ? in[s] : 0.0f;
}

__global__ void k_get_field(Grid g, int c, const float *__restrict__ f, float *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, k = blockIdx.z;
    if (i > g.nx) return;
    long long s = ((long long)k * (g.ny + 1) + j) * (g.nx + 1) + i;
    out[s] = f[c * g.comp + gidx(g, i, j, k)];
}

void launch_set_field(const fdtd_ctx *h, int comp, const float *compact, cudaStream_t s) {
    const Grid &g = h->g;
    dim3 blk(128), grd((g.nx + 1 + 127) / 128, g.ny + 1, g.nz + 1);
    k_set_field<<<grd, blk, 0, s>>>(g, comp, compact, h->fields[h->cur], h->boundary == FDTD_MUR1);
}

void launch_get_field(const fdtd_ctx *h, int comp, float *compact, cudaStream_t s) {
    const Grid &g = h->g;
    dim3 blk(128), grd((g.nx + 1 + 127) / 128, g.ny + 1, g.nz + 1);
    k_get_field<<<grd, blk, 0, s>>>(g, comp, h->fields[h->cur], compact);
}

// ---- energy / stability -----------------------------------------------------
// Pass 1: each block sums E^2 and H^2 (FP64) and counts non-finite values over a
// grid-stride range of the six arrays (entries the update does not keep are
// zero) into partial[3*block].  Pass 2: one block folds the partials.

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_energy_partial(const float4 *__restrict__ f,
                                                        long long comp4, double *partial) {
    double se = 0.0, sh = 0.0, bad = 0.0;
    long long total = 6 * comp4;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        float4 v = f[t];
        double s = (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
        if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w)) bad += 1.0;
        if (t < 3 * comp4) se += s; else sh += s;
    }
    __shared__ double red[3][8];
    se = warp_sum(se); sh = warp_sum(sh); bad = warp_sum(bad);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = se; red[1][w] = sh; red[2][w] = bad; }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        double a = l < nw ? red[0][l] : 0.0, b = l < nw ? red[1][l] : 0.0, c = l < nw ? red[2][l] : 0.0;
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (l == 0) {
            partial[3 * blockIdx.x] = a;
            partial[3 * blockIdx.x + 1] = b;
            partial[3 * blockIdx.x + 2] = c;
        }
    }
}

__global__ void __launch_bounds__(256) k_energy_final(const double *partial, int nblk, double *out) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        a += partial[3 * t]; b += partial[3 * t + 1]; c += partial[3 * t + 2];
    }
    __shared__ double red[3][8];
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = c; }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        a = l < nw ? red[0][l] : 0.0; b = l < nw ? red[1][l] : 0.0; c = l < nw ? red[2][l] : 0.0;
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (l == 0) { out[0] = a; out[1] = b; out[2] = c; }
    }
}

void launch_energy(const fdtd_ctx *h, cudaStream_t s, int *launches) {
    const float4 *f = reinterpret_cast<const float4 *>(h->fields[h->cur]);
    k_energy_partial<<<h->partial_cap, 256, 0, s>>>(f, h->g.comp / 4, h->d_partial);
    k_energy_final<<<1, 256, 0, s>>>(h->d_partial, h->partial_cap, h->d_result);
    *launches = 2;
}

}  // namespace fdtd
