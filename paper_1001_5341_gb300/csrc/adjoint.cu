// adjoint.cu -- transposed steps and the gradient of a detector misfit with
// respect to the shower's charge table (PEC grids without CPML).
//
// The step of Sec. III.A maps u^n = (E^n, H^{n-1/2}) to u^{n+1} linearly:
//   H' = H - kH C_E E,   E' = E + kE C_H H' + S^n,
// with C_E the forward-difference curl and C_H the backward-difference curl.
// On the Yee grid with PEC walls C_H = C_E^T entry by entry, so the transpose
// of the step, acting on the adjoint state mu = (mu_E, mu_H), is again a
// leapfrog:
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
    const double kE = h->kE, kH = h->kH;
    const int active = h->src.active;
    h->kE = -kH;
    h->kH = -kE;
    h->src.active = 0;
    switch (h->kernel) {
    case 1: launch_vtile(h, h->stream); h->launches++; break;
    case 2: launch_fused(h, h->stream); h->launches++; break;
    case 3: launch_strip(h, h->stream); h->launches++; break;
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

bool adjoint_ok(const fdtd_ctx *h) { return h->boundary == FDTD_PEC && h->P == 0; }

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
    h->cur = 0;
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
    h->cur = 0;
    h->steps = 0;
    if (rc == FDTD_OK && !on_device)
        rc = note(h, cudaMemcpyAsync(grad_q, dgrad, sizeof(double) * h->src.nbins, cudaMemcpyDeviceToHost, h->stream));
    if (rc == FDTD_OK) rc = note(h, cudaStreamSynchronize(h->stream));
    cudaFree(gstep);
    if (dgrad) cudaFree(dgrad);
    return rc;
}

}  // extern "C"
