// source_term.cuh -- the moving shower's current on one Ez edge (device).
#pragma once

#include "fdtd_internal.h"

namespace fdtd {

// E increment on edge (i, j, k+1/2) from the charge carried across it during
// step n (FP64, as the integer node index k0 = floor(z/dx) must be decided in
// the same precision as the reference arithmetic).
__device__ __forceinline__ float source_term(const Source &s, int i, int j, int k, long long n) {
    int di = i - s.ic, dj = j - s.jc;
    if (di < -s.L || di > s.L || dj < -s.L || dj > s.L || k < s.kmin || k > s.kmax) return 0.0f;
    double za = s.z0 + s.v * (double)n * s.dt;
    double zb = s.z0 + s.v * (double)(n + 1) * s.dt;
    // C_k(z): fraction of the charge on nodes <= k of the untruncated CIC line
    double ua = za / s.dx, ub = zb / s.dx;
    double ka = floor(ua), kb = floor(ub);
    double ca = (double)k < ka ? 0.0 : ((double)k == ka ? 1.0 - (ua - ka) : 1.0);
    double cb = (double)k < kb ? 0.0 : ((double)k == kb ? 1.0 - (ub - kb) : 1.0);
    double dC = cb - ca;
    if (dC == 0.0) return 0.0f;
    double zm = s.z0 + s.v * ((double)n + 0.5) * s.dt;
    double u = (zm - s.z0) / s.bin_dz;
    if (!(u >= 0.0) || u > (double)(s.nbins - 1)) return 0.0f;
    int b = (int)floor(u);
    double qbar = b >= s.nbins - 1 ? s.q[s.nbins - 1]
                                   : s.q[b] * (1.0 - (u - b)) + s.q[b + 1] * (u - b);
    double wij = s.w[(dj + s.L) * (2 * s.L + 1) + (di + s.L)];
    // -(dt/eps) J with J = -(dx/dt) qbar w dC / dx^3
    return (float)(qbar * wij * s.coef * dC);
}

// The planes k whose Ez edges may carry current during step n: a
// conservative window [klo, khi] around the charge's path (source_term
// decides each edge exactly).  Computed on the host per launch, or on the
// device per step by the persistent batch kernel.
__host__ __device__ inline SourceStep source_window(const Source &s, long long n) {
    SourceStep w;
    w.n = n;
    w.klo = 1;
    w.khi = 0;  // empty
    if (!s.active) return w;
    double za = s.z0 + s.v * (double)n * s.dt, zb = s.z0 + s.v * (double)(n + 1) * s.dt;
    double lo = za < zb ? za : zb, hi = za < zb ? zb : za;
    double klo = floor(lo / s.dx) - 2.0, khi = floor(hi / s.dx) + 2.0;
    if (khi < (double)s.kmin || klo > (double)s.kmax) return w;
    w.klo = klo < (double)s.kmin ? s.kmin : (int)klo;
    w.khi = khi > (double)s.kmax ? s.kmax : (int)khi;
    return w;
}

__device__ __forceinline__ float source_at(const Source &s, const SourceStep &w, int i, int j, int k) {
    if (!s.active || k < w.klo || k > w.khi) return 0.0f;
    return source_term(s, i, j, k, w.n);
}

}  // namespace fdtd
