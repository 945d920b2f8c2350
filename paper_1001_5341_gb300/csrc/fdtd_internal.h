// fdtd_internal.h -- device views and the handle of the GB300 FDTD library.
//
// Layout in HBM.  Each of the six components is a float32 array over the node
// grid (nz+1) x (ny+1) x pitch, x fastest, pitch = nx+1 rounded up to 32
// floats so that every x row starts on a 128-byte boundary.  Two complete
// sets of the six arrays exist (ping-pong): a step reads set `cur` and writes
// set `cur ^ 1`, so no kernel ever reads a value that the same step has
// already overwritten.
//
// CPML memory is kept only in the slabs.  Per axis there are four psi arrays
// (two for the E update, two for the H update) over the slab cells of that
// axis: cells 0..P and N-P..N-1 (W = 2P+1 cells), stored
//   x: [nz][ny][WX]   y: [nz][W][pitch]   z: [W][ny][pitch]   (WX: psi_x_row)
// so that consecutive threads along x touch consecutive floats; the y and z
// rows use the field pitch, so four consecutive columns from a multiple of
// four form one aligned 16-byte vector, and every row of every psi array is a
// multiple of 16 bytes (TMA-addressable).  Every psi array starts on a
// 128-byte boundary.  The E-update
// psi are updated in place by the one thread that owns the cell; the H-update
// psi are ping-ponged like the fields, because a tile of the fused kernel
// recomputes its neighbours' halo H and must read their psi before the update.
// The two-step kernel recomputes halo E as well, so it reads the E psi of one
// set and writes the other: there are two E psi sets, and `ecur` names the one
// holding the current values (the one-step paths update it in place).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/fdtd.h"

namespace fdtd {

struct Grid {
    int nx, ny, nz;
    int pitch;       // floats per x row
    long long plane; // floats per z plane = (ny+1) * pitch
    long long comp;  // floats per component = (nz+1) * plane
};

__host__ __device__ inline long long gidx(const Grid &g, int i, int j, int k) {
    return (long long)k * g.plane + (long long)j * g.pitch + i;
}

// slab cell index of cell i on an axis with N cells and P PML cells, or -1
__host__ __device__ inline int slab_cell(int i, int N, int P) {
    if (P <= 0) return -1;
    if (i <= P) return i;
    if (i >= N - P) return i - (N - P) + (P + 1);
    return -1;
}

// psi roles per axis a: e[a][0..1] and h*[a][0..1] are
//   x: (Ey, Ez) and (Hy, Hz) x-derivative terms
//   y: (Ex, Ez) and (Hx, Hz) y-derivative terms
//   z: (Ex, Ey) and (Hx, Hy) z-derivative terms
struct Cpml {
    int P, W;                 // depth, slab cells per axis (2P+1); P = 0: no CPML
    float *e[3][2];           // E-update psi, in place
    const float *hin[3][2];   // H-update psi at step n-1/2 (read)
    float *hout[3][2];        // H-update psi at step n+1/2 (written)
    const float *aE[3], *bE[3], *aH[3], *bH[3]; // per position index, length n_axis (+1)
};

// An x row holds the low layer's columns 0..P at positions 0..P and the high
// layer's columns N-P..N-1 at positions lo4 + (i - hb), lo4 = P+1 rounded up
// to 4 and hb = N-P rounded down to 4: four consecutive columns from a
// multiple of four sit at four consecutive positions from a multiple of four
// (one aligned 16-byte vector).  Rows are padded to a multiple of four.
__host__ __device__ inline int psi_x_lo4(int P) { return (P + 4) / 4 * 4; }
__host__ __device__ inline int psi_x_hb(int nx, int P) { return (nx - P) / 4 * 4; }
__host__ __device__ inline int psi_x_row(int nx, int P) {
    return (psi_x_lo4(P) + nx - psi_x_hb(nx, P) + 3) / 4 * 4;
}
// position of column i in an x row, or -1 outside the layers
__host__ __device__ inline int psi_x_pos(int i, int nx, int P) {
    if (P <= 0) return -1;
    if (i <= P) return i;
    if (i >= nx - P) return psi_x_lo4(P) + i - psi_x_hb(nx, P);
    return -1;
}
__host__ __device__ inline long long psi_x(const Grid &g, int P, int l, int j, int k) {
    return ((long long)k * g.ny + j) * psi_x_row(g.nx, P) + l;
}
__host__ __device__ inline long long psi_y(const Grid &g, int W, int i, int l, int k) {
    return ((long long)k * W + l) * g.pitch + i;
}
__host__ __device__ inline long long psi_z(const Grid &g, int W, int i, int j, int l) {
    return ((long long)l * g.ny + j) * g.pitch + i;
}

struct Source {
    int active;
    int L, ic, jc;
    int kmin, kmax;           // Ez edges k+1/2 that may carry current
    int nbins;
    double z0, v, dt, dx, bin_dz;
    double coef;              // 1 / (eps dx^2): E-increment per coulomb of charge crossing
    const double *q;          // profile samples
    const double *w;          // lateral weights (2L+1)^2
};

// window of planes whose Ez edges may carry the shower's current in step n
struct SourceStep {
    long long n;
    int klo, khi;
};

struct Probes {
    int n, max_steps;
    const int *ijk;           // [n][3]
    const float *cxy;         // [n][2]: X/r, Y/r about the axis (0,0 on the axis)
    float *trace;             // [n][max_steps][2]
};

struct TimingRec {
    std::vector<cudaEvent_t> ev; // start/stop pairs
    int used = 0;
    int cap = 0;
    bool on = false;
};

}  // namespace fdtd

struct fdtd_ctx {
    fdtd::Grid g;
    int boundary, P;
    double dx, dt, eps_r, eps, kE, kH, mur_m;
    cudaStream_t stream;
    int dev;

    float *fields[2];         // two sets, each 6 * g.comp floats
    int cur;                  // index of the set holding E^n, H^{n-1/2}

    // CPML
    float *psi_block;         // E psi, then two sets of H psi (one allocation)
    size_t psi_floats;        // total floats of psi_block
    float *epsi2;             // second E psi set (psi_floats / 3 floats)
    int ecur;                 // E psi set holding the current values (0: psi_block)
    size_t psi_axis[3];       // floats of one psi array of each axis
    float *coef_block;        // aE,bE,aH,bH per axis
    const float *aE[3], *bE[3], *aH[3], *bH[3];
    int kernel;               // field-update path: 0 unfused sweeps, 1 vector tile,
                              // 2 two steps per pass (vector tile for a last odd step)
    void *vtile;              // host state of the vector-tile path
    void *tb2;                // host state of the two-step path
    int *d_flags;             // device error flags (bits 0-1: a bounded wait gave up,
                              // bit 2: the watchdog saw a non-finite value)
    int watch_every;          // steps between watchdog checks (0: off)
    int num_sms;

    // source
    double *d_q;
    double *d_w;
    fdtd::Source src;

    // detectors
    int np, max_steps;
    int *d_ijk;
    float *d_cxy;
    float *d_trace;
    std::vector<int> h_ijk;
    int probe_ver;            // bumped by every fdtd_set_probes

    // energy / stability scratch
    double *d_partial;        // per-block partial sums
    int partial_cap;
    double *d_result;         // [3]: energy E, energy H, non-finite count

    int64_t steps;
    int64_t launches;
    int status;               // sticky error
    fdtd::TimingRec timing;
};

namespace fdtd {

// psi views of the current step (H psi read from set cur, written to cur^1)
Cpml cpml_view(const fdtd_ctx *h);

// kernels (kernels_basic.cu)
void launch_update_h(const fdtd_ctx *h, cudaStream_t s);
void launch_update_e(const fdtd_ctx *h, cudaStream_t s);
void launch_mur(const fdtd_ctx *h, cudaStream_t s);
void launch_probes(const fdtd_ctx *h, cudaStream_t s);
// watchdog: every component on every WATCH_STRIDE-th z plane (and the last)
// of the set holding the newest fields; sets flag bit 2 on a non-finite value
constexpr int WATCH_STRIDE = 8;
constexpr int FLAG_UNSTABLE = 4;
void launch_watch(const fdtd_ctx *h, cudaStream_t s);
void launch_energy(const fdtd_ctx *h, cudaStream_t s, int *launches);
void launch_set_field(const fdtd_ctx *h, int comp, const float *compact, cudaStream_t s);
void launch_get_field(const fdtd_ctx *h, int comp, float *compact, cudaStream_t s);

// TMA-staged vector-tile z-march over the whole grid, CPML included (kernels_vtile.cu)
int vtile_prepare(fdtd_ctx *h);
void launch_vtile(fdtd_ctx *h, cudaStream_t s);

// n steps of the handle's selected path on stream st (fdtd_step issues them
// on the handle's stream; a batch on its own).  Checks nothing beforehand.
int fdtd_step_on(fdtd_ctx *h, int n, cudaStream_t st);
const char *vtile_name();
void vtile_release(fdtd_ctx *h);

// Two leapfrog steps per pass (temporal blocking, kernels_tb2.cu): tiles of
// 8 rows and 32 lanes recompute a 2-cell halo of the first step; float4
// lanes (120 owned columns) between the x layers, scalar lanes (24 owned
// columns) over them
int tb2_prepare(fdtd_ctx *h);
void launch_tb2(fdtd_ctx *h, cudaStream_t s);          // steps n, n+1
void launch_tb2_probes(fdtd_ctx *h, cudaStream_t s);   // detector slots n, n+1 after launch_tb2
const char *tb2_name(const fdtd_ctx *h);
void tb2_release(fdtd_ctx *h);
float *tb2_probe_values(fdtd_ctx *h);   // the pass's records of E^{n+1} (6 per detector)

// host tables (tables.cpp)
void cpml_coefficients(int n, int P, double dx, double dt, double eps_r, float *aE, float *bE,
                       float *aH, float *bH);

}  // namespace fdtd
