// cyl.cu -- the paper's 2D axisymmetric FDTD (E_r, E_z, H_phi); the ABI and
// its conventions are in cyl.h.
//
// Storage: two sets (ping-pong) of three float32 arrays with nr+1 rows
// (radius) of `pitch` floats (z fastest).  Element (i, j) of a component sits
// at row i, position PADL + j; the PADL floats before column 0 and the floats
// after column nz are never written and stay zero, so that a warp may read a
// band of columns that starts left of column 0 or ends right of column nz.
// Cells outside a component's shape (E_r and H_phi on row nr, E_z and H_phi
// on column nz) are never written either.
//
// Two paths advance the fields:
//  * the two-kernel path (one H launch and one E launch per step, in place on
//    the current set; 36 bytes of DRAM per cell-update), which also runs the
//    steps that are left when a step count is not a multiple of K;
//  * the wavefront path (default): one launch advances K steps, reading the
//    current set once and writing the other set once (24 bytes per cell per
//    launch).  Each warp owns a band of z columns and marches up the rows of
//    one radial segment; time level s is computed one row behind level s-1,
//    all levels in registers, so that every input of a cell of level s (rows
//    r and r+1 of level s-1, row r-1 of level s, columns j-1..j+1 through warp
//    shuffles) is at hand.  A warp's columns overlap its neighbours' by K on
//    each side and its rows start K below its segment, so that the cells it
//    stores depend only on cells it computed.  Rows arrive in shared memory
//    through a ring of bulk asynchronous copies (TMA engine), STAGES rows
//    ahead, one mbarrier per stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/cyl.h"
#include "../../include/fdtd.h"

namespace {

constexpr double kC = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kPi = 3.14159265358979323846;
constexpr int PADL = 16;     // zero floats before column 0 (>= the widest left halo, 16-byte multiple)
constexpr int MSRC = 8;      // faces one step's deposit may touch (|v| dt / d <= 4)
constexpr int NW = 4;        // warps per block of the wavefront kernel
constexpr int LMAX = 1024;   // most rows per segment of the wavefront kernel
constexpr int TUNE_MAX = 48;  // most segment lengths cyl_tune tries
constexpr int NO_ROW = 0x3fffffff;   // detector row past the last one

// ---------------------------------------------------------------------------
// Source: q(z_s) linear in a bin table, cloud-in-cell along z.
// ---------------------------------------------------------------------------
struct Src {
    int active, nbins, nw;
    double z0, bin_dz, v, dt, d;
    const double *q;      // bin table (device)
    const float *coef;    // per ring: w_i / (eps A_i) (device)
};

__device__ __forceinline__ double src_q(const Src &s, double z) {
    const double x = (z - s.z0) / s.bin_dz;
    if (!(x >= 0.0) || x > (double)(s.nbins - 1)) return 0.0;
    int b = (int)floor(x);
    if (b > s.nbins - 2) b = s.nbins - 2;
    const double f = x - (double)b;
    return (1.0 - f) * s.q[b] + f * s.q[b + 1];
}

// cumulative cloud-in-cell weight of the nodes <= j of a unit charge at z
__device__ __forceinline__ double cum(double z, double d, int j) {
    const double x = z / d;
    const double jj = floor(x);
    const double f = x - jj;
    double c = 0.0;
    if ((double)j >= jj) c += 1.0 - f;
    if ((double)j >= jj + 1.0) c += f;
    return c;
}

// First face of the window of step n (n -> n+1); the deposit is zero outside
// jlo .. jlo + MSRC - 1.
__device__ __forceinline__ int src_jlo(const Src &s, long long n) {
    const double za = s.z0 + s.v * (double)n * s.dt, zb = s.z0 + s.v * (double)(n + 1) * s.dt;
    return (int)floor(fmin(za, zb) / s.d) - 1;
}

// qbar dC_j of step n at face j+1/2, to be scaled by coef[i] for ring i.
__device__ __forceinline__ float src_face(const Src &s, long long n, int j) {
    const double za = s.z0 + s.v * (double)n * s.dt, zb = s.z0 + s.v * (double)(n + 1) * s.dt;
    const double qb = src_q(s, s.z0 + s.v * ((double)n + 0.5) * s.dt);
    return (float)(qb * (cum(zb, s.d, j) - cum(za, s.d, j)));
}

struct Set {
    float *Er, *Ez, *Hp;   // element (0, 0) of each component
};

struct Dev {
    int nr, nz, pitch;
    Set f;
    const float2 *rowc;    // per row i: (cA_i, cB_i), E_z += cA_i H(i) - cB_i H(i-1)
};

// ---------------------------------------------------------------------------
// Two-kernel path
// ---------------------------------------------------------------------------
// nstep: index of the step being taken, advanced here so that a captured
// sequence of steps can be replayed (the E and detector kernels read it).
__global__ void k_cyl_h(Dev D, float kH, long long *nstep) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ++*nstep;
    if (i >= D.nr || j >= D.nz) return;
    const long long o = (long long)i * D.pitch + j;
    const float der = D.f.Er[o + 1] - D.f.Er[o];
    const float dez = D.f.Ez[o + D.pitch] - D.f.Ez[o];
    D.f.Hp[o] -= kH * (der - dez);
}

// E update of one step with the boundary: the thread of E_r(i, 1) also sets
// the cap E_r(i, 0), that of E_r(i, nz-1) the cap E_r(i, nz), that of
// E_z(nr-1, j) the wall E_z(nr, j) (first-order Mur from the old and new
// values next to them, or zero for PEC); no other thread of the launch reads
// or writes those cells.
__global__ void k_cyl_e(Dev D, float kE, float mur, int mur_on, Src S, const long long *nstep) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    const long long n = *nstep;
    const int nr = D.nr, nz = D.nz;
    if (i >= nr || j > nz) return;
    const long long o = (long long)i * D.pitch + j;
    float *Er = D.f.Er, *Ez = D.f.Ez;
    const float *Hp = D.f.Hp;
    if (j >= 1 && j <= nz - 1) {
        const float er0 = Er[o];
        const float er1 = er0 - kE * (Hp[o] - Hp[o - 1]);
        Er[o] = er1;
        if (j == 1) Er[o - 1] = mur_on ? er0 + mur * (er1 - Er[o - 1]) : 0.f;
        if (j == nz - 1) Er[o + 1] = mur_on ? er0 + mur * (er1 - Er[o + 1]) : 0.f;
    }
    if (j < nz) {
        const float ez0 = Ez[o];
        const float2 c = D.rowc[i];
        float ez1 = ez0 + c.x * Hp[o] - (i > 0 ? c.y * Hp[o - D.pitch] : 0.f);
        if (S.active && i < S.nw && (unsigned)(j - src_jlo(S, n)) < (unsigned)MSRC)
            ez1 += S.coef[i] * src_face(S, n, j);
        Ez[o] = ez1;
        if (i == nr - 1) Ez[o + D.pitch] = mur_on ? ez0 + mur * (ez1 - Ez[o + D.pitch]) : 0.f;
    }
}

__global__ void k_cyl_probes(Dev D, const int *ij, int np, float *trace, int max_steps, const long long *nstep) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const long long slot = *nstep;
    const int i = ij[2 * p], j = ij[2 * p + 1];
    const long long o = (long long)i * D.pitch + j;
    const float ez = 0.5f * (D.f.Ez[o - 1] + D.f.Ez[o]);
    const float er = i == 0 ? 0.f : 0.5f * (D.f.Er[o - D.pitch] + D.f.Er[o]);
    float *t = trace + ((long long)p * max_steps + slot) * 2;
    t[0] = ez;
    t[1] = er;
}

__global__ void k_cyl_copy(const float *src, int sp, float *dst, int dp, int rows, int cols) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (i < rows && j < cols) dst[(long long)i * dp + j] = src[(long long)i * sp + j];
}

// ---------------------------------------------------------------------------
// Wavefront path
// ---------------------------------------------------------------------------
struct Wave {
    int nr, nz, pitch;
    Set in, out;
    const float2 *rowc;
    float kE, kH, mur;
    int mur_on;
    int U, L, nbands;        // owned columns per band, rows per segment, bands
    Src src;
    long long n0;            // steps done before the launch
    const int *poff;         // per warp (segment-major): first detector record
    const int4 *prec;        // detector records (row, column, id, 0), sorted by warp then row
    float *trace;
    int max_steps;
    int *flags;
    unsigned *tiles;         // [0] next tile, [1] blocks done: zero at launch, the last block zeroes them
    int ntiles;              // segments x groups of NW bands
    int nseg;                // segments; the last one runs to the wall
};

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: gives up after about two seconds of clock cycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (4LL << 30)) return false;
    return true;
}
__device__ __forceinline__ void bulk_load(float *dst, const float *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(bar))
                 : "memory");
}

template <int CPL>
struct Row {
    float er[CPL], ez[CPL], h[CPL];
};

template <int CPL>
__device__ __forceinline__ void lds_row(Row<CPL> &r, const float *st, int lane) {
    constexpr int W = 32 * CPL;
    if constexpr (CPL == 2) {
        const float2 a = reinterpret_cast<const float2 *>(st)[lane];
        const float2 b = reinterpret_cast<const float2 *>(st + W)[lane];
        const float2 c = reinterpret_cast<const float2 *>(st + 2 * W)[lane];
        r.er[0] = a.x; r.er[1] = a.y;
        r.ez[0] = b.x; r.ez[1] = b.y;
        r.h[0] = c.x; r.h[1] = c.y;
    } else {
        static_assert(CPL == 4, "2 or 4 columns per lane");
        const float4 a = reinterpret_cast<const float4 *>(st)[lane];
        const float4 b = reinterpret_cast<const float4 *>(st + W)[lane];
        const float4 c = reinterpret_cast<const float4 *>(st + 2 * W)[lane];
        r.er[0] = a.x; r.er[1] = a.y; r.er[2] = a.z; r.er[3] = a.w;
        r.ez[0] = b.x; r.ez[1] = b.y; r.ez[2] = b.z; r.ez[3] = b.w;
        r.h[0] = c.x; r.h[1] = c.y; r.h[2] = c.z; r.h[3] = c.w;
    }
}

// n of the lane's CPL columns (a prefix) to global memory
template <int CPL>
__device__ __forceinline__ void st_cols(float *p, const float (&v)[CPL], int n) {
    if (n >= CPL) {
        if constexpr (CPL == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int q = 0; q < CPL; ++q)
            if (q < n) p[q] = v[q];
    }
}

// Per-warp march state: rows r - 1 (prv) and r (cur) of every time level in
// registers; the ring position; running offsets of the next row to fetch and
// of the next row to store.
template <int K, int CPL>
struct March {
    Row<CPL> prv[K + 1], cur[K + 1];
    int st;
    uint32_t phase;
    long long ld_off, st_off;
    int prowK;   // next detector row of level K
};

// Per-warp constants and shared-memory tables.
template <int K, int CPL>
struct Band {
    int lane, b, col0, p0, load_end, own0, own1, pfin;
    bool owned, cap_lo, cap_hi;
    float *ring;
    uint64_t *bar;
    const float2 *rowc;   // (cA, cB) of rows p0, p0 + 1, ...
    float *wall;          // [K][32 CPL]: the wall E_z of each level, one row ahead
    int *pc, *prow;       // [K + 1]: detector cursor and its row, per level
};

template <int CPL>
__device__ __forceinline__ void issue_row(const Wave &A, float *ring, uint64_t *bar, long long off, int st) {
    constexpr int W = 32 * CPL, STAGE = 3 * W;
    mbar_expect_tx(&bar[st], STAGE * 4);
    bulk_load(ring + st * STAGE, A.in.Er + off, W * 4, &bar[st]);
    bulk_load(ring + st * STAGE + W, A.in.Ez + off, W * 4, &bar[st]);
    bulk_load(ring + st * STAGE + 2 * W, A.in.Hp + off, W * 4, &bar[st]);
}

// One march step p: load row p (level 0), level s = 1..K computes row p - s,
// level K's row is stored.  FULL handles everything (rows before the segment
// or past the wall, the wall, the source rows, detectors, partial columns);
// the lean form (FULL = false) is taken only where none of that occurs, and
// CAPS adds the end-cap update for the warps that hold column 0 or nz.
template <int K, int CPL, int STAGES, bool FULL, bool CAPS>
__device__ __forceinline__ bool march_step(const Wave &A, const Band<K, CPL> &w, March<K, CPL> &S, int p,
                                           const int *sjlo, const float (*ssrc)[MSRC]) {
    constexpr int W = 32 * CPL, STAGE = 3 * W;
    const int nr = A.nr, nz = A.nz;
    S.prv[0] = S.cur[0];
    if (!FULL || p <= w.load_end) {
        if (!__all_sync(0xffffffffu, mbar_wait(&w.bar[S.st], S.phase))) return false;
        lds_row(S.cur[0], w.ring + S.st * STAGE, w.lane);
        // the warp's reads of the stage are ordered before the refill by the
        // warp barrier (the release/acquire a consumer barrier would give)
        __syncwarp();
        if (w.lane == 0 && p + STAGES <= w.load_end) issue_row<CPL>(A, w.ring, w.bar, S.ld_off, S.st);
        S.ld_off += A.pitch;
        if (++S.st == STAGES) {
            S.st = 0;
            S.phase ^= 1u;
        }
    }
#pragma unroll
    for (int s = 1; s <= K; ++s) {
        const int r = p - s;
        S.prv[s] = S.cur[s];
        if (FULL && (r < w.p0 || r > nr)) continue;
        const Row<CPL> &a = S.prv[s - 1];   // level s-1, row r
        const Row<CPL> &bn = S.cur[s - 1];  // level s-1, row r+1
        Row<CPL> &o = S.cur[s];
        if (!FULL || r < nr) {
            // H_phi(r, j) from E_r(r, j), E_r(r, j+1), E_z(r, j), E_z(r+1, j)
            const float er_right = __shfl_down_sync(0xffffffffu, a.er[0], 1);
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const float eR = q + 1 < CPL ? a.er[q + 1] : er_right;
                o.h[q] = a.h[q] - A.kH * ((eR - a.er[q]) - (bn.ez[q] - a.ez[q]));
            }
            // E_r(r, j) from H_phi(r, j-1), H_phi(r, j)
            const float h_left = __shfl_up_sync(0xffffffffu, o.h[CPL - 1], 1);
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const float hL = q > 0 ? o.h[q - 1] : h_left;
                o.er[q] = a.er[q] - A.kE * (o.h[q] - hL);
            }
            // E_z(r, j) from H_phi(r, j), H_phi(r-1, j); on the axis cB = 0
            const float2 c = w.rowc[r - w.p0];
#pragma unroll
            for (int q = 0; q < CPL; ++q) o.ez[q] = a.ez[q] + c.x * o.h[q] - c.y * S.prv[s].h[q];
            if (FULL && A.src.active && r < A.src.nw) {
                const float cf = __ldg(&A.src.coef[r]);
                const int jlo = sjlo[s - 1];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const unsigned m = (unsigned)(w.col0 + w.lane * CPL + q - jlo);
                    if (m < (unsigned)MSRC) o.ez[q] += cf * ssrc[s - 1][m];
                }
            }
            // end caps: E_r(r, 0) from column 1 (same lane), E_r(r, nz) from column nz - 1
            if (CAPS && w.cap_lo) o.er[0] = A.mur_on ? a.er[1] + A.mur * (o.er[1] - a.er[0]) : 0.f;
            if (CAPS && w.cap_hi) {
                const float old_l = __shfl_up_sync(0xffffffffu, a.er[CPL - 1], 1);
                const float new_l = __shfl_up_sync(0xffffffffu, o.er[CPL - 1], 1);
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    if (w.col0 + w.lane * CPL + q == nz) {
                        const float ol = q > 0 ? a.er[q - 1] : old_l;
                        const float nl = q > 0 ? o.er[q - 1] : new_l;
                        o.er[q] = A.mur_on ? ol + A.mur * (nl - a.er[q]) : 0.f;
                    }
            }
            if (FULL) {
                // the wall E_z(nr, j) of this level, from E_z(nr-1, j) old (a) and
                // new (o) and E_z(nr, j) old (bn); used on the next step
                if (r == nr - 1)
#pragma unroll
                    for (int q = 0; q < CPL; ++q)
                        w.wall[(s - 1) * W + w.lane * CPL + q] =
                            A.mur_on ? a.ez[q] + A.mur * (o.ez[q] - bn.ez[q]) : 0.f;
                // detectors on row r at step n0 + s
                if (r == w.prow[s]) {
                    const float ez_up = __shfl_up_sync(0xffffffffu, o.ez[CPL - 1], 1);
                    int pc = w.pc[s], prow;
                    do {
                        const int4 pr = __ldg(&A.prec[pc]);
                        const int lj = pr.y - w.col0;
                        if (w.lane == lj / CPL) {
                            const int qj = lj % CPL;
                            float ezj = 0.f, ezl = 0.f, erj = 0.f, erb = 0.f;
#pragma unroll
                            for (int q = 0; q < CPL; ++q)
                                if (q == qj) {
                                    ezj = o.ez[q];
                                    erj = o.er[q];
                                    erb = S.prv[s].er[q];
                                    ezl = q > 0 ? o.ez[q > 0 ? q - 1 : 0] : ez_up;
                                }
                            float *t = A.trace + ((long long)pr.z * A.max_steps + A.n0 + s - 1) * 2;
                            t[0] = 0.5f * (ezl + ezj);
                            t[1] = r == 0 ? 0.f : 0.5f * (erb + erj);
                        }
                        ++pc;
                        prow = pc < w.pfin ? __ldg(&A.prec[pc].x) : NO_ROW;
                    } while (prow == r);
                    __syncwarp();
                    if (w.lane == 0) {
                        w.pc[s] = pc;
                        w.prow[s] = prow;
                    }
                    __syncwarp();
                    if (s == K) S.prowK = prow;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                o.er[q] = 0.f;
                o.h[q] = 0.f;
                o.ez[q] = w.wall[(s - 1) * W + w.lane * CPL + q];
            }
        }
    }
    // level K, row p - K: store the owned cells
    const int r = p - K;
    if (w.owned && r >= w.own0 && r < w.own1) {
        const long long o = S.st_off;
        if (FULL || CAPS) {   // the cap warps hold column nz and phantom columns past it
            const int c0 = w.col0 + w.lane * CPL;
            const int nE = nz + 1 - c0, nZ = nz - c0;   // E_r columns <= nz, E_z and H_phi columns < nz
            if (r < nr) {
                st_cols<CPL>(A.out.Er + o, S.cur[K].er, nE);
                st_cols<CPL>(A.out.Hp + o, S.cur[K].h, nZ);
            }
            st_cols<CPL>(A.out.Ez + o, S.cur[K].ez, nZ);
        } else {
            st_cols<CPL>(A.out.Er + o, S.cur[K].er, CPL);
            st_cols<CPL>(A.out.Hp + o, S.cur[K].h, CPL);
            st_cols<CPL>(A.out.Ez + o, S.cur[K].ez, CPL);
        }
    }
    S.st_off += A.pitch;
    return true;
}

// Persistent: the grid is one wave of resident blocks; each block takes tiles
// (segment g, group of NW bands) from an atomic counter until none is left,
// so blocks that draw slow tiles (end caps, source rows, wall, detectors) do
// not hold the launch.  A warp's ring position and parity carry over from
// tile to tile: every row a tile issues is consumed within the tile.
template <int K, int CPL, int MINB, int STAGES>
__global__ void __launch_bounds__(NW * 32, MINB) k_cyl_wave(Wave A) {
    constexpr int W = 32 * CPL;          // columns per warp
    constexpr int HL = K;                // left halo
    constexpr int STAGE = 3 * W;         // floats per ring stage
    static_assert(K % 4 == 0 && K % CPL == 0, "the halo keeps the bulk copies 16-byte aligned");
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[NW][STAGES];
    __shared__ int sjlo[K];
    __shared__ float ssrc[K][MSRC];
    __shared__ __align__(16) float2 srowc[LMAX + 2 * K + 1];   // a last segment may hold L + 1 rows
    __shared__ __align__(16) float swall[NW][K * W];
    __shared__ int spc[NW][K + 1], sprow[NW][K + 1];
    __shared__ int s_tile, s_dead;

    const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
    const int nr = A.nr, nz = A.nz;
    if (A.src.active && tid < K * MSRC) {
        const int s = tid / MSRC, m = tid % MSRC;
        const int jlo = src_jlo(A.src, A.n0 + s);
        if (m == 0) sjlo[s] = jlo;
        ssrc[s][m] = src_face(A.src, A.n0 + s, jlo + m);
    }
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[wi][s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == 0) s_dead = 0;
    int ring_st = 0;            // this warp's next stage and its parity, across tiles
    uint32_t ring_phase = 0;
    const int bxn = (A.nbands + NW - 1) / NW;

    for (;;) {
        __syncthreads();   // the previous tile is done with the shared tables
        if (tid == 0) s_tile = (int)atomicAdd(A.tiles, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= A.ntiles || s_dead) break;
        const int g = tile / bxn, bx = tile - g * bxn;
        // owned rows [own0, own1); the last segment runs to the wall, and it
        // owns row nr - 1 too: the wall value of level s comes from level s at
        // row nr - 1, valid only K rows above the segment's first loaded row
        const int own0 = g * A.L, own1 = g == A.nseg - 1 ? nr + 1 : min(own0 + A.L, nr + 1);
        const int p0 = max(0, own0 - K);
        const int p_end = own1 - 1 + K;
        for (int t = tid; p0 + t <= min(p_end, nr); t += NW * 32) srowc[t] = A.rowc[p0 + t];
        __syncthreads();

        Band<K, CPL> w;
        w.b = bx * NW + wi;
        if (w.b >= A.nbands) continue;
        w.lane = lane;
        w.own0 = own0;
        w.own1 = own1;
        w.p0 = p0;
        w.load_end = min(p_end, nr);
        w.col0 = w.b * A.U - HL;
        const int oc0 = w.b * A.U, oc1 = min(oc0 + A.U, nz + 1);   // owned columns [oc0, oc1)
        w.ring = smem + wi * STAGES * STAGE;
        w.bar = bars[wi];
        w.rowc = srowc;
        w.wall = swall[wi];
        w.pc = spc[wi];
        w.prow = sprow[wi];
        const int c0 = w.col0 + lane * CPL;
        w.owned = c0 >= oc0 && c0 < oc1;                    // a lane owns all or none of its columns
        w.cap_lo = w.b == 0 && lane == HL / CPL;            // holds columns 0 and 1
        w.cap_hi = nz - w.col0 >= 1 && nz - w.col0 < W;     // this warp holds columns nz - 1 and nz
        const bool caps = w.b == 0 || w.cap_hi;

        March<K, CPL> S;
        if (lane == 0)
            for (int s = 0; s < STAGES && p0 + s <= w.load_end; ++s)
                issue_row<CPL>(A, w.ring, w.bar, (long long)(p0 + s) * A.pitch + w.col0, (ring_st + s) % STAGES);
        S.ld_off = (long long)(p0 + STAGES) * A.pitch + w.col0;
        S.st_off = (long long)(p0 - K) * A.pitch + c0;   // row p - K at step p
        {
            const int wid = g * A.nbands + w.b;
            const int pbeg = A.poff[wid];
            w.pfin = A.poff[wid + 1];
            const int r0 = pbeg < w.pfin ? A.prec[pbeg].x : NO_ROW;
            if (lane <= K) {
                w.pc[lane] = pbeg;
                w.prow[lane] = r0;
            }
            S.prowK = r0;
            __syncwarp();
        }
#pragma unroll
        for (int s = 0; s <= K; ++s)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                S.prv[s].er[q] = S.prv[s].ez[q] = S.prv[s].h[q] = 0.f;
                S.cur[s].er[q] = S.cur[s].ez[q] = S.cur[s].h[q] = 0.f;
            }
        S.st = ring_st;
        S.phase = ring_phase;

        // lean steps: every level on a row in [max(p0, source rows), nr - 2], all
        // columns inside [0, nz), no detector on the rows p - K .. p - 1 of the step
        const int src_end = A.src.active ? A.src.nw : 0;
        const int lean_lo = max(p0, src_end) + K, lean_hi = min(nr - 1, p_end);
        int failed_at = -1;
        int p = p0;
        while (p <= p_end) {
            const int stop = min(lean_hi, S.prowK);
            if (p >= lean_lo && p <= stop) {
                bool ok = true;
                if (caps) {
                    for (; ok && p <= stop; ++p) ok = march_step<K, CPL, STAGES, false, true>(A, w, S, p, sjlo, ssrc);
                } else {
                    for (; ok && p + 1 <= stop; p += 2) {
                        ok = march_step<K, CPL, STAGES, false, false>(A, w, S, p, sjlo, ssrc);
                        if (ok) ok = march_step<K, CPL, STAGES, false, false>(A, w, S, p + 1, sjlo, ssrc);
                    }
                    if (ok && p <= stop) {
                        ok = march_step<K, CPL, STAGES, false, false>(A, w, S, p, sjlo, ssrc);
                        ++p;
                    }
                }
                if (!ok) {
                    failed_at = p;
                    break;
                }
            } else {
                if (!march_step<K, CPL, STAGES, true, true>(A, w, S, p, sjlo, ssrc)) {
                    failed_at = p;
                    break;
                }
                ++p;
            }
        }
        ring_st = S.st;
        ring_phase = S.phase;
        if (failed_at >= 0) {
            // give up: flag it, let the copies still in flight land, stop the block
            if (lane == 0) {
                atomicOr(A.flags, 1);
                s_dead = 1;
                int s2 = S.st;
                uint32_t ph = S.phase;
                for (int m = 0; m < STAGES && failed_at + m <= w.load_end; ++m) {
                    // a copy still in flight after these waits may land after the
                    // block ends: flag bit 8 (the handle's status is sticky)
                    bool landed = false;
                    for (int t = 0; t < 4 && !landed; ++t) landed = mbar_wait(&w.bar[s2], ph);
                    if (!landed) atomicOr(A.flags, 8);
                    if (++s2 == STAGES) {
                        s2 = 0;
                        ph ^= 1u;
                    }
                }
            }
            __syncwarp();
        }
    }
    // the last block to finish zeroes the counters for the next launch (the
    // launches of a handle are ordered on its stream), so no memset precedes
    // a launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(A.tiles + 1, 1u) == gridDim.x - 1) {
            atomicExch(A.tiles, 0u);
            atomicExch(A.tiles + 1, 0u);
        }
    }
}

struct Variant {
    int K, CPL, stages;
    void (*fn)(Wave);
    const char *name;
};
// kernel index -> (steps per launch, z columns per lane, rows in flight per warp);
// the third template argument is the resident blocks per SM the registers are bounded for
const Variant kVariants[] = {{0, 0, 0, nullptr, "k_cyl_h+k_cyl_e"},
                             {4, 2, 8, k_cyl_wave<4, 2, 1, 8>, "k_cyl_wave<4,2,1,8>"},
                             {8, 2, 8, k_cyl_wave<8, 2, 1, 8>, "k_cyl_wave<8,2,1,8>"},
                             {4, 4, 8, k_cyl_wave<4, 4, 3, 8>, "k_cyl_wave<4,4,3,8>"},
                             {4, 4, 6, k_cyl_wave<4, 4, 4, 6>, "k_cyl_wave<4,4,4,6>"},
                             {8, 2, 8, k_cyl_wave<8, 2, 4, 8>, "k_cyl_wave<8,2,4,8>"}};
constexpr int kNumKernels = 6;

size_t ring_bytes(const Variant &v) { return (size_t)NW * v.stages * 3 * 32 * v.CPL * sizeof(float); }

}  // namespace

struct cyl_ctx {
    int nr, nz, pitch;
    int boundary;
    double d, dt, eps, kE, kH, mur;
    cudaStream_t stream;
    float *block;
    size_t comp;             // floats per component array
    Set set[2];
    int cur;
    float2 *d_rowc;
    int *d_flags;
    // shower
    double *d_q;
    float *d_coef;
    Src src;
    // detectors
    std::vector<int> pij;    // (i, j) per detector
    int np, max_steps;
    int *d_ij;
    float *d_trace;
    int *d_poff;
    int4 *d_prec;
    // kernel
    int kernel, K, CPL, U, L, nbands, nseg, seg_req;
    long long steps, launches;
    int status;
    // two-kernel path: device step index, and graphs of G2K steps per set
    long long *d_step;
    long long step_host;     // staging of the step index upload
    bool step_ok;            // d_step equals steps - 1
    cudaStream_t gstream;
    cudaEvent_t gev;
    cudaGraphExec_t g2k[2];
    bool graph_off;
    unsigned *d_tiles;       // wavefront tile counters (next tile, blocks done)
    int slots;               // resident blocks of the wavefront kernel in use
};

namespace {

int note(cyl_ctx *h, cudaError_t e) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h && h->status == FDTD_OK) h->status = FDTD_ERR_CUDA;
        return FDTD_ERR_CUDA;
    }
    return FDTD_OK;
}

void free_src(cyl_ctx *h) {
    if (h->d_q) cudaFree(h->d_q);
    if (h->d_coef) cudaFree(h->d_coef);
    h->d_q = nullptr;
    h->d_coef = nullptr;
    h->src = Src{};
}

void free_probes(cyl_ctx *h) {
    if (h->d_ij) cudaFree(h->d_ij);
    if (h->d_trace) cudaFree(h->d_trace);
    if (h->d_poff) cudaFree(h->d_poff);
    if (h->d_prec) cudaFree(h->d_prec);
    h->d_ij = nullptr;
    h->d_trace = nullptr;
    h->d_poff = nullptr;
    h->d_prec = nullptr;
    h->pij.clear();
    h->np = 0;
    h->max_steps = 0;
}

// widest column a warp of any wavefront variant reads, + 1
int read_extent(int nz) {
    int e = nz + 1;
    for (int v = 1; v < kNumKernels; ++v) {
        const int K = kVariants[v].K, W = 32 * kVariants[v].CPL, U = W - 2 * K;
        const int nb = (nz + 1 + U - 1) / U;
        e = std::max(e, (nb - 1) * U - K + W);
    }
    return e;
}

// Resident blocks of the wavefront kernel in use (the persistent grid).
int wave_slots(const cyl_ctx *h) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const Variant &v = kVariants[h->kernel];
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, NW * 32, ring_bytes(v)) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sms * per_sm;
}

// Rows per segment.  A tile marches L + 2K rows (2K of them halo); the
// resident blocks take tiles from a queue.  Tiles differ in speed (caps,
// source rows, wall, detectors) and a block's warps wait for each other at
// every tile, so the launch ends about one tile time after the average
// block: cost = (L + 2K + setup) x (tiles / slots + 1.2), the smallest cost
// wins (measured optimum on the Table I grids: 64, 32 and 16 rows on 8192^2,
// 4096^2 and 2048^2).
int choose_L(cyl_ctx *h) {
    if (h->seg_req > 0) return std::min(std::min(h->seg_req, h->nr + 1), LMAX);
    const double slots = (double)std::max(1, h->slots);
    const long long bx = (h->nbands + NW - 1) / NW;
    int best = std::min(h->nr + 1, LMAX);
    double best_cost = 1e300;
    for (int L = 16; L <= std::min(h->nr + 1 + 15, LMAX); L += 16) {
        const int Lc = std::min(L, h->nr + 1);
        const long long nseg = (h->nr + 1 + Lc - 1) / Lc;
        const double cost = (double)(Lc + 2 * h->K + 8) * ((double)(bx * nseg) / slots + 1.2);
        if (cost < best_cost) {
            best_cost = cost;
            best = Lc;
        }
    }
    return best;
}

// Detector records of the wavefront kernel: per warp (segment, band), sorted by row.
int build_wave_probes(cyl_ctx *h) {
    if (h->d_poff) cudaFree(h->d_poff);
    if (h->d_prec) cudaFree(h->d_prec);
    h->d_poff = nullptr;
    h->d_prec = nullptr;
    if (h->kernel == 0) return FDTD_OK;
    const long long nwarps = (long long)h->nseg * h->nbands;
    std::vector<int> off(nwarps + 1, 0);
    std::vector<long long> key(h->np);
    for (int p = 0; p < h->np; ++p) {
        const int i = h->pij[2 * p], j = h->pij[2 * p + 1];
        key[p] = ((long long)std::min(i / h->L, h->nseg - 1) * h->nbands + j / h->U);
        off[key[p] + 1]++;
    }
    for (long long w = 0; w < nwarps; ++w) off[w + 1] += off[w];
    std::vector<int> order(h->np);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return key[a] != key[b] ? key[a] < key[b] : h->pij[2 * a] < h->pij[2 * b];
    });
    std::vector<int4> rec(std::max(h->np, 1));
    for (int k = 0; k < h->np; ++k) {
        const int p = order[k];
        rec[k] = make_int4(h->pij[2 * p], h->pij[2 * p + 1], p, 0);
    }
    if (cudaMalloc(&h->d_poff, off.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->d_prec, rec.size() * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    if (note(h, cudaMemcpy(h->d_poff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) != FDTD_OK ||
        note(h, cudaMemcpy(h->d_prec, rec.data(), rec.size() * sizeof(int4), cudaMemcpyHostToDevice)) != FDTD_OK)
        return FDTD_ERR_CUDA;
    return FDTD_OK;
}

int configure(cyl_ctx *h, int which, int seg_rows) {
    h->kernel = which;
    h->seg_req = seg_rows;
    if (which == 0) {
        h->K = 1;
        h->CPL = 1;
        h->U = h->L = h->nbands = h->nseg = 0;
    } else {
        const Variant &v = kVariants[which];
        h->K = v.K;
        h->CPL = v.CPL;
        h->U = 32 * v.CPL - 2 * v.K;
        h->nbands = (h->nz + 1 + h->U - 1) / h->U;
        h->slots = wave_slots(h);
        h->L = choose_L(h);
        h->nseg = (h->nr + 1 + h->L - 1) / h->L;
        if (h->nseg > 1 && (h->nr + 1) % h->L == 1) --h->nseg;   // no segment of the wall row alone
    }
    return build_wave_probes(h);
}

// Default kernel by grid size (measured on the Table I grids): below about
// 630^2 cells the two-kernel path replayed from graphs (the wavefront's warps
// are too few to hide their step latency), up to about 1250^2 the wavefront
// with 2 columns per lane (twice the warps), above it 4 columns per lane.
int default_kernel(int nr, int nz) {
    const long long cells = (long long)nr * nz;
    return cells < 400000 ? 0 : cells < 1600000 ? 1 : 3;
}

Dev dev_of(const cyl_ctx *h) {
    Dev D;
    D.nr = h->nr;
    D.nz = h->nz;
    D.pitch = h->pitch;
    D.f = h->set[h->cur];
    D.rowc = h->d_rowc;
    return D;
}

constexpr int G2K = 32;   // steps per captured graph of the two-kernel path

// One step of the two-kernel path on stream st (host counters not touched).
void issue_two_kernel(cyl_ctx *h, cudaStream_t st) {
    const Dev D = dev_of(h);
    const dim3 blk(256), gh((h->nz + 255) / 256, h->nr), ge((h->nz + 1 + 255) / 256, h->nr);
    k_cyl_h<<<gh, blk, 0, st>>>(D, (float)h->kH, h->d_step);
    k_cyl_e<<<ge, blk, 0, st>>>(D, (float)h->kE, (float)h->mur, h->boundary == FDTD_MUR1, h->src, h->d_step);
    if (h->np > 0)
        k_cyl_probes<<<(h->np + 127) / 128, 128, 0, st>>>(D, h->d_ij, h->np, h->d_trace, h->max_steps, h->d_step);
}

void drop_graphs(cyl_ctx *h) {
    for (int c = 0; c < 2; ++c)
        if (h->g2k[c]) {
            cudaGraphExecDestroy(h->g2k[c]);
            h->g2k[c] = nullptr;
        }
}

int sync_step_index(cyl_ctx *h) {
    if (h->step_ok) return FDTD_OK;
    h->step_host = h->steps - 1;
    if (note(h, cudaMemcpyAsync(h->d_step, &h->step_host, sizeof(long long), cudaMemcpyHostToDevice, h->stream)) !=
        FDTD_OK)
        return h->status;
    h->step_ok = true;
    return note(h, cudaStreamSynchronize(h->stream));   // the staging value is read before it changes
}

// n steps of the two-kernel path: whole graphs of G2K steps replayed on a
// private stream (ordered with the handle's stream by events), the rest
// launched directly.
void launch_two_kernel(cyl_ctx *h, int n) {
    if (sync_step_index(h) != FDTD_OK) return;
    int reps = h->graph_off ? 0 : n / G2K;
    if (reps > 0 && !h->g2k[h->cur]) {
        cudaGraph_t graph = nullptr;
        bool ok = cudaEventRecord(h->gev, h->stream) == cudaSuccess &&
                  cudaStreamWaitEvent(h->gstream, h->gev, 0) == cudaSuccess &&
                  cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            for (int s = 0; s < G2K; ++s) issue_two_kernel(h, h->gstream);
            ok = cudaStreamEndCapture(h->gstream, &graph) == cudaSuccess && graph &&
                 cudaGraphInstantiate(&h->g2k[h->cur], graph, 0) == cudaSuccess;
        }
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            h->g2k[h->cur] = nullptr;
            h->graph_off = true;
            reps = 0;
        }
    }
    if (reps > 0) {
        if (note(h, cudaEventRecord(h->gev, h->stream)) || note(h, cudaStreamWaitEvent(h->gstream, h->gev, 0)))
            return;
        for (int r = 0; r < reps; ++r)
            if (note(h, cudaGraphLaunch(h->g2k[h->cur], h->gstream)) != FDTD_OK) return;
        if (note(h, cudaEventRecord(h->gev, h->gstream)) || note(h, cudaStreamWaitEvent(h->stream, h->gev, 0)))
            return;
        h->launches += (long long)reps * G2K * (h->np > 0 ? 3 : 2);
        h->steps += (long long)reps * G2K;
        n -= reps * G2K;
    }
    for (; n > 0; --n) {
        issue_two_kernel(h, h->stream);
        h->launches += h->np > 0 ? 3 : 2;
        h->steps++;
    }
}

void launch_wave(cyl_ctx *h) {
    const Variant &v = kVariants[h->kernel];
    Wave A;
    A.nr = h->nr;
    A.nz = h->nz;
    A.pitch = h->pitch;
    A.in = h->set[h->cur];
    A.out = h->set[h->cur ^ 1];
    A.rowc = h->d_rowc;
    A.kE = (float)h->kE;
    A.kH = (float)h->kH;
    A.mur = (float)h->mur;
    A.mur_on = h->boundary == FDTD_MUR1;
    A.U = h->U;
    A.L = h->L;
    A.nbands = h->nbands;
    A.src = h->src;
    A.n0 = h->steps;
    A.poff = h->d_poff;
    A.prec = h->d_prec;
    A.trace = h->d_trace;
    A.max_steps = h->max_steps;
    A.flags = h->d_flags;
    A.tiles = h->d_tiles;
    A.ntiles = h->nseg * ((h->nbands + NW - 1) / NW);
    A.nseg = h->nseg;
    const int grid = std::min(A.ntiles, std::max(1, h->slots));
    v.fn<<<grid, NW * 32, ring_bytes(v), h->stream>>>(A);
    h->launches++;
    h->cur ^= 1;
    h->steps += v.K;
    h->step_ok = false;
}

size_t comp_rows(const cyl_ctx *h, int comp) { return comp == 1 ? (size_t)h->nr + 1 : (size_t)h->nr; }
size_t comp_cols(const cyl_ctx *h, int comp) { return comp == 0 ? (size_t)h->nz + 1 : (size_t)h->nz; }
float *comp_ptr(cyl_ctx *h, int comp) {
    const Set &s = h->set[h->cur];
    return comp == 0 ? s.Er : comp == 1 ? s.Ez : s.Hp;
}

}  // namespace

extern "C" {

int cyl_create(cyl_t *out, int nr, int nz, double d, double dt, double eps_r, int boundary, void *stream) {
    if (!out) return FDTD_ERR_ARG;
    *out = nullptr;
    if (nr < 4 || nz < 4 || !(d > 0.0) || !(dt > 0.0) || !(eps_r >= 1.0) ||
        (boundary != FDTD_PEC && boundary != FDTD_MUR1))
        return FDTD_ERR_ARG;
    if (nr > 65534 || (long long)(nr + 1) * (nz + 1) > (1LL << 34)) return FDTD_ERR_ARG;   // rows index grid.y
    if (dt > d * std::sqrt(eps_r) / (kC * std::sqrt(2.0))) return FDTD_ERR_CFL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    cyl_ctx *h = new (std::nothrow) cyl_ctx();
    if (!h) return FDTD_ERR_OOM;
    h->nr = nr;
    h->nz = nz;
    h->pitch = (PADL + read_extent(nz) + 31) / 32 * 32;
    h->boundary = boundary;
    h->d = d;
    h->dt = dt;
    h->eps = eps_r / (kMu0 * kC * kC);
    h->kE = dt / (h->eps * d);
    h->kH = dt / (kMu0 * d);
    const double S = kC / std::sqrt(eps_r) * dt / d;
    h->mur = (S - 1.0) / (S + 1.0);
    h->stream = static_cast<cudaStream_t>(stream);
    h->comp = (size_t)(nr + 1) * h->pitch;
    const size_t bytes = 6 * h->comp * sizeof(float);
    std::vector<float2> rowc(nr + 1);
    rowc[0] = make_float2((float)(4.0 * h->kE), 0.f);
    for (int i = 1; i <= nr; ++i)
        rowc[i] = make_float2((float)(h->kE * (i + 0.5) / i), (float)(h->kE * (i - 0.5) / i));
    if (cudaMalloc(&h->block, bytes) != cudaSuccess || cudaMalloc(&h->d_rowc, (nr + 1) * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&h->d_flags, sizeof(int)) != cudaSuccess || cudaMalloc(&h->d_step, sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&h->d_tiles, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->d_tiles, 0, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->gev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cyl_destroy(h);
        return FDTD_ERR_OOM;
    }
    for (int s = 0; s < 2; ++s) {
        float *base = h->block + 3 * s * h->comp + PADL;
        h->set[s] = Set{base, base + h->comp, base + 2 * h->comp};
    }
    for (int v = 1; v < kNumKernels; ++v)   // dynamic + static shared memory may pass 48 KB
        note(h, cudaFuncSetAttribute(kVariants[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ring_bytes(kVariants[v])));
    note(h, cudaMemsetAsync(h->block, 0, bytes, h->stream));
    note(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream));
    note(h, cudaMemcpyAsync(h->d_rowc, rowc.data(), rowc.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
    note(h, cudaStreamSynchronize(h->stream));
    if (h->status == FDTD_OK) h->status = configure(h, default_kernel(nr, nz), 0);
    if (h->status != FDTD_OK) {
        const int st = h->status;
        cyl_destroy(h);
        return st;
    }
    *out = h;
    return FDTD_OK;
}

void cyl_destroy(cyl_t h) {
    if (!h) return;
    if (h->gstream) cudaStreamSynchronize(h->gstream);
    drop_graphs(h);
    free_src(h);
    free_probes(h);
    if (h->block) cudaFree(h->block);
    if (h->d_rowc) cudaFree(h->d_rowc);
    if (h->d_flags) cudaFree(h->d_flags);
    if (h->d_step) cudaFree(h->d_step);
    if (h->d_tiles) cudaFree(h->d_tiles);
    if (h->gev) cudaEventDestroy(h->gev);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    delete h;
}

int cyl_set_kernel(cyl_t h, int which, int seg_rows) {
    if (!h || which < 0 || which >= kNumKernels || seg_rows < 0) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    const int st = configure(h, which, seg_rows);
    if (st != FDTD_OK && h->status == FDTD_OK) h->status = st;
    return st;
}
int cyl_tune(cyl_t h, int launches, int *steps_used) {
    if (steps_used) *steps_used = 0;
    if (!h || launches < 1 || launches > 8) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (h->kernel == 0) return FDTD_OK;   // the two-kernel path has no segments
    // candidates: 12 rows and up (steps of 4 to 64, 8 to 128, 16 beyond) until
    // the tiles fit one wave of the resident blocks (longer segments then only
    // lengthen every tile); at most TUNE_MAX of them
    const long long bx = (h->nbands + NW - 1) / NW;
    const long long slots = std::max(1, h->slots);
    std::vector<int> cand;
    for (int L = 12; L <= std::min(h->nr + 1, LMAX) && (int)cand.size() < TUNE_MAX;
         L += L < 64 ? 4 : L < 128 ? 8 : 16) {
        cand.push_back(L);
        long long nseg = (h->nr + 1 + L - 1) / L;
        if (nseg > 1 && (h->nr + 1) % L == 1) --nseg;
        if (nseg * bx <= slots) break;
    }
    const long long need = (long long)cand.size() * launches * h->K;
    if (h->np > 0 && h->steps + need > h->max_steps) return FDTD_ERR_CAPACITY;
    std::vector<cudaEvent_t> ev(launches + 1, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            for (auto &f : ev)
                if (f) cudaEventDestroy(f);
            return FDTD_ERR_CUDA;
        }
    const int kernel = h->kernel;
    int best = h->L;
    float best_ms = -1.f;
    int used = 0;
    for (int L : cand) {
        if (configure(h, kernel, L) != FDTD_OK) break;
        cudaEventRecord(ev[0], h->stream);
        for (int i = 0; i < launches; ++i) {
            launch_wave(h);
            cudaEventRecord(ev[i + 1], h->stream);
        }
        used += launches * h->K;
        if (note(h, cudaEventSynchronize(ev[launches])) != FDTD_OK || h->status != FDTD_OK) break;
        float ms = -1.f;   // the fastest launch of the candidate
        for (int i = 0; i < launches; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess && (ms < 0.f || t < ms)) ms = t;
        }
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = L;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    cudaGetLastError();
    if (steps_used) *steps_used = used;
    if (h->status != FDTD_OK) return h->status;
    const int st = configure(h, kernel, best);
    if (st != FDTD_OK && h->status == FDTD_OK) h->status = st;
    return st;
}

int cyl_kernel_info(cyl_t h, int *which, int *steps_per_launch, int *seg_rows) {
    if (!h) return FDTD_ERR_ARG;
    if (which) *which = h->kernel;
    if (steps_per_launch) *steps_per_launch = h->K;
    if (seg_rows) *seg_rows = h->L;
    return FDTD_OK;
}

int cyl_set_shower(cyl_t h, const double *q, int n_bins, double z0, double bin_dz, double v, const double *w,
                   int nw) {
    if (!h || !q || !w || n_bins < 2 || !(bin_dz > 0.0) || nw < 1 || nw > h->nr + 1 || !std::isfinite(z0) ||
        !std::isfinite(v) || std::fabs(v) * h->dt > 4.0 * h->d)
        return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (note(h, cudaStreamSynchronize(h->gstream)) != FDTD_OK) return h->status;
    drop_graphs(h);
    free_src(h);
    std::vector<float> coef(nw);
    for (int i = 0; i < nw; ++i) {
        const double A = i == 0 ? kPi * h->d * h->d / 4.0 : 2.0 * kPi * (double)i * h->d * h->d;
        coef[i] = (float)(w[i] / (h->eps * A));
    }
    if (cudaMalloc(&h->d_q, n_bins * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_coef, nw * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        free_src(h);
        return FDTD_ERR_OOM;
    }
    if (note(h, cudaMemcpy(h->d_q, q, n_bins * sizeof(double), cudaMemcpyHostToDevice)) != FDTD_OK ||
        note(h, cudaMemcpy(h->d_coef, coef.data(), nw * sizeof(float), cudaMemcpyHostToDevice)) != FDTD_OK)
        return h->status;
    h->src.active = 1;
    h->src.nbins = n_bins;
    h->src.nw = std::min(nw, h->nr);   // ring nr lies on the wall, whose E_z the boundary sets
    h->src.z0 = z0;
    h->src.bin_dz = bin_dz;
    h->src.v = v;
    h->src.dt = h->dt;
    h->src.d = h->d;
    h->src.q = h->d_q;
    h->src.coef = h->d_coef;
    return FDTD_OK;
}

int cyl_set_probes(cyl_t h, const double *rz, int n, int max_steps) {
    if (!h || n < 0 || (n > 0 && !rz) || max_steps < 0) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    std::vector<int> ij(2 * (size_t)n);
    for (int p = 0; p < n; ++p) {
        if (!std::isfinite(rz[2 * p]) || !std::isfinite(rz[2 * p + 1])) return FDTD_ERR_ARG;
        const double fi = std::floor(rz[2 * p] / h->d + 0.5), fj = std::floor(rz[2 * p + 1] / h->d + 0.5);
        if (fi < 0 || fi >= h->nr || fj < 1 || fj >= h->nz) return FDTD_ERR_ARG;
        ij[2 * p] = (int)fi;
        ij[2 * p + 1] = (int)fj;
    }
    if (note(h, cudaStreamSynchronize(h->gstream)) != FDTD_OK) return h->status;
    drop_graphs(h);
    free_probes(h);
    if (n == 0) {
        // the wavefront kernel reads its (empty) per-warp lists
        const int st = build_wave_probes(h);
        if (st != FDTD_OK && h->status == FDTD_OK) h->status = st;
        return st;
    }
    const size_t tbytes = std::max<size_t>((size_t)n * max_steps * 2 * sizeof(float), 16);
    if (cudaMalloc(&h->d_ij, ij.size() * sizeof(int)) != cudaSuccess || cudaMalloc(&h->d_trace, tbytes) != cudaSuccess) {
        cudaGetLastError();
        free_probes(h);
        return FDTD_ERR_OOM;
    }
    if (note(h, cudaMemcpy(h->d_ij, ij.data(), ij.size() * sizeof(int), cudaMemcpyHostToDevice)) != FDTD_OK ||
        note(h, cudaMemsetAsync(h->d_trace, 0, tbytes, h->stream)) != FDTD_OK)
        return h->status;
    h->pij = ij;
    h->np = n;
    h->max_steps = max_steps;
    const int st = build_wave_probes(h);
    if (st != FDTD_OK && h->status == FDTD_OK) h->status = st;
    return st;
}

int cyl_step(cyl_t h, int n) {
    if (!h || n < 0) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (h->np > 0 && h->steps + n > h->max_steps) return FDTD_ERR_CAPACITY;
    if (h->kernel > 0)
        for (; n >= h->K; n -= h->K) launch_wave(h);
    if (n > 0) launch_two_kernel(h, n);
    return note(h, cudaGetLastError());
}

int cyl_sync(cyl_t h) {
    if (!h) return FDTD_ERR_ARG;
    if (note(h, cudaStreamSynchronize(h->stream)) != FDTD_OK) return h->status;
    int flag = 0;
    if (note(h, cudaMemcpy(&flag, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost)) != FDTD_OK) return h->status;
    if (flag && h->status == FDTD_OK) h->status = FDTD_ERR_TIMEOUT;
    return h->status;
}

int cyl_probes(cyl_t h, float *out, int on_device) {
    if (!h || !out) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (h->np == 0) return FDTD_OK;
    const size_t bytes = (size_t)h->np * h->max_steps * 2 * sizeof(float);
    if (bytes &&
        note(h, cudaMemcpyAsync(out, h->d_trace, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream)) != FDTD_OK)
        return h->status;
    return cyl_sync(h);
}

int cyl_fields(cyl_t h, int comp, float *out, int on_device) {
    if (!h || !out || comp < 0 || comp > 2) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    const int rows = (int)comp_rows(h, comp), cols = (int)comp_cols(h, comp);
    if (on_device) {
        const dim3 g((cols + 255) / 256, rows);
        k_cyl_copy<<<g, 256, 0, h->stream>>>(comp_ptr(h, comp), h->pitch, out, cols, rows, cols);
        h->launches++;
        if (note(h, cudaGetLastError()) != FDTD_OK) return h->status;
        return cyl_sync(h);
    }
    if (note(h, cudaMemcpy2DAsync(out, cols * sizeof(float), comp_ptr(h, comp), h->pitch * sizeof(float),
                                  cols * sizeof(float), rows, cudaMemcpyDeviceToHost, h->stream)) != FDTD_OK)
        return h->status;
    return cyl_sync(h);
}

int cyl_set_field(cyl_t h, int comp, const float *in, int on_device) {
    if (!h || !in || comp < 0 || comp > 2) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    const int rows = (int)comp_rows(h, comp), cols = (int)comp_cols(h, comp);
    if (note(h, cudaMemcpy2DAsync(comp_ptr(h, comp), h->pitch * sizeof(float), in, cols * sizeof(float),
                                  cols * sizeof(float), rows,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream)) !=
        FDTD_OK)
        return h->status;
    return cyl_sync(h);
}

int cyl_reset(cyl_t h) {
    if (!h) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (note(h, cudaMemsetAsync(h->block, 0, 6 * h->comp * sizeof(float), h->stream)) != FDTD_OK) return h->status;
    if (h->d_trace &&
        note(h, cudaMemsetAsync(h->d_trace, 0, (size_t)h->np * h->max_steps * 2 * sizeof(float), h->stream)) !=
            FDTD_OK)
        return h->status;
    h->steps = 0;
    h->cur = 0;
    h->step_ok = false;
    return cyl_sync(h);
}

const char *cyl_kernel_name(cyl_t h) { return h ? kVariants[h->kernel].name : "none"; }

int cyl_steps_done(cyl_t h, int64_t *steps) {
    if (!h || !steps) return FDTD_ERR_ARG;
    *steps = h->steps;
    return FDTD_OK;
}

int cyl_launch_count(cyl_t h, int64_t *launches) {
    if (!h || !launches) return FDTD_ERR_ARG;
    *launches = h->launches;
    return FDTD_OK;
}

}  // extern "C"
