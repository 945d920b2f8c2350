// kernels_tb2.cu -- two leapfrog steps per pass over the whole grid
// (temporal blocking of the Yee scheme, Sec. III.A; shower current of
// Sec. III.B; the CPML, this library's choice of absorbing boundary, and the
// detectors included).
//
// One launch takes E^n, H^{n-1/2} (set cur) to E^{n+2}, H^{n+3/2} (set cur^1):
// the fields are read once and written once for two steps, 24 B + 24 B per
// cell, so 24 B per cell-update instead of 48 B.
//
// Tiles.  A wide block owns up to 120 columns [i0, i0+120) by TY = 8 rows
// [j0, j0+8) and marches up a chunk of z planes [k0, k1).  It computes the
// first step (level 1: H^{n+1/2}, E^{n+1}) on a larger region and the second
// (level 2: H^{n+3/2}, E^{n+2}) on its own cells:
//   lanes: lane L holds the four columns i0-4+4L .. i0-4+4L+3 as float4, so
//     the block computes columns [i0-4, i0+124); the values of a level stay
//     correct where their stencil stays inside that range, which leaves two
//     correct columns left and three right of the owned ones after level 2
//     (x neighbours by warp shuffle);
//   warps: warp w (0..10) is row j0-2+w; level-1 H on rows j0-2 .. j0+8,
//     level-1 E on j0-1 .. j0+8, level-2 H on j0-1 .. j0+7, level-2 E on the
//     owned rows (y neighbours through shared exchange rows).
// On a CPML grid the x layers belong to narrow blocks (scalar lanes: 32
// computed columns, 24 owned), and the wide blocks lie where neither their
// owned cells nor the halo values those depend on (columns i0-2 .. end) meet
// an x layer, so the wide blocks carry no x CPML code at all (tile_col).
// Every value of the halo is computed from the same inputs with the same
// arithmetic as by the tile that owns it, so it is that tile's value; values
// of nodes outside the grid, and the components a cell owns on the grid's low
// faces, are zero, as the one-step paths leave them.
//
// z march.  Iteration p (from k0-2 to k1) waits for input plane p+1 (TMA ring
// of stages, bounded waits), then:
//   A  level-1 H at plane p (planes p, p+1 of the stage);
//   B  level-1 E at plane p (level-1 H of plane p-1 kept in registers);
//   C  level-2 H at plane q = p-1 (level-1 E of plane p-1 kept in registers,
//      and of plane p from B);
//   D  level-2 E at plane q (level-2 H of plane q-1 kept in registers);
//      stores of the owned H and E of plane q.
// Exchange rows: A writes Hx, Hz of its row for B of the warp above (two
// buffers, by the parity of p); C writes level-2 Hx, Hz for D of the warp
// above; D writes the level-1 Ex, Ez of plane p for the next iteration's C
// of the warp below.
//
// Synchronisation.  No block barrier inside the march: a row warp signals an
// mbarrier of its own when its row of an exchange buffer is written and
// waits only for the rows it reads (B for A's row below, D for C's row
// below, and before signalling its A row, for the B row above from the last
// iteration, which C reads).  Those waits also order every rewrite of a row
// after its reads: warp w rewrites its A row of one parity two iterations
// later, after it has seen the warp above finish the iteration in between;
// its C row one iteration later, after the warp above read it (that warp's D
// precedes its B-row signal); its B row after the warp below finished its C,
// which D waits for.  A barrier's waits are parity waits, so its phase must
// never run two ahead of a waiter: the warp above cannot finish iteration p
// (B waits for this warp's A row of p) before this warp has waited for its
// B row of p-1, and likewise for the other rows.  A twelfth warp refills the
// ring: plane r goes into the stage of plane r - ns once every row warp has
// signalled that stage empty.  Every wait is bounded; a warp whose wait
// expires stops, and the warps that wait for it stop in turn.
//
// CPML.  The first step of a halo cell needs the CPML memory of that cell, so
// the stages carry psi boxes (x, y, z) where the tile meets a layer.  The
// level-1 memory stays in registers for level 2; level 2 writes the H psi to
// the other H set (as the one-step path does) and the E psi to the other E
// set (the one-step paths update E psi in place, which a neighbour's halo
// would read after it changed).  z chunks are split so that only the chunks
// of the two layers carry z boxes.
//
// Detectors.  The level-1 E of the six cells of a detector's readout (Ex at
// i-1, i; Ey at j-1, j; Ez at k-1, k) go to a small buffer from the tile that
// owns them; the readout of step n+1 reads them, that of step n+2 reads the
// fields.  A block's records are sorted by plane; those of plane q are served
// in the next iteration, one per thread, from the shared rows that hold the
// level-1 E of plane q (Ex, Ez in the exchange rows, Ey in rows of its own),
// so thousands of detectors in one tile cost a few loads per plane.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fdtd_internal.h"
#include "source_term.cuh"
#include "tma_pipe.cuh"

namespace fdtd {
namespace {

using namespace tma;

constexpr int TY = 8;                 // owned rows
constexpr int NWR = TY + 3;           // row warps: rows j0-2 .. j0+TY
constexpr int NT = 32 * (NWR + 1);    // and one warp that refills the stage ring
constexpr int BR = TY + 4;            // box rows j0-2 .. j0+TY+1
constexpr int NSMAX = 8;

// mbarriers of a block: the stage ring (full: the stage's copies landed;
// empty: every row warp is done with it) and the exchange rows (a row warp's
// row of an exchange buffer is written)
struct Bars {
    uint64_t full[NSMAX], empty[NSMAX];
    uint64_t xa[2][NWR], xb[NWR], xc[NWR];
};
constexpr int BAR_BYTES = 512;
static_assert(sizeof(Bars) <= BAR_BYTES, "barrier area");

// Tile geometry for lanes of VW columns (VW = 4: float4 lanes of the wide
// tiles; VW = 1: scalar lanes of the narrow tiles over the x layers)
template <int VW>
struct Geo {
    static constexpr int TXC = 32 * VW;          // computed columns i0-4 .. i0+TXC-5
    static constexpr int TXO = TXC - 8;          // owned columns (lanes 4/VW .. 31-4/VW)
    static constexpr int BOX = TXC * BR;         // floats of a field or y/z psi box
    static constexpr int FIELDS = 6 * BOX;
    static constexpr unsigned FIELD_BYTES = 4u * FIELDS;
    static constexpr int XROW = 2 * TXC;         // exchange floats per warp row (two components)
    static constexpr int XBUF = NWR * XROW;      // one exchange buffer
    // CPML coefficient table (floats): aH, bH, aE, bE of the computed columns,
    // of the rows j0-2 .. j0+TY+1, of the planes kstart .. kstart+zt-1
    static constexpr int CX = 0;
    static constexpr int CY = 4 * TXC;
    static constexpr int CZ = CY + 4 * BR;
    static constexpr int LO = 4 / VW;            // first owned lane
    static constexpr int HI = 31 - 4 / VW;       // last owned lane
    // shared memory: barriers, four exchange buffers (A's two, B's, C's),
    // coefficient table, ring
    __host__ __device__ static constexpr int head_floats(int zt) {
        return (4 * XBUF + CZ + 4 * zt + 31) / 32 * 32;
    }
};

// ---- lane vectors: the same code for float4 and scalar lanes ----
template <int VW> struct Vec;
template <> struct Vec<4> { typedef float4 T; typedef uint4 U; };
template <> struct Vec<1> { typedef float T; typedef unsigned U; };

template <typename V> __device__ __forceinline__ V ldv(const float *p) { return *reinterpret_cast<const V *>(p); }
template <typename V> __device__ __forceinline__ void stv(float *p, V v) { *reinterpret_cast<V *>(p) = v; }
template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
__device__ __forceinline__ float axpy(float a, float s, float d) { return a + s * d; }
__device__ __forceinline__ float cpmls(float &psi, float a, float b, float d) { return cpml1(psi, a, b, d); }
__device__ __forceinline__ float cpmlv(float &psi, float a, float b, float d) { return cpml1(psi, a, b, d); }
__device__ __forceinline__ float first(float v) { return v; }
__device__ __forceinline__ float last(float v) { return v; }
__device__ __forceinline__ float right(float, float r) { return r; }
__device__ __forceinline__ float left(float, float l) { return l; }
__device__ __forceinline__ unsigned umask(const unsigned *m, float) { return m[0]; }
__device__ __forceinline__ void stn(float *p, float v, int) { *p = v; }
__device__ __forceinline__ void add_source(float &v, const Source &s, const SourceStep &w, int c0, int j, int k) {
    v += source_at(s, w, c0, j, k);
}
// the float4 forms (tma_pipe.cuh) in the same overload sets as the scalar forms
using tma::axpy;
using tma::cpmlv;
using tma::operator-;
__device__ __forceinline__ float4 cpmls(float4 &psi, float a, float b, float4 d) { return cpml4(psi, a, b, d); }
__device__ __forceinline__ float first(float4 v) { return v.x; }
__device__ __forceinline__ float last(float4 v) { return v.w; }
// the vector one column to the right (x+1) / left (x-1), edge element given
__device__ __forceinline__ float4 right(float4 v, float r) { return make_float4(v.y, v.z, v.w, r); }
__device__ __forceinline__ float4 left(float4 v, float l) { return make_float4(l, v.x, v.y, v.z); }
// v with the elements outside the mask set to +0 (bitwise, so a non-finite
// value outside the state never leaks in)
__device__ __forceinline__ float mk(float v, unsigned b) { return __uint_as_float(__float_as_uint(v) & b); }
template <bool MASK>
__device__ __forceinline__ float4 keep(float4 v, uint4 b) {
    if (!MASK) return v;
    return make_float4(mk(v.x, b.x), mk(v.y, b.y), mk(v.z, b.z), mk(v.w, b.w));
}
template <bool MASK>
__device__ __forceinline__ float keep(float v, unsigned b) {
    if (!MASK) return v;
    return mk(v, b);
}
template <typename U> __device__ __forceinline__ U uzero();
template <> __device__ __forceinline__ uint4 uzero<uint4>() { return make_uint4(0u, 0u, 0u, 0u); }
template <> __device__ __forceinline__ unsigned uzero<unsigned>() { return 0u; }
__device__ __forceinline__ uint4 umask(const unsigned *m, float4) { return make_uint4(m[0], m[1], m[2], m[3]); }
// store the first n (1..VW) elements; one vector store when n == VW
__device__ __forceinline__ void stn(float *p, float4 v, int n) { st4n(p, v, n); }
// a store of an owned lane: in the instances without masks (a block clear
// of the grid's faces) every owned lane holds VW columns on the grid (tile
// ends are multiples of four), so the vector store needs no count
template <bool MASK, typename V> __device__ __forceinline__ void stw(float *p, V v, int n) {
    if (MASK) stn(p, v, n);
    else stv(p, v);
}
// the shower's current on the lane's Ez edges
__device__ __forceinline__ void add_source(float4 &v, const Source &s, const SourceStep &w, int c0, int j, int k) {
    v.x += source_at(s, w, c0, j, k);
    v.y += source_at(s, w, c0 + 1, j, k);
    v.z += source_at(s, w, c0 + 2, j, k);
    v.w += source_at(s, w, c0 + 3, j, k);
}

// Tensor maps; fields and y/z psi per tile width (wd 0: float4 lanes, 128
// columns; wd 1: scalar lanes, 32 columns)
struct Maps {
    CUtensorMap f[2][2][6]; // fields [wd][set][component]
    CUtensorMap x[4][2];    // psi x: xHy, xHz [field set], xEy, xEz [E psi set]
    CUtensorMap y[2][4][2]; // psi y [wd]: yHx, yHz, yEx, yEz
    CUtensorMap z[2][4][2]; // psi z [wd]: zHx, zHy, zEx, zEy
};

// Tile columns: nl narrow ones (scalar lanes, up to 24 owned columns) over
// [0, a), nw wide ones (float4 lanes, up to 120) over [a, b), then narrow ones
// over [b, nx).  On a CPML grid the wide tiles stay clear of the x layers
// (their owned results depend on columns i0-2 .. end+1 only), so the x layers'
// CPML memory is updated by the narrow tiles alone, one column per lane.
struct TileCol {
    int i0, w, vw;
};
__host__ __device__ inline TileCol tile_col(int tc, int a, int b, int nl, int nw, int nx) {
    TileCol t;
    if (tc < nl) {
        t.i0 = 24 * tc;
        t.w = a - t.i0 < 24 ? a - t.i0 : 24;
        t.vw = 1;
    } else if (tc < nl + nw) {
        t.i0 = a + 120 * (tc - nl);
        t.w = b - t.i0 < 120 ? b - t.i0 : 120;
        t.vw = 4;
    } else {
        t.i0 = b + 24 * (tc - nl - nw);
        t.w = nx - t.i0 < 24 ? nx - t.i0 : 24;
        t.vw = 1;
    }
    return t;
}

struct Args {
    Grid g;
    float *out[6];          // output field set
    Cpml pm;                // psi read (hin: H set cur, e: E set ecur) and coefficients
    float *eout[3][2];      // E psi written (set ecur^1); H psi: pm.hout
    int ta, tb, nl, nw, tiles_x, tiles_y;   // tile columns (tile_col), tiles_x = their number
    int za, zb, cm, m;      // z chunks: m of cm planes over [za, zb), then [0, za), [zb, nz)
    int zt;                 // planes of the z coefficient table
    int smem_floats;        // floats of dynamic shared memory after the barriers
    int xlo4, xhb, xbw;     // x psi: high half start, first column of the high half, box width
    int xplane;             // floats of an x psi plane (ny rows)
    int cur, ecur;
    Source src;
    SourceStep ss1, ss2;    // current of steps n and n+1
    float kE, kH;
    int *flags;
    const int4 *prec;       // detector records {k, j, i, slot * 4 + component}
    const int *pidx;        // records of block b: [pidx[b], pidx[b+1])
    float *pbuf;            // level-1 values of the records
};

struct Blk {
    int i0, j0, k0, k1, kstart, nplanes;
    int iend;               // end of the owned columns
    bool src_blk, hx, hy, hz;
    int l0;                 // first y slab row of the y box
    int xo, yo, zo, stage, ns;
    int xlo, xhi, nxb, xb;
    int pbeg, pend;
};

template <int VW>
__device__ __forceinline__ void issue_plane(const Args &A, const Maps &M, const Blk &B, float *st, uint64_t *bar,
                                            int r) {
    typedef Geo<VW> G;
    const int p = B.kstart + r;
    const int lz = (B.hz && p >= 0 && p < A.g.nz) ? slab_cell(p, A.g.nz, A.pm.P) : -1;
    unsigned bytes = G::FIELD_BYTES;
    if (B.hx) bytes += 16u * (unsigned)(B.nxb * A.xbw * BR);
    if (B.hy) bytes += 16u * G::BOX;
    if (lz >= 0) bytes += 16u * G::BOX;
    mbar_expect_tx(bar, bytes);
    constexpr int WD = VW == 4 ? 0 : 1;
#pragma unroll
    for (int c = 0; c < 6; ++c) tma_load(st + c * G::BOX, &M.f[WD][A.cur][c], bar, B.i0 - 4, B.j0 - 2, p);
    if (B.hx)
        for (int a = 0; a < 4; ++a) {
            float *d = st + B.xo + a * B.nxb * B.xb;
            const CUtensorMap *mp = &M.x[a][a < 2 ? A.cur : A.ecur];
            if (B.xlo >= 0) tma_load(d + B.xlo * B.xb, mp, bar, 0, B.j0 - 2, p);
            if (B.xhi >= 0) tma_load(d + B.xhi * B.xb, mp, bar, A.xlo4, B.j0 - 2, p);
        }
    if (B.hy)
        for (int a = 0; a < 4; ++a)
            tma_load(st + B.yo + a * G::BOX, &M.y[WD][a][a < 2 ? A.cur : A.ecur], bar, B.i0 - 4, B.l0, p);
    if (lz >= 0)
        for (int a = 0; a < 4; ++a)
            tma_load(st + B.zo + a * G::BOX, &M.z[WD][a][a < 2 ? A.cur : A.ecur], bar, B.i0 - 4, B.j0 - 2, lz);
}

template <int VW>
struct Lane {
    typedef typename Vec<VW>::U U;
    int lane, w, c0, j;
    bool rowin;
    bool own;          // stores level-2 values: owned lane and row, on the grid
    int nval;          // columns of the lane on the grid
    U mcol;            // all bits of an element whose column lies in [0, nx)
    U mcol0;           // the same without column 0
    int ly;            // y slab row of j, or -1
    bool xl;           // the lane's columns lie in an x half (row on the grid)
    int xs, xpos;      // x psi: offset in a stage's x array (box row 0), position of column c0
    unsigned yoff, zoff, xoff;   // the lane's psi offsets in plane 0 / slab plane 0
};

// Per-plane element masks of the six components: the state a cell keeps
// (all bits) or a zero that the one-step paths leave there (no bits): nodes
// outside the grid, and the components a cell owns on the grid's low faces.
template <typename U>
struct Masks {
    U hx, hy, hz, ex, ey, ez;
};
template <int VW>
__device__ __forceinline__ Masks<typename Vec<VW>::U> masks(const Lane<VW> &L, int k, int nz) {
    typedef typename Vec<VW>::U U;
    const U z = uzero<U>();
    const bool in = L.rowin && k >= 0 && k < nz, fj = L.j != 0, fk = k != 0;
    Masks<U> m;
    m.hx = in ? L.mcol0 : z;
    m.hy = in && fj ? L.mcol : z;
    m.hz = in && fk ? L.mcol : z;
    m.ex = in && fj && fk ? L.mcol : z;
    m.ey = in && fk ? L.mcol0 : z;
    m.ez = in && fj ? L.mcol0 : z;
    return m;
}

constexpr unsigned FULL = 0xffffffffu;

// Register state carried from one iteration to the next.
template <typename V>
struct State {
    V ex1p, ey1p, ez1p;   // level-1 E at plane p-1
    V hx1p, hy1p, hz1p;   // level-1 H at plane p-1
    V hx2p, hy2p;         // level-2 H at plane p-2
    // level-1 CPML memory at plane p-1 (H terms 0, 1; E terms 0, 1 per axis)
    V yH0, yH1, yE0, yE1, zH0, zH1, zE0, zE1, xH0, xH1, xE0, xE1;
};

struct RingPos {
    int s0, s1;
    uint32_t ph1;
};

// element e of lane src's vector (every lane of the warp takes part)
__device__ __forceinline__ float shfl_elem(float v, int src, int) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_elem(float4 v, int src, int e) {
    const float x = __shfl_sync(0xffffffffu, v.x, src), y = __shfl_sync(0xffffffffu, v.y, src);
    const float z = __shfl_sync(0xffffffffu, v.z, src), w = __shfl_sync(0xffffffffu, v.w, src);
    return e == 0 ? x : e == 1 ? y : e == 2 ? z : w;
}

// The records of plane q of the warp's row from position pc of the block's
// list (every row warp walks the list; a warp serves its own row's records
// from the level-1 E of plane q it holds, column col in lane col / VW);
// returns the new position.  Only the instances of blocks with records (REC)
// carry it.
template <int VW, typename V>
__device__ __forceinline__ int serve_records(const int4 *__restrict__ prec, int pend, int pc, int q, int row, int ib,
                                          const V &ex, const V &ey, const V &ez, float *pbuf) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int i = pc + lane;
        const bool live = i < pend;
        const int4 r = live ? prec[i] : make_int4(0, 0, 0, 0);
        const bool now = live && r.x == q;   // (q is -1 .. -3 in the first iterations of the bottom chunk)
        const unsigned bal = __ballot_sync(0xffffffffu, now);
        if (bal) {
            const int col = r.z - ib, c = r.w & 3;
            // (the host assigns a record to the block that owns its cell; a
            // record outside the block's columns is skipped, never read out of range)
            const bool mine = now && r.y == row && col >= 0 && col < 32 * VW;
            const int src = mine ? col / VW : lane, e = mine ? col % VW : 0;
            const float vx = shfl_elem(ex, src, e), vy = shfl_elem(ey, src, e), vz = shfl_elem(ez, src, e);
            if (mine) pbuf[r.w >> 2] = c == 0 ? vx : c == 1 ? vy : vz;
        }
        const int cnt = __popc(bal);
        pc += cnt;
        if (cnt < 32) return pc;
    }
}

// a row warp's signal: its lanes' shared stores before one arrival
__device__ __forceinline__ void signal(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// a row warp's wait expired: record it and stop (the warps that wait for
// this one give up in turn; the refill warp lets the copies in flight land)
__device__ __forceinline__ bool fail(const Args &A) {
    if ((threadIdx.x & 31) == 0) atomicOr(A.flags, 1);
    return false;
}

// The refill warp (one thread): planes 0 .. ns-1 into the empty ring, then
// plane r into stage r % ns once every row warp is done with plane r - ns.
template <int VW>
__device__ __forceinline__ void refill(const Args &A, const Maps &M, const Blk &B, Bars *bar, float *ring) {
    for (int r = 0; r < B.ns && r < B.nplanes; ++r) issue_plane<VW>(A, M, B, ring + r * B.stage, &bar->full[r], r);
    for (int r = B.ns; r < B.nplanes; ++r) {
        const int s = r % B.ns;
        if (!mbar_wait(&bar->empty[s], ((r - B.ns) / B.ns) & 1)) {
            // a row warp stopped: let the copies in flight (planes r-ns ..
            // r-1) land before the block ends; one that does not land within
            // these waits may land after it: flag bit 8 (the handle's status
            // is sticky)
            atomicOr(A.flags, 1);
            for (int t = r - B.ns; t < r; ++t) {
                bool landed = false;
                for (int n = 0; n < 4 && !landed; ++n) landed = mbar_wait(&bar->full[t % B.ns], (t / B.ns) & 1);
                if (!landed) atomicOr(A.flags, 8);
            }
            return;
        }
        issue_plane<VW>(A, M, B, ring + s * B.stage, &bar->full[s], r);
    }
}

template <int VW, bool HX, bool HY, bool HZ, bool MASK, bool REC>
__device__ __forceinline__ bool plane(const Args &A, const Maps &M, const Lane<VW> &L, const Blk &B, Bars *bar,
                                      float *ring, float *X, const float *CT, int rel, RingPos &rp,
                                      State<typename Vec<VW>::T> &S, int &pc) {
    typedef typename Vec<VW>::T V;
    typedef Geo<VW> G;
    constexpr int TXC = G::TXC, BOX = G::BOX, XROW = G::XROW, XBUF = G::XBUF, CX = G::CX, CY = G::CY, CZ = G::CZ;
    const Grid &g = A.g;
    const Cpml &pm = A.pm;
    const int w = L.w;
    const int p = B.kstart + rel, q = p - 1;
    const float kH = A.kH, kE = A.kE;
    constexpr bool STAGE_IN_B = HX || HY || HZ;   // B reads E psi from the stage
    bool ok = true;
    if (rel == 0) ok = mbar_wait(&bar->full[0], 0);
    ok = ok && mbar_wait(&bar->full[rp.s1], rp.ph1);
    if (__any_sync(FULL, !ok)) return fail(A);
    const float *s0 = ring + rp.s0 * B.stage;   // plane p
    const float *s1 = ring + rp.s1 * B.stage;   // plane p+1
    // A's buffer alternates with the plane; B's and C's are single
    float *XA = X + (rel & 1) * XBUF, *XB = X + 2 * XBUF, *XC = X + 3 * XBUF;
    const int bc0 = VW * L.lane;
    const int lzp = (HZ && p >= 0 && p < g.nz) ? slab_cell(p, g.nz, pm.P) : -1;
    const int lzq = (HZ && q >= 0 && q < g.nz) ? slab_cell(q, g.nz, pm.P) : -1;
    const V z4 = vzero<V>();
    const bool yl = HY && L.ly >= 0;
    const float *PY = s0 + B.yo + (L.ly - B.l0) * TXC + bc0;
    const float *PZ = s0 + B.zo + w * TXC + bc0;
    const float *PX = s0 + B.xo + L.xs + w * A.xbw;
    const int XA4 = B.nxb * B.xb;   // floats per x psi array in a stage
    Masks<typename Vec<VW>::U> mp, mq;
    if (MASK) mp = masks<VW>(L, p, g.nz);

    // ---- A: level-1 H at plane p (rows j0-2 .. j0+TY) ----
    const V ex0 = ldv<V>(s0 + 0 * BOX + w * TXC + bc0);
    const V ey0 = ldv<V>(s0 + 1 * BOX + w * TXC + bc0);
    const V ez0 = ldv<V>(s0 + 2 * BOX + w * TXC + bc0);
    V hx1, hy1, hz1;
    V yH0 = z4, yH1 = z4, zH0 = z4, zH1 = z4, xH0 = z4, xH1 = z4;
    {
        const V hx = ldv<V>(s0 + 3 * BOX + w * TXC + bc0);
        const V hy = ldv<V>(s0 + 4 * BOX + w * TXC + bc0);
        const V hz = ldv<V>(s0 + 5 * BOX + w * TXC + bc0);
        const V exU = ldv<V>(s0 + 0 * BOX + (w + 1) * TXC + bc0);   // row j+1
        const V ezU = ldv<V>(s0 + 2 * BOX + (w + 1) * TXC + bc0);
        const V exN = ldv<V>(s1 + 0 * BOX + w * TXC + bc0);         // plane p+1
        const V eyN = ldv<V>(s1 + 1 * BOX + w * TXC + bc0);
        const float eyR = __shfl_down_sync(FULL, first(ey0), 1);             // column +4 (lane 31: unused)
        const float ezR = __shfl_down_sync(FULL, first(ez0), 1);
        V dyEz = ezU - ez0, dzEy = eyN - ey0;                      // Hx
        V dzEx = exN - ex0, dxEz = right(ez0, ezR) - ez0;          // Hy
        V dxEy = right(ey0, eyR) - ey0, dyEx = exU - ex0;          // Hz
        if (yl) {
            const float a = CT[CY + w], b = CT[CY + BR + w];
            yH0 = ldv<V>(PY);
            yH1 = ldv<V>(PY + BOX);
            dyEz = cpmls(yH0, a, b, dyEz);
            dyEx = cpmls(yH1, a, b, dyEx);
        }
        if (HZ && lzp >= 0) {
            const float a = CT[CZ + rel], b = CT[CZ + A.zt + rel];
            zH0 = ldv<V>(PZ);
            zH1 = ldv<V>(PZ + BOX);
            dzEy = cpmls(zH0, a, b, dzEy);
            dzEx = cpmls(zH1, a, b, dzEx);
        }
        if (HX) {
            const V a = ldv<V>(CT + CX + bc0), b = ldv<V>(CT + CX + TXC + bc0);
            xH0 = L.xl ? ldv<V>(PX) : z4;
            xH1 = L.xl ? ldv<V>(PX + XA4) : z4;
            dxEz = cpmlv(xH0, a, b, dxEz);
            dxEy = cpmlv(xH1, a, b, dxEy);
        }
        hx1 = keep<MASK>(axpy(hx, -kH, dyEz - dzEy), mp.hx);
        hy1 = keep<MASK>(axpy(hy, -kH, dzEx - dxEz), mp.hy);
        hz1 = keep<MASK>(axpy(hz, -kH, dxEy - dyEx), mp.hz);
        stv(XA + w * XROW + bc0, hx1);
        stv(XA + w * XROW + TXC + bc0, hz1);
    }
    // B's rows of the warp above (level-1 E of plane q, written in the last
    // iteration's D) before this warp's A rows are signalled: the warp above
    // cannot finish this iteration before then, so that barrier is never two
    // phases ahead of this wait; it also tells this warp that the warp above
    // is done with the A and C rows it rewrites
    if (w + 1 < NWR && rel >= 1 && __any_sync(FULL, !mbar_wait(&bar->xb[w + 1], (rel - 1) & 1)))
        return fail(A);
    signal(&bar->xa[rel & 1][w]);
    // the warp is done with stage p (read by A, and by B where it carries psi)
    if (!STAGE_IN_B) signal(&bar->empty[rp.s0]);

    // detector records of plane q of the warp's row: its level-1 E are the
    // warp's registers of the last iteration; the records of a plane are
    // contiguous in the block's sorted list
    if (REC) pc = serve_records<VW>(A.prec, B.pend, pc, q, L.j, B.i0 - 4, S.ex1p, S.ey1p, S.ez1p, A.pbuf);

    // ---- B: level-1 E at plane p (rows j0-1 .. j0+TY) ----
    V ex1 = z4, ey1 = z4, ez1 = z4;
    V yE0 = z4, yE1 = z4, zE0 = z4, zE1 = z4, xE0 = z4, xE1 = z4;
    if (w >= 1) {
        // A's rows of the warp below
        if (__any_sync(FULL, !mbar_wait(&bar->xa[rel & 1][w - 1], (rel >> 1) & 1))) return fail(A);
        const V hzD = ldv<V>(XA + (w - 1) * XROW + TXC + bc0);   // row j-1
        const V hxD = ldv<V>(XA + (w - 1) * XROW + bc0);
        const float hzL = __shfl_up_sync(FULL, last(hz1), 1);           // column -1 (lane 0: unused)
        const float hyL = __shfl_up_sync(FULL, last(hy1), 1);
        V dyHz = hz1 - hzD, dzHy = hy1 - S.hy1p;                  // Ex
        V dzHx = hx1 - S.hx1p, dxHz = hz1 - left(hz1, hzL);       // Ey
        V dxHy = hy1 - left(hy1, hyL), dyHx = hx1 - hxD;          // Ez
        if (yl) {
            const float a = CT[CY + 2 * BR + w], b = CT[CY + 3 * BR + w];
            yE0 = ldv<V>(PY + 2 * BOX);
            yE1 = ldv<V>(PY + 3 * BOX);
            dyHz = cpmls(yE0, a, b, dyHz);
            dyHx = cpmls(yE1, a, b, dyHx);
        }
        if (HZ && lzp >= 0) {
            const float a = CT[CZ + 2 * A.zt + rel], b = CT[CZ + 3 * A.zt + rel];
            zE0 = ldv<V>(PZ + 2 * BOX);
            zE1 = ldv<V>(PZ + 3 * BOX);
            dzHy = cpmls(zE0, a, b, dzHy);
            dzHx = cpmls(zE1, a, b, dzHx);
        }
        if (HX) {
            const V a = ldv<V>(CT + CX + 2 * TXC + bc0), b = ldv<V>(CT + CX + 3 * TXC + bc0);
            xE0 = L.xl ? ldv<V>(PX + 2 * XA4) : z4;
            xE1 = L.xl ? ldv<V>(PX + 3 * XA4) : z4;
            dxHz = cpmlv(xE0, a, b, dxHz);
            dxHy = cpmlv(xE1, a, b, dxHy);
        }
        ex1 = axpy(ex0, kE, dyHz - dzHy);
        ey1 = axpy(ey0, kE, dzHx - dxHz);
        ez1 = axpy(ez0, kE, dxHy - dyHx);
        if (B.src_blk) add_source(ez1, A.src, A.ss1, L.c0, L.j, p);
        ex1 = keep<MASK>(ex1, mp.ex);
        ey1 = keep<MASK>(ey1, mp.ey);
        ez1 = keep<MASK>(ez1, mp.ez);
    }

    if (STAGE_IN_B) signal(&bar->empty[rp.s0]);

    // ---- C: level-2 H at plane q = p-1 (rows j0-1 .. j0+TY-1) ----
    V hx2 = z4, hy2 = z4, hz2 = z4;
    if (MASK) mq = masks<VW>(L, q, g.nz);
    if (p >= B.k0 && w >= 1 && w <= TY + 1) {
        const V exU = ldv<V>(XB + (w + 1) * XROW + bc0);         // level-1 E of plane q, row j+1
        const V ezU = ldv<V>(XB + (w + 1) * XROW + TXC + bc0);
        const float eyR = __shfl_down_sync(FULL, first(S.ey1p), 1);
        const float ezR = __shfl_down_sync(FULL, first(S.ez1p), 1);
        V dyEz = ezU - S.ez1p, dzEy = ey1 - S.ey1p;
        V dzEx = ex1 - S.ex1p, dxEz = right(S.ez1p, ezR) - S.ez1p;
        V dxEy = right(S.ey1p, eyR) - S.ey1p, dyEx = exU - S.ex1p;
        if (yl) {
            const float a = CT[CY + w], b = CT[CY + BR + w];
            dyEz = cpmls(S.yH0, a, b, dyEz);
            dyEx = cpmls(S.yH1, a, b, dyEx);
        }
        if (HZ && lzq >= 0) {
            const float a = CT[CZ + rel - 1], b = CT[CZ + A.zt + rel - 1];
            dzEy = cpmls(S.zH0, a, b, dzEy);
            dzEx = cpmls(S.zH1, a, b, dzEx);
        }
        if (HX) {
            const V a = ldv<V>(CT + CX + bc0), b = ldv<V>(CT + CX + TXC + bc0);
            dxEz = cpmlv(S.xH0, a, b, dxEz);
            dxEy = cpmlv(S.xH1, a, b, dxEy);
        }
        hx2 = keep<MASK>(axpy(S.hx1p, -kH, dyEz - dzEy), mq.hx);
        hy2 = keep<MASK>(axpy(S.hy1p, -kH, dzEx - dxEz), mq.hy);
        hz2 = keep<MASK>(axpy(S.hz1p, -kH, dxEy - dyEx), mq.hz);
        stv(XC + w * XROW + bc0, hx2);
        stv(XC + w * XROW + TXC + bc0, hz2);
        if (L.own && q >= B.k0 && q < B.k1) {
            const unsigned o = (unsigned)L.c0 + (unsigned)L.j * (unsigned)g.pitch + (unsigned)q * (unsigned)g.plane;
            stw<MASK>(A.out[3] + o, hx2, L.nval);
            stw<MASK>(A.out[4] + o, hy2, L.nval);
            stw<MASK>(A.out[5] + o, hz2, L.nval);
            if (yl) {
                const unsigned oy = L.yoff + (unsigned)q * (unsigned)(pm.W * g.pitch);
                stw<MASK>(pm.hout[1][0] + oy, S.yH0, L.nval);
                stw<MASK>(pm.hout[1][1] + oy, S.yH1, L.nval);
            }
            if (HZ && lzq >= 0) {
                const unsigned oz = L.zoff + (unsigned)lzq * (unsigned)(g.ny * g.pitch);
                stw<MASK>(pm.hout[2][0] + oz, S.zH0, L.nval);
                stw<MASK>(pm.hout[2][1] + oz, S.zH1, L.nval);
            }
            if (HX && L.xl) {
                const unsigned ox = L.xoff + (unsigned)q * (unsigned)A.xplane;
                stw<MASK>(pm.hout[0][0] + ox, S.xH0, L.nval);
                stw<MASK>(pm.hout[0][1] + ox, S.xH1, L.nval);
            }
        }
    }
    signal(&bar->xc[w]);

    // ---- D: level-2 E at plane q (owned rows); level-1 E rows for the next C ----
    // C's rows of the warp below; every warp from the third up waits for them,
    // which also tells it that the warp below is done with the B rows it
    // rewrites at the end of D
    if (w >= 2 && __any_sync(FULL, !mbar_wait(&bar->xc[w - 1], rel & 1))) return fail(A);
    if (p >= B.k0 + 1 && w >= 2 && w <= TY + 1) {
        const V hzD = ldv<V>(XC + (w - 1) * XROW + TXC + bc0);
        const V hxD = ldv<V>(XC + (w - 1) * XROW + bc0);
        const float hzL = __shfl_up_sync(FULL, last(hz2), 1);
        const float hyL = __shfl_up_sync(FULL, last(hy2), 1);
        V dyHz = hz2 - hzD, dzHy = hy2 - S.hy2p;
        V dzHx = hx2 - S.hx2p, dxHz = hz2 - left(hz2, hzL);
        V dxHy = hy2 - left(hy2, hyL), dyHx = hx2 - hxD;
        if (yl) {
            const float a = CT[CY + 2 * BR + w], b = CT[CY + 3 * BR + w];
            dyHz = cpmls(S.yE0, a, b, dyHz);
            dyHx = cpmls(S.yE1, a, b, dyHx);
        }
        if (HZ && lzq >= 0) {
            const float a = CT[CZ + 2 * A.zt + rel - 1], b = CT[CZ + 3 * A.zt + rel - 1];
            dzHy = cpmls(S.zE0, a, b, dzHy);
            dzHx = cpmls(S.zE1, a, b, dzHx);
        }
        if (HX) {
            const V a = ldv<V>(CT + CX + 2 * TXC + bc0), b = ldv<V>(CT + CX + 3 * TXC + bc0);
            dxHz = cpmlv(S.xE0, a, b, dxHz);
            dxHy = cpmlv(S.xE1, a, b, dxHy);
        }
        V ex2 = axpy(S.ex1p, kE, dyHz - dzHy);
        V ey2 = axpy(S.ey1p, kE, dzHx - dxHz);
        V ez2 = axpy(S.ez1p, kE, dxHy - dyHx);
        if (L.own && q < B.k1) {
            if (B.src_blk) add_source(ez2, A.src, A.ss2, L.c0, L.j, q);
            const unsigned o = (unsigned)L.c0 + (unsigned)L.j * (unsigned)g.pitch + (unsigned)q * (unsigned)g.plane;
            stw<MASK>(A.out[0] + o, keep<MASK>(ex2, mq.ex), L.nval);
            stw<MASK>(A.out[1] + o, keep<MASK>(ey2, mq.ey), L.nval);
            stw<MASK>(A.out[2] + o, keep<MASK>(ez2, mq.ez), L.nval);
            if (yl) {
                const unsigned oy = L.yoff + (unsigned)q * (unsigned)(pm.W * g.pitch);
                stw<MASK>(A.eout[1][0] + oy, S.yE0, L.nval);
                stw<MASK>(A.eout[1][1] + oy, S.yE1, L.nval);
            }
            if (HZ && lzq >= 0) {
                const unsigned oz = L.zoff + (unsigned)lzq * (unsigned)(g.ny * g.pitch);
                stw<MASK>(A.eout[2][0] + oz, S.zE0, L.nval);
                stw<MASK>(A.eout[2][1] + oz, S.zE1, L.nval);
            }
            if (HX && L.xl) {
                const unsigned ox = L.xoff + (unsigned)q * (unsigned)A.xplane;
                stw<MASK>(A.eout[0][0] + ox, S.xE0, L.nval);
                stw<MASK>(A.eout[0][1] + ox, S.xE1, L.nval);
            }
        }
    }
    // level-1 Ex, Ez of plane p for the next iteration's C of the warp below
    if (w >= 1) {
        stv(XB + w * XROW + bc0, ex1);
        stv(XB + w * XROW + TXC + bc0, ez1);
    }
    signal(&bar->xb[w]);
    // carry to the next plane
    S.ex1p = ex1; S.ey1p = ey1; S.ez1p = ez1;
    S.hx1p = hx1; S.hy1p = hy1; S.hz1p = hz1;
    S.hx2p = hx2; S.hy2p = hy2;
    S.yH0 = yH0; S.yH1 = yH1; S.yE0 = yE0; S.yE1 = yE1;
    S.zH0 = zH0; S.zH1 = zH1; S.zE0 = zE0; S.zE1 = zE1;
    S.xH0 = xH0; S.xH1 = xH1; S.xE0 = xE0; S.xE1 = xE1;
    rp.s0 = rp.s1;
    rp.s1 = rp.s1 + 1;
    if (rp.s1 == B.ns) {
        rp.s1 = 0;
        rp.ph1 ^= 1u;
    }
    return true;
}

template <int VW, bool HX, bool HY, bool HZ, bool MASK, bool REC>
__device__ __forceinline__ void march(const Args &A, const Maps &M, const Lane<VW> &L, const Blk &B, Bars *bar,
                                      float *ring, float *X, const float *CT) {
    typedef typename Vec<VW>::T V;
    State<V> S;
    const V z4 = vzero<V>();
    S.ex1p = S.ey1p = S.ez1p = S.hx1p = S.hy1p = S.hz1p = S.hx2p = S.hy2p = z4;
    S.yH0 = S.yH1 = S.yE0 = S.yE1 = S.zH0 = S.zH1 = S.zE0 = S.zE1 = S.xH0 = S.xH1 = S.xE0 = S.xE1 = z4;
    RingPos rp{0, 1, 0u};   // two stages at least
    int pc = B.pbeg;
    for (int rel = 0; rel + 1 < B.nplanes; ++rel)
        if (!plane<VW, HX, HY, HZ, MASK, REC>(A, M, L, B, bar, ring, X, CT, rel, rp, S, pc)) return;
}

// the instance of a block's case: which psi boxes it carries, whether it
// meets a face of the grid
template <int VW, bool HX, bool HY, bool HZ>
__device__ __forceinline__ void march_edge(bool edge, const Args &A, const Maps &M, const Lane<VW> &L, const Blk &B,
                                           Bars *bar, float *ring, float *X, const float *CT) {
    // blocks with detector records run an instance with the record service
    if (B.pbeg < B.pend) {
        if (edge) march<VW, HX, HY, HZ, true, true>(A, M, L, B, bar, ring, X, CT);
        else march<VW, HX, HY, HZ, false, true>(A, M, L, B, bar, ring, X, CT);
    } else {
        if (edge) march<VW, HX, HY, HZ, true, false>(A, M, L, B, bar, ring, X, CT);
        else march<VW, HX, HY, HZ, false, false>(A, M, L, B, bar, ring, X, CT);
    }
}
template <int VW, bool HX, bool HY>
__device__ __forceinline__ void march_z(bool hz, bool edge, const Args &A, const Maps &M, const Lane<VW> &L,
                                        const Blk &B, Bars *bar, float *ring, float *X, const float *CT) {
    if (hz) march_edge<VW, HX, HY, true>(edge, A, M, L, B, bar, ring, X, CT);
    else march_edge<VW, HX, HY, false>(edge, A, M, L, B, bar, ring, X, CT);
}

// one block of the launch: tile column T, tile row ty
template <int VW>
__device__ __forceinline__ void run_block(const Args &A, const Maps &M, const TileCol T, int ty) {
    typedef Geo<VW> G;
    constexpr int TXC = G::TXC, BOX = G::BOX, FIELDS = G::FIELDS, XBUF = G::XBUF, CX = G::CX,
                  CY = G::CY, CZ = G::CZ;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Bars *bar = reinterpret_cast<Bars *>(smem_raw);
    float *X = reinterpret_cast<float *>(smem_raw + BAR_BYTES);   // exchange rows
    float *CT = X + 4 * XBUF;                                      // CPML coefficients
    float *ring = X + G::head_floats(A.zt);                        // stage ring

    const Grid &g = A.g;
    const Cpml &pm = A.pm;
    const int P = pm.P;
    const int tid = threadIdx.x;
    Blk B;
    const int tile = (int)blockIdx.x;
    B.i0 = T.i0;
    B.iend = T.i0 + T.w;
    B.j0 = ty * TY;
    {
        // chunk-major launch order: the middle chunks first, the two layer
        // chunks last
        const int c = (int)blockIdx.y;
        if (c < A.m) {
            B.k0 = A.za + c * A.cm;
            B.k1 = min(A.zb, B.k0 + A.cm);
        } else if (c == A.m && A.za > 0) {
            B.k0 = 0;
            B.k1 = A.za;
        } else {
            B.k0 = A.zb;
            B.k1 = g.nz;
        }
        B.hz = P > 0 && c >= A.m;
        const int b = c * A.tiles_x * A.tiles_y + tile;
        B.pbeg = A.pidx ? A.pidx[b] : 0;
        B.pend = A.pidx ? A.pidx[b + 1] : 0;
    }
    B.kstart = B.k0 - 2;
    B.nplanes = B.k1 - B.k0 + 4;   // input planes k0-2 .. k1+1
    B.src_blk = A.src.active && B.i0 - 4 <= A.src.ic + A.src.L && B.i0 + TXC - 5 >= A.src.ic - A.src.L &&
                B.j0 - 2 <= A.src.jc + A.src.L && B.j0 + TY + 1 >= A.src.jc - A.src.L;
    B.hx = B.hy = false;
    B.l0 = 0;
    B.xlo = B.xhi = -1;
    B.nxb = 0;
    B.xb = (A.xbw * BR + 31) / 32 * 32;
    if (P > 0) {
        const int ilo = max(B.i0 - 4, 0), ihi = min(B.i0 + TXC - 5, g.nx - 1);
        if (VW == 1 && ilo <= P) B.xlo = B.nxb++;
        if (VW == 1 && ihi >= g.nx - P) B.xhi = B.nxb++;
        B.hx = B.nxb > 0;
        int lmin = 1 << 30;
        for (int j = max(B.j0 - 2, 0); j < min(B.j0 + TY + 2, g.ny); ++j) {
            const int l = slab_cell(j, g.ny, P);
            if (l >= 0 && l < lmin) lmin = l;
        }
        B.hy = lmin < (1 << 30);
        B.l0 = B.hy ? lmin : 0;
    }
    B.xo = FIELDS;
    B.yo = B.xo + 4 * B.nxb * B.xb;
    B.zo = B.yo + (B.hy ? 4 * BOX : 0);
    B.stage = B.zo + (B.hz ? 4 * BOX : 0);
    B.ns = min(NSMAX, (A.smem_floats - G::head_floats(A.zt)) / B.stage);

    if (tid == 0) {
        for (int s = 0; s < B.ns; ++s) {
            mbar_init(&bar->full[s], 1);
            mbar_init(&bar->empty[s], NWR);
        }
        for (int w = 0; w < NWR; ++w) {
            mbar_init(&bar->xa[0][w], 1);
            mbar_init(&bar->xa[1][w], 1);
            mbar_init(&bar->xb[w], 1);
            mbar_init(&bar->xc[w], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (P > 0) {
        for (int t = tid; t < TXC; t += NT) {
            const int i = B.i0 - 4 + t;
            const bool in = i >= 0 && i < g.nx;
            CT[CX + t] = in ? pm.aH[0][i] : 0.f;
            CT[CX + TXC + t] = in ? pm.bH[0][i] : 0.f;
            CT[CX + 2 * TXC + t] = in ? pm.aE[0][i] : 0.f;
            CT[CX + 3 * TXC + t] = in ? pm.bE[0][i] : 0.f;
        }
        for (int t = tid; t < BR; t += NT) {
            const int j = B.j0 - 2 + t;
            const bool in = j >= 0 && j < g.ny;
            CT[CY + t] = in ? pm.aH[1][j] : 0.f;
            CT[CY + BR + t] = in ? pm.bH[1][j] : 0.f;
            CT[CY + 2 * BR + t] = in ? pm.aE[1][j] : 0.f;
            CT[CY + 3 * BR + t] = in ? pm.bE[1][j] : 0.f;
        }
        if (B.hz)
            for (int t = tid; t < A.zt; t += NT) {
                const int k = B.kstart + t;
                const bool in = k >= 0 && k < g.nz;
                CT[CZ + t] = in ? pm.aH[2][k] : 0.f;
                CT[CZ + A.zt + t] = in ? pm.bH[2][k] : 0.f;
                CT[CZ + 2 * A.zt + t] = in ? pm.aE[2][k] : 0.f;
                CT[CZ + 3 * A.zt + t] = in ? pm.bE[2][k] : 0.f;
            }
    }
    __syncthreads();   // the only block barrier: barriers and coefficients are set
    if (tid >= 32 * NWR) {
        if (tid == 32 * NWR) refill<VW>(A, M, B, bar, ring);
        return;
    }

    Lane<VW> L;
    L.lane = tid & 31;
    L.w = tid >> 5;
    L.c0 = B.i0 - 4 + VW * L.lane;
    L.j = B.j0 - 2 + L.w;
    L.rowin = L.j >= 0 && L.j < g.ny;
    {
        typedef typename Vec<VW>::T V;
        unsigned m[4];
        for (int e = 0; e < VW; ++e) m[e] = (L.c0 + e >= 0 && L.c0 + e < g.nx) ? 0xffffffffu : 0u;
        L.mcol = umask(m, V());
        if (L.c0 == 0) m[0] = 0u;
        L.mcol0 = umask(m, V());
    }
    L.nval = L.c0 >= 0 && L.c0 < g.nx ? min(VW, g.nx - L.c0) : 0;
    L.own = L.lane >= G::LO && L.lane <= G::HI && L.w >= 2 && L.w <= TY + 1 && L.rowin && L.nval > 0 &&
            L.c0 < B.iend;
    if (L.own) L.nval = min(L.nval, B.iend - L.c0);
    L.ly = (P > 0 && L.rowin) ? slab_cell(L.j, g.ny, P) : -1;
    L.xl = false;
    L.xs = L.xpos = 0;
    L.yoff = L.ly >= 0 ? (unsigned)psi_y(g, pm.W, L.c0, L.ly, 0) : 0u;
    L.zoff = (L.rowin && L.nval > 0) ? (unsigned)psi_z(g, pm.W, L.c0, L.j, 0) : 0u;
    if (B.hx && L.rowin && L.nval > 0) {
        if (B.xlo >= 0 && L.c0 < A.xlo4) {
            L.xl = true;
            L.xpos = L.c0;
            L.xs = B.xlo * B.xb + L.c0;
        } else if (B.xhi >= 0 && L.c0 >= A.xhb) {
            L.xl = true;
            L.xpos = A.xlo4 + L.c0 - A.xhb;
            L.xs = B.xhi * B.xb + (L.c0 - A.xhb);
        }
    }
    L.xoff = L.xl ? (unsigned)psi_x(g, P, L.xpos, L.j, 0) : 0u;

    // blocks whose computed region stays clear of the faces need no masks
    const bool edge = B.i0 - 4 < 1 || B.i0 + TXC - 5 > g.nx - 1 || B.j0 - 2 < 1 || B.j0 + TY > g.ny - 1 ||
                      B.k0 - 2 < 1 || B.k1 > g.nz - 1;
    if (VW == 1) {   // the narrow tiles of the x layers: always with masks
        if (B.hx) {
            if (B.hy) march_z<VW, true, true>(B.hz, true, A, M, L, B, bar, ring, X, CT);
            else march_z<VW, true, false>(B.hz, true, A, M, L, B, bar, ring, X, CT);
        } else {
            if (B.hy) march_z<VW, false, true>(B.hz, true, A, M, L, B, bar, ring, X, CT);
            else march_z<VW, false, false>(B.hz, true, A, M, L, B, bar, ring, X, CT);
        }
    } else {         // the wide tiles never meet an x layer
        if (B.hy) march_z<VW, false, true>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
        else march_z<VW, false, false>(B.hz, edge, A, M, L, B, bar, ring, X, CT);
    }
}

__global__ void __launch_bounds__(NT, 1) k_tb2(const Args A, const __grid_constant__ Maps M) {
    const int tile = (int)blockIdx.x;
    const int ty = tile / A.tiles_x;
    const TileCol T = tile_col(tile - ty * A.tiles_x, A.ta, A.tb, A.nl, A.nw, A.g.nx);
    if (T.vw == 1) run_block<1>(A, M, T, ty);
    else run_block<4>(A, M, T, ty);
}

constexpr CUtensorMapL2promotion kPromotion = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;

struct HostState {
    Maps maps;
    int ta, tb, nl, nw;                        // tile columns (tile_col)
    int tiles_x, tiles_y, za, zb, cm, m, zt, chunks, smem_floats;
    int xlo4, xhb, xbw;
    size_t smem;
    // detector records, rebuilt when the handle's detectors change
    int probe_ver;
    std::vector<int4> h_rec;
    std::vector<int> h_idx;
    int4 *d_rec;
    int *d_idx;
    float *d_pbuf;
};

// tile column of column i (tile_col inverted)
int tile_of(const HostState *st, int i, int nx) {
    i = std::min(std::max(i, 0), nx - 1);   // a readout cell outside the grid: the edge tile
    int tc;
    if (i < st->ta) tc = i / 24;
    else if (i < st->tb) tc = st->nl + (i - st->ta) / 120;
    else tc = st->nl + st->nw + (i - st->tb) / 24;
    return tc;
}

// chunk of plane k (the kernel's chunk decoding, inverted)
int chunk_of(const HostState *st, int k) {
    if (k < st->za) return st->m;
    if (k >= st->zb) return st->m + (st->za > 0 ? 1 : 0);
    return (k - st->za) / st->cm;
}

int build_records(fdtd_ctx *h, HostState *st) {
    cudaFree(st->d_rec);
    cudaFree(st->d_idx);
    cudaFree(st->d_pbuf);
    st->d_rec = nullptr;
    st->d_idx = nullptr;
    st->d_pbuf = nullptr;
    st->probe_ver = h->probe_ver;
    if (h->np == 0) return FDTD_OK;
    const int tiles = st->tiles_x * st->tiles_y;
    const int blocks = tiles * st->chunks;
    // the six cells of each detector's readout: Ex at i-1, i; Ey at j-1, j; Ez at k-1, k
    struct Rec { int b; int4 r; };
    std::vector<Rec> recs;
    recs.reserve(6 * (size_t)h->np);
    for (int t = 0; t < h->np; ++t) {
        const int i = h->h_ijk[3 * t], j = h->h_ijk[3 * t + 1], k = h->h_ijk[3 * t + 2];
        const int cell[6][4] = {{i - 1, j, k, 0}, {i, j, k, 0}, {i, j - 1, k, 1},
                                {i, j, k, 1},     {i, j, k - 1, 2}, {i, j, k, 2}};
        for (int s = 0; s < 6; ++s) {
            const int ci = cell[s][0], cj = cell[s][1], ck = cell[s][2];
            const int b = chunk_of(st, ck) * tiles + (cj / TY) * st->tiles_x + tile_of(st, ci, h->g.nx);
            recs.push_back({b, make_int4(ck, cj, ci, (6 * t + s) * 4 + cell[s][3])});
        }
    }
    std::stable_sort(recs.begin(), recs.end(),
                     [](const Rec &a, const Rec &b) { return a.b < b.b || (a.b == b.b && a.r.x < b.r.x); });
    st->h_rec.resize(recs.size());
    st->h_idx.assign(blocks + 1, 0);
    for (size_t n = 0; n < recs.size(); ++n) {
        st->h_rec[n] = recs[n].r;
        st->h_idx[recs[n].b + 1]++;
    }
    for (int b = 0; b < blocks; ++b) st->h_idx[b + 1] += st->h_idx[b];
    if (cudaMalloc(&st->d_rec, sizeof(int4) * recs.size()) != cudaSuccess ||
        cudaMalloc(&st->d_idx, sizeof(int) * (blocks + 1)) != cudaSuccess ||
        cudaMalloc(&st->d_pbuf, sizeof(float) * 6 * (size_t)h->np) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    if (cudaMemcpy(st->d_rec, st->h_rec.data(), sizeof(int4) * recs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(st->d_idx, st->h_idx.data(), sizeof(int) * (blocks + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    return FDTD_OK;
}

}  // namespace

const char *tb2_name(const fdtd_ctx *) { return "tblock2-120x8"; }

int tb2_prepare(fdtd_ctx *h) {
    typedef Geo<4> G4;
    typedef Geo<1> G1;
    const Grid &g = h->g;
    const int P = h->P;
    if (h->boundary == FDTD_MUR1) return FDTD_ERR_ARG;   // the Mur faces need E^{n+1} between the steps
    if ((unsigned long long)g.comp >= (1ull << 32) || g.pitch % 4 != 0) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    const int xlo4 = P > 0 ? psi_x_lo4(P) : 0, xhb = P > 0 ? psi_x_hb(g.nx, P) : 0;
    const int WX = P > 0 ? psi_x_row(g.nx, P) : 0;
    const int xbw = P > 0 ? (xlo4 > WX - xlo4 ? xlo4 : WX - xlo4) : 4;
    if (P > 0 && (g.nx < 2 * P + 8 || xbw > 256 || !h->epsi2)) return FDTD_ERR_ARG;
    EncodeTiled encode = encoder();
    if (!encode) return FDTD_ERR_CUDA;
    HostState *st = new (std::nothrow) HostState();
    if (!st) return FDTD_ERR_OOM;
    st->xlo4 = xlo4;
    st->xhb = xhb;
    st->xbw = xbw;
    bool ok = true;
    const int TXCW[2] = {G4::TXC, G1::TXC};   // box width of the wide and the narrow tiles
    for (int wd = 0; wd < 2; ++wd)
        for (int s = 0; s < 2; ++s)
            for (int c = 0; c < 6; ++c)
                ok = ok && encode3(encode, &st->maps.f[wd][s][c], h->fields[s] + (size_t)c * g.comp, g.nx + 1,
                                   g.ny + 1, g.nz + 1, g.pitch, g.plane, TXCW[wd], BR, kPromotion);
    if (P > 0) {
        // H psi sets follow the field set; E psi sets are psi_block's first
        // third and epsi2
        const size_t set = 2 * (h->psi_axis[0] + h->psi_axis[1] + h->psi_axis[2]);
        const int W = 2 * P + 1;
        for (int s = 0; s < 2; ++s) {
            size_t off = 0;
            for (int axis = 0; axis < 3; ++axis)
                for (int t = 0; t < 2; ++t) {
                    const float *hp = h->psi_block + set * (1 + s) + off;
                    const float *ep = (s == 0 ? h->psi_block : h->epsi2) + off;
                    off += h->psi_axis[axis];
                    for (int half = 0; half < 2; ++half) {
                        const float *base = half == 0 ? hp : ep;
                        const int a = 2 * half + t;
                        if (axis == 0)
                            ok = ok && encode3(encode, &st->maps.x[a][s], base, WX, g.ny, g.nz, WX,
                                               (cuuint64_t)g.ny * WX, xbw, BR, kPromotion);
                        for (int wd = 0; wd < 2 && axis > 0; ++wd) {
                            if (axis == 1)
                                ok = ok && encode3(encode, &st->maps.y[wd][a][s], base, g.nx, W, g.nz, g.pitch,
                                                   (cuuint64_t)W * g.pitch, TXCW[wd], BR, kPromotion);
                            else
                                ok = ok && encode3(encode, &st->maps.z[wd][a][s], base, g.nx, g.ny, W, g.pitch,
                                                   (cuuint64_t)g.ny * g.pitch, TXCW[wd], BR, kPromotion);
                        }
                    }
                }
        }
    }
    if (!ok) {
        delete st;
        return FDTD_ERR_CUDA;
    }
    // tile columns: narrow tiles over the x layers [0, a), [b, nx) (a, b
    // multiples of 4 with a - 2 > P and b + 1 < nx - P), wide tiles between;
    // a grid too narrow for a wide part is all narrow tiles
    if (P > 0) {
        st->ta = (P + 3 + 3) / 4 * 4;
        st->tb = (g.nx - P - 2) / 4 * 4;
        if (st->tb - st->ta < 24) {
            st->ta = st->tb = g.nx;
        } else {
            // a last wide tile of r < 120 columns costs a whole wide block:
            // move those columns to the narrow tiles where their last tiles
            // have room for them
            const int r = (st->tb - st->ta) % G4::TXO;
            const int room_l = (st->ta + 23) / 24 * 24 - st->ta;
            const int room_r = ((g.nx - st->tb + 23) / 24 * 24 - (g.nx - st->tb)) / 4 * 4;
            if (r > 0 && st->tb - st->ta > G4::TXO && r <= room_l + room_r) {
                const int dl = std::min(r, room_l);
                st->ta += dl;
                st->tb -= r - dl;
            }
        }
    } else {
        st->ta = st->tb = 0;
    }
    if (P == 0) {
        st->nl = 0;
        st->nw = (g.nx + G4::TXO - 1) / G4::TXO;
        st->tiles_x = st->nw;
        st->ta = 0;
        st->tb = g.nx;
    } else {
        st->nl = (st->ta + G1::TXO - 1) / G1::TXO;
        st->nw = (st->tb - st->ta + G4::TXO - 1) / G4::TXO;
        st->tiles_x = st->nl + st->nw + (g.nx - st->tb + G1::TXO - 1) / G1::TXO;
    }
    st->tiles_y = (g.ny + TY - 1) / TY;
    // z chunks: the planes of a middle chunk (k0-2 .. k1+1) stay clear of the
    // z layers, so only the two layer chunks [0, za), [zb, nz) carry z boxes;
    // a grid too short for a middle part is one layer chunk
    if (P > 0) {
        st->za = P + 3;
        st->zb = g.nz - P - 2;
        if (st->zb - st->za < 8) st->za = st->zb = g.nz;
    } else {
        st->za = 0;
        st->zb = g.nz;
    }
    // Middle chunks: the fewest waves x chunk length, with chunks of at most
    // CM_MAX planes.  The blocks of a wave march up z side by side and read
    // each other's halo rows; over a long march they drift apart by more
    // planes than L2 keeps, and the halo rows come from DRAM twice (measured:
    // 139 -> 147 Gcell/s on 384x384x1536 and 169 -> 181 on 640x640x2048 with
    // chunks of about 150 planes instead of 300-500; below 64 planes the
    // warm-up planes cost more than L2 saves).
    constexpr long long CM_MAX = 160;
    const int mid = st->zb - st->za;
    const long long sms = h->num_sms > 0 ? h->num_sms : 1;
    const long long tiles = (long long)st->tiles_x * st->tiles_y;
    long long m = 0, best = -1;
    const long long m_lo = std::max(1LL, (mid + CM_MAX - 1) / CM_MAX);
    const long long m_hi = std::max(m_lo, (long long)(mid / 16));
    if (mid > 0)
        for (long long mm = m_lo; mm <= m_hi; ++mm) {
            const long long cm = (mid + mm - 1) / mm;
            const long long cost = (tiles * mm + sms - 1) / sms * (cm + 7);
            if (best < 0 || cost < best) { best = cost; m = mm; }
        }
    st->cm = m > 0 ? (int)((mid + m - 1) / m) : 1;
    st->m = m > 0 ? (mid + st->cm - 1) / st->cm : 0;
    st->chunks = st->m + (st->za > 0 ? 1 : 0) + (st->zb < g.nz ? 1 : 0);
    const int layer = std::max(st->za, g.nz - st->zb);
    st->zt = P > 0 ? layer + 4 : 1;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const long long xb = (xbw * BR + 31) / 32 * 32;
    // largest stages: wide tiles with y and z boxes; narrow ones with two x
    // halves, y and z
    const long long big4 = G4::FIELDS + 8LL * G4::BOX;
    const long long big1 = G1::FIELDS + 8 * xb + 8LL * G1::BOX;
    const long long floats = (long long)max_smem / 4 - BAR_BYTES / 4;
    st->smem_floats = (int)floats;
    st->smem = 4 * (size_t)floats + BAR_BYTES;
    if (floats - G4::head_floats(st->zt) < 2 * big4 || floats - G1::head_floats(st->zt) < 2 * big1 ||
        cudaFuncSetAttribute(k_tb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem) != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FDTD_ERR_CUDA;
    }
    st->probe_ver = -1;
    h->tb2 = st;
    return FDTD_OK;
}

void tb2_release(fdtd_ctx *h) {
    HostState *st = static_cast<HostState *>(h->tb2);
    if (st) {
        cudaFree(st->d_rec);
        cudaFree(st->d_idx);
        cudaFree(st->d_pbuf);
    }
    delete st;
    h->tb2 = nullptr;
}

void launch_tb2(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->tb2);
    if (st->probe_ver != h->probe_ver) {
        const int rc = build_records(h, st);
        if (rc != FDTD_OK && h->status == FDTD_OK) h->status = rc;
    }
    const Grid &g = h->g;
    Args a;
    a.g = g;
    float *out = h->fields[h->cur ^ 1];
    for (int c = 0; c < 6; ++c) a.out[c] = out + (size_t)c * g.comp;
    a.pm = cpml_view(h);
    h->ecur ^= 1;   // the E psi set this pass writes
    const Cpml other = cpml_view(h);
    h->ecur ^= 1;
    for (int ax = 0; ax < 3; ++ax)
        for (int t = 0; t < 2; ++t) a.eout[ax][t] = other.e[ax][t];
    a.ta = st->ta;
    a.tb = st->tb;
    a.nl = st->nl;
    a.nw = st->nw;
    a.tiles_x = st->tiles_x;
    a.tiles_y = st->tiles_y;
    a.za = st->za;
    a.zb = st->zb;
    a.cm = st->cm;
    a.m = st->m;
    a.zt = st->zt;
    a.smem_floats = st->smem_floats;
    a.xlo4 = st->xlo4;
    a.xhb = st->xhb;
    a.xbw = st->xbw;
    a.xplane = g.ny * (h->P > 0 ? psi_x_row(g.nx, h->P) : 0);
    a.cur = h->cur;
    a.ecur = h->ecur;
    a.src = h->src;
    a.ss1 = source_window(h->src, h->steps);
    a.ss2 = source_window(h->src, h->steps + 1);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.flags = h->d_flags;
    a.prec = st->d_rec;
    a.pidx = st->d_idx;
    a.pbuf = st->d_pbuf;
    dim3 grid(st->tiles_x * st->tiles_y, st->chunks);
    k_tb2<<<grid, NT, st->smem, s>>>(a, st->maps);
}

float *tb2_probe_values(fdtd_ctx *h) {
    HostState *st = static_cast<HostState *>(h->tb2);
    return st ? st->d_pbuf : nullptr;
}

}  // namespace fdtd
