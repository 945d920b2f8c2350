// batch.cu -- many simulations in one persistent kernel (batch.h).
//
// Work queue.  Every step of every simulation is two kinds of items:
//   F: item = (simulation q, tile of 128 columns x 8 rows, z chunk of q): the
//      one-pass step of that tile (H^{n+1/2} and E^{n+1} with the shower's
//      current, Sec. III.A-B), the block body of the handle's tile path
//      (vtile_tile.cuh), with q's tensor maps;
//   M: item = (q, face, piece of MUR_PIECE face nodes) for the six Mur faces of
//      a Mur grid, and (q, detectors) for a grid with detectors: the boundary,
//      then the readout of E^{n+1} (the code of the handle's own Mur and
//      detector kernels).  An x face is a strided walk through memory (one
//      node per row), so faces are cut into pieces that many SMs share.
// The blocks (one per SM, all resident: a cooperative launch) take items from
// one atomic counter in the order (step, kind, simulation, item).  (Placing a
// simulation's M items a wave of F items after its own, for L2 hits on its
// faces, measured slower: the waits grew more than the reads shrank.)  An item
// waits only for its own simulation: an F item of step s for all F and M
// items of step s-1 of that simulation, an M item for all its F items of
// step s; completion is counted per simulation and kind.  A simulation thus
// runs its Mur faces and detectors, and starts its next step, while the
// blocks still finish other simulations' tiles: no grid-wide barrier inside a
// launch.  Every wait is for items taken earlier from the counter (by blocks
// that are running), so the launch cannot deadlock; each wait is bounded
// (FDTD_ERR_TIMEOUT when it gives up).  The numbers are those of the handle
// stepped on its tile path (fdtd_set_kernel 1), bit for bit.
// The kernel takes PEC and Mur grids: its tile arguments come from memory (a
// copy per item in shared memory), not from the parameter bank, and with them
// the CPML instances of the tile body need more registers than a block of
// nine warps has (168 per thread); a grid with CPML layers steps alone.
// Simulations keep their own ping-pong sets: in step s of a launch,
// simulation q reads set cur_q ^ (s & 1).  At the end of a launch block 0
// advances each descriptor's set index and step count, so that the captured
// graph can be replayed unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/batch.h"
#include "cell_update.cuh"
#include "fdtd_internal.h"
#include "vtile_tile.cuh"

using namespace fdtd;

namespace {

constexpr int MAX_STEPS_PER_LAUNCH = 64;
constexpr int NT = vt::NT;
constexpr int MUR_PIECE = 2048;   // face nodes per M item

// A simulation of the persistent kernel.
struct BSim {
    vt::Args a[2];         // tile arguments for field set 0 and 1 (ss and flags set per step)
    const vt::Maps *maps;  // its tensor maps (device copy)
    int tiles, items;      // tiles per chunk; F items (tiles x chunks)
    float mur;
    int mface[7];          // M items before face f (pieces of MUR_PIECE nodes); mface[6]: all faces
    Probes pr;
    int cur;
    long long n;           // steps done
};

struct BArgs {
    BSim *sims;
    int nsim;
    const int *fstart;     // [nsim + 1] prefix sums of F items
    const int *mstart;     // [nsim + 1] prefix sums of M items
    const int *seg;        // [nseg + 1] item order within a step: segment g holds items
                           // [seg[g], seg[g+1]) of kind and simulation segq[g] (2 q + 1 for M)
    const int *segq;
    int nseg;
    int steps;
    unsigned *ctr;         // [1 + 2 nsim] work counter, then F and M items done per simulation; zero at launch
    unsigned *bar;         // [2] barrier count and generation, zero at launch
    int *flags;
    long long spin;        // clock cycles a wait may take
};

// Wait (bounded by spin cycles; thread 0) until *c >= target.  False when the
// wait gave up (flag bit 1 set) or another block recorded a failure.
__device__ bool wait_count(const unsigned *c, unsigned target, int *flags, long long spin) {
    const volatile unsigned *v = c;
    if (*v >= target) return true;
    const long long t0 = clock64();
    while (*v < target) {
        if (*(volatile int *)flags) return false;
        if (clock64() - t0 > spin) {
            atomicOr(flags, 2);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Grid-wide barrier: arrive, then wait (bounded by spin cycles) for the
// generation to move.  A block whose wait gives up sets flag bit 1.  Returns
// false when the launch must stop: this wait gave up, or some block recorded
// a failure (a barrier or a pipeline wait) before arriving; every block that
// passes the barrier then sees that flag, so they leave together.
__device__ bool grid_sync(unsigned *bar, int *flags, long long spin) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > spin) {
                    atomicOr(flags, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (*(volatile int *)flags) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int find_sim(const int *start, int nsim, int it) {
    int lo = 0, hi = nsim - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(NT, 1) k_batch(BArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(16) vt::Args s_a;   // the item's tile arguments
    __shared__ int s_go, s_step, s_q, s_item;   // s_item: F item index, or -1 - M item index
    const int tid = threadIdx.x;
    const int fitems = A.fstart[A.nsim], mitems = A.mstart[A.nsim];   // per step
    // an earlier launch (or a block of this one) gave up: the simulations are
    // in an unknown state.  One read per block, so that its threads leave
    // together (thread 0 alone drives the work queue).
    __shared__ int s_stop;
    if (tid == 0) s_stop = *(volatile int *)A.flags;
    __syncthreads();
    if (s_stop) return;
    const unsigned per_step = (unsigned)(fitems + mitems);
    const unsigned total = per_step * (unsigned)A.steps;
    unsigned *doneF = A.ctr + 1, *doneM = A.ctr + 1 + A.nsim;
    for (;;) {
        if (tid == 0) {
            const unsigned it = atomicAdd(A.ctr, 1u);
            int ok = it < total;
            if (ok) {
                const int s = (int)(it / per_step), r = (int)(it % per_step);
                const int g = find_sim(A.seg, A.nseg, r);
                const bool f = (A.segq[g] & 1) == 0;
                const int q = A.segq[g] >> 1;
                const unsigned nf = (unsigned)(A.fstart[q + 1] - A.fstart[q]);
                const unsigned nm = (unsigned)(A.mstart[q + 1] - A.mstart[q]);
                // an F item: all of q's step s-1 done; an M item: q's F items of step s done
                ok = f ? wait_count(doneF + q, nf * s, A.flags, A.spin) && wait_count(doneM + q, nm * s, A.flags, A.spin)
                       : wait_count(doneF + q, nf * (s + 1), A.flags, A.spin);
                __threadfence();
                // the other blocks' stores of the fields, ahead of this block's tensor loads
                asm volatile("fence.proxy.async.global;" ::: "memory");
                s_step = s;
                s_q = q;
                s_item = f ? r - A.seg[g] : -1 - (r - A.seg[g]);
            }
            s_go = ok;
        }
        __syncthreads();
        if (!s_go) break;
        const int s = s_step, q = s_q, item = s_item;
        const BSim &S = A.sims[q];
        const int cur = S.cur ^ (s & 1);
        if (item >= 0) {
            // ---- F: a tile ----
            {
                static_assert(sizeof(vt::Args) % 8 == 0, "Args copied in 8-byte words");
                const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&S.a[cur]);
                unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_a);
                for (int w = tid; w < (int)(sizeof(vt::Args) / 8); w += NT) dst[w] = src[w];
            }
            __syncthreads();
            if (tid == 0) {
                s_a.ss = source_window(s_a.src, S.n + s);
                s_a.flags = A.flags;
            }
            __syncthreads();
            const int ns = vt::tile_block<false>(s_a, *S.maps, item % S.tiles, item / S.tiles, smem_raw);
            vt::end_tile(smem_raw, ns);
        } else {
            // ---- M: a piece of a Mur face, or the detectors, of E^{n+1} ----
            const vt::Args &a = S.a[cur];
            const Grid &g = a.g;
            const float *in = S.a[cur ^ 1].oex;   // E^n: the set this step reads
            float *out = a.oex;                   // E^{n+1}
            const int m = -1 - item;
            if (m < S.mface[6]) {
                // a piece of face f: (a, b) over (j, k), (i, k) or (i, j)
                int f = 0;
                while (m >= S.mface[f + 1]) ++f;
                const int ax = f >> 1;
                const int na = (ax == 0 ? g.ny : g.nx) + 1, nb = (ax == 2 ? g.ny : g.nz) + 1;
                const int c0 = (m - S.mface[f]) * MUR_PIECE, c1 = min(c0 + MUR_PIECE, na * nb);
                for (int c = c0 + tid; c < c1; c += NT) mur_cell(g, in, out, S.mur, f, c % na, c / na);
            } else {
                const Probes &p = S.pr;
                for (int t = tid; t < p.n; t += NT) {
                    const int i = p.ijk[3 * t], j = p.ijk[3 * t + 1], k = p.ijk[3 * t + 2];
                    const long long c = gidx(g, i, j, k);
                    const float *Ex = out, *Ey = out + g.comp, *Ez = out + 2 * g.comp;
                    const float ex = 0.5f * (Ex[c - 1] + Ex[c]);
                    const float ey = 0.5f * (Ey[c - g.pitch] + Ey[c]);
                    const float ez = 0.5f * (Ez[c - g.plane] + Ez[c]);
                    float *o = p.trace + ((long long)t * p.max_steps + S.n + s) * 2;
                    o[0] = ez;
                    o[1] = p.cxy[2 * t] * ex + p.cxy[2 * t + 1] * ey;
                }
            }
        }
        // the item's stores, then its count (release to the items that wait for it)
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(item >= 0 ? doneF + q : doneM + q, 1u);
    }
    // every item of the launch done before the descriptors advance
    if (!grid_sync(A.bar, A.flags, A.spin)) return;
    if (blockIdx.x == 0)
        for (int q = tid; q < A.nsim; q += NT) {
            A.sims[q].cur ^= A.steps & 1;
            A.sims[q].n += A.steps;
        }
}

}  // namespace

// Streams over which the simulations that step alone are spread (their
// launches rarely fill the GPU one at a time).
constexpr int SOLO_STREAMS = 8;

struct fdtd_batch {
    std::vector<fdtd_t> sims;
    int dev, sms;
    cudaStream_t stream;
    cudaEvent_t ev;
    BSim *d_sims;
    vt::Maps *d_maps;
    int *d_fstart, *d_mstart, *d_seg, *d_segq;
    int nseg;
    unsigned *d_ctr, *d_bar;
    int *d_flags;
    int chunk_planes, steps_per_launch;
    size_t smem;           // dynamic shared memory of the persistent kernel
    long long floats;      // its floats after the ring barriers
    long long solo_cells;  // simulations of at least this many cells step alone (-1: none)
    std::vector<char> solo;
    cudaStream_t solo_st[SOLO_STREAMS];   // the solo simulations, spread over these
    cudaEvent_t solo_ev[SOLO_STREAMS];
    int nshared;           // simulations inside the persistent kernel
    long long spin;        // clock cycles a grid-barrier wait may take
    int blocks;
    int graph_ok;          // -1 unknown, 0 direct launches, 1 graphs
    std::map<int, cudaGraphExec_t> graphs;   // steps per launch -> executable graph
    int status;
};

namespace {

int note(fdtd_batch *b, cudaError_t e) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->status == FDTD_OK) b->status = FDTD_ERR_CUDA;
        return FDTD_ERR_CUDA;
    }
    return FDTD_OK;
}

void drop_graphs(fdtd_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Descriptors and item prefix sums from the handles' current state.  A
// simulation whose grid the tile path cannot run (no tile state on its
// handle), or which has CPML layers, steps alone.
int refresh(fdtd_batch *b) {
    const int all = (int)b->sims.size();
    std::vector<fdtd_ctx *> shared;
    b->solo.assign(all, 0);
    for (int q = 0; q < all; ++q) {
        const fdtd_ctx *h = b->sims[q];
        const long long cells = (long long)h->g.nx * h->g.ny * h->g.nz;
        b->solo[q] = !h->vtile || h->P > 0 || (b->solo_cells >= 0 && cells >= b->solo_cells);
        if (!b->solo[q]) shared.push_back(b->sims[q]);
    }
    const int n = (int)shared.size();
    b->nshared = n;
    if (n == 0) return FDTD_OK;
    std::vector<BSim> d(n);
    std::vector<vt::Maps> maps(n);
    std::vector<int> fs(n + 1, 0), ms(n + 1, 0);
    for (int q = 0; q < n; ++q) {
        fdtd_ctx *h = shared[q];
        const vt::HostState *vs = static_cast<const vt::HostState *>(h->vtile);
        const Grid &g = h->g;
        // z chunks of about chunk_planes planes between the layers
        const int mid = h->P > 0 ? g.nz - 2 * h->P - 1 : g.nz;
        vt::Chunks z;
        if (!vt::z_chunks(g.nz, h->P, vs->xbw, (mid + b->chunk_planes - 1) / b->chunk_planes, b->floats, z)) {
            if (b->status == FDTD_OK) b->status = FDTD_ERR_CUDA;
            return b->status;
        }
        BSim &S = d[q];
        std::memset(&S, 0, sizeof(S));
        const int cur = h->cur;
        for (int c = 0; c < 2; ++c) {
            vt::Args &a = S.a[c];
            a.g = g;
            float *out = h->fields[c ^ 1];
            const size_t cc = (size_t)g.comp;
            a.oex = out; a.oey = out + cc; a.oez = out + 2 * cc;
            a.ohx = out + 3 * cc; a.ohy = out + 4 * cc; a.ohz = out + 5 * cc;
            h->cur = c;
            a.pml = cpml_view(h);
            a.tiles_x = vs->tiles_x;
            a.tiles_y = vs->tiles_y;
            a.za = z.za;
            a.zb = z.zb;
            a.cm = z.cm;
            a.m = z.m;
            a.zc = z.zc;
            a.ring = z.ring;
            a.xlo4 = vs->xlo4;
            a.xhb = vs->xhb;
            a.xbw = vs->xbw;
            a.cur = c;
            a.ecur = h->ecur;
            a.src = h->src;
            a.kE = (float)h->kE;
            a.kH = (float)h->kH;
        }
        h->cur = cur;
        maps[q] = vs->maps;
        S.maps = b->d_maps + q;
        S.tiles = vs->tiles_x * vs->tiles_y;
        S.items = S.tiles * z.chunks;
        S.mur = (float)h->mur_m;
        S.mface[0] = 0;
        for (int f = 0; f < 6; ++f) {
            const int ax = f >> 1;
            const long long na = (ax == 0 ? g.ny : g.nx) + 1, nb = (ax == 2 ? g.ny : g.nz) + 1;
            S.mface[f + 1] = S.mface[f] + (h->boundary == FDTD_MUR1 ? (int)((na * nb + MUR_PIECE - 1) / MUR_PIECE) : 0);
        }
        S.pr = Probes{h->np, h->max_steps, h->d_ijk, h->d_cxy, h->d_trace};
        S.cur = h->cur;
        S.n = h->steps;
        fs[q + 1] = fs[q] + S.items;
        ms[q + 1] = ms[q] + S.mface[6] + (h->np > 0 ? 1 : 0);
    }
    // item order of a step: the F items of each simulation in turn, then the
    // M items of each
    std::vector<int> seg{0}, segq;
    for (int kind = 0; kind < 2; ++kind)
        for (int q = 0; q < n; ++q) {
            const int count = kind == 0 ? fs[q + 1] - fs[q] : ms[q + 1] - ms[q];
            if (count <= 0) continue;
            segq.push_back(2 * q + kind);
            seg.push_back(seg.back() + count);
        }
    b->nseg = (int)segq.size();
    if (note(b, cudaMemcpyAsync(b->d_seg, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_segq, segq.data(), segq.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_sims, d.data(), n * sizeof(BSim), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_maps, maps.data(), n * sizeof(vt::Maps), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_fstart, fs.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_mstart, ms.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream)))
        return b->status;
    // pageable sources: the copies complete before the next host change of d, maps, fs, ms
    return note(b, cudaStreamSynchronize(b->stream));
}

// The persistent kernel's shared memory (all an SM's block may take) and grid
// (every block resident).
int size_grid(fdtd_batch *b) {
    cudaFuncAttributes fa;
    int optin = 0, per = 0;
    if (cudaFuncGetAttributes(&fa, k_batch) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    b->smem = ((size_t)optin - fa.sharedSizeBytes) / 1024 * 1024;
    b->floats = ((long long)b->smem - vt::BAR_BYTES) / 4;
    if (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, NT, b->smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    b->blocks = per * b->sms;
    return FDTD_OK;
}

cudaError_t issue(fdtd_batch *b, int steps) {
    BArgs A;
    A.sims = b->d_sims;
    A.nsim = b->nshared;
    A.fstart = b->d_fstart;
    A.mstart = b->d_mstart;
    A.seg = b->d_seg;
    A.segq = b->d_segq;
    A.nseg = b->nseg;
    A.steps = steps;
    A.ctr = b->d_ctr;
    A.bar = b->d_bar;
    A.flags = b->d_flags;
    A.spin = b->spin;
    cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, (1 + 2 * (size_t)b->nshared) * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->blocks);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch, A);
}

// One persistent launch of `steps` steps: a replay of its captured graph, or
// a direct launch when capture is not available.
int launch(fdtd_batch *b, int steps) {
    if (b->graph_ok != 0) {
        auto it = b->graphs.find(steps);
        if (it == b->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const cudaError_t e1 = issue(b, steps);
                const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
                ok = e1 == cudaSuccess && e2 == cudaSuccess && graph &&
                     cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            }
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                cudaGetLastError();
                if (exec) cudaGraphExecDestroy(exec);
                b->graph_ok = 0;
            } else {
                b->graph_ok = 1;
                it = b->graphs.emplace(steps, exec).first;
            }
        }
        if (b->graph_ok == 1) return note(b, cudaGraphLaunch(it->second, b->stream));
    }
    return note(b, issue(b, steps));
}

// One untimed step (it builds the graph), then `trial` steps timed on the
// batch's stream; *used counts every step the trial advanced.
int time_trial(fdtd_batch *b, int warm, int trial, float *ms, int *used) {
    *used = 0;
    int rc = fdtd_batch_step(b, warm);
    if (rc != FDTD_OK) return rc;
    *used += warm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    rc = note(b, cudaEventRecord(e0, b->stream));
    if (rc == FDTD_OK) rc = fdtd_batch_step(b, trial);
    if (rc == FDTD_OK) {
        *used += trial;
        rc = note(b, cudaEventRecord(e1, b->stream));
    }
    if (rc == FDTD_OK) rc = fdtd_batch_sync(b);
    if (rc == FDTD_OK) cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" {

int fdtd_batch_create(fdtd_batch_t *out, const fdtd_t *sims, int n) {
    if (!out) return FDTD_ERR_ARG;
    *out = nullptr;
    if (!sims || n < 1) return FDTD_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    for (int q = 0; q < n; ++q) {
        if (!sims[q] || sims[q]->dev != dev) return FDTD_ERR_ARG;
        if (sims[q]->status != FDTD_OK) return sims[q]->status;
        for (int r = 0; r < q; ++r)
            if (sims[r] == sims[q]) return FDTD_ERR_ARG;
    }
    fdtd_batch *b = new (std::nothrow) fdtd_batch();
    if (!b) return FDTD_ERR_OOM;
    b->sims.assign(sims, sims + n);
    b->dev = dev;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->chunk_planes = 256;
    b->steps_per_launch = 8;
    b->solo_cells = -1;
    b->nshared = n;
    b->spin = FDTD_BATCH_DEFAULT_WAIT_CYCLES;
    b->graph_ok = -1;
    b->status = FDTD_OK;
    bool streams_ok = true;
    for (int k = 0; k < SOLO_STREAMS; ++k)
        streams_ok = streams_ok && cudaStreamCreateWithFlags(&b->solo_st[k], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&b->solo_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!streams_ok || cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b->d_sims, n * sizeof(BSim)) != cudaSuccess ||
        cudaMalloc(&b->d_maps, n * sizeof(vt::Maps)) != cudaSuccess ||
        cudaMalloc(&b->d_fstart, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_seg, (2 * n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_segq, 2 * n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_mstart, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_ctr, (1 + 2 * (size_t)n) * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->d_flags, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        fdtd_batch_destroy(b);
        return FDTD_ERR_OOM;
    }
    if (note(b, cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream)) != FDTD_OK ||
        note(b, cudaMemsetAsync(b->d_flags, 0, sizeof(int), b->stream)) != FDTD_OK ||
        note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK || size_grid(b) != FDTD_OK) {
        fdtd_batch_destroy(b);
        return FDTD_ERR_CUDA;
    }
    *out = b;
    return FDTD_OK;
}

void fdtd_batch_destroy(fdtd_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->d_sims) cudaFree(b->d_sims);
    if (b->d_maps) cudaFree(b->d_maps);
    if (b->d_fstart) cudaFree(b->d_fstart);
    if (b->d_seg) cudaFree(b->d_seg);
    if (b->d_segq) cudaFree(b->d_segq);
    if (b->d_mstart) cudaFree(b->d_mstart);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->d_flags) cudaFree(b->d_flags);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    for (int k = 0; k < SOLO_STREAMS; ++k) {
        if (b->solo_st[k]) {
            cudaStreamSynchronize(b->solo_st[k]);
            cudaStreamDestroy(b->solo_st[k]);
        }
        if (b->solo_ev[k]) cudaEventDestroy(b->solo_ev[k]);
    }
    delete b;
}

int fdtd_batch_step(fdtd_batch_t b, int n) {
    if (!b || n < 0) return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    for (fdtd_t h : b->sims) {
        if (h->status != FDTD_OK) return h->status;
        if (h->np > 0 && h->steps + n > h->max_steps) return FDTD_ERR_CAPACITY;
    }
    if (n == 0) return FDTD_OK;
    // order after earlier work on the handles' streams
    for (fdtd_t h : b->sims) {
        if (note(b, cudaEventRecord(b->ev, h->stream)) || note(b, cudaStreamWaitEvent(b->stream, b->ev, 0)))
            return b->status;
    }
    if (refresh(b) != FDTD_OK) return b->status;
    const int all = (int)b->sims.size();
    if (b->nshared > 0) {
        int left = n;
        while (left > 0 && b->status == FDTD_OK) {
            const int s = std::min(left, b->steps_per_launch);
            launch(b, s);
            left -= s;
        }
    }
    // the simulations that step alone: their own selected path, after the
    // persistent launches (which then have the GPU to themselves), spread
    // largest first over the solo streams, each to the least loaded one
    std::vector<int> order;
    for (int q = 0; q < all; ++q)
        if (b->solo[q]) order.push_back(q);
    if (!order.empty() && b->status == FDTD_OK) {
        auto cells = [&](int q) { return (long long)b->sims[q]->g.nx * b->sims[q]->g.ny * b->sims[q]->g.nz; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cells(x) > cells(y); });
        const int ns = std::min<int>(SOLO_STREAMS, (int)order.size());
        if (note(b, cudaEventRecord(b->ev, b->stream)) != FDTD_OK) return b->status;
        for (int k = 0; k < ns; ++k)
            if (note(b, cudaStreamWaitEvent(b->solo_st[k], b->ev, 0)) != FDTD_OK) return b->status;
        long long load[SOLO_STREAMS] = {0};
        for (int q : order) {
            int k = 0;
            for (int j = 1; j < ns; ++j)
                if (load[j] < load[k]) k = j;
            load[k] += cells(q);
            if (fdtd::fdtd_step_on(b->sims[q], n, b->solo_st[k]) != FDTD_OK) {
                b->status = b->sims[q]->status;
                break;
            }
        }
        for (int k = 0; k < ns; ++k)
            if (note(b, cudaEventRecord(b->solo_ev[k], b->solo_st[k])) != FDTD_OK ||
                note(b, cudaStreamWaitEvent(b->stream, b->solo_ev[k], 0)) != FDTD_OK)
                return b->status;
    }
    for (int q = 0; q < all; ++q)
        if (!b->solo[q]) {
            b->sims[q]->cur ^= n & 1;
            b->sims[q]->steps += n;
        }
    // order later work on the handles' streams after the batch
    if (note(b, cudaEventRecord(b->ev, b->stream)) != FDTD_OK) return b->status;
    for (fdtd_t h : b->sims)
        if (note(b, cudaStreamWaitEvent(h->stream, b->ev, 0)) != FDTD_OK) return b->status;
    return b->status;
}

int fdtd_batch_sync(fdtd_batch_t b) {
    if (!b) return FDTD_ERR_ARG;
    if (note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK) return b->status;
    int f = 0;
    if (note(b, cudaMemcpy(&f, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost)) != FDTD_OK) return b->status;
    if (f) {
        // a grid barrier gave up: the simulations of the persistent kernel
        // were left part-way through a step
        if (b->status == FDTD_OK) b->status = FDTD_ERR_TIMEOUT;
        for (size_t q = 0; q < b->sims.size(); ++q)
            if (q >= b->solo.size() || !b->solo[q])
                if (b->sims[q]->status == FDTD_OK) b->sims[q]->status = FDTD_ERR_TIMEOUT;
    }
    return b->status;
}

int fdtd_batch_set_wait_limit(fdtd_batch_t b, long long cycles) {
    if (!b || cycles < 0) return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    if (note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK) return b->status;
    drop_graphs(b);   // the limit is a launch argument, baked into the graphs
    b->spin = cycles == 0 ? FDTD_BATCH_DEFAULT_WAIT_CYCLES : cycles;
    return FDTD_OK;
}

int fdtd_batch_set_config(fdtd_batch_t b, int chunk_planes, int steps_per_launch) {
    if (!b || chunk_planes < 1 || steps_per_launch < 1 || steps_per_launch > MAX_STEPS_PER_LAUNCH)
        return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    if (note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK) return b->status;
    drop_graphs(b);
    b->chunk_planes = chunk_planes;
    b->steps_per_launch = steps_per_launch;
    return FDTD_OK;
}

int fdtd_batch_get_config(fdtd_batch_t b, int *chunk_planes, int *steps_per_launch) {
    if (!b) return FDTD_ERR_ARG;
    if (chunk_planes) *chunk_planes = b->chunk_planes;
    if (steps_per_launch) *steps_per_launch = b->steps_per_launch;
    return FDTD_OK;
}

int fdtd_batch_set_solo(fdtd_batch_t b, long long min_cells) {
    if (!b || min_cells < -1) return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    if (note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK) return b->status;
    drop_graphs(b);
    b->solo_cells = min_cells;
    return FDTD_OK;
}

int fdtd_batch_get_solo(fdtd_batch_t b, long long *min_cells, int *n_solo) {
    if (!b) return FDTD_ERR_ARG;
    if (min_cells) *min_cells = b->solo_cells;
    if (n_solo) {
        int k = 0;
        for (fdtd_t h : b->sims)
            if (!h->vtile || h->P > 0 || (b->solo_cells >= 0 && (long long)h->g.nx * h->g.ny * h->g.nz >= b->solo_cells))
                ++k;
        *n_solo = k;
    }
    return FDTD_OK;
}

int fdtd_batch_tune(fdtd_batch_t b, int trial_steps, int *steps_used) {
    if (!b || trial_steps < 1) return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    const int spl0 = b->steps_per_launch, spl = std::min(spl0, trial_steps);
    int used = 0;
    // first the solo threshold, with the current launch configuration: none,
    // every simulation alone, or a power of two between the smallest and the
    // largest grid
    {
        long long lo = 1LL << 62, hi = 0;
        for (fdtd_t h : b->sims) {
            const long long c = (long long)h->g.nx * h->g.ny * h->g.nz;
            lo = std::min(lo, c);
            hi = std::max(hi, c);
        }
        std::vector<long long> cand{-1, lo};
        for (long long t = 2; t <= hi; t <<= 1)
            if (t > lo) cand.push_back(t);
        long long best = b->solo_cells;
        float best_ms = 1e30f;
        for (long long t : cand) {
            int rc = fdtd_batch_set_solo(b, t);
            float ms = 0.f;
            int u = 0;
            if (rc == FDTD_OK) rc = time_trial(b, spl, trial_steps, &ms, &u);
            used += u;
            if (rc != FDTD_OK) {
                if (steps_used) *steps_used = used;
                return rc;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        fdtd_batch_set_solo(b, best);
    }
    // then the z chunk length of the persistent kernel's tiles, if it has work
    const int cpl[4] = {64, 128, 256, 512};
    float best_ms = 1e30f;
    int best_c = b->chunk_planes, rc = FDTD_OK;
    refresh(b);
    if (b->nshared > 0)
        for (int c : cpl) {
            if ((rc = fdtd_batch_set_config(b, c, spl)) != FDTD_OK) break;
            float ms = 0.f;
            int u = 0;
            rc = time_trial(b, spl, trial_steps, &ms, &u);
            used += u;
            if (rc != FDTD_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_c = c;
            }
        }
    if (steps_used) *steps_used = used;
    if (rc != FDTD_OK) return rc;
    return fdtd_batch_set_config(b, best_c, spl0);
}

int fdtd_batch_graph_mode(fdtd_batch_t b) { return b ? b->graph_ok : -1; }

}  // extern "C"
