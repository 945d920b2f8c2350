// batch.cu -- many simulations in one persistent kernel (batch.h).
//
// Work queue.  For each step the kernel runs three phases; in each phase every
// block takes items from an atomic counter until the phase's items are gone:
//   H: item = (simulation q, slab of planes of q): H^{n+1/2} of its cells;
//   E: same items: E^{n+1} with the shower's current;
//   M: item = (q, face) for the six Mur faces of a Mur grid, and (q, detectors)
//      for a grid with detectors: the boundary, then the readout of E^{n+1}.
// Between phases a grid-wide barrier (all blocks are resident: cooperative
// launch) with a bounded wait.  Every cell goes through cell_h / cell_e /
// mur_cell, the code of the unfused path, so the numbers are the same.
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

using namespace fdtd;

namespace {

constexpr int MAX_STEPS_PER_LAUNCH = 64;

struct BSim {
    Grid g;
    float *f[2];
    Cpml pml[2];           // views for cur = 0 and cur = 1
    float kE, kH, mur;
    int mur_on;
    Source src;
    Probes pr;
    int cur;
    long long n;           // steps done
    int planes;            // z planes per H/E item
};

struct BArgs {
    BSim *sims;
    int nsim;
    const int *hstart;     // [nsim + 1] prefix sums of H/E items
    const int *mstart;     // [nsim + 1] prefix sums of M items
    int steps;
    unsigned *ctr;         // [3 * steps] queue counters, zero at launch
    unsigned *bar;         // [2] barrier count and generation, zero at launch
    int *flags;
    long long spin;        // clock cycles a barrier wait may take
};

// Grid-wide barrier: arrive, then wait (bounded by spin cycles) for the
// generation to move.  A block whose wait gives up sets flag bit 1 and stops;
// the others then give up at this barrier or the next, so the launch ends.
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

__global__ void __launch_bounds__(256, 6) k_batch(BArgs A) {   // 40 registers: 6 blocks per SM
    __shared__ int s_item;
    // the item's simulation, copied once per item: the per-cell code then
    // reads it from shared memory, which no global store can alias
    __shared__ Grid s_g;
    __shared__ Cpml s_pml;
    __shared__ Source s_src;
    __shared__ Probes s_pr;
    __shared__ float s_k[3];
    __shared__ int s_q, s_mur;
    __shared__ long long s_n;
    __shared__ const float *s_in;
    __shared__ float *s_out;
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int hitems = A.hstart[A.nsim], mitems = A.mstart[A.nsim];
    // an earlier launch (or a block of this one) gave up: the simulations are
    // in an unknown state.  One read per block, so that its threads leave
    // together (thread 0 alone drives the work queue).
    __shared__ int s_stop;
    if (tid == 0) s_stop = *(volatile int *)A.flags;
    __syncthreads();
    if (s_stop) return;
    for (int s = 0; s < A.steps; ++s) {
        for (int phase = 0; phase < 3; ++phase) {
            const int total = phase < 2 ? hitems : mitems;
            unsigned *ctr = A.ctr + 3 * s + phase;
            for (;;) {
                if (tid == 0) {
                    const int it = (int)atomicAdd(ctr, 1u);
                    s_item = it;
                    if (it < total) {
                        const int q = find_sim(phase < 2 ? A.hstart : A.mstart, A.nsim, it);
                        const BSim &S = A.sims[q];
                        const int cur = S.cur ^ (s & 1);
                        s_q = q;
                        s_g = S.g;
                        s_pml = S.pml[cur];
                        s_src = S.src;
                        s_pr = S.pr;
                        s_k[0] = S.kE;
                        s_k[1] = S.kH;
                        s_k[2] = S.mur;
                        s_mur = S.mur_on;
                        s_n = S.n + s;
                        s_in = S.f[cur];
                        s_out = S.f[cur ^ 1];
                    }
                }
                __syncthreads();
                const int it = s_item;
                if (it >= total) {
                    __syncthreads();
                    break;
                }
                const Grid g = s_g;
                const float *in = s_in;
                float *out = s_out;
                if (phase < 2) {
                    const int planes = A.sims[s_q].planes;
                    const int k0 = (it - A.hstart[s_q]) * planes, k1 = min(k0 + planes, g.nz);
                    const int rows = g.ny * (k1 - k0);
                    for (int row = warp; row < rows; row += nwarps) {
                        const int kk = row / g.ny, j = row - kk * g.ny, k = k0 + kk;
                        for (int i = lane; i < g.nx; i += 32) {
                            if (phase == 0)
                                cell_h(g, in, in + 3 * g.comp, out + 3 * g.comp, s_pml, s_k[1], i, j, k);
                            else
                                cell_e(g, in, out + 3 * g.comp, out, s_pml, s_k[0], s_src, s_n, i, j, k);
                        }
                    }
                } else {
                    const int m = it - A.mstart[s_q];
                    if (s_mur && m < 6) {
                        // face m: (a, b) over (j, k), (i, k) or (i, j)
                        const int ax = m >> 1;
                        const int na = (ax == 0 ? g.ny : g.nx) + 1, nb = (ax == 2 ? g.ny : g.nz) + 1;
                        for (int c = tid; c < na * nb; c += nt) mur_cell(g, in, out, s_k[2], m, c % na, c / na);
                    } else {
                        const Probes &p = s_pr;
                        for (int t = tid; t < p.n; t += nt) {
                            const int i = p.ijk[3 * t], j = p.ijk[3 * t + 1], k = p.ijk[3 * t + 2];
                            const long long c = gidx(g, i, j, k);
                            const float *Ex = out, *Ey = out + g.comp, *Ez = out + 2 * g.comp;
                            const float ex = 0.5f * (Ex[c - 1] + Ex[c]);
                            const float ey = 0.5f * (Ey[c - g.pitch] + Ey[c]);
                            const float ez = 0.5f * (Ez[c - g.plane] + Ez[c]);
                            float *o = p.trace + ((long long)t * p.max_steps + s_n) * 2;
                            o[0] = ez;
                            o[1] = p.cxy[2 * t] * ex + p.cxy[2 * t + 1] * ey;
                        }
                    }
                }
                __syncthreads();   // the item's shared copy is free again
            }
            if (!grid_sync(A.bar, A.flags, A.spin)) return;
        }
    }
    if (blockIdx.x == 0)
        for (int q = tid; q < A.nsim; q += nt) {
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
    int *d_hstart, *d_mstart;
    unsigned *d_ctr, *d_bar;
    int *d_flags;
    int threads, cells_per_item, steps_per_launch;
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

// Descriptors and item prefix sums from the handles' current state.
int refresh(fdtd_batch *b) {
    const int all = (int)b->sims.size();
    std::vector<fdtd_ctx *> shared;
    b->solo.assign(all, 0);
    for (int q = 0; q < all; ++q) {
        const fdtd_ctx *h = b->sims[q];
        const long long cells = (long long)h->g.nx * h->g.ny * h->g.nz;
        b->solo[q] = b->solo_cells >= 0 && cells >= b->solo_cells;
        if (!b->solo[q]) shared.push_back(b->sims[q]);
    }
    const int n = (int)shared.size();
    b->nshared = n;
    if (n == 0) return FDTD_OK;
    std::vector<BSim> d(n);
    std::vector<int> hs(n + 1, 0), ms(n + 1, 0);
    for (int q = 0; q < n; ++q) {
        fdtd_ctx *h = shared[q];
        BSim &S = d[q];
        S.g = h->g;
        S.f[0] = h->fields[0];
        S.f[1] = h->fields[1];
        const int cur = h->cur;
        for (int c = 0; c < 2; ++c) {
            h->cur = c;
            S.pml[c] = cpml_view(h);
        }
        h->cur = cur;
        S.kE = (float)h->kE;
        S.kH = (float)h->kH;
        S.mur = (float)h->mur_m;
        S.mur_on = h->boundary == FDTD_MUR1;
        S.src = h->src;
        S.pr = Probes{h->np, h->max_steps, h->d_ijk, h->d_cxy, h->d_trace};
        S.cur = h->cur;
        S.n = h->steps;
        const long long plane = (long long)h->g.nx * h->g.ny;
        S.planes = (int)std::max<long long>(1, std::min<long long>(h->g.nz, b->cells_per_item / std::max(1LL, plane)));
        while (S.planes > 1 && plane * S.planes >= (1LL << 31)) --S.planes;
        hs[q + 1] = hs[q] + (h->g.nz + S.planes - 1) / S.planes;
        ms[q + 1] = ms[q] + (S.mur_on ? 6 : 0) + (h->np > 0 ? 1 : 0);
    }
    if (note(b, cudaMemcpyAsync(b->d_sims, d.data(), n * sizeof(BSim), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_hstart, hs.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream)) ||
        note(b, cudaMemcpyAsync(b->d_mstart, ms.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream)))
        return b->status;
    // pageable sources: the copies complete before the next host change of d, hs, ms
    return note(b, cudaStreamSynchronize(b->stream));
}

int size_grid(fdtd_batch *b) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, b->threads, 0) != cudaSuccess || per < 1) {
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
    A.hstart = b->d_hstart;
    A.mstart = b->d_mstart;
    A.steps = steps;
    A.ctr = b->d_ctr;
    A.bar = b->d_bar;
    A.flags = b->d_flags;
    A.spin = b->spin;
    cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, 3 * steps * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->blocks);
    cfg.blockDim = dim3(b->threads);
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
    b->threads = 256;
    b->cells_per_item = 1 << 16;
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
        cudaMalloc(&b->d_hstart, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_mstart, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_ctr, 3 * MAX_STEPS_PER_LAUNCH * sizeof(unsigned)) != cudaSuccess ||
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
    if (b->d_hstart) cudaFree(b->d_hstart);
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

int fdtd_batch_set_config(fdtd_batch_t b, int threads, int cells_per_item, int steps_per_launch) {
    if (!b || (threads != 128 && threads != 256) || cells_per_item < 1 || steps_per_launch < 1 ||
        steps_per_launch > MAX_STEPS_PER_LAUNCH)
        return FDTD_ERR_ARG;
    if (b->status != FDTD_OK) return b->status;
    if (note(b, cudaStreamSynchronize(b->stream)) != FDTD_OK) return b->status;
    drop_graphs(b);
    b->threads = threads;
    b->cells_per_item = cells_per_item;
    b->steps_per_launch = steps_per_launch;
    return size_grid(b);
}

int fdtd_batch_get_config(fdtd_batch_t b, int *threads, int *cells_per_item, int *steps_per_launch) {
    if (!b) return FDTD_ERR_ARG;
    if (threads) *threads = b->threads;
    if (cells_per_item) *cells_per_item = b->cells_per_item;
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
            if (b->solo_cells >= 0 && (long long)h->g.nx * h->g.ny * h->g.nz >= b->solo_cells) ++k;
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
    const int thr[2] = {128, 256};
    const int cpi[4] = {1 << 14, 1 << 16, 1 << 18, 1 << 20};
    // then the launch configuration of the persistent kernel, if it has work
    float best_ms = 1e30f;
    int best_t = b->threads, best_c = b->cells_per_item, rc = FDTD_OK;
    refresh(b);
    if (b->nshared > 0)
        for (int t : thr)
            for (int c : cpi) {
                if ((rc = fdtd_batch_set_config(b, t, c, spl)) != FDTD_OK) break;
                float ms = 0.f;
                int u = 0;
                rc = time_trial(b, spl, trial_steps, &ms, &u);
                used += u;
                if (rc != FDTD_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_t = t;
                    best_c = c;
                }
            }
    if (steps_used) *steps_used = used;
    if (rc != FDTD_OK) return rc;
    return fdtd_batch_set_config(b, best_t, best_c, spl0);
}

int fdtd_batch_graph_mode(fdtd_batch_t b) { return b ? b->graph_ok : -1; }

}  // extern "C"
