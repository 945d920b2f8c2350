// kernels_noalloc.cu -- field energy of caller-owned device arrays with a
// scratch area compiled into the library: the call allocates no memory.
//
// Same two-pass reduction as the handle's energy check: pass 1 reduces
// |E|^2, |H|^2 and a non-finite count per block into a partial slot, pass 2
// reduces the slots into three totals.  The slots and the totals live in a
// fixed __device__ array; its address is looked up once per device and
// context (a device reset makes a new primary context, which loads the module
// again, possibly at another address).
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/fdtd.h"

namespace {

constexpr double kC = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
constexpr int kTotals = 3 * FDTD_ENERGY_SCRATCH_BLOCKS;   // offset of the three totals

// pass-1 slots (E sum, H sum, non-finite count per block), then the totals;
// each call writes every slot it reads before reading it
__device__ __align__(256) double g_energy_scratch[3 * FDTD_ENERGY_SCRATCH_BLOCKS + 3];

// device address of g_energy_scratch per device (looked up on first use),
// valid for the context it was looked up in
std::atomic<double *> g_scratch_addr[kMaxDevices];
std::atomic<void *> g_scratch_ctx[kMaxDevices];

typedef CUresult (*CtxGetCurrent)(CUcontext *);

// the calling thread's current context (the primary context of the current
// device once the runtime has initialised it), or null
void *current_context() {
    static std::atomic<CtxGetCurrent> fn{nullptr};
    CtxGetCurrent f = fn.load();
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        f = reinterpret_cast<CtxGetCurrent>(p);
        fn.store(f);
    }
    CUcontext c = nullptr;
    return f(&c) == CUDA_SUCCESS ? static_cast<void *>(c) : nullptr;
}

__device__ __forceinline__ double warp_total(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// three block sums into out[0..2] (thread 0)
__device__ __forceinline__ void block_total(double a, double b, double c, double *out) {
    __shared__ double red[3][kThreads / 32];
    a = warp_total(a);
    b = warp_total(b);
    c = warp_total(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = c; }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? red[0][l] : 0.0;
        b = l < nw ? red[1][l] : 0.0;
        c = l < nw ? red[2][l] : 0.0;
        a = warp_total(a);
        b = warp_total(b);
        c = warp_total(c);
        if (l == 0) { out[0] = a; out[1] = b; out[2] = c; }
    }
}

// f: n floats, the first n_e of them E components
__global__ void __launch_bounds__(kThreads) k_energy_slots(const float *__restrict__ f, long long n_e, long long n,
                                                           double *slots) {
    double se = 0.0, sh = 0.0, bad = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float v = f[t];
        const double s = (double)v * v;
        if (!isfinite(v)) bad += 1.0;
        if (t < n_e) se += s; else sh += s;
    }
    block_total(se, sh, bad, slots + 3 * blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_energy_totals(double *scratch, int nslots) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < nslots; t += blockDim.x) {
        a += scratch[3 * t];
        b += scratch[3 * t + 1];
        c += scratch[3 * t + 2];
    }
    block_total(a, b, c, scratch + kTotals);
}

}  // namespace

extern "C" int fdtd_energy_noalloc(const float *d_fields, int nx, int ny, int nz, double dx, double eps_r,
                                   int nblocks, void *stream, double *energy) {
    if (!d_fields || !energy || nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(eps_r > 0.0) || nblocks < 0)
        return FDTD_ERR_ARG;
    if (nblocks > FDTD_ENERGY_SCRATCH_BLOCKS) return FDTD_ERR_CAPACITY;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    // before the runtime's first use of the device no context is current yet;
    // the lookup below then makes the primary context current
    void *ctx = current_context();
    double *scratch = g_scratch_addr[dev].load();
    if (!scratch || !ctx || g_scratch_ctx[dev].load() != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FDTD_ERR_CUDA;
        }
        scratch = static_cast<double *>(p);
        g_scratch_addr[dev].store(scratch);
        g_scratch_ctx[dev].store(current_context());
    }
    if (nblocks == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return FDTD_ERR_CUDA;
        }
        nblocks = 4 * (sms > 0 ? sms : 1);
        if (nblocks > FDTD_ENERGY_SCRATCH_BLOCKS) nblocks = FDTD_ENERGY_SCRATCH_BLOCKS;
    }
    const long long nodes = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_energy_slots<<<nblocks, kThreads, 0, s>>>(d_fields, 3 * nodes, 6 * nodes, scratch);
    k_energy_totals<<<1, kThreads, 0, s>>>(scratch, nblocks);
    double r[3];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(r, scratch + kTotals, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    const double eps = eps_r / (kMu0 * kC * kC), v = dx * dx * dx;
    *energy = 0.5 * eps * r[0] * v + 0.5 * kMu0 * r[1] * v;
    return r[2] > 0.0 ? FDTD_ERR_UNSTABLE : FDTD_OK;
}
