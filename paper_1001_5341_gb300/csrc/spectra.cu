// Spectra of detector traces (Sec. V): E_omega(f) = dt sum_m g_m x_{first+m}
// exp(i 2 pi f t_{first+m}), t_n = t0 + n dt, the time factor of eq. GreenMethod.
//
// One block per (trace, group of SPEC_FB frequencies).  Its threads stride
// over the gated samples; each forms x = sum_c a_c X[n][c] times the Tukey
// weight once and rotates it by the SPEC_FB phases.  A phase is the fraction
// of a cycle in 64-bit fixed point, advanced by an integer add per sample, so
// no rounding builds up along the trace; its top 32 bits give the angle for
// sincospif.  Partial sums are float32 within a thread and float64 across the
// block.  The work is a few dozen ALU instructions per (sample, frequency);
// the traces (n_traces x n_t x n_comp floats) are read once per frequency
// group, from L2 after the first.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "spectra.h"

namespace {

constexpr int SPEC_THREADS = 256;
constexpr int SPEC_FB = 8;            // frequencies per block
constexpr int SPEC_MAX_COMP = 4;

struct TraceParam {
    float a[SPEC_MAX_COMP];           // component weights
    int first, count;                 // gate
};

struct FreqParam {
    unsigned long long a, b;          // cycles of f t0 and of f dt, fraction x 2^64
};

// Fraction of x in [0, 1) as a 64-bit fixed-point number.
unsigned long long fixed_fraction(double x) {
    double fr = x - std::floor(x);
    if (!(fr >= 0.0 && fr < 1.0)) fr = 0.0;
    return (unsigned long long)std::ldexp(fr, 64);
}

__global__ void __launch_bounds__(SPEC_THREADS)
k_trace_spectrum(const float *__restrict__ X, int n_t, int n_comp, const TraceParam *__restrict__ tp,
                 const FreqParam *__restrict__ fp, int n_freq, float taper, double dt, float *__restrict__ out) {
    const int tr = blockIdx.x;
    const int k0 = blockIdx.y * SPEC_FB;
    const TraceParam P = tp[tr];
    const float *x = X + ((size_t)tr * n_t + P.first) * n_comp;

    unsigned long long ph[SPEC_FB], step[SPEC_FB];
    float re[SPEC_FB], im[SPEC_FB];
#pragma unroll
    for (int k = 0; k < SPEC_FB; ++k) {
        ph[k] = step[k] = 0ull;
        if (k0 + k < n_freq) {
            const FreqParam F = fp[k0 + k];
            ph[k] = F.a + (unsigned long long)(P.first + (int)threadIdx.x) * F.b;
            step[k] = F.b * (unsigned long long)SPEC_THREADS;
        }
        re[k] = im[k] = 0.f;
    }
    const bool tapered = taper > 0.f && P.count > 1;
    const float inv = P.count > 1 ? 1.f / (float)(P.count - 1) : 0.f;
    const float half = 0.5f * taper;

    for (int m = threadIdx.x; m < P.count; m += SPEC_THREADS) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < SPEC_MAX_COMP; ++c)
            if (c < n_comp) v = fmaf(P.a[c], x[(size_t)m * n_comp + c], v);
        if (tapered) {
            const float u = (float)m * inv;
            if (u < half)
                v *= 0.5f * (1.f - cospif(2.f * u / taper));
            else if (u > 1.f - half)
                v *= 0.5f * (1.f - cospif(2.f * (1.f - u) / taper));
        }
#pragma unroll
        for (int k = 0; k < SPEC_FB; ++k) {
            // signed top word: the phase in half-turns, in [-1, 1)
            const float turns = (float)(int)(ph[k] >> 32) * 4.656612873077393e-10f;
            float s, c;
            sincospif(turns, &s, &c);
            re[k] = fmaf(v, c, re[k]);
            im[k] = fmaf(v, s, im[k]);
            ph[k] += step[k];
        }
    }

    __shared__ double red[SPEC_THREADS / 32][2 * SPEC_FB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < SPEC_FB; ++k) {
        double r = re[k], i = im[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r += __shfl_down_sync(0xffffffffu, r, o);
            i += __shfl_down_sync(0xffffffffu, i, o);
        }
        if (lane == 0) {
            red[warp][2 * k] = r;
            red[warp][2 * k + 1] = i;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * SPEC_FB) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < SPEC_THREADS / 32; ++w) s += red[w][threadIdx.x];
        const int k = threadIdx.x >> 1;
        if (k0 + k < n_freq) out[((size_t)tr * n_freq + k0 + k) * 2 + (threadIdx.x & 1)] = (float)(s * dt);
    }
}

// Device (or managed) memory that kernels may read; a host pointer is refused
// before anything is launched.
bool device_pointer(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int fdtd_trace_spectrum(const float *traces, int n_traces, int n_t, int n_comp, const double *coef,
                                   const int *gate, double taper, double dt, double t0, const double *freq,
                                   int n_freq, float *out, int on_device, void *stream) {
    if (!traces || !freq || !out || n_traces < 1 || n_t < 1 || n_freq < 1 || n_comp < 1 ||
        n_comp > SPEC_MAX_COMP || !(taper >= 0.0 && taper <= 1.0) || !(dt > 0.0) || !std::isfinite(dt) ||
        !std::isfinite(t0))
        return FDTD_ERR_ARG;
    if ((n_freq + SPEC_FB - 1) / SPEC_FB > 65535 || n_traces > 0x7fffffff / 2) return FDTD_ERR_ARG;
    if (!device_pointer(traces) || (on_device && !device_pointer(out))) return FDTD_ERR_ARG;

    std::vector<TraceParam> tp(n_traces);
    for (int p = 0; p < n_traces; ++p) {
        TraceParam &T = tp[p];
        for (int c = 0; c < SPEC_MAX_COMP; ++c) {
            double a = c < n_comp ? (coef ? coef[(size_t)p * n_comp + c] : (c == 0 ? 1.0 : 0.0)) : 0.0;
            if (!std::isfinite(a)) return FDTD_ERR_ARG;
            T.a[c] = (float)a;
        }
        T.first = gate ? gate[2 * p] : 0;
        T.count = gate ? gate[2 * p + 1] : n_t;
        if (T.first < 0 || T.count < 0 || (long long)T.first + T.count > n_t) return FDTD_ERR_ARG;
    }
    std::vector<FreqParam> fp(n_freq);
    for (int k = 0; k < n_freq; ++k) {
        const double f = freq[k];
        if (!std::isfinite(f) || !std::isfinite(f * t0) || !std::isfinite(f * dt)) return FDTD_ERR_ARG;
        fp[k].a = fixed_fraction(f * t0);
        fp[k].b = fixed_fraction(f * dt);
    }

    cudaStream_t s = (cudaStream_t)stream;
    const size_t tp_bytes = sizeof(TraceParam) * (size_t)n_traces;
    const size_t tp_pad = (tp_bytes + 15) & ~(size_t)15;
    const size_t par_bytes = tp_pad + sizeof(FreqParam) * (size_t)n_freq;
    const size_t out_bytes = sizeof(float) * 2 * (size_t)n_traces * n_freq;
    char *dpar = nullptr;
    float *dout = nullptr;
    if (cudaMallocAsync((void **)&dpar, par_bytes + (on_device ? 0 : out_bytes), s) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    dout = on_device ? out : (float *)(dpar + par_bytes);
    int rc = FDTD_OK;
    if (cudaMemcpyAsync(dpar, tp.data(), tp_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dpar + tp_pad, fp.data(), sizeof(FreqParam) * (size_t)n_freq, cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        rc = FDTD_ERR_CUDA;
    if (rc == FDTD_OK) {
        dim3 grid(n_traces, (n_freq + SPEC_FB - 1) / SPEC_FB);
        k_trace_spectrum<<<grid, SPEC_THREADS, 0, s>>>(traces, n_t, n_comp, (const TraceParam *)dpar,
                                                       (const FreqParam *)(dpar + tp_pad), n_freq, (float)taper,
                                                       dt, dout);
        if (cudaGetLastError() != cudaSuccess) rc = FDTD_ERR_CUDA;
    }
    if (rc == FDTD_OK && !on_device) {
        if (cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = FDTD_ERR_CUDA;
    }
    cudaFreeAsync(dpar, s);
    if (!on_device && cudaStreamSynchronize(s) != cudaSuccess) rc = FDTD_ERR_CUDA;
    return rc;
}

extern "C" int fdtd_theta_coef(const double *theta, int n, double *coef) {
    if (!theta || !coef || n < 1) return FDTD_ERR_ARG;
    for (int t = 0; t < n; ++t)
        if (!std::isfinite(theta[t])) return FDTD_ERR_ARG;
    for (int t = 0; t < n; ++t) {
        coef[2 * t] = -std::sin(theta[t]);
        coef[2 * t + 1] = std::cos(theta[t]);
    }
    return FDTD_OK;
}
