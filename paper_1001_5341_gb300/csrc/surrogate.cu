// surrogate.cu -- forward/backward kernels and the optimiser step of the
// learned near-field surrogate (declarations and contracts: surrogate.h).
//
// The GEMM with both operands K-major (and 16-byte rows) runs on the
// fifth-generation tensor cores (tcgen05, TMEM, TMA: gemm_tc.cu).  The other
// operand layouts run on the warp-level mma.sync m16n8k16 bf16 instruction:
// 64x64 block tiles, 32-deep k slices staged in shared memory (either operand
// layout, transposed while staging), four warps of 32x32, f32 accumulators,
// fused bias / ReLU / bf16-copy epilogue.  The
// convolutions, the elementwise steps and the reductions are plain SIMT
// kernels: they are a few percent of the network's arithmetic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fdtd.h"
#include "../../include/surrogate.h"

namespace {

typedef unsigned short bf16raw;   // storage of one bfloat16

__device__ __forceinline__ float bf(const bf16raw v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
__device__ __forceinline__ bf16raw tobf(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

int launched() {
    if (cudaGetLastError() != cudaSuccess) return FDTD_ERR_CUDA;
    return FDTD_OK;
}

// ---- GEMM ------------------------------------------------------------------

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8, GT = 128;

template <bool AK, bool BK>
__global__ void __launch_bounds__(GT) k_gemm(const bf16raw *__restrict__ A, int lda, const bf16raw *__restrict__ B,
                                             int ldb, float *Y, int ldy, bf16raw *Yb, int M, int N, int K,
                                             const float *__restrict__ bias, int relu, int accumulate) {
    __shared__ __align__(16) bf16raw As[GBM][GBK + GPAD];
    __shared__ __align__(16) bf16raw Bs[GBN][GBK + GPAD];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int wm = warp >> 1, wn = warp & 1;       // warp tile (32x32) inside the block tile
    const int g = lane >> 2, t4 = lane & 3;        // mma fragment coordinates
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = 0; k0 < K; k0 += GBK) {
        // stage A (64 x 32) and B (64 x 32), reading along the contiguous axis
#pragma unroll 4
        for (int e = t; e < GBM * GBK; e += GT) {
            int m, k;
            if (AK) { m = e / GBK; k = e % GBK; } else { m = e % GBM; k = e / GBM; }
            const int gm = m0 + m, gk = k0 + k;
            bf16raw v = 0;
            if (gm < M && gk < K) v = AK ? A[(long long)gm * lda + gk] : A[(long long)gk * lda + gm];
            As[m][k] = v;
        }
#pragma unroll 4
        for (int e = t; e < GBN * GBK; e += GT) {
            int n, k;
            if (BK) { n = e / GBK; k = e % GBK; } else { n = e % GBN; k = e / GBN; }
            const int gn = n0 + n, gk = k0 + k;
            bf16raw v = 0;
            if (gn < N && gk < K) v = BK ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[n][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + g;
                a[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t4]);
                a[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t4]);
                a[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t4 + 8]);
                a[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn * 32 + j * 8 + g;
                b[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t4]);
                b[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
        }
        __syncthreads();
    }
    // epilogue: c0,c1 at (row g, cols 2t4, 2t4+1), c2,c3 at row g+8
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * t4 + (r & 1);
                if (m >= M || n >= N) continue;
                const long long o = (long long)m * ldy + n;
                float v = acc[i][j][r];
                if (accumulate) v += Y[o];
                if (bias) v += bias[n];
                if (relu) v = fmaxf(v, 0.f);
                Y[o] = v;
                if (Yb) Yb[o] = tobf(v);
            }
}

// ---- convolution -------------------------------------------------------------

__global__ void k_conv_fwd(const float *__restrict__ x, int xs, const bf16raw *__restrict__ w,
                           const float *__restrict__ bias, float *y, int B, int cin, int lin, int cout, int k,
                           int stride, int pad, int lout, int relu) {
    const long long total = (long long)B * cout * lout;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(id % lout), o = (int)((id / lout) % cout), b = (int)(id / ((long long)lout * cout));
        float s = bias ? bias[o] : 0.f;
        const float *xb = x + (long long)b * xs;
        for (int c = 0; c < cin; ++c)
            for (int tt = 0; tt < k; ++tt) {
                const int i = l * stride + tt - pad;
                if (i >= 0 && i < lin) s += bf(w[(o * cin + c) * k + tt]) * xb[c * lin + i];
            }
        y[id] = relu ? fmaxf(s, 0.f) : s;
    }
}

__device__ __forceinline__ float block_sum(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid on thread 0
}

// dw[o][c][t], one block per (o, c); db[o] from the blocks with c == 0
__global__ void k_conv_bwd_w(const float *__restrict__ x, int xs, const float *__restrict__ y,
                             const float *__restrict__ dy, int dys, float *dw, float *db, int B, int cin, int lin,
                             int cout, int k, int stride, int pad, int lout) {
    __shared__ float red[32];
    const int o = blockIdx.x / cin, c = blockIdx.x % cin;
    float acc[8];
    for (int tt = 0; tt < 8; ++tt) acc[tt] = 0.f;
    float accb = 0.f;
    const long long total = (long long)B * lout;
    for (long long id = threadIdx.x; id < total; id += blockDim.x) {
        const int l = (int)(id % lout), b = (int)(id / lout);
        const long long yo = (long long)b * cout * lout + (long long)o * lout + l;
        const float dz = y[yo] > 0.f ? dy[(long long)b * dys + (long long)o * lout + l] : 0.f;
        if (dz == 0.f) continue;
        accb += dz;
        const float *xb = x + (long long)b * xs + (long long)c * lin;
        for (int tt = 0; tt < k; ++tt) {
            const int i = l * stride + tt - pad;
            if (i >= 0 && i < lin) acc[tt] += dz * xb[i];
        }
    }
    for (int tt = 0; tt < k; ++tt) {
        const float s = block_sum(acc[tt], red);
        if (threadIdx.x == 0) dw[(o * cin + c) * k + tt] = s;
    }
    const float sb = block_sum(accb, red);
    if (threadIdx.x == 0 && c == 0) db[o] = sb;
}

__global__ void k_conv_bwd_x(const bf16raw *__restrict__ w, const float *__restrict__ y,
                             const float *__restrict__ dy, int dys, float *dx, int B, int cin, int lin, int cout,
                             int k, int stride, int pad, int lout) {
    const long long total = (long long)B * cin * lin;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(id % lin), c = (int)((id / lin) % cin), b = (int)(id / ((long long)lin * cin));
        float s = 0.f;
        for (int tt = 0; tt < k; ++tt) {
            const int num = i + pad - tt;
            if (num < 0 || num % stride) continue;
            const int l = num / stride;
            if (l >= lout) continue;
            for (int o = 0; o < cout; ++o) {
                const long long yo = (long long)b * cout * lout + (long long)o * lout + l;
                if (y[yo] > 0.f) s += bf(w[(o * cin + c) * k + tt]) * dy[(long long)b * dys + (long long)o * lout + l];
            }
        }
        dx[id] = s;
    }
}

// ---- elementwise and reductions ------------------------------------------------

__global__ void k_relu_bwd(const float *y, const float *dy, float *dz, bf16raw *dzb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = y[i] > 0.f ? dy[i] : 0.f;
        dz[i] = v;
        if (dzb) dzb[i] = tobf(v);
    }
}

// one block per 32 columns: a warp per column stripe, threads over rows
__global__ void k_bias_grad(const float *dz, int ldz, int M, int N, float *db) {
    __shared__ float red[8][33];
    const int col = blockIdx.x * 32 + (threadIdx.x & 31), ry = threadIdx.x >> 5;
    float s = 0.f;
    if (col < N)
        for (int m = ry; m < M; m += 8) s += dz[(long long)m * ldz + col];
    red[ry][threadIdx.x & 31] = s;
    __syncthreads();
    if (ry == 0 && col < N) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += red[r][threadIdx.x & 31];
        db[col] = t;
    }
}

__global__ void k_cast(const float *x, bf16raw *y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = tobf(x[i]);
}

__global__ void k_concat(const float *a, int na, const float *c, int nc, bf16raw *out, int B) {
    const int w = na + nc;
    const long long n = (long long)B * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % w);
        const long long b = i / w;
        out[i] = tobf(f < na ? a[b * na + f] : c[b * nc + (f - na)]);
    }
}

__global__ void k_mse(const float *y, const float *t, long long n, float *dy, float *loss) {
    __shared__ float red[32];
    float s = 0.f;
    const float inv = 1.0f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d * inv;
        s += d * d;
    }
    const float b = block_sum(s, red);
    if (loss && threadIdx.x == 0) atomicAdd(loss, b * inv);
}

__global__ void k_adam(float *w, bf16raw *wb, const float *g, float *m, float *v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = tobf(wi);
    }
}

// one warp per row: the row's peak |q|, then the division
__global__ void k_normalize(const float *q, int B, int n, float *qn, float *s) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    const float *qr = q + (long long)row * n;
    float m = 0.f;
    for (int i = lane; i < n; i += 32) m = fmaxf(m, fabsf(qr[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    for (int i = lane; i < n; i += 32) qn[(long long)row * n + i] = qr[i] * inv;
    if (lane == 0) s[row] = m;
}

__global__ void k_features(const float *rz, int B, float r0, float rs, float z0, float zs, float *out) {
    const long long n = (long long)B * 64;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % 64);
        const long long b = i / 64;
        const float u = (rz[2 * b] - r0) / rs, v = (rz[2 * b + 1] - z0) / zs;
        float val = 0.f;
        if (f == 0) {
            val = u;
        } else if (f == 1) {
            val = v;
        } else if (f < 62) {
            const int q = (f - 2) / 4, r = (f - 2) % 4;
            const float a = 3.14159265358979f * (float)(q + 1) * (r < 2 ? u : v);
            val = (r & 1) ? cosf(a) : sinf(a);
        }
        out[i] = val;
    }
}

__global__ void k_scale_rows(float *y, int B, int n, const float *s, float c, int invert) {
    const long long total = (long long)B * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float sb = s[i / n];
        y[i] *= invert ? (sb != 0.f ? c / sb : 0.f) : c * sb;
    }
}

__global__ void k_pairs(const float *rz, int B, int K, float z0, float dz, float *out) {
    const long long n = (long long)B * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / K;
        const int k = (int)(i % K);
        out[2 * i] = rz[2 * b];
        out[2 * i + 1] = rz[2 * b + 1] - z0 - (float)k * dz;
    }
}

// retarded-time placement of bin k's response at antenna b: integer sample
// offset ci, interpolation weight f, amplitude 1/R
struct Place {
    int ci;
    float f, a;
};
__device__ __forceinline__ Place place(const float *rz, long long b, int k, int shift, float z0, float dz,
                                       float cps) {
    const float r = rz[2 * b], d = rz[2 * b + 1] - z0 - (float)k * dz;
    const float R = fmaxf(sqrtf(r * r + d * d), 0.5f * dz);
    const float c = (float)(shift * k) + R / cps;
    Place p;
    p.ci = (int)floorf(c);
    p.f = c - (float)p.ci;
    p.a = 1.f / R;
    return p;
}

// one thread per output sample, a loop over the bins
__global__ void k_assemble(const float *__restrict__ G, const float *__restrict__ qn, const float *__restrict__ rz,
                           int B, int K, int Tg, int shift, int T, float z0, float dz, float cps, int J0,
                           float *out) {
    const long long n = (long long)B * T;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(id % T);
        const long long b = id / T;
        float s = 0.f;
        for (int k = 0; k < K; ++k) {
            const Place p = place(rz, b, k, shift, z0, dz, cps);
            const int j = i - p.ci + J0;
            if (j < 0) continue;
            const float *g = G + (b * K + k) * (long long)Tg;
            const float g0 = j < Tg ? g[j] : 0.f, g1 = (j >= 1 && j - 1 < Tg) ? g[j - 1] : 0.f;
            s += qn[b * K + k] * p.a * ((1.f - p.f) * g0 + p.f * g1);
        }
        out[id] = s;
    }
}

__global__ void k_assemble_bwd(const float *__restrict__ dout, const float *__restrict__ qn,
                               const float *__restrict__ rz, int B, int K, int Tg, int shift, int T, float z0,
                               float dz, float cps, int J0, float *dG, bf16raw *dGb) {
    const long long n = (long long)B * K * Tg;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(id % Tg);
        const long long bk = id / Tg;
        const long long b = bk / K;
        const int k = (int)(bk % K);
        const Place p = place(rz, b, k, shift, z0, dz, cps);
        const int i0 = j + p.ci - J0, i1 = i0 + 1;
        const float d0 = (i0 >= 0 && i0 < T) ? dout[b * T + i0] : 0.f;
        const float d1 = (i1 >= 0 && i1 < T) ? dout[b * T + i1] : 0.f;
        const float v = qn[bk] * p.a * ((1.f - p.f) * d0 + p.f * d1);
        dG[id] = v;
        if (dGb) dGb[id] = tobf(v);
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

// ---- lattice surrogate: bin responses on the grid's own lattice ----------------
// G[(ir * D + d) * T + tau] (bf16): response of antenna radial class ir to a
// unit profile bin at axial lattice offset d - moff (bins), tau samples after
// the bin's own time origin.  Antenna b has class ant[2b] and axial lattice
// index ant[2b+1]; bin k's offset is m - k, its time origin S k - J samples
// (J lead samples: the bin's charge starts to move one bin early).

__device__ __forceinline__ float val(const bf16raw v) { return bf(v); }
__device__ __forceinline__ float val(const float v) { return v; }

// Tab: bf16raw (with an optional second bf16 table Glo of the remainders) or float
template <typename Tab>
__global__ void __launch_bounds__(256) k_lat_fwd(const Tab *__restrict__ G, const bf16raw *__restrict__ Glo,
                                                 const float *__restrict__ q, const int *__restrict__ ant, int K,
                                                 int NR, int D, int T, int S, int J, int moff,
                                                 float *__restrict__ y) {
    __shared__ float qs[1024];
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < K; k += blockDim.x) qs[k] = q[(long long)b * K + k];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int ir = ant[2 * b], m = ant[2 * b + 1];
    float acc = 0.f;
    if (ir >= 0 && ir < NR) {
        const long long base = (long long)ir * D * T;
        for (int k = 0; k < K && S * k - J <= t; ++k) {
            const int d = m - k + moff, tau = t - S * k + J;
            if (d >= 0 && d < D && tau < T && qs[k] != 0.f) {
                const long long i = base + (long long)d * T + tau;
                float gv = val(G[i]);
                if (Glo) gv += bf(Glo[i]);
                acc += qs[k] * gv;
            }
        }
    }
    y[(long long)b * T + t] = acc;
}

__global__ void __launch_bounds__(256) k_lat_bwd(const float *__restrict__ dy, const float *__restrict__ q,
                                                 const int *__restrict__ ant, int K, int NR, int D, int T, int S,
                                                 int J, int moff, float *__restrict__ dG) {
    __shared__ float qs[1024];
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < K; k += blockDim.x) qs[k] = q[(long long)b * K + k];
    __syncthreads();
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= T) return;
    const int ir = ant[2 * b], m = ant[2 * b + 1];
    if (ir < 0 || ir >= NR) return;
    float *g = dG + (long long)ir * D * T;
    const float *r = dy + (long long)b * T;
    for (int k = 0; k < K && tau + S * k - J < T; ++k) {
        const int d = m - k + moff, t = tau + S * k - J;
        if (d >= 0 && d < D && t >= 0 && qs[k] != 0.f) atomicAdd(&g[(long long)d * T + tau], qs[k] * r[t]);
    }
}

// hi = bf16(x), lo = bf16(x - hi): x = hi + lo to about 2^-17 relative
__global__ void k_split_bf16(const float *__restrict__ x, bf16raw *__restrict__ hi, bf16raw *__restrict__ lo,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const bf16raw h = tobf(x[i]);
        hi[i] = h;
        lo[i] = tobf(x[i] - bf(h));
    }
}

// W[a][k][t] = G[ir_a][m_a - k + moff][t - S k + J] (0 where that time or the
// offset is off the table): antenna a's weights, a K x T matrix, for the GEMM
__global__ void k_lat_weights(const bf16raw *__restrict__ G, const int *__restrict__ ant, int K, int NR, int D,
                              int T, int S, int J, int moff, bf16raw *__restrict__ W) {
    const int a = blockIdx.z, k = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int ir = ant[2 * a], d = ant[2 * a + 1] - k + moff, tau = t - S * k + J;
    bf16raw v = 0;
    if (ir >= 0 && ir < NR && d >= 0 && d < D && tau >= 0 && tau < T) v = G[((long long)ir * D + d) * T + tau];
    W[((long long)a * K + k) * T + t] = v;
}

// The same weights K-major: W[a][t][koff + k] (row stride ldw), for the
// tcgen05 GEMM; one thread per (a, t, k), k fastest
__global__ void k_lat_weights_kmajor(const bf16raw *__restrict__ G, const int *__restrict__ ant, int A, int K, int NR,
                                     int D, int T, int S, int J, int moff, bf16raw *__restrict__ W, int ldw,
                                     int koff) {
    const long long n = (long long)A * T * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const long long at = i / K;
        const int t = (int)(at % T), a = (int)(at / T);
        const int ir = ant[2 * a], d = ant[2 * a + 1] - k + moff, tau = t - S * k + J;
        bf16raw v = 0;
        if (ir >= 0 && ir < NR && d >= 0 && d < D && tau >= 0 && tau < T) v = G[((long long)ir * D + d) * T + tau];
        W[at * ldw + koff + k] = v;
    }
}

// out[r] = [hi(x[r]), hi(x[r]), lo(x[r]), 0 ...] (row stride ld >= 3K): the A
// operand of the split-precision product [hi, hi, lo] [W_hi; W_lo; W_hi]
__global__ void k_split3_bf16(const float *__restrict__ x, int rows, int K, bf16raw *__restrict__ out, int ld) {
    const long long n = (long long)rows * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ld);
        const long long r = i / ld;
        bf16raw v = 0;
        if (c < 3 * K) {
            const float xv = x[r * K + c % K];
            const bf16raw h = tobf(xv);
            v = c < 2 * K ? h : tobf(xv - bf(h));
        }
        out[i] = v;
    }
}

}  // namespace

namespace fdtd {
namespace gtc {
// gemm_tc.cu: the tcgen05 kernel's layout for this product (-1: none), the
// path selected by sur_gemm_set_path, and its launch
int tc_layout(const void *A, int lda, int a_kmajor, const void *B, int ldb, int b_kmajor, int K);
int tc_path();
int gemm_tc(int layout, const void *A, int lda, const void *B, int ldb, float *Y, int ldy, void *Yb, int M, int N,
            int K, const float *bias, int relu, int accumulate, cudaStream_t s);
}  // namespace gtc
}  // namespace fdtd

extern "C" {

int sur_gemm_bf16(const void *A, int lda, int a_kmajor, const void *B, int ldb, int b_kmajor, float *Y, int ldy,
                  void *Yb, int M, int N, int K, const float *bias, int relu, int accumulate, void *stream) {
    if (!A || !B || !Y || M < 1 || N < 1 || K < 1 || lda < 1 || ldb < 1 || ldy < N) return FDTD_ERR_ARG;
    if ((a_kmajor ? lda < K : lda < M) || (b_kmajor ? ldb < K : ldb < N)) return FDTD_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // both operands K-major with 16-byte rows: the tcgen05 kernel; else mma.sync
    const int layout = fdtd::gtc::tc_layout(A, lda, a_kmajor, B, ldb, b_kmajor, K);
    if (layout >= 0) return fdtd::gtc::gemm_tc(layout, A, lda, B, ldb, Y, ldy, Yb, M, N, K, bias, relu, accumulate, s);
    if (fdtd::gtc::tc_path() >= 2) return FDTD_ERR_ARG;   // the tcgen05 kernel alone was asked for
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    const bf16raw *a = static_cast<const bf16raw *>(A), *b = static_cast<const bf16raw *>(B);
    bf16raw *yb = static_cast<bf16raw *>(Yb);
    if (a_kmajor && b_kmajor)
        k_gemm<true, true><<<grid, GT, 0, s>>>(a, lda, b, ldb, Y, ldy, yb, M, N, K, bias, relu, accumulate);
    else if (a_kmajor)
        k_gemm<true, false><<<grid, GT, 0, s>>>(a, lda, b, ldb, Y, ldy, yb, M, N, K, bias, relu, accumulate);
    else if (b_kmajor)
        k_gemm<false, true><<<grid, GT, 0, s>>>(a, lda, b, ldb, Y, ldy, yb, M, N, K, bias, relu, accumulate);
    else
        k_gemm<false, false><<<grid, GT, 0, s>>>(a, lda, b, ldb, Y, ldy, yb, M, N, K, bias, relu, accumulate);
    return launched();
}

int sur_conv1d_fwd(const float *x, int xs, const void *w, const float *bias, float *y, int B, int cin, int lin,
                   int cout, int k, int stride, int pad, int relu, void *stream) {
    if (!x || !w || !y || B < 1 || cin < 1 || lin < 1 || cout < 1 || k < 1 || k > 8 || stride < 1 || pad < 0 ||
        xs < cin * lin)
        return FDTD_ERR_ARG;
    const int lout = (lin + 2 * pad - k) / stride + 1;
    if (lout < 1) return FDTD_ERR_ARG;
    const long long n = (long long)B * cout * lout;
    k_conv_fwd<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, xs, static_cast<const bf16raw *>(w), bias, y, B, cin, lin, cout, k, stride, pad, lout, relu);
    return launched();
}

int sur_conv1d_bwd(const float *x, int xs, const void *w, const float *y, const float *dy, int dys, float *dx,
                   float *dw, float *db, int B, int cin, int lin, int cout, int k, int stride, int pad,
                   void *stream) {
    if (!x || !w || !y || !dy || !dw || !db || B < 1 || cin < 1 || lin < 1 || cout < 1 || k < 1 || k > 8 ||
        stride < 1 || pad < 0 || xs < cin * lin)
        return FDTD_ERR_ARG;
    const int lout = (lin + 2 * pad - k) / stride + 1;
    if (lout < 1 || dys < cout * lout) return FDTD_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_conv_bwd_w<<<cout * cin, 256, 0, s>>>(x, xs, y, dy, dys, dw, db, B, cin, lin, cout, k, stride, pad, lout);
    if (dx) {
        const long long n = (long long)B * cin * lin;
        k_conv_bwd_x<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const bf16raw *>(w), y, dy, dys, dx, B, cin,
                                                        lin, cout, k, stride, pad, lout);
    }
    return launched();
}

int sur_relu_bwd(const float *y, const float *dy, float *dz, void *dzb, long long n, void *stream) {
    if (!y || !dy || !dz || n < 1) return FDTD_ERR_ARG;
    k_relu_bwd<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, dy, dz,
                                                                                  static_cast<bf16raw *>(dzb), n);
    return launched();
}

int sur_bias_grad(const float *dz, int ldz, int M, int N, float *db, void *stream) {
    if (!dz || !db || M < 1 || N < 1 || ldz < N) return FDTD_ERR_ARG;
    k_bias_grad<<<(N + 31) / 32, 256, 0, static_cast<cudaStream_t>(stream)>>>(dz, ldz, M, N, db);
    return launched();
}

int sur_cast_bf16(const float *x, void *y, long long n, void *stream) {
    if (!x || !y || n < 1) return FDTD_ERR_ARG;
    k_cast<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, static_cast<bf16raw *>(y), n);
    return launched();
}

int sur_concat_bf16(const float *a, int na, const float *c, int nc, void *out, int B, void *stream) {
    if (!a || !c || !out || na < 1 || nc < 1 || B < 1) return FDTD_ERR_ARG;
    const long long n = (long long)B * (na + nc);
    k_concat<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, na, c, nc,
                                                                               static_cast<bf16raw *>(out), B);
    return launched();
}

int sur_mse(const float *y, const float *t, long long n, float *dy, float *loss, void *stream) {
    if (!y || !t || !dy || n < 1) return FDTD_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return FDTD_ERR_CUDA;
    k_mse<<<grid_for(n, 256), 256, 0, s>>>(y, t, n, dy, loss);
    return launched();
}

int sur_adam(float *w, void *wb, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
             float eps, int t, void *stream) {
    if (!w || !g || !m || !v || n < 1 || t < 1) return FDTD_ERR_ARG;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(w, static_cast<bf16raw *>(wb), g, m, v,
                                                                              n, lr, b1, b2, eps, c1, c2);
    return launched();
}

int sur_normalize_rows(const float *q, int B, int n, float *qn, float *s, void *stream) {
    if (!q || !qn || !s || B < 1 || n < 1) return FDTD_ERR_ARG;
    k_normalize<<<(B + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(q, B, n, qn, s);
    return launched();
}

int sur_antenna_features(const float *rz, int B, float r0, float rs, float z0, float zs, float *out, void *stream) {
    if (!rz || !out || B < 1 || !(rs != 0.f) || !(zs != 0.f)) return FDTD_ERR_ARG;
    k_features<<<grid_for((long long)B * 64, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(rz, B, r0, rs, z0, zs,
                                                                                               out);
    return launched();
}

int sur_scale_rows(float *y, int B, int n, const float *s, float c, int invert, void *stream) {
    if (!y || !s || B < 1 || n < 1) return FDTD_ERR_ARG;
    k_scale_rows<<<grid_for((long long)B * n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, B, n, s, c,
                                                                                               invert);
    return launched();
}

int sur_pairs(const float *rz, int B, int K, float z0, float dz, float *out, void *stream) {
    if (!rz || !out || B < 1 || K < 1) return FDTD_ERR_ARG;
    k_pairs<<<grid_for((long long)B * K, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(rz, B, K, z0, dz, out);
    return launched();
}

int sur_assemble(const float *G, const float *qn, const float *rz, int B, int K, int Tg, int shift, int T, float z0,
                 float dz, float cps, int J0, float *out, void *stream) {
    if (!G || !qn || !rz || !out || B < 1 || K < 1 || Tg < 1 || shift < 0 || T < 1 || !(dz > 0.f) || !(cps > 0.f) ||
        J0 < 0)
        return FDTD_ERR_ARG;
    k_assemble<<<grid_for((long long)B * T, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        G, qn, rz, B, K, Tg, shift, T, z0, dz, cps, J0, out);
    return launched();
}

int sur_assemble_bwd(const float *dout, const float *qn, const float *rz, int B, int K, int Tg, int shift, int T,
                     float z0, float dz, float cps, int J0, float *dG, void *dGb, void *stream) {
    if (!dout || !qn || !rz || !dG || B < 1 || K < 1 || Tg < 1 || shift < 0 || T < 1 || !(dz > 0.f) ||
        !(cps > 0.f) || J0 < 0)
        return FDTD_ERR_ARG;
    k_assemble_bwd<<<grid_for((long long)B * K * Tg, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        dout, qn, rz, B, K, Tg, shift, T, z0, dz, cps, J0, dG, static_cast<bf16raw *>(dGb));
    return launched();
}

int sur_lattice_fwd(const void *G, const void *Glo, const float *q, const int *ant, int B, int K, int NR, int D,
                    int T, int S, int J, int moff, float *y, void *stream) {
    if (!G || !q || !ant || !y || B < 1 || B > 65535 || K < 1 || K > 1024 || NR < 1 || D < 1 || T < 1 || S < 0 ||
        J < 0)
        return FDTD_ERR_ARG;
    k_lat_fwd<bf16raw><<<dim3((T + 255) / 256, B), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16raw *>(G), static_cast<const bf16raw *>(Glo), q, ant, K, NR, D, T, S, J, moff, y);
    return launched();
}

int sur_lattice_fwd_f32(const float *G, const float *q, const int *ant, int B, int K, int NR, int D, int T, int S,
                        int J, int moff, float *y, void *stream) {
    if (!G || !q || !ant || !y || B < 1 || B > 65535 || K < 1 || K > 1024 || NR < 1 || D < 1 || T < 1 || S < 0 ||
        J < 0)
        return FDTD_ERR_ARG;
    k_lat_fwd<float><<<dim3((T + 255) / 256, B), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        G, nullptr, q, ant, K, NR, D, T, S, J, moff, y);
    return launched();
}

int sur_split_bf16(const float *x, void *hi, void *lo, long long n, void *stream) {
    if (!x || !hi || !lo || n < 1) return FDTD_ERR_ARG;
    k_split_bf16<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, static_cast<bf16raw *>(hi), static_cast<bf16raw *>(lo), n);
    return launched();
}

int sur_lattice_bwd(const float *dy, const float *q, const int *ant, int B, int K, int NR, int D, int T, int S,
                    int J, int moff, float *dG, void *stream) {
    if (!dy || !q || !ant || !dG || B < 1 || B > 65535 || K < 1 || K > 1024 || NR < 1 || D < 1 || T < 1 || S < 0 ||
        J < 0)
        return FDTD_ERR_ARG;
    k_lat_bwd<<<dim3((T + 255) / 256, B), 256, 0, static_cast<cudaStream_t>(stream)>>>(dy, q, ant, K, NR, D, T, S,
                                                                                         J, moff, dG);
    return launched();
}

int sur_lattice_weights_kmajor(const void *G, const int *ant, int A, int K, int NR, int D, int T, int S, int J,
                               int moff, void *W, int ldw, int koff, void *stream) {
    if (!G || !ant || !W || A < 1 || K < 1 || NR < 1 || D < 1 || T < 1 || S < 0 || J < 0 || koff < 0 ||
        ldw < koff + K)
        return FDTD_ERR_ARG;
    const long long n = (long long)A * T * K;
    k_lat_weights_kmajor<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16raw *>(G), ant, A, K, NR, D, T, S, J, moff, static_cast<bf16raw *>(W), ldw, koff);
    return launched();
}

int sur_split3_bf16(const float *x, int rows, int K, void *out, int ld, void *stream) {
    if (!x || !out || rows < 1 || K < 1 || ld < 3 * K) return FDTD_ERR_ARG;
    k_split3_bf16<<<grid_for((long long)rows * ld, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, rows, K, static_cast<bf16raw *>(out), ld);
    return launched();
}

int sur_lattice_weights(const void *G, const int *ant, int A, int K, int NR, int D, int T, int S, int J, int moff,
                        void *W, void *stream) {
    if (!G || !ant || !W || A < 1 || A > 65535 || K < 1 || K > 65535 || NR < 1 || D < 1 || T < 1 || S < 0 || J < 0)
        return FDTD_ERR_ARG;
    k_lat_weights<<<dim3((T + 255) / 256, K, A), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16raw *>(G), ant, K, NR, D, T, S, J, moff, static_cast<bf16raw *>(W));
    return launched();
}

}  // extern "C"
