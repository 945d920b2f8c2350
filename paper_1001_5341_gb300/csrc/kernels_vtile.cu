// kernels_vtile.cu -- one-pass leapfrog step over the whole grid (path 1):
// one block per (tile, z chunk), the block body of vtile_tile.cuh.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "fdtd_internal.h"
#include "vtile_tile.cuh"

namespace fdtd {
namespace {

using namespace vt;

// the form without block barriers: NW warps and the refill warp
__global__ void __launch_bounds__(NT + 32, 1) k_vtile(const Args A, const __grid_constant__ Maps M) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    tile_block<true, true>(A, M, (int)blockIdx.x, (int)blockIdx.y, smem_raw);
}

constexpr CUtensorMapL2promotion kPromotion =
    VT_L2PROMO == 0 ? CU_TENSOR_MAP_L2_PROMOTION_NONE
    : VT_L2PROMO == 1 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
    : VT_L2PROMO == 2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B;

bool encode3(EncodeTiled encode, CUtensorMap *m, const float *base, cuuint64_t d0, cuuint64_t d1, cuuint64_t d2,
             cuuint64_t s1, cuuint64_t s2, cuuint32_t b0, cuuint32_t b1) {
    return tma::encode3(encode, m, base, d0, d1, d2, s1, s2, b0, b1, kPromotion);
}

}  // namespace

const char *vtile_name() { return "fused-vtile-128x8"; }

int vtile_prepare(fdtd_ctx *h) {
    const Grid &g = h->g;
    const int P = h->P;
    if ((unsigned long long)g.comp >= (1ull << 32) || g.pitch % 4 != 0) return FDTD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((unsigned long long)h->psi_axis[a] >= (1ull << 32)) return FDTD_ERR_ARG;
    // the x layers must not share a group of four columns; x boxes within the
    // TMA box extent
    const int xlo4 = P > 0 ? psi_x_lo4(P) : 0, xhb = P > 0 ? psi_x_hb(g.nx, P) : 0;
    const int WX = P > 0 ? psi_x_row(g.nx, P) : 0;
    const int xbw = P > 0 ? (xlo4 > WX - xlo4 ? xlo4 : WX - xlo4) : 4;
    if (P > 0 && (g.nx < 2 * P + 8 || xbw > 256 || g.nz < 2 * P + 2)) return FDTD_ERR_ARG;
    EncodeTiled encode = encoder();
    if (!encode) return FDTD_ERR_CUDA;
    HostState *st = new (std::nothrow) HostState();
    if (!st) return FDTD_ERR_OOM;
    st->xlo4 = xlo4;
    st->xhb = xhb;
    st->xbw = xbw;
    bool ok = true;
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 6; ++c)
            ok = ok && encode3(encode, &st->maps.f[s][c], h->fields[s] + (size_t)c * g.comp, g.nx + 1, g.ny + 1,
                               g.nz + 1, g.pitch, g.plane, fb_w(c), fb_r(c));
    if (P > 0) {
        // psi block: E psi, then H psi set 0, then H psi set 1 (each set the
        // x, y, z arrays in turn, two per axis); the H set read when cur == s
        // is set s.  The second E psi set (epsi2, same layout) is the one the
        // two-step path leaves current every other launch.
        const size_t set = 2 * (h->psi_axis[0] + h->psi_axis[1] + h->psi_axis[2]);
        const int W = 2 * P + 1;
        for (int s = 0; s < 2; ++s) {
            size_t off = 0;
            for (int axis = 0; axis < 3; ++axis)
                for (int t = 0; t < 2; ++t) {
                    const float *hp = h->psi_block + set * (1 + s) + off;   // H array t of axis, field set s
                    const float *ep = (s == 0 ? h->psi_block : h->epsi2) + off;  // E array t of axis, E set s
                    off += h->psi_axis[axis];
                    for (int half = 0; half < 2; ++half) {
                        const float *base = half == 0 ? hp : ep;
                        const int a = 2 * half + t;
                        CUtensorMap *m = axis == 0 ? &st->maps.x[a][s] : axis == 1 ? &st->maps.y[a][s] : &st->maps.z[a][s];
                        if (axis == 0)
                            ok = ok && encode3(encode, m, base, WX, g.ny, g.nz, WX, (cuuint64_t)g.ny * WX, xbw, PR);
                        else if (axis == 1)
                            ok = ok && encode3(encode, m, base, g.nx, W, g.nz, g.pitch, (cuuint64_t)W * g.pitch, PW, PR);
                        else
                            ok = ok && encode3(encode, m, base, g.nx, g.ny, W, g.pitch, (cuuint64_t)g.ny * g.pitch, PW, PR);
                    }
                }
        }
    }
    if (!ok) {
        delete st;
        return FDTD_ERR_CUDA;
    }
    st->tiles_x = (g.nx + TXC - 1) / TXC;
    st->tiles_y = (g.ny + BY - 1) / BY;
    // z chunks: the layers [0, P] and [nz-P, nz) as chunks of their own, the
    // planes between them in m chunks of cm.  With one block per SM, the
    // middle blocks run in ceil(tiles m / SMs) waves of about cm + 4 plane
    // times each (warm-up plane and pipeline fill); m minimises that, chunks
    // of at least 16 planes.  More chunks where the coefficient table of a
    // long chunk leaves the ring too small for two of the largest stages.
    const int mid = P > 0 ? g.nz - 2 * P - 1 : g.nz;
    const long long sms = h->num_sms > 0 ? h->num_sms : 1;
    const long long tiles = (long long)st->tiles_x * st->tiles_y;
    // chunks of at most CM_MAX planes: the blocks of a wave share halo rows
    // through L2 only while they stay within a few planes of each other
    constexpr long long CM_MAX = 160;
    const long long m_lo = std::max(1LL, (mid + CM_MAX - 1) / CM_MAX);
    const long long m_hi = std::max(m_lo, (long long)(mid / 16));
    long long m = m_lo, best = -1;
    for (long long mm = m_lo; mm <= m_hi; ++mm) {
        const long long cm = (mid + mm - 1) / mm;
        const long long cost = (tiles * mm + sms - 1) / sms * (cm + 4);
        if (best < 0 || cost < best) { best = cost; m = mm; }
    }
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const bool fits = z_chunks(g.nz, P, xbw, m, (long long)max_smem / 4 - BAR_BYTES / 4, st->z);
    st->smem = BAR_BYTES + 4 * (size_t)(head_floats(st->z.zc) + st->z.ring);
    if (!fits ||
        cudaFuncSetAttribute(k_vtile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem) != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return FDTD_ERR_CUDA;
    }
    h->vtile = st;
    return FDTD_OK;
}

void vtile_release(fdtd_ctx *h) {
    delete static_cast<HostState *>(h->vtile);
    h->vtile = nullptr;
}

void launch_vtile(fdtd_ctx *h, cudaStream_t s) {
    HostState *st = static_cast<HostState *>(h->vtile);
    const Grid &g = h->g;
    Args a;
    a.g = g;
    float *out = h->fields[h->cur ^ 1];
    const size_t c = (size_t)g.comp;
    a.oex = out; a.oey = out + c; a.oez = out + 2 * c; a.ohx = out + 3 * c; a.ohy = out + 4 * c; a.ohz = out + 5 * c;
    a.pml = cpml_view(h);
    a.tiles_x = st->tiles_x;
    a.tiles_y = st->tiles_y;
    a.za = st->z.za;
    a.zb = st->z.zb;
    a.cm = st->z.cm;
    a.m = st->z.m;
    a.zc = st->z.zc;
    a.ring = st->z.ring;
    a.xlo4 = st->xlo4;
    a.xhb = st->xhb;
    a.xbw = st->xbw;
    a.cur = h->cur;
    a.ecur = h->ecur;
    a.src = h->src;
    a.ss = source_window(h->src, h->steps);
    a.kE = (float)h->kE;
    a.kH = (float)h->kH;
    a.flags = h->d_flags;
    dim3 grid(st->tiles_x * st->tiles_y, st->z.chunks);
    k_vtile<<<grid, NT + 32, st->smem, s>>>(a, st->maps);
}

}  // namespace fdtd
