// tma_pipe.cuh -- inline-PTX pieces of the TMA-staged z-march kernels:
// mbarrier pipeline stages, 3-D tensor loads, float4 arithmetic of the field
// update and the CPML recursion, and the host-side tensor-map encoder.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {
namespace tma {

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
// one arrival on a barrier (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}
// make a barrier's memory free for a new mbar_init (no arrival or
// transaction may be pending on it)
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sa(bar)) : "memory");
}
// 3-D tiled tensor load into shared memory, completion counted on bar
__device__ __forceinline__ void tma_load(float *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
// a + s * d, elementwise
__device__ __forceinline__ float4 axpy(float4 a, float s, float4 d) {
    return make_float4(a.x + s * d.x, a.y + s * d.y, a.z + s * d.z, a.w + s * d.w);
}

// CPML recursion psi <- b psi + a d; the derivative becomes d + psi
__device__ __forceinline__ float cpml1(float &psi, float a, float b, float d) {
    psi = b * psi + a * d;
    return d + psi;
}
__device__ __forceinline__ float4 cpml4(float4 &psi, float a, float b, float4 d) {
    return make_float4(cpml1(psi.x, a, b, d.x), cpml1(psi.y, a, b, d.y), cpml1(psi.z, a, b, d.z),
                       cpml1(psi.w, a, b, d.w));
}
// elementwise coefficients
__device__ __forceinline__ float4 cpmlv(float4 &psi, float4 a, float4 b, float4 d) {
    return make_float4(cpml1(psi.x, a.x, b.x, d.x), cpml1(psi.y, a.y, b.y, d.y), cpml1(psi.z, a.z, b.z, d.z),
                       cpml1(psi.w, a.w, b.w, d.w));
}

// zero the whole vector (all) or its first element (first): the components a
// cell owns on the grid's low faces are not updated
__device__ __forceinline__ float4 mask(float4 v, bool all, bool first) {
    if (all) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (first) v.x = 0.f;
    return v;
}
// store the first n (1..4) elements; a 16-byte store when n == 4
__device__ __forceinline__ void st4n(float *p, float4 v, int n) {
    if (n == 4) {
        *reinterpret_cast<float4 *>(p) = v;
    } else {
        p[0] = v.x;
        if (n > 1) p[1] = v.y;
        if (n > 2) p[2] = v.z;
    }
}

// ---- host ----

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, or null
inline EncodeTiled encoder() {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return nullptr;
    }
    return reinterpret_cast<EncodeTiled>(fn);
}

// 3-D float32 tensor map: extents d0 (innermost) .. d2, strides s1, s2 in
// floats, box b0 x b1 x 1; loads outside the extents read zeros
inline bool encode3(EncodeTiled encode, CUtensorMap *m, const float *base, cuuint64_t d0, cuuint64_t d1,
                    cuuint64_t d2, cuuint64_t s1, cuuint64_t s2, cuuint32_t b0, cuuint32_t b1,
                    CUtensorMapL2promotion promo) {
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1 * 4, s2 * 4};
    cuuint32_t box[3] = {b0, b1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace fdtd
