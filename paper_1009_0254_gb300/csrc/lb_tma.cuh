// lb_tma.cuh -- TMA, mbarrier and tile helpers shared by the TMA-staged step kernels.
#pragma once

#include <cuda.h>

#include "lb_internal.cuh"

namespace lbf {

template <int TX, int TY, typename T>
struct TmaTile {
    static constexpr int XO = Elem<T>::XO;                              // 16 bytes of elements
    static constexpr int BW = TX + 2 * XO;                              // box width (elements)
    static constexpr int BH = TY + 2;                                   // box height
    static constexpr int PLANE_BYTES = BW * BH * (int)sizeof(T);
    static constexpr int PS = ((PLANE_BYTES + 127) / 128) * 128 / (int)sizeof(T);   // plane stride (elements)
    static constexpr int STAGE = Q * PS;                                // elements per stage
    static constexpr int STAGE_BYTES = STAGE * (int)sizeof(T);
    static constexpr int RW = TX + 2, RH = TY + 2;                      // density tile + ring
    static constexpr int SMEM_BYTES = 2 * STAGE_BYTES + RW * RH * 4 + 2 * 8;
    static constexpr uint32_t TX_BYTES = Q * PLANE_BYTES;
};

static __constant__ int kCYt[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s: far beyond any healthy tile load

// Bounded wait on an mbarrier phase (false once limit_ns have passed); the decision to give
// up is made by the caller collectively (__syncthreads_or) so that no thread of the block
// is left at a barrier.
__device__ __forceinline__ bool mbar_wait_bounded_ns(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const uint64_t t0 = global_ns();
        while (!(ok = mbar_try_wait(bar, parity)))
            if (global_ns() - t0 > limit_ns) break;
    }
    return ok;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    return mbar_wait_bounded_ns(bar, parity, WAIT_LIMIT_NS);
}

// The nine pulled deviations of the node whose unshifted box index is b: plane i is read at
// b - cx_i (its y shift is already in the box origin).
template <int PS, typename T>
__device__ __forceinline__ void load9_ps(const T* S, int b, float f[Q]) {
    f[0] = Elem<T>::load(S[b], 0);
    f[1] = Elem<T>::load(S[PS + b - 1], 1);
    f[2] = Elem<T>::load(S[2 * PS + b], 2);
    f[3] = Elem<T>::load(S[3 * PS + b + 1], 3);
    f[4] = Elem<T>::load(S[4 * PS + b], 4);
    f[5] = Elem<T>::load(S[5 * PS + b - 1], 5);
    f[6] = Elem<T>::load(S[6 * PS + b + 1], 6);
    f[7] = Elem<T>::load(S[7 * PS + b + 1], 7);
    f[8] = Elem<T>::load(S[8 * PS + b - 1], 8);
}

}  // namespace lbf
