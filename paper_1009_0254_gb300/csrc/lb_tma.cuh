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
    // real-space correlated noise: h00, h10, h01, h11 (float2 each) of the tile's nodes and of
    // the column left of it and the row below it, (TX + 1) x (TY + 1) nodes, after the mbarriers
    static constexpr int HW = TX + 1;
    static constexpr int HN = (TX + 1) * (TY + 1);
    static constexpr int H_BYTES = 4 * HN * 8;
    static constexpr int H_OFFSET = SMEM_BYTES;        // 16-byte aligned: RW, RH even
    static_assert(H_OFFSET % 16 == 0, "H must be 16-byte aligned");
    // whether H fits in the memory of one stage (FP32 storage): the engines put it in the
    // stage just consumed and refill that stage after the collision pass
    static constexpr bool H_IN_STAGE = H_BYTES <= STAGE_BYTES;
};

static __constant__ int kCYt[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// cuTensorMapEncodeTiled of the driver, looked up once per process (thread-safe); null if
// the driver does not provide it
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

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
template <int PS, typename T, bool GF = false>
__device__ __forceinline__ void load9_ps(const T* S, int b, float f[Q]) {
    auto ld = [](T v, int i) -> float {
        if constexpr (GF) return Elem<T>::load_g(v);
        else return Elem<T>::load(v, i);
    };
    f[0] = ld(S[b], 0);
    f[1] = ld(S[PS + b - 1], 1);
    f[2] = ld(S[2 * PS + b], 2);
    f[3] = ld(S[3 * PS + b + 1], 3);
    f[4] = ld(S[4 * PS + b], 4);
    f[5] = ld(S[5 * PS + b - 1], 5);
    f[6] = ld(S[6 * PS + b + 1], 6);
    f[7] = ld(S[7 * PS + b + 1], 7);
    f[8] = ld(S[8 * PS + b - 1], 8);
}

// Real-space correlated noise of a tile (LB_NOISE_FULL_RS): the contributions h_d(q) of a
// node q of the tile, or of the column left of it / row below it (local coordinates -1),
// go to H[d][(ly + 1) * HW + lx + 1]; the (xi_4, xi_9) of a tile node are then
// h00(r) + h10(r - e_x) + h01(r - e_y) + h11(r - e_x - e_y).
template <int HW, typename Args>
__device__ __forceinline__ void stencil_store(const Args& a, float2* H, int HN, int lx, int ly, uint32_t node) {
    float h[8];
    stencil_h(a, node, h);
    const int q = (ly + 1) * HW + lx + 1;
    H[q] = make_float2(h[0], h[1]);
    H[HN + q] = make_float2(h[2], h[3]);
    H[2 * HN + q] = make_float2(h[4], h[5]);
    H[3 * HN + q] = make_float2(h[6], h[7]);
}

// the halo nodes of the tile at (x0, y0): j in [0, TY] -> column x0 - 1, rows y0 - 1 ..
// y0 + TY - 1; j in (TY, TX + TY] -> row y0 - 1, columns x0 .. x0 + TX - 1 (periodic; nodes
// past a ragged edge are skipped, no tile node reads them).  They go to the last threads of
// the block, which form no density-ring node, so the work before the tile's barrier evens out.
template <int TX, int TY, int HW, typename Args>
__device__ __forceinline__ void stencil_halo(const Args& a, float2* H, int HN, int x0, int y0, int nx, int ny,
                                             int tid, int nthreads) {
    for (int j = nthreads - 1 - tid; j < TX + TY + 1; j += nthreads) {
        int lx, ly;
        if (j <= TY) { lx = -1; ly = j - 1; }
        else { lx = j - (TY + 1); ly = -1; }
        int gx = x0 + lx, gy = y0 + ly;
        if (gx < 0) gx += nx;
        if (gy < 0) gy += ny;
        if (gx < nx && gy < ny) stencil_store<HW>(a, H, HN, lx, ly, (uint32_t)gy * (uint32_t)nx + (uint32_t)gx);
    }
}

template <int HW>
__device__ __forceinline__ float2 stencil_xi(const float2* H, int HN, int lx, int ly) {
    const int q = (ly + 1) * HW + lx + 1;
    const float2 a = H[q], b = H[HN + q - 1], c = H[2 * HN + q - HW], d = H[3 * HN + q - HW - 1];
    return make_float2((a.x + b.x) + (c.x + d.x), (a.y + b.y) + (c.y + d.y));
}

}  // namespace lbf
