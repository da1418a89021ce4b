// lb_step_sweep.cu -- the fused fluctuating D2Q9 step as a warp-autonomous vertical sweep.
//
// Same arithmetic as the other step kernels (collide_node); the data movement avoids
// shared memory and block barriers altogether:
//   * each warp owns a strip of 32 columns (lane = column) and H rows and walks it upward;
//   * the pulled populations of the row being collided stay in registers, the next row's
//     are loaded (coalesced, one 128-byte line per plane and warp) one iteration ahead;
//   * the density is kept as a rolling window of three rows in registers; the east/west
//     neighbours come from warp shuffles, lanes 0 and 31 also form the density of the two
//     halo columns x0-1 and x0+32 (the only redundant work besides the strip's two halo
//     rows);
//   * the next row's loads are issued before the current row's random numbers and
//     moments, which cover their latency.
#include "lb_collide.cuh"

namespace lbf {

constexpr int SWEEP_H = 64;          // rows per strip
constexpr int SWEEP_WARPS = 4;       // strips (warps) per CTA, side by side

// Element offsets are 32-bit here: the launcher only uses this kernel while the nine
// planes of a buffer hold fewer than 2^31 elements.
template <typename T>
__device__ __forceinline__ void pull_row(const T* __restrict__ s, uint32_t P, uint32_t pitch, uint32_t c, float f[Q]) {
    f[0] = Elem<T>::load(s[c], 0);
    f[1] = Elem<T>::load(s[P + c - 1u], 1);
    f[2] = Elem<T>::load(s[2u * P + c - pitch], 2);
    f[3] = Elem<T>::load(s[3u * P + c + 1u], 3);
    f[4] = Elem<T>::load(s[4u * P + c + pitch], 4);
    f[5] = Elem<T>::load(s[5u * P + c - pitch - 1u], 5);
    f[6] = Elem<T>::load(s[6u * P + c - pitch + 1u], 6);
    f[7] = Elem<T>::load(s[7u * P + c + pitch + 1u], 7);
    f[8] = Elem<T>::load(s[8u * P + c + pitch - 1u], 8);
}

// density deviation of the halo column this lane is responsible for (lane 0: x0-1,
// lane 31: x0+32), zero on the other lanes
template <typename T>
__device__ __forceinline__ float halo_rho(const T* __restrict__ s, uint32_t P, uint32_t pitch, uint32_t ch, bool halo) {
    if (!halo) return 0.0f;
    float h[Q];
    pull_row(s, P, pitch, ch, h);
    return drho_of(h);
}

template <int MODE, typename T, int MINB>
__global__ void __launch_bounds__(SWEEP_WARPS * 32, MINB) step_sweep_kernel(const StepArgs a) {
    const Grid g = a.g;
    const uint32_t P = (uint32_t)g.plane;
    const T* __restrict__ src = static_cast<const T*>(a.src);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int x0 = (blockIdx.x * SWEEP_WARPS + warp) * 32;
    if (x0 >= g.nx) return;                       // whole warp beyond the lattice
    const int x = x0 + lane;                      // x <= nx + 31 stays inside the padded row
    const int y0 = blockIdx.y * SWEEP_H;
    const int y1 = min(y0 + SWEEP_H, g.ny);
    const bool own_col = x < g.nx;
    // the west halo is always inside [-1, nx]; the east one only matters if column x0+31 is ours
    const bool halo = (lane == 0) || (lane == 31 && x0 + 31 < g.nx);
    const int xh = lane == 0 ? x0 - 1 : x0 + 32;  // halo column of lanes 0 and 31

    // rolling window: rows y-1 (m), y (c), y+1 (p)
    float fc[Q], fn[Q];
    const uint32_t pitch = (uint32_t)g.pitch;
    uint32_t cn = (uint32_t)g.at(x, y0 - 1), chn = (uint32_t)g.at(xh, y0 - 1);
    pull_row(src, P, pitch, cn, fn);
    float rm = drho_of(fn);
    float hm = halo_rho(src, P, pitch, chn, halo);
    cn += pitch; chn += pitch;
    pull_row(src, P, pitch, cn, fc);
    float rc = drho_of(fc);
    float hc = halo_rho(src, P, pitch, chn, halo);

    for (int y = y0; y < y1; ++y) {
        // next row (y + 1 <= ny is inside the ghost rows)
        cn += pitch; chn += pitch;
        pull_row(src, P, pitch, cn, fn);
        const float hp = halo_rho(src, P, pitch, chn, halo);
        const float rp = drho_of(fn);

        // 3x3 density neighbourhood from the window and the shuffles
        Nbr r;
        r.C = rc;
        r.N = rp;
        r.S = rm;
        float e = __shfl_down_sync(0xffffffffu, rc, 1), w = __shfl_up_sync(0xffffffffu, rc, 1);
        float ne = __shfl_down_sync(0xffffffffu, rp, 1), nw = __shfl_up_sync(0xffffffffu, rp, 1);
        float se = __shfl_down_sync(0xffffffffu, rm, 1), sw = __shfl_up_sync(0xffffffffu, rm, 1);
        if (lane == 31) { e = hc; ne = hp; se = hm; }
        if (lane == 0) { w = hc; nw = hp; sw = hm; }
        r.E = e; r.W = w; r.NE = ne; r.NW = nw; r.SE = se; r.SW = sw;

        if (own_col) {
            const uint32_t node = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
            float2 z = make_float2(0.f, 0.f);
            if (MODE == 2) z = a.xi49[(long long)y * g.nx + x];
            float o[Q];
            collide_node<MODE>(a, fc, r, node, z, o);
            store9(static_cast<T*>(a.dst), P, g, x, y, o);
        }
        // slide the window
        rm = rc; rc = rp;
        hm = hc; hc = hp;
#pragma unroll
        for (int i = 0; i < Q; ++i) fc[i] = fn[i];
    }
}

template <typename T, int MINB>
static void launch_sweep_t(const StepArgs& a, int noise_mode, cudaStream_t s) {
    dim3 grid((a.g.nx + 32 * SWEEP_WARPS - 1) / (32 * SWEEP_WARPS), (a.g.ny + SWEEP_H - 1) / SWEEP_H);
    dim3 block(32 * SWEEP_WARPS);
    switch (noise_mode) {
        case 0: step_sweep_kernel<0, T, MINB><<<grid, block, 0, s>>>(a); break;
        case 1: step_sweep_kernel<1, T, MINB><<<grid, block, 0, s>>>(a); break;
        default: step_sweep_kernel<2, T, MINB><<<grid, block, 0, s>>>(a); break;
    }
}

bool sweep_fits(const Grid& g) { return (long long)Q * g.plane < (1ll << 31); }

// occupancy: 8 resident CTAs per SM (<= 64 registers) or 6 (<= 85 registers)
cudaError_t launch_step_sweep(const StepArgs& a, int noise_mode, int fp16, int occ6, cudaStream_t s) {
    if (fp16) {
        if (occ6) launch_sweep_t<__half, 6>(a, noise_mode, s);
        else launch_sweep_t<__half, 8>(a, noise_mode, s);
    } else {
        if (occ6) launch_sweep_t<float, 6>(a, noise_mode, s);
        else launch_sweep_t<float, 8>(a, noise_mode, s);
    }
    return cudaGetLastError();
}

}  // namespace lbf
