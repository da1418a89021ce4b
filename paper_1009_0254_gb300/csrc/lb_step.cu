// lb_step.cu -- the fused fluctuating D2Q9 step for sm_103a.
//
// One launch performs one time step of [GACV] Eq. (fluct-lin-lbe) on every node:
//   pull   f_i(r,t) = f*_i(r - c_i, t-1)                               (Eq. gen-lbe)
//   rho    density on the CTA tile plus a one-node ring, in shared memory
//   grad   Appendix B Laplacian and the isotropic gradient of rho
//   m      moments m = T f in deviation form (Table I basis, Eq. Tmat)
//   m^eq   Table II with p0 = cs2 rho, C_n = 0, m^F = 0
//   relax  m*_a = m_a + lambda_a (m_a - m_a^eq) + xi_a,  a = 4..9        (Eq. fluct-lin-lbe)
//   noise  xi from Philox4x32-10 keyed (seed, t, node, tag) (Sec. IV); for the
//          correlated mode xi_4, xi_9 read from the k-space synthesis or, built in real
//          space, summed over the 2 x 2 box of draws below-left of the node
//   back   f*_i = w_i sum_a T_ai m*_a / N_a                                 (Sec. III A)
//   store  f*_i(r,t) with its periodic ghost copies.
// Everything is FP32 on deviations from the rest state fbar_i, which keeps the
// small fluctuations (~sqrt(kT)) at full relative precision; with FP64 storage the
// arithmetic is FP64 too (this kernel is the FP64 path).
#include "lb_collide.cuh"

namespace lbf {

template <int BX, int BY>
struct Tile {
    static constexpr int RX = BX + 2;
    static constexpr int RY = BY + 2;
    static constexpr int RING = 2 * RX + 2 * BY;
};

// Pulled deviations at (x, y): f_i(x, y) = f*_i(x - cx_i, y - cy_i).
template <typename T>
__device__ __forceinline__ void pull9(const T* __restrict__ s, long long P, int pitch, long long c,
                                      typename Arith<T>::type f[Q]) {
    f[0] = Elem<T>::load(s[c], 0);
    f[1] = Elem<T>::load(s[P + c - 1], 1);                   // c = ( 1, 0)
    f[2] = Elem<T>::load(s[2 * P + c - pitch], 2);           // c = ( 0, 1)
    f[3] = Elem<T>::load(s[3 * P + c + 1], 3);               // c = (-1, 0)
    f[4] = Elem<T>::load(s[4 * P + c + pitch], 4);           // c = ( 0,-1)
    f[5] = Elem<T>::load(s[5 * P + c - pitch - 1], 5);       // c = ( 1, 1)
    f[6] = Elem<T>::load(s[6 * P + c - pitch + 1], 6);       // c = (-1, 1)
    f[7] = Elem<T>::load(s[7 * P + c + pitch + 1], 7);       // c = (-1,-1)
    f[8] = Elem<T>::load(s[8 * P + c + pitch - 1], 8);       // c = ( 1,-1)
}

// contributions h_d of node q (tile coordinates lx, ly >= -1) to the real-space correlated
// noise, in the arithmetic type (stencil_h in lb_internal.cuh)
template <int HW, typename Args, typename V>
__device__ __forceinline__ void stencil_put(const Args& a, V* H, int HN, int lx, int ly, uint32_t node) {
    decltype(V().x) h[8];
    stencil_h(a, node, h);
    const int q = (ly + 1) * HW + lx + 1;
    H[q].x = h[0]; H[q].y = h[1];
    H[HN + q].x = h[2]; H[HN + q].y = h[3];
    H[2 * HN + q].x = h[4]; H[2 * HN + q].y = h[5];
    H[3 * HN + q].x = h[6]; H[3 * HN + q].y = h[7];
}

template <int BX, int BY, int MODE, typename T, bool POLY>
__global__ void __launch_bounds__(BX * BY) step_kernel(const StepArgsT<typename Arith<T>::type> a) {
    using TL = Tile<BX, BY>;
    using R = typename Arith<T>::type;
    using V = typename Arith<T>::vec2;
    __shared__ R rs[TL::RY][TL::RX];
    // real-space correlated noise (MODE 3): h00, h10, h01, h11 of the tile's nodes and of the
    // column left of it and the row below it
    constexpr int HW = BX + 1, HN = (BX + 1) * (BY + 1);
    __shared__ V H[MODE == 3 ? 4 * HN : 1];
    const Grid g = a.g;
    const T* __restrict__ src = static_cast<const T*>(a.src);
    const long long P = g.plane;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = (x < g.nx) && (y < g.ny);

    // 1. density on the tile (plus the first column/row past a ragged edge)
    R f[Q];
    if (x <= g.nx && y <= g.ny) {
        pull9(src, P, g.pitch, g.at(x, y), f);
        rs[ty + 1][tx + 1] = drho_of(f);
    } else {
        rs[ty + 1][tx + 1] = R(0);
    }
    // 2. density on the one-node ring around the tile
    const int tid = ty * BX + tx;
    for (int q = tid; q < TL::RING; q += BX * BY) {
        int hx, hy;
        if (q < TL::RX) {
            hx = q - 1; hy = -1;
        } else if (q < 2 * TL::RX) {
            hx = q - TL::RX - 1; hy = BY;
        } else if (q < 2 * TL::RX + BY) {
            hx = -1; hy = q - 2 * TL::RX;
        } else {
            hx = BX; hy = q - 2 * TL::RX - BY;
        }
        const int gx = x0 + hx, gy = y0 + hy;
        R v = R(0);
        if (gx >= -1 && gx <= g.nx && gy >= -1 && gy <= g.ny) {
            R h[Q];
            pull9(src, P, g.pitch, g.at(gx, gy), h);
            v = drho_of(h);
        }
        rs[hy + 1][hx + 1] = v;
    }
    if (MODE == 3) {
        if (own) stencil_put<HW>(a, H, HN, tx, ty, (uint32_t)y * (uint32_t)g.nx + (uint32_t)x);
        for (int j = tid; j < BX + BY + 1; j += BX * BY) {
            int lx, ly;
            if (j <= BY) { lx = -1; ly = j - 1; }
            else { lx = j - (BY + 1); ly = -1; }
            int gx = x0 + lx, gy = y0 + ly;
            if (gx < 0) gx += g.nx;
            if (gy < 0) gy += g.ny;
            if (gx < g.nx && gy < g.ny) stencil_put<HW>(a, H, HN, lx, ly, (uint32_t)gy * (uint32_t)g.nx + (uint32_t)gx);
        }
    }
    __syncthreads();
    if (!own) return;

    // 3.-8. stencil, moments, equilibrium, noise, relaxation, back-transform
    NbrT<R> r;
    r.C = rs[ty + 1][tx + 1];
    r.E = rs[ty + 1][tx + 2]; r.W = rs[ty + 1][tx];
    r.N = rs[ty + 2][tx + 1]; r.S = rs[ty][tx + 1];
    r.NE = rs[ty + 2][tx + 2]; r.NW = rs[ty + 2][tx];
    r.SE = rs[ty][tx + 2]; r.SW = rs[ty][tx];
    const uint32_t node = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
    typename Arith<T>::vec2 z{};
    if (MODE == 2) z = a.xi49[(long long)y * g.nx + x];
    if (MODE == 3) {
        const int q = (ty + 1) * HW + tx + 1;
        const V h00 = H[q], h10 = H[HN + q - 1], h01 = H[2 * HN + q - HW], h11 = H[3 * HN + q - HW - 1];
        z.x = (h00.x + h10.x) + (h01.x + h11.x);
        z.y = (h00.y + h10.y) + (h01.y + h11.y);
    }
    R o[Q];
    collide_node<MODE, POLY>(a, f, r, node, z, o);

    // 9. store (own node plus periodic ghosts)
    store9(static_cast<T*>(a.dst), P, g, x, y, o);
}

template <typename T, bool POLY>
static void launch_p(const StepArgsT<typename Arith<T>::type>& a, int noise_mode, cudaStream_t s) {
    constexpr int BX = 32, BY = 16;
    dim3 block(BX, BY);
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY);
    switch (noise_mode) {
        case 0: step_kernel<BX, BY, 0, T, POLY><<<grid, block, 0, s>>>(a); break;
        case 1: step_kernel<BX, BY, 1, T, POLY><<<grid, block, 0, s>>>(a); break;
        case 3: step_kernel<BX, BY, 3, T, POLY><<<grid, block, 0, s>>>(a); break;
        case 4: step_kernel<BX, BY, 4, T, POLY><<<grid, block, 0, s>>>(a); break;
        default: step_kernel<BX, BY, 2, T, POLY><<<grid, block, 0, s>>>(a); break;
    }
}

// the double-well equation of state (a.eos) is a separate instantiation
template <typename T>
static void launch_t(const StepArgsT<typename Arith<T>::type>& a, int noise_mode, cudaStream_t s) {
    if (a.eos) launch_p<T, true>(a, noise_mode, s);
    else launch_p<T, false>(a, noise_mode, s);
}

cudaError_t launch_step_simple(const StepArgs& a, int noise_mode, int fp16, cudaStream_t s) {
    if (fp16) launch_t<__half>(a, noise_mode, s);
    else launch_t<float>(a, noise_mode, s);
    return cudaGetLastError();
}

cudaError_t launch_step_simple_d(const StepArgsD& a, int noise_mode, cudaStream_t s) {
    launch_t<double>(a, noise_mode, s);
    return cudaGetLastError();
}

}  // namespace lbf
