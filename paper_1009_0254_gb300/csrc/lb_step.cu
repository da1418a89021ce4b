// lb_step.cu -- the fused fluctuating D2Q9 step for sm_103a.
//
// One launch performs one time step of [GACV] Eq. (fluct-lin-lbe) on every node:
//   pull   f_i(r,t) = f*_i(r - c_i, t-1)                               (Eq. gen-lbe)
//   rho    density on the CTA tile plus a one-node ring, in shared memory
//   grad   Appendix B Laplacian and the isotropic gradient of rho
//   m      moments m = T f in deviation form (Table I basis, Eq. Tmat)
//   m^eq   Table II with p0 = cs2 rho, C_n = 0, m^F = 0
//   relax  m*_a = m_a + lambda_a (m_a - m_a^eq) + xi_a,  a = 4..9        (Eq. fluct-lin-lbe)
//   noise  xi from Philox4x32-10 keyed (seed, t, node, tag) (Sec. IV), or for the
//          correlated mode xi_4, xi_9 read from the k-space synthesis
//   back   f*_i = w_i sum_a T_ai m*_a / N_a                                 (Sec. III A)
//   store  f*_i(r,t) with its periodic ghost copies.
// Everything is FP32 on deviations from the rest state fbar_i, which keeps the
// small fluctuations (~sqrt(kT)) at full relative precision.
#include "lb_internal.cuh"

namespace lbf {

template <int BX, int BY>
struct Tile {
    static constexpr int RX = BX + 2;
    static constexpr int RY = BY + 2;
    static constexpr int RING = 2 * RX + 2 * BY;
};

// Pulled deviations at (x, y): f_i(x, y) = f*_i(x - cx_i, y - cy_i).
__device__ __forceinline__ void pull9(const float* __restrict__ s, long long P, int pitch, long long c,
                                      float f[Q]) {
    f[0] = __ldg(s + c);
    f[1] = __ldg(s + P + c - 1);                   // c = ( 1, 0)
    f[2] = __ldg(s + 2 * P + c - pitch);           // c = ( 0, 1)
    f[3] = __ldg(s + 3 * P + c + 1);               // c = (-1, 0)
    f[4] = __ldg(s + 4 * P + c + pitch);           // c = ( 0,-1)
    f[5] = __ldg(s + 5 * P + c - pitch - 1);       // c = ( 1, 1)
    f[6] = __ldg(s + 6 * P + c - pitch + 1);       // c = (-1, 1)
    f[7] = __ldg(s + 7 * P + c + pitch + 1);       // c = (-1,-1)
    f[8] = __ldg(s + 8 * P + c + pitch - 1);       // c = ( 1,-1)
}

// density deviation with one fixed summation order (used for the node and the ring)
__device__ __forceinline__ float drho_of(const float f[Q]) {
    const float sa = (f[1] + f[3]) + (f[2] + f[4]);
    const float sd = (f[5] + f[7]) + (f[6] + f[8]);
    return f[0] + sa + sd;
}

template <int BX, int BY, int MODE>
__global__ void __launch_bounds__(BX * BY) step_kernel(const StepArgs a) {
    using TL = Tile<BX, BY>;
    __shared__ float rs[TL::RY][TL::RX];
    const Grid g = a.g;
    const long long P = g.plane;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = (x < g.nx) && (y < g.ny);

    // 1. density on the tile (plus the first column/row past a ragged edge)
    float f[Q];
    if (x <= g.nx && y <= g.ny) {
        pull9(a.src, P, g.pitch, g.at(x, y), f);
        rs[ty + 1][tx + 1] = drho_of(f);
    } else {
        rs[ty + 1][tx + 1] = 0.0f;
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
        float v = 0.0f;
        if (gx >= -1 && gx <= g.nx && gy >= -1 && gy <= g.ny) {
            float h[Q];
            pull9(a.src, P, g.pitch, g.at(gx, gy), h);
            v = drho_of(h);
        }
        rs[hy + 1][hx + 1] = v;
    }
    __syncthreads();
    if (!own) return;

    // 3. stencils on the density (deviations; the constant rho0 drops out)
    const float rC = rs[ty + 1][tx + 1];
    const float rE = rs[ty + 1][tx + 2], rW = rs[ty + 1][tx];
    const float rN = rs[ty + 2][tx + 1], rS = rs[ty][tx + 1];
    const float rNE = rs[ty + 2][tx + 2], rNW = rs[ty + 2][tx];
    const float rSE = rs[ty][tx + 2], rSW = rs[ty][tx];
    // Appendix B: sum_{i != 1} w_i [rho(r+c_i) + rho(r-c_i) - 2 rho(r)] / sigma_s^2
    const float lap = (4.0f * ((rE + rW) + (rN + rS)) + ((rNE + rSW) + (rNW + rSE)) - 20.0f * rC) * (1.0f / 6.0f);
    // d_alpha rho = 3 sum_i w_i c_i,alpha rho(r + c_i)
    const float gxr = (rE - rW) * (1.0f / 3.0f) + ((rNE - rSW) + (rSE - rNW)) * (1.0f / 12.0f);
    const float gyr = (rN - rS) * (1.0f / 3.0f) + ((rNE - rSW) + (rNW - rSE)) * (1.0f / 12.0f);

    // 4. moments of the deviations (rows of T, Eq. Tmat)
    const float sa = (f[1] + f[3]) + (f[2] + f[4]);
    const float sd = (f[5] + f[7]) + (f[6] + f[8]);
    const float drho = f[0] + sa + sd;
    const float ax = f[1] - f[3], ay = f[2] - f[4];
    const float dx = (f[5] - f[7]) + (f[8] - f[6]);
    const float dy = (f[5] - f[7]) + (f[6] - f[8]);
    const float jx = ax + dx, jy = ay + dy;
    const float m4 = -2.0f * f[0] + sa + 4.0f * sd;
    const float m5 = (f[1] + f[3]) - (f[2] + f[4]);
    const float m6 = (f[5] + f[7]) - (f[6] + f[8]);
    const float m7 = 2.0f * dx - ax;
    const float m8 = 2.0f * dy - ay;
    const float m9 = 2.0f * f[0] - 4.0f * sa + 8.0f * sd;

    // 5. equilibrium deviations, Table II
    const float rho = a.rho0 + drho;
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv;
    const float iso = a.cs2m * drho - a.kappa * rho * lap;        // p0 - rho s^2 - k rho lap, minus rest value
    const float e_eq = 3.0f * (jx * ux + jy * uy) + 6.0f * iso;
    const float pww_eq = (jx * ux - jy * uy) + a.kappa * (gxr * gxr - gyr * gyr);
    const float pxy_eq = jx * uy + a.kappa * gxr * gyr;
    const float eps_eq = -6.0f * iso - 3.0f * a.kappa * (gxr * gxr + gyr * gyr);

    // 6. noise
    float xi4 = 0.f, xi5 = 0.f, xi6 = 0.f, xi7 = 0.f, xi8 = 0.f, xi9 = 0.f;
    if (MODE != 0) {
        const uint32_t node = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
        const uint4 r0 = philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_MODES_5_8), a.key0, a.key1);
        const float2 g01 = gauss_pair(r0.x, r0.y);
        const float2 g23 = gauss_pair(r0.z, r0.w);
        xi5 = a.s5 * g01.x;
        xi6 = a.s6 * g01.y;
        xi7 = a.s7 * g23.x;
        xi8 = a.s7 * g23.y;
        if (MODE == 1) {
            const uint4 r1 = philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_MODES_4_9), a.key0, a.key1);
            const float2 n49 = gauss_pair(r1.x, r1.y);
            xi4 = a.L44 * n49.x;
            xi9 = a.L94 * n49.x + a.L99 * n49.y;
        } else {
            const float2 z = a.xi49[(long long)y * g.nx + x];
            xi4 = z.x;
            xi9 = z.y;
        }
    }

    // 7. relaxation of the non-conserved modes, Eq. (fluct-lin-lbe)
    const float m4s = m4 + a.lb * (m4 - e_eq) + xi4;
    const float m5s = m5 + a.ls * (m5 - pww_eq) + xi5;
    const float m6s = m6 + a.ls * (m6 - pxy_eq) + xi6;
    const float m7s = m7 + a.lq * m7 + xi7;
    const float m8s = m8 + a.lq * m8 + xi8;
    const float m9s = m9 + a.le * (m9 - eps_eq) + xi9;

    // 8. back to populations: f*_i = w_i sum_a T_ai m*_a / N_a
    const float u1 = drho, u2 = 3.0f * jx, u3 = 3.0f * jy;
    const float u4 = 0.25f * m4s, u5 = 2.25f * m5s, u6 = 9.0f * m6s;
    const float u7 = 1.5f * m7s, u8 = 1.5f * m8s, u9 = 0.0625f * m9s;
    const float base_a = u1 + u4 - 4.0f * u9;               // common to the axis directions
    const float base_d = u1 + 4.0f * u4 + 8.0f * u9;        // common to the diagonals
    float o[Q];
    o[0] = (4.0f / 9.0f) * (u1 - 2.0f * u4 + 2.0f * u9);
    o[1] = (1.0f / 9.0f) * (base_a + u2 + u5 - u7);
    o[2] = (1.0f / 9.0f) * (base_a + u3 - u5 - u8);
    o[3] = (1.0f / 9.0f) * (base_a - u2 + u5 + u7);
    o[4] = (1.0f / 9.0f) * (base_a - u3 - u5 + u8);
    o[5] = (1.0f / 36.0f) * (base_d + u2 + u3 + u6 + 2.0f * u7 + 2.0f * u8);
    o[6] = (1.0f / 36.0f) * (base_d - u2 + u3 - u6 - 2.0f * u7 + 2.0f * u8);
    o[7] = (1.0f / 36.0f) * (base_d - u2 - u3 + u6 - 2.0f * u7 - 2.0f * u8);
    o[8] = (1.0f / 36.0f) * (base_d + u2 - u3 - u6 + 2.0f * u7 - 2.0f * u8);

    // 9. store (own node plus periodic ghosts)
#pragma unroll
    for (int i = 0; i < Q; ++i) store_with_ghosts(a.dst + i * P, g, x, y, o[i]);
}

cudaError_t launch_step(const StepArgs& a, int noise_mode, cudaStream_t s) {
    constexpr int BX = 32, BY = 16;
    dim3 block(BX, BY);
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY);
    switch (noise_mode) {
        case 0: step_kernel<BX, BY, 0><<<grid, block, 0, s>>>(a); break;
        case 1: step_kernel<BX, BY, 1><<<grid, block, 0, s>>>(a); break;
        default: step_kernel<BX, BY, 2><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace lbf
