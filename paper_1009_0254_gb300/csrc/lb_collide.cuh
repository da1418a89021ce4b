// lb_collide.cuh -- the per-node fluctuating collision of [GACV] Eq. (fluct-lin-lbe),
// shared by the step kernels.  Input: the nine pulled FP32 deviations f_i(r,t) - fbar_i
// and the density deviations on the 3x3 neighbourhood; output: the nine post-collision
// deviations f*_i(r,t) - fbar_i.
#pragma once

#include "lb_internal.cuh"

namespace lbf {

// density deviation with one fixed summation order (used for a node and for the ring)
__device__ __forceinline__ float drho_of(const float f[Q]) {
    const float sa = (f[1] + f[3]) + (f[2] + f[4]);
    const float sd = (f[5] + f[7]) + (f[6] + f[8]);
    return f[0] + sa + sd;
}

// Density deviations around the node: C centre, E/W = x +- 1, N/S = y +- 1.
struct Nbr {
    float C, E, W, N, S, NE, NW, SE, SW;
};

// MODE 0: no noise; 1: uncorrelated (long-wavelength or diagonal); 2: correlated
// (xi_4, xi_9 given in xi49).  A carries the relaxation and noise factors, the time and
// the Philox key (StepArgs with precomputed round keys, or a per-replica record): Args.
template <int MODE, typename Args>
__device__ __forceinline__ void collide_node(const Args& a, const float f[Q], const Nbr& r, uint32_t node,
                                             float2 xi49, float o[Q]) {
    // Appendix B: sum_{i != 1} w_i [rho(r+c_i) + rho(r-c_i) - 2 rho(r)] / sigma_s^2
    const float lap = (4.0f * ((r.E + r.W) + (r.N + r.S)) + ((r.NE + r.SW) + (r.NW + r.SE)) - 20.0f * r.C) *
                      (1.0f / 6.0f);
    // d_alpha rho = 3 sum_i w_i c_i,alpha rho(r + c_i)
    const float gx = (r.E - r.W) * (1.0f / 3.0f) + ((r.NE - r.SW) + (r.SE - r.NW)) * (1.0f / 12.0f);
    const float gy = (r.N - r.S) * (1.0f / 3.0f) + ((r.NE - r.SW) + (r.NW - r.SE)) * (1.0f / 12.0f);

    // moments of the deviations (rows of T, Eq. Tmat)
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

    // equilibrium deviations, Table II (p0 = cs2 rho, C_n = 0)
    const float rho = a.rho0 + drho;
    const float inv = rcp_approx(rho);
    const float ux = jx * inv, uy = jy * inv;
    const float iso = a.cs2m * drho - a.kappa * rho * lap;
    const float e_eq = 3.0f * (jx * ux + jy * uy) + 6.0f * iso;
    const float pww_eq = (jx * ux - jy * uy) + a.kappa * (gx * gx - gy * gy);
    const float pxy_eq = jx * uy + a.kappa * gx * gy;
    const float eps_eq = -6.0f * iso - 3.0f * a.kappa * (gx * gx + gy * gy);

    // noise, Sec. IV
    float xi4 = 0.f, xi5 = 0.f, xi6 = 0.f, xi7 = 0.f, xi8 = 0.f, xi9 = 0.f;
    if (MODE != 0) {
        // one Philox draw per node and step: words 0, 1 -> nu_5..nu_8, word 2 -> (nu_4, nu_9)
        const uint4 r0 = philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_NODE), a.rk);
        const float2 g01 = gauss_pair(r0.x);
        const float2 g23 = gauss_pair(r0.y);
        xi5 = a.s5 * g01.x;
        xi6 = a.s6 * g01.y;
        xi7 = a.s7 * g23.x;
        xi8 = a.s7 * g23.y;
        if (MODE == 1) {
            const float2 n49 = gauss_pair(r0.z);
            xi4 = a.L44 * n49.x + a.L49 * n49.y;
            xi9 = a.L94 * n49.x + a.L99 * n49.y;
        } else {
            xi4 = xi49.x;
            xi9 = xi49.y;
        }
    }

    // relaxation of the non-conserved modes, Eq. (fluct-lin-lbe), as increments
    // D_a = m*_a - m_a = lambda_a (m_a - m_a^eq) + xi_a (zero for the conserved a = 1..3)
    const float D4 = a.lb * (m4 - e_eq) + xi4;
    const float D5 = a.ls * (m5 - pww_eq) + xi5;
    const float D6 = a.ls * (m6 - pxy_eq) + xi6;
    const float D7 = a.lq * m7 + xi7;
    const float D8 = a.lq * m8 + xi8;
    const float D9 = a.le * (m9 - eps_eq) + xi9;

    // back to populations: f*_i = f_i + w_i sum_{a>=4} T_ai D_a / N_a (Sec. III A)
    const float d4 = 0.25f * D4, d5 = 2.25f * D5, d6 = 9.0f * D6;
    const float d7 = 1.5f * D7, d8 = 1.5f * D8, d9 = 0.0625f * D9;
    const float A = d4 - 4.0f * d9;                 // T_4i - 4 T_9i part of the axis directions
    const float A1 = A + d5, A2 = A - d5;
    const float Dd = 4.0f * d4 + 8.0f * d9;         // the same for the diagonals
    const float D1 = Dd + d6, D2 = Dd - d6;
    const float P = 2.0f * (d7 + d8), M = 2.0f * (d7 - d8);
    o[0] = f[0] + (8.0f / 9.0f) * (d9 - d4);
    o[1] = f[1] + (1.0f / 9.0f) * (A1 - d7);
    o[2] = f[2] + (1.0f / 9.0f) * (A2 - d8);
    o[3] = f[3] + (1.0f / 9.0f) * (A1 + d7);
    o[4] = f[4] + (1.0f / 9.0f) * (A2 + d8);
    o[5] = f[5] + (1.0f / 36.0f) * (D1 + P);
    o[6] = f[6] + (1.0f / 36.0f) * (D2 - M);
    o[7] = f[7] + (1.0f / 36.0f) * (D1 - P);
    o[8] = f[8] + (1.0f / 36.0f) * (D2 + M);
}

}  // namespace lbf
