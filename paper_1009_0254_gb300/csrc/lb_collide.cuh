// lb_collide.cuh -- the per-node fluctuating collision of [GACV] Eq. (fluct-lin-lbe),
// shared by the step kernels.  Input: the nine pulled FP32 deviations f_i(r,t) - fbar_i
// and the density deviations on the 3x3 neighbourhood; output: the nine post-collision
// deviations f*_i(r,t) - fbar_i.
#pragma once

#include "lb_internal.cuh"

namespace lbf {

// density deviation with one fixed summation order (used for a node and for the ring)
template <typename R>
__device__ __forceinline__ R drho_of(const R f[Q]) {
    const R sa = (f[1] + f[3]) + (f[2] + f[4]);
    const R sd = (f[5] + f[7]) + (f[6] + f[8]);
    return f[0] + sa + sd;
}

// Density deviations around the node: C centre, E/W = x +- 1, N/S = y +- 1.
template <typename R>
struct NbrT {
    R C, E, W, N, S, NE, NW, SE, SW;
};
using Nbr = NbrT<float>;

// MODE 0: no noise; 1: uncorrelated (long-wavelength or diagonal); 2 and 3: correlated
// (xi_4, xi_9 given in xi49: from the k-space synthesis, or built in real space);
// 4: uncorrelated with Xi(0) at the node's own density and sound speed.  A carries the
// relaxation and noise factors, the time and the Philox key (StepArgs with precomputed
// round keys, or a per-replica record): Args.  R is the arithmetic type (float, or double
// for FP64 storage); every constant is an exact rational or rounded in R.
// density deviation of scaled deviations g_i = (f_i - fbar_i) / w_i (the FP16 storage form)
template <typename R>
__device__ __forceinline__ R drho_of_g(const R g[Q]) {
    const R sa = (g[1] + g[3]) + (g[2] + g[4]);
    const R sd = (g[5] + g[7]) + (g[6] + g[8]);
    return R(4) / R(9) * g[0] + (R(1) / R(9) * sa + R(1) / R(36) * sd);
}

// POLY: the bulk pressure is the double well's quartic in drho (Args carries e2..e4);
// otherwise p0 = cs2 rho and no polynomial code is compiled.
// GF: f and o hold the scaled deviations g_i = (f_i - fbar_i) / w_i instead of f_i - fbar_i
// (the weights move into the moment sums and out of the back-transform, so FP16 storage
// needs no scaling on load or store).
template <int MODE, bool POLY = false, bool GF = false, typename Args, typename R, typename X2>
__device__ __forceinline__ void collide_node(const Args& a, const R f[Q], const NbrT<R>& r, uint32_t node,
                                             X2 xi49, R o[Q]) {
    const R c6 = R(1) / R(6), c3 = R(1) / R(3), c12 = R(1) / R(12);
    // Appendix B: sum_{i != 1} w_i [rho(r+c_i) + rho(r-c_i) - 2 rho(r)] / sigma_s^2
    const R lap = (R(4) * ((r.E + r.W) + (r.N + r.S)) + ((r.NE + r.SW) + (r.NW + r.SE)) - R(20) * r.C) * c6;
    // d_alpha rho = 3 sum_i w_i c_i,alpha rho(r + c_i)
    const R gx = (r.E - r.W) * c3 + ((r.NE - r.SW) + (r.SE - r.NW)) * c12;
    const R gy = (r.N - r.S) * c3 + ((r.NE - r.SW) + (r.NW - r.SE)) * c12;

    // moments of the deviations (rows of T, Eq. Tmat); with GF the sums over the axis and
    // diagonal velocities carry their weights 1/9 and 1/36, the rest velocity 4/9
    const R wa = GF ? R(1) / R(9) : R(1), wd = GF ? R(1) / R(36) : R(1), w0 = GF ? R(4) / R(9) : R(1);
    const R sa0 = (f[1] + f[3]) + (f[2] + f[4]);
    const R sd0 = (f[5] + f[7]) + (f[6] + f[8]);
    const R sa = GF ? wa * sa0 : sa0, sd = GF ? wd * sd0 : sd0, g0 = GF ? w0 * f[0] : f[0];
    const R drho = g0 + sa + sd;
    const R ax = GF ? wa * (f[1] - f[3]) : f[1] - f[3], ay = GF ? wa * (f[2] - f[4]) : f[2] - f[4];
    const R dx0 = (f[5] - f[7]) + (f[8] - f[6]);
    const R dy0 = (f[5] - f[7]) + (f[6] - f[8]);
    const R dx = GF ? wd * dx0 : dx0, dy = GF ? wd * dy0 : dy0;
    const R jx = ax + dx, jy = ay + dy;
    const R m4 = R(-2) * g0 + sa + R(4) * sd;
    const R m5 = GF ? wa * ((f[1] + f[3]) - (f[2] + f[4])) : (f[1] + f[3]) - (f[2] + f[4]);
    const R m6 = GF ? wd * ((f[5] + f[7]) - (f[6] + f[8])) : (f[5] + f[7]) - (f[6] + f[8]);
    const R m7 = R(2) * dx - ax;
    const R m8 = R(2) * dy - ay;
    const R m9 = R(2) * g0 - R(4) * sa + R(8) * sd;

    // equilibrium deviations, Table II (C_n = 0): p0 - sigma_s^2 rho relative to the rest
    // state, linear (p0 = cs2 rho) or the double well's quartic in drho (Sec. II A)
    const R rho = a.rho0 + drho;
    const R inv = recip(rho);
    const R ux = jx * inv, uy = jy * inv;
    R dp = a.cs2m;
    if constexpr (POLY) dp += drho * (a.e2 + drho * (a.e3 + drho * a.e4));
    const R iso = dp * drho - a.kappa * rho * lap;
    const R e_eq = R(3) * (jx * ux + jy * uy) + R(6) * iso;
    const R pww_eq = (jx * ux - jy * uy) + a.kappa * (gx * gx - gy * gy);
    const R pxy_eq = jx * uy + a.kappa * gx * gy;
    const R eps_eq = R(-6) * iso - R(3) * a.kappa * (gx * gx + gy * gy);

    // noise, Sec. IV
    R xi4 = R(0), xi5 = R(0), xi6 = R(0), xi7 = R(0), xi8 = R(0), xi9 = R(0);
    if (MODE != 0) {
        // one Philox draw per node and step: words 0, 1 -> nu_5..nu_8, word 2 -> (nu_4, nu_9)
        const uint4 r0 = philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_NODE), a.rk);
        R n5, n6, n7, n8;
        gauss_word(r0.x, &n5, &n6);
        gauss_word(r0.y, &n7, &n8);
        if constexpr (MODE == 4) {
            // Xi(0) of Eq. (noise-yeo) at this node's density and sound speed (Sec. IV for
            // inhomogeneous systems), Cholesky of the (4,9) block with negative pivots at 0
            const R c = a.cq[0] + drho * (a.cq[1] + drho * (a.cq[2] + drho * a.cq[3]));
            const R y44 = rho * (a.lu[0] + a.lu[1] * c);
            const R y49 = rho * (a.lu[2] + a.lu[3] * c);
            const R y99 = rho * (a.lu[4] + a.lu[5] * c);
            const R sr = sqrt_fast(fmax(rho, R(0)));
            xi5 = sr * a.lu[6] * n5;
            xi6 = sr * a.lu[7] * n6;
            xi7 = sr * a.lu[8] * n7;
            xi8 = sr * a.lu[8] * n8;
            const R L44 = sqrt_fast(fmax(y44, R(0)));
            const R L94 = L44 > R(0) ? y49 * recip(L44) : R(0);
            const R L99 = sqrt_fast(fmax(y99 - L94 * L94, R(0)));
            R n4, n9;
            gauss_word(r0.z, &n4, &n9);
            xi4 = L44 * n4;
            xi9 = L94 * n4 + L99 * n9;
        } else {
            xi5 = a.s5 * n5;
            xi6 = a.s6 * n6;
            xi7 = a.s7 * n7;
            xi8 = a.s7 * n8;
        }
        if (MODE == 1) {
            R n4, n9;
            gauss_word(r0.z, &n4, &n9);
            xi4 = a.L44 * n4 + a.L49 * n9;
            xi9 = a.L94 * n4 + a.L99 * n9;
        } else if (MODE == 2 || MODE == 3) {
            xi4 = xi49.x;
            xi9 = xi49.y;
        }
    }

    // relaxation of the non-conserved modes, Eq. (fluct-lin-lbe), as increments
    // D_a = m*_a - m_a = lambda_a (m_a - m_a^eq) + xi_a (zero for the conserved a = 1..3)
    const R D4 = a.lb * (m4 - e_eq) + xi4;
    const R D5 = a.ls * (m5 - pww_eq) + xi5;
    const R D6 = a.ls * (m6 - pxy_eq) + xi6;
    const R D7 = a.lq * m7 + xi7;
    const R D8 = a.lq * m8 + xi8;
    const R D9 = a.le * (m9 - eps_eq) + xi9;

    // back to populations: f*_i = f_i + w_i sum_{a>=4} T_ai D_a / N_a (Sec. III A)
    const R d4 = R(0.25) * D4, d5 = R(2.25) * D5, d6 = R(9) * D6;
    const R d7 = R(1.5) * D7, d8 = R(1.5) * D8, d9 = R(0.0625) * D9;
    const R A = d4 - R(4) * d9;                    // T_4i - 4 T_9i part of the axis directions
    const R A1 = A + d5, A2 = A - d5;
    const R Dd = R(4) * d4 + R(8) * d9;            // the same for the diagonals
    const R D1 = Dd + d6, D2 = Dd - d6;
    const R P = R(2) * (d7 + d8), M = R(2) * (d7 - d8);
    // the rest velocity's increment is w_0 (T_40 D4/N4 + T_90 D9/N9) = (4/9)(2 d9 - 2 d4)
    if constexpr (GF) {
        o[0] = f[0] + R(2) * (d9 - d4);
        o[1] = f[1] + (A1 - d7);
        o[2] = f[2] + (A2 - d8);
        o[3] = f[3] + (A1 + d7);
        o[4] = f[4] + (A2 + d8);
        o[5] = f[5] + (D1 + P);
        o[6] = f[6] + (D2 - M);
        o[7] = f[7] + (D1 - P);
        o[8] = f[8] + (D2 + M);
    } else {
        const R u0 = R(8) / R(9), u1 = R(1) / R(9), u5 = R(1) / R(36);
        o[0] = f[0] + u0 * (d9 - d4);
        o[1] = f[1] + u1 * (A1 - d7);
        o[2] = f[2] + u1 * (A2 - d8);
        o[3] = f[3] + u1 * (A1 + d7);
        o[4] = f[4] + u1 * (A2 + d8);
        o[5] = f[5] + u5 * (D1 + P);
        o[6] = f[6] + u5 * (D2 - M);
        o[7] = f[7] + u5 * (D1 - P);
        o[8] = f[8] + u5 * (D2 + M);
    }
}

}  // namespace lbf
