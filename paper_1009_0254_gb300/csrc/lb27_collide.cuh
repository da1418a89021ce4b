// lb27_collide.cuh -- the per-node fluctuating collision on the D3Q27 lattice.
//
// [GACV] Sec. IV: the noise construction holds on any DdQn lattice; this is the paper's
// D2Q9 model carried to D3Q27 in the tensor-product basis
//   modes   m_(a,b,c) = sum_i p_a(c_ix) p_b(c_iy) p_c(c_iz) f_i, p_0 = 1, p_1 = c,
//           p_2 = 3c^2 - 1 (orthogonal under the D1Q3 weights 2/3, 1/6, 1/6 whose products
//           are the D3Q27 weights; the c_z-independent modes are the D2Q9 basis of Table I)
//   m^eq    rho, j, second-order modes of P^th + rho u u (Eq. press-ten, p0 = cs2 rho or the
//           double well's bulk pressure, Coef3); the
//           fourth-order p_2a p_2b = -3 (p0 - rho/3 - kappa rho lap rho) - (3/2) kappa |grad rho|^2
//           (Table II's eps on fields uniform along an axis), the sixth-order
//           p_2x p_2y p_2z = 3 (p0 - rho/3 - kappa rho lap rho) - (3/2) kappa |grad rho|^2, others 0
//   relax   lambda_b on p_2x + p_2y + p_2z, lambda_s on the traceless second order, one ghost
//           rate above; xi from Xi(0) (Eq. noise-matrix-k0)
// Index conventions: velocity i = 9 ix + 3 iy + iz with components v = (0, 1, -1); mode
// k = 9 a + 3 b + c.  The three-point transforms below act along one axis at a time.
#pragma once

#include "lb3_collide.cuh"

namespace lbf3 {

constexpr int Q27 = 27;

// moments of a 3-point line (f(0), f(+1), f(-1)) -> (p_0, p_1, p_2 projections)
template <typename R>
__host__ __device__ __forceinline__ void fwd3(R& f0, R& f1, R& f2) {
    const R s = f1 + f2, d = f1 - f2;
    const R m2 = R(2) * s - f0;
    f0 = f0 + s;
    f1 = d;
    f2 = m2;
}

// weighted back-transform of one axis with the 1/n_a of that axis folded in:
// g(c) = w1(c) sum_a p_a(c) h_a / n_a, n = (1, 1/3, 2), w1 = (2/3, 1/6, 1/6)
template <typename R>
__host__ __device__ __forceinline__ void bwd3(R& h0, R& h1, R& h2) {
    const R g0 = (R(2) / R(3)) * (h0 - R(0.5) * h2);
    const R e = h0 + h2, o = R(3) * h1;
    const R gp = (R(1) / R(6)) * (e + o), gm = (R(1) / R(6)) * (e - o);
    h0 = g0;
    h1 = gp;
    h2 = gm;
}

// m[27] from f[27] (three passes: x, y, z)
template <typename R>
__host__ __device__ __forceinline__ void moments27(const R f[Q27], R m[Q27]) {
#pragma unroll
    for (int k = 0; k < Q27; ++k) m[k] = f[k];
#pragma unroll
    for (int j = 0; j < 9; ++j) fwd3(m[j], m[9 + j], m[18 + j]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) fwd3(m[9 * a + c], m[9 * a + 3 + c], m[9 * a + 6 + c]);
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) fwd3(m[3 * ab], m[3 * ab + 1], m[3 * ab + 2]);
}

// Density deviations on the 3x3x3 neighbourhood, nb[9 ix + 3 iy + iz] = rho(r + c_i).
// xi[k] is the noise of mode k (zero for the conserved modes and without noise).
template <typename R>
__host__ __device__ __forceinline__ void collide27(const Coef3<R>& a, const R f[Q27], const R nb[Q27],
                                                   const R xi[Q27], R o[Q27]) {
    // Appendix B's stencils with the D3Q27 weights (products of 2/3, 1/6, 1/6):
    // lap = 6 sum_{i != 0} w_i rho(r + c_i) - 6 (1 - 8/27) rho(r), d_a rho = 3 sum_i w_i c_ia rho(r + c_i)
    // Both are formed by the same three-point sums along each axis.
    R t[Q27];
#pragma unroll
    for (int k = 0; k < Q27; ++k) t[k] = nb[k];
    // weighted sums along z, then y, then x: s0 = w-weighted sum, s1 = w-weighted first moment
    // (w1(+1) - w1(-1) parts), kept separately for each axis's role
    R wz0[9], wz1[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const R p = t[3 * j + 1], mn = t[3 * j + 2];
        wz0[j] = (R(2) / R(3)) * t[3 * j] + (R(1) / R(6)) * (p + mn);
        wz1[j] = (R(1) / R(6)) * (p - mn);
    }
    // along y: index j = 3 ix + iy
    R wy00[3], wy10[3], wy01[3];
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
        const int b = 3 * ix;
        wy00[ix] = (R(2) / R(3)) * wz0[b] + (R(1) / R(6)) * (wz0[b + 1] + wz0[b + 2]);
        wy10[ix] = (R(1) / R(6)) * (wz0[b + 1] - wz0[b + 2]);                              // y moment
        wy01[ix] = (R(2) / R(3)) * wz1[b] + (R(1) / R(6)) * (wz1[b + 1] + wz1[b + 2]);    // z moment
    }
    const R S = (R(2) / R(3)) * wy00[0] + (R(1) / R(6)) * (wy00[1] + wy00[2]);    // sum_i w_i rho(r + c_i)
    const R Mx = (R(1) / R(6)) * (wy00[1] - wy00[2]);
    const R My = (R(2) / R(3)) * wy10[0] + (R(1) / R(6)) * (wy10[1] + wy10[2]);
    const R Mz = (R(2) / R(3)) * wy01[0] + (R(1) / R(6)) * (wy01[1] + wy01[2]);
    const R lap = R(6) * S - R(6) * nb[0];         // 6 (sum_{i != 0} w_i rho_i - (1 - w_0) rho)
    const R gx = R(3) * Mx, gy = R(3) * My, gz = R(3) * Mz;

    R m[Q27];
    moments27(f, m);
    const R drho = m[0];
    const R jx = m[9], jy = m[3], jz = m[1];
    const R rho = a.rho0 + drho;
    const R inv = recip19(rho);
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const R g2 = (gx * gx + gy * gy) + gz * gz;
    const R klap = a.kappa * rho * lap;
    const R dd = pressure_slope(a, drho);
    const R base2 = (dd * drho - R(3) * klap) - R(1.5) * a.kappa * g2;
    // second order (deviations): p_2a: 3 Pi_aa - rho; p_1a p_1b: Pi_ab
    const R e18 = base2 + R(3) * (jx * ux + a.kappa * gx * gx);      // (2,0,0)
    const R e6 = base2 + R(3) * (jy * uy + a.kappa * gy * gy);       // (0,2,0)
    const R e2 = base2 + R(3) * (jz * uz + a.kappa * gz * gz);       // (0,0,2)
    const R e12 = jx * uy + a.kappa * gx * gy;                       // (1,1,0)
    const R e4 = jy * uz + a.kappa * gy * gz;                        // (0,1,1)
    const R e10 = jx * uz + a.kappa * gx * gz;                       // (1,0,1)
    const R e44 = (R(3) * klap - dd * drho) - R(1.5) * a.kappa * g2;  // p_2a p_2b
    const R e26 = (dd * drho - R(3) * klap) - R(1.5) * a.kappa * g2;  // p_2x p_2y p_2z

    // increments D = Lambda (m - m^eq) + xi; the p_2 block relaxes its mean at lambda_b
    R D[Q27];
#pragma unroll
    for (int k = 0; k < Q27; ++k) D[k] = a.lg * m[k] + xi[k];
    D[0] = R(0); D[1] = R(0); D[3] = R(0); D[9] = R(0);
    const R dx2 = m[18] - e18, dy2 = m[6] - e6, dz2 = m[2] - e2;
    const R mean = ((dx2 + dy2) + dz2) * (R(1) / R(3));
    const R bulk = (a.lb - a.ls) * mean;
    D[18] = (a.ls * dx2 + bulk) + xi[18];
    D[6] = (a.ls * dy2 + bulk) + xi[6];
    D[2] = (a.ls * dz2 + bulk) + xi[2];
    D[12] = a.ls * (m[12] - e12) + xi[12];
    D[4] = a.ls * (m[4] - e4) + xi[4];
    D[10] = a.ls * (m[10] - e10) + xi[10];
    D[24] = a.lg * (m[24] - e44) + xi[24];
    D[8] = a.lg * (m[8] - e44) + xi[8];
    D[20] = a.lg * (m[20] - e44) + xi[20];
    D[26] = a.lg * (m[26] - e26) + xi[26];

    // back to populations: delta f_i = w_i sum_k T_ki D_k / N_k, three weighted passes (z, y, x)
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) bwd3(D[3 * ab], D[3 * ab + 1], D[3 * ab + 2]);
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int c = 0; c < 3; ++c) bwd3(D[9 * a2 + c], D[9 * a2 + 3 + c], D[9 * a2 + 6 + c]);
#pragma unroll
    for (int j = 0; j < 9; ++j) bwd3(D[j], D[9 + j], D[18 + j]);
#pragma unroll
    for (int i = 0; i < Q27; ++i) o[i] = f[i] + D[i];
}

}  // namespace lbf3
